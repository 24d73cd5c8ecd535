"""Closed-form flows and conservation laws that pin the oracle's full step
(streaming Eq. 1, collision Eq. 2 / TRT, PSM rule Eq. 4, force and torque
Eq. 10 / 11).

* Poiseuille (Guo body force, half-way bounce-back walls): the parabola is the
  exact steady state for TRT with Lambda = 3/16 and for BGK at
  tau = 1/2 + sqrt(3/16); at other tau BGK misses it by O(1/ny^2).
* Couette (moving half-way bounce-back wall): linear profile, exact for any tau.
* Taylor-Green vortex: decay rate nu (kx^2 + ky^2), nu = c_s^2 (tau - 1/2).
* A moving body in a periodic box: total mass constant; momentum change per
  step equals the solid's momentum transfer S_F of Eq. 10.
* Torque reference-point shift: T_R' = T_R + (R - R') x F.
* A body spinning in fluid at rest is braked: omega . T < 0.
"""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

CS2 = 1.0 / 3.0


def _feq_np(c, w, i, rho, u):
    # vectorised Eq. 3 used only to build initial states; its output is an
    # input of the oracle, not an expected value
    cu = u @ c[i].astype(float)
    uu = (u ** 2).sum(-1)
    return w[i] * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))


@pytest.mark.parametrize("fluid,tau,exact", [(0, 0.5 + np.sqrt(3 / 16), True), (1, 0.8, True), (1, 0.56, True),
                                             (0, 0.8, False)])
def test_poiseuille(oracle_mod, fluid, tau, exact):
    O = oracle_mod
    ny, F = 8, 1e-6
    cfg = O.Config(nx=1, ny=ny, nz=1, bc_z=0, walls_y=1, force=(F, 0, 0), fluid=fluid, tau=tau)
    sim = O.Sim(cfg, threads=1)
    sim.init_eq(1.0, (0, 0, 0))
    sim.step(int(30 * ny * ny / ((tau - 0.5) / 3)))
    c, _, _ = O.lattice(19)
    f = sim.get_f()
    rho = f.sum(0)
    ux = ((np.einsum("i,izyx->zyx", c[:, 0].astype(float), f) + F / 2) / rho)[0, :, 0]
    nu = CS2 * (tau - 0.5)
    y = np.arange(ny)
    ua = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    err = np.abs(ux - ua).max() / ua.max()
    if exact:
        assert err < 1e-9
    else:
        assert err > 1e-3


@pytest.mark.parametrize("tau", [0.6, 1.3])
def test_couette(oracle_mod, tau):
    O = oracle_mod
    ny, U = 10, 0.01
    cfg = O.Config(nx=2, ny=ny, nz=1, bc_z=0, walls_y=1, wall_u_hi=(U, 0, 0), fluid=0, tau=tau)
    sim = O.Sim(cfg, threads=1)
    sim.init_eq(1.0, (0, 0, 0))
    sim.step(int(40 * ny * ny / (CS2 * (tau - 0.5))))
    rho, u = sim.macroscopic()
    y = np.arange(ny)
    ua = U * (y + 0.5) / ny
    assert np.abs(u[0, :, 0, 0] - ua).max() / U < 1e-9


@pytest.mark.parametrize("Q,fluid,tau", [(19, 0, 0.8), (19, 1, 0.6), (27, 0, 0.7)])
def test_taylor_green_decay(oracle_mod, Q, fluid, tau):
    O = oracle_mod
    N, U = 64, 0.01
    k = 2 * np.pi / N
    x = np.arange(N) + 0.0
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.zeros((4, N, N, 3))
    u[..., 0] = -U * np.cos(k * X) * np.sin(k * Y)
    u[..., 1] = U * np.sin(k * X) * np.cos(k * Y)
    c, w, _ = O.lattice(Q)
    f0 = np.stack([_feq_np(c, w, i, np.ones((4, N, N)), u) for i in range(Q)])
    sim = O.Sim(O.Config(nx=N, ny=N, nz=4, Q=Q, bc_z=0, fluid=fluid, tau=tau))
    sim.set_f(f0)
    mode = -np.cos(k * X) * np.sin(k * Y)

    def amp():
        _, uu = sim.macroscopic()
        return (uu[..., 0] * mode).sum() / (mode ** 2).sum() / 4

    sim.step(20)
    a1 = amp()
    sim.step(200)
    a2 = amp()
    rate = np.log(a1 / a2) / 200
    nu = CS2 * (tau - 0.5)
    assert abs(rate / (2 * nu * k * k) - 1) < 1e-2


def _moving_body_sim(O, Q=19, solid=1, fluid=1, n=16):
    sub, lo = O.voxelize(W.ELLIPSOID, (5.0, 3.0, 2.0), 2)
    cfg = O.Config(nx=n, ny=n, nz=n, Q=Q, bc_z=0, fluid=fluid, tau=0.6, solid=solid, weighting=1)
    sim = O.Sim(cfg)
    sim.add_body(O.BodySpec(sub=sub, s=2, lo=lo, R0=(8.0, 8.3, 7.9), omega=(0.002, -0.001, 0.02),
                            v=(0.002, 0.0, -0.001)))
    sim.init_eq(1.0, (0.0, 0.01, 0.02))
    return sim


@pytest.mark.parametrize("Q,solid", [(19, 1), (19, 2), (19, 3), (27, 1)])
def test_mass_conservation_and_momentum_balance(oracle_mod, Q, solid):
    O = oracle_mod
    sim = _moving_body_sim(O, Q=Q, solid=solid)
    c, _, _ = O.lattice(Q)
    f = sim.get_f()
    m0 = f.sum()
    P = [np.einsum("ia,izyx->a", c.astype(float), f)]
    for _ in range(40):
        sim.step(1)
        f = sim.get_f()
        P.append(np.einsum("ia,izyx->a", c.astype(float), f))
    assert abs(f.sum() - m0) / m0 < 1e-13
    ft = sim.force_torque()
    dP = np.diff(np.array(P), axis=0)
    # the fluid's momentum gain each step is the momentum the solid gives it
    assert np.abs(dP + ft[:, 0, :3]).max() < 1e-10
    assert np.abs(ft[:, 0, :3]).max() > 1e-4


def test_torque_reference_shift(oracle_mod):
    """Same world geometry, reference point moved by an integer vector d:
    T' = T + (R - R') x F with F unchanged."""
    O = oracle_mod
    sub, lo = O.voxelize(W.ELLIPSOID, (4.0, 2.5, 2.0), 2)
    res = []
    for d in (np.zeros(3), np.array([2.0, -1.0, 3.0])):
        cfg = O.Config(nx=12, ny=12, nz=16, bc_z=1, u_in=(0, 0, 0.03), fluid=0, tau=0.8)
        sim = O.Sim(cfg)
        R0 = np.array([6.0, 6.0, 8.0]) + d
        sim.add_body(O.BodySpec(sub=sub, s=2, lo=lo - d, R0=tuple(R0)))
        sim.init_eq(1.0, (0, 0, 0.03))
        sim.step(15)
        res.append((R0, sim.force_torque()[:, 0]))
    (R, a), (Rp, b) = res
    assert np.abs(a[:, :3] - b[:, :3]).max() < 1e-15
    pred = a[:, 3:] + np.cross(R - Rp, a[:, :3])
    assert np.abs(b[:, 3:] - pred).max() < 1e-13
    assert np.abs(a[:, 2]).max() > 1e-4  # drag along the flow


def test_spinning_body_is_braked(oracle_mod):
    O = oracle_mod
    sub, lo = O.voxelize(W.ELLIPSOID, (5.0, 2.0, 2.0), 2)
    for wz in (0.01, -0.01):
        cfg = O.Config(nx=16, ny=16, nz=8, bc_z=0, fluid=0, tau=0.8)
        sim = O.Sim(cfg)
        sim.add_body(O.BodySpec(sub=sub, s=2, lo=lo, R0=(8.0, 8.0, 4.0), omega=(0, 0, wz)))
        sim.init_eq(1.0, (0, 0, 0))
        sim.step(30)
        T = sim.force_torque()[:, 0, 3:]
        assert np.all(wz * T[5:, 2] < 0)


def test_drag_points_downstream(oracle_mod):
    """A static sphere in an inflow along +z is pushed along +z (Eq. 10 with the
    body-force sign reading)."""
    O = oracle_mod
    sub, lo = O.voxelize(W.SPHERE, (3.0,), 2)
    cfg = O.Config(nx=12, ny=12, nz=16, bc_z=1, u_in=(0, 0, 0.02), fluid=0, tau=0.8)
    sim = O.Sim(cfg)
    sim.add_body(O.BodySpec(sub=sub, s=2, lo=lo, R0=(6.0, 6.0, 8.0)))
    sim.init_eq(1.0, (0, 0, 0.02))
    sim.step(30)
    F = sim.force_torque()[:, 0, :3]
    assert np.all(F[:, 2] > 0)
    assert np.abs(F[:, :2]).max() < 1e-3 * np.abs(F[:, 2]).max()


def test_rotating_sphere_stokes_torque(oracle_mod):
    """Torque on a slowly rotating sphere (surface speed 5e-3, Re << 1) in a
    periodic box against Stokes' closed form T = -8 pi rho nu R^3 omega (the
    torque on the body, opposing the rotation): within 5 % at R = 5 and closer
    than at R = 4 (the PSM boundary converges with resolution; R = 6 in a 48^3
    box gives 1 %); the other components vanish by symmetry.  This pins the
    magnitude of Eq. 11 with the remap and u_s of a rotating body (SC1, Eq. 6)."""
    O = oracle_mod
    tau, om, s = 0.8, 1e-3, 3
    nu = CS2 * (tau - 0.5)
    err = {}
    for N, R, steps in ((24, 4.0, 400), (32, 5.0, 500)):
        cfg = O.Config(nx=N, ny=N, nz=N, Q=19, bc_z=0, fluid=0, tau=tau, solid=1, weighting=1)
        sim = O.Sim(cfg)
        sub, lo = O.voxelize(W.SPHERE, (R,), s)
        sim.add_body(O.BodySpec(sub=sub, s=s, lo=lo, R0=(N / 2, N / 2, N / 2), omega=(0.0, 0.0, om)))
        sim.init_eq(1.0, (0, 0, 0))
        sim.step(steps)
        ft = sim.force_torque()[:, 0]
        T0 = -8.0 * np.pi * nu * R ** 3 * om
        assert abs(ft[-1, 5] / ft[-101, 5] - 1) < 5e-3  # steady
        assert np.abs(ft[-1, :5]).max() < 1e-12 * abs(T0)
        err[R] = abs(ft[-1, 5] / T0 - 1)
    assert err[5.0] < 0.05
    assert err[5.0] < err[4.0]
