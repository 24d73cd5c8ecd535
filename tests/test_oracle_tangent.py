"""Pin of the oracle's tangent-linear model (the reference for the adjoint).

The tangent-linear model is the oracle's own step run on dual numbers; it is
checked here against central finite differences of the plain FP64 oracle, for
every cell of a small grid (derivative with respect to a per-cell fraction
perturbation delta), for the angular velocity (with the geometry sequence
frozen, as both sides define it) and for the inflow velocity (ghost planes and
initial state).  The functional is the mean torque about z on the body over
the run: J = (1/N) sum_n T_z(n).
"""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

NX, NY, NZ, STEPS = 6, 6, 8, 10
U_IN = 0.03
OMEGA = (0.0, 0.0, 0.05)


def _cfg(O, u_in=U_IN):
    return O.Config(nx=NX, ny=NY, nz=NZ, bc_z=1, u_in=(0.0, 0.0, u_in), fluid=1, tau=0.62, solid=1, weighting=1)


def _body(O):
    sub, lo = O.voxelize(W.ELLIPSOID, (2.6, 1.4, 1.2), 2)
    return O.BodySpec(sub=sub, s=2, lo=lo, R0=(3.0, 3.1, 4.0), omega=OMEGA)


def J_plain(O, delta=None, u_in=U_IN, omega_us=None):
    sim = O.Sim(_cfg(O, u_in), threads=1)
    sim.add_body(_body(O))
    if omega_us is not None:
        sim.set_us_omega(0, omega_us)
    sim.init_eq(1.0, (0.0, 0.0, u_in))
    if delta is not None:
        sim.set_delta(delta)
    sim.step(STEPS)
    return sim.force_torque()[:, 0, 5].mean()


def J_tangent(O, d_delta=None, d_omega=(0, 0, 0), d_u=0.0):
    sim = O.TangentSim(_cfg(O), d_u_in=(0.0, 0.0, d_u), threads=1)
    sim.add_body(_body(O), d_omega=d_omega)
    sim.init_eq(1.0, (0.0, 0.0, U_IN), du=(0.0, 0.0, d_u))
    sim.set_delta(None, d_delta)
    sim.step(STEPS)
    v, t = sim.force_torque()
    return v[:, 0, 5].mean(), t[:, 0, 5].mean()


def test_tangent_value_matches_plain(oracle_mod):
    O = oracle_mod
    v, _ = J_tangent(O)
    assert abs(v - J_plain(O)) <= 1e-15 * max(1.0, abs(v))


def test_tangent_vs_fd_every_cell(oracle_mod):
    O = oracle_mod
    n = NX * NY * NZ
    h = 1e-6
    j0 = J_plain(O)
    scale = abs(j0)
    worst = 0.0
    nonzero = 0
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        _, tl = J_tangent(O, d_delta=e)
        fd = (J_plain(O, delta=h * e) - J_plain(O, delta=-h * e)) / (2 * h)
        worst = max(worst, abs(tl - fd))
        nonzero += abs(tl) > 1e-9 * scale
    # central FD error ~ h^2 J''' + eps_mach J / h
    assert worst < 1e-8 * max(scale, 1e-6) + 1e-12
    assert nonzero > n // 4


def test_tangent_vs_fd_omega_and_inflow(oracle_mod):
    O = oracle_mod
    _, tl_w = J_tangent(O, d_omega=(0.0, 0.0, 1.0))
    h = 1e-6
    fd_w = (J_plain(O, omega_us=(0, 0, OMEGA[2] + h)) - J_plain(O, omega_us=(0, 0, OMEGA[2] - h))) / (2 * h)
    assert abs(tl_w - fd_w) < 1e-7 * abs(fd_w)
    _, tl_u = J_tangent(O, d_u=1.0)
    fd_u = (J_plain(O, u_in=U_IN + h) - J_plain(O, u_in=U_IN - h)) / (2 * h)
    assert abs(tl_u - fd_u) < 1e-7 * abs(fd_u)
    assert abs(fd_w) > 0 and abs(fd_u) > 0


def test_tangent_gradient_every_direction_vs_fd(oracle_mod):
    """oracle.tangent_gradient (one tangent-linear run per cell, per omega
    axis and per inflow axis: the per-cell reference the GPU adjoint is
    compared with) against central differences of the plain FP64 oracle, for
    every cell and all three components of omega and u_in."""
    O = oracle_mod
    u = np.array([0.004, -0.003, U_IN])
    cfg = O.Config(nx=NX, ny=NY, nz=NZ, bc_z=1, u_in=tuple(u), fluid=1, tau=0.62, solid=1, weighting=1)
    body = _body(O)
    J, gd, gw, gu = O.tangent_gradient(cfg, [body], STEPS, 1.0, tuple(u))

    def Jp(delta=None, uu=u, om=None):
        c = O.Config(nx=NX, ny=NY, nz=NZ, bc_z=1, u_in=tuple(uu), fluid=1, tau=0.62, solid=1, weighting=1)
        sim = O.Sim(c, threads=1)
        sim.add_body(body)
        if om is not None:
            sim.set_us_omega(0, om)
        sim.init_eq(1.0, tuple(uu))
        if delta is not None:
            sim.set_delta(delta)
        sim.step(STEPS)
        return sim.force_torque()[:, 0, 5].mean()

    assert abs(J - Jp()) <= 1e-15 * abs(J)
    h = 1e-6
    n = NX * NY * NZ
    fd = np.zeros(n)
    for c in range(n):
        e = np.zeros(n)
        e[c] = h
        fd[c] = (Jp(delta=e) - Jp(delta=-e)) / (2 * h)
    assert np.abs(gd.reshape(-1) - fd).max() < 1e-8 * abs(J) + 1e-12
    for k in range(3):
        dk = np.eye(3)[k] * h
        fw = (Jp(om=np.array(OMEGA) + dk) - Jp(om=np.array(OMEGA) - dk)) / (2 * h)
        fu = (Jp(uu=u + dk) - Jp(uu=u - dk)) / (2 * h)
        assert abs(gw[0, k] - fw) < 1e-7 * max(abs(fw), abs(gw[0, 2])), (k, gw[0, k], fw)
        assert abs(gu[k] - fu) < 1e-7 * max(abs(fu), abs(gu[2])), (k, gu[k], fu)
