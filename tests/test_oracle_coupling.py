"""Pins of the oracle's two-way coupling (a body moving under the force and
torque the fluid exerts on it, as in the paper's settling-sphere validation,
Sec. 4): total momentum of fluid and body, the first step from rest, the
limit of an infinitely heavy body (the prescribed motion), and the torque-free
isotropic rotation."""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W


def _sim(O, n=16, bc_z=0, omega=(0.0, 0.0, 0.0), v=(0.0, 0.0, 0.0), u0=(0.0, 0.0, 0.0), Q=19, solid=1):
    sub, lo = O.voxelize(W.SPHERE, (3.0,), 2)
    cfg = O.Config(nx=n, ny=n, nz=n, Q=Q, bc_z=bc_z, u_in=u0, fluid=1, tau=0.6, solid=solid, weighting=1)
    sim = O.Sim(cfg)
    sim.add_body(O.BodySpec(sub=sub, s=2, lo=lo, R0=(8.0, 8.2, 7.9), omega=omega, v=v))
    sim.init_eq(1.0, u0)
    return sim


def _fluid_momentum(O, sim, Q=19):
    c, _, _ = O.lattice(Q)
    return np.einsum("ia,izyx->a", c.astype(float), sim.get_f())


@pytest.mark.parametrize("solid", [1, 2, 3])
def test_total_momentum_of_fluid_and_body(oracle_mod, solid):
    """Periodic box: P_fluid + m v changes by exactly F_ext per step."""
    O = oracle_mod
    sim = _sim(O, v=(0.01, -0.005, 0.02), omega=(0.0, 0.01, 0.02), u0=(0.0, 0.01, -0.01), solid=solid)
    # sphere of radius 3 (about 113 cells) at three times the fluid density:
    # explicit coupling needs the body heavier than the fluid it displaces
    m, Fext = 340.0, np.array([0.0, 0.0, -2e-3])
    sim.set_body_dynamics(0, m, np.eye(3) * 0.4 * 340.0 * 9.0, Fext)
    P0 = _fluid_momentum(O, sim) + m * sim.body_state(0)["v"]
    for n in range(1, 25):
        sim.step(1)
        P = _fluid_momentum(O, sim) + m * sim.body_state(0)["v"]
        # round-off of the FP64 sums (the momentum balance of a step holds to
        # ~1e-12 absolute here); a wrong sign or factor would be ~1e-3 per step
        assert np.abs(P - (P0 + n * Fext)).max() <= 1e-11 * n
    assert np.abs(sim.force_torque()[:, 0, :3]).max() > 1e-4  # the fluid does push the body


def test_first_step_from_rest_is_free_fall(oracle_mod):
    """Body and fluid at rest in equilibrium: no fluid force at step 0, so
    v_1 = F_ext / m and R_1 = R_0 + v_1 exactly."""
    O = oracle_mod
    sim = _sim(O)
    m, Fext = 40.0, np.array([1e-3, 0.0, -3e-3])
    sim.set_body_dynamics(0, m, np.eye(3) * 100.0, Fext)
    R0 = sim.body_state(0)["R"].copy()
    sim.step(1)
    assert np.array_equal(sim.force_torque()[0, 0], np.zeros(6))
    st = sim.body_state(0)
    assert np.allclose(st["v"], Fext / m, rtol=0, atol=1e-18)
    assert np.allclose(st["R"], R0 + Fext / m, rtol=0, atol=1e-15)


def test_infinitely_heavy_body_follows_the_prescribed_motion(oracle_mod):
    O = oracle_mod
    a = _sim(O, omega=(0.0, 0.0, 0.03), v=(0.01, 0.0, 0.0), u0=(0.0, 0.0, 0.02), bc_z=1)
    b = _sim(O, omega=(0.0, 0.0, 0.03), v=(0.01, 0.0, 0.0), u0=(0.0, 0.0, 0.02), bc_z=1)
    b.step(3)
    a.step(3)
    b.set_body_dynamics(0, 1e30, np.eye(3) * 1e30)
    a.step(20)
    b.step(20)
    fa, fb = a.force_torque(), b.force_torque()
    assert np.abs(fa - fb).max() <= 1e-9 * np.abs(fa).max()
    assert np.abs(a.get_f() - b.get_f()).max() <= 1e-12


def test_torque_free_isotropic_rotation(oracle_mod):
    """Isotropic inertia, no torque (the fluid's is negligible against a huge
    inertia): omega stays and Q_n equals n successive rotations by omega, the
    prescribed Q_n = Rot(omega n) Q0 to round-off."""
    O = oracle_mod
    w = np.array([0.01, -0.02, 0.03])
    sim = _sim(O, omega=tuple(w))
    sim.set_body_dynamics(0, 1e30, np.eye(3) * 1e30)
    sim.step(30)
    st = sim.body_state(0)
    Qp, _ = O.pose(np.eye(3).reshape(-1), (8.0, 8.2, 7.9), w, (0, 0, 0), 30)
    assert np.abs(st["Q"] - np.asarray(Qp).reshape(3, 3)).max() <= 1e-13
    assert np.abs(st["omega"] - w).max() <= 1e-13
    assert np.abs(st["Q"] @ st["Q"].T - np.eye(3)).max() <= 1e-14
