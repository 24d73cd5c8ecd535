"""Two-way coupling on the GPU (psm_set_body_dynamics): a heavy sphere settling
under gravity and spinning, against the oracle's integrator; total momentum of
fluid and body; the infinitely heavy limit against prescribed motion."""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

from helpers import ft_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()


def settling(storage="fp64", streaming="aa", bc_z=0, solid=2):
    """A sphere of radius 3 at three times the fluid density (about 340 in
    lattice units), gravity minus buoyancy along -z, spinning about x."""
    return W.Case("settle", 20, 20, 28, Q=19, storage=storage, streaming=streaming, fluid="bgk", tau=0.7,
                  solid=solid, weighting=1, bc_z=bc_z, u_in=(0.0, 0.0, 0.0), steps=40,
                  bodies=[W.BodyCase(W.SPHERE, (3.0,), 2, (10.0, 10.3, 18.2), omega=(0.004, 0.0, 0.0))])


MASS, GRAV = 340.0, (0.0, 0.0, -0.05)


def run_pair(case, steps):
    import oracle

    from paper_2502_20049_gb300 import psm
    from oracle.cases import sim_from_case

    I = np.eye(3) * 0.4 * MASS * 9.0
    sol = psm.Solver.from_case(case)
    sol.set_body_dynamics(0, MASS, I, GRAV)
    sim = sim_from_case(case)
    sim.set_body_dynamics(0, MASS, I, GRAV)
    sol.step(steps)
    sim.step(steps)
    return sol, sim


@pytest.mark.parametrize("streaming,solid", [("aa", 2), ("twogrid", 1), ("aa", 1)])
def test_settling_sphere_fp64_matches_oracle(streaming, solid):
    case = settling(streaming=streaming, solid=solid)
    sol, sim = run_pair(case, case.steps)
    g, o = sol.body_state(0), sim.body_state(0)
    for k in ("R", "v", "omega", "L"):
        assert np.abs(g[k] - o[k]).max() <= 1e-12 * max(np.abs(o[k]).max(), 1e-3), k
    assert np.abs(g["Q"] - o["Q"]).max() <= 1e-13
    assert ft_err(dict(ft=sol.force_torque(0)[:, None, :]), dict(ft=sim.force_torque())) <= 1e-11
    _, u = sol.macroscopic()
    _, ou = sim.macroscopic()
    assert np.abs(u - ou).max() <= 1e-12
    assert o["v"][2] < -0.002  # it does settle


def test_settling_sphere_fp32_matches_oracle():
    case = settling(storage="fp32")
    sol, sim = run_pair(case, case.steps)
    g, o = sol.body_state(0), sim.body_state(0)
    assert np.abs(g["v"] - o["v"]).max() <= 1e-4 * np.abs(o["v"]).max()
    assert np.abs(g["R"] - o["R"]).max() <= 1e-4


def test_total_momentum_fp64():
    """Periodic box: P_fluid + m v changes by exactly F_ext per step."""
    from paper_2502_20049_gb300 import psm

    case = settling()
    sol = psm.Solver.from_case(case)
    sol.set_body_dynamics(0, MASS, np.eye(3) * 1224.0, GRAV)
    c, _, _ = psm.lattice_velocities(19)

    def P():
        return np.einsum("ia,izyx->a", c.astype(float), sol.get_state()) + MASS * sol.body_state(0)["v"]

    P0 = P()
    for n in (10, 25):
        sol.step(n - sol.step_count)
        assert np.abs(P() - (P0 + n * np.array(GRAV))).max() <= 1e-11 * n


def test_infinitely_heavy_body_follows_prescribed_motion():
    from paper_2502_20049_gb300 import psm

    case = settling(streaming="twogrid")
    a = psm.Solver.from_case(case)
    b = psm.Solver.from_case(case)
    b.set_body_dynamics(0, 1e30, np.eye(3) * 1e30)
    a.step(20)
    b.step(20)
    fa, fb = a.force_torque(0), b.force_torque(0)
    assert np.abs(fa - fb).max() <= 1e-9 * np.abs(fa).max()


def test_coupling_guards():
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(settling())
    with pytest.raises(psm.PSMError):
        sol.set_body_dynamics(0, -1.0, np.eye(3))
    with pytest.raises(psm.PSMError):
        sol.set_body_dynamics(0, 1.0, [[1, 2, 0], [0, 1, 0], [0, 0, 1]])  # not symmetric
    sol.set_body_dynamics(0, MASS, np.eye(3) * 1224.0, GRAV)
    with pytest.raises(psm.PSMError) as ei:
        sol.record(2)
    assert ei.value.code == -5
    sol.step(3)
    e = sol.eps()
    assert e.sum() > 0
