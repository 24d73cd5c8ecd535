"""Pins of the oracle's per-cell PSM collision (Eq. 2, TRT, Eq. 4, Eq. 7-9).

A 1x1x1 fully periodic grid streams every population back into its own cell,
so one oracle step is exactly one collision.  A large translating box body
makes the cell solid with u_s = v; the per-cell perturbation delta sets any
eps + delta.  The checks are moment identities and special cases derived from
the equations (mass, momentum balance against the recorded force, the
equilibrium fixed point, the B = 1 limits of SC1/SC2/SC3, the relaxation of
the non-equilibrium parts), so a wrong opposite index, sign, velocity argument
or weighting fails one of them.
"""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W


def one_cell(O, Q, f, eps, us, fluid=0, tau=0.8, solid=1, weighting=1, lam=3.0 / 16.0):
    cfg = O.Config(nx=1, ny=1, nz=1, Q=Q, bc_z=0, fluid=fluid, tau=tau, solid=solid, weighting=weighting,
                   trt_lambda=lam)
    sim = O.Sim(cfg, threads=1)
    sub, lo = O.voxelize(W.BOX, (50.0, 50.0, 50.0), 0)
    sim.add_body(O.BodySpec(sub=sub, s=0, lo=lo, R0=(0.5, 0.5, 0.5), v=tuple(us)))
    sim.set_f(np.asarray(f).reshape(Q, 1, 1, 1))
    sim.set_delta(np.array([eps - 1.0]))
    sim.step(1)
    return sim.get_f().reshape(Q), sim.force_torque()[0, 0]


def feqv(O, Q, rho, u):
    return np.array([O.feq(Q, i, rho, u) for i in range(Q)])


CASES = [(Q, fl, sc) for Q in (19, 27) for fl in (0, 1) for sc in (1, 2, 3)]


@pytest.mark.parametrize("Q,fluid,solid", CASES)
def test_mass_and_momentum_balance(oracle_mod, Q, fluid, solid):
    O = oracle_mod
    c, w, _ = O.lattice(Q)
    f = W.random_positive(Q, seed=W.SEED + Q + 10 * fluid + solid)
    us = (0.01, -0.02, 0.015)
    for eps in (0.0, 0.3, 1.0):
        post, ft = one_cell(O, Q, f, eps, us, fluid=fluid, solid=solid)
        assert abs(post.sum() - f.sum()) < 1e-15 * 16
        dj = c.T @ post - c.T @ f
        # momentum the solid gives the fluid = -(force on the body), Eq. 10
        assert np.abs(dj + ft[:3]).max() < 1e-15 * 16
        if eps == 0.0:
            assert np.abs(dj).max() < 1e-15 * 16


@pytest.mark.parametrize("Q,fluid,solid", CASES)
def test_equilibrium_fixed_point(oracle_mod, Q, fluid, solid):
    """f = f^eq(rho, u_s) with u = u_s is left unchanged for any B."""
    O = oracle_mod
    us = np.array([0.02, 0.01, -0.03])
    f = feqv(O, Q, 1.07, us)
    for eps in (0.0, 0.5, 1.0):
        post, ft = one_cell(O, Q, f, eps, us, fluid=fluid, solid=solid)
        assert np.abs(post - f).max() < 1e-15 * 8
        assert np.abs(ft).max() < 1e-15 * 8


@pytest.mark.parametrize("Q", [19, 27])
def test_full_solid_limits(oracle_mod, Q):
    """B = 1: SC1 leaves momentum rho u_s, SC3 2 rho u_s - j, SC2 j - (j - rho u_s)/tau."""
    O = oracle_mod
    c, w, _ = O.lattice(Q)
    f = W.random_positive(Q, seed=W.SEED + 7 * Q)
    rho, j = f.sum(), c.T @ f
    us = np.array([0.03, -0.01, 0.02])
    tau = 0.8
    expect = {1: rho * us, 2: j - (j - rho * us) / tau, 3: 2 * rho * us - j}
    for sc in (1, 2, 3):
        post, _ = one_cell(O, Q, f, 1.0, us, solid=sc, tau=tau)
        assert np.abs(c.T @ post - expect[sc]).max() < 1e-15 * 16, sc


@pytest.mark.parametrize("Q", [19, 27])
def test_fluid_relaxation(oracle_mod, Q):
    """B = 0: BGK relaxes f - f^eq by (1 - 1/tau); TRT relaxes the even / odd parts by
    (1 - omega+) / (1 - omega-), Lambda = (1/omega+ - 1/2)(1/omega- - 1/2)."""
    O = oracle_mod
    c, w, opp = O.lattice(Q)
    f = W.random_positive(Q, seed=W.SEED + 3 * Q)
    rho, u = f.sum(), (c.T @ f) / f.sum()
    fe = feqv(O, Q, rho, u)
    tau = 0.7
    post, _ = one_cell(O, Q, f, 0.0, (0, 0, 0), fluid=0, tau=tau)
    assert np.abs((post - fe) - (1 - 1 / tau) * (f - fe)).max() < 1e-15 * 8
    lam = 3.0 / 16.0
    wp = 1 / tau
    wm = 1 / (lam / (tau - 0.5) + 0.5)
    assert abs((1 / wp - 0.5) * (1 / wm - 0.5) - lam) < 1e-15
    post, _ = one_cell(O, Q, f, 0.0, (0, 0, 0), fluid=1, tau=tau, lam=lam)
    ne, ne_post = f - fe, post - fe
    ev, od = 0.5 * (ne + ne[opp]), 0.5 * (ne - ne[opp])
    ev_p, od_p = 0.5 * (ne_post + ne_post[opp]), 0.5 * (ne_post - ne_post[opp])
    assert np.abs(ev_p - (1 - wp) * ev).max() < 1e-15 * 8
    assert np.abs(od_p - (1 - wm) * od).max() < 1e-15 * 8
    # TRT with omega- = omega+ (Lambda = (tau - 1/2)^2) is BGK
    post_trt, _ = one_cell(O, Q, f, 0.0, (0, 0, 0), fluid=1, tau=tau, lam=(tau - 0.5) ** 2)
    post_bgk, _ = one_cell(O, Q, f, 0.0, (0, 0, 0), fluid=0, tau=tau)
    assert np.abs(post_trt - post_bgk).max() < 1e-15 * 8


@pytest.mark.parametrize("weighting", [0, 1])
@pytest.mark.parametrize("solid", [1, 2, 3])
def test_psm_rule_is_linear_blend(oracle_mod, weighting, solid):
    """Eq. 4: the post-collision state is linear in B between the B = 0 (pure fluid)
    and B = 1 (pure solid) results, with B given by Eq. 5 / Eq. 6."""
    O = oracle_mod
    Q = 19
    f = W.random_positive(Q, seed=W.SEED + 99)
    us = (0.01, 0.0, -0.02)
    tau = 0.65
    p0, _ = one_cell(O, Q, f, 0.0, us, solid=solid, weighting=weighting, tau=tau)
    p1, _ = one_cell(O, Q, f, 1.0, us, solid=solid, weighting=weighting, tau=tau)
    for eps in (0.2, 0.55, 0.9):
        pe, _ = one_cell(O, Q, f, eps, us, solid=solid, weighting=weighting, tau=tau)
        B = eps if weighting == 0 else eps * (tau - 0.5) / ((1 - eps) + (tau - 0.5))
        assert np.abs(pe - ((1 - B) * p0 + B * p1)).max() < 1e-15 * 16
