"""Pins of the oracle's lattice tables and equilibrium (Sec. 2.1, Eq. 3).

The velocity sets and weights are fixed by the isotropy conditions that make
the lattice Boltzmann equation recover Navier-Stokes; the equilibrium is fixed
by its moments.  A wrong weight, a missing direction, a wrong opposite index or
a wrong sign in Eq. 3 fails one of these.
"""

import itertools

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

CS2 = 1.0 / 3.0


@pytest.mark.parametrize("Q", [19, 27])
def test_velocity_set(oracle_mod, Q):
    c, w, opp = oracle_mod.lattice(Q)
    assert c.shape == (Q, 3)
    # distinct velocities, all in {-1,0,1}^3; D3Q19 excludes the 8 corners
    assert len({tuple(v) for v in c}) == Q
    n2 = (c ** 2).sum(1)
    expect = {19: {0: 1, 1: 6, 2: 12}, 27: {0: 1, 1: 6, 2: 12, 3: 8}}[Q]
    assert {k: int((n2 == k).sum()) for k in set(n2.tolist())} == expect
    # opposite directions
    assert np.array_equal(c[opp], -c)
    assert np.array_equal(opp[opp], np.arange(Q))


@pytest.mark.parametrize("Q", [19, 27])
def test_isotropy(oracle_mod, Q):
    c, w, _ = oracle_mod.lattice(Q)
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - CS2 * d).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.abs(m4 - iso).max() < 1e-15


@pytest.mark.parametrize("Q", [19, 27])
def test_equilibrium_moments(oracle_mod, Q):
    """Sum f^eq = rho, sum c f^eq = rho u, sum c c f^eq = rho c_s^2 I + rho u u."""
    c, w, _ = oracle_mod.lattice(Q)
    g = W.rng(W.SEED + Q)
    for _ in range(20):
        rho = g.uniform(0.5, 1.5)
        u = g.uniform(-0.1, 0.1, size=3)
        fe = np.array([oracle_mod.feq(Q, i, rho, u) for i in range(Q)])
        assert abs(fe.sum() - rho) < 1e-15 * 8
        assert np.abs(np.einsum("i,ia->a", fe, c) - rho * u).max() < 1e-15 * 8
        P = np.einsum("i,ia,ib->ab", fe, c, c)
        assert np.abs(P - (rho * CS2 * np.eye(3) + rho * np.outer(u, u))).max() < 1e-14


def test_equilibrium_sign_reading(oracle_mod):
    """Eq. 3 as printed (+u^2/(2 c_s^2)) would give sum f^eq = rho (1 + u^2/c_s^2):
    the oracle's reading (-u^2/(2 c_s^2)) is the only sign that conserves mass."""
    Q = 19
    c, w, _ = oracle_mod.lattice(Q)
    rho, u = 1.1, np.array([0.03, -0.02, 0.05])
    cu = c @ u
    uu = u @ u
    printed = w * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) + uu / (2 * CS2))
    assert abs(printed.sum() - rho * (1 + uu / CS2)) < 1e-14
    oracle_sum = sum(oracle_mod.feq(Q, i, rho, u) for i in range(Q))
    assert abs(oracle_sum - rho) < 1e-15 * 8


@pytest.mark.parametrize("mode,tau", list(itertools.product([0, 1], [0.55, 0.8, 1.5])))
def test_weighting(oracle_mod, mode, tau):
    """Eq. 5 / Eq. 6 special cases: B(0)=0, B(1)=1, monotone; Eq. 6 at tau-1/2 = 1
    is eps/(2-eps) and tends to Eq. 5 as tau grows."""
    B = lambda e, t=tau: oracle_mod.weighting(mode, e, t)
    assert B(0.0) == 0.0
    assert abs(B(1.0) - 1.0) < 1e-15
    es = np.linspace(0, 1, 101)
    vals = np.array([B(e) for e in es])
    assert np.all(np.diff(vals) > 0)
    if mode == 0:
        assert np.array_equal(vals, es)
    else:
        assert np.all(vals <= es + 1e-15)  # (1 - eps) >= 0 in the denominator => B <= eps
        for e in (0.25, 0.5, 0.75):
            assert abs(oracle_mod.weighting(1, e, 1.5) - e / (2 - e)) < 1e-15
        assert abs(oracle_mod.weighting(1, 0.3, 1e9) - 0.3) < 1e-8
