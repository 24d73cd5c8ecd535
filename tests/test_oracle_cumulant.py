"""Pins of the oracle's cumulant collision on D3Q19 (Geier et al. 2015: listed
in Sec. 2.2, the operator of every performance run in Sec. 5.1).

The oracle computes central moments, cumulants, relaxes them and solves a
linear system back to PDFs.  These tests check its output against facts that
do not go through that code:

* mass and momentum are conserved;
* with every rate 1 and zero momentum the result is rho w_i (the D3Q19 weights
  carry exactly the cumulant equilibrium of a fluid at rest);
* the cumulants of input and output, taken from their textbook definition
  (Taylor coefficients of log sum_i f_i exp(xi . c_i), computed here as a
  truncated power series), relax as the definition says, one family at a time;
* the operator commutes with the lattice symmetries (rotations, reflections);
* its output at rates 1 is a fixed point for any rates;
* its equilibrium has the closed-form (factorised Maxwellian) raw moments;
* a Taylor-Green vortex decays with the shear viscosity c_s^2 (tau - 1/2).
A wrong exponent, index, sign or rate in any family fails one of them.
"""

import itertools
import math

import numpy as np
import pytest

CS2 = 1.0 / 3.0


def oracle_cell(O, tau=0.8, rates=(1.0, 1.0, 1.0)):
    """An oracle with one periodic cell and no body: collide_at is the pure
    fluid operator."""
    cfg = O.Config(nx=1, ny=1, nz=1, Q=19, bc_z=0, fluid=2, tau=tau, cum_rates=tuple(rates))
    return O.Sim(cfg, threads=1)


def collide(sim, f):
    post, g, e = sim.collide_at(0, 0, 0, 0, f)
    assert e == 0.0 and not g.any()
    return post


def near_eq(O, rng, rho=1.0, u=(0.03, -0.02, 0.05), noise=2e-3):
    c, w, _ = O.lattice(19)
    f = np.array([O.feq(19, i, rho, u) for i in range(19)])
    return f + noise * rng.standard_normal(19) * w


# ---------------------------------------------------------------------------
# Cumulants from their definition: truncated power series in (x, y, z) with
# every exponent <= 2 (the ring modulo x^3, y^3, z^3).
# ---------------------------------------------------------------------------
def _mul(a, b):
    out = np.zeros((3, 3, 3))
    for i, j, k in itertools.product(range(3), repeat=3):
        if a[i, j, k] == 0.0:
            continue
        for p, q, r in itertools.product(range(3 - i), range(3 - j), range(3 - k)):
            out[i + p, j + q, k + r] += a[i, j, k] * b[p, q, r]
    return out


def cumulants(c, f):
    """K[a, b, c] = a! b! c! [x^a y^b z^c] log(sum_i f_i exp(x c_ix + y c_iy + z c_iz))
    for a, b, c <= 2 (normalised cumulants; K[0,0,0] = log rho)."""
    M = np.zeros((3, 3, 3))
    for i in range(len(f)):
        for a, b, cc in itertools.product(range(3), repeat=3):
            M[a, b, cc] += f[i] * c[i, 0] ** a * c[i, 1] ** b * c[i, 2] ** cc / (
                math.factorial(a) * math.factorial(b) * math.factorial(cc))
    rho = M[0, 0, 0]
    X = M / rho
    X[0, 0, 0] = 0.0
    L = np.zeros((3, 3, 3))
    P = np.zeros((3, 3, 3))
    P[0, 0, 0] = 1.0
    for n in range(1, 7):
        P = _mul(P, X)
        L += (-1) ** (n + 1) * P / n
    L[0, 0, 0] = math.log(rho)
    for a, b, cc in itertools.product(range(3), repeat=3):
        L[a, b, cc] *= math.factorial(a) * math.factorial(b) * math.factorial(cc)
    return L


THIRD = [(2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1), (1, 0, 2), (0, 1, 2)]
FOURTH = [(2, 2, 0), (2, 0, 2), (0, 2, 2)]
OFFDIAG = [(1, 1, 0), (1, 0, 1), (0, 1, 1)]


def test_cumulant_series_matches_moments(oracle_mod):
    """The series route itself: normalised cumulants of order <= 3 equal the
    central moments over rho (a check of the test's own definition)."""
    O = oracle_mod
    c, w, _ = O.lattice(19)
    f = near_eq(O, np.random.default_rng(1))
    rho = f.sum()
    u = (f[:, None] * c).sum(0) / rho
    K = cumulants(c, f)
    d = c - u
    assert abs(K[1, 0, 0] - u[0]) < 1e-14
    assert abs(K[2, 1, 0] - (f * d[:, 0] ** 2 * d[:, 1]).sum() / rho) < 1e-14
    assert abs(K[1, 1, 0] - (f * d[:, 0] * d[:, 1]).sum() / rho) < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_conservation(oracle_mod, seed):
    O = oracle_mod
    rng = np.random.default_rng(seed)
    c, w, _ = O.lattice(19)
    f = rng.uniform(0.02, 0.06, 19)
    sim = oracle_cell(O, tau=rng.uniform(0.52, 1.5), rates=tuple(rng.uniform(0.3, 1.9, 3)))
    post = collide(sim, f)
    assert abs(post.sum() - f.sum()) < 1e-14
    assert np.abs((post[:, None] * c).sum(0) - (f[:, None] * c).sum(0)).max() < 1e-14


def test_rest_state_closed_form(oracle_mod):
    """Rates 1, zero momentum: the output is rho w_i whatever the input."""
    O = oracle_mod
    c, w, opp = O.lattice(19)
    sim = oracle_cell(O, tau=1.0)
    for seed in range(3):
        f = np.random.default_rng(seed).uniform(0.02, 0.06, 19)
        f = 0.5 * (f + f[opp])  # zero momentum
        post = collide(sim, f)
        assert np.abs(post - f.sum() * w).max() < 1e-15


@pytest.mark.parametrize("tau,rates", [(0.8, (1.0, 1.0, 1.0)), (0.56, (1.3, 0.7, 1.6)), (1.4, (0.6, 1.8, 0.4))])
def test_cumulants_relax_by_definition(oracle_mod, tau, rates):
    O = oracle_mod
    c, w, _ = O.lattice(19)
    ws, wb, w3, w4 = 1.0 / tau, rates[0], rates[1], rates[2]
    rng = np.random.default_rng(7)
    for _ in range(3):
        f = near_eq(O, rng, rho=rng.uniform(0.9, 1.1), u=rng.uniform(-0.08, 0.08, 3), noise=5e-3)
        post = collide(oracle_cell(O, tau=tau, rates=rates), f)
        K, Kp = cumulants(c, f), cumulants(c, post)
        tol = 1e-12
        assert abs(Kp[0, 0, 0] - K[0, 0, 0]) < tol
        for e in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
            assert abs(Kp[e] - K[e]) < tol
        for e in OFFDIAG:
            assert abs(Kp[e] - (1 - ws) * K[e]) < tol
        tr, trp = K[2, 0, 0] + K[0, 2, 0] + K[0, 0, 2], Kp[2, 0, 0] + Kp[0, 2, 0] + Kp[0, 0, 2]
        assert abs(trp - (tr + wb * (3 * CS2 - tr))) < tol
        for a, b in [((2, 0, 0), (0, 2, 0)), ((2, 0, 0), (0, 0, 2))]:
            assert abs((Kp[a] - Kp[b]) - (1 - ws) * (K[a] - K[b])) < tol
        for e in THIRD:
            assert abs(Kp[e] - (1 - w3) * K[e]) < tol
        for e in FOURTH:
            assert abs(Kp[e] - (1 - w4) * K[e]) < tol


def _perm(c, R):
    """Index map P with c[P[i]] = R c[i]."""
    rc = c @ R.T
    return np.array([int(np.where((c == r).all(1))[0][0]) for r in rc])


@pytest.mark.parametrize("R", [
    np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]),   # 90 degrees about z
    np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]]),   # 90 degrees about x
    np.array([[-1, 0, 0], [0, 1, 0], [0, 0, 1]]),   # reflection x -> -x
    np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]]),    # swap x and y
])
def test_lattice_symmetry(oracle_mod, R):
    O = oracle_mod
    c, w, _ = O.lattice(19)
    P = _perm(c, R)
    sim = oracle_cell(O, tau=0.6, rates=(1.2, 0.8, 1.5))
    f = near_eq(O, np.random.default_rng(3), noise=1e-2)
    g = np.empty(19)
    g[P] = f  # population of direction c_i moves to direction R c_i
    post_f, post_g = collide(sim, f), collide(sim, g)
    expect = np.empty(19)
    expect[P] = post_f
    assert np.abs(post_g - expect).max() < 1e-15


def test_equilibrium_is_fixed_point(oracle_mod):
    O = oracle_mod
    f = near_eq(O, np.random.default_rng(5), noise=1e-2)
    feqc = collide(oracle_cell(O, tau=1.0), f)
    again = collide(oracle_cell(O, tau=0.57, rates=(1.4, 0.6, 1.7)), feqc)
    assert np.abs(again - feqc).max() < 1e-15


def test_equilibrium_closed_form(oracle_mod):
    """At rates 1 the output is the cumulant equilibrium at (rho, u), whose raw
    moments factorise into one-dimensional Maxwellian moments:
    sum_i f_i c_ix^a c_iy^b c_iz^c = rho m_a(u_x) m_b(u_y) m_c(u_z) with
    m_0 = 1, m_1 = u, m_2 = c_s^2 + u^2 (every cumulant above second order
    zero).  On D3Q19 these 19 moments fix the 19 populations.  Eq. 3 shares
    the moments up to second order; its fourth moments differ at O(u^2)."""
    O = oracle_mod
    c, w, _ = O.lattice(19)
    sim = oracle_cell(O, tau=1.0)
    E = [e for e in itertools.product(range(3), repeat=3) if min(e) == 0]  # not all three non-zero
    assert len(E) == 19

    def m1(e, v):
        return (1.0, v, CS2 + v * v)[e]

    for rho, u in [(1.03, (0.06, -0.04, 0.05)), (0.97, (-0.1, 0.02, 0.0)), (1.0, (0.0, 0.0, 0.08))]:
        u = np.array(u)
        fe = np.array([O.feq(19, i, rho, u) for i in range(19)])
        fc = collide(sim, fe)
        for e in E:
            mom = (fc * c[:, 0] ** e[0] * c[:, 1] ** e[1] * c[:, 2] ** e[2]).sum()
            assert abs(mom - rho * m1(e[0], u[0]) * m1(e[1], u[1]) * m1(e[2], u[2])) < 2e-15
            if sum(e) <= 2:
                assert abs(mom - (fe * c[:, 0] ** e[0] * c[:, 1] ** e[1] * c[:, 2] ** e[2]).sum()) < 2e-15


def _feq_np(c, w, i, rho, u):
    cu = u[..., 0] * c[i, 0] + u[..., 1] * c[i, 1] + u[..., 2] * c[i, 2]
    uu = (u ** 2).sum(-1)
    return w[i] * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))


@pytest.mark.parametrize("tau", [0.8, 0.6])
def test_taylor_green_decay_shear_viscosity(oracle_mod, tau):
    O = oracle_mod
    N, U = 32, 0.01
    k = 2 * np.pi / N
    x = np.arange(N) + 0.0
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.zeros((1, N, N, 3))
    u[..., 0] = -U * np.cos(k * X) * np.sin(k * Y)
    u[..., 1] = U * np.sin(k * X) * np.cos(k * Y)
    c, w, _ = O.lattice(19)
    f0 = np.stack([_feq_np(c, w, i, np.ones((1, N, N)), u) for i in range(19)])
    sim = O.Sim(O.Config(nx=N, ny=N, nz=1, Q=19, bc_z=0, fluid=2, tau=tau))
    sim.set_f(f0)
    mode = -np.cos(k * X) * np.sin(k * Y)

    def amp():
        _, uu = sim.macroscopic()
        return (uu[..., 0] * mode).sum() / (mode ** 2).sum()

    sim.step(10)
    a1 = amp()
    sim.step(100)
    a2 = amp()
    rate = np.log(a1 / a2) / 100
    nu = CS2 * (tau - 0.5)
    assert abs(rate / (2 * nu * k * k) - 1) < 1e-2


def test_rejects_unsupported(oracle_mod):
    O = oracle_mod
    with pytest.raises(ValueError):
        O.Sim(O.Config(nx=2, ny=2, nz=2, Q=27, fluid=2))
    with pytest.raises(ValueError):
        O.Sim(O.Config(nx=2, ny=2, nz=2, Q=19, fluid=2, force=(1e-5, 0.0, 0.0)))


def test_relaxation_property_random(oracle_mod):
    """The definition check over random states and rates (hypothesis)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    O = oracle_mod
    c, w, _ = O.lattice(19)

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(rho=st.floats(0.85, 1.15), u=st.tuples(*[st.floats(-0.12, 0.12)] * 3), noise=st.floats(0.0, 0.02),
               seed=st.integers(0, 2 ** 31 - 1), tau=st.floats(0.51, 2.0),
               rates=st.tuples(*[st.floats(0.05, 1.95)] * 3))
    def check(rho, u, noise, seed, tau, rates):
        rng = np.random.default_rng(seed)
        f = np.array([O.feq(19, i, rho, u) for i in range(19)]) + noise * rng.standard_normal(19) * w
        post = collide(oracle_cell(O, tau=tau, rates=rates), f)
        K, Kp = cumulants(c, f), cumulants(c, post)
        ws, wb, w3, w4 = 1.0 / tau, rates[0], rates[1], rates[2]
        tol = 1e-11
        assert abs(post.sum() - f.sum()) < 1e-13
        for e in OFFDIAG:
            assert abs(Kp[e] - (1 - ws) * K[e]) < tol
        tr, trp = K[2, 0, 0] + K[0, 2, 0] + K[0, 0, 2], Kp[2, 0, 0] + Kp[0, 2, 0] + Kp[0, 0, 2]
        assert abs(trp - (tr + wb * (3 * CS2 - tr))) < tol
        for e in THIRD:
            assert abs(Kp[e] - (1 - w3) * K[e]) < tol
        for e in FOURTH:
            assert abs(Kp[e] - (1 - w4) * K[e]) < tol

    check()
