"""Parity at the full workload sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one.

The GPU runs a workload for some steps; the pre-collision PDFs of every
upstream neighbour x - c_i of a set of sampled cells x are exported
(psm_get_cells), the GPU takes one more step, and the sampled cells' new PDFs
are compared, population by population, with the oracle: f_i(x, n+1) is the
oracle's collision (remap, Eq. 4-9) of the upstream cell x - c_i at the pose
of step n applied to the exported PDFs, or the ghost value f^eq_i(rho0, u_in)
where x - c_i lies in a ghost plane.  Samples: uniform over the grid, around
every body (where eps is fractional and the solid collision acts), and on both
z boundary planes.

Tolerance per population (absolute): the GPU computes in FP32 and rounds to
its storage precision, the oracle computes in FP64 from the same inputs:
FP32 2e-6, FP16 (shifted) 2e-5, BF16 (shifted) 2e-4.
"""

import numpy as np
import pytest

from helpers import perm_lib_to_oracle
from paper_2502_20049_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp32": 2e-6, "fp16": 2e-5, "bf16": 2e-4}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()


def sample_cells(case, n_rand=96, n_body=96, n_bc=32, seed=W.SEED):
    rng = W.rng(seed)
    nx, ny, nz = case.nx, case.ny, case.nz
    pts = [np.stack([rng.integers(0, nx, n_rand), rng.integers(0, ny, n_rand), rng.integers(0, nz, n_rand)], 1)]
    for b in case.bodies:
        p = np.asarray(b.params, dtype=float)
        if b.kind == W.ROTOR:
            he = np.array([p[0] + p[2], p[0] + p[2], max(p[1] / 2, 0.5 * np.hypot(p[3], p[4]))])
        elif b.kind == W.SPHERE:
            he = np.array([p[0]] * 3)
        else:
            he = p[:3]
        off = rng.uniform(-1.0, 1.0, size=(n_body // len(case.bodies), 3)) * (he + 1.0)
        c = np.floor(np.asarray(b.R0) + off).astype(np.int64)
        pts.append(c)
    zb = np.stack([rng.integers(0, nx, n_bc), rng.integers(0, ny, n_bc), np.where(np.arange(n_bc) % 2, nz - 1, 0)], 1)
    pts.append(zb)
    P = np.concatenate(pts)
    P[:, 0] %= nx
    P[:, 1] %= ny
    P[:, 2] = np.clip(P[:, 2], 0, nz - 1)
    flat = (P[:, 2] * ny + P[:, 1]) * nx + P[:, 0]
    return np.unique(flat)


def check_one_step(case, steps_before):
    import oracle
    from oracle.cases import sim_from_case
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(case)
    sol.step(steps_before)
    n = sol.step_count
    c_lib, _, _ = psm.lattice_velocities(case.Q)
    perm = perm_lib_to_oracle(case.Q)
    cells = sample_cells(case)
    nx, ny, nz = case.nx, case.ny, case.nz
    x = cells % nx
    y = (cells // nx) % ny
    z = cells // (nx * ny)
    # upstream cells x - c_i (None where the population comes from a ghost plane)
    up = {}
    for k in range(cells.size):
        for i in range(case.Q):
            zs = z[k] - c_lib[i, 2]
            if zs < 0 or zs >= nz:
                if case.bc_z == 1:
                    continue
                zs %= nz
            xs, ys = (x[k] - c_lib[i, 0]) % nx, (y[k] - c_lib[i, 1]) % ny
            up[(k, i)] = int((zs * ny + ys) * nx + xs)
    ucells = np.unique(np.array(list(up.values()), dtype=np.int64))
    F = sol.get_cells(ucells)  # pre-collision PDFs at step n, library order
    index = {int(c): j for j, c in enumerate(ucells)}
    sol.step(1)
    G = sol.get_cells(cells)  # PDFs at step n + 1
    sim = sim_from_case(case, init=False)
    post_cache = {}
    ghost = np.array([oracle.feq(case.Q, perm[i], case.rho0, case.u_in) for i in range(case.Q)])
    worst = 0.0
    for k in range(cells.size):
        for i in range(case.Q):
            u = up.get((k, i))
            if u is None:
                expect = ghost[i]
            else:
                if u not in post_cache:
                    fin = np.zeros(case.Q)
                    fin[perm] = F[index[u]]  # library order -> oracle order
                    uz, r = divmod(u, nx * ny)
                    uy, ux = divmod(r, nx)
                    post, _, _ = sim.collide_at(n, ux, uy, uz, fin)
                    post_cache[u] = post
                expect = post_cache[u][perm[i]]
            worst = max(worst, abs(G[k, i] - expect))
    return worst, cells.size, n


def test_c2_full_256_fp32_twogrid_tma():
    case = W.c2_ellipsoid().with_(streaming="twogrid")
    worst, ns, n = check_one_step(case, 37)
    print(f"256^3 FP32 two-grid: {ns} cells, step {n}: max |df| {worst:.2e}")
    assert worst <= TOL["fp32"]


@pytest.mark.parametrize("steps_before", [20, 21])
def test_c3_full_d3q27_fp16_aa(steps_before):
    case = W.c3_rotor("fp16").with_(streaming="aa")
    worst, ns, n = check_one_step(case, steps_before)
    print(f"512x512x640 D3Q27 FP16 AA: {ns} cells, step {n}: max |df| {worst:.2e}")
    assert worst <= TOL["fp16"]


def test_c5_full_1e9_fp16_aa():
    case = W.c5_large().with_(streaming="aa")
    worst, ns, n = check_one_step(case, 11)
    print(f"1024x1024x960 FP16 AA: {ns} cells, step {n}: max |df| {worst:.2e}")
    assert worst <= TOL["fp16"]


@pytest.mark.parametrize("storage,streaming,steps_before", [("fp32", "twogrid", 37), ("fp16", "twogrid", 37),
                                                            ("fp16", "aa", 21)])
def test_c2_full_256_cumulant(storage, streaming, steps_before):
    """The cumulant variants bench.py times (256^3, default rates)."""
    case = W.c2_ellipsoid().with_(streaming=streaming, storage=storage, fluid="cumulant")
    worst, ns, n = check_one_step(case, steps_before)
    print(f"256^3 cumulant {storage} {streaming}: {ns} cells, step {n}: max |df| {worst:.2e}")
    assert worst <= TOL[storage]
