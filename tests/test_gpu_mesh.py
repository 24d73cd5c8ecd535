"""GPU triangle-mesh voxeliser (psm_geom_voxelize_mesh) against the oracle's
brute-force exact ray parity, bit for bit, and one PSM run with a
mesh-voxelised body against the oracle."""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

from helpers import u_err, ft_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()


def meshes():
    rng = np.random.default_rng(W.SEED + 11)
    R = W.rot("z", 0.61) @ W.rot("y", 0.27) @ W.rot("x", 1.3)
    return {
        "icosphere": W.icosphere(5.3, 2, centre=(0.13, -0.07, 0.21)),
        "box_through_centres": W.box_mesh((1.125, -0.875, 0.375), (4.625, 2.375, 3.125)),
        "rotated_cube": W.transform_mesh(W.box_mesh((-3, -3, -3), (3, 3, 3)), R, shift=0.1 * rng.random(3)),
        "torus": W.torus_mesh(6.0, 2.0, 40, 20),
        "components": W.merge_meshes(W.icosphere(2.5, 1, centre=(-6.0, 0.0, 0.0)),
                                     W.icosphere(2.0, 1, centre=(6.0, 1.0, 0.5)),
                                     W.transform_mesh(W.torus_mesh(3.0, 1.0, 24, 12), W.rot("x", 0.5))),
    }


# s = 3 (eight words per brick) on the small meshes: the oracle's brute force
# costs sub-cells x triangles
CASES = [(name, s) for name in ["icosphere", "box_through_centres", "rotated_cube", "torus", "components"]
         for s in (0, 1, 2)] + [("box_through_centres", 3), ("rotated_cube", 3)]


@pytest.mark.parametrize("name,s", CASES)
def test_mesh_voxeliser_equals_oracle(oracle_mod, name, s):
    from paper_2502_20049_gb300 import psm

    v, t = meshes()[name]
    g = psm.voxelize_mesh(v, t, s)
    sub, lo = oracle_mod.voxelize_mesh(v, t, s)
    assert np.array_equal(g.lo, lo)
    got = g.subcells()
    assert got.shape == sub.shape
    assert np.array_equal(got, sub), int((got != sub).sum())
    assert sub.sum() > 0


def test_mesh_voxeliser_device_inputs_and_large_mesh(oracle_mod):
    """Torch tensors on the device as inputs; a 20,480-triangle sphere of
    radius 40 at s = 2 (about 1e7 sub-cells) against the oracle on sampled
    rows and against the polyhedron volume."""
    import torch

    from paper_2502_20049_gb300 import psm

    v, t = W.icosphere(40.0, 5)
    g = psm.voxelize_mesh(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), 2)
    h = psm.voxelize_mesh(v, t, 2)
    assert np.array_equal(g.words(), h.words())
    sub = g.subcells()
    V = v.astype(np.float64)
    vol = sum(np.dot(V[a], np.cross(V[b], V[c])) for a, b, c in t) / 6.0
    assert abs(sub.sum() / 64.0 - vol) / vol < 2e-3


def test_psm_run_with_mesh_body_matches_oracle(oracle_mod):
    """FP64 two-grid run with a rotating torus voxelised from its mesh: the GPU
    (library mesh voxeliser) against the oracle (its own mesh voxeliser)."""
    import oracle

    from paper_2502_20049_gb300 import psm

    v, t = W.torus_mesh(5.0, 1.8, 32, 16)
    s = 2
    case = W.Case("mesh_torus", 24, 24, 16, Q=19, storage="fp64", streaming="twogrid", fluid="trt", tau=0.6,
                  bc_z=1, u_in=(0.0, 0.0, 0.03), steps=12, bodies=[])
    R0, omega, Q0 = (12.0, 12.0, 8.0), (0.0, 0.0, 0.04), np.eye(3).reshape(-1)
    sol = psm.Solver.from_case(case)
    sol.set_geometry(0, psm.voxelize_mesh(v, t, s), Q0, R0, omega, (0.0, 0.0, 0.0))
    sol.init_equilibrium(case.rho0, case.u_in)
    sol.step(case.steps)
    sub, lo = oracle_mod.voxelize_mesh(v, t, s)
    cfg = oracle.Config(nx=case.nx, ny=case.ny, nz=case.nz, Q=19, bc_z=1, rho0=1.0, u_in=tuple(case.u_in), fluid=1,
                        tau=case.tau, trt_lambda=case.trt_lambda, solid=case.solid, weighting=case.weighting)
    sim = oracle.Sim(cfg)
    sim.add_body(oracle.BodySpec(sub=sub, s=s, lo=lo, R0=R0, Q0=Q0, omega=omega, v=(0.0, 0.0, 0.0)))
    sim.init_eq(1.0, case.u_in)
    sim.step(case.steps)
    rho, u = sol.macroscopic()
    orho, ou = sim.macroscopic()
    assert np.abs(u - ou).max() / 0.03 <= 1e-12
    g = dict(ft=sol.force_torque(0)[:, None, :])
    o = dict(ft=sim.force_torque())
    assert ft_err(g, o) <= 1e-12
    assert np.abs(o["ft"]).max() > 0
