"""Shared test helpers: run a workload case on the CUDA path and on the oracle.

Both sides take their inputs from paper_2502_20049_gb300.workloads; the oracle
voxelises the bodies itself.  No expected value comes from the CUDA path.
"""

import numpy as np

from paper_2502_20049_gb300 import workloads as W

def perm_lib_to_oracle(Q):
    """perm[i] = oracle index of the library's direction i (same velocity)."""
    import oracle
    from paper_2502_20049_gb300 import psm

    c_lib, _, _ = psm.lattice_velocities(Q)
    c_or, _, _ = oracle.lattice(Q)
    return np.array([int(np.flatnonzero((c_or == c_lib[i]).all(1))[0]) for i in range(Q)])


def oracle_sim(case: W.Case, threads=None):
    from oracle.cases import sim_from_case

    return sim_from_case(case, threads=threads)


def run_oracle(case: W.Case, steps=None):
    sim = oracle_sim(case)
    sim.step(case.steps if steps is None else steps)
    rho, u = sim.macroscopic()
    return dict(f=sim.get_f(), ft=sim.force_torque(), rho=rho, u=u, sim=sim)


def run_gpu(case: W.Case, steps=None):
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(case)
    sol.step(case.steps if steps is None else steps)
    rho, u = sol.macroscopic()
    ft = np.stack([sol.force_torque(b) for b in range(len(case.bodies))], axis=1) if case.bodies else None
    return dict(f=sol.get_state(), ft=ft, rho=rho, u=u, solver=sol)


def u_err(a, b, case):
    return np.abs(a["u"] - b["u"]).max() / np.linalg.norm(case.u_in)


def ft_err(a, b, lever=1.0):
    """Force/torque error of series a against b: max |dF| over the force
    components relative to the largest |F| of b, and max |dT| relative to
    max(largest |T| of b, largest |F| of b x a lever arm of `lever` cells), so
    that components that vanish by symmetry are compared at the scale of the
    ones that do not.  The torque about z (the one the adjoint's J is built on)
    is also compared at its own scale, max |dT_z| / max |T_z| of b, wherever it
    is at least a tenth of that body's torque scale above (a torque that is
    only round-off, as on a sphere in axial flow, is not)."""
    fa, fb = np.asarray(a["ft"]), np.asarray(b["ft"])
    sF = np.abs(fb[..., :3]).max()
    sT = max(np.abs(fb[..., 3:]).max(), sF * lever)
    eF = np.abs(fa[..., :3] - fb[..., :3]).max() / max(sF, 1e-300)
    eT = np.abs(fa[..., 3:] - fb[..., 3:]).max() / max(sT, 1e-300)
    eTz = 0.0
    ta, tb = fa.reshape(-1, fa.shape[-2], 6) if fa.ndim == 3 else fa[:, None], \
        fb.reshape(-1, fb.shape[-2], 6) if fb.ndim == 3 else fb[:, None]
    for body in range(tb.shape[1]):
        sTz = np.abs(tb[:, body, 5]).max()
        scale = max(np.abs(tb[:, body, 3:]).max(), np.abs(tb[:, body, :3]).max() * lever)
        if sTz > 0 and sTz >= 0.1 * scale:
            eTz = max(eTz, np.abs(ta[:, body, 5] - tb[:, body, 5]).max() / sTz)
    return max(eF, eT, eTz)


def assert_ft_same(fa, fb, storage):
    """Force/torque series of two runs with bit-identical states.  Kernels with
    the same tiling reduce in the same order and agree bit for bit; the TMA
    kernel gives 2-byte storage tiles of two cells per thread, so its warps
    hold other cells and their FP32 partial sums (32 cells, then added in
    FP64) round differently: 1e-6 of the largest component (a few FP32
    round-offs of a warp's terms)."""
    fa, fb = np.asarray(fa), np.asarray(fb)
    if storage in ("fp16", "bf16"):
        assert np.abs(fa - fb).max() <= 1e-6 * np.abs(fb).max()
    else:
        assert np.array_equal(fa, fb)
