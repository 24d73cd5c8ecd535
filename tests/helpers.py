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


def ft_err(a, b):
    """max |FT_a - FT_b| per component, relative to the component's max |FT_b|."""
    fa, fb = a["ft"], b["ft"]
    scale = np.abs(fb).max(axis=0, keepdims=True)
    scale = np.maximum(scale, 1e-300)
    return (np.abs(fa - fb) / scale).max()
