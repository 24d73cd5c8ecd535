"""Build an oracle simulation from a synthetic workload case (test
infrastructure only, like the rest of this package)."""

import numpy as np

from . import BodySpec, Config, Sim, voxelize

FLUID = {"bgk": 0, "trt": 1, "cumulant": 2}


def sim_from_case(case, threads=None, init: bool = True) -> Sim:
    """Oracle Sim for a paper_2502_20049_gb300.workloads.Case: same grid,
    collision and bodies (voxelised by the oracle), equilibrium initial state
    at (rho0, u_in) (init=False: no state is allocated, for one-cell
    collisions of grids too large to hold).  The oracle always computes in
    FP64; the case's storage precision does not apply to it."""
    cfg = Config(nx=case.nx, ny=case.ny, nz=case.nz, Q=case.Q, bc_z=case.bc_z, rho0=case.rho0,
                 u_in=tuple(case.u_in), fluid=FLUID[case.fluid], tau=case.tau, trt_lambda=case.trt_lambda,
                 solid=case.solid, weighting=case.weighting, cum_rates=tuple(case.cum_rates))
    sim = Sim(cfg, threads=threads)
    for b in case.bodies:
        sub, lo = voxelize(b.kind, b.params, b.s)
        sim.add_body(BodySpec(sub=sub, s=b.s, lo=lo, R0=tuple(b.R0), Q0=np.array(b.Q0), omega=tuple(b.omega),
                              v=tuple(b.v)))
    if init:
        sim.init_eq(case.rho0, case.u_in)
    return sim
