"""z-slab decomposition (Sec. 5.2: one block of the lattice per GPU, the
populations crossing block faces exchanged every step) on the CPU.

The FP64 oracle, split into z-slabs that are each periodic in z and know their
world offset, stepped with the face exchange of paper_2502_20049_gb300.slabs,
equals the undecomposed oracle bit for bit in every PDF (the oracle streams
on two grids), on a domain periodic in z and on one bounded by equilibrium
ghost planes; force, torque and mass summed over the slabs agree to round-off
(the order of the sums differs).  Two and three gloo ranks exchange through
torch.distributed point-to-point (DistRing); one process holding all slabs
(LocalRing) covers one to four slabs, D3Q19 and D3Q27.
"""

import os
import socket

import numpy as np
import pytest

from paper_2502_20049_gb300 import slabs as S
from paper_2502_20049_gb300 import workloads as W


def case(Q=19, bc_z=1, nz=18):
    bodies = [W.BodyCase(W.ELLIPSOID, (4.0, 2.5, 3.0), 2, (6.2, 5.1, nz * 0.45), omega=(0.01, 0.02, 0.03),
                         v=(0.0, 0.0, 0.02)),
              W.BodyCase(W.BOX, (1.5, 1.5, 2.0), 1, (3.0, 7.5, nz * 0.8), omega=(0.0, 0.0, -0.04),
                         v=(0.01, 0.0, -0.03))]
    return W.Case("slabs", 12, 10, nz, Q=Q, storage="fp64", streaming="twogrid", fluid="trt", tau=0.7, solid=1,
                  weighting=1, bc_z=bc_z, u_in=(0.01, -0.005, 0.02), steps=25, bodies=bodies)


class OracleSlab:
    """One z-slab of a case as an oracle simulation (periodic in z, world offset z0)."""

    def __init__(self, c, z0, nz):
        import oracle

        self.O = oracle
        self.Q, self.nz, self.rho0, self.u_in = c.Q, nz, c.rho0, tuple(c.u_in)
        cfg = oracle.Config(nx=c.nx, ny=c.ny, nz=nz, Q=c.Q, bc_z=0, rho0=c.rho0, u_in=tuple(c.u_in),
                            fluid={"bgk": 0, "trt": 1}[c.fluid], tau=c.tau, trt_lambda=c.trt_lambda, solid=c.solid,
                            weighting=c.weighting, z0=z0)
        self.sim = oracle.Sim(cfg, threads=1)
        for b in c.bodies:
            sub, lo = oracle.voxelize(b.kind, b.params, b.s)
            self.sim.add_body(oracle.BodySpec(sub=sub, s=b.s, lo=lo, R0=tuple(b.R0), Q0=np.array(b.Q0),
                                              omega=tuple(b.omega), v=tuple(b.v)))
        self.sim.init_eq(c.rho0, c.u_in)

    def velocities(self):
        return self.O.lattice(self.Q)[0]

    def get_face(self, z, slots):
        import torch

        return torch.from_numpy(self.sim.get_f()[slots, z].copy())

    def set_face(self, z, slots, values):
        f = self.sim.get_f()
        f[slots, z] = np.asarray(values)
        self.sim.set_f(f)

    def fill_inflow(self, z, slots, dirs):
        f = self.sim.get_f()
        for i, d in zip(slots, dirs):
            f[i, z] = self.O.feq(self.Q, d, self.rho0, self.u_in)
        self.sim.set_f(f)


def reference(c):
    import oracle
    from oracle.cases import sim_from_case

    sim = sim_from_case(c, threads=1)
    sim.step(c.steps)
    return sim.get_f(), sim.force_torque()


def run_local(c, world):
    parts = S.partition(c.nz, world)
    slabs = [OracleSlab(c, z0, n) for z0, n in parts]
    dec = S.Decomposition(slabs, S.LocalRing(world), "twogrid", bounded=c.bc_z == 1)
    dec.prepare()
    dec.run(c.steps, lambda s: s.sim.step(1))
    f = np.concatenate([s.sim.get_f() for s in slabs], axis=1)
    ft = dec.allreduce([s.sim.force_torque() for s in slabs])[0]
    return f, ft


def check(c, f, ft, ref):
    fr, ftr = ref
    assert np.array_equal(f, fr), np.abs(f - fr).max()
    assert np.abs(ft - ftr).max() <= 1e-12 * np.abs(ftr).max()
    assert abs(f.sum() - fr.sum()) <= 1e-12 * fr.sum()
    assert np.abs(ftr).max() > 0


def test_partition_and_moves():
    assert S.partition(18, 4) == [(0, 5), (5, 5), (10, 4), (14, 4)]
    assert S.partition(7, 1) == [(0, 7)]
    with pytest.raises(ValueError):
        S.partition(3, 4)
    assert S.moves("twogrid", 4, "before") == [] and len(S.moves("twogrid", 4, "after")) == 2
    assert S.moves("aa", 2, "before") == [] and S.moves("aa", 2, "after") == []
    assert S.moves("aa", 3, "before") == [("hi", "down", +1), ("lo", "up", -1)]
    assert S.moves("aa", 3, "after") == [("lo", "up", +1), ("hi", "down", -1)]
    up, down, opp = S.face_slots(np.array([[0, 0, 0], [0, 0, 1], [0, 0, -1], [1, 0, 1], [-1, 0, -1]]))
    assert up == [1, 3] and down == [2, 4] and opp == [0, 2, 1, 4, 3]


@pytest.mark.parametrize("bc_z", [0, 1])
@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_local_ring_equals_undecomposed(oracle_mod, world, bc_z):
    c = case(bc_z=bc_z)
    check(c, *run_local(c, world), reference(c))


@pytest.mark.parametrize("bc_z", [0, 1])
def test_local_ring_d3q27(oracle_mod, bc_z):
    c = case(Q=27, bc_z=bc_z, nz=13).with_(steps=15)
    check(c, *run_local(c, 3), reference(c))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, bc_z, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist

    dist.init_process_group("gloo")
    try:
        c = case(bc_z=bc_z)
        z0, n = S.partition(c.nz, world)[rank]
        slab = OracleSlab(c, z0, n)
        dec = S.Decomposition([slab], S.DistRing(), "twogrid", bounded=bc_z == 1)
        dec.prepare()
        dec.run(c.steps, lambda s: s.sim.step(1))
        ft = dec.allreduce([slab.sim.force_torque()])[0]
        out.put((rank, z0, slab.sim.get_f(), ft))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,bc_z", [(2, 1), (3, 0)])
def test_gloo_ranks_equal_undecomposed(oracle_mod, world, bc_z):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, bc_z, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c = case(bc_z=bc_z)
    f = np.concatenate([r[2] for r in res], axis=1)
    for r in res[1:]:
        assert np.array_equal(r[3], res[0][3])  # every rank holds the same all-reduced sums
    check(c, f, res[0][3], reference(c))
