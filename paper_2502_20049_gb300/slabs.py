"""z-slab decomposition of a PSM run (Sec. 5.2 runs one block of the lattice
per GPU, exchanges the populations that cross block faces every time step and
sums the force and torque over the blocks).

Each rank holds the planes [z0, z0 + nz) of the domain in a solver that is
periodic in z and knows its offset (``psm_set_z_offset``: cell centres, hence
the remap, u_s and the torque lever arm, are world positions).  A population
that leaves the slab through one face therefore wraps into the slots of the
opposite face of the same slab; the exchange moves it on to the neighbouring
slab.  With lo = plane 0, hi = plane nz - 1, UP = {i : c_z(i) = +1} and
DOWN = {i : c_z(i) = -1} (each solver's own direction order):

  two-grid step (push or pull)   after the step:   lo/UP -> rank + 1,  hi/DOWN -> rank - 1
  AA pattern, odd step           before the step:  hi/DOWN -> rank + 1, lo/UP -> rank - 1
                                 after the step:   lo/UP -> rank + 1,  hi/DOWN -> rank - 1
  AA pattern, even step          nothing crosses a face

(in the AA odd step a cell reads and writes the same slot of its neighbour:
the move before it brings the neighbour's value in to be read, the move after
it returns the value written).  The ranks form a ring: on a domain periodic in
z that is the whole story.  On a domain bounded by equilibrium ghost planes in
z the slots that a ring move fills at the domain's ends (rank 0's lo/UP after
a step, and before an AA odd step its hi/DOWN; rank N - 1's hi/DOWN after a
step, and before an AA odd step its lo/UP) take the inflow equilibrium
instead, of the slot's own direction in the natural layout and of the
opposite direction in the AA swapped layout.

A slab's own state is the domain's state on its planes after every
two-grid step and after every even number of AA steps (natural layout); in
the AA swapped layout, after an odd number of steps, a face cell's incoming
populations still sit in the neighbouring slab's slots until the next odd
step's exchange, so export the slabs (psm_get_state) after an even number.

Per exchange a face moves |UP| = 5 (D3Q19) or 9 (D3Q27) planes of nx * ny
values each way.  The force, torque and mass of the domain are the sums of the
slabs' (FP64, ``allreduce``).

Two transports: ``DistRing`` (one slab per process, torch.distributed
point-to-point: NCCL between GPUs, each rank receiving into its own buffers,
or gloo on CPU) and ``LocalRing`` (all slabs in one process, moved by copies).
A slab is any object with ``Q``, ``nz``, ``velocities()`` (c[Q, 3] in its
direction order), ``get_face(z, slots)`` -> [len(slots), ny, nx],
``set_face(z, slots, values)`` and ``fill_inflow(z, slots, dirs)``;
``PsmSlab`` adapts a ``psm.Solver``.
"""

from __future__ import annotations

import numpy as np


def partition(nz: int, world: int):
    """[(z0, nz_r)] for ranks 0..world-1: contiguous slabs, sizes differing by at most one."""
    if world < 1 or nz < world:
        raise ValueError(f"cannot split {nz} planes over {world} ranks")
    base, extra = divmod(nz, world)
    out, z0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z0, n))
        z0 += n
    return out


def face_slots(c):
    """(UP, DOWN, opp): direction indices with c_z = +1 and c_z = -1, and the opposite of each direction."""
    c = np.asarray(c)
    up = [i for i in range(len(c)) if c[i, 2] == 1]
    down = [i for i in range(len(c)) if c[i, 2] == -1]
    opp = [int(np.flatnonzero((c == -c[i]).all(1))[0]) for i in range(len(c))]
    return up, down, opp


def moves(streaming: str, step: int, when: str):
    """The face moves around step `step` (0-based global step index):
    list of (face, set, direction) with face 'lo'/'hi', set 'up'/'down',
    direction +1 (to rank + 1) or -1."""
    after = [("lo", "up", +1), ("hi", "down", -1)]
    if streaming == "twogrid":
        return after if when == "after" else []
    if step % 2 == 0:
        return []
    return [("hi", "down", +1), ("lo", "up", -1)] if when == "before" else after


class LocalRing:
    """All slabs of the ring in this process: a move is a rotation of the list."""

    def __init__(self, n: int):
        self.n = n
        self.ranks = list(range(n))

    def shift(self, faces, direction: int):
        # faces[k] is the face of slab k; slab k + direction receives it
        return [faces[(k - direction) % self.n] for k in range(self.n)]

    def allreduce(self, values):
        total = values[0]
        for v in values[1:]:
            total = total + v
        return [total for _ in values]


class DistRing:
    """One slab per process over torch.distributed (point-to-point to the ring
    neighbours; a GPU rank sends from and receives into its own device memory)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.n = dist.get_world_size(group)
        self.ranks = [self.rank]

    def _peer(self, r: int) -> int:
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def shift(self, faces, direction: int):
        import torch

        (face,) = faces
        if self.n == 1:
            return [face]
        send = face.contiguous()
        recv = torch.empty_like(send)
        d = self.dist
        ops = [d.P2POp(d.isend, send, self._peer((self.rank + direction) % self.n), self.group),
               d.P2POp(d.irecv, recv, self._peer((self.rank - direction) % self.n), self.group)]
        for req in d.batch_isend_irecv(ops):
            req.wait()
        return [recv]

    def allreduce(self, values):
        import torch

        (v,) = values
        t = torch.as_tensor(np.asarray(v, dtype=np.float64)).clone()
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, group=self.group)
        return [t.cpu().numpy()]


class Decomposition:
    """The exchange schedule of a ring of slabs.

    slabs: the slabs this process holds (one per rank with DistRing, all of
    them with LocalRing), in ring order; ring: LocalRing or DistRing;
    streaming: 'aa' or 'twogrid'; bounded: the domain's z ends are ghost
    planes (True) or periodic (False)."""

    def __init__(self, slabs, ring, streaming: str, bounded: bool):
        self.slabs = list(slabs)
        self.ring = ring
        self.streaming = streaming
        self.bounded = bounded
        self.step = 0
        up, down, opp = face_slots(self.slabs[0].velocities())
        self.sets = {"up": up, "down": down}
        self.opp = opp

    def _z(self, slab, face):
        return 0 if face == "lo" else slab.nz - 1

    def _ends(self, layout: str, before_odd: bool):
        """Refill the slots a ring move fills at the domain's ends with the inflow equilibrium."""
        if not self.bounded:
            return
        for slab, rank in zip(self.slabs, self.ring.ranks):
            for face, key, end in (("lo", "up", 0), ("hi", "down", self.ring.n - 1)):
                if before_odd:  # the swapped-layout slots read from beyond the end faces
                    face, key = ("hi", "down") if face == "lo" else ("lo", "up")
                if rank != end:
                    continue
                slots = self.sets[key]
                dirs = [self.opp[i] for i in slots] if layout == "swapped" else slots
                slab.fill_inflow(self._z(slab, face), slots, dirs)

    def prepare(self):
        """Before the first step (natural layout): the inflow equilibrium at the ends."""
        self._ends("natural", before_odd=False)

    def _move(self, when: str):
        for face, key, direction in moves(self.streaming, self.step, when):
            slots = self.sets[key]
            faces = [s.get_face(self._z(s, face), slots) for s in self.slabs]
            got = self.ring.shift(faces, direction)
            for s, v in zip(self.slabs, got):
                s.set_face(self._z(s, face), slots, v)
        if when == "before" and self.streaming == "aa" and self.step % 2 == 1:
            self._ends("swapped", before_odd=True)
        if when == "after" and moves(self.streaming, self.step, "after"):
            self._ends("natural", before_odd=False)

    def run(self, n: int, step_fn):
        """n time steps: step_fn(slab) advances one slab by one step."""
        for _ in range(n):
            self._move("before")
            for s in self.slabs:
                step_fn(s)
            self._move("after")
            self.step += 1

    def allreduce(self, values):
        """Sum per-slab FP64 values (force/torque, mass) over the ring."""
        return self.ring.allreduce(values)


class PsmSlab:
    """A psm.Solver as one slab (faces are torch views of its PDF buffer)."""

    def __init__(self, solver, z0: int):
        self.sol = solver
        self.Q = solver.cfg.Q
        self.nz = solver.cfg.nz
        solver.set_z_offset(z0)

    def velocities(self):
        from . import psm

        return psm.lattice_velocities(self.Q)[0]

    def get_face(self, z, slots):
        import torch

        return torch.stack([self.sol.slot_plane(i, z) for i in slots]).clone()

    def set_face(self, z, slots, values):
        for k, i in enumerate(slots):
            self.sol.slot_plane(i, z).copy_(values[k])

    def fill_inflow(self, z, slots, dirs):
        for i, d in zip(slots, dirs):
            self.sol.fill_slot_plane(i, z, d)
