"""Synthetic workloads and seeded input generators.

This module holds no arithmetic of the method: only sizes, body parameters,
seeds and random-number draws.  Both the CUDA path (through the binding) and
the CPU oracle (in the tests and the CPU baseline) take their inputs from here.

The bodies stand in for the paper's meshes (the CROR rotor of Sec. 3 and the
cube / bunny / rotor of Table I-III are not available): an analytic sphere,
ellipsoid, box and a synthetic counter-rotating rotor (hub cylinder with
twisted thin elliptic blades).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

SEED = 20250227

# analytic shape kinds shared by the library voxeliser and the oracle voxeliser
SPHERE, ELLIPSOID, BOX, ROTOR = 0, 1, 2, 3


@dataclass(frozen=True)
class Rotor:
    """One rotor of the synthetic counter-rotating open rotor.

    Body frame: hub axis = z.  Hub: cylinder of radius r_hub and length hub_len.
    Blades k = 0..n_blades-1 at azimuth phase + 2 pi k / n_blades, spanning radii
    r_hub .. r_hub + span, elliptic section chord x thickness, pitch (from the
    rotation plane) pitch_root_deg at the root, decreasing linearly by
    twist_deg to the tip; hand = -1 mirrors the pitch.
    """

    r_hub: float = 20.0
    hub_len: float = 40.0
    span: float = 120.0
    chord: float = 24.0
    thickness: float = 4.0
    pitch_root_deg: float = 60.0
    twist_deg: float = 30.0
    phase: float = 0.0
    n_blades: int = 6
    hand: int = 1

    def params(self):
        return (self.r_hub, self.hub_len, self.span, self.chord, self.thickness, self.pitch_root_deg,
                self.twist_deg, self.phase, float(self.n_blades), float(self.hand))

    def scaled(self, k: float) -> "Rotor":
        return replace(self, r_hub=self.r_hub * k, hub_len=self.hub_len * k, span=self.span * k,
                       chord=self.chord * k, thickness=self.thickness * k)


@dataclass
class BodyCase:
    kind: int
    params: tuple
    s: int
    R0: tuple
    omega: tuple = (0.0, 0.0, 0.0)
    v: tuple = (0.0, 0.0, 0.0)
    Q0: tuple = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)


@dataclass
class Case:
    """One synthetic PSM run: grid, lattice, collision, bodies, steps."""

    name: str
    nx: int
    ny: int
    nz: int
    Q: int = 19
    storage: str = "fp32"         # fp64 | fp32 | fp16 | bf16
    streaming: str = "aa"         # aa | twogrid
    fluid: str = "bgk"            # bgk | trt | cumulant (D3Q19)
    tau: float = 0.8
    trt_lambda: float = 3.0 / 16.0
    cum_rates: tuple = (1.0, 1.0, 1.0)  # cumulant: bulk, third-order, fourth-order rates
    solid: int = 1                # SC1 / SC2 / SC3 (Eq. 7 / 8 / 9)
    weighting: int = 1            # 0: Eq. 5, 1: Eq. 6
    bc_z: int = 1                 # 0 periodic, 1 equilibrium inlet/outlet planes
    rho0: float = 1.0
    u_in: tuple = (0.0, 0.0, 0.01)
    steps: int = 200
    bodies: list = field(default_factory=list)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def with_(self, **kw) -> "Case":
        return replace(self, **kw)


def c1_sphere() -> Case:
    """D3Q19 BGK, 32^3, FP64, sphere r=6 centred, s=3 (8^3 supersampling), 200 steps."""
    return Case("c1_sphere_32", 32, 32, 32, Q=19, storage="fp64", fluid="bgk", tau=0.8, u_in=(0.0, 0.0, 0.01),
                steps=200, bodies=[BodyCase(SPHERE, (6.0,), 3, (16.0, 16.0, 16.0))])


def c2_ellipsoid(scale: float = 1.0, n: int = 256, steps: int = 1000, omega_z: float = 2e-4) -> Case:
    """D3Q19 TRT, n^3, FP32, uniform inflow 0.05, tau 0.55, rotating ellipsoid 40/20/8 (x scale) about z."""
    c = n / 2.0
    return Case(f"c2_ellipsoid_{n}", n, n, n, Q=19, storage="fp32", fluid="trt", tau=0.55, u_in=(0.0, 0.0, 0.05),
                steps=steps,
                bodies=[BodyCase(ELLIPSOID, (40.0 * scale, 20.0 * scale, 8.0 * scale), 2, (c, c, c),
                                 omega=(0.0, 0.0, omega_z))])


def rotor_pair(scale: float, axis_xy: tuple, z_front: float, z_back: float, omega: float, s: int = 2):
    front = Rotor().scaled(scale)
    back = replace(Rotor(n_blades=5, phase=math.pi / 5, hand=-1).scaled(scale))
    return [BodyCase(ROTOR, front.params(), s, (axis_xy[0], axis_xy[1], z_front), omega=(0.0, 0.0, omega)),
            BodyCase(ROTOR, back.params(), s, (axis_xy[0], axis_xy[1], z_back), omega=(0.0, 0.0, -omega))]


def c3_rotor(storage: str = "fp32", scale: float = 1.0, dims=(512, 512, 640), steps: int = 2000) -> Case:
    """D3Q27, counter-rotating rotor (6 + 5 blades) at +-3e-4 rad/step, inflow 0.04."""
    nx, ny, nz = dims
    k = scale
    return Case(f"c3_rotor_{nx}x{ny}x{nz}_{storage}", nx, ny, nz, Q=27, storage=storage, fluid="bgk", tau=0.55,
                u_in=(0.0, 0.0, 0.04), steps=steps,
                bodies=rotor_pair(k, (nx / 2.0, ny / 2.0), nz * 0.375, nz * 0.5625, 3e-4))


def c4_adjoint(n: int = 128, steps: int = 512) -> Case:
    """D3Q19 TRT FP32, n^3, ellipsoid 20/10/4 rotating about z at 2e-4, inflow 0.05."""
    c = n / 2.0
    k = n / 256.0
    return Case(f"c4_adjoint_{n}", n, n, n, Q=19, storage="fp32", fluid="trt", tau=0.55, u_in=(0.0, 0.0, 0.05),
                steps=steps,
                bodies=[BodyCase(ELLIPSOID, (80.0 * k, 40.0 * k, 16.0 * k), 2, (c, c, c), omega=(0.0, 0.0, 2e-4))])


def c5_large(dims=(1024, 1024, 960), steps: int = 500) -> Case:
    """D3Q19 BGK, AA in place, FP16 shifted storage, rotor of c3 scaled x2."""
    nx, ny, nz = dims
    return Case(f"c5_rotor_{nx}x{ny}x{nz}_fp16", nx, ny, nz, Q=19, storage="fp16", fluid="bgk", tau=0.55,
                u_in=(0.0, 0.0, 0.04), steps=steps,
                bodies=rotor_pair(2.0 * nx / 1024.0, (nx / 2.0, ny / 2.0), nz * 0.375, nz * 0.625, 3e-4))


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_positive(shape, seed: int = SEED, lo: float = 0.02, hi: float = 0.06) -> np.ndarray:
    """Uniform random values in [lo, hi) (used as PDF sets far from equilibrium)."""
    return rng(seed).uniform(lo, hi, size=shape)


def random_unit(shape, seed: int = SEED) -> np.ndarray:
    """Uniform random values in [-1, 1)."""
    return rng(seed).uniform(-1.0, 1.0, size=shape)


def pick_cells(mask: np.ndarray, k: int, seed: int = SEED) -> np.ndarray:
    """k distinct flat indices drawn uniformly from the True cells of mask."""
    idx = np.flatnonzero(mask.reshape(-1))
    return np.sort(rng(seed).choice(idx, size=min(k, idx.size), replace=False))


# ---------------------------------------------------------------------------
# Synthetic closed triangle meshes (inputs of the mesh voxeliser; the paper's
# CROR and bunny meshes are not available).  Vertices float32 [nv, 3] in body
# frame lattice units, triangles int32 [nt, 3], outward orientation.
# ---------------------------------------------------------------------------
def box_mesh(lo, hi):
    """Axis-aligned box [lo, hi] as 12 triangles."""
    (x0, y0, z0), (x1, y1, z1) = lo, hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float32)
    t = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4],
                  [1, 2, 6], [1, 6, 5], [2, 3, 7], [2, 7, 6], [3, 0, 4], [3, 4, 7]], dtype=np.int32)
    return v, t


def icosphere(radius: float, subdiv: int, centre=(0.0, 0.0, 0.0)):
    """Sphere approximated by a subdivided icosahedron (vertices on the sphere)."""
    g = (1.0 + 5 ** 0.5) / 2.0
    v = [[-1, g, 0], [1, g, 0], [-1, -g, 0], [1, -g, 0], [0, -1, g], [0, 1, g], [0, -1, -g], [0, 1, -g],
         [g, 0, -1], [g, 0, 1], [-g, 0, -1], [-g, 0, 1]]
    f = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
         [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5], [2, 4, 11],
         [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    for _ in range(subdiv):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                mid[key] = len(v) - 1
            return mid[key]

        f = [t for a, b, c in f for t in ([a, m(a, b), m(c, a)], [b, m(b, c), m(a, b)], [c, m(c, a), m(b, c)],
                                          [m(a, b), m(b, c), m(c, a)])]
    return (np.array(v) * radius + np.array(centre)).astype(np.float32), np.array(f, dtype=np.int32)


def torus_mesh(R: float, r: float, nu: int = 48, nv: int = 24):
    """Torus about the z axis (tube radius r around the circle of radius R)."""
    u = 2 * np.pi * np.arange(nu) / nu
    w = 2 * np.pi * np.arange(nv) / nv
    U, Wv = np.meshgrid(u, w, indexing="ij")
    x = (R + r * np.cos(Wv)) * np.cos(U)
    y = (R + r * np.cos(Wv)) * np.sin(U)
    z = r * np.sin(Wv)
    v = np.stack([x, y, z], -1).reshape(-1, 3).astype(np.float32)
    tri = []
    for i in range(nu):
        for j in range(nv):
            a, b = i * nv + j, ((i + 1) % nu) * nv + j
            c, d = ((i + 1) % nu) * nv + (j + 1) % nv, i * nv + (j + 1) % nv
            tri += [[a, b, c], [a, c, d]]
    return v, np.array(tri, dtype=np.int32)


def merge_meshes(*meshes):
    """Disjoint closed meshes as one (components must not intersect)."""
    vs, ts, off = [], [], 0
    for v, t in meshes:
        vs.append(v)
        ts.append(t + off)
        off += len(v)
    return np.concatenate(vs).astype(np.float32), np.concatenate(ts).astype(np.int32)


def transform_mesh(mesh, R=None, shift=(0.0, 0.0, 0.0)):
    v, t = mesh
    v = v.astype(np.float64)
    if R is not None:
        v = v @ np.asarray(R, dtype=np.float64).T
    return (v + np.asarray(shift)).astype(np.float32), t


def rot(axis: str, angle: float):
    c, s = np.cos(angle), np.sin(angle)
    if axis == "x":
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == "y":
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
