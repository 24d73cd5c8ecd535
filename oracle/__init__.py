"""FP64 CPU oracle of the PSM lattice Boltzmann step (arXiv 2502.20049).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct restatement of the
method that the CUDA library is checked against.  Only the test suite, the
smoke check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library; the C++ source is
``psm_oracle.cpp`` next to this file and is compiled with
``-ffp-contract=off`` so that every float/double operation rounds on its own.

What each function follows (sections and equations of the paper):

* :func:`lattice` -- D3Q19 / D3Q27 velocity sets (Sec. 2.2 names them).
* :func:`feq` -- Eq. 3, read with ``-u.u/(2 c_s^2)`` (the printed ``+`` is a
  typo: with it the zeroth moment is not rho).
* :func:`weighting` -- Eq. 5 (``mode=0``) and Eq. 6 (``mode=1``).
* :class:`Sim` -- one step = remap (Sec. 3) -> Eq. 4 with Eq. 2 / TRT / the
  cumulant operator of Sec. 2.2 / Sec. 5.1 (D3Q19) and the solid
  collision Eq. 7 / 8 / 9 -> force and torque Eq. 10 / 11 -> streaming Eq. 1.
* :func:`voxelize`, :func:`remap` -- the super-sampled geometry field and its
  per-step interpolation onto the lattice (Sec. 3).
* :class:`TangentSim` -- the same code on dual numbers: exact directional
  derivatives of the force/torque series (the reference the adjoint is
  checked against).

Parity status: every function above is pinned by the tests in
``tests/test_oracle_*.py`` (closed forms, invariants, brute force).  The torque
magnitude is pinned on a slowly rotating sphere (Stokes' closed form); the
synthetic rotor's torque has no closed form of its own, but each ingredient
(its voxelisation, the remap, the torque sum) is pinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psm_oracle.cpp")
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

KIND_SPHERE, KIND_ELLIPSOID, KIND_BOX, KIND_ROTOR = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, FP contraction off)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", tmp, _SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.POINTER
            d, i, l, vp = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
            dp, ip, u8p = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_uint8)
            sig = {
                "or_lattice": (i, [i, ip, dp, ip]),
                "or_feq": (d, [i, i, d, dp]),
                "or_weighting": (d, [i, d, d]),
                "or_shape_box": (i, [i, dp, ip, dp]),
                "or_voxelize": (i, [i, dp, i, u8p]),
                "or_inside": (i, [i, dp, d, d, d]),
                "or_mesh_box": (i, [vp, l, i, vp, dp]),
                "or_voxelize_mesh": (i, [vp, l, vp, l, i, u8p]),
                "or_remap": (i, [u8p, i, i, i, i, dp, dp, dp, dp, dp, l, i, i, i, dp]),
                "or_pose": (i, [dp, dp, dp, dp, l, dp, dp]),
                "or_create": (vp, [vp]),
                "or_destroy": (None, [vp]),
                "or_set_threads": (i, [vp, i]),
                "or_get_threads": (i, [vp]),
                "or_add_body": (i, [vp, u8p, i, i, i, i, dp, dp, dp, dp, dp]),
                "or_init_eq": (i, [vp, d, dp]),
                "or_set_body_us_omega": (i, [vp, i, dp]),
                "or_set_body_dynamics": (i, [vp, i, d, dp, dp, dp]),
                "or_body_state": (i, [vp, i, dp]),
                "or_set_f": (i, [vp, dp]),
                "or_get_f": (i, [vp, dp]),
                "or_set_delta": (i, [vp, dp]),
                "or_step": (i, [vp, i]),
                "or_step_count": (l, [vp]),
                "or_ft": (i, [vp, dp]),
                "or_eps": (i, [vp, l, dp, ip]),
                "or_macroscopic": (i, [vp, dp, dp]),
                "or_update_cells": (i, [vp, P(ctypes.c_long), l, dp]),
                "or_collide_at": (i, [vp, l, i, i, i, dp, dp, dp, dp]),
                "ort_create": (vp, [vp, dp]),
                "ort_destroy": (None, [vp]),
                "ort_set_threads": (i, [vp, i]),
                "ort_add_body": (i, [vp, u8p, i, i, i, i, dp, dp, dp, dp, dp, dp]),
                "ort_init_eq": (i, [vp, d, dp, dp]),
                "ort_set_delta": (i, [vp, dp, dp]),
                "ort_step": (i, [vp, i]),
                "ort_ft": (i, [vp, dp, dp]),
                "ort_get_f": (i, [vp, dp, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _d3(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("Q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc_z", ctypes.c_int), ("walls_y", ctypes.c_int),
        ("wall_u_lo", ctypes.c_double * 3), ("wall_u_hi", ctypes.c_double * 3),
        ("force", ctypes.c_double * 3), ("rho0", ctypes.c_double), ("u_in", ctypes.c_double * 3),
        ("fluid", ctypes.c_int), ("tau", ctypes.c_double), ("trt_lambda", ctypes.c_double),
        ("solid", ctypes.c_int), ("weighting", ctypes.c_int), ("cum_rates", ctypes.c_double * 3),
        ("z0", ctypes.c_int),
    ]


@dataclass
class Config:
    """Oracle configuration (mirrors ``or_config`` in psm_oracle.cpp).

    ``bc_z``: 0 periodic, 1 equilibrium ghost planes f^eq(rho0, u_in) at z=-1 and
    z=nz.  ``fluid``: 0 BGK (Eq. 2), 1 TRT, 2 cumulant (D3Q19; ``cum_rates`` =
    bulk, third-order and fourth-order rates; the shear rate is 1/tau).
    ``solid``: 1/2/3 = Eq. 7/8/9.
    ``weighting``: 0 Eq. 5, 1 Eq. 6.  ``walls_y`` and ``force`` are oracle-only
    (half-way bounce-back walls and a Guo body force, used by the pins).
    ``z0``: world z index of plane 0 (the grid is the slab [z0, z0 + nz) of a
    larger domain; the geometry uses world cell centres).
    """

    nx: int
    ny: int
    nz: int
    Q: int = 19
    bc_z: int = 1
    rho0: float = 1.0
    u_in: tuple = (0.0, 0.0, 0.0)
    fluid: int = 0
    tau: float = 0.8
    trt_lambda: float = 3.0 / 16.0
    solid: int = 1
    weighting: int = 1
    walls_y: int = 0
    wall_u_lo: tuple = (0.0, 0.0, 0.0)
    wall_u_hi: tuple = (0.0, 0.0, 0.0)
    force: tuple = (0.0, 0.0, 0.0)
    cum_rates: tuple = (1.0, 1.0, 1.0)
    z0: int = 0

    def _c(self):
        c = _Cfg()
        c.Q, c.nx, c.ny, c.nz = self.Q, self.nx, self.ny, self.nz
        c.bc_z, c.walls_y = self.bc_z, self.walls_y
        for k in range(3):
            c.wall_u_lo[k] = self.wall_u_lo[k]
            c.wall_u_hi[k] = self.wall_u_hi[k]
            c.force[k] = self.force[k]
            c.u_in[k] = self.u_in[k]
            c.cum_rates[k] = self.cum_rates[k]
        c.rho0, c.fluid, c.tau, c.trt_lambda = self.rho0, self.fluid, self.tau, self.trt_lambda
        c.solid, c.weighting = self.solid, self.weighting
        c.z0 = self.z0
        return c


def lattice(Q: int):
    """(c[Q,3] int, w[Q], opp[Q]) in the oracle's own direction order."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    rc = _lib().or_lattice(Q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                           opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise ValueError(f"unsupported stencil Q={Q}")
    return c.astype(np.int64), w, opp.astype(np.int64)


def feq(Q: int, i: int, rho: float, u) -> float:
    """Eq. 3 (sign-corrected) for direction i of the oracle's order."""
    u = _d3(u)
    return _lib().or_feq(Q, i, rho, _dp(u))


def weighting(mode: int, eps: float, tau: float) -> float:
    """B(eps): Eq. 5 (mode 0) or Eq. 6 (mode 1)."""
    return _lib().or_weighting(mode, eps, tau)


def shape_box(kind: int, params):
    """Coarse-cell dims and body-frame origin of an analytic shape's geometry box."""
    p = _d3(params)
    dims = np.zeros(3, dtype=np.int32)
    lo = np.zeros(3)
    _lib().or_shape_box(kind, _dp(p), dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(lo))
    return tuple(int(v) for v in dims), lo


def voxelize(kind: int, params, s: int):
    """Binary super-sampled geometry field of an analytic shape (Sec. 3).

    Returns (sub[nsz, nsy, nsx] uint8, lo[3]); sub-cell size 2^-s, bit = sub-cell
    centre inside the shape.
    """
    p = _d3(params)
    dims, lo = shape_box(kind, p)
    n = 1 << s
    sub = np.zeros((dims[2] * n, dims[1] * n, dims[0] * n), dtype=np.uint8)
    _lib().or_voxelize(kind, _dp(p), s, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return sub, lo


def voxelize_mesh(vertices, triangles, s: int):
    """Binary super-sampled field of a closed triangle mesh by brute-force ray
    parity in exact integer arithmetic (Sec. 3; rules in psm_oracle.cpp).

    vertices [nv, 3] (float32 body-frame lattice units), triangles [nt, 3]
    (int32).  Returns (sub[nsz, nsy, nsx] uint8, lo[3])."""
    v = np.ascontiguousarray(vertices, dtype=np.float32)
    t = np.ascontiguousarray(triangles, dtype=np.int32)
    dims = np.zeros(3, dtype=np.int64)
    lo = np.zeros(3)
    if _lib().or_mesh_box(v.ctypes.data, len(v), s, dims.ctypes.data, _dp(lo)) != 0:
        raise ValueError("mesh outside the supported box or s out of 0..3")
    n = 1 << s
    sub = np.zeros((dims[2] * n, dims[1] * n, dims[0] * n), dtype=np.uint8)
    if _lib().or_voxelize_mesh(v.ctypes.data, len(v), t.ctypes.data, len(t), s,
                               sub.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))) != 0:
        raise ValueError("bad mesh")
    return sub, lo


def inside(kind: int, params, x: float, y: float, z: float) -> bool:
    p = _d3(params)
    return bool(_lib().or_inside(kind, _dp(p), x, y, z))


def pose(Q0, R0, omega, v, n: int):
    """Rotation Q_n (world <- body, 3x3) and reference point R_n at step n."""
    Qo = np.zeros(9)
    Ro = np.zeros(3)
    _lib().or_pose(_dp(_d3(Q0)), _dp(_d3(R0)), _dp(_d3(omega)), _dp(_d3(v)), int(n), _dp(Qo), _dp(Ro))
    return Qo.reshape(3, 3), Ro


def remap(sub, s, lo, Q0, R0, omega, v, n, shape):
    """eps[nz, ny, nx] of one body at the pose of step n (Sec. 3)."""
    sub = np.ascontiguousarray(sub, dtype=np.uint8)
    nsz, nsy, nsx = sub.shape
    nx, ny, nz = shape
    eps = np.zeros((nz, ny, nx))
    _lib().or_remap(sub.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nsx, nsy, nsz, s, _dp(_d3(lo)),
                    _dp(_d3(Q0)), _dp(_d3(R0)), _dp(_d3(omega)), _dp(_d3(v)), int(n), nx, ny, nz, _dp(eps))
    return eps


IDENTITY = np.eye(3).reshape(-1)


@dataclass
class BodySpec:
    """A rigid body for the oracle: geometry field + motion (Sec. 3)."""

    sub: np.ndarray
    s: int
    lo: np.ndarray
    R0: tuple
    Q0: np.ndarray = field(default_factory=lambda: IDENTITY.copy())
    omega: tuple = (0.0, 0.0, 0.0)
    v: tuple = (0.0, 0.0, 0.0)


class Sim:
    """FP64 oracle simulation (two-grid, natural pre-collision state f[Q,nz,ny,nx])."""

    def __init__(self, cfg: Config, threads: int | None = None):
        self.cfg = cfg
        self._h = _lib().or_create(ctypes.byref(cfg._c()))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        if threads is not None:
            _lib().or_set_threads(self._h, int(threads))
        self.nbodies = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib().or_destroy(h)
            self._h = None

    @property
    def threads(self) -> int:
        return _lib().or_get_threads(self._h)

    @property
    def shape(self):
        c = self.cfg
        return (c.Q, c.nz, c.ny, c.nx)

    def add_body(self, b: BodySpec) -> int:
        sub = np.ascontiguousarray(b.sub, dtype=np.uint8)
        nsz, nsy, nsx = sub.shape
        self.nbodies += 1
        return _lib().or_add_body(self._h, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nsx, nsy, nsz,
                                  b.s, _dp(_d3(b.lo)), _dp(_d3(b.Q0)), _dp(_d3(b.R0)), _dp(_d3(b.omega)),
                                  _dp(_d3(b.v)))

    def init_eq(self, rho: float = 1.0, u=(0.0, 0.0, 0.0)):
        _lib().or_init_eq(self._h, rho, _dp(_d3(u)))

    def set_us_omega(self, body: int, omega):
        """Angular velocity used in u_s only (the geometry keeps its pose sequence)."""
        if _lib().or_set_body_us_omega(self._h, int(body), _dp(_d3(omega))) != 0:
            raise IndexError(body)

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape)
        _lib().or_set_f(self._h, _dp(f))

    def get_f(self):
        f = np.zeros(self.shape)
        _lib().or_get_f(self._h, _dp(f))
        return f

    def set_delta(self, d):
        if d is None:
            _lib().or_set_delta(self._h, None)
            return
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1)
        _lib().or_set_delta(self._h, _dp(d))

    def step(self, n: int = 1):
        _lib().or_step(self._h, int(n))

    @property
    def step_count(self) -> int:
        return _lib().or_step_count(self._h)

    def set_body_dynamics(self, b: int, mass: float, inertia, force_ext=(0.0, 0.0, 0.0), torque_ext=(0.0, 0.0, 0.0)):
        """Two-way coupling of body b from the current step (semi-implicit Euler
        of the rigid-body equations of motion under the force and torque of each
        step plus constant external loads)."""
        Ib = np.ascontiguousarray(inertia, dtype=np.float64).reshape(9)
        if _lib().or_set_body_dynamics(self._h, b, float(mass), _dp(Ib), _dp(_d3(force_ext)),
                                       _dp(_d3(torque_ext))) != 0:
            raise ValueError("bad body dynamics")

    def body_state(self, b: int):
        """dict R, v, Q (3x3), omega, L of body b for the next step."""
        out = np.zeros(21)
        _lib().or_body_state(self._h, b, _dp(out))
        return dict(R=out[0:3], v=out[3:6], Q=out[6:15].reshape(3, 3), omega=out[15:18], L=out[18:21])

    def force_torque(self):
        """[steps, nbodies, 6] force and torque ON each body (-S of Eq. 10/11)."""
        nb = max(self.nbodies, 1)
        out = np.zeros(max(self.step_count * nb * 6, 1))
        _lib().or_ft(self._h, _dp(out))
        return out[: self.step_count * self.nbodies * 6].reshape(self.step_count, self.nbodies, 6)

    def eps(self, n: int | None = None):
        """(eps[nz,ny,nx], owner[nz,ny,nx]) at the pose of step n (default: current)."""
        n = self.step_count if n is None else n
        c = self.cfg
        e = np.zeros((c.nz, c.ny, c.nx))
        o = np.zeros((c.nz, c.ny, c.nx), dtype=np.int32)
        _lib().or_eps(self._h, int(n), _dp(e), o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return e, o

    def update_cells(self, cells):
        """f_i(x, n+1) [len(cells), Q] at flat cell indices, from the current state
        (no step is taken); oracle direction order."""
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
        out = np.zeros((cells.size, self.cfg.Q))
        rc = _lib().or_update_cells(self._h, cells.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), cells.size,
                                    _dp(out))
        if rc != 0:
            raise IndexError("cell index out of range")
        return out

    def collide_at(self, n: int, x: int, y: int, z: int, f_in):
        """(post[Q], g[3], eps) of cell (x, y, z) at the pose of step n from given
        pre-collision PDFs f_in[Q] (oracle direction order)."""
        f_in = np.ascontiguousarray(f_in, dtype=np.float64).reshape(self.cfg.Q)
        post = np.zeros(self.cfg.Q)
        g = np.zeros(3)
        e = np.zeros(1)
        if _lib().or_collide_at(self._h, int(n), int(x), int(y), int(z), _dp(f_in), _dp(post), _dp(g), _dp(e)) != 0:
            raise IndexError((x, y, z))
        return post, g, float(e[0])

    def macroscopic(self):
        """(rho[nz,ny,nx], u[nz,ny,nx,3]) with u = j / rho."""
        c = self.cfg
        rho = np.zeros((c.nz, c.ny, c.nx))
        u = np.zeros((c.nz, c.ny, c.nx, 3))
        _lib().or_macroscopic(self._h, _dp(rho), _dp(u))
        return rho, u


class TangentSim:
    """Tangent-linear oracle: the same step on dual numbers.

    Seeds are set at construction (``d_u_in``), per body (``d_omega``) and per
    cell (``set_delta(delta, d_delta)``); :meth:`force_torque` returns values
    and exact directional derivatives of the force/torque series.  The eps
    sequence is taken at the nominal angular velocity (frozen geometry).
    """

    def __init__(self, cfg: Config, d_u_in=(0.0, 0.0, 0.0), threads: int | None = None):
        self.cfg = cfg
        self._h = _lib().ort_create(ctypes.byref(cfg._c()), _dp(_d3(d_u_in)))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        if threads is not None:
            _lib().ort_set_threads(self._h, int(threads))
        self.nbodies = 0
        self.steps = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib().ort_destroy(h)
            self._h = None

    @property
    def shape(self):
        c = self.cfg
        return (c.Q, c.nz, c.ny, c.nx)

    def add_body(self, b: BodySpec, d_omega=(0.0, 0.0, 0.0)) -> int:
        sub = np.ascontiguousarray(b.sub, dtype=np.uint8)
        nsz, nsy, nsx = sub.shape
        self.nbodies += 1
        return _lib().ort_add_body(self._h, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nsx, nsy, nsz,
                                   b.s, _dp(_d3(b.lo)), _dp(_d3(b.Q0)), _dp(_d3(b.R0)), _dp(_d3(b.omega)),
                                   _dp(_d3(d_omega)), _dp(_d3(b.v)))

    def init_eq(self, rho: float = 1.0, u=(0.0, 0.0, 0.0), du=(0.0, 0.0, 0.0)):
        _lib().ort_init_eq(self._h, rho, _dp(_d3(u)), _dp(_d3(du)))

    def set_delta(self, d=None, dd=None):
        c = self.cfg
        n = c.nx * c.ny * c.nz
        d = np.zeros(n) if d is None else np.ascontiguousarray(d, dtype=np.float64).reshape(-1)
        dd = np.zeros(n) if dd is None else np.ascontiguousarray(dd, dtype=np.float64).reshape(-1)
        _lib().ort_set_delta(self._h, _dp(d), _dp(dd))

    def step(self, n: int = 1):
        _lib().ort_step(self._h, int(n))
        self.steps += n

    def force_torque(self):
        """(values, tangents), each [steps, nbodies, 6]."""
        m = self.steps * self.nbodies * 6
        v = np.zeros(max(m, 1))
        t = np.zeros(max(m, 1))
        _lib().ort_ft(self._h, _dp(v), _dp(t))
        shp = (self.steps, self.nbodies, 6)
        return v[:m].reshape(shp), t[:m].reshape(shp)

    def get_f(self):
        v = np.zeros(self.shape)
        t = np.zeros(self.shape)
        _lib().ort_get_f(self._h, _dp(v), _dp(t))
        return v, t


def tangent_gradient(cfg: Config, bodies, steps: int, rho0: float, u_in, weights=None, threads: int = 1):
    """FP64 gradient of J = sum_{n, b, k} w[n, b, k] FT[n, b, k] over `steps`
    steps from the equilibrium f^eq(rho0, u_in), as directional derivatives of
    the tangent-linear model, one run per direction (the definition of each
    partial derivative, no reverse sweep):
      grad_delta[z, y, x]: seed e_c on the per-cell perturbation delta of cell c,
      grad_omega[b, k]:    seed on component k of body b's angular velocity
                           (through u_s; the geometry sequence is frozen),
      grad_u_in[k]:        seed on component k of the inflow, in the ghost
                           planes and in the initial state.
    bodies: BodySpec list; weights [steps, nbodies, 6] (None: mean T_z of
    body 0).  Test infrastructure, like the rest of this package."""
    nb = len(bodies)
    if weights is None:
        weights = np.zeros((steps, nb, 6))
        weights[:, 0, 5] = 1.0 / steps
    weights = np.asarray(weights, dtype=np.float64).reshape(steps, nb, 6)

    def run(d_delta=None, d_omega=None, d_u=(0.0, 0.0, 0.0)):
        sim = TangentSim(cfg, d_u_in=d_u, threads=threads)
        for b, spec in enumerate(bodies):
            sim.add_body(spec, d_omega=(0.0, 0.0, 0.0) if d_omega is None or d_omega[0] != b else d_omega[1])
        sim.init_eq(rho0, u_in, du=d_u)
        if d_delta is not None:
            sim.set_delta(None, d_delta)
        sim.step(steps)
        v, t = sim.force_torque()
        return float((v * weights).sum()), float((t * weights).sum())

    n = cfg.nx * cfg.ny * cfg.nz
    J = run()[0]
    g_delta = np.zeros(n)
    e = np.zeros(n)
    for c in range(n):
        e[c] = 1.0
        g_delta[c] = run(d_delta=e)[1]
        e[c] = 0.0
    g_omega = np.zeros((nb, 3))
    for b in range(nb):
        for k in range(3):
            g_omega[b, k] = run(d_omega=(b, tuple(1.0 if j == k else 0.0 for j in range(3))))[1]
    g_u = np.array([run(d_u=tuple(1.0 if j == k else 0.0 for j in range(3)))[1] for k in range(3)])
    return J, g_delta.reshape(cfg.nz, cfg.ny, cfg.nx), g_omega, g_u
