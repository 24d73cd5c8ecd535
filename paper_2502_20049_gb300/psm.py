"""Python binding of libpsm (include/psm.h): argument marshalling only.

Every step of the PSM path runs in the CUDA library; this module converts
Python / numpy / torch arguments to the C ABI and back.  It raises
:class:`PSMError` for a non-zero status.  If ``libpsm.so`` has not been built,
loading fails loudly: there is no CPU fallback.

PyTorch supplies the CUDA stream (``torch.cuda.current_stream()``) and, where a
caller passes a torch CUDA tensor as an output, the device memory it is written
to.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpsm.so")
_LOCK = threading.Lock()
_LIB = None

PSM_OK = 0
ERRORS = {-1: "PSM_ERR_ARG", -2: "PSM_ERR_CUDA", -3: "PSM_ERR_OOM", -4: "PSM_ERR_NONFINITE", -5: "PSM_ERR_STATE",
          -6: "PSM_ERR_UNSUPPORTED"}
PSM_MAX_BODIES = 4
STORAGE = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
STREAMING = {"aa": 0, "twogrid": 1}
FLUID = {"bgk": 0, "trt": 1, "cumulant": 2}
STORAGE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}


class PSMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("bc_z", ctypes.c_int),
                ("rho0", ctypes.c_double), ("u_in", ctypes.c_double * 3)]


class Lattice(ctypes.Structure):
    _fields_ = [("stencil", ctypes.c_int), ("streaming", ctypes.c_int), ("storage", ctypes.c_int)]


class Collision(ctypes.Structure):
    _fields_ = [("fluid", ctypes.c_int), ("tau", ctypes.c_double), ("trt_lambda", ctypes.c_double),
                ("solid", ctypes.c_int), ("weighting", ctypes.c_int), ("cum_omega", ctypes.c_double * 3)]


class GeomField(ctypes.Structure):
    _fields_ = [("bricks", ctypes.POINTER(ctypes.c_uint64)), ("gx", ctypes.c_int64), ("gy", ctypes.c_int64),
                ("gz", ctypes.c_int64), ("s", ctypes.c_int), ("lo", ctypes.c_double * 3)]


class RotorParams(ctypes.Structure):
    _fields_ = [("r_hub", ctypes.c_double), ("hub_len", ctypes.c_double), ("span", ctypes.c_double),
                ("chord", ctypes.c_double), ("thickness", ctypes.c_double), ("pitch_root_deg", ctypes.c_double),
                ("twist_deg", ctypes.c_double), ("phase", ctypes.c_double), ("n_blades", ctypes.c_int),
                ("hand", ctypes.c_int)]


class BodyDynamics(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("inertia", ctypes.c_double * 9), ("force_ext", ctypes.c_double * 3),
                ("torque_ext", ctypes.c_double * 3)]


def lib() -> ctypes.CDLL:
    """Load libpsm.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                                  f"g.build()'` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            i, d, vp, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
            H = vp
            sig = {
                "psm_last_error": (ctypes.c_char_p, []),
                "psm_lattice_velocities": (i, [i, P(i), P(d), P(i)]),
                "psm_geom_voxelize_sphere": (i, [d, i, P(GeomField)]),
                "psm_geom_voxelize_ellipsoid": (i, [d, d, d, i, P(GeomField)]),
                "psm_geom_voxelize_box": (i, [d, d, d, i, P(GeomField)]),
                "psm_geom_voxelize_rotor": (i, [P(RotorParams), i, P(GeomField)]),
                "psm_geom_free": (i, [P(GeomField)]),
                "psm_geom_voxelize_mesh": (i, [vp, i64, vp, i64, i, P(GeomField)]),
                "psm_create": (i, [P(Grid), P(Lattice), P(Collision), vp, P(H)]),
                "psm_create_with_buffers": (i, [P(Grid), P(Lattice), P(Collision), vp, P(vp), i, P(H)]),
                "psm_init_equilibrium_field": (i, [H, vp, vp]),
                "psm_get_pdfs": (i, [H, vp]),
                "psm_force_torque_raw": (i, [H, i, i64, i64, vp]),
                "psm_set_remap": (i, [H, i]),
                "psm_set_body_dynamics": (i, [H, i, P(BodyDynamics)]),
                "psm_body_state": (i, [H, i, vp]),
                "psm_destroy": (i, [H]),
                "psm_init_equilibrium": (i, [H, d, P(d)]),
                "psm_set_state": (i, [H, vp]),
                "psm_get_state": (i, [H, vp]),
                "psm_get_macroscopic": (i, [H, vp, vp]),
                "psm_get_cells": (i, [H, vp, i64, vp]),
                "psm_get_eps": (i, [H, vp]),
                "psm_set_geometry": (i, [H, i, P(GeomField), P(d), P(d), P(d), P(d)]),
                "psm_num_bodies": (i, [H, P(i)]),
                "psm_step": (i, [H, i]),
                "psm_step_count": (i, [H, P(i64)]),
                "psm_force_torque": (i, [H, i, i64, i64, vp]),
                "psm_series_capacity": (i, [H, P(i64)]),
                "psm_mass": (i, [H, P(d)]),
                "psm_synchronize": (i, [H]),
                "psm_set_kernel_variant": (i, [H, i]),
                "psm_set_eps_delta": (i, [H, vp]),
                "psm_record": (i, [H, i, i]),
                "psm_backward": (i, [H, vp, vp, vp, vp]),
                "psm_kernel_variant": (i, [H, P(i)]),
                "psm_tma_layout": (i, [i, i, i, i, P(i)]),
                "psm_check_device_buffer": (i, [vp, i64]),
                "psm_set_z_offset": (i, [H, i64]),
                "psm_set_us_omega": (i, [H, i, P(d)]),
                "psm_slot_plane": (i, [H, i, i, P(vp)]),
                "psm_fill_slot_plane": (i, [H, i, i, i]),
                "psm_mass_noalloc": (i, [vp, i, i, i64, d, vp, P(d)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def check_device_buffer(ptr: int, nbytes: int) -> tuple[int, str]:
    """psm_check_device_buffer: (status, message) for a raw pointer and a size
    in bytes (status 0 = device memory of the current device, large enough)."""
    rc = lib().psm_check_device_buffer(ctypes.c_void_p(ptr), int(nbytes))
    return rc, (lib().psm_last_error() or b"").decode() if rc else ""


def check(rc: int):
    if rc != PSM_OK:
        msg = lib().psm_last_error()
        raise PSMError(rc, msg.decode() if msg else "")


def _d(arr, n):
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr(out, dtype, count):
    """(pointer, keepalive) for an output/input array: numpy host array or torch tensor."""
    if hasattr(out, "data_ptr"):  # torch tensor, host or device
        if out.numel() != count:
            raise ValueError(f"expected {count} elements, got {out.numel()}")
        if str(out.dtype).replace("torch.", "") != np.dtype(dtype).name or not out.is_contiguous():
            raise ValueError(f"expected a contiguous {np.dtype(dtype).name} tensor, got {out.dtype}")
        return ctypes.c_void_p(out.data_ptr()), out
    if not isinstance(out, np.ndarray) or out.dtype != dtype or out.size != count or not out.flags.c_contiguous:
        raise ValueError(f"expected a C-contiguous {dtype} array of {count} elements")
    return ctypes.c_void_p(out.ctypes.data), out


def current_stream() -> int:
    """cudaStream_t of torch's current stream (0 when torch has no CUDA)."""
    try:
        import torch

        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def lattice_velocities(Q: int):
    """(c[Q,3], w[Q], opp[Q]) in the library's direction order."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    check(lib().psm_lattice_velocities(Q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return c.astype(np.int64), w, opp.astype(np.int64)


def tma_layout(storage: str, Q: int, mode: int, fluid: str = "bgk") -> dict:
    """Shared-memory layout of the TMA-staged step kernel (psm_tma_layout; host
    only): mode 0 two-grid, 1 AA even, 2 AA odd."""
    out = (ctypes.c_int * 4)()
    check(lib().psm_tma_layout(STORAGE[storage], Q, mode, FLUID[fluid], out))
    return dict(smem=out[0], stages=out[1], blocks_per_sm=out[2], cells_per_thread=out[3])


class Geometry:
    """A host geometry field returned by a library voxeliser (freed on delete)."""

    def __init__(self):
        self.field = GeomField()

    def __del__(self):
        if getattr(self, "field", None) is not None and self.field.bricks:
            lib().psm_geom_free(ctypes.byref(self.field))

    @property
    def dims(self):
        return (self.field.gx, self.field.gy, self.field.gz)

    @property
    def s(self) -> int:
        return self.field.s

    @property
    def lo(self):
        return np.array(self.field.lo[:])

    def words(self) -> np.ndarray:
        wpb = 8 if self.field.s == 3 else 1
        n = self.field.gx * self.field.gy * self.field.gz * wpb
        return np.ctypeslib.as_array(self.field.bricks, shape=(n,)).copy()

    def subcells(self) -> np.ndarray:
        """Unpack to one byte per sub-cell, [gz*n, gy*n, gx*n] (x fastest)."""
        s = self.field.s
        n = 1 << s
        gx, gy, gz = self.dims
        wpb = 8 if s == 3 else 1
        words = self.words().reshape(gz, gy, gx, wpb)
        bits = np.unpackbits(words.view(np.uint8).reshape(gz, gy, gx, wpb * 8), axis=-1, bitorder="little")
        bits = bits[..., : n * n * n].reshape(gz, gy, gx, n, n, n)  # [.., sz, sy, sx]
        return np.ascontiguousarray(bits.transpose(0, 3, 1, 4, 2, 5).reshape(gz * n, gy * n, gx * n))


def voxelize(kind: int, params, s: int) -> Geometry:
    """Library voxeliser for an analytic shape kind of :mod:`workloads`."""
    g = Geometry()
    p = list(params)
    if kind == W.SPHERE:
        rc = lib().psm_geom_voxelize_sphere(p[0], s, ctypes.byref(g.field))
    elif kind == W.ELLIPSOID:
        rc = lib().psm_geom_voxelize_ellipsoid(p[0], p[1], p[2], s, ctypes.byref(g.field))
    elif kind == W.BOX:
        rc = lib().psm_geom_voxelize_box(p[0], p[1], p[2], s, ctypes.byref(g.field))
    elif kind == W.ROTOR:
        r = RotorParams(p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], int(p[8]), int(p[9]))
        rc = lib().psm_geom_voxelize_rotor(ctypes.byref(r), s, ctypes.byref(g.field))
    else:
        raise ValueError(f"unknown shape kind {kind}")
    check(rc)
    return g


def voxelize_mesh(vertices, triangles, s: int) -> Geometry:
    """GPU voxeliser of a closed triangle mesh (psm_geom_voxelize_mesh):
    vertices [nv, 3] float32, triangles [nt, 3] int32 (numpy, or torch tensors
    on the host or the device)."""
    g = Geometry()
    if hasattr(vertices, "data_ptr"):
        vp, nv = ctypes.c_void_p(vertices.data_ptr()), vertices.shape[0]
    else:
        vertices = np.ascontiguousarray(vertices, dtype=np.float32)
        vp, nv = ctypes.c_void_p(vertices.ctypes.data), len(vertices)
    if hasattr(triangles, "data_ptr"):
        tp, nt = ctypes.c_void_p(triangles.data_ptr()), triangles.shape[0]
    else:
        triangles = np.ascontiguousarray(triangles, dtype=np.int32)
        tp, nt = ctypes.c_void_p(triangles.ctypes.data), len(triangles)
    check(lib().psm_geom_voxelize_mesh(vp, nv, tp, nt, s, ctypes.byref(g.field)))
    return g


@dataclass
class SolverConfig:
    nx: int
    ny: int
    nz: int
    Q: int = 19
    streaming: str = "aa"
    storage: str = "fp32"
    fluid: str = "bgk"
    tau: float = 0.8
    trt_lambda: float = 3.0 / 16.0
    solid: int = 1
    weighting: int = 1
    bc_z: int = 1
    cum_rates: tuple = (1.0, 1.0, 1.0)  # cumulant: bulk, third-order, fourth-order rates
    rho0: float = 1.0
    u_in: tuple = (0.0, 0.0, 0.0)


class Solver:
    """One libpsm handle (psm_create ... psm_destroy)."""

    def __init__(self, cfg: SolverConfig, stream: int | None = None, buffers=None, keep: bool = False):
        """buffers: caller-owned device PDF buffers (torch tensors or raw
        pointers; one for AA, two for two-grid), kept alive by the solver and
        never freed by it (psm_create_with_buffers); keep: their contents are
        the initial state."""
        self.cfg = cfg
        grid = Grid(cfg.nx, cfg.ny, cfg.nz, cfg.bc_z, cfg.rho0, (ctypes.c_double * 3)(*cfg.u_in))
        lat = Lattice(cfg.Q, STREAMING[cfg.streaming], STORAGE[cfg.storage])
        col = Collision(FLUID[cfg.fluid], cfg.tau, cfg.trt_lambda, cfg.solid, cfg.weighting,
                        (ctypes.c_double * 3)(*cfg.cum_rates))
        self._h = ctypes.c_void_p()
        self.stream = current_stream() if stream is None else stream
        self._buffers = buffers
        if buffers is None:
            check(lib().psm_create(ctypes.byref(grid), ctypes.byref(lat), ctypes.byref(col),
                                   ctypes.c_void_p(self.stream), ctypes.byref(self._h)))
        else:
            ptrs = [b.data_ptr() if hasattr(b, "data_ptr") else int(b) for b in buffers]
            arr = (ctypes.c_void_p * 2)(*(ptrs + [0] * (2 - len(ptrs))))
            check(lib().psm_create_with_buffers(ctypes.byref(grid), ctypes.byref(lat), ctypes.byref(col),
                                                ctypes.c_void_p(self.stream), arr, 1 if keep else 0,
                                                ctypes.byref(self._h)))
        self._geoms = []

    @classmethod
    def from_case(cls, case: "W.Case", stream: int | None = None, init: bool = True,
                  geoms: dict | None = None) -> "Solver":
        """A solver for a workload case.  geoms: a dict that caches the
        voxelised fields by (kind, params, s) across solvers (the field is
        copied to the device by psm_set_geometry, so one host field serves
        any number of handles)."""
        cfg = SolverConfig(case.nx, case.ny, case.nz, Q=case.Q, streaming=case.streaming, storage=case.storage,
                           fluid=case.fluid, tau=case.tau, trt_lambda=case.trt_lambda, solid=case.solid,
                           weighting=case.weighting, bc_z=case.bc_z, rho0=case.rho0, u_in=tuple(case.u_in),
                           cum_rates=tuple(case.cum_rates))
        s = cls(cfg, stream=stream)
        for bi, b in enumerate(case.bodies):
            key = (b.kind, tuple(b.params), b.s)
            if geoms is not None and key in geoms:
                g = geoms[key]
            else:
                g = voxelize(b.kind, b.params, b.s)
                if geoms is not None:
                    geoms[key] = g
            s.set_geometry(bi, g, b.Q0, b.R0, b.omega, b.v)
        if init:
            s.init_equilibrium(case.rho0, case.u_in)
        return s

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        self.close()

    @property
    def shape(self):
        c = self.cfg
        return (c.Q, c.nz, c.ny, c.nx)

    @property
    def ncell(self) -> int:
        c = self.cfg
        return c.nx * c.ny * c.nz

    def init_equilibrium(self, rho: float, u):
        _, up = _d(u, 3)
        check(lib().psm_init_equilibrium(self._h, rho, up))

    def init_equilibrium_field(self, rho, u):
        """f = f^eq(rho(x), u(x)) per cell: rho [nz, ny, nx], u [nz, ny, nx, 3]
        (numpy or torch, host or device, float64)."""
        if not hasattr(rho, "data_ptr"):
            rho = np.ascontiguousarray(rho, dtype=np.float64)
        if not hasattr(u, "data_ptr"):
            u = np.ascontiguousarray(u, dtype=np.float64)
        rp, k1 = _ptr(rho, np.float64, self.ncell)
        up, k2 = _ptr(u, np.float64, 3 * self.ncell)
        check(lib().psm_init_equilibrium_field(self._h, rp, up))

    def set_body_dynamics(self, body: int, mass: float, inertia, force_ext=(0.0, 0.0, 0.0),
                          torque_ext=(0.0, 0.0, 0.0)):
        """Two-way coupling of a body from the current step (psm_set_body_dynamics)."""
        d = BodyDynamics(float(mass), (ctypes.c_double * 9)(*np.asarray(inertia, dtype=float).reshape(9)),
                         (ctypes.c_double * 3)(*force_ext), (ctypes.c_double * 3)(*torque_ext))
        check(lib().psm_set_body_dynamics(self._h, body, ctypes.byref(d)))

    def body_state(self, body: int = 0):
        """dict R, v, Q (3x3), omega, L of a body for the next step."""
        out = np.zeros(21)
        check(lib().psm_body_state(self._h, body, ctypes.c_void_p(out.ctypes.data)))
        return dict(R=out[0:3], v=out[3:6], Q=out[6:15].reshape(3, 3), omega=out[15:18], L=out[18:21])

    def set_remap(self, every_step: bool):
        """Remap the geometry every step (True) or freeze the poses now (False)."""
        check(lib().psm_set_remap(self._h, 1 if every_step else 0))

    STORAGE_DTYPES = {"fp64": np.float64, "fp32": np.float32, "fp16": np.float16, "bf16": np.uint16}

    def get_pdfs(self, out=None):
        """Stored PDFs (shifted, natural layout) in the storage precision:
        [Q, nz, ny, nx] numpy array (BF16 as its raw 16-bit patterns) unless
        out (numpy or torch, host or device) is given."""
        dt = self.STORAGE_DTYPES[self.cfg.storage]
        if out is None:
            out = np.zeros(self.shape, dtype=dt)
        n = int(np.prod(self.shape))
        if hasattr(out, "data_ptr"):
            if out.numel() * out.element_size() != n * np.dtype(dt).itemsize:
                raise ValueError("output buffer has the wrong size")
            p = ctypes.c_void_p(out.data_ptr())
        else:
            p, keep = _ptr(out, dt, n)
        check(lib().psm_get_pdfs(self._h, p))
        return out

    def set_geometry(self, body: int, geom: Geometry, Q0, R0, omega, v):
        a, Qp = _d(Q0, 9)
        b, Rp = _d(R0, 3)
        c, wp = _d(omega, 3)
        e, vp = _d(v, 3)
        check(lib().psm_set_geometry(self._h, body, ctypes.byref(geom.field), Qp, Rp, wp, vp))
        self._geoms.append(geom)

    def set_geometry_bits(self, body: int, sub: np.ndarray, s: int, lo, Q0, R0, omega, v):
        """Attach a field given as one byte per sub-cell [nsz, nsy, nsx] (packed here)."""
        n = 1 << s
        nsz, nsy, nsx = sub.shape
        gx, gy, gz = nsx // n, nsy // n, nsz // n
        b = sub.reshape(gz, n, gy, n, gx, n).transpose(0, 2, 4, 1, 3, 5).reshape(gz, gy, gx, n * n * n)
        wpb = 8 if s == 3 else 1
        padded = np.zeros((gz, gy, gx, wpb * 64), dtype=np.uint8)
        padded[..., : n * n * n] = b
        words = np.packbits(padded, axis=-1, bitorder="little").view(np.uint64).reshape(-1).copy()
        g = Geometry()
        g._words = words
        g.field.bricks = words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        g.field.gx, g.field.gy, g.field.gz, g.field.s = gx, gy, gz, s
        for k in range(3):
            g.field.lo[k] = float(lo[k])
        try:
            self.set_geometry(body, g, Q0, R0, omega, v)
        finally:
            g.field.bricks = ctypes.POINTER(ctypes.c_uint64)()  # numpy owns the words
        self._geoms.pop()

    def set_us_omega(self, body: int, omega):
        """Angular velocity of body's u_s (the pose keeps its own; psm_set_us_omega)."""
        a, p = _d(omega, 3)
        check(lib().psm_set_us_omega(self._h, int(body), p))

    @property
    def num_bodies(self) -> int:
        n = ctypes.c_int()
        check(lib().psm_num_bodies(self._h, ctypes.byref(n)))
        return n.value

    def step(self, n: int = 1):
        check(lib().psm_step(self._h, int(n)))

    @property
    def step_count(self) -> int:
        n = ctypes.c_int64()
        check(lib().psm_step_count(self._h, ctypes.byref(n)))
        return n.value

    def force_torque(self, body: int = 0, step_from: int = 0, count: int | None = None, out=None):
        """[count, 6] force and torque on the body (FP64, host unless out is given)."""
        if count is None:
            count = self.step_count - step_from
        if out is None:
            out = np.zeros((count, 6))
        p, keep = _ptr(out, np.float64, count * 6)
        check(lib().psm_force_torque(self._h, body, step_from, count, p))
        return out

    def force_torque_raw(self, body: int = 0, step_from: int = 0, count: int | None = None):
        """[count, 6] with the printed sign of Eq. 10 / 11 (minus force_torque)."""
        if count is None:
            count = self.step_count - step_from
        out = np.zeros((count, 6))
        check(lib().psm_force_torque_raw(self._h, body, step_from, count, ctypes.c_void_p(out.ctypes.data)))
        return out

    def mass(self) -> float:
        m = ctypes.c_double()
        check(lib().psm_mass(self._h, ctypes.byref(m)))
        return m.value

    def get_state(self, out=None):
        if out is None:
            out = np.zeros(self.shape)
        p, keep = _ptr(out, np.float64, int(np.prod(self.shape)))
        check(lib().psm_get_state(self._h, p))
        return out

    def set_state(self, f):
        if hasattr(f, "data_ptr"):
            p, keep = _ptr(f, np.float64, int(np.prod(self.shape)))
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
            p, keep = _ptr(f, np.float64, int(np.prod(self.shape)))
        check(lib().psm_set_state(self._h, p))

    def get_cells(self, cells):
        """[len(cells), Q] natural FP64 PDFs of flat cell indices (library order)."""
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
        out = np.zeros((cells.size, self.cfg.Q))
        check(lib().psm_get_cells(self._h, ctypes.c_void_p(cells.ctypes.data), cells.size,
                                  ctypes.c_void_p(out.ctypes.data)))
        return out

    def macroscopic(self, rho=None, u=None):
        """(rho[nz, ny, nx], u[nz, ny, nx, 3]) in FP64, into new numpy arrays or
        the given ones (numpy or torch, host or device)."""
        c = self.cfg
        rho = np.zeros((c.nz, c.ny, c.nx)) if rho is None else rho
        u = np.zeros((c.nz, c.ny, c.nx, 3)) if u is None else u
        pr, kr = _ptr(rho, np.float64, self.ncell)
        pu, ku = _ptr(u, np.float64, 3 * self.ncell)
        check(lib().psm_get_macroscopic(self._h, pr, pu))
        return rho, u

    def eps(self):
        c = self.cfg
        e = np.zeros((c.nz, c.ny, c.nx), dtype=np.float32)
        check(lib().psm_get_eps(self._h, ctypes.c_void_p(e.ctypes.data)))
        return e

    def synchronize(self):
        check(lib().psm_synchronize(self._h))

    def set_eps_delta(self, delta):
        """Per-cell additive eps perturbation (float32 [nz, ny, nx], numpy or torch); None removes it."""
        if delta is None:
            check(lib().psm_set_eps_delta(self._h, None))
            return
        if hasattr(delta, "data_ptr"):
            d = delta.detach().to(dtype=__import__("torch").float32).contiguous()
            p, keep = _ptr(d, np.float32, self.ncell)
        else:
            d = np.ascontiguousarray(delta, dtype=np.float32)
            p, keep = _ptr(d, np.float32, self.ncell)
        check(lib().psm_set_eps_delta(self._h, p))

    def record(self, K: int, init_from_inflow: bool = False, sequential: bool = False):
        """Checkpoint the trajectory every K steps from now on (K = 0 stops);
        sequential: one set of recompute buffers (psm_backward recomputes and
        sweeps each segment in turn)."""
        flags = (1 if init_from_inflow else 0) | (2 if sequential else 0)
        check(lib().psm_record(self._h, int(K), flags))

    def backward(self, dJ_dFT=None, grad_eps=None):
        """Adjoint gradients of J = sum w * FT over the recorded steps.

        Returns (grad_eps [nz, ny, nx] (or the given buffer), grad_omega
        [nbodies, 3], grad_uin [3]).  dJ_dFT None = mean torque about z on body 0.
        """
        c = self.cfg
        nb = self.num_bodies
        w = None
        if dJ_dFT is not None:
            w = np.ascontiguousarray(dJ_dFT, dtype=np.float64)
        if grad_eps is None:
            grad_eps = np.zeros((c.nz, c.ny, c.nx))
        gp, keep = _ptr(grad_eps, np.float64, self.ncell)
        gw = np.zeros((max(nb, 1), 3))
        gu = np.zeros(3)
        check(lib().psm_backward(self._h, None if w is None else ctypes.c_void_p(w.ctypes.data), gp,
                                 ctypes.c_void_p(gw.ctypes.data), ctypes.c_void_p(gu.ctypes.data)))
        return grad_eps, gw[:nb], gu

    KERNELS = {"auto": 0, "plain": 1, "tma": 2}

    @property
    def kernel_variant(self) -> str:
        """'plain' or 'tma': the step kernel psm_step uses."""
        v = ctypes.c_int()
        check(lib().psm_kernel_variant(self._h, ctypes.byref(v)))
        return {1: "plain", 2: "tma"}[v.value]

    def set_kernel_variant(self, name: str):
        check(lib().psm_set_kernel_variant(self._h, self.KERNELS[name]))

    def bytes_per_cell_update(self) -> int:
        """Algorithmic bytes per cell update: one read and one write of every PDF."""
        return 2 * self.cfg.Q * STORAGE_BYTES[self.cfg.storage]

    # ---- z-slab decomposition (psm_set_z_offset, psm_slot_plane, psm_fill_slot_plane) ----

    def set_z_offset(self, z0: int):
        """This handle's lattice is the planes [z0, z0 + nz) of a larger domain."""
        check(lib().psm_set_z_offset(self._h, int(z0)))

    def slot_plane_ptr(self, slot: int, z: int) -> int:
        """Device address of slot `slot` of plane z in the buffer the next step reads."""
        p = ctypes.c_void_p()
        check(lib().psm_slot_plane(self._h, int(slot), int(z), ctypes.byref(p)))
        return p.value

    def slot_plane(self, slot: int, z: int):
        """A torch view [ny, nx] of slot `slot` of plane z (no copy; valid until the next step)."""
        import torch

        c = self.cfg
        typestr = {"fp64": "<f8", "fp32": "<f4", "fp16": "<f2", "bf16": "<f2"}[c.storage]

        class _View:
            __cuda_array_interface__ = {"shape": (c.ny, c.nx), "typestr": typestr,
                                        "data": (self.slot_plane_ptr(slot, z), False), "version": 3}

        t = torch.as_tensor(_View(), device="cuda")
        return t.view(torch.bfloat16) if c.storage == "bf16" else t

    def fill_slot_plane(self, slot: int, z: int, direction: int | None = None):
        """Set slot `slot` of plane z to the inflow equilibrium of `direction`
        (default: the slot's own; stream-ordered)."""
        d = slot if direction is None else direction
        check(lib().psm_fill_slot_plane(self._h, int(slot), int(z), int(d)))
