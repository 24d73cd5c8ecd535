"""psm_mass_noalloc: the allocation-free mass reduction (its scratch is a static
device array), checked through the C ABI against psm_mass on the same state,
on two calls in a row.  This file is collected last so that a stopping run has
already run every other test; it also passes alone in a fresh process (the
first call on the device sets up the scratch address)."""

import ctypes

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__ as g

    g.build()
    from paper_2502_20049_gb300 import psm

    L = psm.lib()
    fn = L.psm_mass_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double)]
    return psm, fn


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_noalloc_mass_matches_psm_mass_twice(storage):
    import torch

    psm, fn = _lib()
    case = W.c2_ellipsoid(scale=0.25, n=64, steps=0, omega_z=0.01).with_(storage=storage)
    sol = psm.Solver.from_case(case)
    stream = torch.cuda.current_stream()
    for rnd in range(2):
        sol.step(7)
        ref = sol.mass()
        f = torch.empty(sol.shape, dtype=torch.float64, device="cuda")
        sol.get_state(out=f)  # natural layout, unshifted, FP64, device
        out = ctypes.c_double()
        rc = fn(ctypes.c_void_p(f.data_ptr()), psm.STORAGE["fp64"], 19, sol.ncell, 0.0,
                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
        assert rc == 0, psm.lib().psm_last_error()
        assert abs(out.value - ref) <= 1e-12 * abs(ref), (rnd, out.value, ref)
        # the same field stored shifted in FP32: the library's own storage format
        f32 = (f - torch.tensor(psm.lattice_velocities(19)[1], device="cuda").view(19, 1, 1, 1)).to(torch.float32)
        out32 = ctypes.c_double()
        rc = fn(ctypes.c_void_p(f32.data_ptr()), psm.STORAGE["fp32"], 19, sol.ncell, 1.0,
                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out32))
        assert rc == 0
        assert abs(out32.value - ref) <= 1e-6 * abs(ref)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    psm, fn = _lib()
    import torch

    f = torch.zeros(19, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    rc = fn(ctypes.c_void_p(f.data_ptr()), 0, 19, (1 << 30) + 1, 0.0, None, ctypes.byref(out))
    assert rc == -1
    assert b"2^30" in psm.lib().psm_last_error()
    rc = fn(ctypes.c_void_p(f.data_ptr()), 0, 19, 1, 0.0, None, ctypes.byref(out))
    assert rc == 0 and out.value == 0.0
