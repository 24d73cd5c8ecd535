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


@pytest.mark.parametrize("Q", [19, 27])
def test_noalloc_half_precision_and_d3q27(Q):
    """The FP16- and BF16-shifted instantiations (and D3Q27): the state of a
    solver, stored shifted in the 2-byte format with rho0 = 1, summed by
    psm_mass_noalloc equals the FP64 sum of those same 2-byte values (1e-12
    relative: only the order differs) and psm_mass within the formats'
    rounding (half an ulp of each stored value), on two calls in a row."""
    import torch

    psm, fn = _lib()
    if Q == 19:
        case = W.c2_ellipsoid(scale=0.25, n=64, steps=0, omega_z=0.01).with_(storage="fp32")
    else:
        case = W.c3_rotor("fp32", scale=0.125, dims=(64, 64, 80), steps=0)
    sol = psm.Solver.from_case(case)
    stream = torch.cuda.current_stream()
    w = torch.tensor(psm.lattice_velocities(Q)[1], device="cuda").view(Q, 1, 1, 1)
    for rnd in range(2):
        sol.step(5)
        ref = sol.mass()
        f = torch.empty(sol.shape, dtype=torch.float64, device="cuda")
        sol.get_state(out=f)
        for storage, dt, ulp in (("fp16", torch.float16, 2.0 ** -10), ("bf16", torch.bfloat16, 2.0 ** -7)):
            g = (f - w).to(dt)
            exact = float(g.double().sum()) + float(sol.ncell)
            bound = 0.5 * ulp * float((f - w).abs().sum()) * 2.0
            out = ctypes.c_double()
            rc = fn(ctypes.c_void_p(g.data_ptr()), psm.STORAGE[storage], Q, sol.ncell, 1.0,
                    ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
            assert rc == 0, psm.lib().psm_last_error()
            assert abs(out.value - exact) <= 1e-12 * abs(exact), (storage, rnd, out.value, exact)
            assert abs(out.value - ref) <= bound, (storage, rnd, out.value, ref, bound)


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
