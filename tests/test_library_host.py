"""Host-side checks of libpsm that need no GPU: the shared library loads and
exports every function include/psm.h declares, the lattice tables agree with
the oracle's, the voxelisers agree with the oracle's bit for bit, and argument
validation fails with PSM_ERR_ARG before any CUDA call."""

import os
import re

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def psm():
    from paper_2502_20049_gb300 import build as B

    B.build()
    from paper_2502_20049_gb300 import psm as P

    return P


def declared_functions():
    src = open(os.path.join(ROOT, "include", "psm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(psm_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(psm):
    names = declared_functions()
    assert len(names) >= 20
    L = psm.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("Q", [19, 27])
def test_lattice_matches_oracle(psm, oracle_mod, Q):
    c, w, opp = psm.lattice_velocities(Q)
    co, wo, _ = oracle_mod.lattice(Q)
    assert {tuple(v) for v in c} == {tuple(v) for v in co}
    for i in range(Q):
        j = int(np.flatnonzero((co == c[i]).all(1))[0])
        assert w[i] == wo[j]
    assert np.array_equal(c[opp], -c)


CASES = [(W.SPHERE, (3.3,)), (W.ELLIPSOID, (4.5, 2.25, 1.7)), (W.BOX, (2.5, 1.5, 3.25)),
         (W.ROTOR, W.Rotor().scaled(0.08).params()),
         (W.ROTOR, W.Rotor(n_blades=5, phase=0.6283185307179586, hand=-1).scaled(0.08).params())]


@pytest.mark.parametrize("s", [0, 1, 2, 3])
@pytest.mark.parametrize("kind,params", CASES)
def test_voxeliser_matches_oracle(psm, oracle_mod, kind, params, s):
    g = psm.voxelize(kind, params, s)
    sub, lo = oracle_mod.voxelize(kind, params, s)
    assert np.array_equal(g.lo, lo)
    assert np.array_equal(g.subcells(), sub)
    assert sub.sum() > 0


def test_pack_roundtrip(psm, oracle_mod):
    """set_geometry_bits packs the oracle-style byte field into the documented brick layout."""
    for s in (0, 1, 2, 3):
        g = psm.voxelize(W.ELLIPSOID, (3.0, 2.0, 1.5), s)
        sub = g.subcells()
        n = 1 << s
        gx, gy, gz = g.dims
        b = sub.reshape(gz, n, gy, n, gx, n).transpose(0, 2, 4, 1, 3, 5).reshape(gz, gy, gx, n ** 3)
        wpb = 8 if s == 3 else 1
        padded = np.zeros((gz, gy, gx, wpb * 64), dtype=np.uint8)
        padded[..., : n ** 3] = b
        words = np.packbits(padded, axis=-1, bitorder="little").view(np.uint64).reshape(-1)
        assert np.array_equal(words, g.words())


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(tau=0.3), dict(u_in=(0.0, 0.0, 0.31)), dict(Q=15),
                                 dict(storage="fp8"), dict(nx=0), dict(rho0=0.0), dict(solid=4), dict(weighting=2),
                                 dict(fluid="trt", trt_lambda=0.0), dict(bc_z=3)])
def test_create_rejects_bad_arguments(psm, bad):
    kw = dict(nx=8, ny=8, nz=8)
    kw.update(bad)
    try:
        cfg = psm.SolverConfig(**kw)
        with pytest.raises(psm.PSMError) as ei:
            psm.Solver(cfg, stream=0)
        assert ei.value.code == -1
        assert psm.lib().psm_last_error()
    except KeyError:
        pass  # an unknown enum name never reaches the library


@pytest.mark.parametrize("bad,code", [(dict(fluid="cumulant", Q=27), -6), (dict(fluid="cumulant", cum_rates=(2.0, 1.0, 1.0)), -1),
                                      (dict(fluid="cumulant", cum_rates=(1.0, -0.5, 1.0)), -1),
                                      (dict(fluid="cumulant", cum_rates=(1.0, 1.0, float("nan"))), -1)])
def test_create_rejects_bad_cumulant(psm, bad, code):
    """The cumulant operator is D3Q19 only (PSM_ERR_UNSUPPORTED for D3Q27) and
    its rates lie in (0, 2) (0 selects 1); both fail before any CUDA call."""
    kw = dict(nx=8, ny=8, nz=8)
    kw.update(bad)
    with pytest.raises(psm.PSMError) as ei:
        psm.Solver(psm.SolverConfig(**kw), stream=0)
    assert ei.value.code == code


def test_voxeliser_rejects_bad_arguments(psm):
    with pytest.raises(psm.PSMError) as ei:
        psm.voxelize(W.SPHERE, (-1.0,), 2)
    assert ei.value.code == -1
    with pytest.raises(psm.PSMError):
        psm.voxelize(W.SPHERE, (2.0,), 4)


@pytest.mark.parametrize("bufs,flags", [([0, 0], 0), ([0x1008, 0x2000], 0), ([0x1000, 0x1000], 0),
                                        ([0x1000, 0x2000], 4)])
def test_create_with_buffers_rejects_bad_buffers(psm, bufs, flags):
    """NULL, misaligned or equal caller buffers and unknown flags fail before
    any CUDA call (the pointers are never dereferenced)."""
    import ctypes

    cfg = psm.SolverConfig(8, 8, 8, streaming="twogrid")
    grid = psm.Grid(cfg.nx, cfg.ny, cfg.nz, cfg.bc_z, cfg.rho0, (ctypes.c_double * 3)(*cfg.u_in))
    lat = psm.Lattice(cfg.Q, psm.STREAMING[cfg.streaming], psm.STORAGE[cfg.storage])
    col = psm.Collision(psm.FLUID[cfg.fluid], cfg.tau, cfg.trt_lambda, cfg.solid, cfg.weighting)
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 2)(*bufs)
    rc = psm.lib().psm_create_with_buffers(ctypes.byref(grid), ctypes.byref(lat), ctypes.byref(col), None, arr,
                                           flags, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_host_buffers_are_rejected_before_any_launch(psm):
    """Caller-owned memory that is host memory (a numpy array passed through
    ctypes) is refused with PSM_ERR_ARG by psm_check_device_buffer,
    psm_create_with_buffers and psm_mass_noalloc.  Without a GPU the pointer
    cannot be classified at all and the answer is the same; on a GPU the
    reason is that it is host memory.  Nothing is launched either way."""
    import ctypes

    a = np.zeros(19 * 8 * 8 * 8, dtype=np.float64)
    b = np.zeros_like(a)
    rc, msg = psm.check_device_buffer(a.ctypes.data, a.nbytes)
    assert rc == -1 and msg
    cfg = psm.SolverConfig(8, 8, 8, streaming="twogrid", storage="fp64")
    grid = psm.Grid(cfg.nx, cfg.ny, cfg.nz, cfg.bc_z, cfg.rho0, (ctypes.c_double * 3)(*cfg.u_in))
    lat = psm.Lattice(cfg.Q, psm.STREAMING[cfg.streaming], psm.STORAGE[cfg.storage])
    col = psm.Collision(psm.FLUID[cfg.fluid], cfg.tau, cfg.trt_lambda, cfg.solid, cfg.weighting)
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 2)(a.ctypes.data, b.ctypes.data)
    rc = psm.lib().psm_create_with_buffers(ctypes.byref(grid), ctypes.byref(lat), ctypes.byref(col), None, arr, 1,
                                           ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"PDF buffer 0" in psm.lib().psm_last_error()
    out = ctypes.c_double(7.0)
    rc = psm.lib().psm_mass_noalloc(ctypes.c_void_p(a.ctypes.data), psm.STORAGE["fp64"], 19, 512, 0.0, None,
                                    ctypes.byref(out))
    assert rc == -1 and out.value == 7.0
    assert b"psm_mass_noalloc: f" in psm.lib().psm_last_error()


def test_null_handle_calls_are_argument_errors(psm):
    import ctypes

    L = psm.lib()
    assert L.psm_set_remap(None, 0) == -1
    assert L.psm_get_pdfs(None, None) == -1
    assert L.psm_init_equilibrium_field(None, None, None) == -1
    assert L.psm_force_torque_raw(None, 0, 0, 0, None) == -1


@pytest.mark.parametrize("case", ["open", "index", "degenerate", "nan", "s"])
def test_mesh_voxeliser_rejects_bad_meshes(psm, case):
    """Argument errors of the mesh voxeliser are found on the host (no kernel runs)."""
    v, t = W.box_mesh((0, 0, 0), (2, 2, 2))
    s = 2
    if case == "open":
        t = t[:-1]
    elif case == "index":
        t = t.copy()
        t[0, 0] = 99
    elif case == "degenerate":
        t = t.copy()
        t[0, 1] = t[0, 0]
    elif case == "nan":
        v = v.copy()
        v[0, 0] = np.nan
    else:
        s = 4
    with pytest.raises(psm.PSMError) as ei:
        psm.voxelize_mesh(v, t, s)
    assert ei.value.code == -1


def test_tma_stage_budget(psm):
    """The TMA step kernel's stages fit the shared memory of the resident blocks
    it is sized for (228 KB per SM, 1 KB reserved and 6 KB of static shared
    memory per block; at most 227 KB per block), for every storage, stencil,
    streaming step and fluid operator; two cells per thread exactly for the
    D3Q19 two-grid and the D3Q19/D3Q27 AA even BGK/TRT steps in 2-byte storage.
    Host only."""
    for storage in ("fp64", "fp32", "fp16", "bf16"):
        for Q in (19, 27):
            for mode in (0, 1, 2):
                for fluid in ("bgk", "trt", "cumulant"):
                    if fluid == "cumulant" and Q == 27:
                        with pytest.raises(psm.PSMError) as ei:
                            psm.tma_layout(storage, Q, mode, fluid)
                        assert ei.value.code == -6
                        continue
                    L = psm.tma_layout(storage, Q, mode, fluid)
                    key = (storage, Q, mode, fluid, L)
                    assert 2 <= L["stages"] <= 8, key
                    assert L["smem"] <= 227 * 1024, key
                    assert L["blocks_per_sm"] * (L["smem"] + 1024 + 6144) <= 228 * 1024, key
                    two = (storage in ("fp16", "bf16") and fluid != "cumulant"
                           and ((mode == 0 and Q == 19) or mode == 1))
                    assert L["cells_per_thread"] == (2 if two else 1), key
    with pytest.raises(psm.PSMError):
        psm.tma_layout("fp32", 15, 0, "bgk")


@pytest.mark.parametrize("compiler,flags", [("gcc", ["-x", "c", "-std=c99"]), ("g++", ["-x", "c++", "-std=c++17"])])
def test_header_is_plain_c(tmp_path, compiler, flags):
    """include/psm.h compiles as strict C99 (and as C++): plain types, no C++ in the
    ABI.  A translation unit fills the structs and takes the address of every
    declared function (compile only, no GPU)."""
    import shutil
    import subprocess

    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not available")
    names = declared_functions()
    src = ['#include "psm.h"', "typedef void (*fnp)(void);",
           "static const fnp table[] = {" + ", ".join(f"(fnp){n}" for n in names) + "};",
           "int psm_header_check(void) {",
           "  psm_grid g = {64, 64, 64, PSM_BC_EQ_INLET_OUTLET, 1.0, {0.0, 0.0, 0.05}};",
           "  psm_lattice l = {PSM_D3Q19, PSM_STREAM_AA, PSM_FP16_SHIFTED};",
           "  psm_collision c = {PSM_CUMULANT, 0.6, 0.1875, PSM_SC1, PSM_B_TAU_WEIGHTED, {1.0, 1.0, 1.0}};",
           "  psm_handle h = 0;",
           "  (void)g; (void)l; (void)c; (void)h;",
           "  return (int)(sizeof table / sizeof table[0]);",
           "}"]
    f = tmp_path / "check.c"
    f.write_text("\n".join(src) + "\n")
    out = subprocess.run([compiler] + flags + ["-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                                               os.path.join(ROOT, "include"), "-c", str(f), "-o",
                                               str(tmp_path / "check.o")], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr


def test_binding_checks_output_buffers(psm):
    """The binding refuses torch outputs of the wrong dtype, shape or layout
    before it hands a pointer to the library."""
    import torch

    with pytest.raises(ValueError):
        psm._ptr(torch.zeros(8, dtype=torch.float32), np.float64, 8)
    with pytest.raises(ValueError):
        psm._ptr(torch.zeros(7, dtype=torch.float64), np.float64, 8)
    with pytest.raises(ValueError):
        psm._ptr(torch.zeros(4, 4, dtype=torch.float64).t(), np.float64, 16)
    with pytest.raises(ValueError):
        psm._ptr(np.zeros(8, dtype=np.float32), np.float64, 8)
    p, keep = psm._ptr(torch.zeros(8, dtype=torch.float64), np.float64, 8)
    assert p.value == keep.data_ptr()
