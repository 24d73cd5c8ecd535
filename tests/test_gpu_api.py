"""GPU checks of the ABI's state and geometry controls: caller-owned PDF
buffers, PDFs in the storage precision, equilibrium initialisation from
per-cell fields, the remap switch and the printed-sign force/torque."""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()


def small(storage="fp32", streaming="twogrid", omega=(0.0, 0.0, 0.02), v=(0.0, 0.0, 0.0), bc_z=1):
    return W.Case("api", 32, 16, 24, Q=19, storage=storage, streaming=streaming, fluid="trt", tau=0.6, bc_z=bc_z,
                  u_in=(0.0, 0.01, 0.03), steps=9,
                  bodies=[W.BodyCase(W.ELLIPSOID, (6.0, 3.0, 2.5), 2, (16.0, 8.0, 12.0), omega=omega, v=v)])


def cfg_of(case):
    from paper_2502_20049_gb300 import psm

    return psm.SolverConfig(case.nx, case.ny, case.nz, Q=case.Q, streaming=case.streaming, storage=case.storage,
                            fluid=case.fluid, tau=case.tau, trt_lambda=case.trt_lambda, solid=case.solid,
                            weighting=case.weighting, bc_z=case.bc_z, rho0=case.rho0, u_in=tuple(case.u_in))


def with_bodies(sol, case):
    from paper_2502_20049_gb300 import psm

    for bi, b in enumerate(case.bodies):
        sol.set_geometry(bi, psm.voxelize(b.kind, b.params, b.s), b.Q0, b.R0, b.omega, b.v)
    return sol


TORCH_DT = {"fp64": "float64", "fp32": "float32", "fp16": "float16", "bf16": "bfloat16"}


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("streaming", ["twogrid", "aa"])
def test_caller_owned_buffers_match_library_buffers(storage, streaming):
    import torch

    from paper_2502_20049_gb300 import psm

    case = small(storage, streaming)
    ref = psm.Solver.from_case(case)
    nbuf = 2 if streaming == "twogrid" else 1
    bufs = [torch.zeros((case.Q, case.nz, case.ny, case.nx), dtype=getattr(torch, TORCH_DT[storage]), device="cuda")
            for _ in range(nbuf)]
    mine = with_bodies(psm.Solver(cfg_of(case), buffers=bufs), case)
    assert float(bufs[0].float().abs().sum()) > 0  # initialised to f^eq in the caller's memory
    ref.step(case.steps)
    mine.step(case.steps)
    assert np.array_equal(ref.get_state(), mine.get_state())
    assert np.array_equal(ref.force_torque(0), mine.force_torque(0))
    mine.close()
    assert torch.isfinite(bufs[0].float()).all()  # still the caller's, not freed


@pytest.mark.parametrize("streaming", ["twogrid", "aa"])
def test_caller_buffers_keep_continue_a_run(streaming):
    """A state exported with get_pdfs (storage precision, natural layout) and
    handed over with PSM_BUFFERS_KEEP continues the run bit for bit (after an
    even number of steps the AA state is in the natural layout)."""
    import torch

    from paper_2502_20049_gb300 import psm

    case = small("fp32", streaming, omega=(0.0, 0.0, 0.0))
    ref = psm.Solver.from_case(case)
    ref.step(6)
    t = torch.from_numpy(ref.get_pdfs()).cuda()
    bufs = [t] if streaming == "aa" else [t, torch.zeros_like(t)]
    mine = with_bodies(psm.Solver(cfg_of(case), buffers=bufs, keep=True), case)
    ref.step(5)
    mine.step(5)
    assert np.array_equal(ref.get_pdfs(), mine.get_pdfs())


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
def test_get_pdfs_is_the_shifted_state(storage):
    from paper_2502_20049_gb300 import psm

    case = small(storage, "aa")
    s = psm.Solver.from_case(case)
    s.step(7)  # odd AA step: the stored layout is swapped, get_pdfs un-swaps it
    raw = s.get_pdfs()
    if storage == "bf16":
        raw = (raw.astype(np.uint32) << 16).view(np.float32)
    _, w, _ = psm.lattice_velocities(case.Q)
    full = s.get_state()
    d = np.abs(raw.astype(np.float64) + w[:, None, None, None] * case.rho0 - full)
    # stored populations: the same values; the ghost-plane populations of the
    # end planes are the ghost value, rounded to the storage type by get_pdfs
    assert d[:, 1:-1].max() <= 1e-15
    assert d.max() <= {"fp64": 1e-15, "fp32": 1e-8, "fp16": 1e-4, "bf16": 1e-3}[storage]


def test_init_equilibrium_field_uniform_and_varying():
    from paper_2502_20049_gb300 import psm

    case = small("fp64", "twogrid")
    a = psm.Solver.from_case(case)
    b = psm.Solver.from_case(case)
    rho = np.full((case.nz, case.ny, case.nx), 1.01)
    u = np.zeros((case.nz, case.ny, case.nx, 3))
    u[...] = (0.01, -0.02, 0.03)
    a.init_equilibrium(1.01, (0.01, -0.02, 0.03))
    b.init_equilibrium_field(rho, u)
    assert np.array_equal(a.get_state(), b.get_state())
    rng = np.random.default_rng(W.SEED + 9)
    rho = 1.0 + 0.05 * rng.random((case.nz, case.ny, case.nx))
    u = 0.05 * (rng.random((case.nz, case.ny, case.nx, 3)) - 0.5)
    b.init_equilibrium_field(rho, u)
    f = b.get_state()
    c, w, _ = psm.lattice_velocities(case.Q)
    cu = np.einsum("qk,zyxk->qzyx", c.astype(float), u)
    uu = (u * u).sum(-1)
    feq = w[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    inner = (slice(None), slice(1, -1))  # populations entering from a ghost plane take the ghost value
    assert np.abs(f[inner] - feq[inner]).max() <= 1e-15
    with pytest.raises(psm.PSMError):
        b.init_equilibrium_field(-rho, u)


def test_remap_switch():
    from paper_2502_20049_gb300 import psm

    # a static body: remapping every step or never gives the same bits
    case = small("fp32", "twogrid", omega=(0.0, 0.0, 0.0))
    a = psm.Solver.from_case(case)
    b = psm.Solver.from_case(case)
    b.set_remap(False)
    a.step(case.steps)
    b.step(case.steps)
    assert np.array_equal(a.get_state(), b.get_state())
    # a rotating body frozen at step 3 keeps that step's eps
    case = small("fp32", "twogrid", omega=(0.0, 0.0, 0.05))
    s = psm.Solver.from_case(case)
    s.step(3)
    e3 = s.eps()
    s.set_remap(False)
    s.step(4)
    assert np.array_equal(s.eps(), e3)
    s.set_remap(True)
    assert not np.array_equal(s.eps(), e3)
    s.record(2)
    with pytest.raises(psm.PSMError) as ei:
        s.set_remap(False)
    assert ei.value.code == -5


def test_force_torque_raw_is_the_printed_sign():
    from paper_2502_20049_gb300 import psm

    s = psm.Solver.from_case(small())
    s.step(5)
    ft = s.force_torque(0)
    assert np.abs(ft).max() > 0
    assert np.array_equal(s.force_torque_raw(0), -ft)


def test_device_buffer_check_classifies_memory():
    """psm_check_device_buffer (host only, launches nothing): host and
    page-locked host memory are refused, device memory of the current device
    is accepted, and a size beyond the allocation is refused."""
    import torch

    from paper_2502_20049_gb300 import psm

    a = np.zeros(1000)
    rc, msg = psm.check_device_buffer(a.ctypes.data, a.nbytes)
    assert rc == -1 and "host memory" in msg, msg
    p = torch.zeros(1000, dtype=torch.float64, pin_memory=True)
    rc, msg = psm.check_device_buffer(p.data_ptr(), 8000)
    assert rc == -1 and "page-locked" in msg, msg
    d = torch.zeros(1000, dtype=torch.float64, device="cuda")
    assert psm.check_device_buffer(d.data_ptr(), 8000)[0] == 0
    rc, msg = psm.check_device_buffer(d.data_ptr(), 1 << 40)
    assert rc == -1 and "bytes needed" in msg, msg


def test_entry_points_refuse_host_and_short_buffers():
    """psm_create_with_buffers and psm_mass_noalloc refuse host memory and a
    device allocation shorter than Q * ncell values with PSM_ERR_ARG before
    any launch.  Each pointer is first shown to be refused by the check alone,
    so no kernel ever sees it."""
    import ctypes

    import torch

    from paper_2502_20049_gb300 import psm

    cfg = psm.SolverConfig(64, 64, 64, streaming="twogrid", storage="fp32")
    need = 19 * 64 ** 3 * 4
    host = [np.zeros(19 * 64 ** 3, dtype=np.float32) for _ in range(2)]
    short = [torch.zeros(16, dtype=torch.float32, device="cuda") for _ in range(2)]
    for ptrs, why in (([h.ctypes.data for h in host], "host memory"), ([t.data_ptr() for t in short], "bytes needed")):
        for q in ptrs:
            rc, msg = psm.check_device_buffer(q, need)
            assert rc == -1 and why in msg, msg
        with pytest.raises(psm.PSMError) as ei:
            psm.Solver(cfg, buffers=ptrs)
        assert ei.value.code == -1 and why in str(ei.value)
        out = ctypes.c_double(3.0)
        rc = psm.lib().psm_mass_noalloc(ctypes.c_void_p(ptrs[0]), psm.STORAGE["fp32"], 19, 64 ** 3, 1.0, None,
                                        ctypes.byref(out))
        assert rc == -1 and out.value == 3.0
        assert why.encode() in psm.lib().psm_last_error()
