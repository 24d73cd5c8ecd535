"""GPU discrete adjoint (psm_record / psm_backward, through the C ABI) against
the oracle's tangent-linear model and against central finite differences.

J = mean torque about z on body 0 over the recorded steps.  The tangent-linear
model is the oracle's own FP64 step on dual numbers (pinned against FP64
finite differences in test_oracle_tangent.py); a directional derivative there
must equal the inner product of the GPU gradient with the same direction.
"""

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()


def small_case(storage="fp64", fluid="trt", solid=1, weighting=1, streaming="aa", steps=24, bc_z=1):
    return W.Case("adj_small", 12, 12, 16, Q=19, storage=storage, streaming=streaming, fluid=fluid, tau=0.62,
                  solid=solid, weighting=weighting, bc_z=bc_z, u_in=(0.0, 0.0, 0.03), steps=steps,
                  bodies=[W.BodyCase(W.ELLIPSOID, (4.0, 2.2, 1.8), 2, (6.0, 6.2, 8.0), omega=(0.0, 0.0, 0.04))])


def gpu_grad(case, K=4):
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(case)
    sol.record(K, init_from_inflow=True)
    sol.step(case.steps)
    ge, gw, gu = sol.backward()
    J = sol.force_torque(0)[:, 5].mean()
    return J, ge, gw, gu


def oracle_tl(case, d_delta=None, d_omega=(0, 0, 0), d_u=(0, 0, 0)):
    import oracle

    cfg = oracle.Config(nx=case.nx, ny=case.ny, nz=case.nz, Q=case.Q, bc_z=case.bc_z, rho0=case.rho0,
                        u_in=tuple(case.u_in), fluid={"bgk": 0, "trt": 1}[case.fluid], tau=case.tau,
                        trt_lambda=case.trt_lambda, solid=case.solid, weighting=case.weighting)
    sim = oracle.TangentSim(cfg, d_u_in=d_u)
    b = case.bodies[0]
    sub, lo = oracle.voxelize(b.kind, b.params, b.s)
    sim.add_body(oracle.BodySpec(sub=sub, s=b.s, lo=lo, R0=b.R0, Q0=np.array(b.Q0), omega=b.omega, v=b.v),
                 d_omega=d_omega)
    sim.init_eq(case.rho0, case.u_in, du=d_u)
    sim.set_delta(None, d_delta)
    sim.step(case.steps)
    v, t = sim.force_torque()
    return v[:, 0, 5].mean(), t[:, 0, 5].mean()


CASES = [dict(), dict(fluid="bgk"), dict(solid=2), dict(solid=3), dict(weighting=0), dict(streaming="twogrid"),
         dict(bc_z=0)]


@pytest.mark.parametrize("kw", CASES)
def test_adjoint_fp64_matches_tangent_linear(kw):
    case = small_case(**kw)
    J, ge, gw, gu = gpu_grad(case)
    v = W.random_unit((case.nz, case.ny, case.nx), seed=W.SEED + 5)
    J_or, dv = oracle_tl(case, d_delta=v)
    assert abs(J - J_or) <= 1e-12 * abs(J_or)
    ip = float((ge * v).sum())
    print(f"{kw}: <grad, v> {ip:.12e} vs tangent {dv:.12e}")
    assert abs(ip - dv) <= 1e-9 * abs(dv)
    _, dw = oracle_tl(case, d_omega=(0.0, 0.0, 1.0))
    assert abs(gw[0, 2] - dw) <= 1e-9 * abs(dw)
    _, dwx = oracle_tl(case, d_omega=(1.0, 0.0, 0.0))
    assert abs(gw[0, 0] - dwx) <= 1e-9 * max(abs(dwx), 1e-3 * abs(dw))
    _, du = oracle_tl(case, d_u=(0.0, 0.0, 1.0))
    assert abs(gu[2] - du) <= 1e-9 * abs(du)


def tiny_case(fluid="trt", solid=1, weighting=1, streaming="aa", bc_z=1, at_ghost=False, steps=12):
    """6 x 6 x 8 cells, a rotating ellipsoid (at_ghost: low in z, covering the
    planes next to the lower ghost plane, and a second, translating box)."""
    z = 1.4 if at_ghost else 4.0
    bodies = [W.BodyCase(W.ELLIPSOID, (2.2, 1.5, 1.2), 2, (3.0, 3.1, z), omega=(0.01, -0.02, 0.05))]
    if at_ghost:
        bodies.append(W.BodyCase(W.BOX, (1.0, 1.0, 1.0), 1, (3.2, 2.8, 6.3), omega=(0.0, 0.03, 0.0),
                                 v=(0.01, 0.0, -0.02)))
    return W.Case("adj_tiny", 6, 6, 8, Q=19, storage="fp64", streaming=streaming, fluid=fluid, tau=0.62,
                  solid=solid, weighting=weighting, bc_z=bc_z, u_in=(0.004, -0.003, 0.03), steps=steps,
                  bodies=bodies)


def oracle_gradient(case):
    import oracle

    cfg = oracle.Config(nx=case.nx, ny=case.ny, nz=case.nz, Q=case.Q, bc_z=case.bc_z, rho0=case.rho0,
                        u_in=tuple(case.u_in), fluid={"bgk": 0, "trt": 1}[case.fluid], tau=case.tau,
                        trt_lambda=case.trt_lambda, solid=case.solid, weighting=case.weighting)
    specs = []
    for b in case.bodies:
        sub, lo = oracle.voxelize(b.kind, b.params, b.s)
        specs.append(oracle.BodySpec(sub=sub, s=b.s, lo=lo, R0=b.R0, Q0=np.array(b.Q0), omega=b.omega, v=b.v))
    return oracle.tangent_gradient(cfg, specs, case.steps, case.rho0, tuple(case.u_in))


PER_CELL = [dict(), dict(fluid="bgk"), dict(solid=2), dict(solid=3), dict(weighting=0), dict(streaming="twogrid"),
            dict(bc_z=0), dict(at_ghost=True), dict(at_ghost=True, streaming="twogrid", solid=3)]


@pytest.mark.parametrize("kw", PER_CELL)
def test_adjoint_fp64_every_cell_matches_oracle(kw):
    """The GPU FP64 gradient, cell by cell, against the oracle's FP64 gradient
    (one tangent-linear run per cell; pinned against central differences of
    the plain oracle in test_oracle_tangent.py): 1e-9 relative per cell plus
    1e-11 of max |grad|; grad_omega and grad_u_in component by component."""
    case = tiny_case(**kw)
    J, ge, gw, gu = gpu_grad(case, K=4)
    J_or, gd, gw_or, gu_or = oracle_gradient(case)
    assert abs(J - J_or) <= 1e-12 * abs(J_or)
    scale = np.abs(gd).max()
    err = np.abs(ge - gd)
    bound = 1e-9 * np.abs(gd) + 1e-11 * scale
    worst = int(np.argmax(err - bound))
    print(f"{kw}: max |grad_gpu - grad_oracle| = {err.max():.3e} (max |grad| {scale:.3e}); "
          f"omega {np.abs(gw - gw_or[:len(gw)]).max():.3e}, u_in {np.abs(gu - gu_or).max():.3e}")
    assert np.all(err <= bound), (np.unravel_index(worst, ge.shape), ge.reshape(-1)[worst], gd.reshape(-1)[worst])
    assert (np.abs(gd) > 1e-6 * scale).sum() > case.cells // 4
    gscale = np.abs(gw_or).max()
    assert np.all(np.abs(gw - gw_or) <= 1e-9 * np.abs(gw_or) + 1e-11 * gscale), (gw, gw_or)
    assert np.all(np.abs(gu - gu_or) <= 1e-9 * np.abs(gu_or) + 1e-11 * np.abs(gu_or).max()), (gu, gu_or)


@pytest.mark.parametrize("solid", [1, 2, 3])
@pytest.mark.parametrize("fluid", ["trt", "bgk"])
def test_adjoint_fluid_tiles_match_tangent_linear(solid, fluid):
    """A small body in a long periodic box: most tiles hold no body and take
    the adjoint's fluid-only path (B = 0), the rest the general one."""
    case = W.Case("adj_sparse", 64, 8, 20, Q=19, storage="fp64", streaming="aa", fluid=fluid, tau=0.6,
                  solid=solid, weighting=1, bc_z=0, u_in=(0.02, 0.0, 0.03), steps=16,
                  bodies=[W.BodyCase(W.SPHERE, (2.5,), 2, (12.0, 4.0, 10.0), omega=(0.0, 0.0, 0.05))])
    J, ge, gw, gu = gpu_grad(case)
    v = W.random_unit((case.nz, case.ny, case.nx), seed=W.SEED + 8)
    J_or, dv = oracle_tl(case, d_delta=v)
    assert abs(J - J_or) <= 1e-12 * abs(J_or)
    ip = float((ge * v).sum())
    assert abs(ip - dv) <= 1e-9 * abs(dv)
    # a direction supported only on the fluid-only tiles (planes far from the body)
    far = np.zeros_like(v)
    far[:3] = v[:3]
    far[17:] = v[17:]
    _, dfar = oracle_tl(case, d_delta=far)
    assert abs(float((ge * far).sum()) - dfar) <= 1e-9 * abs(dfar)
    _, dw = oracle_tl(case, d_omega=(0.0, 0.0, 1.0))
    assert abs(gw[0, 2] - dw) <= 1e-9 * abs(dw)
    _, du = oracle_tl(case, d_u=(0.0, 0.0, 1.0))
    assert abs(gu[2] - du) <= 1e-9 * abs(du)


@pytest.mark.parametrize("storage,tol", [("fp32", 1e-3), ("fp16", 2e-2)])
def test_adjoint_reduced_precision_matches_tangent_linear(storage, tol):
    case = small_case(storage=storage)
    J, ge, gw, gu = gpu_grad(case)
    v = W.random_unit((case.nz, case.ny, case.nx), seed=W.SEED + 6)
    _, dv = oracle_tl(case, d_delta=v)
    _, dw = oracle_tl(case, d_omega=(0.0, 0.0, 1.0))
    _, du = oracle_tl(case, d_u=(0.0, 0.0, 1.0))
    ip = float((ge * v).sum())
    errs = (abs(ip - dv) / abs(dv), abs(gw[0, 2] - dw) / abs(dw), abs(gu[2] - du) / abs(du))
    print(f"{storage} adjoint relative errors (delta, omega, u_in): {errs}")
    assert max(errs) <= tol


def fd_richardson(J_of, n, c, h):
    """Central difference at h and h/2 combined by Richardson extrapolation
    (truncation error O(h^4)).  The solid fraction enters through B(eps) with
    B' = (1 + t) / t at eps = 1 (t = tau - 1/2: 21 at tau = 0.55), and B > 1
    makes a fully solid cell anti-dissipative, so J(delta) is strongly curved
    there: at h = 1e-4 even Richardson differences are biased by ~1 % and at
    h = 1e-3 the perturbed run can blow up.  The checks use h = 1e-6 in FP64
    (the differences converge to the adjoint as h shrinks)."""
    def D(hh):
        d = np.zeros(n, np.float32)
        d[c] = hh
        return (J_of(d) - J_of(-d)) / (2 * hh)

    return (4 * D(h / 2) - D(h)) / 3


def swept_cells(case, k=16, every=8):
    from paper_2502_20049_gb300 import psm

    mask = np.zeros((case.nz, case.ny, case.nx), bool)
    sol = psm.Solver.from_case(case)
    for n in range(0, case.steps, every):
        mask |= sol.eps() > 0
        sol.step(every)
    return W.pick_cells(mask, k)


def J_fp64(case):
    from paper_2502_20049_gb300 import psm

    c64 = case.with_(storage="fp64")

    def J_of(delta):
        s = psm.Solver.from_case(c64)
        s.set_eps_delta(delta)
        s.step(c64.steps)
        return s.force_torque(0)[:, 5].mean()

    return J_of


def test_adjoint_fp64_vs_central_fd_16_cells():
    """GPU FP64 adjoint vs FP64 central differences (h = 1e-6, Richardson) of
    the GPU forward on 16 seeded cells of the body's swept region."""
    case = W.c4_adjoint(n=32, steps=48).with_(storage="fp64")
    case.bodies[0].omega = (0.0, 0.0, 0.01)
    J, ge, _, _ = gpu_grad(case, K=8)
    J_of = J_fp64(case)
    scale = np.abs(ge).max()
    for c in swept_cells(case):
        fd = fd_richardson(J_of, case.cells, c, 1e-6)
        g = ge.reshape(-1)[c]
        assert abs(g - fd) <= 1e-5 * abs(fd) + 1e-7 * scale, (c, g, fd)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_adjoint_c4_full_vs_fp64_fd(storage):
    """The adjoint workload at full size: 128^3, 512 steps, checkpoint every 64
    steps, TRT tau 0.55, against FP64 central differences (h = 1e-6,
    Richardson) of the GPU forward on 16 seeded cells of the swept region.
    FP64 adjoint: 1e-5 relative per cell plus 1e-7 of max|grad| (the
    difference's round-off floor).  FP32 forward and adjoint (the
    gradient of the FP32 trajectory): 1e-2 relative per cell (the relative
    error of each cell is printed)."""
    case = W.c4_adjoint().with_(storage=storage)
    J, ge, gw, gu = gpu_grad(case, K=64)
    cells = swept_cells(case, every=64)
    J_of = J_fp64(case)
    scale = np.abs(ge).max()
    worst_rel, worst_scaled, fp64_ok = 0.0, 0.0, True
    for c in cells:
        fd = fd_richardson(J_of, case.cells, c, 1e-6)
        g = ge.reshape(-1)[c]
        rel = abs(g - fd) / max(abs(fd), 1e-300)
        print(f"{storage} cell {c}: adjoint {g:.9e} fd {fd:.9e} rel {rel:.3e} (max |grad| {scale:.3e})")
        worst_rel = max(worst_rel, rel if abs(fd) > 1e-3 * scale else 0.0)
        worst_scaled = max(worst_scaled, abs(g - fd) / scale)
        # FP64: 1e-5 relative per cell plus 1e-7 of max|grad|, the round-off floor of a
        # central difference at h = 1e-6 (about eps_mach |J| / h), which dominates for
        # cells whose derivative is ~1e-3 of the largest
        fp64_ok = fp64_ok and abs(g - fd) <= 1e-5 * abs(fd) + 1e-7 * scale
    print(f"C4 128^3 {storage} adjoint vs FP64 FD, 16 cells: worst relative {worst_rel:.3e}, "
          f"worst / max|grad| {worst_scaled:.3e}")
    if storage == "fp64":
        assert fp64_ok and worst_scaled <= 1e-6
    else:
        assert worst_rel <= 1e-2 and worst_scaled <= 1e-3


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_adjoint_c4_full_omega_and_inflow_vs_fp64_fd(storage):
    """The adjoint workload at full size (128^3, 512 steps, checkpoint every 64):
    d J / d omega_z and d J / d u_in,z against central differences of the FP64
    GPU forward at the relative step h = 1e-4 of the configuration, Richardson
    extrapolated.  omega is varied in u_s only (psm_set_us_omega: the geometry
    sequence stays the nominal one, as the adjoint defines the derivative);
    u_in in the ghost planes and the initial equilibrium (the recording
    declares the initial state f^eq(rho0, u_in)).  FP64: 1e-6 relative; FP32
    forward and adjoint: 1e-2."""
    from paper_2502_20049_gb300 import psm

    case = W.c4_adjoint().with_(storage=storage)
    J, ge, gw, gu = gpu_grad(case, K=64)
    c64 = case.with_(storage="fp64")
    w0 = np.array(c64.bodies[0].omega, dtype=float)
    u0 = np.array(c64.u_in, dtype=float)

    def J_of(omega=None, u_in=None):
        c = c64 if u_in is None else c64.with_(u_in=tuple(u_in))
        sol = psm.Solver.from_case(c)
        if omega is not None:
            sol.set_us_omega(0, omega)
        sol.step(c.steps)
        j = sol.force_torque(0)[:, 5].mean()
        sol.close()
        return j

    def rich(f, x0, k, hrel):
        h = hrel * abs(x0[k])

        def D(hh):
            e = np.zeros(3)
            e[k] = hh
            return (f(x0 + e) - f(x0 - e)) / (2 * hh)

        return (4 * D(h / 2) - D(h)) / 3

    fd_w = rich(lambda w: J_of(omega=w), w0, 2, 1e-4)
    fd_u = rich(lambda u: J_of(u_in=u), u0, 2, 1e-4)
    ew, eu = abs(gw[0, 2] - fd_w) / abs(fd_w), abs(gu[2] - fd_u) / abs(fd_u)
    print(f"C4 128^3 {storage}: dJ/domega_z adjoint {gw[0, 2]:.9e} fd {fd_w:.9e} rel {ew:.2e}; "
          f"dJ/du_in,z adjoint {gu[2]:.9e} fd {fd_u:.9e} rel {eu:.2e}")
    tol = 1e-6 if storage == "fp64" else 1e-2
    assert ew <= tol and eu <= tol


def test_autograd_function_fp64():
    import torch

    from paper_2502_20049_gb300.autograd import PSMTorque

    case = small_case()
    eps_delta = torch.zeros((case.nz, case.ny, case.nx), dtype=torch.float64, device="cuda", requires_grad=True)
    omega = torch.tensor(case.bodies[0].omega, dtype=torch.float64, requires_grad=True)
    u_in = torch.tensor(case.u_in, dtype=torch.float64, requires_grad=True)
    J = PSMTorque.apply(eps_delta, omega, u_in, case, case.steps, 4)
    J.backward()
    v = W.random_unit((case.nz, case.ny, case.nx), seed=W.SEED + 7)
    J_or, dv = oracle_tl(case, d_delta=v)
    _, dw = oracle_tl(case, d_omega=(0.0, 0.0, 1.0))
    assert abs(float(J.detach()) - J_or) <= 1e-12 * abs(J_or)
    assert abs(float((eps_delta.grad.cpu().numpy() * v).sum()) - dv) <= 1e-9 * abs(dv)
    assert abs(float(omega.grad[2]) - dw) <= 1e-9 * abs(dw)


@pytest.mark.parametrize("storage", ["fp16", "fp32"])
@pytest.mark.parametrize("streaming", ["aa", "twogrid"])
def test_backward_tma_recompute_equals_plain(storage, streaming):
    """A TMA-tiled grid (64 x 8 x 16): the backward pass recomputes each segment
    with the TMA two-grid kernel on its own tiling (two cells per thread for
    FP16) whatever the forward's streaming; its gradients equal those of the
    plain-kernel recompute (bit-identical states, same adjoint kernel)."""
    from paper_2502_20049_gb300 import psm

    case = W.Case("adj_tma", 64, 8, 16, Q=19, storage=storage, streaming=streaming, fluid="trt", tau=0.62,
                  u_in=(0.0, 0.0, 0.03), steps=24,
                  bodies=[W.BodyCase(W.ELLIPSOID, (6.0, 2.5, 2.0), 2, (30.0, 4.1, 8.0), omega=(0.0, 0.0, 0.04))])
    out = []
    for variant in ("tma", "plain"):
        sol = psm.Solver.from_case(case)
        sol.set_kernel_variant(variant)
        sol.record(8, init_from_inflow=True)
        sol.step(case.steps)
        out.append((sol.get_state(), *sol.backward()))
    (sa, ga, wa, ua), (sb, gb, wb, ub) = out
    assert np.array_equal(sa, sb)
    assert np.array_equal(ga, gb)
    assert np.abs(ga).max() > 0
    assert np.array_equal(wa, wb) and np.array_equal(ua, ub)


def test_backward_without_record_is_state_error():
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(small_case())
    sol.step(2)
    with pytest.raises(psm.PSMError) as ei:
        sol.backward()
    assert ei.value.code == -5


@pytest.mark.parametrize("storage,streaming", [("fp32", "aa"), ("fp64", "twogrid"), ("fp16", "aa")])
def test_backward_overlapped_recompute_equals_one_segment(storage, streaming):
    """psm_backward recomputes the segment before the current one on a second
    stream while the adjoint sweeps the current one (several segments: K = 4,
    6 or 8 of 24 steps); with PSM_RECORD_SEQUENTIAL, or with one segment
    (K = 24), it recomputes and sweeps in turn on the solver's stream.  The
    recomputed states equal the recorded ones bit for bit either way, so every
    gradient agrees bit for bit."""
    from paper_2502_20049_gb300 import psm

    case = W.Case("adj_overlap", 64, 8, 16, Q=19, storage=storage, streaming=streaming, fluid="trt", tau=0.62,
                  u_in=(0.0, 0.0, 0.03), steps=24,
                  bodies=[W.BodyCase(W.ELLIPSOID, (6.0, 2.5, 2.0), 2, (30.0, 4.1, 8.0), omega=(0.0, 0.0, 0.04))])
    out = {}
    for K, seq in ((24, False), (4, False), (6, False), (8, False), (4, True), (8, True)):
        sol = psm.Solver.from_case(case)
        sol.record(K, init_from_inflow=True, sequential=seq)
        sol.step(case.steps)
        out[K, seq] = sol.backward()
        if K == 8 and not seq:
            out["again"] = sol.backward()  # a second pass over the same recording
        sol.close()
    g0, w0, u0 = out[24, False]
    assert np.abs(g0).max() > 0 and np.abs(w0).max() > 0
    for key, (g, w, u) in out.items():
        assert np.array_equal(g, g0), (key, np.abs(g - g0).max())
        assert np.array_equal(w, w0) and np.array_equal(u, u0), key


def test_record_rejects_unknown_flags():
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(small_case())
    with pytest.raises(psm.PSMError) as ei:
        psm.check(psm.lib().psm_record(sol._h, 4, 4))
    assert ei.value.code == -1
    sol.close()
