"""z-slab decomposition on the GPU (Sec. 5.2: one block of the lattice per GPU,
populations crossing block faces exchanged every step).

Several handles on one GPU each hold a z-slab (psm_set_z_offset, periodic in
z); the exchange of paper_2502_20049_gb300.slabs moves the face slots between
their PDF buffers with device copies (psm_slot_plane) and refills the
domain's ends with the inflow equilibrium (psm_fill_slot_plane).  The
decomposed run equals the undecomposed one bit for bit in every PDF, for the
AA pattern (moves before and after odd steps) and two-grid streaming (after
every step), on a periodic domain and on one bounded by ghost planes, in FP64
and FP32; in FP16 storage bit for bit on the periodic domain and within FP16
rounding where the ends hold the inflow equilibrium (stored in FP16 by the
slab, kept in FP32 by the undecomposed kernel).  Force and torque summed over
the slabs agree to round-off (another summation order).  The handles run one
after the other on one stream; no kernel waits for another.  The states are
compared after an even number of steps: in the AA pattern's swapped layout
(after an odd number) a face cell's populations sit in the neighbouring
slab's slots until the next odd step's exchange, so a slab alone cannot
export them.
"""

import numpy as np
import pytest

from paper_2502_20049_gb300 import slabs as S
from paper_2502_20049_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()


def case(storage, streaming, bc_z, Q=19, nz=30):
    bodies = [W.BodyCase(W.ELLIPSOID, (7.0, 4.0, 5.0), 2, (15.3, 8.2, nz * 0.45), omega=(0.01, 0.02, 0.03),
                         v=(0.0, 0.0, 0.02)),
              W.BodyCase(W.BOX, (2.5, 2.0, 3.0), 1, (24.0, 9.0, nz * 0.75), omega=(0.0, 0.0, -0.04),
                         v=(0.01, 0.0, -0.03))]
    return W.Case("slabs_gpu", 32, 16, nz, Q=Q, storage=storage, streaming=streaming, fluid="trt", tau=0.7,
                  bc_z=bc_z, u_in=(0.01, -0.005, 0.02), steps=26, bodies=bodies)


def undecomposed(c):
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(c)
    sol.step(c.steps)
    out = sol.get_state(), np.stack([sol.force_torque(b) for b in range(len(c.bodies))], 1)
    sol.close()
    return out


def decomposed(c, world):
    from paper_2502_20049_gb300 import psm

    slabs = []
    for z0, n in S.partition(c.nz, world):
        sol = psm.Solver.from_case(c.with_(nz=n, bc_z=0), init=False)
        slab = S.PsmSlab(sol, z0)
        sol.init_equilibrium(c.rho0, c.u_in)
        slabs.append(slab)
    dec = S.Decomposition(slabs, S.LocalRing(world), c.streaming, bounded=c.bc_z == 1)
    dec.prepare()
    dec.run(c.steps, lambda s: s.sol.step(1))
    f = np.concatenate([s.sol.get_state() for s in slabs], axis=1)
    ft = dec.allreduce([np.stack([s.sol.force_torque(b) for b in range(len(c.bodies))], 1) for s in slabs])[0]
    for s in slabs:
        s.sol.close()
    return f, ft


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("streaming", ["aa", "twogrid"])
@pytest.mark.parametrize("bc_z", [0, 1])
def test_slabs_equal_undecomposed(storage, streaming, bc_z):
    c = case(storage, streaming, bc_z)
    fr, ftr = undecomposed(c)
    for world in (2, 3):
        f, ft = decomposed(c, world)
        if storage == "fp16" and bc_z == 1:
            err = np.abs(f - fr).max()
            assert err <= 2e-3 * np.linalg.norm(c.u_in), (world, err)
            assert np.abs(ft - ftr).max() <= 1e-2 * np.abs(ftr).max()
        else:
            assert np.array_equal(f, fr), (world, np.abs(f - fr).max())
            assert np.abs(ft - ftr).max() <= 1e-12 * np.abs(ftr).max(), world
    assert np.abs(ftr).max() > 0


def test_slabs_d3q27_aa():
    c = case("fp32", "aa", 1, Q=27, nz=21).with_(steps=14)
    fr, ftr = undecomposed(c)
    f, ft = decomposed(c, 3)
    assert np.array_equal(f, fr)
    assert np.abs(ft - ftr).max() <= 1e-12 * np.abs(ftr).max()


def test_slab_entry_points_check_arguments():
    from paper_2502_20049_gb300 import psm

    sol = psm.Solver.from_case(case("fp32", "aa", 0, nz=8).with_(bodies=[]))
    for bad in ((19, 0), (-1, 0), (0, 8), (0, -1)):
        with pytest.raises(psm.PSMError) as ei:
            sol.slot_plane_ptr(*bad)
        assert ei.value.code == -1
    with pytest.raises(psm.PSMError):
        sol.fill_slot_plane(0, 0, 19)
    with pytest.raises(psm.PSMError):
        sol.set_z_offset(-1)
    sol.set_z_offset(8)
    with pytest.raises(psm.PSMError) as ei:
        sol.record(2)
    assert ei.value.code == -6
    # the plane views alias the PDF buffer: a fill with the inflow equilibrium
    # (shifted) of direction 5, then of its opposite, shows in the view
    c, w, opp = psm.lattice_velocities(19)
    u = np.array([0.01, -0.005, 0.02])
    for d in (5, int(opp[5])):
        sol.fill_slot_plane(5, 3, d)
        v = sol.slot_plane(5, 3)
        cu = float(c[d] @ u)
        expect = w[d] * (3 * cu + 4.5 * cu * cu - 1.5 * float(u @ u))
        assert v.shape == (16, 32)
        assert np.allclose(v.cpu().numpy(), expect, rtol=1e-6, atol=1e-9)
    sol.close()
