"""Pins of the oracle's geometry mapping (Sec. 3): super-sampled binary geometry
field, per-step transform of cell centres into the body frame, average over the
2^s x 2^s x 2^s sub-cells -> eps.

* identity pose with the sub-grid aligned to the lattice: eps equals the
  brute-force fraction of sub-cell centres inside the analytic body, exactly;
* a rotation by 90 degrees about an integer point permutes eps exactly;
* the centroid of eps follows the pose within half a sub-cell;
* sum eps matches the analytic volume for rotated bodies (Eq. 12 with dx^3):
  within 1 % for single poses of bodies as thin as 5 cells, within 1e-3 for
  the 100-step average of Sec. 3.1 at s >= 2 for bodies >= 12 cells across;
* the volume error of a cube rotating about all three axes falls with the
  resolution N and from s = 0 to s >= 1 (the trend of Table I).
"""

import os

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_cube_volume_error.txt")


def brute_eps(inside_fn, R0, shape, s, region):
    """eps by direct super-sampling of each cell (no geometry field, no transform)."""
    n = 1 << s
    nx, ny, nz = shape
    eps = np.zeros((nz, ny, nx))
    (x0, x1), (y0, y1), (z0, z1) = region
    off = (np.arange(n) + 0.5) / n
    for z in range(z0, z1):
        for y in range(y0, y1):
            xs = np.arange(x0, x1)
            px = (xs[:, None] - R0[0] + off[None, :])           # [cells, n]
            py = (y - R0[1] + off)
            pz = (z - R0[2] + off)
            X = px[:, None, None, :]
            Y = py[None, None, :, None]
            Z = pz[None, :, None, None]
            ins = inside_fn(X, Y, Z)
            eps[z, y, x0:x1] = ins.reshape(len(xs), -1).mean(1)
    return eps


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_identity_sphere_equals_bruteforce(oracle_mod, s):
    O = oracle_mod
    r = 6.0
    sub, lo = O.voxelize(W.SPHERE, (r,), s)
    R0 = (16.0, 16.0, 16.0)
    eps = O.remap(sub, s, lo, np.eye(3), R0, (0, 0, 0), (0, 0, 0), 0, (32, 32, 32))
    ref = brute_eps(lambda X, Y, Z: X * X + Y * Y + Z * Z <= r * r, R0, (32, 32, 32), s,
                    ((8, 24), (8, 24), (8, 24)))
    assert np.array_equal(eps, ref)
    assert eps.max() == 1.0 and (eps > 0).sum() > 100


def test_identity_ellipsoid_and_rotor_equal_bruteforce(oracle_mod):
    O = oracle_mod
    a, b, c = 7.0, 4.0, 2.5
    sub, lo = O.voxelize(W.ELLIPSOID, (a, b, c), 2)
    R0 = (12.0, 10.0, 9.0)
    eps = O.remap(sub, 2, lo, np.eye(3), R0, (0, 0, 0), (0, 0, 0), 0, (24, 20, 18))
    ref = brute_eps(lambda X, Y, Z: (X / a) ** 2 + (Y / b) ** 2 + (Z / c) ** 2 <= 1.0, R0, (24, 20, 18), 2,
                    ((0, 24), (0, 20), (0, 18)))
    assert np.array_equal(eps, ref)
    # rotor: brute force through the oracle's own point test
    rotor = W.Rotor().scaled(0.1)
    p = rotor.params()
    sub, lo = O.voxelize(W.ROTOR, p, 1)
    R0 = (10.0, 10.0, 6.0)
    eps = O.remap(sub, 1, lo, np.eye(3), R0, (0, 0, 0), (0, 0, 0), 0, (20, 20, 12))
    vin = np.vectorize(lambda x, y, z: O.inside(W.ROTOR, p, x, y, z))
    ref = brute_eps(lambda X, Y, Z: vin(X, Y, Z), R0, (20, 20, 12), 1, ((0, 20), (0, 20), (0, 12)))
    assert np.array_equal(eps, ref)
    assert (eps > 0).sum() > 50


def test_quarter_turn_permutes_eps(oracle_mod):
    O = oracle_mod
    sub, lo = O.voxelize(W.ELLIPSOID, (5.0, 3.0, 2.0), 2)
    R0 = (8.0, 8.0, 5.0)
    steps = 10
    om = (0.0, 0.0, (np.pi / 2) / steps)
    e0 = O.remap(sub, 2, lo, np.eye(3), R0, om, (0, 0, 0), 0, (16, 16, 10))
    e90 = O.remap(sub, 2, lo, np.eye(3), R0, om, (0, 0, 0), steps, (16, 16, 10))
    # world cell (x, y) at 90 deg sees the body point of cell (y, 15 - x) at 0 deg
    assert np.array_equal(e90, np.transpose(e0, (0, 2, 1))[:, :, ::-1])
    assert not np.array_equal(e90, e0)


@pytest.mark.parametrize("kind,params,vol", [
    (W.SPHERE, (6.0,), 4.0 / 3.0 * np.pi * 216.0),
    (W.ELLIPSOID, (9.0, 5.0, 3.0), 4.0 / 3.0 * np.pi * 135.0),
    (W.BOX, (4.5, 3.0, 2.5), 8 * 4.5 * 3.0 * 2.5),
])
def test_rotated_volume_single_poses(oracle_mod, kind, params, vol):
    """Single poses of rotated and translated bodies as thin as 5 cells: sum
    eps within 1 % of the analytic volume at s = 2.  (A single pose fluctuates
    by a few 1e-3 even for bodies 12 cells across; the 1e-3 bound holds for the
    time average of the next test.)"""
    O = oracle_mod
    s = 2
    sub, lo = O.voxelize(kind, params, s)
    th = 0.7
    Q0 = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    R0 = (16.3, 15.8, 16.1)
    for n in (0, 37, 101):
        eps = O.remap(sub, s, lo, Q0, R0, (0.004, 0.011, 0.007), (0.01, 0, -0.02), n, (32, 32, 32))
        assert abs(eps.sum() - vol) / vol < 1e-2
        assert eps.min() >= 0 and eps.max() <= 1


@pytest.mark.parametrize("kind,params,vol", [
    (W.SPHERE, (6.0,), 4.0 / 3.0 * np.pi * 216.0),
    (W.ELLIPSOID, (12.0, 8.0, 6.0), 4.0 / 3.0 * np.pi * 576.0),
    (W.BOX, (7.0, 6.5, 6.0), 8 * 7.0 * 6.5 * 6.0),
])
def test_rotated_volume_time_average(oracle_mod, kind, params, vol):
    """Sec. 3.1 verifies the mapping by the solid volume (Eq. 12, read with
    dx^3 and eps) averaged over 100 steps of a body rotating about all three
    axes.  Bodies whose half-widths are all >= 6 cells: the averaged volume is
    within 1e-3 of the analytic one for s = 2 and 3, and the error falls from
    s = 0 to s = 1 to s = 2."""
    O = oracle_mod
    th = 0.7
    Q0 = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    R0 = (14.3, 13.8, 14.1)
    err = []
    for s in (0, 1, 2, 3):
        sub, lo = O.voxelize(kind, params, s)
        v = [O.remap(sub, s, lo, Q0, R0, (0.011, 0.017, 0.013), (0, 0, 0), n, (28, 28, 28)).sum() for n in range(100)]
        err.append(abs(np.mean(v) - vol) / vol)
    print(kind, params, ["%.2e" % e for e in err])
    assert err[2] <= 1e-3 and err[3] <= 1e-3
    assert err[0] > err[1] > err[2]


@pytest.mark.parametrize("s", [1, 2, 3])
def test_centroid_follows_pose(oracle_mod, s):
    """The centroid of eps is the centroid of the geometry field carried by the
    pose, R_n + Q_n c_body (pose from scipy's rotation vectors, not the
    oracle's), within half a sub-cell per axis: snapping each cell's block to
    the nearest sub-grid point moves it by at most h/2 = 2^-(s+1) (bodies many
    sub-cells thick, so that the snapping shifts average over the surface),
    and a lookup that were off by half a sub-cell or more, or that rotated the
    wrong way, would exceed it."""
    from scipy.spatial.transform import Rotation

    O = oracle_mod
    th = 0.7
    Q0 = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    R0 = np.array([14.3, 13.8, 14.1])
    om = np.array([0.011, 0.017, 0.013])
    v = np.array([0.003, -0.002, 0.001])
    ax = np.arange(28) + 0.5
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    h = 1.0 / (1 << s)
    worst = 0.0
    for kind, params in [(W.SPHERE, (6.0,)), (W.ELLIPSOID, (12.0, 8.0, 6.0)), (W.BOX, (7.0, 6.5, 6.0))]:
        sub, lo = O.voxelize(kind, params, s)
        nz, ny, nx = sub.shape
        bz, by, bx = np.meshgrid((np.arange(nz) + 0.5) * h + lo[2], (np.arange(ny) + 0.5) * h + lo[1],
                                 (np.arange(nx) + 0.5) * h + lo[0], indexing="ij")
        cb = np.array([(sub * bx).sum(), (sub * by).sum(), (sub * bz).sum()]) / sub.sum()
        for k in range(0, 100, 3):
            e = O.remap(sub, s, lo, Q0, tuple(R0), tuple(om), tuple(v), k, (28, 28, 28))
            c = np.array([(e * X).sum(), (e * Y).sum(), (e * Z).sum()]) / e.sum()
            expect = R0 + v * k + Rotation.from_rotvec(om * k).as_matrix() @ Q0 @ cb
            worst = max(worst, np.abs(c - expect).max())
    print(f"s={s}: centroid within {worst:.4f} cells of the pose (bound {h / 2})")
    assert worst <= h / 2


def test_cube_volume_error_trend_table1(oracle_mod):
    O = oracle_mod
    golden = np.loadtxt(GOLDEN)
    assert golden.shape == (3, 5)
    err = {}
    for N in (10, 20):
        for s in (0, 1, 2, 3):
            sub, lo = O.voxelize(W.BOX, (N / 2.0,) * 3, s)
            n = 2 * N
            vols = [O.remap(sub, s, lo, np.eye(3), (n / 2,) * 3, (0.013, 0.009, 0.005), (0, 0, 0), 4 * k,
                            (n, n, n)).sum() for k in range(12)]
            err[N, s] = np.mean(np.abs(np.array(vols) - N ** 3)) / N ** 3
    # Table I: s = 0 is the worst column and the error falls with N
    for N in (10, 20):
        assert err[N, 0] > max(err[N, 1], err[N, 2], err[N, 3])
        assert err[N, 3] < err[N, 1]
    for s in (0, 1, 2, 3):
        assert err[20, s] < err[10, s]
    gd = {int(r[0]): r[1:] for r in golden}
    assert gd[20][0] > max(gd[20][1:]) and gd[40][0] > max(gd[40][1:])


def test_out_of_box_is_zero_and_multibody(oracle_mod):
    """Bits outside the stored box count as 0; two bodies: eps = min(1, sum),
    owner = argmax (lower id on ties)."""
    O = oracle_mod
    sub, lo = O.voxelize(W.BOX, (2.0, 2.0, 2.0), 1)
    cfg = O.Config(nx=16, ny=8, nz=8, bc_z=0)
    sim = O.Sim(cfg)
    sim.add_body(O.BodySpec(sub=sub, s=1, lo=lo, R0=(5.0, 4.0, 4.0)))
    sim.add_body(O.BodySpec(sub=sub, s=1, lo=lo, R0=(8.0, 4.0, 4.0)))
    eps, owner = sim.eps(0)
    e0 = O.remap(sub, 1, lo, np.eye(3), (5.0, 4.0, 4.0), (0, 0, 0), (0, 0, 0), 0, (16, 8, 8))
    e1 = O.remap(sub, 1, lo, np.eye(3), (8.0, 4.0, 4.0), (0, 0, 0), (0, 0, 0), 0, (16, 8, 8))
    assert np.array_equal(eps, np.minimum(1.0, e0 + e1))
    exp_owner = np.where(e0 + e1 == 0, -1, np.where(e1 > e0, 1, 0))
    assert np.array_equal(owner, exp_owner)
    assert ((e0 > 0) & (e1 > 0)).sum() > 0  # the boxes overlap in x = 6..7
