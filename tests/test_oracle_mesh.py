"""Pins of the oracle's triangle-mesh voxeliser (Sec. 3): the analytic box
voxeliser where both apply, the half-open closed form its tie rule gives for a
box whose faces pass through sub-cell centres, an exact big-integer half-space
test for convex polyhedra, and the polyhedron volume for a sphere mesh."""

import math

import numpy as np
import pytest

from paper_2502_20049_gb300 import workloads as W


def centres(sub_shape, lo, s):
    """World coordinates of the sub-cell centres along each axis (z, y, x order of the array)."""
    h = 2.0 ** -s
    nz, ny, nx = sub_shape
    return (lo[2] + (np.arange(nz) + 0.5) * h, lo[1] + (np.arange(ny) + 0.5) * h, lo[0] + (np.arange(nx) + 0.5) * h)


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_box_on_subcell_boundaries_equals_analytic_box(oracle_mod, s):
    h = (3.25, 2.5, 1.75) if s >= 2 else (3.0, 2.0, 1.0)
    sub, lo = oracle_mod.voxelize_mesh(*W.box_mesh([-a for a in h], h), s)
    zc, yc, xc = centres(sub.shape, lo, s)
    expect = ((np.abs(zc)[:, None, None] <= h[2]) & (np.abs(yc)[None, :, None] <= h[1])
              & (np.abs(xc)[None, None, :] <= h[0]))
    assert np.array_equal(sub.astype(bool), expect)
    # the analytic voxeliser of the same box, on the cells both fields cover
    ref, rlo = oracle_mod.voxelize(W.BOX, h, s)
    off = [int(round((lo[k] - rlo[k]) * 2 ** s)) for k in range(3)]
    part = ref[off[2]:off[2] + sub.shape[0], off[1]:off[1] + sub.shape[1], off[0]:off[0] + sub.shape[2]]
    assert part.shape == sub.shape and np.array_equal(part, sub)


def test_box_through_subcell_centres_is_half_open(oracle_mod):
    """Faces through sample points: the tie rule (centre moved by (delta^2,
    delta) in (y, z); crossings at or ahead of the centre counted) makes the
    inside set x0 < x <= x1, y0 <= y < y1, z0 <= z < z1 exactly."""
    s = 2
    lo_b, hi_b = (1.125, -0.875, 0.375), (4.625, 2.375, 3.125)  # all at sub-cell centres (k + 1/2) / 4
    sub, lo = oracle_mod.voxelize_mesh(*W.box_mesh(lo_b, hi_b), s)
    zc, yc, xc = centres(sub.shape, lo, s)
    ex = (xc > lo_b[0]) & (xc <= hi_b[0])
    ey = (yc >= lo_b[1]) & (yc < hi_b[1])
    ez = (zc >= lo_b[2]) & (zc < hi_b[2])
    assert np.array_equal(sub.astype(bool), ez[:, None, None] & ey[None, :, None] & ex[None, None, :])


def _q(x, lo, s):
    """The quantisation of the voxeliser: round half away from zero of (x - lo) 2^(s+8)."""
    y = (float(x) - lo) * 2.0 ** (s + 8)
    return int(math.copysign(math.floor(abs(y) + 0.5), y))


def test_convex_polyhedron_equals_exact_halfspace_test(oracle_mod):
    """Random rotated and shifted icosahedron (convex): a centre is inside iff it
    lies behind every face plane, decided with Python's exact integers on the
    quantised vertices; centres on a plane are skipped."""
    s = 2
    rng = np.random.default_rng(W.SEED)
    R = W.rot("z", 0.37) @ W.rot("x", 1.1)
    v, t = W.transform_mesh(W.icosphere(4.3, 0), R, shift=(0.3, -0.21, 0.17) + 0.1 * rng.random(3))
    sub, lo = oracle_mod.voxelize_mesh(v, t, s)
    Q = [[_q(v[i][k], lo[k], s) for k in range(3)] for i in range(len(v))]
    faces = []
    for a, b, c in t:
        A, B, C = Q[a], Q[b], Q[c]
        e1 = [B[k] - A[k] for k in range(3)]
        e2 = [C[k] - A[k] for k in range(3)]
        n = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]]
        faces.append((A, n))  # outward normal for the outward-oriented mesh
    nz, ny, nx = sub.shape
    checked = 0
    for az in range(nz):
        for ay in range(ny):
            for ax in range(nx):
                P = [256 * ax + 128, 256 * ay + 128, 256 * az + 128]
                d = [sum(n[k] * (P[k] - A[k]) for k in range(3)) for A, n in faces]
                if any(x == 0 for x in d):
                    continue
                assert sub[az, ay, ax] == (1 if all(x < 0 for x in d) else 0), (az, ay, ax)
                checked += 1
    assert checked > 0.99 * nz * ny * nx and sub.sum() > 100


@pytest.mark.parametrize("s", [1, 2])
def test_sphere_mesh_volume(oracle_mod, s):
    """Sum of sub-cell volumes vs the polyhedron's volume (divergence theorem),
    within area x half the sub-cell diagonal."""
    v, t = W.icosphere(5.0, 2)
    sub, _ = oracle_mod.voxelize_mesh(v, t, s)
    V = v.astype(np.float64)
    vol = sum(np.dot(V[a], np.cross(V[b], V[c])) for a, b, c in t) / 6.0
    area = sum(0.5 * np.linalg.norm(np.cross(V[b] - V[a], V[c] - V[a])) for a, b, c in t)
    got = sub.sum() * 8.0 ** -s
    assert abs(got - vol) <= area * 0.5 * math.sqrt(3) * 2.0 ** -s
    assert abs(got - vol) / vol < 0.05
