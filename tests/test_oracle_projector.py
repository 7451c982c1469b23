"""Pins of the FP64 oracle projector (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: hand-derived chords, the total chord through a box or a voxel (closed
form), the adjoint identity, the block partition of Eq. 3, a rotation symmetry,
the magnification of a point's shadow, and the matrix sizes the paper prints.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import projector as P
from paper_1903_11874_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- independent helpers written for the tests --------------------------------

def ray_points(geom, a, v, u):
    """Ray end points from the stated conventions (re-derived here)."""
    th = geom.angles[a]
    uc = (u - (geom.nu - 1) / 2.0) * geom.du
    vc = (v - (geom.nv - 1) / 2.0) * geom.dv
    er = np.array([math.cos(th), math.sin(th), 0.0])
    eu = np.array([-math.sin(th), math.cos(th), 0.0])
    if geom.kind == "par2d":
        far = 10.0 * (geom.nx * geom.dx + geom.ny * geom.dy)
        base = uc * eu
        return base - far * er, base + far * er
    src = geom.dso * er
    det = -(geom.dsd - geom.dso) * er + uc * eu + np.array([0.0, 0.0, vc])
    return src, det


def box_chord(p0, p1, lo, hi):
    """Length of segment p0-p1 inside the axis-aligned box [lo, hi] (slab clip)."""
    d = p1 - p0
    t0, t1 = 0.0, 1.0
    for k in range(3):
        if abs(d[k]) < 1e-300:
            # a ray lying in a face belongs to the voxel above it (half-open)
            if p0[k] < lo[k] or p0[k] >= hi[k]:
                return 0.0
            continue
        a, b = (lo[k] - p0[k]) / d[k], (hi[k] - p0[k]) / d[k]
        t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
    return max(0.0, t1 - t0) * float(np.linalg.norm(d))


def lies_in_face(p0, p1, lo, hi):
    """Ray parallel to an axis and (within rounding) inside one of the box's
    faces: ownership there is a convention, pinned separately."""
    d = p1 - p0
    nd = float(np.linalg.norm(d))
    for k in range(3):
        if abs(d[k]) <= 1e-12 * nd and min(abs(p0[k] - lo[k]), abs(p0[k] - hi[k])) < 1e-9:
            return True
    return False


def vol_box(geom):
    h = np.array([geom.nx * geom.dx, geom.ny * geom.dy, geom.nz * geom.dz]) / 2.0
    return -h, h


def _angles(n, span, off=0.1):
    # offset keeps every ray clear of voxel faces (ownership there is rounding)
    return off + np.arange(n) * (span / n)


def small_geoms():
    return [
        P.Geometry("par2d", 12, 10, 1, 1.0, 1.3, 1.0, 7, 17, 1, 0.9, 1.0,
                   angles=_angles(7, math.pi)),
        P.Geometry("fan2d", 11, 13, 1, 1.1, 0.9, 1.0, 9, 19, 1, 1.7, 1.0, dso=40.0, dsd=85.0,
                   angles=_angles(9, 2 * math.pi)),
        P.Geometry("cone3d", 9, 8, 7, 1.0, 1.2, 0.8, 6, 13, 11, 1.9, 1.5, dso=30.0, dsd=60.0,
                   angles=_angles(6, 2 * math.pi)),
    ]


# ---- pins ---------------------------------------------------------------------

def test_hand_derived_2x2_chords():
    gold = json.load(open(os.path.join(GOLDEN, "chords_2x2_par2d.json")))
    a = math.sqrt(2.0) - 1.0
    expect = np.array([[a if s == "a" else float(s) for s in row] for row in gold["rows"]])
    geom = P.Geometry("par2d", 2, 2, 1, 1.0, 1.0, 1.0, 4, 2, 1, 1.0, 1.0,
                      angles=np.deg2rad(np.array(gold["angles_deg"], dtype=np.float64)))
    A = P.dense_matrix(geom)
    np.testing.assert_allclose(A, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("gi", range(3))
def test_total_chord_through_volume_box(gi):
    geom = small_geoms()[gi]
    ones = np.ones(geom.n_cols)
    y = P.fp(geom, ones).reshape(-1)
    lo, hi = vol_box(geom)
    k = 0
    for a in range(geom.n_views):
        for v in range(geom.nv):
            for u in range(geom.nu):
                p0, p1 = ray_points(geom, a, v, u)
                assert abs(y[k] - box_chord(p0, p1, lo, hi)) <= 1e-10 * (1 + abs(y[k]))
                k += 1


@pytest.mark.parametrize("gi", range(3))
def test_single_voxel_chords(gi):
    geom = small_geoms()[gi]
    rng = np.random.default_rng(5)
    lo, _ = vol_box(geom)
    h = np.array([geom.dx, geom.dy, geom.dz])
    for vox in rng.choice(geom.n_cols, size=6, replace=False):
        ix, iy, iz = vox % geom.nx, (vox // geom.nx) % geom.ny, vox // (geom.nx * geom.ny)
        vlo = lo + np.array([ix, iy, iz]) * h
        e = np.zeros(geom.n_cols)
        e[vox] = 1.0
        y = P.fp(geom, e).reshape(-1)
        k = 0
        for a in range(geom.n_views):
            for v in range(geom.nv):
                for u in range(geom.nu):
                    p0, p1 = ray_points(geom, a, v, u)
                    if not lies_in_face(p0, p1, vlo, vlo + h):
                        assert abs(y[k] - box_chord(p0, p1, vlo, vlo + h)) <= 1e-10
                    k += 1


def test_ray_in_a_face_belongs_to_the_voxel_above():
    """Reading of the paper's silence on ties: a ray lying exactly in a voxel
    face is owned by the voxel on the + side (half-open voxels)."""
    geom = P.Geometry("par2d", 4, 4, 1, 1.0, 1.0, 1.0, 2, 3, 1, 1.0, 1.0,
                      angles=np.array([0.0, 0.5 * math.pi]))
    A = P.dense_matrix(geom).reshape(2, 3, 4, 4)
    # view 0: rays along +x at y = -1, 0, 1 lie in faces between pixel rows
    for u, y in enumerate((-1, 0, 1)):
        expect = np.zeros((4, 4))
        expect[y + 2, :] = 1.0
        np.testing.assert_allclose(A[0, u], expect, rtol=0, atol=1e-12)
    # view 1 (90 deg, axis-aligned exactly): rays along +y at x = 1, 0, -1 lie
    # in faces between pixel columns
    for u, x in enumerate((1, 0, -1)):
        expect = np.zeros((4, 4))
        expect[:, x + 2] = 1.0
        np.testing.assert_allclose(A[1, u], expect, rtol=0, atol=1e-12)


def test_axis_aligned_view_angles_are_exact():
    """Angles within 1e-9 rad of a multiple of 90 deg give exact axis
    directions (double cos(pi / 2) is 6e-17); other angles are untouched."""
    for k in range(-4, 9):
        c, s = P.view_cos_sin(k * (math.pi / 2))
        assert (c, s) == ((1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0))[k % 4]
    t = 2 * math.pi * 90 / 360
    assert P.view_cos_sin(t) == (0.0, 1.0)
    for t in (1e-6, math.pi / 2 + 1e-6, 0.3, -2.0):
        assert P.view_cos_sin(t) == (math.cos(t), math.sin(t))
    # the C traversal applies the same rule: a 90-deg cone view whose central
    # column lies in the x = 0 face puts the whole ray into the + side column
    geom = P.Geometry("cone3d", 4, 4, 2, 1.0, 1.0, 1.0, 1, 3, 3, 1.0, 1.0, dso=10.0, dsd=20.0,
                      angles=np.array([2 * math.pi * 90 / 360]))
    A = P.dense_matrix(geom).reshape(3, 3, 2, 4, 4)
    col = A[1, 1]                      # centre pixel: the ray x = 0, z = 0 along -y
    expect = np.zeros((2, 4, 4))
    expect[1, :, 2] = 1.0              # + side in x (column 2) and in z (slice 1)
    np.testing.assert_allclose(col, expect, rtol=0, atol=1e-12)


def test_disc_chords_converge_first_order():
    """Uniform disc of radius R: a ray at distance s from the centre sees a
    chord 2 sqrt(R^2 - s^2); the pixelised disc's error shrinks with the pixel."""
    errs = []
    for n in (32, 64, 128):
        d = 2.0 / n
        c = (np.arange(n) + 0.5) * d - 1.0
        X, Y = np.meshgrid(c, c, indexing="xy")
        disc = (X ** 2 + Y ** 2 <= 0.7 ** 2).astype(np.float64)
        geom = P.Geometry("par2d", n, n, 1, d, d, 1.0, 8, 41, 1, 0.03, 1.0)
        y = P.fp(geom, disc.reshape(-1))[:, 0, :]
        s = (np.arange(41) - 20) * 0.03
        exact = 2.0 * np.sqrt(np.maximum(0.49 - s ** 2, 0.0))
        errs.append(np.abs(y - exact[None, :]).mean())
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]
    assert errs[2] < 0.02


@pytest.mark.parametrize("gi", range(3))
def test_adjoint_identity(gi):
    geom = small_geoms()[gi]
    x = synth.normal_array(geom.n_cols, 1)
    r = synth.normal_array(geom.n_rows, 2)
    ax = P.fp(geom, x).reshape(-1)
    atr = P.bp(geom, r).reshape(-1)
    lhs, rhs = float(ax @ r), float(x @ atr)
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.abs(ax).sum() * np.abs(r).max())
    # every sub-block A_I^J of a 3 x 2 partition as well
    M, N = 3, 2
    for i in range(M):
        views = P.row_block_views(geom, M, i)
        for j in range(N):
            blk = P.column_block(geom, N, j)
            ax = P.fp(geom, x, views, blk).reshape(-1)
            atr = P.bp(geom, r, views, blk).reshape(-1)
            lhs, rhs = float(ax @ r), float(x @ atr)
            assert abs(lhs - rhs) <= 1e-12 * (1.0 + np.abs(ax).sum() * np.abs(r).max())


@pytest.mark.parametrize("gi", range(3))
def test_dense_matrix_columns_equal_rows(gi):
    """A built column by column from FP of unit vectors equals A built row by
    row from BP of unit residuals and A assembled from single-ray traces."""
    geom = small_geoms()[gi]
    A = P.dense_matrix(geom)
    cols = np.stack([P.fp(geom, np.eye(1, geom.n_cols, j).reshape(-1)).reshape(-1)
                     for j in range(0, geom.n_cols, 7)], axis=1)
    np.testing.assert_allclose(A[:, ::7], cols, rtol=0, atol=1e-12)
    rows = np.stack([P.bp(geom, np.eye(1, geom.n_rows, i).reshape(-1)).reshape(-1)
                     for i in range(0, geom.n_rows, 11)], axis=0)
    np.testing.assert_allclose(A[::11, :], rows, rtol=0, atol=1e-12)
    assert (A >= 0).all()                                 # Sec. 1: non-negative entries
    hmin = min(geom.dx, geom.dy, geom.dz)
    assert P.count_rows(geom, np.arange(geom.n_rows)) == int((A > 1e-4 * hmin).sum())


@pytest.mark.parametrize("gi", range(3))
def test_block_partition_sums(gi):
    """Eq. 3: A_I x = sum_j A_I^{J_j} x_{J_j} and the row blocks tile y."""
    geom = small_geoms()[gi]
    x = synth.uniform_array(geom.n_cols, 3)
    full = P.fp(geom, x)
    M, N = 4, 3
    acc = np.zeros_like(full)
    for j in range(N):
        for i in range(M):
            acc += P.fp(geom, x, P.row_block_views(geom, M, i), P.column_block(geom, N, j))
    np.testing.assert_allclose(acc, full, rtol=1e-13, atol=1e-12)
    views = np.concatenate([P.row_block_views(geom, M, i) for i in range(M)])
    assert sorted(views.tolist()) == list(range(geom.n_views))


def test_parallel_rotation_symmetry():
    """Rotating the image by +90 degrees shifts the parallel-beam views by 90
    degrees (and flips the detector when the shift wraps past 180)."""
    n, nv = 16, 36
    # 24 bins of 0.7: no ray lies in a pixel face (ownership there is not
    # rotation invariant)
    geom = P.Geometry("par2d", n, n, 1, 1.0, 1.0, 1.0, nv, 24, 1, 0.7, 1.0)
    f = synth.uniform_array((n, n), 7)
    g = f[::-1, :].T                                     # g(p) = f(R^-1 p), R = +90 deg
    pf = P.fp(geom, f.reshape(-1))[:, 0, :]
    pg = P.fp(geom, g.reshape(-1))[:, 0, :]
    q = nv // 2
    for a in range(nv):
        if a < q:
            np.testing.assert_allclose(pg[a + q], pf[a], rtol=1e-11, atol=1e-11)
        else:
            np.testing.assert_allclose(pg[a - q][::-1], pf[a], rtol=1e-11, atol=1e-11)


def test_cone_point_shadow_position():
    """A voxel's shadow falls where the magnification says: detector
    u = dsd (X . e_u) / (dso - X . e_r), v = dsd X_z / (dso - X . e_r)."""
    geom = P.Geometry("cone3d", 16, 16, 16, 1.0, 1.0, 1.0, 8, 64, 64, 0.5, 0.5, dso=60.0, dsd=110.0)
    ix, iy, iz = 12, 4, 13
    X = np.array([ix - 7.5, iy - 7.5, iz - 7.5])
    e = np.zeros(geom.n_cols)
    e[(iz * 16 + iy) * 16 + ix] = 1.0
    y = P.fp(geom, e)
    for a in range(geom.n_views):
        th = geom.angles[a]
        er = np.array([math.cos(th), math.sin(th), 0.0])
        eu = np.array([-math.sin(th), math.cos(th), 0.0])
        mag = geom.dsd / (geom.dso - X @ er)
        u_exp = mag * (X @ eu) / geom.du + (geom.nu - 1) / 2.0
        v_exp = mag * X[2] / geom.dv + (geom.nv - 1) / 2.0
        img = y[a]
        vv, uu = np.nonzero(img)
        w = img[vv, uu]
        assert abs((uu * w).sum() / w.sum() - u_exp) < 0.6
        assert abs((vv * w).sum() / w.sum() - v_exp) < 0.6


def _matches_printed(value, printed: str) -> bool:
    """value rounds to the printed number (half a unit of its last digit)."""
    mant, _, exp = printed.partition("e")
    decimals = len(mant.partition(".")[2])
    half_ulp = 0.5 * 10.0 ** (int(exp or 0) - decimals)
    return abs(value - float(printed)) <= half_ulp


def test_paper_matrix_sizes():
    gold = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    for case in gold["cases"]:
        vol = case.get("volume") or case["image"] + [1]
        det = case["detector"]
        kind = case["kind"]
        geom = P.Geometry(kind, vol[0], vol[1], vol[2], 1.0, 1.0, 1.0, case["views"],
                          det[0], det[1], 1.0, 1.0, dso=1000.0, dsd=1500.0)
        assert _matches_printed(geom.n_rows, case["rows"]), case["cite"]
        assert _matches_printed(geom.n_cols, case["cols"]), case["cite"]


@pytest.mark.parametrize("gi", [1, 2])
def test_v_band_contains_every_hit_row(gi):
    """Rows outside the detector band of a column block see none of it."""
    geom = small_geoms()[gi]
    N = 3 if geom.nz > 1 else 2
    for j in range(N):
        blk = P.column_block(geom, N, j)
        ind = np.zeros(geom.n_cols)
        ind[P.column_block_voxels(geom, N, j)] = 1.0
        y = P.fp(geom, ind, None, blk)
        for a in range(geom.n_views):
            lo, hi = P.v_band(geom, a, N, j)
            hit = np.nonzero(y[a].sum(axis=1) > 0)[0]
            if hit.size:
                assert lo <= hit.min() and hit.max() <= hi
