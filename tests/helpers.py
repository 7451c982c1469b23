"""Shared test helpers: one geometry spec feeds both the CUDA library and the
oracle (each builds its own tables from it)."""
import math

import numpy as np

SPECS = {
    # config-1 workload: 64^2 image, 90 parallel views over 180 deg, 96 unit bins
    "config1": dict(kind="par2d", nx=64, ny=64, nz=1, dx=1.0, dy=1.0, dz=1.0, n_views=90,
                    nu=96, nv=1, du=1.0, dv=1.0, M=4, N=4),
    # Sec. 3.1 set-up: fan beam, 16^2, OP = OD = 50, 30 unit elements, 10 deg steps
    "paper2d": dict(kind="fan2d", nx=16, ny=16, nz=1, dx=1.0, dy=1.0, dz=1.0, n_views=36,
                    nu=30, nv=1, du=1.0, dv=1.0, dso=50.0, dsd=100.0, M=4, N=2),
    # small cone beam spanning several CTA tiles with ragged tails in u and v
    # (angles offset by 0.05 rad: no ray lies in an x or y face; the odd detector's
    # centre row lies exactly in the z = 0 face on both sides)
    "cone_small": dict(kind="cone3d", nx=40, ny=36, nz=32, dx=1.0, dy=1.0, dz=1.0, n_views=24,
                       nu=45, nv=37, du=1.6, dv=1.6, dso=120.0, dsd=240.0, M=4, N=4,
                       angles=0.05 + np.arange(24) * (2 * math.pi / 24)),
    # degenerate cone beam: views at exact multiples of 45 deg (rays in voxel
    # faces, x / y crossing ties), even volume sides (the central rays lie in
    # the x = 0, y = 0 and z = 0 faces), a detector wider and taller than the
    # volume's shadow (rays that miss), one view per row block and one slice per
    # column block
    "cone_axes": dict(kind="cone3d", nx=24, ny=20, nz=16, dx=1.0, dy=1.0, dz=1.0, n_views=8,
                      nu=41, nv=33, du=1.6, dv=1.6, dso=60.0, dsd=120.0, M=8, N=16,
                      angles=np.arange(8) * (math.pi / 4)),
    # parallel beam whose bins all lie in pixel faces at 0 and 90 deg: unit
    # bins at integer offsets, including the two outer faces y = +-8 (the + side
    # convention puts the lower one inside, the upper one outside) and the
    # boundaries between the 4-row column blocks
    "par_faces": dict(kind="par2d", nx=16, ny=16, nz=1, dx=1.0, dy=1.0, dz=1.0, n_views=4,
                      nu=19, nv=1, du=1.0, dv=1.0, M=2, N=4,
                      angles=np.arange(4) * (math.pi / 4)),
    # the solver's block-count limits: M = 64 row blocks (one view each) and
    # M x N = 1024 residual-weighted pairs
    "limits": dict(kind="cone3d", nx=16, ny=16, nz=16, dx=1.0, dy=1.0, dz=1.0, n_views=64,
                   nu=21, nv=19, du=1.3, dv=1.3, dso=60.0, dsd=120.0, M=64, N=16),
    # Sec. 5, Table 1 case 1: 256^3 (1 mm), 360 views at 1 deg, 400^2 detector of
    # 1 mm, source 1536 mm / detector 1000 mm from the centre; M = 5 groups of 72
    # views (a seeded random partition, as in Sec. 5), N = 8
    "paper_case1": dict(kind="cone3d", nx=256, ny=256, nz=256, dx=1.0, dy=1.0, dz=1.0,
                        n_views=360, nu=400, nv=400, du=1.0, dv=1.0, dso=1536.0, dsd=2536.0,
                        M=5, N=8),
    # config-2 workload: 256^3, 360 views, 256^2 detector at 1.6 mm, DSO 500 / DSD 1000
    "config2": dict(kind="cone3d", nx=256, ny=256, nz=256, dx=1.0, dy=1.0, dz=1.0,
                    n_views=360, nu=256, nv=256, du=1.6, dv=1.6, dso=500.0, dsd=1000.0, M=8, N=8),
}


def paper_partition(seed=5):
    """360 views in 5 equal random groups (Sec. 5's random partition)."""
    vb = np.repeat(np.arange(5, dtype=np.int32), 72)
    np.random.default_rng(seed).shuffle(vb)
    return vb


def spec(name, **over):
    s = dict(SPECS[name])
    s.update(over)
    return s


def oracle_geom(s):
    from oracle import projector as P
    kw = {k: v for k, v in s.items() if k not in ("M", "N", "view_block")}
    return P.Geometry(**kw)


def gpu_geom(s):
    from paper_1903_11874_gb300 import binding as B
    return B.Geometry(**s)


def rows_of_blocks(og, M, blocks):
    from oracle import projector as P
    views = np.concatenate([P.row_block_views(og, M, i) for i in blocks])
    return P.rows_of_views(og, np.sort(views))


def col_range(og, N, blocks):
    from oracle import projector as P
    blocks = sorted(blocks)
    assert blocks == list(range(blocks[0], blocks[-1] + 1))
    return P.column_block(og, N, blocks[0])[0], P.column_block(og, N, blocks[-1])[1]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# FP32 error model of one ray sum z = L sum_k s_k x_k:
# every crossing parameter is within a few ulps of the chord, so each segment
# carries an absolute length error of order 4 u T (T = chord, u = 2^-24) and
# the FP32 accumulation adds at most n u sum |s_k x_k|. With n <= 2 nx the
# per-ray bound is |dz| <= (8 n u) * (A |x|)_row; a ray-independent floor
# covers segments split differently at exact ties.
U32 = 2.0 ** -24


def fp_tolerance(abs_proj, n_max):
    return 8.0 * n_max * U32 * abs_proj + 1e-6 * float(np.max(abs_proj) + 1e-30)


def angle_list(n, span, off=0.0):
    return off + np.arange(n) * (span / n)


def uniform_angles(kind, n):
    return angle_list(n, math.pi if kind == "par2d" else 2 * math.pi)
