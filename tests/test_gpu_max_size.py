"""The largest workload (Table 1 case 3: 1024^3 voxels, 360 x 2000^2 rays) on
the GPU projector: A 1 on sampled rays equals the ray's chord through the
volume box (slab method, FP64), a closed form. At this size the flat voxel
index passes 2^30 and the row index 2^30, so the test guards the index
arithmetic as well as the traversal."""
import math

import numpy as np
import pytest

from helpers import fp_tolerance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1903_11874_gb300 import binding as B  # noqa: E402


def chord(p0, p1, lo, hi):
    d = p1 - p0
    t0, t1 = 0.0, 1.0
    for k in range(3):
        a, b = (lo[k] - p0[k]) / d[k], (hi[k] - p0[k]) / d[k]
        t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
    return max(0.0, t1 - t0) * float(np.linalg.norm(d))


def test_case3_total_chords():
    n, nd, V = 1024, 2000, 360
    h, p, dso, dsd = 256.0 / n, 400.0 / nd, 1536.0, 2536.0
    gg = B.Geometry(M=1, N=1, kind="cone3d", nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, n_views=V, nu=nd,
                    nv=nd, du=p, dv=p, dso=dso, dsd=dsd)
    assert gg.n_rows == V * nd * nd and gg.n_cols == n ** 3
    x = torch.ones(gg.n_cols, device="cuda:0")
    y = torch.zeros(gg.n_rows, device="cuda:0")
    B.bsgd_forward_project(gg, x, y)
    del x
    rng = np.random.default_rng(11)
    rows = np.unique(rng.integers(0, gg.n_rows, 20000))
    rows = np.concatenate([rows, [0, gg.n_rows - 1, gg.n_rows // 2]])
    got = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    lo, hi = -np.full(3, 128.0), np.full(3, 128.0)
    ref = np.empty(rows.size)
    for k, row in enumerate(rows):
        a, rem = divmod(int(row), nd * nd)
        v, u = divmod(rem, nd)
        b = a * 2 * math.pi / V
        er = np.array([math.cos(b), math.sin(b), 0.0])
        eu = np.array([-math.sin(b), math.cos(b), 0.0])
        src = dso * er
        det = -(dsd - dso) * er + (u - (nd - 1) / 2) * p * eu + np.array([0.0, 0.0, (v - (nd - 1) / 2) * p])
        ref[k] = chord(src, det, lo, hi)
    assert (ref > 0).sum() > 0.5 * rows.size        # most sampled rays meet the volume
    tol = fp_tolerance(ref, 3 * n)
    assert np.all(np.abs(got - ref) <= tol)
