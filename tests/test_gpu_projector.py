"""GPU parity of the Siddon projector against the FP64 oracle, through the C ABI.

Element-by-element comparison on seeded inputs at sizes the oracle finishes in
seconds (several CTA tiles, ragged tails), sampled rays / voxels at the
config-2 size in the bench's launch configuration, the FP32 adjoint test, the
update count, storage dtypes, batches and block selections.
"""
import numpy as np
import pytest

from helpers import (fp_tolerance, gpu_geom, oracle_geom, rel_l2, rows_of_blocks, spec, col_range)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import projector as P  # noqa: E402
from paper_1903_11874_gb300 import binding as B  # noqa: E402
from paper_1903_11874_gb300 import synth  # noqa: E402

DEV = "cuda:0"
SMALL = ["config1", "paper2d", "cone_small"]


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def _nmax(s):
    return 2 * (s["nx"] + s["ny"] + s["nz"])


@pytest.mark.parametrize("name", SMALL)
def test_forward_projection_matches_oracle(name):
    s = spec(name)
    og, gg = oracle_geom(s), gpu_geom(s)
    x = synth.uniform_array(og.n_cols, 11)
    y = torch.zeros(og.n_rows, device=DEV)
    B.bsgd_forward_project(gg, _cuda(x), y)
    ref = P.fp(og, x).reshape(-1)
    tol = fp_tolerance(P.fp(og, np.abs(x)).reshape(-1), _nmax(s))
    got = y.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) - tol)
    assert rel_l2(got, ref) < 1e-5


@pytest.mark.parametrize("name", SMALL)
def test_back_projection_matches_oracle(name):
    s = spec(name)
    og, gg = oracle_geom(s), gpu_geom(s)
    r = synth.normal_array(og.n_rows, 12)
    x = torch.zeros(og.n_cols, device=DEV)
    B.bsgd_back_project(gg, _cuda(r), x)
    ref = P.bp(og, r).reshape(-1)
    tol = fp_tolerance(P.bp(og, np.abs(r)).reshape(-1), _nmax(s))
    got = x.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) - tol)
    assert rel_l2(got, ref) < 1e-5


@pytest.mark.parametrize("name", SMALL + ["config2"])
def test_adjoint_identity_fp32(name):
    """<A x, r> = <x, A^T r> for the FP32 kernels (target 1e-6 relative)."""
    s = spec(name)
    gg = gpu_geom(s)
    x = _cuda(synth.uniform_array(gg.n_cols, 1, dtype=np.float32))
    r = _cuda(synth.normal_array(gg.n_rows, 2, dtype=np.float32))
    ax = torch.zeros(gg.n_rows, device=DEV)
    atr = torch.zeros(gg.n_cols, device=DEV)
    B.bsgd_forward_project(gg, x, ax)
    B.bsgd_back_project(gg, r, atr)
    lhs = float(torch.dot(ax.double(), r.double()))
    rhs = float(torch.dot(x.double(), atr.double()))
    scale = float(torch.dot(ax.double().abs(), r.double().abs()))
    assert abs(lhs - rhs) <= 1e-6 * scale


@pytest.mark.parametrize("name", ["config1", "cone_small"])
def test_block_restricted_projection(name):
    """A_S^B x over a subset of row blocks and a contiguous run of column
    blocks; rows outside S untouched, voxels outside B untouched."""
    s = spec(name)
    og, gg = oracle_geom(s), gpu_geom(s)
    M, N = s["M"], s["N"]
    rb, cb = [1, 3], [1, 2]
    x = synth.uniform_array(og.n_cols, 4)
    y = torch.full((og.n_rows,), 7.0, device=DEV)
    B.bsgd_forward_project(gg, _cuda(x), y, row_blocks=rb, col_blocks=cb)
    rows = rows_of_blocks(og, M, rb)
    blk = col_range(og, N, cb)
    ref = P.fp_rows(og, x, rows, blk)
    got = y.cpu().double().numpy()
    tol = fp_tolerance(P.fp_rows(og, np.abs(x), rows, blk), _nmax(s))
    assert np.all(np.abs(got[rows] - ref) <= tol)
    others = np.setdiff1d(np.arange(og.n_rows), rows)
    assert np.all(got[others] == 7.0)
    # BP into the same blocks, accumulate onto existing values
    r = synth.normal_array(og.n_rows, 5)
    base = synth.uniform_array(og.n_cols, 6)
    xg = _cuda(base)
    B.bsgd_back_project(gg, _cuda(r), xg, row_blocks=rb, col_blocks=cb, scale=0.5, accumulate=True)
    refb = base + 0.5 * P.bp_rows(og, r[rows], rows, blk)
    tolb = 0.5 * fp_tolerance(P.bp_rows(og, np.abs(r[rows]), rows, blk), _nmax(s)) + 1e-6
    assert np.all(np.abs(xg.cpu().double().numpy() - refb) <= tolb)


@pytest.mark.parametrize("name", SMALL)
def test_update_count_matches_oracle(name):
    s = spec(name)
    og, gg = oracle_geom(s), gpu_geom(s)
    for rb, cb in [(None, None), ([0], [1])]:
        n_gpu = B.bsgd_count_updates(gg, row_blocks=rb, col_blocks=cb)
        rows = np.arange(og.n_rows) if rb is None else rows_of_blocks(og, s["M"], rb)
        blk = None if cb is None else col_range(og, s["N"], cb)
        n_orc = P.count_rows(og, rows, blk)
        # both sides skip edge / corner slivers (< 1e-4 voxel); a true piece
        # within FP32 rounding of that threshold may still flip
        assert abs(n_gpu - n_orc) <= 1e-5 * n_orc + 2


@pytest.mark.parametrize("xt,yt", [(torch.bfloat16, torch.float32), (torch.float16, torch.float32),
                                   (torch.float32, torch.bfloat16)])
def test_storage_dtypes(xt, yt):
    s = spec("cone_small")
    og, gg = oracle_geom(s), gpu_geom(s)
    xg = _cuda(synth.uniform_array(og.n_cols, 7), xt)
    x = xg.float().cpu().double().numpy()            # the values the kernel reads
    y = torch.zeros(og.n_rows, device=DEV, dtype=yt)
    B.bsgd_forward_project(gg, xg, y)
    ref = P.fp(og, x).reshape(-1)
    tol = fp_tolerance(P.fp(og, np.abs(x)).reshape(-1), _nmax(s))
    if yt != torch.float32:                           # one output rounding
        tol = tol + np.abs(ref) * 2.0 ** -8
    assert np.all(np.abs(y.float().cpu().double().numpy() - ref) <= tol)


def test_batch_equals_single():
    s = spec("cone_small")
    gg = gpu_geom(s)
    xs = _cuda(synth.uniform_array((3, gg.n_cols), 8))
    yb = torch.zeros(3, gg.n_rows, device=DEV)
    B.bsgd_forward_project(gg, xs, yb, batch=3)
    for b in range(3):
        y1 = torch.zeros(gg.n_rows, device=DEV)
        B.bsgd_forward_project(gg, xs[b].contiguous(), y1)
        assert torch.equal(y1, yb[b])
    rb = torch.zeros(3, gg.n_cols, device=DEV)
    B.bsgd_back_project(gg, yb, rb, batch=3)
    r1 = torch.zeros(gg.n_cols, device=DEV)
    B.bsgd_back_project(gg, yb[1].contiguous(), r1)
    assert torch.allclose(r1, rb[1], rtol=1e-5, atol=1e-5 * float(r1.abs().max()))


def test_config2_sampled_rays_and_voxels():
    """Config-2 size (256^3, 360 x 256^2) in the solver's launch shape: one
    (row block, z-slab) pair. FP on 400 sampled rays and BP of the pair on
    every voxel of the slab against the oracle."""
    s = spec("config2")
    og, gg = oracle_geom(s), gpu_geom(s)
    x = synth.ellipsoid_phantom(256, 256, 256, 10, seed=0).reshape(-1).astype(np.float64) * 0.01
    i, j = 3, 5
    y = torch.zeros(og.n_rows, device=DEV)
    B.bsgd_forward_project(gg, _cuda(x), y, row_blocks=[i], col_blocks=[j])
    rows = rows_of_blocks(og, 8, [i])
    rng = np.random.default_rng(3)
    pick = rows[rng.choice(rows.size, 400, replace=False)]
    blk = P.column_block(og, 8, j)
    ref = P.fp_rows(og, x, pick, blk)
    tol = fp_tolerance(P.fp_rows(og, np.abs(x), pick, blk), _nmax(s))
    got = y.cpu().double().numpy()[pick]
    assert np.all(np.abs(got - ref) <= tol)
    # BP of a seeded residual over the pair (the whole slab)
    r = synth.normal_array(og.n_rows, 9).astype(np.float32).astype(np.float64)
    xg = torch.zeros(og.n_cols, device=DEV)
    B.bsgd_back_project(gg, _cuda(r), xg, row_blocks=[i], col_blocks=[j])
    vox = P.column_block_voxels(og, 8, j)
    refb = P.bp_rows(og, r[rows], rows, blk)[vox]
    tolb = fp_tolerance(P.bp_rows(og, np.abs(r[rows]), rows, blk)[vox], _nmax(s))
    gotb = xg.cpu().double().numpy()[vox]
    assert np.all(np.abs(gotb - refb) <= tolb)
    # zero-mean noise: every (ray, voxel) length carries the FP32 rounding of
    # the ray's own geometry (the source sits ~630 voxels from the volume
    # corner: ~6e-8 * 630 ~ 4e-5 voxel), and the signed terms do not telescope,
    # so rel-L2 ~ 4e-5 / (mean segment ~0.7) ~ 6e-5; bound 1e-4
    assert rel_l2(gotb, refb) < 1e-4


def test_fp_is_deterministic_and_bp_within_rounding():
    """The FP of a ray is one thread's fixed-order sum: two runs agree bit for
    bit (also through the solver's fused pass). The BP scatters with float
    atomics whose order varies: two runs agree to FP32 rounding."""
    s = spec("cone_small")
    gg = gpu_geom(s)
    x = _cuda(synth.uniform_array(gg.n_cols, 31))
    r = _cuda(synth.normal_array(gg.n_rows, 32))
    ys = []
    for _ in range(2):
        y = torch.zeros(gg.n_rows, device=DEV)
        B.bsgd_forward_project(gg, x, y)
        ys.append(y)
    assert torch.equal(ys[0], ys[1])
    bs = []
    for _ in range(2):
        b = torch.zeros(gg.n_cols, device=DEV)
        B.bsgd_back_project(gg, r, b)
        bs.append(b.double())
    scale = float(bs[0].abs().max())
    assert float((bs[0] - bs[1]).abs().max()) <= 1e-5 * scale
