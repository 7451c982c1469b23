"""Degenerate inputs on the GPU path against the FP64 oracle: views at exact
multiples of 45 degrees (rays lying in voxel faces, tied x / y crossings),
rays that miss the volume, one view per row block and one slice per column
block, non-contiguous column-block lists, a zero sinogram, and calls that do
no work."""
import numpy as np
import pytest

from helpers import fp_tolerance, gpu_geom, oracle_geom, rel_l2, rows_of_blocks, spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bsgd as OB  # noqa: E402
from oracle import projector as P  # noqa: E402
from paper_1903_11874_gb300 import binding as B  # noqa: E402
from paper_1903_11874_gb300 import synth  # noqa: E402

DEV = "cuda:0"


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, torch.float32)


def _nmax(s):
    return 2 * (s["nx"] + s["ny"] + s["nz"])


def _geoms(name="cone_axes"):
    s = spec(name)
    return s, oracle_geom(s), gpu_geom(s)


@pytest.mark.parametrize("name", ["cone_axes", "par_faces"])
def test_axis_views_forward_and_back_projection(name):
    s, og, gg = _geoms(name)
    x = synth.uniform_array(og.n_cols, 21)
    y = torch.zeros(og.n_rows, device=DEV)
    B.bsgd_forward_project(gg, _cuda(x), y)
    ref = P.fp(og, x).reshape(-1)
    tol = fp_tolerance(P.fp(og, np.abs(x)).reshape(-1), _nmax(s))
    got = y.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) - tol)
    # the detector overhangs the volume's shadow: some rays meet nothing
    chords = P.fp(og, np.ones(og.n_cols)).reshape(-1)
    if name == "cone_axes":
        assert (chords == 0).sum() > 0.1 * og.n_rows
    else:
        # view 0: bins 1..16 (y = -8 .. 7) each own one full pixel row, the
        # bins at y = 8 and 9 and y = -9 miss
        np.testing.assert_allclose(chords[:19], [0] + [16] * 16 + [0, 0], rtol=0, atol=1e-12)
        assert np.all(np.abs(got[:19][chords[:19] == 0]) == 0)
    assert np.all(np.abs(got[chords == 0]) <= tol[chords == 0])
    r = synth.normal_array(og.n_rows, 22)
    xb = torch.zeros(og.n_cols, device=DEV)
    B.bsgd_back_project(gg, _cuda(r), xb)
    refb = P.bp(og, r).reshape(-1)
    tolb = fp_tolerance(P.bp(og, np.abs(r)).reshape(-1), _nmax(s))
    gotb = xb.cpu().double().numpy()
    assert np.all(np.abs(gotb - refb) <= tolb), np.max(np.abs(gotb - refb) - tolb)


def test_single_view_and_single_slice_blocks():
    """Row blocks of one view, column blocks of one slice, and a column-block
    list with two separate runs ([2, 3] and [9]) given out of order."""
    s, og, gg = _geoms()
    M, N = s["M"], s["N"]
    x = synth.uniform_array(og.n_cols, 23)
    rb, cb = [6, 0, 3], [9, 3, 2]
    y = torch.full((og.n_rows,), -1.0, device=DEV)
    B.bsgd_forward_project(gg, _cuda(x), y, row_blocks=rb, col_blocks=cb)
    got = y.cpu().double().numpy()
    rows = rows_of_blocks(og, M, sorted(rb))
    ref = np.zeros(rows.size)
    tol = np.zeros(rows.size)
    for blocks in ([2, 3], [9]):
        lo, hi = P.column_block(og, N, blocks[0])[0], P.column_block(og, N, blocks[-1])[1]
        ref += P.fp_rows(og, x, rows, (lo, hi))
        tol += fp_tolerance(P.fp_rows(og, np.abs(x), rows, (lo, hi)), _nmax(s))
    assert np.all(np.abs(got[rows] - ref) <= tol)
    others = np.setdiff1d(np.arange(og.n_rows), rows)
    assert np.all(got[others] == -1.0)
    # BP of the same blocks: voxels outside the listed slices keep their value
    r = synth.normal_array(og.n_rows, 24)
    xb = torch.full((og.n_cols,), 5.0, device=DEV)
    B.bsgd_back_project(gg, _cuda(r), xb, row_blocks=rb, col_blocks=cb)
    gotb = xb.cpu().double().numpy()
    refb = np.full(og.n_cols, 5.0)
    inside = np.zeros(og.n_cols, bool)
    plane = og.nx * og.ny                      # column blocks are z-slabs
    for blocks in ([2, 3], [9]):
        lo, hi = P.column_block(og, N, blocks[0])[0], P.column_block(og, N, blocks[-1])[1]
        v0, v1 = lo * plane, hi * plane
        part = P.bp_rows(og, r[rows], rows, (lo, hi))
        refb[v0:v1] = part[v0:v1]
        inside[v0:v1] = True
        tolb = fp_tolerance(P.bp_rows(og, np.abs(r[rows]), rows, (lo, hi)), _nmax(s))[v0:v1]
        assert np.all(np.abs(gotb[v0:v1] - refb[v0:v1]) <= tolb)
    assert inside.sum() == 3 * plane
    assert np.all(gotb[~inside] == 5.0)


def test_update_count_with_face_rays():
    s, og, gg = _geoms()
    n_gpu = B.bsgd_count_updates(gg)
    n_orc = P.count_rows(og, np.arange(og.n_rows), None)
    assert abs(n_gpu - n_orc) <= 1e-5 * n_orc + 2


@pytest.mark.parametrize("name,epochs", [("cone_axes", 2), ("par_faces", 10)])
def test_trajectory_with_single_view_single_slice_blocks(name, epochs):
    """cone_axes: 128 pairs of (one view, one slice); par_faces: rays in
    pixel faces and on block boundaries. Uniform draws shared with the oracle
    by the sampling spec give the same image."""
    s, og, gg = _geoms(name)
    M, N = s["M"], s["N"]
    if og.nz > 1:
        xt = synth.ellipsoid_phantom(og.nx, og.ny, og.nz, 4, seed=3).astype(np.float64).reshape(-1)
    else:
        xt = synth.ellipse_phantom(og.nx, og.ny, 4, seed=3).reshape(-1)
    y = P.fp(og, xt).reshape(-1).astype(np.float32).astype(np.float64)
    mu = 0.25 * OB.step_strip(og, N, 1.0, 30)
    iters = epochs * M * N
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=9)
    st = B.State(gg, prm, _cuda(y))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, iters)
    torch.cuda.synchronize()
    ost = OB.bsgd(og, y, OB.Params(M, N, 1 / M, 1 / N, mu, seed=9), iters)
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-5
    assert st.query()["iteration"] == iters


@pytest.mark.parametrize("cells", [False, True])
def test_zero_sinogram_leaves_zero_image(cells):
    """y = 0 from x = 0: every residual and every BP weight is zero, the
    residual-weighted draw falls back on its floor, and the image stays
    exactly zero (no NaN from the zero weights)."""
    s, og, gg = _geoms()
    M, N = s["M"], s["N"]
    kw = dict(cells=B.CELLS_GEOMETRIC, n_cells=4) if cells else {}
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=1e-3, seed=2,
                        pair_sampling=B.PAIRS_RESIDUAL, **kw)
    st = B.State(gg, prm, torch.zeros(gg.n_rows, device=DEV))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, 3 * M * N)
    torch.cuda.synchronize()
    assert torch.count_nonzero(x).item() == 0
    q = st.query()
    assert q["residual_norm"] == 0.0 and q["iteration"] == 3 * M * N
    tr = st.read_trace(3 * M * N)
    assert np.all(tr[:, 0] == 1)
    assert np.all((tr[:, 1] >= 0) & (tr[:, 1] < M)) and np.all((tr[:, 2] >= 0) & (tr[:, 2] < N))


def test_calls_without_work():
    """Zero iterations, accumulate onto an existing sinogram with x = 0, and a
    BP of a zero residual change nothing."""
    s, og, gg = _geoms()
    M, N = s["M"], s["N"]
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=1e-3, seed=2)
    st = B.State(gg, prm, _cuda(synth.uniform_array(og.n_rows, 25)))
    x = _cuda(synth.uniform_array(og.n_cols, 26))
    x0 = x.clone()
    st.block_step(x, 0)
    torch.cuda.synchronize()
    assert torch.equal(x, x0) and st.query()["iteration"] == 0
    y0 = _cuda(synth.uniform_array(og.n_rows, 27))
    y = y0.clone()
    B.bsgd_forward_project(gg, torch.zeros(og.n_cols, device=DEV), y, accumulate=True)
    assert torch.equal(y, y0)
    B.bsgd_back_project(gg, torch.zeros(og.n_rows, device=DEV), x, accumulate=True)
    assert torch.equal(x, x0)


def test_block_count_limits():
    """M = 64 row blocks and M x N = 1024 pairs, the largest the device sampler
    takes: residual-weighted draws replayed by the oracle give the same image,
    and the oracle's own sampler agrees with the draws; then 64 pairs per
    iteration (alpha = 1/8, gamma = 1/2, uniform) against the oracle's
    trajectory."""
    s, og, gg = _geoms("limits")
    M, N = s["M"], s["N"]
    assert M * N == 1024
    xt = synth.ellipsoid_phantom(og.nx, og.ny, og.nz, 4, seed=5).astype(np.float64).reshape(-1)
    y = P.fp(og, xt).reshape(-1).astype(np.float32).astype(np.float64)
    mu = 0.25 * OB.step_strip(og, N, 1.0, 30)
    iters = 300
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=6,
                        pair_sampling=B.PAIRS_RESIDUAL)
    st = B.State(gg, prm, _cuda(y))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, iters)
    torch.cuda.synchronize()
    tr = st.read_trace(iters)
    po = OB.Params(M, N, 1 / M, 1 / N, mu, seed=6, pair_sampling="residual")
    ost = OB.BSGDState(og, y, po)
    agree = 0
    for t in tr:
        assert int(t[0]) == 1
        sel = OB.Selection([(int(t[1]), int(t[2]))], [None])
        agree += OB.sample(og, po, ost.it, ost.r, ost.bands, ost.cell_w).pairs == sel.pairs
        ost.step(sel)
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-5
    assert agree >= iters - 2
    # 8 x 8 = 64 pairs per iteration (the work list's capacity)
    kM, kN, iters = 8, 8, 12
    prm = B.SolveParams(alpha=kM / M, gamma=kN / N, step_rule=B.STEP_FIXED, mu=mu, seed=7)
    st = B.State(gg, prm, _cuda(y))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, iters)
    torch.cuda.synchronize()
    assert np.all(st.read_trace(iters)[:, 0] == kM * kN)
    ost = OB.bsgd(og, y, OB.Params(M, N, kM / M, kN / N, mu, seed=7), iters)
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-5
