"""Full-size parity of the fused solver kernels from a non-zero state.

The first iteration from x = 0 forward projects a zero slab, so it checks
neither the FP sums of the fused kernels nor their z / r epilogue. Here the
GPU runs several iterations at the bench's full size and launch shape, chosen
so that slabs are revisited: later FPs walk non-zero images, residuals are
formed from several blocks' non-zero z^j, and the BP weights are the deltas
r - r~ of a refreshed snapshot. The FP64 oracle runs the same draws; every
voxel of the touched slabs, and the residual of the last drawn rows element
by element, are compared.
"""
import numpy as np
import pytest

from helpers import U32, fp_tolerance, gpu_geom, oracle_geom, paper_partition, rel_l2, spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bsgd as OB  # noqa: E402
from oracle import projector as OP  # noqa: E402
from oracle import rng as ORNG  # noqa: E402
from paper_1903_11874_gb300 import binding as B  # noqa: E402

DEV = "cuda:0"


def replay_rows(pairs, stride):
    """Trace rows of one pair per iteration: [1, i, j, then -1 (no cells)]."""
    t = np.full((len(pairs), stride), -1, dtype=np.int32)
    for k, (i, j) in enumerate(pairs):
        t[k, :3] = (1, i, j)
    return t


def residual_bound(ost, og, rows, n_max):
    """Per-row tolerance of r = y - sum_j z^j: the FP error bound of each
    block's ray sum (the oracle's |z^j| stands for A^J |x_J|: x stays
    non-negative here up to a few 1e-5 of its largest value, which the caller
    checks) plus the rounding of r."""
    absz = np.abs(ost.z[:, rows]).sum(axis=0)
    return fp_tolerance(absz, n_max) + 2 * U32 * np.abs(ost.y[rows])


def test_config2_fused_kernel_from_a_nonzero_state():
    """Config 2 (256^3, 360 x 256^2, 8 x 8 blocks, residual-weighted pairs,
    one pair per iteration: fpbp_solve_kernel). Five replayed pairs revisit
    slabs 3 and 4 (a non-zero FP in the 2nd, 4th and 5th, a refreshed
    snapshot in the 4th, the residual of a row formed from two blocks'
    non-zero z^j in the 5th), then one pair is drawn by the device's
    residual-weighted sampler; one block_step call runs all six, as the bench
    launches an epoch."""
    s = spec("config2")
    og, gg = oracle_geom(s), gpu_geom(s)
    M, N = s["M"], s["N"]
    y = np.abs(np.random.default_rng(7).standard_normal(og.n_rows)).astype(np.float32)
    mu = 1e-5
    designed = [(0, 3), (1, 3), (0, 4), (0, 3), (1, 4)]
    n = len(designed) + 1
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=9,
                        pair_sampling=B.PAIRS_RESIDUAL)
    st = B.State(gg, prm, torch.from_numpy(y).to(DEV))
    st.set_replay(replay_rows(designed, st.trace_stride))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, n)
    r_gpu = torch.empty(gg.n_rows, device=DEV)
    st.read_residual(r_gpu)
    torch.cuda.synchronize()
    tr = st.read_trace(n)
    pairs = [(int(t[1]), int(t[2])) for t in tr]
    assert pairs[:len(designed)] == designed and all(int(t[0]) == 1 for t in tr)

    po = OB.Params(M, N, 1 / M, 1 / N, mu, seed=9, pair_sampling="residual")
    ost = OB.bsgd(og, y.astype(np.float64), po, n,
                  replay=[OB.Selection([p], [None]) for p in pairs])
    got = x.cpu().double().numpy()
    assert ost.x.min() >= -1e-3 * ost.x.max()
    touched = sorted({j for _, j in pairs})
    for j in touched:
        vox = OP.column_block_voxels(og, N, j)
        assert rel_l2(got[vox], ost.x[vox]) <= 1e-5, j
    other = np.setdiff1d(np.arange(og.n_cols),
                         np.concatenate([OP.column_block_voxels(og, N, j) for j in touched]))
    assert not got[other].any()
    # the residual of the last pair's row block, element by element
    i_last = pairs[-1][0]
    rows = OP.rows_of_views(og, OP.row_block_views(og, M, i_last))
    r = r_gpu.cpu().double().numpy()[rows]
    tol = residual_bound(ost, og, rows, og.nx + og.ny + og.nz // N)
    assert np.all(np.abs(r - ost.r[rows]) <= tol)
    q = st.query()
    assert abs(q["residual_norm"] - ost.residual_norm()) <= 1e-5 * ost.residual_norm()


def revisiting_seed(M, N, kM, kN, iters):
    """Smallest seed whose uniform draws (the SplitMix64 spec, the same on
    both sides) revisit a column block of an earlier iteration in every
    iteration after the first, and repeat a row block once."""
    for seed in range(1, 10000):
        cols = [set(ORNG.choose_k_of_n(seed, it, ORNG.LANE_COLS, N, kN)) for it in range(iters)]
        rws = [tuple(ORNG.choose_k_of_n(seed, it, ORNG.LANE_ROWS, M, kM)) for it in range(iters)]
        seen, ok = set(cols[0]), True
        for c in cols[1:]:
            ok &= bool(c & seen) and len(c) == kN
            seen |= c
        if ok and len(set(rws)) < iters:
            return seed
    raise AssertionError("no seed found")


def test_case1_fused_multi_block_kernel_from_a_nonzero_state():
    """Table 1 case 1 (Sec. 5: 256^3, 360 views, 400^2 detector, the paper's
    random partition into M = 5 groups, N = 8, alpha = 1/5, gamma = 2/8): two
    column blocks per iteration run through fpbpm_solve_kernel. Two
    iterations with a seed whose draws revisit a slab and repeat the row block
    (a non-zero FP and a refreshed snapshot in the second), against the
    oracle drawing the same pairs."""
    vb = paper_partition()
    s = spec("paper_case1", view_block=vb)
    og, gg = oracle_geom(s), gpu_geom(s)
    M, N, iters = 5, 8, 2
    seed = revisiting_seed(M, N, 1, 2, iters)
    y = np.abs(np.random.default_rng(3).standard_normal(og.n_rows)).astype(np.float32)
    mu = 5e-6
    prm = B.SolveParams(alpha=1 / M, gamma=2 / N, step_rule=B.STEP_FIXED, mu=mu, seed=seed)
    st = B.State(gg, prm, torch.from_numpy(y).to(DEV))
    st.profile(True)
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, iters)
    r_gpu = torch.empty(gg.n_rows, device=DEV)
    st.read_residual(r_gpu)
    torch.cuda.synchronize()
    prof = st.read_profile()
    assert prof["fpbp"]["launches"] == iters and prof["fp"]["launches"] == 0

    po = OB.Params(M, N, 1 / M, 2 / N, mu, seed=seed, view_block=vb)
    ost = OB.bsgd(og, y.astype(np.float64), po, iters)
    tr = st.read_trace(iters)
    assert [sorted((int(t[1 + 2 * p]), int(t[2 + 2 * p])) for p in range(2)) for t in tr] == \
        [sorted(sel.pairs) for sel in ost.history]
    got = x.cpu().double().numpy()
    assert ost.x.min() >= -1e-3 * ost.x.max()
    touched = sorted({j for sel in ost.history for _, j in sel.pairs})
    for j in touched:
        vox = OP.column_block_voxels(og, N, j)
        assert rel_l2(got[vox], ost.x[vox]) <= 1e-5, j
    i_last = ost.history[-1].pairs[0][0]
    rows = OP.rows_of_views(og, OP.row_block_views(og, M, i_last, vb))
    r = r_gpu.cpu().double().numpy()[rows]
    tol = residual_bound(ost, og, rows, og.nx + og.ny + og.nz // N)
    assert np.all(np.abs(r - ost.r[rows]) <= tol)
