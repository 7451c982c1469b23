"""Parity at the paper's Table 1 case 1 geometry (Sec. 5), full size.

Two column blocks per iteration (gamma = 2/8), so the FP, the residual
recomputation and the BP run as separate kernels; the row blocks are the
paper's random partition of the views into 5 groups.
"""
import numpy as np
import pytest

from helpers import gpu_geom, oracle_geom, paper_partition, rel_l2, spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import projector as OP  # noqa: E402
from paper_1903_11874_gb300 import binding as B  # noqa: E402


def test_case1_first_iteration():
    """From x = 0 the first iteration gives x_J = mu (A_I^J)^T y on both drawn
    slabs (every voxel checked) and leaves the other voxels at 0."""
    vb = paper_partition()
    s = spec("paper_case1", view_block=vb)
    og, gg = oracle_geom(s), gpu_geom(s)
    y = np.abs(np.random.default_rng(1).standard_normal(og.n_rows)).astype(np.float32)
    mu = 1e-6
    prm = B.SolveParams(alpha=1 / 5, gamma=2 / 8, step_rule=B.STEP_FIXED, mu=mu, seed=3)
    st = B.State(gg, prm, torch.from_numpy(y).cuda())
    x = torch.zeros(gg.n_cols, device="cuda:0")
    st.block_step(x, 1)
    torch.cuda.synchronize()
    tr = st.read_trace(1)
    assert tr[0, 0] == 2
    pairs = [(int(tr[0, 1 + 2 * p]), int(tr[0, 2 + 2 * p])) for p in range(2)]
    assert pairs[0][0] == pairs[1][0] and pairs[0][1] != pairs[1][1]
    i = pairs[0][0]
    rows = OP.rows_of_views(og, OP.row_block_views(og, 5, i, vb))
    assert rows.size == 72 * 400 * 400
    got = x.cpu().double().numpy()
    touched = []
    for _, j in pairs:
        vox = OP.column_block_voxels(og, 8, j)
        ref = mu * OP.bp_rows(og, y[rows].astype(np.float64), rows, OP.column_block(og, 8, j))[vox]
        assert rel_l2(got[vox], ref) <= 1e-5
        touched.append(vox)
    other = np.setdiff1d(np.arange(og.n_cols), np.concatenate(touched))
    assert not got[other].any()
