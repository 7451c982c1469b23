"""Pins of the FP64 BSGD oracle (CPU only).

Against the paper: Algorithm 1 literal vs the snapshot form; the special cases
the paper names (gamma = 1 is SAG, Sec. 2; all blocks at once is gradient
descent); the fixed point of Sec. 4 (the least-squares solution, computed here
with a library solve on the explicit matrix); convergence on the paper's 2D
set-up (Sec. 3.1) and the config-1 phantom; the power-iteration step against an
SVD; the sampling weights against brute-force sums over rays.
"""
import math

import numpy as np
import pytest

from oracle import bsgd as B
from oracle import projector as P
from oracle import rng
from oracle.tv import tv_prox
from paper_1903_11874_gb300 import synth

RHO = 0.25   # step fraction of 1/max_J ||A^J||^2 (rho = 1 diverges under block sampling)


def paper_2d_geom():
    """Sec. 3.1: fan beam, K = 16, OP = OD = 50, 30 unit detector elements,
    10 degree steps over a full turn (A in R^{1080 x 256})."""
    return P.Geometry("fan2d", 16, 16, 1, 1.0, 1.0, 1.0, 36, 30, 1, 1.0, 1.0, dso=50.0, dsd=100.0)


_CACHE = {}


def paper_2d_problem():
    if "p" not in _CACHE:
        geom = paper_2d_geom()
        A = P.dense_matrix(geom)
        x_true = synth.ellipse_phantom(16, 16, 6, 0).reshape(-1)
        y = synth.gaussian_noise_at_snr(A @ x_true, 17.5, 1)     # SNR 17.5 dB (Sec. 3.1)
        x_ls = np.linalg.lstsq(A, y, rcond=None)[0]
        _CACHE["p"] = (geom, A, y, x_ls)
    return _CACHE["p"]


def test_paper_2d_setup_size():
    geom, A, _, _ = paper_2d_problem()
    assert A.shape == (1080, 256)


@pytest.mark.parametrize("M,N,alpha,gamma", [(4, 2, 1.0, 1.0), (4, 2, 0.5, 0.5), (3, 4, 1 / 3, 0.5)])
def test_literal_equals_snapshot(M, N, alpha, gamma):
    geom, _, y, _ = paper_2d_problem()
    prm = B.Params(M, N, alpha, gamma, RHO * B.step_strip(geom, N), seed=4)
    x_lit, hist = B.bsgd_literal(geom, y, prm, 40)
    st = B.bsgd(geom, y, prm, 40)
    assert [s.pairs for s in hist] == [s.pairs for s in st.history]
    np.testing.assert_allclose(st.x, x_lit, rtol=0, atol=1e-12 * np.abs(x_lit).max())


def test_all_blocks_is_gradient_descent():
    """M = N = 1, alpha = gamma = 1: x <- x + mu A^T (y - A x)."""
    geom, A, y, _ = paper_2d_problem()
    mu = 0.9 / np.linalg.norm(A, 2) ** 2
    st = B.bsgd(geom, y, B.Params(1, 1, 1.0, 1.0, mu), 30)
    x = np.zeros(A.shape[1])
    for _ in range(30):
        x = x + mu * A.T @ (y - A @ x)
    np.testing.assert_allclose(st.x, x, rtol=0, atol=1e-11 * np.abs(x).max())


def test_gamma_one_is_sag():
    """gamma = 1 (Sec. 2): memory g-hat^i = A_i^T (y_i - A_i x) refreshed for the
    sampled row block, x moves along the sum of all memories (SAG)."""
    geom, A, y, _ = paper_2d_problem()
    M = 4
    prm = B.Params(M, 1, 1.0 / M, 1.0, 0.2 / np.linalg.norm(A, 2) ** 2, seed=2)
    st = B.bsgd(geom, y, prm, 60)
    per = geom.nv * geom.nu
    blocks = [np.concatenate([np.arange(a * per, (a + 1) * per)
                              for a in P.row_block_views(geom, M, i)]) for i in range(M)]
    x = np.zeros(A.shape[1])
    mem = np.zeros((M, A.shape[1]))
    for it in range(60):
        i = rng.choose_k_of_n(prm.seed, it, rng.LANE_ROWS, M, 1)[0]
        Ai = A[blocks[i]]
        mem[i] = Ai.T @ (y[blocks[i]] - Ai @ x)
        x = x + prm.mu * mem.sum(axis=0)
    np.testing.assert_allclose(st.x, x, rtol=0, atol=1e-11 * np.abs(x).max())


def test_fixed_point_is_least_squares():
    """Sec. 4: the fixed point is the LS solution; with alpha = gamma = 1
    (Sec. 3.1, M = 4, N = 2) the distance DS = ||x - x_lsq|| goes to 0, and at
    the fixed point z^j = A^j x and g = A^T (y - A x) = 0."""
    geom, A, y, x_ls = paper_2d_problem()
    prm = B.Params(4, 2, 1.0, 1.0, B.step_strip(geom, 2), seed=1)
    st = B.bsgd(geom, y, prm, 2000)
    assert np.linalg.norm(st.x - x_ls) < 2e-6 * np.linalg.norm(x_ls)
    assert np.linalg.norm(st.g) < 1e-5 * np.linalg.norm(A.T @ y)
    for j in range(2):
        vox = P.column_block_voxels(geom, 2, j)
        # z^j holds A^J x from before the last update, which moved x by ~1e-6
        np.testing.assert_allclose(st.z[j], A[:, vox] @ st.x[vox], atol=1e-7 * np.abs(st.z[j]).max())


@pytest.mark.parametrize("M,N", [(8, 8), (4, 16)])
def test_block_sampling_approaches_least_squares(M, N):
    """Sec. 3.1 (Fig. 5): alpha = 1/M, gamma = 1/N still approaches x_lsq."""
    geom, _, y, x_ls = paper_2d_problem()
    prm = B.Params(M, N, 1.0 / M, 1.0 / N, RHO * B.step_strip(geom, N), seed=3)
    st = B.BSGDState(geom, y, prm)
    ds = []
    for ep in range(100):
        for _ in range(prm.epoch_len):
            st.step()
        if ep % 25 == 24:
            ds.append(np.linalg.norm(st.x - x_ls) / np.linalg.norm(x_ls))
    assert ds[-1] < 0.05
    assert ds[-1] < 0.5 * ds[0]


@pytest.mark.parametrize("pairs,cells", [("uniform", "geometric"), ("uniform", "uniform"),
                                         ("residual", "none")])
def test_importance_sampling_keeps_least_squares_fixed_point(pairs, cells):
    """BSGD-IM (Algorithm 2) with SAG memory per sub-detector cell (the halves
    DE / DF of Fig. 3), BSGD-RAN (uniform cells) and residual-weighted pairs all
    head to x_lsq."""
    geom, _, y, x_ls = paper_2d_problem()
    prm = B.Params(4, 2, 0.25, 0.5, RHO * B.step_strip(geom, 2), seed=5,
                   pair_sampling=pairs, cells=cells, n_cells=2 if cells != "none" else 1)
    st = B.BSGDState(geom, y, prm)
    ds = []
    for ep in range(150):
        for _ in range(prm.epoch_len):
            st.step()
        if ep % 50 == 49:
            ds.append(np.linalg.norm(st.x - x_ls) / np.linalg.norm(x_ls))
    assert ds[-1] < 0.03 and ds[-1] < 0.5 * ds[0]


def test_noise_free_convergence_to_phantom():
    """Config-1 geometry (64^2 image, 90 parallel views over 180 deg, 96 unit
    bins, 4 x 4 blocks, alpha = gamma = 1/4, 50 epochs): the relative error to
    the phantom falls every epoch."""
    geom = P.Geometry("par2d", 64, 64, 1, 1.0, 1.0, 1.0, 90, 96, 1, 1.0, 1.0)
    xt = synth.ellipse_phantom(64, 64, 6, 0).reshape(-1)
    y = P.fp(geom, xt).reshape(-1)
    prm = B.Params(4, 4, 0.25, 0.25, RHO * B.step_strip(geom, 4), seed=1)
    st = B.BSGDState(geom, y, prm)
    errs = []
    for ep in range(50):
        for _ in range(prm.epoch_len):
            st.step()
        errs.append(np.linalg.norm(st.x - xt) / np.linalg.norm(xt))
    assert all(b <= a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.13


def test_power_iteration_matches_svd():
    geom, A, _, _ = paper_2d_problem()
    for j in range(2):
        vox = P.column_block_voxels(geom, 2, j)
        s = np.linalg.svd(A[:, vox], compute_uv=False)[0]
        assert abs(B.power_iteration(geom, 2, j, 300) - s * s) < 1e-9 * s * s
        assert abs(B.power_iteration(geom, 2, j, 30) - s * s) < 1e-2 * s * s


def small_cone():
    return P.Geometry("cone3d", 10, 9, 12, 1.0, 1.1, 0.9, 8, 14, 12, 1.5, 1.6, dso=40.0,
                      dsd=80.0, angles=0.05 + np.arange(8) * (2 * math.pi / 8))


def test_residual_pair_weights_brute_force():
    geom = small_cone()
    M, N = 4, 3
    prm = B.Params(M, N, 1 / M, 1 / N, 1.0, pair_sampling="residual")
    r = synth.normal_array(geom.n_rows, 3)
    bands = [[P.row_block_v_band(geom, M, N, i, j) for j in range(N)] for i in range(M)]
    W = B.residual_pair_weights(geom, prm, r, bands)
    ref = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            views = set(P.row_block_views(geom, M, i).tolist())
            lo = min(P.v_band(geom, a, N, j)[0] for a in views)
            hi = max(P.v_band(geom, a, N, j)[1] for a in views)
            for row in range(geom.n_rows):
                a, v = row // (geom.nv * geom.nu), (row // geom.nu) % geom.nv
                if a in views and lo <= v <= hi:
                    ref[i, j] += r[row] ** 2
    ref += B.RESIDUAL_FLOOR * ref.sum() / ref.size + 1e-300
    np.testing.assert_allclose(W, ref, rtol=1e-12)


def test_geometric_cell_weights_brute_force():
    geom = small_cone()
    N = 3
    prm = B.Params(2, N, 0.5, 1 / N, 1.0, cells="geometric", n_cells=4)
    A = P.dense_matrix(geom)
    for j in range(N):
        w = B.geometric_cell_weights(geom, prm, j)
        vox = P.column_block_voxels(geom, N, j)
        for a in range(geom.n_views):
            tot = A[P.rows_of_views(geom, [a])][:, vox].sum()
            for s in range(4):
                exp = A[P.rows_of_cell(geom, a, s, 4)][:, vox].sum()
                assert abs(w[a, s] - max(exp, B.CELL_FLOOR * tot)) <= 1e-10 * (1 + tot)


# --------------------------------------------------------------------------
# BSGD-TV (Algorithm 4). The paper's objective, Eq. (TVequ), is
# ||y - A x||^2 + 2 lambda TV(x); halved it is 1/2 ||y - A x||^2 + lambda TV(x),
# whose ISTA step with step length mu (gradient A^T r, the factor 2 of
# Algorithm 1 folded into mu) is x <- prox(x + mu A^T r) with
# prox(b) = argmin_t ||t - b||^2 + 2 mu lambda TV(t), i.e. tv_prox(b, kappa = mu lambda).
# In the paper's own step length (half of this mu) that weight reads 4 mu lambda,
# twice what Algorithm 4 prints; the objective decides.

def test_bsgd_tv_all_blocks_is_ista():
    """M = N = 1, alpha = gamma = 1: one iteration per epoch, so Algorithm 4 is
    ISTA on 1/2 ||y - A x||^2 + lambda TV(x): every iterate equals
    tv_prox(x + mu A^T (y - A x), mu lambda), the matrix product taken on the
    explicit matrix of the paper's 2D set-up (Sec. 3.1)."""
    geom, A, y, _ = paper_2d_problem()
    mu = 0.9 / np.linalg.norm(A, 2) ** 2
    lam = 0.05 * float(np.abs(A.T @ y).max())
    prm = B.Params(1, 1, 1.0, 1.0, mu, tv_lambda=lam, tv_iters=15)
    st = B.BSGDState(geom, y, prm)
    x = np.zeros(A.shape[1])
    moved = 0.0
    for _ in range(12):
        st.step()
        b = x + mu * A.T @ (y - A @ x)
        x = tv_prox(b.reshape(16, 16), mu * lam, 15).reshape(-1)
        moved = max(moved, float(np.linalg.norm(x - b)))
        np.testing.assert_allclose(st.x, x, rtol=0, atol=1e-12 * np.abs(x).max())
    assert moved > 1e-3 * np.linalg.norm(x)          # the prox is active


def test_bsgd_tv_prox_on_the_epoch_boundary_only():
    """1/(alpha gamma) = 4 iterations per epoch: the TV-regularised state equals
    the plain Algorithm 1 state driven through the same draws, with
    tv_prox(x, mu lambda) applied by hand after iterations 4, 8 and 12 and at
    no other time."""
    geom, A, y, _ = paper_2d_problem()
    mu = RHO * B.step_strip(geom, 2)
    lam = 0.05 * float(np.abs(A.T @ y).max())
    tv = B.BSGDState(geom, y, B.Params(2, 2, 0.5, 0.5, mu, seed=6, tv_lambda=lam, tv_iters=10))
    plain = B.BSGDState(geom, y, B.Params(2, 2, 0.5, 0.5, mu, seed=6))
    assert tv.prm.epoch_len == 4
    for it in range(1, 13):
        sel = tv.step()
        plain.step(sel)
        if it % 4 == 0:
            before = plain.x.copy()
            plain.x = tv_prox(plain.x.reshape(16, 16), mu * lam, 10).reshape(-1)
            assert np.linalg.norm(plain.x - before) > 1e-4 * np.linalg.norm(before)
        np.testing.assert_allclose(tv.x, plain.x, rtol=0, atol=1e-12 * np.abs(plain.x).max())


def test_bsgd_tv_small_lambda_is_plain_bsgd():
    """lambda -> 0: the prox tends to the identity and BSGD-TV to Algorithm 1."""
    geom, _, y, _ = paper_2d_problem()
    mu = RHO * B.step_strip(geom, 2)
    a = B.bsgd(geom, y, B.Params(2, 2, 0.5, 0.5, mu, seed=6, tv_lambda=1e-12), 12)
    b = B.bsgd(geom, y, B.Params(2, 2, 0.5, 0.5, mu, seed=6), 12)
    np.testing.assert_allclose(a.x, b.x, rtol=0, atol=1e-9 * np.abs(b.x).max())


# --------------------------------------------------------------------------
# Starting image x0 != 0: z^j = A^j x0_J, r = y - sum_j z^j, r~ = 0, g = 0

def test_start_from_x0_all_blocks_is_gradient_descent_from_x0():
    """M = N = 1: the iterates are gradient descent started at x0."""
    geom, A, y, _ = paper_2d_problem()
    mu = 0.9 / np.linalg.norm(A, 2) ** 2
    x0 = synth.normal_array(A.shape[1], 21)
    st = B.bsgd(geom, y, B.Params(1, 1, 1.0, 1.0, mu), 25, x0=x0)
    x = x0.copy()
    for _ in range(25):
        x = x + mu * A.T @ (y - A @ x)
    np.testing.assert_allclose(st.x, x, rtol=0, atol=1e-11 * np.abs(x).max())


def test_start_at_the_least_squares_solution_stays_there():
    """Sec. 4: x_lsq is the fixed point. Started there with every block in
    every iteration (M = 4, N = 2, alpha = gamma = 1), each iteration's memories
    sum to g = A^T (y - A x_lsq) = 0, so x does not move; the memories z^j of
    the start give r = y - A x_lsq."""
    geom, A, y, x_ls = paper_2d_problem()
    prm = B.Params(4, 2, 1.0, 1.0, B.step_strip(geom, 2), seed=9)
    st = B.BSGDState(geom, y, prm, x0=x_ls)
    np.testing.assert_allclose(st.r, y - A @ x_ls, rtol=0, atol=1e-12 * np.abs(y).max())
    for j in range(2):
        vox = P.column_block_voxels(geom, 2, j)
        np.testing.assert_allclose(st.z[j], A[:, vox] @ x_ls[vox], rtol=0, atol=1e-12 * np.abs(y).max())
    for _ in range(5):
        st.step()
    assert np.linalg.norm(st.x - x_ls) <= 1e-9 * np.linalg.norm(x_ls)
