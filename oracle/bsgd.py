"""FP64 BSGD oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this module. It runs the paper's iteration step by step, in the paper's order,
with every FP and BP done by the FP64 Siddon projector in oracle/projector.py.

Readings of the paper used here (the design notes list each of them too):
  * gradient of 1/2 ||y - A x||^2 is A^T r, so the factor 2 printed in
    Algorithm 1's BP step is folded into mu (Sec. 1, Eq. 2 vs Algorithm 1);
  * "randomly select" = uniform without replacement within an iteration,
    i.i.d. across iterations, drawn from the SplitMix64 spec in oracle/rng.py;
  * one epoch = 1/(alpha*gamma) iterations (Sec. 3.4, effective epochs);
  * sub-detector cells keep SAG memory per cell (snapshot form below), so the
    fixed point stays the least-squares solution of Sec. 4 for any sampling law;
  * residual-weighted pair sampling: p(i, j) ~ sum of r^2 over the detector
    rows R_ij of J_j's shadow in the views of I_i, plus a small floor;
  * Algorithm 3 counts k in epochs (the paper tests every M epochs); the
    effective update direction of a window is the sum of the directions g_J
    the window's updates applied; ||r|| is the maintained ||y - sum_j z^j||;
    the test starts once three residual checkpoints exist (k >= 2M), and the
    criterion |theta^e - theta^(e-1)| > t1 is used once two cosines exist.
"""
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import projector as P
from . import rng
from .tv import tv_prox


@dataclass
class Params:
    M: int
    N: int
    alpha: float
    gamma: float
    mu: float
    seed: int = 1
    pair_sampling: str = "uniform"     # "uniform" | "residual"
    cells: str = "none"                # "none" | "geometric" | "uniform"
    n_cells: int = 1                   # 1, 2 (2D halves) or 4 (3D quadrants)
    tv_lambda: float = 0.0
    tv_iters: int = 20
    view_block: Optional[np.ndarray] = None
    # Algorithm 3 (automatic step length): a test every `auto_window` epochs
    # (0: M epochs, as in the paper)
    auto_mu: bool = False
    auto_window: int = 0
    auto_eps: float = 0.1
    auto_delta: float = 0.4
    auto_t1: float = 0.2
    auto_t2: float = 0.5

    @property
    def kM(self) -> int:
        return max(1, int(round(self.alpha * self.M)))

    @property
    def kN(self) -> int:
        return max(1, int(round(self.gamma * self.N)))

    @property
    def epoch_len(self) -> int:
        """Iterations per (effective) epoch: 1/(alpha*gamma)."""
        return max(1, int(round(1.0 / (self.alpha * self.gamma))))


RESIDUAL_FLOOR = 1e-9   # relative floor of the residual weights (per pair)
CELL_FLOOR = 1e-12      # relative floor of the geometric cell weights


@dataclass
class Selection:
    """What one iteration works on: the pairs (i, j) and, per pair, the cell
    chosen for every view of I_i (None without sub-detector sampling)."""
    pairs: List[tuple]
    cells: List[Optional[np.ndarray]] = field(default_factory=list)


# --------------------------------------------------------------------------
# Sampling

def geometric_cell_weights(geom, prm: Params, j: int) -> np.ndarray:
    """w[a, s] = 1^T A_{(a, s)}^{J_j} 1: total chord length inside J_j's box of
    the rays of cell s at view a (the density proxy of Sec. 2.1: the fraction of
    a block's projection on each sub-detector), floored relative to the view's
    sum so that every cell stays reachable."""
    block = P.column_block(geom, prm.N, j)
    ones = np.zeros(geom.n_cols)
    ones[P.column_block_voxels(geom, prm.N, j)] = 1.0
    y = P.fp(geom, ones, None, block)          # (views, nv, nu)
    v, u = np.meshgrid(np.arange(geom.nv), np.arange(geom.nu), indexing="ij")
    cell = P.cell_of_pixel(geom, v, u, prm.n_cells)
    w = np.zeros((geom.n_views, prm.n_cells))
    for s in range(prm.n_cells):
        w[:, s] = y[:, cell == s].sum(axis=1)
    tot = w.sum(axis=1, keepdims=True)
    return np.maximum(w, CELL_FLOOR * tot)


def residual_pair_weights(geom, prm: Params, r: np.ndarray, bands) -> np.ndarray:
    """W[i, j] = sum over views a in I_i, rows v in R_ij, all u of r^2, plus a
    floor RESIDUAL_FLOOR * mean(W) (and 1e-300) so that no pair has weight 0."""
    r3 = r.reshape(geom.sino_shape)
    W = np.zeros((prm.M, prm.N))
    for i in range(prm.M):
        views = P.row_block_views(geom, prm.M, i, prm.view_block)
        S = (r3[views] ** 2).sum(axis=(0, 2))          # per detector row v
        for j in range(prm.N):
            lo, hi = bands[i][j]
            W[i, j] = S[lo:hi + 1].sum() if lo <= hi else 0.0
    return W + RESIDUAL_FLOOR * W.sum() / W.size + 1e-300


def sample(geom, prm: Params, it: int, r: np.ndarray, bands, cell_w) -> Selection:
    if prm.pair_sampling == "uniform":
        I = rng.choose_k_of_n(prm.seed, it, rng.LANE_ROWS, prm.M, prm.kM)
        J = rng.choose_k_of_n(prm.seed, it, rng.LANE_COLS, prm.N, prm.kN)
        pairs = [(i, j) for i in I for j in J]
    elif prm.pair_sampling == "residual":
        if prm.kM != 1 or prm.kN != 1:
            raise ValueError("residual pair sampling draws one pair per iteration")
        W = residual_pair_weights(geom, prm, r, bands).reshape(-1)
        k = rng.choose_weighted(rng.uniform(prm.seed, it, rng.LANE_PAIR), W)
        pairs = [(k // prm.N, k % prm.N)]
    else:
        raise ValueError(prm.pair_sampling)
    cells = []
    for p, (i, j) in enumerate(pairs):
        if prm.cells == "none":
            cells.append(None)
            continue
        views = P.row_block_views(geom, prm.M, i, prm.view_block)
        choice = np.zeros(views.size, dtype=np.int64)
        for k, a in enumerate(views):
            u = rng.uniform(prm.seed, it, rng.LANE_CELLS + p * views.size + k)
            if prm.cells == "uniform":
                choice[k] = min(int(u * prm.n_cells), prm.n_cells - 1)
            else:
                choice[k] = rng.choose_weighted(u, cell_w[j][a])
        cells.append(choice)
    return Selection(pairs, cells)


def selection_rows(geom, prm: Params, i: int, cells) -> np.ndarray:
    """Row index set of pair (i, .): all rows of I_i, or the chosen cells' rows
    (the set I-hat_t of Algorithm 2)."""
    views = P.row_block_views(geom, prm.M, i, prm.view_block)
    if cells is None:
        return P.rows_of_views(geom, views)
    return np.concatenate([P.rows_of_cell(geom, int(a), int(s), prm.n_cells)
                           for a, s in zip(views, cells)])


# --------------------------------------------------------------------------
# Step size

def power_iteration(geom, N: int, j: int, iters: int = 30, views=None) -> float:
    """lambda_J ~ ||A^J||_2^2 (rows = all views unless given): v0 = 1/sqrt|J|
    on J, v <- A^T A v / ||A^T A v||, then lambda = ||A^J v||^2."""
    block = P.column_block(geom, N, j)
    vox = P.column_block_voxels(geom, N, j)
    views = np.arange(geom.n_views) if views is None else np.asarray(views)
    rows = P.rows_of_views(geom, views)
    v = np.zeros(geom.n_cols)
    v[vox] = 1.0 / math.sqrt(vox.size)
    for _ in range(iters):
        w = P.bp_rows(geom, P.fp_rows(geom, v, rows, block), rows, block)
        nrm = math.sqrt(float(np.dot(w, w)))
        if nrm == 0.0:
            return 0.0
        v = w / nrm
    z = P.fp_rows(geom, v, rows, block)
    return float(np.dot(z, z))


def step_strip(geom, N: int, rho: float = 1.0, iters: int = 30) -> float:
    """mu = rho / max_J ||A^J||^2 (g_J aggregates every row block, so the
    column strip A^J is the operator whose Lipschitz constant bounds the step)."""
    return rho / max(power_iteration(geom, N, j, iters) for j in range(N))


# --------------------------------------------------------------------------
# Algorithm 1, literal form

def bsgd_literal(geom, y, prm: Params, n_iters: int, replay=None):
    """Algorithm 1 exactly as printed (memories z^j in R^r, g-hat^i in R^c),
    uniform sampling only. Returns (x, history)."""
    r_, c_ = geom.n_rows, geom.n_cols
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    x = np.zeros(c_)
    z = np.zeros((prm.N, r_))
    ghat = np.zeros((prm.M, c_))
    r = y.copy()
    hist = []
    for it in range(n_iters):
        sel = replay[it] if replay is not None else sample(geom, prm, it, r, None, None)
        rows = {i: selection_rows(geom, prm, i, None) for i, _ in sel.pairs}
        for i, j in sel.pairs:                                  # z^j_{I_i} = A x_J
            z[j, rows[i]] = P.fp_rows(geom, x, rows[i], P.column_block(geom, prm.N, j))
        r = y - z.sum(axis=0)                                   # r = y - sum_j z^j
        for i, j in sel.pairs:                                  # g-hat^i_J = A^T r_I
            vox = P.column_block_voxels(geom, prm.N, j)
            full = P.bp_rows(geom, r[rows[i]], rows[i], P.column_block(geom, prm.N, j))
            ghat[i, vox] = full[vox]
        g = ghat.sum(axis=0)                                    # g = sum_i g-hat^i
        for j in sorted({j for _, j in sel.pairs}):             # x_J += mu g_J
            vox = P.column_block_voxels(geom, prm.N, j)
            x[vox] += prm.mu * g[vox]
        hist.append(sel)
    return x, hist


# --------------------------------------------------------------------------
# Snapshot form (the form the CUDA path implements)

class BSGDState:
    """State of the snapshot form: z^j (N x r), residual snapshots rt^j (N x r),
    r, aggregated g and x. For a selected pair with rows R,
        g_J += (A_R^J)^T (r_R - rt^J_R),  rt^J_R = r_R,
    which equals replacing g-hat^i_J by (A_{I_i}^J)^T r_{I_i} when R = I_i and is
    SAG memory per sub-detector cell otherwise."""

    def __init__(self, geom, y, prm: Params, x0=None):
        self.geom, self.prm = geom, prm
        self.y = np.asarray(y, dtype=np.float64).reshape(-1)
        r_, c_ = geom.n_rows, geom.n_cols
        self.x = np.zeros(c_) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
        self.z = np.zeros((prm.N, r_))
        if x0 is not None:                                      # z^j = A^j x0_J
            allrows = np.arange(r_, dtype=np.int64)
            for j in range(prm.N):
                self.z[j] = P.fp_rows(geom, self.x, allrows, P.column_block(geom, prm.N, j))
        self.rt = np.zeros((prm.N, r_))
        self.g = np.zeros(c_)
        self.r = self.y - self.z.sum(axis=0)
        self.it = 0
        self.bands = [[P.row_block_v_band(geom, prm.M, prm.N, i, j, prm.view_block)
                       for j in range(prm.N)] for i in range(prm.M)]
        self.cell_w = ([geometric_cell_weights(geom, prm, j) for j in range(prm.N)]
                       if prm.cells == "geometric" else None)
        self.history = []
        self.mu = prm.mu
        if prm.auto_mu:
            self.tuner = AutoMu(prm.auto_window or prm.M, prm.auto_eps, prm.auto_delta,
                                prm.auto_t1, prm.auto_t2, self.residual_norm(), c_)

    def step(self, sel: Optional[Selection] = None):
        geom, prm = self.geom, self.prm
        if sel is None:
            sel = sample(geom, prm, self.it, self.r, self.bands, self.cell_w)
        rows = [selection_rows(geom, prm, i, c) for (i, _), c in zip(sel.pairs, sel.cells or [None] * len(sel.pairs))]
        for (i, j), R in zip(sel.pairs, rows):
            self.z[j, R] = P.fp_rows(geom, self.x, R, P.column_block(geom, prm.N, j))
        self.r = self.y - self.z.sum(axis=0)
        for (i, j), R in zip(sel.pairs, rows):
            P.bp_rows(geom, self.r[R] - self.rt[j, R], R, P.column_block(geom, prm.N, j), out=self.g)
            self.rt[j, R] = self.r[R]
        for j in sorted({j for _, j in sel.pairs}):
            vox = P.column_block_voxels(geom, prm.N, j)
            self.x[vox] += self.mu * self.g[vox]
            if prm.auto_mu:
                self.tuner.eud[vox] += self.g[vox]
        self.it += 1
        if prm.tv_lambda > 0.0 and self.it % prm.epoch_len == 0:   # Algorithm 4
            # Eq. 10 is the TV of a 2D image; volumes use the 3D extension
            shape = geom.vol_shape if geom.nz > 1 else (geom.ny, geom.nx)
            self.x = tv_prox(self.x.reshape(shape), self.mu * prm.tv_lambda,
                             prm.tv_iters).reshape(-1)
        if prm.auto_mu and self.it % (prm.epoch_len * self.tuner.window) == 0:   # Algorithm 3
            self.mu = self.tuner.test(self.mu, self.residual_norm())
        self.history.append(sel)
        return sel

    def residual_norm(self) -> float:
        return float(np.linalg.norm(self.r))


class AutoMu:
    """Algorithm 3. At the end of window e (every `window` epochs) the
    effective update direction gbar^e (the sum of the directions the window's
    updates applied) gives theta^e = cos(gbar^e, gbar^(e-1)). With the residual
    norms rho^e, rho^(e-1), rho^(e-2) at the last three window ends (rho^0 at
    the start):
      rho^e < rho^(e-1) < rho^(e-2)                       ->  mu <- (1 + eps) mu
      rho^e > rho^(e-1) > rho^(e-2) and (theta^e < t2 or
                            |theta^e - theta^(e-1)| > t1)  ->  mu <- (1 - delta) mu
    A cosine with a zero direction counts as 1."""

    def __init__(self, window, eps, delta, t1, t2, rho0, n_cols):
        self.window, self.eps, self.delta, self.t1, self.t2 = window, eps, delta, t1, t2
        self.rho = [rho0]                 # residual norm at each window end
        self.theta = []                   # cosine at each window end (None for e = 1)
        self.eud = np.zeros(n_cols)
        self.eud_prev = None
        self.mu_log = []

    @staticmethod
    def cosine(a, b) -> float:
        na, nb = float(np.linalg.norm(a)), float(np.linalg.norm(b))
        return 1.0 if na == 0.0 or nb == 0.0 else float(np.dot(a, b)) / (na * nb)

    def decide(self, mu: float, rho, theta, theta_prev) -> float:
        """The test of Algorithm 3 on the last three residual norms
        rho = (rho^(e-2), rho^(e-1), rho^e) and the cosines theta^e and
        theta^(e-1) (None where not defined yet)."""
        r2, r1, r0 = rho
        if r0 < r1 < r2:
            return mu * (1.0 + self.eps)
        if r0 > r1 > r2:
            c2 = theta is not None and theta < self.t2
            c1 = theta is not None and theta_prev is not None and abs(theta - theta_prev) > self.t1
            if c1 or c2:
                return mu * (1.0 - self.delta)
        return mu

    def test(self, mu: float, rho_now: float) -> float:
        theta = self.cosine(self.eud, self.eud_prev) if self.eud_prev is not None else None
        self.rho.append(rho_now)
        if len(self.rho) >= 3:
            theta_prev = self.theta[-1] if self.theta else None
            mu = self.decide(mu, self.rho[-3:], theta, theta_prev)
        self.theta.append(theta)
        self.eud_prev, self.eud = self.eud, np.zeros_like(self.eud)
        self.mu_log.append(mu)
        return mu


def bsgd(geom, y, prm: Params, n_iters: int, x0=None, replay=None):
    """Run n_iters iterations of the snapshot form; returns the state."""
    st = BSGDState(geom, y, prm, x0)
    for k in range(n_iters):
        st.step(None if replay is None else replay[k])
    return st
