"""GPU parity of the BSGD iteration against the FP64 oracle, through the C ABI.

Uniform sampling draws the same blocks on both sides (the SplitMix64 spec is
implemented independently on each), so whole trajectories are compared. Where
a floating-point weight decides the draw (residual pairs, geometric cells), the
oracle replays the GPU's recorded choices and the test checks separately that
the GPU's own choices agree with the oracle's sampler.
"""
import numpy as np
import pytest

from helpers import gpu_geom, oracle_geom, rel_l2, spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bsgd as OB  # noqa: E402
from oracle import projector as OP  # noqa: E402
from oracle import tv as OT  # noqa: E402
from paper_1903_11874_gb300 import binding as B  # noqa: E402
from paper_1903_11874_gb300 import synth  # noqa: E402

DEV = "cuda:0"
RHO = 0.25

_CACHE = {}


def problem(name):
    """(spec, oracle geometry, GPU geometry, y (FP32-rounded), mu)."""
    if name not in _CACHE:
        s = spec(name)
        og, gg = oracle_geom(s), gpu_geom(s)
        if og.nz > 1:
            xt = synth.ellipsoid_phantom(og.nx, og.ny, og.nz, 6, seed=0).astype(np.float64)
        else:
            xt = synth.ellipse_phantom(og.nx, og.ny, 6, seed=0)
        y = OP.fp(og, xt.reshape(-1)).reshape(-1).astype(np.float32).astype(np.float64)
        mu = RHO * OB.step_strip(og, s["N"], 1.0, 30)
        _CACHE[name] = (s, og, gg, y, mu, xt.reshape(-1))
    return _CACHE[name]


def gpu_run(gg, y, prm, iters, x=None, storage=torch.float32):
    st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
    if x is None:
        x = torch.zeros(gg.n_cols, device=DEV, dtype=storage)
    st.block_step(x, iters)
    torch.cuda.synchronize()
    return st, x


def oracle_replay(trace, n_pairs_max, max_views, M, og, prm_o, cells):
    sels = []
    for t in trace:
        np_ = int(t[0])
        pairs = [(int(t[1 + 2 * p]), int(t[2 + 2 * p])) for p in range(np_)]
        cl = []
        for p, (i, _) in enumerate(pairs):
            if not cells:
                cl.append(None)
                continue
            nv = OP.row_block_views(og, M, i).size
            base = 1 + 2 * np_ + p * max_views
            cl.append(np.array(t[base:base + nv], dtype=np.int64))
        sels.append(OB.Selection(pairs, cl))
    return sels


@pytest.mark.parametrize("kM,kN", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_device_sampler_follows_the_spec(kM, kN):
    s, og, gg, y, mu, _ = problem("paper2d")
    M, N = s["M"], s["N"]
    prm = B.SolveParams(alpha=kM / M, gamma=kN / N, step_rule=B.STEP_FIXED, mu=mu, seed=11)
    st, _ = gpu_run(gg, y, prm, 40)
    tr = st.read_trace(40)
    po = OB.Params(M, N, kM / M, kN / N, mu, seed=11)
    for it in range(40):
        exp = OB.sample(og, po, it, None, None, None).pairs
        got = [(int(tr[it, 1 + 2 * p]), int(tr[it, 2 + 2 * p])) for p in range(int(tr[it, 0]))]
        assert got == exp, it


def test_config1_trajectory_matches_oracle():
    """Config 1: 64^2, 90 x 96 parallel beam, 4 x 4 blocks, alpha = gamma = 1/4,
    uniform sampling, 50 epochs (800 iterations): final x within 1e-5."""
    s, og, gg, y, mu, xt = problem("config1")
    M, N = s["M"], s["N"]
    iters = 50 * 16
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_FIXED, mu=mu, seed=1)
    st, x = gpu_run(gg, y, prm, iters)
    ost = OB.bsgd(og, y, OB.Params(M, N, 0.25, 0.25, mu, seed=1), iters)
    got = x.cpu().double().numpy()
    assert rel_l2(got, ost.x) <= 1e-5
    rep = st.query()
    assert rep["iteration"] == iters
    assert abs(rep["residual_norm"] - ost.residual_norm()) <= 1e-4 * np.linalg.norm(y)
    assert rel_l2(got, xt) < 0.13       # and it is a reconstruction


@pytest.mark.parametrize("name", ["config1", "cone_small"])
def test_fused_and_split_kernels_agree(name):
    """With one column block per iteration FP, residual and BP of a ray run in
    one kernel; the split path (FP kernel, then BP kernel) gives the same
    iterates, the same residual-driven choices and the same update count, up to
    the order of the float atomics in g."""
    s, og, gg, y, mu, _ = problem(name)
    M, N = s["M"], s["N"]
    out = []
    for split in (False, True):
        prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=4,
                            pair_sampling=B.PAIRS_RESIDUAL)
        st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
        st.set_split(split)
        x = torch.zeros(gg.n_cols, device=DEV)
        st.profile(True)
        st.block_step(x, 24)
        prof = st.read_profile()
        out.append((x.cpu().double().numpy(), st.read_trace(24), st.query(), prof))
    (xf, tf, qf, pf), (xs, ts, qs, ps) = out
    assert pf["fpbp"]["launches"] == 24 and pf["fp"]["launches"] == 0
    assert ps["fp"]["launches"] == 24 and ps["bp"]["launches"] == 24 and ps["fpbp"]["launches"] == 0
    assert rel_l2(xf, xs) <= 1e-5
    assert np.array_equal(tf, ts)
    assert qf["updates"] == qs["updates"]
    assert abs(qf["residual_norm"] - qs["residual_norm"]) <= 1e-5 * qs["residual_norm"]


def test_several_column_blocks_per_iteration():
    """alpha = gamma = 1/2 on the paper's 2D set-up: two column blocks share a
    row block, so r is formed after both blocks' FPs (the multi-block fused
    pass), against the literal form of Algorithm 1."""
    s, og, gg, y, mu, _ = problem("paper2d")
    M, N = s["M"], s["N"]
    prm = B.SolveParams(alpha=0.5, gamma=1.0, step_rule=B.STEP_FIXED, mu=mu, seed=5)
    _, x = gpu_run(gg, y, prm, 60)
    x_lit, _ = OB.bsgd_literal(og, y, OB.Params(M, N, 0.5, 1.0, mu, seed=5), 60)
    assert rel_l2(x.cpu().double().numpy(), x_lit) <= 1e-5


@pytest.mark.parametrize("kM,kN", [(1, 2), (2, 2), (1, 3), (1, 4), (2, 4)])
def test_several_column_blocks_fused_pass(kM, kN):
    """kN column blocks per iteration (uniform draws, no cells) run FP,
    residual and BP in one pass over the bounding box of the drawn blocks'
    bands: the same trajectory as the FP64 oracle, and as the split path
    (FP pass, residual pass, BP pass) up to the order of the float atomics."""
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    iters = 3 * (M // kM) * (N // kN)
    out = []
    for split in (False, True):
        prm = B.SolveParams(alpha=kM / M, gamma=kN / N, step_rule=B.STEP_FIXED, mu=mu, seed=8)
        st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
        st.set_split(split)
        x = torch.zeros(gg.n_cols, device=DEV)
        st.profile(True)
        st.block_step(x, iters)
        prof = st.read_profile()
        out.append((x.cpu().double().numpy(), st.read_trace(iters), st.query(), prof))
    (xf, tf, qf, pf), (xs, ts, qs, ps) = out
    assert pf["fpbp"]["launches"] == iters and pf["fp"]["launches"] == 0 and pf["residual"]["launches"] == 0
    assert ps["fp"]["launches"] == iters and ps["fpbp"]["launches"] == 0
    assert np.array_equal(tf, ts) and np.all(tf[:, 0] == kM * kN)
    assert rel_l2(xf, xs) <= 1e-6
    assert qf["updates"] == qs["updates"]
    assert abs(qf["residual_norm"] - qs["residual_norm"]) <= 1e-6 * np.linalg.norm(y)
    ost = OB.bsgd(og, y, OB.Params(M, N, kM / M, kN / N, mu, seed=8), iters)
    assert rel_l2(xf, ost.x) <= 1e-5
    assert abs(qf["residual_norm"] - ost.residual_norm()) <= 1e-4 * np.linalg.norm(y)


@pytest.mark.parametrize("pairs,cells", [(B.PAIRS_UNIFORM, B.CELLS_GEOMETRIC),
                                         (B.PAIRS_UNIFORM, B.CELLS_UNIFORM),
                                         (B.PAIRS_RESIDUAL, B.CELLS_NONE),
                                         (B.PAIRS_RESIDUAL, B.CELLS_GEOMETRIC)])
def test_importance_sampling_replay_and_choices(pairs, cells):
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    iters = 48
    use_cells = cells != B.CELLS_NONE
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=3,
                        pair_sampling=pairs, cells=cells, n_cells=4 if use_cells else 1)
    st, x = gpu_run(gg, y, prm, iters)
    tr = st.read_trace(iters)
    names = {B.CELLS_NONE: "none", B.CELLS_GEOMETRIC: "geometric", B.CELLS_UNIFORM: "uniform"}
    po = OB.Params(M, N, 1 / M, 1 / N, mu, seed=3,
                   pair_sampling="uniform" if pairs == B.PAIRS_UNIFORM else "residual",
                   cells=names[cells], n_cells=4 if use_cells else 1)
    sels = oracle_replay(tr, 1, gg.info.max_views_per_block, M, og, po, use_cells)
    ost = OB.BSGDState(og, y, po)
    agree = total = 0
    for sel in sels:
        own = OB.sample(og, po, ost.it, ost.r, ost.bands, ost.cell_w)
        total += 1
        agree += own.pairs == sel.pairs and all(
            (a is None and b is None) or np.array_equal(a, b) for a, b in zip(own.cells, sel.cells))
        ost.step(sel)
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-5
    # FP32 vs FP64 weights may flip a draw that lands within rounding of a CDF step
    assert agree >= total - 1


def test_power_iteration_matches_oracle():
    s, og, gg, _, _, _ = problem("cone_small")
    for j in range(s["N"]):
        lam_g = B.bsgd_power_iteration(gg, j, 30)
        lam_o = OB.power_iteration(og, s["N"], j, 30)
        assert abs(lam_g - lam_o) <= 1e-5 * lam_o
    # STRIP rule inside the state: mu = rho / max_J lambda_J
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_STRIP, rho=RHO, power_iters=30)
    st = B.State(gg, prm, torch.zeros(gg.n_rows, device=DEV))
    assert abs(st.query()["mu"] - problem("cone_small")[4]) <= 1e-5 * problem("cone_small")[4]


def test_device_replay_of_a_recorded_trace():
    """bsgd_state_set_replay: a second state consuming the first one's trace
    (residual pairs with geometric cells, then two column blocks per iteration)
    takes the same blocks and cells and gives the same image; iterations after
    the replayed ones sample again."""
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    for prm in (B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=14,
                              pair_sampling=B.PAIRS_RESIDUAL, cells=B.CELLS_GEOMETRIC, n_cells=4),
                B.SolveParams(alpha=1 / M, gamma=2 / N, step_rule=B.STEP_FIXED, mu=mu, seed=15)):
        a, xa = gpu_run(gg, y, prm, 30)
        ta = a.read_trace(30)
        other = B.SolveParams(**{**prm.__dict__, "seed": prm.seed + 100})
        b = B.State(gg, other, torch.from_numpy(y.astype(np.float32)).to(DEV))
        b.set_replay(ta[:20])
        xb = torch.zeros(gg.n_cols, device=DEV)
        b.block_step(xb, 20)
        torch.cuda.synchronize()
        assert np.array_equal(b.read_trace(20), ta[:20])
        xa20 = gpu_run(gg, y, prm, 20)[1]
        assert rel_l2(xb.cpu().double().numpy(), xa20.cpu().double().numpy()) <= 1e-6
        b.block_step(xb, 10)       # past the replayed part: b's own seed draws
        torch.cuda.synchronize()
        assert not np.array_equal(b.read_trace(30)[20:], ta[20:])


def test_block_step_rule_matches_oracle():
    """BSGD_STEP_BLOCK: mu = rho / max over (row block, column block) of the
    power-iteration estimate of ||A_(I_i)^(J_j)||^2, against the oracle's power
    iteration restricted to each row block's views; per-pair estimates through
    bsgd_power_iteration's row-block list as well."""
    s, og, gg, _, _, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    lam = np.zeros((M, N))
    for i in range(M):
        views = OP.row_block_views(og, M, i)
        for j in range(N):
            lam[i, j] = OB.power_iteration(og, N, j, 20, views=views)
            got = B.bsgd_power_iteration(gg, j, 20, row_blocks=[i])
            assert abs(got - lam[i, j]) <= 1e-5 * lam[i, j]
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_BLOCK, rho=RHO, power_iters=20)
    st = B.State(gg, prm, torch.zeros(gg.n_rows, device=DEV))
    mu = RHO / lam.max()
    assert abs(st.query()["mu"] - mu) <= 1e-5 * mu
    # the estimate is kept with the geometry: a second state takes the same mu
    st2 = B.State(gg, B.SolveParams(**{**prm.__dict__, "rho": 2 * RHO}),
                  torch.zeros(gg.n_rows, device=DEV))
    assert st2.query()["mu"] == 2 * st.query()["mu"]
    # a row block sees part of the strip: its norm is below the strip's
    strip = max(OB.power_iteration(og, N, j, 20) for j in range(N))
    assert lam.max() < strip


@pytest.mark.parametrize("name", ["config1", "cone_small"])
def test_tv_prox_matches_oracle(name):
    s, og, gg, _, _, xt = problem(name)
    b = xt + 0.1 * synth.normal_array(og.n_cols, 21)
    kappa = 0.05
    xg = torch.from_numpy(b.astype(np.float32)).to(DEV)
    B.bsgd_tv_prox(gg, xg, kappa, 20)
    shape = og.vol_shape if og.nz > 1 else (og.ny, og.nx)
    ref = OT.tv_prox(b.astype(np.float32).astype(np.float64).reshape(shape), kappa, 20).reshape(-1)
    assert rel_l2(xg.cpu().double().numpy(), ref) <= 1e-5


def test_tv_prox_ragged_volume_matches_oracle():
    """A 37 x 29 x 19 volume: sides that are no multiple of the fused FGP
    pass's 32 x 8 columns, and a depth that splits into z-chunks of 10 and 9
    planes (each chunk recomputes u of the plane below it). The halo, edge and
    chunk-boundary handling against the oracle's prox."""
    gg = B.Geometry(M=1, N=1, kind="cone3d", nx=37, ny=29, nz=19, dx=1.0, dy=1.0, dz=1.0, n_views=4,
                    nu=16, nv=16, du=4.0, dv=4.0, dso=100.0, dsd=200.0)
    b = np.random.default_rng(5).random(37 * 29 * 19).astype(np.float32)
    kappa = 0.05
    xg = torch.from_numpy(b).to(DEV)
    B.bsgd_tv_prox(gg, xg, kappa, 20)
    ref = OT.tv_prox(b.astype(np.float64).reshape(19, 29, 37), kappa, 20).reshape(-1)
    assert rel_l2(xg.cpu().double().numpy(), ref) <= 1e-5
    gg.close()


def test_bsgd_tv_matches_oracle():
    """Algorithm 4: the prox runs after every 1/(alpha gamma) iterations."""
    s, og, gg, y, mu, _ = problem("config1")
    M, N = s["M"], s["N"]
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_FIXED, mu=mu, seed=2,
                        tv_lambda=2.0, tv_iters=10)
    _, x = gpu_run(gg, y, prm, 48)
    ost = OB.bsgd(og, y, OB.Params(M, N, 0.25, 0.25, mu, seed=2, tv_lambda=2.0, tv_iters=10), 48)
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-5


@pytest.mark.parametrize("storage", [B.F32, B.BF16])
def test_bsgd_tv_volume_matches_oracle(storage):
    """Algorithm 4 on a volume (3D TV), with FP32 storage and with BF16
    storage, where the prox reads and writes the image with its low-order
    term: within 1e-5 (FP32) and 1e-2 (BF16) of the FP64 oracle."""
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    tdt = torch.bfloat16 if storage == B.BF16 else torch.float32
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=3,
                        tv_lambda=0.5, tv_iters=10, storage=storage)
    _, x = gpu_run(gg, y, prm, 48, storage=tdt)
    ost = OB.bsgd(og, y, OB.Params(M, N, 1 / M, 1 / N, mu, seed=3, tv_lambda=0.5, tv_iters=10), 48)
    assert rel_l2(x.float().cpu().double().numpy(), ost.x) <= (1e-5 if storage == B.F32 else 1e-2)


@pytest.mark.parametrize("storage", [B.BF16, B.F16])
def test_reduced_precision_storage(storage):
    """Sinogram, image and solver state stored in BF16 / FP16 with FP32 ray sums
    and accumulation: within 1e-2 of the FP64 oracle after 50 epochs."""
    s, og, gg, y, mu, _ = problem("config1")
    M, N = s["M"], s["N"]
    iters = 50 * 16
    tdt = torch.bfloat16 if storage == B.BF16 else torch.float16
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_FIXED, mu=mu, seed=1,
                        storage=storage)
    _, x = gpu_run(gg, y, prm, iters, storage=tdt)
    ost = OB.bsgd(og, y, OB.Params(M, N, 0.25, 0.25, mu, seed=1), iters)
    assert rel_l2(x.float().cpu().double().numpy(), ost.x) <= 1e-2


def test_switching_between_fused_and_split_passes():
    """One state alternates the multi-block fused pass and the split passes
    between block_step calls (they share z, r~, r, S and the draws): the
    trajectory is the oracle's."""
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    prm = B.SolveParams(alpha=1 / M, gamma=2 / N, step_rule=B.STEP_FIXED, mu=mu, seed=12)
    st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.profile(True)
    for split in (False, True, False, True):
        st.set_split(split)
        st.block_step(x, 5)
    torch.cuda.synchronize()
    prof = st.read_profile()
    assert prof["fpbp"]["launches"] == 10 and prof["fp"]["launches"] == 10
    ost = OB.bsgd(og, y, OB.Params(M, N, 1 / M, 2 / N, mu, seed=12), 20)
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-5
    assert abs(st.query()["residual_norm"] - ost.residual_norm()) <= 1e-4 * np.linalg.norm(y)


@pytest.mark.parametrize("kM,kN,cells", [(1, 2, B.CELLS_GEOMETRIC), (1, 4, B.CELLS_GEOMETRIC),
                                           (2, 2, B.CELLS_UNIFORM)])
def test_several_column_blocks_with_cells(kM, kN, cells):
    """Algorithm 2's detector cells with several column blocks per iteration
    (the paper's BSGD-IM set-up draws 4 of 8 column blocks): the fused pass
    walks block j only for the rays of the cell drawn for pair (i, j). Same
    draws and image as the split path; the oracle replaying the GPU's draws
    gives the same image."""
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    iters = 2 * (M // kM) * (N // kN)
    out = []
    for split in (False, True):
        prm = B.SolveParams(alpha=kM / M, gamma=kN / N, step_rule=B.STEP_FIXED, mu=mu, seed=6,
                            cells=cells, n_cells=4)
        st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
        st.set_split(split)
        x = torch.zeros(gg.n_cols, device=DEV)
        st.profile(True)
        st.block_step(x, iters)
        prof = st.read_profile()
        out.append((x.cpu().double().numpy(), st.read_trace(iters), st.query(), prof))
    (xf, tf, qf, pf), (xs, ts, qs, ps) = out
    assert pf["fpbp"]["launches"] == iters and ps["fp"]["launches"] == iters
    assert np.array_equal(tf, ts)
    assert rel_l2(xf, xs) <= 1e-6 and qf["updates"] == qs["updates"]
    names = {B.CELLS_GEOMETRIC: "geometric", B.CELLS_UNIFORM: "uniform"}
    po = OB.Params(M, N, kM / M, kN / N, mu, seed=6, cells=names[cells], n_cells=4)
    sels = oracle_replay(tf, kM * kN, gg.info.max_views_per_block, M, og, po, True)
    assert all(len(sel.pairs) == kM * kN for sel in sels)
    ost = OB.BSGDState(og, y, po)
    for sel in sels:
        ost.step(sel)
    assert rel_l2(xf, ost.x) <= 1e-5


@pytest.mark.parametrize("storage", [B.BF16, B.F16])
def test_reduced_precision_several_column_blocks(storage):
    """16-bit storage through the multi-block fused pass (alpha = 1/4, gamma =
    2/4 on the small cone beam): the fused and the split path round z, r and
    r~ at the same points, so they agree to the order of the float atomics,
    and both stay within 1e-2 of the FP64 oracle."""
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    iters = 3 * 8
    tdt = torch.bfloat16 if storage == B.BF16 else torch.float16
    xs = []
    for split in (False, True):
        prm = B.SolveParams(alpha=1 / M, gamma=2 / N, step_rule=B.STEP_FIXED, mu=mu, seed=2,
                            storage=storage)
        st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
        st.set_split(split)
        x = torch.zeros(gg.n_cols, device=DEV, dtype=tdt)
        st.block_step(x, iters)
        torch.cuda.synchronize()
        xs.append(x.float().cpu().double().numpy())
    ost = OB.bsgd(og, y, OB.Params(M, N, 1 / M, 2 / N, mu, seed=2), iters)
    assert rel_l2(xs[0], xs[1]) <= 1e-3
    assert rel_l2(xs[0], ost.x) <= 1e-2


def test_solve_with_host_buffers_equals_block_steps():
    s, og, gg, y, mu, _ = problem("config1")
    prm = B.SolveParams(alpha=0.25, gamma=0.25, epochs=3, step_rule=B.STEP_FIXED, mu=mu, seed=4)
    yh = y.astype(np.float32)
    xh = np.zeros(og.n_cols, dtype=np.float32)
    rep = B.bsgd_solve(gg, prm, yh, xh)
    _, x = gpu_run(gg, y, prm, 3 * 16)
    assert rep["iteration"] == 48
    assert rel_l2(xh, x.cpu().numpy()) <= 1e-6


def test_config2_first_iteration():
    """Config 2 at full size (256^3, 360 x 256^2, 8 x 8 blocks, residual-weighted
    pairs) in the bench's launch shape. From x = 0 the first iteration gives
    x_J = mu (A_I^J)^T y for the drawn pair: checked on every voxel of the slab."""
    s = spec("config2")
    og, gg = oracle_geom(s), gpu_geom(s)
    rng = np.random.default_rng(0)
    y = np.abs(rng.standard_normal(og.n_rows)).astype(np.float32)
    mu = 1e-6
    prm = B.SolveParams(alpha=1 / 8, gamma=1 / 8, step_rule=B.STEP_FIXED, mu=mu, seed=9,
                        pair_sampling=B.PAIRS_RESIDUAL)
    st, x = gpu_run(gg, y.astype(np.float64), prm, 1)
    tr = st.read_trace(1)
    i, j = int(tr[0, 1]), int(tr[0, 2])
    rows = OP.rows_of_views(og, OP.row_block_views(og, 8, i))
    blk = OP.column_block(og, 8, j)
    vox = OP.column_block_voxels(og, 8, j)
    ref = mu * OP.bp_rows(og, y[rows].astype(np.float64), rows, blk)[vox]
    got = x.cpu().double().numpy()
    assert rel_l2(got[vox], ref) <= 1e-5
    other = np.setdiff1d(np.arange(og.n_cols), vox)
    assert not got[other].any()


@pytest.mark.parametrize("name,frac", [("cone_small", 1.0), ("config2", 0.35)])
def test_compact_band_storage(name, frac):
    """z^j and r~^j keep the rows of block j's band only: their length is the
    sum over (view, block) of the band areas, i.e. the rays of all pairs, and
    (for thin slabs) a small part of N full sinograms."""
    s = spec(name)
    gg = gpu_geom(s)
    M, N = s["M"], s["N"]
    assert gg.compact_rows == sum(gg.pair_rays(i, j) for i in range(M) for j in range(N))
    assert gg.compact_rows <= frac * N * gg.n_rows


def test_switch_to_whole_views_matches_oracle():
    """BSGD-IM (geometric cells, uniform pairs) for two epochs, then the
    iterations after Algorithm 2's suggestion: whole views, uniform pairs. The
    cell memories carry over (snapshot form), so the oracle replays the GPU's
    cells for the first phase and samples whole views for the second."""
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    k1, k2 = 32, 32
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=6,
                        pair_sampling=B.PAIRS_UNIFORM, cells=B.CELLS_GEOMETRIC, n_cells=4)
    st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, k1)
    st.set_sampling(B.PAIRS_UNIFORM, B.CELLS_NONE)
    st.block_step(x, k2)
    torch.cuda.synchronize()
    tr = st.read_trace(k1 + k2)
    assert (tr[k1:, 3:] == -1).all()                     # no cells after the switch
    po = OB.Params(M, N, 1 / M, 1 / N, mu, seed=6, cells="geometric", n_cells=4)
    ost = OB.BSGDState(og, y, po)
    for sel in oracle_replay(tr[:k1], 1, gg.info.max_views_per_block, M, og, po, True):
        ost.step(sel)
    import dataclasses
    ost.prm = dataclasses.replace(po, cells="none", n_cells=1)
    for _ in range(k2):
        ost.step()
    assert [h.pairs for h in ost.history[k1:]] == [
        [(int(t[1]), int(t[2]))] for t in tr[k1:]]
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-5


def test_solve_final_uniform_epochs_equals_manual_switch():
    s, og, gg, y, mu, _ = problem("cone_small")
    M, N = s["M"], s["N"]
    kw = dict(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=8,
              pair_sampling=B.PAIRS_RESIDUAL, cells=B.CELLS_GEOMETRIC, n_cells=4)
    xh = np.zeros(gg.n_cols, dtype=np.float32)
    B.bsgd_solve(gg, B.SolveParams(epochs=3, final_uniform_epochs=1, **kw), y.astype(np.float32), xh)
    st = B.State(gg, B.SolveParams(**kw), torch.from_numpy(y.astype(np.float32)).to(DEV))
    x = torch.zeros(gg.n_cols, device=DEV)
    st.block_step(x, 2 * M * N)
    st.set_sampling(B.PAIRS_UNIFORM, B.CELLS_NONE)
    st.block_step(x, M * N)
    assert rel_l2(xh, x.cpu().double().numpy()) <= 1e-5
    with pytest.raises(B.BSGDError):
        B.State(gg, B.SolveParams(alpha=2 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu),
                torch.from_numpy(y.astype(np.float32)).to(DEV)).set_sampling(B.PAIRS_RESIDUAL, B.CELLS_NONE)


# --------------------------------------------------------------------------
# Starting image x0 != 0 (the first block step sets z^j = A^j x0_J and
# r = y - sum_j z^j before its first iteration)

def warm_x0(og, xt, seed):
    return (0.5 * xt + 0.05 * synth.normal_array(og.n_cols, seed)).astype(np.float32)


def test_warm_start_one_call_solve_matches_oracle():
    """Config 1 through bsgd_solve with host buffers, x holding x0 on entry:
    three epochs of uniform draws (the same on both sides) against the oracle
    started at the same x0."""
    s, og, gg, y, mu, xt = problem("config1")
    M, N = s["M"], s["N"]
    x0 = warm_x0(og, xt, 31)
    prm = B.SolveParams(alpha=0.25, gamma=0.25, epochs=3, step_rule=B.STEP_FIXED, mu=mu, seed=3)
    xh = x0.copy()
    rep = B.bsgd_solve(gg, prm, y.astype(np.float32), xh)
    ost = OB.bsgd(og, y, OB.Params(M, N, 0.25, 0.25, mu, seed=3), 48, x0=x0.astype(np.float64))
    assert rep["iteration"] == 48
    assert rel_l2(xh, ost.x) <= 1e-5
    assert abs(rep["residual_norm"] - ost.residual_norm()) <= 1e-5 * np.linalg.norm(y)
    # the start mattered: from zero the same draws end elsewhere
    assert rel_l2(OB.bsgd(og, y, OB.Params(M, N, 0.25, 0.25, mu, seed=3), 48).x, ost.x) > 1e-3


@pytest.mark.parametrize("extra", [dict(auto_mu=True), dict(tv_lambda=0.02, tv_iters=10)])
def test_warm_start_with_auto_mu_or_tv_matches_oracle(extra):
    """The start from x0 combined with Algorithm 3 (whose first residual norm
    is the warm start's) and with Algorithm 4 (the prox after every epoch):
    config 1, four epochs of uniform draws, against the oracle from the same
    x0; Algorithm 3's step decisions agree."""
    s, og, gg, y, mu, xt = problem("config1")
    M, N = s["M"], s["N"]
    x0 = warm_x0(og, xt, 34)
    mu0 = 2.0 * mu if extra.get("auto_mu") else mu
    prm = B.SolveParams(alpha=0.25, gamma=0.25, epochs=4, step_rule=B.STEP_FIXED, mu=mu0, seed=5,
                        auto_window=1 if extra.get("auto_mu") else 0, **extra)
    xh = x0.copy()
    rep = B.bsgd_solve(gg, prm, y.astype(np.float32), xh)
    okw = dict(extra)
    if extra.get("auto_mu"):
        okw["auto_window"] = 1
    ost = OB.bsgd(og, y, OB.Params(M, N, 0.25, 0.25, mu0, seed=5, **okw), 64,
                  x0=x0.astype(np.float64))
    assert rel_l2(xh, ost.x) <= 1e-5
    assert rep["mu"] == pytest.approx(ost.mu, rel=1e-9)


@pytest.mark.parametrize("storage", [torch.float32, torch.bfloat16])
def test_warm_start_block_steps_match_oracle(storage):
    """cone_small, residual-weighted pairs with geometric cells: a state whose
    first block step is given x0; the oracle, started at the same x0 (rounded
    to the storage type), replays the GPU's draws. FP32 within 1e-5, BF16
    storage within 1e-2."""
    s, og, gg, y, mu, xt = problem("cone_small")
    M, N = s["M"], s["N"]
    code = B.F32 if storage == torch.float32 else B.BF16
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=17,
                        pair_sampling=B.PAIRS_RESIDUAL, cells=B.CELLS_GEOMETRIC, n_cells=4,
                        storage=code)
    x0 = torch.from_numpy(warm_x0(og, xt, 32)).to(DEV).to(storage)
    iters = 24
    st, x = gpu_run(gg, y, prm, iters, x=x0.clone())
    tr = st.read_trace(iters)
    po = OB.Params(M, N, 1 / M, 1 / N, mu, seed=17, pair_sampling="residual", cells="geometric",
                   n_cells=4)
    sels = oracle_replay(tr, 1, gg.info.max_views_per_block, M, og, po, True)
    ost = OB.bsgd(og, y, po, iters, x0=x0.float().cpu().double().numpy(), replay=sels)
    tol = 1e-5 if storage == torch.float32 else 1e-2
    assert rel_l2(x.float().cpu().numpy(), ost.x) <= tol
    assert abs(st.query()["residual_norm"] - ost.residual_norm()) <= tol * ost.residual_norm()


def test_zero_start_does_not_read_x():
    """zero_start = 1: bsgd_solve starts from x0 = 0 whatever x holds."""
    s, og, gg, y, mu, _ = problem("config1")
    kw = dict(alpha=0.25, gamma=0.25, epochs=2, step_rule=B.STEP_FIXED, mu=mu, seed=4)
    xa = np.zeros(og.n_cols, dtype=np.float32)
    B.bsgd_solve(gg, B.SolveParams(**kw), y.astype(np.float32), xa)
    xb = synth.normal_array(og.n_cols, 33).astype(np.float32)
    B.bsgd_solve(gg, B.SolveParams(zero_start=True, **kw), y.astype(np.float32), xb)
    assert rel_l2(xb, xa) <= 1e-6
