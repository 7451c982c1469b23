"""Checkpoint / resume of a solver state (bsgd_state_save / bsgd_state_restore).

Every draw is a function of (seed, iteration), so a state restored from a
checkpoint and given the x of the save continues exactly as the uninterrupted
run: the same draws (bit-exact trace) and the same image up to the order of the
float atomics of the BP.
"""
import numpy as np
import pytest

from helpers import gpu_geom, oracle_geom, rel_l2, spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bsgd as OB  # noqa: E402
from oracle import projector as OP  # noqa: E402
from paper_1903_11874_gb300 import binding as B  # noqa: E402
from paper_1903_11874_gb300 import synth  # noqa: E402

DEV = "cuda:0"
_CACHE = {}


def problem():
    if not _CACHE:
        s = spec("cone_small")
        og, gg = oracle_geom(s), gpu_geom(s)
        xt = synth.ellipsoid_phantom(og.nx, og.ny, og.nz, 6, seed=0).astype(np.float64)
        y = OP.fp(og, xt.reshape(-1)).reshape(-1).astype(np.float32)
        mu = 0.25 * OB.step_strip(og, s["N"], 1.0, 30)
        _CACHE.update(s=s, gg=gg, y=y, mu=mu)
    return _CACHE["s"], _CACHE["gg"], _CACHE["y"], _CACHE["mu"]


def params(kind, M, N, mu):
    base = dict(step_rule=B.STEP_FIXED, mu=mu, seed=21)
    if kind == "residual":
        return B.SolveParams(alpha=1 / M, gamma=1 / N, pair_sampling=B.PAIRS_RESIDUAL, **base)
    if kind == "multi_cells":
        return B.SolveParams(alpha=1 / M, gamma=2 / N, cells=B.CELLS_GEOMETRIC, n_cells=4, **base)
    if kind == "bf16":
        return B.SolveParams(alpha=1 / M, gamma=1 / N, storage=B.BF16, **base)
    if kind == "auto_mu":
        return B.SolveParams(alpha=1 / M, gamma=1 / N, auto_mu=True, auto_window=1, **base)
    if kind == "tv":
        return B.SolveParams(alpha=1 / M, gamma=1 / N, tv_lambda=1e-3, tv_iters=10, **base)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["residual", "multi_cells", "bf16", "auto_mu", "tv"])
def test_resume_equals_uninterrupted(kind):
    s, gg, y, mu = problem()
    M, N = s["M"], s["N"]
    prm = params(kind, M, N, mu)
    xdt = torch.bfloat16 if kind == "bf16" else torch.float32
    k1, k2 = 23, 41                     # the save falls inside an epoch
    yd = torch.from_numpy(y).to(DEV)
    a = B.State(gg, prm, yd)
    x = torch.zeros(gg.n_cols, device=DEV, dtype=xdt)
    a.block_step(x, k1)
    blob = a.save()
    x_saved = x.clone()
    a.block_step(x, k2)
    torch.cuda.synchronize()
    qa, ta = a.query(), a.read_trace(k1 + k2)

    b = B.State(gg, prm, yd)
    b.restore(blob)
    xb = x_saved.clone()
    b.block_step(xb, k2)
    torch.cuda.synchronize()
    qb, tb = b.query(), b.read_trace(k1 + k2)
    assert np.array_equal(ta, tb)
    assert qb["iteration"] == qa["iteration"] == k1 + k2
    assert qb["updates"] == qa["updates"]
    assert qb["mu"] == pytest.approx(qa["mu"], rel=1e-12)
    assert rel_l2(xb.float().cpu().numpy(), x.float().cpu().numpy()) <= (2e-3 if kind == "bf16" else 1e-6)
    assert abs(qb["residual_norm"] - qa["residual_norm"]) <= 1e-5 * qa["residual_norm"]

    # rolling the first state back to the checkpoint gives the same run again
    a.restore(blob)
    xr = x_saved.clone()
    a.block_step(xr, k2)
    torch.cuda.synchronize()
    assert np.array_equal(a.read_trace(k1 + k2), ta)
    assert rel_l2(xr.float().cpu().numpy(), x.float().cpu().numpy()) <= (2e-3 if kind == "bf16" else 1e-6)


def test_restore_rejects_other_states():
    s, gg, y, mu = problem()
    M, N = s["M"], s["N"]
    yd = torch.from_numpy(y).to(DEV)
    a = B.State(gg, params("residual", M, N, mu), yd)
    a.block_step(torch.zeros(gg.n_cols, device=DEV), 5)
    blob = a.save()
    other_seed = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu, seed=22,
                               pair_sampling=B.PAIRS_RESIDUAL)
    with pytest.raises(B.BSGDError):
        B.State(gg, other_seed, yd).restore(blob)
    two_cols = B.SolveParams(alpha=1 / M, gamma=2 / N, step_rule=B.STEP_FIXED, mu=mu, seed=21)
    with pytest.raises(B.BSGDError):
        B.State(gg, two_cols, yd).restore(blob)
    with pytest.raises(B.BSGDError):
        B.State(gg, params("residual", M, N, mu), yd).restore(blob[: len(blob) // 2])
    with pytest.raises(B.BSGDError):
        B.State(gg, params("residual", M, N, mu), yd).restore(b"\0" * len(blob))
