"""GPU parity of Algorithm 3 (automatic step length) against the FP64 oracle.

Uniform sampling draws the same blocks on both sides, so the two runs take the
same decisions: the step after every window must match exactly (it is mu0
times a product of (1 + eps) and (1 - delta) factors), and the residual norms
and the image follow the oracle within the FP32 trajectory tolerance.
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
    """Sec. 3.1 set-up (fan beam, 16^2, 36 views, 30 elements, SNR 17.5 dB)
    with 4 x 4 blocks; y rounded to FP32 for both sides."""
    if "p" not in _CACHE:
        s = spec("paper2d", N=4)
        og, gg = oracle_geom(s), gpu_geom(s)
        A = OP.dense_matrix(og)
        x_true = synth.ellipse_phantom(16, 16, 6, 0).reshape(-1)
        y = synth.gaussian_noise_at_snr(A @ x_true, 17.5, 1).astype(np.float32).astype(np.float64)
        _CACHE["p"] = (og, gg, y, OB.step_strip(og, 4))
    return _CACHE["p"]


@pytest.mark.parametrize("rho,windows", [(0.25, 8), (2.0, 16)])
def test_auto_mu_matches_oracle(rho, windows):
    """rho = 0.25: the residual falls, mu grows by 1.1 per window; rho = 2:
    fixed-step BSGD diverges, the tuner cuts the step and recovers."""
    og, gg, y, base = problem()
    mu0 = rho * base
    ost = OB.BSGDState(og, y, OB.Params(4, 4, 0.25, 0.25, mu0, seed=2, auto_mu=True))
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_FIXED, mu=mu0, seed=2, auto_mu=True)
    st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
    x = torch.zeros(gg.n_cols, device=DEV)
    per = 16 * 4                       # epochs of 16 iterations, a test every M = 4 epochs
    mus, rn_gpu, rn_orc = [], [], []
    for _ in range(windows):
        st.block_step(x, per)
        for _ in range(per):
            ost.step()
        q = st.query()
        mus.append(q["mu"])
        rn_gpu.append(q["residual_norm"])
        rn_orc.append(ost.residual_norm())
    np.testing.assert_allclose(mus, ost.tuner.mu_log, rtol=1e-12)
    np.testing.assert_allclose(rn_gpu, rn_orc, rtol=1e-4)
    assert rel_l2(x.cpu().double().numpy(), ost.x) <= 1e-4
    if rho > 1:
        assert min(mus) < 0.5 * mu0
    else:
        assert mus[-1] == pytest.approx(mu0 * 1.1 ** (windows - 1), rel=1e-12)


def test_one_call_solve_takes_the_same_steps():
    og, gg, y, base = problem()
    prm = B.SolveParams(alpha=0.25, gamma=0.25, epochs=24, step_rule=B.STEP_FIXED, mu=2 * base,
                        seed=2, auto_mu=True)
    st = B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
    st.block_step(torch.zeros(gg.n_cols, device=DEV), 24 * 16)
    xh = np.zeros(gg.n_cols, dtype=np.float32)
    rep = B.bsgd_solve(gg, prm, y.astype(np.float32), xh)
    assert rep["mu"] == pytest.approx(st.query()["mu"], rel=1e-12)
    assert rep["mu"] != 2 * base


@pytest.mark.parametrize("bad", [dict(auto_eps=0.0), dict(auto_delta=1.0), dict(auto_delta=0.0),
                                 dict(auto_t1=0.0), dict(auto_window=-1), dict(tv_lambda=1e-3)])
def test_argument_checks(bad):
    og, gg, y, base = problem()
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_FIXED, mu=base, auto_mu=True, **bad)
    with pytest.raises(B.BSGDError) as ei:
        B.State(gg, prm, torch.from_numpy(y.astype(np.float32)).to(DEV))
    assert ei.value.status == 1


def test_not_served():
    geo = dict(kind="cone3d", nx=32, ny=32, nz=32, dx=1.0, dy=1.0, dz=1.0, n_views=24, nu=32,
               nv=32, du=1.6, dv=1.6, dso=500.0, dsd=1000.0)
    prm = B.SolveParams(alpha=0.25, gamma=0.25, step_rule=B.STEP_FIXED, mu=1e-3, auto_mu=True)
    srv = B.Server(budget_bytes=1 << 30, max_slots=2)
    try:
        with pytest.raises(B.BSGDError) as ei:
            srv.submit(geo, 4, 4, prm, np.zeros(24 * 32 * 32, np.float32))
        assert ei.value.status == 1
    finally:
        srv.close()
