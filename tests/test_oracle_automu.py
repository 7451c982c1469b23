"""Oracle pins for Algorithm 3 (automatic step length).

The tuner is a heuristic, so what is pinned is its stated rule and its stated
purpose: the decision table of Algorithm 3 on hand-made residual / cosine
sequences, the effective update direction as the direction the window's
updates applied (Delta x / mu), geometric growth of mu while the residual falls,
and recovery from a step that makes fixed-step BSGD diverge (Sec. 5, Fig. auto).
"""
import numpy as np
import pytest

from oracle import bsgd as B
from oracle import projector as P
from paper_1903_11874_gb300 import synth


def tuner():
    return B.AutoMu(window=4, eps=0.1, delta=0.4, t1=0.2, t2=0.5, rho0=1.0, n_cols=3)


@pytest.mark.parametrize("rho,theta,theta_prev,factor", [
    ((3.0, 2.0, 1.0), 0.9, 0.9, 1.1),      # residual fell twice: grow
    ((3.0, 2.0, 1.0), -1.0, 0.9, 1.1),     # ... whatever the cosines
    ((1.0, 2.0, 3.0), 0.9, 0.85, 1.0),     # rose twice, directions steady: keep
    ((1.0, 2.0, 3.0), 0.4, 0.45, 0.6),     # rose twice, cosine below t2: shrink
    ((1.0, 2.0, 3.0), 0.9, 0.6, 0.6),      # rose twice, cosine jumped by > t1: shrink
    ((1.0, 2.0, 3.0), 0.9, None, 1.0),     # second cosine not defined yet
    ((1.0, 2.0, 3.0), None, None, 1.0),    # no cosine yet
    ((1.0, 3.0, 2.0), 0.1, 0.9, 1.0),      # not monotone: keep
    ((3.0, 1.0, 2.0), 0.1, 0.9, 1.0),
    ((2.0, 2.0, 1.0), 0.9, 0.9, 1.0),      # ties are not a decrease
])
def test_decision_table(rho, theta, theta_prev, factor):
    assert tuner().decide(2.0, rho, theta, theta_prev) == pytest.approx(2.0 * factor, rel=1e-15)


def test_cosine():
    a = np.array([1.0, 2.0, -2.0])
    assert B.AutoMu.cosine(a, 3 * a) == pytest.approx(1.0)
    assert B.AutoMu.cosine(a, -a) == pytest.approx(-1.0)
    assert B.AutoMu.cosine(a, np.array([2.0, -1.0, 0.0])) == pytest.approx(0.0, abs=1e-15)
    assert B.AutoMu.cosine(a, np.zeros(3)) == 1.0


_CACHE = {}


def problem():
    """The paper's 2D set-up of Sec. 3.1 (fan beam, 16 x 16, 36 views of 30
    elements, SNR 17.5 dB), its LS residual norm, and the strip step bound."""
    if "p" not in _CACHE:
        geom = P.Geometry("fan2d", 16, 16, 1, 1.0, 1.0, 1.0, 36, 30, 1, 1.0, 1.0, dso=50.0, dsd=100.0)
        A = P.dense_matrix(geom)
        x_true = synth.ellipse_phantom(16, 16, 6, 0).reshape(-1)
        y = synth.gaussian_noise_at_snr(A @ x_true, 17.5, 1)
        x_ls = np.linalg.lstsq(A, y, rcond=None)[0]
        _CACHE["p"] = (geom, y, float(np.linalg.norm(y - A @ x_ls)), B.step_strip(geom, 4))
    return _CACHE["p"]


def run(rho, auto, windows, seed=2):
    geom, y, _, base = problem()
    prm = B.Params(4, 4, 0.25, 0.25, rho * base, seed=seed, auto_mu=auto)
    st = B.BSGDState(geom, y, prm)
    rn, xs = [st.residual_norm()], [st.x.copy()]
    for _ in range(windows):
        for _ in range(prm.epoch_len * 4):
            st.step()
        rn.append(st.residual_norm())
        xs.append(st.x.copy())
    return st, np.array(rn), xs


def test_eud_is_the_applied_direction():
    """A window's effective update direction is what its updates applied:
    gbar = (x_end - x_start) / mu while mu is unchanged within the window."""
    st, _, xs = run(0.25, True, 1)
    mu0 = st.prm.mu
    np.testing.assert_allclose(st.tuner.eud_prev, (xs[1] - xs[0]) / mu0, rtol=0,
                               atol=1e-10 * np.abs(st.tuner.eud_prev).max())
    assert st.tuner.theta == [None] and st.tuner.mu_log == [mu0]


def test_mu_grows_geometrically_while_the_residual_falls():
    st, rn, _ = run(0.25, True, 6)
    mu0 = st.prm.mu
    assert np.all(np.diff(rn) < 0)                       # residual falls every window
    expect = [mu0] + [mu0 * 1.1 ** e for e in range(1, 6)]
    np.testing.assert_allclose(st.tuner.mu_log, expect, rtol=1e-14)


def test_recovers_from_a_step_that_diverges():
    """Sec. 5 (Fig. auto): with twice the strip step, fixed-step BSGD diverges;
    with Algorithm 3 the step is cut and the residual returns to the LS level."""
    _, _, rls, _ = problem()
    _, rn_fixed, _ = run(2.0, False, 25)
    st, rn_auto, _ = run(2.0, True, 25)
    assert rn_fixed[-1] > 100 * rn_fixed[0]
    assert min(st.tuner.mu_log) < 0.5 * st.prm.mu        # the step was cut
    assert rn_auto[-1] < 1.02 * rls
