"""Pins of the oracle's sampling spec and TV prox (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import rng, tv
from paper_1903_11874_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    gold = json.load(open(os.path.join(GOLDEN, "splitmix64_seed0.json")))
    got = [rng.splitmix64(gold["seed"], n) for n in (1, 2, 3)]
    assert got == [int(h, 16) for h in gold["outputs_hex"]]


def test_uniform_draws_in_unit_interval_and_lane_independent():
    us = [rng.uniform(7, it, lane) for it in range(50) for lane in range(20)]
    assert all(0.0 <= u < 1.0 for u in us)
    assert len(set(us)) == len(us)
    assert abs(np.mean(us) - 0.5) < 0.03


def _chi2_ok(counts, probs, n):
    exp = np.asarray(probs) * n
    chi2 = float(((np.asarray(counts) - exp) ** 2 / exp).sum())
    dof = len(counts) - 1
    return chi2 < dof + 6.0 * math.sqrt(2.0 * dof)      # far tail of chi2(dof)


def test_choose_k_of_n_uniform_over_subsets():
    n, k, draws = 5, 2, 20000
    counts = {}
    for it in range(draws):
        s = tuple(rng.choose_k_of_n(3, it, rng.LANE_ROWS, n, k))
        assert len(set(s)) == k and list(s) == sorted(s)
        counts[s] = counts.get(s, 0) + 1
    assert len(counts) == math.comb(n, k)
    c = np.array(list(counts.values()))
    assert _chi2_ok(c, np.full(c.size, 1.0 / c.size), draws)


def test_choose_weighted_frequencies():
    w = np.array([0.5, 0.0, 2.0, 1.0, 0.25])
    draws = 20000
    counts = np.zeros(w.size)
    for it in range(draws):
        counts[rng.choose_weighted(rng.uniform(9, it, 0), w)] += 1
    assert counts[1] == 0
    nz = w > 0
    assert _chi2_ok(counts[nz], w[nz] / w.sum(), draws)


def test_choose_weighted_boundaries():
    w = [1.0, 1.0, 2.0]
    assert rng.choose_weighted(0.0, w) == 0
    assert rng.choose_weighted(0.25, w) == 1          # u*total = 1.0 = cdf[0]: next
    assert rng.choose_weighted(0.4999, w) == 1
    assert rng.choose_weighted(0.5, w) == 2
    assert rng.choose_weighted(0.9999999, w) == 2


# ---- TV (Algorithm 4, Eq. 10) ------------------------------------------------------

def test_tv_value_is_eq10():
    x = synth.normal_array((5, 7), 1)
    ref = 0.0
    for c in range(5):
        for d in range(7):
            dc = x[c, d] - x[c - 1, d] if c > 0 else 0.0
            dd = x[c, d] - x[c, d - 1] if d > 0 else 0.0
            ref += math.sqrt(dc * dc + dd * dd)
    assert abs(tv.tv_value(x) - ref) < 1e-12 * ref


@pytest.mark.parametrize("shape", [(6, 5), (4, 5, 3)])
def test_difference_operator_adjoint(shape):
    x = synth.normal_array(shape, 2)
    p = [synth.normal_array(shape, 3 + k) for k in range(len(shape))]
    lhs = sum(float((dk * pk).sum()) for dk, pk in zip(tv.grad_backward(x), p))
    rhs = float((x * tv.grad_backward_adjoint(p)).sum())
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_prox_two_pixel_closed_form():
    """1 x 2 image [a, b]: TV = |b - a|; the prox shrinks the jump by kappa on
    each side, or merges the pixels at their mean when |b - a| <= 2 kappa."""
    for a, b, kappa in [(0.0, 1.0, 0.2), (0.3, -0.9, 0.1), (0.2, 0.5, 0.4)]:
        out = tv.tv_prox(np.array([[a, b]]), kappa, n_iter=3000)
        if abs(b - a) <= 2 * kappa:
            exp = [(a + b) / 2] * 2
        else:
            s = math.copysign(1.0, b - a)
            exp = [a + kappa * s, b - kappa * s]
        np.testing.assert_allclose(out[0], exp, atol=1e-8)


def test_prox_identity_cases():
    const = np.full((6, 6), 0.7)
    np.testing.assert_allclose(tv.tv_prox(const, 0.5, 20), const, atol=1e-14)
    x = synth.normal_array((6, 6), 4)
    np.testing.assert_array_equal(tv.tv_prox(x, 0.0, 20), x)
    np.testing.assert_allclose(tv.tv_prox(x, 1e-9, 20), x, atol=1e-8)


@pytest.mark.parametrize("shape", [(12, 10), (6, 5, 7)])
def test_prox_duality_gap_closes(shape):
    b = synth.normal_array(shape, 5)
    kappa = 0.3
    gaps = []
    for n in (10, 100, 1000):
        _, p = tv.tv_prox(b, kappa, n, return_dual=True)
        gaps.append(tv.duality_gap(b, kappa, p))
    assert all(g >= -1e-9 for g in gaps)
    assert gaps[2] < gaps[1] < gaps[0]
    assert gaps[2] < 1e-3 * gaps[0]


def test_prox_minimises_against_brute_force():
    """3 x 3 image: no point found by a derivative-free search from several
    starts has a lower objective than the FGP result."""
    from scipy.optimize import minimize
    b = synth.normal_array((3, 3), 6)
    kappa = 0.25

    def obj(t):
        t = t.reshape(3, 3)
        return float(((t - b) ** 2).sum()) + 2 * kappa * tv.tv_value(t)

    t_fgp = tv.tv_prox(b, kappa, 5000)
    best = min(minimize(obj, b.reshape(-1) + 0.1 * synth.normal_array(9, 10 + s),
                        method="Powell", options={"xtol": 1e-10, "ftol": 1e-14,
                                                  "maxfev": 200000}).fun
               for s in range(4))
    assert obj(t_fgp.reshape(-1)) <= best + 1e-9
