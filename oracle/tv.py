"""TV proximal step of BSGD-TV in FP64 -- TEST INFRASTRUCTURE ONLY.

Algorithm 4 replaces x, once every 1/(alpha*gamma) iterations, by a TV
de-noising step argmin_t ||t - x||^2 + w TV(t), with the isotropic TV of
Eq. 10, built from backward differences x[c] - x[c - e_k].

The weight w: Algorithm 4 prints 2 mu lambda, with mu the step of a gradient
2 A^T r. The oracle folds that factor 2 into its step (its gradient is A^T r,
so its mu is twice the paper's) and uses w = 2 mu lambda in its own mu, which
is 4 mu lambda in the paper's: the weight of ISTA's proximal step for the
paper's objective, Eq. (TVequ), ||y - A x||^2 + 2 lambda TV(x) (equivalently
1/2 ||y - A x||^2 + lambda TV(x) with step mu). The printed weight is half of
that; the objective decides.

The paper does not say how the minimiser is found; the oracle uses FGP (Beck
and Teboulle 2009, the FISTA paper the text cites), whose problem statement
min ||t - b||^2 + 2 kappa TV(t) is this one with kappa = mu * lambda (mu in
the oracle's convention). Readings: a difference with a missing neighbour
(index 0 along that axis) is zero; 3D volumes use sqrt(dx^2 + dy^2 + dz^2); no
non-negativity constraint.
"""
import numpy as np


def grad_backward(x: np.ndarray):
    """D x: per axis k, x[c] - x[c - e_k], zero at index 0 along k."""
    out = []
    for k in range(x.ndim):
        d = np.zeros_like(x)
        sl_hi = [slice(None)] * x.ndim
        sl_lo = [slice(None)] * x.ndim
        sl_hi[k] = slice(1, None)
        sl_lo[k] = slice(0, -1)
        d[tuple(sl_hi)] = x[tuple(sl_hi)] - x[tuple(sl_lo)]
        out.append(d)
    return out


def grad_backward_adjoint(p):
    """D^T p, from <D x, p> = <x, D^T p>:
    (D^T p)[c] = sum_k p_k[c] [c_k >= 1] - p_k[c + e_k] [c_k <= n_k - 2]."""
    out = np.zeros_like(p[0])
    nd = out.ndim
    for k in range(nd):
        pk = p[k].copy()
        sl0 = [slice(None)] * nd
        sl0[k] = 0
        pk[tuple(sl0)] = 0.0
        out += pk
        sl_hi = [slice(None)] * nd
        sl_lo = [slice(None)] * nd
        sl_hi[k] = slice(1, None)
        sl_lo[k] = slice(0, -1)
        out[tuple(sl_lo)] -= pk[tuple(sl_hi)]
    return out


def tv_value(x: np.ndarray) -> float:
    """Isotropic TV of Eq. 10 (and its 3D extension)."""
    d = grad_backward(x)
    return float(np.sum(np.sqrt(sum(dk * dk for dk in d))))


def _project_unit(p):
    nrm = np.sqrt(sum(pk * pk for pk in p))
    scale = np.maximum(1.0, nrm)
    return [pk / scale for pk in p]


def tv_prox(b: np.ndarray, kappa: float, n_iter: int = 20, return_dual: bool = False):
    """FGP for argmin_t ||t - b||^2 + 2 kappa TV(t).

    Dual: t = b - kappa D^T p with |p[c]| <= 1. Projected gradient on the dual
    with step 1/(kappa L), L = 4 * ndim >= ||D||^2, plus FISTA momentum.
    """
    b = np.asarray(b, dtype=np.float64)
    if kappa <= 0.0:
        return (b.copy(), None) if return_dual else b.copy()
    L = 4.0 * b.ndim
    zeros = [np.zeros_like(b) for _ in range(b.ndim)]
    p_prev = [z.copy() for z in zeros]
    r = [z.copy() for z in zeros]
    t = 1.0
    for _ in range(n_iter):
        u = b - kappa * grad_backward_adjoint(r)
        du = grad_backward(u)
        p = _project_unit([rk + du_k / (kappa * L) for rk, du_k in zip(r, du)])
        t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        w = (t - 1.0) / t_next
        r = [pk + w * (pk - qk) for pk, qk in zip(p, p_prev)]
        p_prev, t = p, t_next
    out = b - kappa * grad_backward_adjoint(p_prev)
    return (out, p_prev) if return_dual else out


def duality_gap(b: np.ndarray, kappa: float, p) -> float:
    """Primal ||t - b||^2 + 2 kappa TV(t) at t = b - kappa D^T p minus the dual
    value ||b||^2 - ||b - kappa D^T p||^2 (>= 0 for feasible p)."""
    t = b - kappa * grad_backward_adjoint(p)
    primal = float(np.sum((t - b) ** 2)) + 2.0 * kappa * tv_value(t)
    dual = float(np.sum(b * b)) - float(np.sum(t * t))
    return primal - dual
