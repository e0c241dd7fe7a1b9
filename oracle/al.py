"""Multi-round active learning (the outer loop of Section 5), float64 -- test infrastructure only.

The paper's experiments alternate two steps for a fixed number of rounds: train the
multinomial logistic-regression classifier of eq. 1 on the labelled set, then select a batch
of ``b`` pool points with Relax + Round and reveal their labels.  This module restates that
loop on synthetic labels (the Gaussian-mixture component of each point):

* ``softmax_probs`` -- eq. 1, ``h_i = softmax(W x_i)`` with ``W`` of shape c x d;
* ``lr_loss`` / ``lr_gradient`` -- the ridge-regularised negative log-likelihood
  ``sum_i -log h_{i, y_i} + (gamma/2) ||W||_F^2`` and its gradient
  ``sum_i (h_i - e_{y_i}) x_i^T + gamma W``;
* ``lr_fit`` -- its minimiser by Newton's method with the dense Hessian
  ``sum_i H_i + gamma I`` (``H_i`` of eq. 2, from ``exact.hessian_sum``) and Armijo
  backtracking;
* ``active_learning`` -- the loop, with ``approx.relax`` and ``approx.round_select``.

Readings (the paper does not state them): the classifier is refit by
ridge-regularised maximum likelihood with its own ridge ``gamma`` (1.0 by default, the
usual unit-strength penalty), warm-started from the previous round's ``W`` (zero at first);
``H_o`` keeps the problem's ridge ``lam``; the labelled set is the initial rows followed by
the picks in selection order; the pool shrinks to the points not yet picked, in index order;
round ``r`` draws its Hutchinson probes with seed ``seed + r``.
"""
import numpy as np

from . import approx, exact


def softmax_probs(X, W):
    """``h_i = softmax(W x_i)`` for every row of X (eq. 1)."""
    L = np.asarray(X, np.float64) @ np.asarray(W, np.float64).T
    L = L - L.max(axis=1, keepdims=True)
    E = np.exp(L)
    return E / E.sum(axis=1, keepdims=True)


def lr_loss(X, y, W, gamma):
    """``sum_i -log softmax(W x_i)_{y_i} + (gamma/2) ||W||_F^2``."""
    h = softmax_probs(X, W)
    return float(-np.sum(np.log(h[np.arange(len(y)), y])) + 0.5 * gamma * np.sum(W * W))


def lr_gradient(X, y, W, gamma):
    """``sum_i (h_i - e_{y_i}) x_i^T + gamma W`` (c x d)."""
    X = np.asarray(X, np.float64)
    R = softmax_probs(X, W)
    R[np.arange(len(y)), y] -= 1.0
    return R.T @ X + gamma * W


def lr_fit(X, y, c, gamma, W0=None, iters=50, tol=1e-12):
    """Newton's method on ``lr_loss``: solve ``(sum_i H_i + gamma I) vec(dW) = vec(grad)``
    with the dense Hessian of eq. 2, backtrack until the Armijo condition holds.  The vec of
    a c x d matrix stacks its rows (index ``k d + e``), the layout of ``exact.hessian_dense``."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y)
    d = X.shape[1]
    W = np.zeros((c, d)) if W0 is None else np.asarray(W0, np.float64).copy()
    g0 = None
    for _ in range(iters):
        f = lr_loss(X, y, W, gamma)
        g = lr_gradient(X, y, W, gamma)
        gn = np.linalg.norm(g)
        g0 = gn if g0 is None else g0
        if gn <= tol * max(1.0, g0):
            break
        Hs = exact.hessian_sum(X, softmax_probs(X, W), np.ones(len(y))) + gamma * np.eye(c * d)
        dW = np.linalg.solve(Hs, g.reshape(-1)).reshape(c, d)
        gd = float(np.sum(g * dW))
        step = 1.0
        while lr_loss(X, y, W - step * dW, gamma) > f - 1e-4 * step * gd and step > 1e-12:
            step *= 0.5
        W = W - step * dW
    return W


class _Pool:
    """The Relax / Round problem of one round (the fields ``approx`` reads)."""

    def __init__(self, X, h, Xo, ho, lam):
        self.X, self.h, self.Xo, self.ho, self.lam = X, h, Xo, ho, lam


def active_learning(Xp, yp, Xl, yl, c, rounds, b, *, lam=1e-3, gamma=1.0, s=10, T=20,
                    seed=1, tol=0.1, maxit=100, fixed_iters=None, eta=None):
    """Run ``rounds`` rounds; returns ``(picks (rounds x b) pool indices, final W)`` where the
    final ``W`` is refit on the last labelled set."""
    Xp = np.asarray(Xp, np.float64)
    Xl = np.asarray(Xl, np.float64).reshape(-1, Xp.shape[1])
    yl = list(np.asarray(yl, np.int64))
    yp = np.asarray(yp, np.int64)
    remaining = list(range(Xp.shape[0]))
    W = np.zeros((c, Xp.shape[1]))
    picks = []
    for r in range(rounds):
        if len(yl):
            W = lr_fit(Xl, np.array(yl), c, gamma, W0=W)
        Xr = Xp[remaining]
        prob = _Pool(Xr, softmax_probs(Xr, W), Xl, softmax_probs(Xl, W), lam)
        z, _ = approx.relax(prob, b, s, T, seed + r, tol=tol, maxit=maxit,
                            fixed_iters=fixed_iters)
        local = approx.round_select(prob, z, b, eta=eta)
        chosen = [remaining[i] for i in local]
        picks.append(chosen)
        Xl = np.vstack([Xl, Xp[chosen]])
        yl.extend(int(yp[i]) for i in chosen)
        taken = set(chosen)
        remaining = [i for i in remaining if i not in taken]
    W = lr_fit(Xl, np.array(yl), c, gamma, W0=W)
    return np.array(picks), W
