"""Exact-FIRAL (Algorithm 1) with dense dc x dc matrices, float64 -- test infrastructure only.

Only for tiny inputs (d c up to a few hundred): every Hessian is formed
explicitly from its definition.  Notation follows Section 2 of the paper:
``H_i`` (eq. 2), ``H_o, H_p, H_z`` (eq. 3), ``f(z)`` (eqs. 4, 5), ``g_i``
(eq. 6), ``Sigma_z`` (eq. 7), the tilde transform (eq. 8) and the FTRL
matrices ``A_t`` (eqs. 9, 10).

Readings taken where the paper is loose (shared with the approximate oracle):
full c-class softmax with ``d~ = d c``; ``H_o`` = sum of the labelled
Hessians plus ``lam I``; ``H_p`` = pool *average*; ``z`` iterated on the
budget simplex (``sum z = b``); step size ``beta_t = beta0 / ||g_t||_inf``;
the Round step minimises the tilded objective of eq. 9 and never picks a
point twice; ties go to the lowest index.
"""
from itertools import combinations

import numpy as np

from .approx import nu_bisect, block_of


def hessian_dense(x, h):
    """Fisher matrix of one point, eq. 2: ``[diag(h) - h h^T] (x) (x x^T)`` (dc x dc).

    Row/column index ``k d + e`` matches ``vec`` stacking the columns of a d x c matrix.
    """
    x = np.asarray(x, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    return np.kron(np.diag(h) - np.outer(h, h), np.outer(x, x))


def hessian_sum(X, h, w):
    """``sum_i w_i H_i`` over the rows of X (eq. 3 with weights)."""
    d, c = X.shape[1], h.shape[1]
    out = np.zeros((d * c, d * c))
    for i in range(X.shape[0]):
        if w[i] != 0.0:
            out += w[i] * hessian_dense(X[i], h[i])
    return out


def h_o(prob):
    """``H_o``: labelled Hessians plus the ridge ``lam I`` (eq. 3)."""
    Xo = np.asarray(prob.Xo, np.float64)
    ho = np.asarray(prob.ho, np.float64)
    D = Xo.shape[1] * ho.shape[1]
    return hessian_sum(Xo, ho, np.ones(Xo.shape[0])) + prob.lam * np.eye(D)


def h_p(prob):
    """``H_p``: average Hessian of the unlabelled pool (eq. 3, scaled by 1/n)."""
    X = np.asarray(prob.X, np.float64)
    n = X.shape[0]
    return hessian_sum(X, np.asarray(prob.h, np.float64), np.full(n, 1.0 / n))


def sigma(prob, z, Ho=None):
    """``Sigma_z = H_o + H_z`` (eq. 7)."""
    Ho = h_o(prob) if Ho is None else Ho
    return Ho + hessian_sum(np.asarray(prob.X, np.float64), np.asarray(prob.h, np.float64),
                            np.asarray(z, np.float64))


def objective(prob, z, Ho=None, Hp=None):
    """``f(z) = Sigma_z^{-1} . H_p = Tr(Sigma_z^{-1} H_p)`` (eqs. 4, 5)."""
    S = sigma(prob, z, Ho)
    Hp = h_p(prob) if Hp is None else Hp
    return float(np.trace(np.linalg.solve(S, Hp)))


def gradient(prob, z, Ho=None, Hp=None):
    """``g_i = -H_i . Sigma_z^{-1} H_p Sigma_z^{-1}`` for every pool point (eq. 6)."""
    S = sigma(prob, z, Ho)
    Hp = h_p(prob) if Hp is None else Hp
    Sinv = np.linalg.inv(S)
    M = Sinv @ Hp @ Sinv
    X = np.asarray(prob.X, np.float64)
    h = np.asarray(prob.h, np.float64)
    return np.array([-np.sum(hessian_dense(X[i], h[i]) * M) for i in range(X.shape[0])])


def relax(prob, b, T, beta0=1.0, z0=None):
    """Exact Relax: entropic mirror descent on ``f`` (Algorithm 1, Relax part).

    ``z`` stays on the budget simplex ``{z >= 0, sum z = b}``; each step is
    ``z <- z exp(-beta_t g)``, ``z <- b z / sum(z)`` with ``beta_t = beta0/||g||_inf``.
    Returns ``(z, history)`` with the objective before every step.
    """
    n = prob.X.shape[0]
    Ho, Hp = h_o(prob), h_p(prob)
    z = np.full(n, b / n) if z0 is None else np.asarray(z0, np.float64).copy()
    hist = []
    for _ in range(T):
        hist.append(objective(prob, z, Ho, Hp))
        g = gradient(prob, z, Ho, Hp)
        beta = beta0 / np.max(np.abs(g))
        z = z * np.exp(-beta * g)
        z = b * z / z.sum()
    return z, hist


def _block_diagonal(M, d, c):
    """``B(M)``: keep the c diagonal d x d blocks of M (Definition 1)."""
    out = np.zeros_like(M)
    for k in range(c):
        sl = slice(k * d, (k + 1) * d)
        out[sl, sl] = M[sl, sl]
    return out


def round_exact(prob, z_diamond, b, eta=None, block_diag=False, exclude_selected=True,
                details=False):
    """Exact Round: FTRL greedy selection of ``b`` points (Algorithm 1, Round part).

    Each iteration picks ``argmin_i Tr[(A_t + eta/b H~_o + eta H~_i)^{-1}]``
    (eq. 9) with ``A_1 = sqrt(d~) I`` and ``A_{t+1} = nu I + eta H~_t``, ``nu``
    such that ``Tr(A^{-2}) = 1`` (eq. 10).  ``block_diag=True`` replaces every
    Hessian (``H_i``, ``H_o`` and ``Sigma_diamond``) by its block diagonal, the
    assumption under which Proposition 1 holds.  ``details=True`` also returns the
    minimised trace of every pick and the ``nu`` that defined ``A_t`` for it
    (``nu_1 = sqrt(d~)``).
    """
    X = np.asarray(prob.X, np.float64)
    h = np.asarray(prob.h, np.float64)
    n, d = X.shape
    c = h.shape[1]
    D = d * c
    eta = 8.0 * np.sqrt(D) if eta is None else eta
    bd = (lambda M: _block_diagonal(M, d, c)) if block_diag else (lambda M: M)
    Ho = bd(h_o(prob))
    Sd = bd(Ho + hessian_sum(X, h, np.asarray(z_diamond, np.float64)))
    ev, Q = np.linalg.eigh(Sd)
    Sm12 = (Q / np.sqrt(ev)) @ Q.T          # Sigma_diamond^{-1/2}
    tilde = lambda M: Sm12 @ M @ Sm12        # eq. 8
    Ho_t = tilde(Ho)
    Hi_t = [tilde(bd(hessian_dense(X[i], h[i]))) for i in range(n)]
    A = np.sqrt(D) * np.eye(D)
    Ht = np.zeros((D, D))
    chosen, r_pick, nus = [], [], [np.sqrt(D)]
    for _ in range(b):
        base = A + (eta / b) * Ho_t
        r = np.full(n, np.inf)
        for i in range(n):
            if exclude_selected and i in chosen:
                continue
            r[i] = np.trace(np.linalg.inv(base + eta * Hi_t[i]))
        it = int(np.argmin(r))
        chosen.append(it)
        r_pick.append(float(r[it]))
        Ht = Ht + Ho_t / b + Hi_t[it]
        lam, V = np.linalg.eigh(eta * Ht)
        nu = nu_bisect(lam)
        nus.append(float(nu))
        A = (V * (nu + lam)) @ V.T
    if details:
        return chosen, r_pick, nus[:b]
    return chosen


def subset_objective(prob, S, Ho=None, Hp=None):
    """``f(1_S)``: the integer objective of eq. 4 for the index set ``S``."""
    z = np.zeros(prob.X.shape[0])
    z[list(S)] = 1.0
    return objective(prob, z, Ho, Hp)


def brute_force_best(prob, b):
    """``min_{|S| = b} f(1_S)`` by enumeration (tiny pools only); returns (f*, S*)."""
    Ho, Hp = h_o(prob), h_p(prob)
    best = (np.inf, None)
    for S in combinations(range(prob.X.shape[0]), b):
        f = subset_objective(prob, S, Ho, Hp)
        if f < best[0]:
            best = (f, S)
    return best


def block_diag_of(M, d, c):
    """The c diagonal blocks of a dense dc x dc matrix, shape (c, d, d)."""
    return np.stack([block_of(M, k, d) for k in range(c)])
