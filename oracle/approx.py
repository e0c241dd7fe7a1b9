"""Approx-FIRAL (Algorithms 2 and 3), matrix-free, float64 -- test infrastructure only.

Each function restates one step of the paper in plain numpy:

* ``hessian_apply``  -- Lemma 1, summed over points with weights (the H_p / Sigma_z
  matvecs of Section 3.1);
* ``block_diag``     -- the block diagonal B_k(H_i) = h_i^k (1 - h_i^k) x_i x_i^T (eq. 13);
* ``pcg``            -- conjugate gradients with the block-Jacobi preconditioner
  B(Sigma_z)^{-1} (Algorithm 2, lines 5-8);
* ``grad_hutchinson`` -- the Hutchinson gradient estimator (eq. 11, Algorithm 2 line 9);
* ``md_step``        -- the entropic mirror-descent update (Algorithm 2, lines 10-11);
* ``relax``          -- Algorithm 2;
* ``round_select``   -- Algorithm 3 with the Proposition 1 score (eq. 14) and
  Lemma 2's block Sherman-Morrison form;
* ``nu_bisect``      -- the scalar root of eq. 10 / Algorithm 3 line 10.

Layout: a vector of length ``d~ = d c`` is ``vec(V)`` of a d x c matrix, so its
element ``k d + e`` is ``V[e, k]``.  A block of ``s`` vectors is a (d~, s) array.

Readings where the paper is silent or loose:
full c-class softmax; ``H_o = sum_{X_o} H_i + lam I``; ``H_p`` is the pool
average; z lives on the budget simplex; ``beta_t = beta0 / ||g_t||_inf``; CG
starts from zero, stops a column when its true recursive residual satisfies
``||r_j|| <= tol ||b_j||`` (or after a fixed count); the Round score uses
``B_k^{-1} Sigma_k B_k^{-1}`` in its numerator, as the proof of Proposition 1
derives (the statement prints ``Sigma_k^{-1}``); eta defaults to
``8 sqrt(d~)`` (Theorem 1 with epsilon = 1); no point is selected twice and
ties go to the lowest index.

Sums over points may be split into consecutive chunks (``chunk=``) to bound
memory; that only regroups the sum of eq. 3.
"""
import numpy as np

from .probes import rademacher


# ----------------------------------------------------------------------------------------
# Hessian algebra
# ----------------------------------------------------------------------------------------

def _as64(a):
    return np.asarray(a, dtype=np.float64)


def hessian_apply(X, h, w, V, chunk=None):
    """``sum_i w_i H_i V`` by Lemma 1, for a block V of shape (d c, s).

    Per point and column: gamma = V_j^T x_i; alpha = gamma . h_i;
    gamma <- (gamma - alpha) * h_i; H_i v_j = vec(x_i gamma^T).
    """
    X, h, w, V = _as64(X), _as64(h), _as64(w), _as64(V)
    n, d = X.shape
    c = h.shape[1]
    s = V.shape[1]
    out = np.zeros((c, d, s))
    Vm = V.reshape(c, d, s)                          # Vm[k, e, j] = V_j[e, k]
    step = max(n, 1) if chunk is None else chunk
    for a in range(0, n, step):
        Xa, ha, wa = X[a:a + step], h[a:a + step], w[a:a + step]
        for j in range(s):
            gamma = Xa @ Vm[:, :, j].T               # (points, c): gamma_i = V_j^T x_i
            alpha = np.sum(gamma * ha, axis=1)       # alpha_i = gamma_i^T h_i
            gamma = (gamma - alpha[:, None]) * ha    # (gamma_i - alpha_i) * h_i
            out[:, :, j] += (Xa.T @ (wa[:, None] * gamma)).T   # sum_i w_i x_i gamma_i^T
    return out.reshape(c * d, s)


def block_diag(X, h, w):
    """``sum_i w_i B_k(H_i)`` with ``B_k(H_i) = h_i^k (1 - h_i^k) x_i x_i^T`` (eq. 13); (c, d, d)."""
    X, h, w = _as64(X), _as64(h), _as64(w)
    wk = w[:, None] * h * (1.0 - h)                  # (n, c)
    return np.einsum("ik,ie,if->kef", wk, X, X)


def block_of(M, k, d):
    """The k-th diagonal d x d block of a dc x dc matrix (Definition 1)."""
    return M[k * d:(k + 1) * d, k * d:(k + 1) * d]


class Operators:
    """The two Hessian operators of Algorithm 2 for one problem.

    ``Sigma_z V = H_o V + sum_{pool} z_i H_i V`` with ``H_o V = lam V + sum_{X_o} H_i V``
    (eqs. 3, 7), and ``H_p V = (1/n) sum_{pool} H_i V``.
    """

    def __init__(self, prob, chunk=None):
        self.X, self.h = _as64(prob.X), _as64(prob.h)
        self.Xo, self.ho = _as64(prob.Xo), _as64(prob.ho)
        self.lam = float(prob.lam)
        self.n, self.d = self.X.shape
        self.c = self.h.shape[1]
        self.D = self.d * self.c
        self.chunk = chunk

    def ho_apply(self, V):
        return self.lam * V + hessian_apply(self.Xo, self.ho, np.ones(self.Xo.shape[0]), V)

    def sigma_apply(self, z, V):
        return self.ho_apply(V) + hessian_apply(self.X, self.h, z, V, self.chunk)

    def hp_apply(self, V):
        return hessian_apply(self.X, self.h, np.full(self.n, 1.0 / self.n), V, self.chunk)

    def ho_blocks(self):
        """``B(H_o)``: labelled blocks plus ``lam I``."""
        return (block_diag(self.Xo, self.ho, np.ones(self.Xo.shape[0]))
                + self.lam * np.eye(self.d)[None])

    def precond_blocks(self, z):
        """``B(Sigma_z) = B(H_o) + sum_pool z_i B(H_i)`` (Definition 1, eq. 13)."""
        return self.ho_blocks() + block_diag(self.X, self.h, z)

    def sigma_dense(self, z):
        """Dense Sigma_z assembled column by column from ``sigma_apply`` (small d~ only)."""
        return self.sigma_apply(z, np.eye(self.D))


# ----------------------------------------------------------------------------------------
# Preconditioned conjugate gradients (Algorithm 2, lines 5-8)
# ----------------------------------------------------------------------------------------

def block_cholesky(blocks):
    """Lower Cholesky factors of the c SPD blocks."""
    return np.linalg.cholesky(blocks)


def block_solve(chol, R):
    """Apply ``B^{-1}`` block by block: column j, block k gets ``B_k^{-1} r_j[k]``."""
    c, d, _ = chol.shape
    s = R.shape[1]
    Rm = R.reshape(c, d, s)
    out = np.empty_like(Rm)
    for k in range(c):
        y = np.linalg.solve(chol[k], Rm[k])
        out[k] = np.linalg.solve(chol[k].T, y)
    return out.reshape(c * d, s)


def pcg(apply_A, B, apply_M, tol=0.1, maxit=100, fixed_iters=None):
    """Preconditioned CG on every column of B (x0 = 0).

    Column j stops when ``||r_j|| <= tol ||b_j||`` (true recursive residual,
    unpreconditioned norm) or when ``p^T A p <= 0``; with ``fixed_iters`` every
    column runs exactly that many iterations (``tol`` ignored).  Returns
    ``(X, iters, relres)``.
    """
    B = _as64(B)
    s = B.shape[1]
    Xs = np.zeros_like(B)
    R = B.copy()
    bn = np.linalg.norm(B, axis=0)
    active = bn > 0
    Z = apply_M(R)
    P = Z.copy()
    rho = np.sum(R * Z, axis=0)
    iters = np.zeros(s, dtype=np.int64)
    nsteps = fixed_iters if fixed_iters is not None else maxit
    if fixed_iters is None:
        active &= ~(np.linalg.norm(R, axis=0) <= tol * bn)
    for _ in range(nsteps):
        if not active.any():
            break
        Q = apply_A(P)
        pq = np.sum(P * Q, axis=0)
        active &= pq > 0
        a = np.where(active, rho / np.where(active, pq, 1.0), 0.0)
        Xs += a * P
        R -= a * Q
        iters += active
        rn = np.linalg.norm(R, axis=0)
        if fixed_iters is None:
            active &= ~(rn <= tol * bn)
        Z = apply_M(R)
        rho_new = np.sum(R * Z, axis=0)
        beta = np.where(active, rho_new / np.where(rho != 0, rho, 1.0), 0.0)
        P = np.where(active, Z + beta * P, P)
        rho = np.where(active, rho_new, rho)
    relres = np.linalg.norm(B - apply_A(Xs), axis=0) / np.where(bn > 0, bn, 1.0)
    return Xs, iters, relres


def block_pcg(apply_A, B, apply_M, tol=0.1, maxit=100, fixed_iters=None):
    """Block preconditioned CG (O'Leary, 1980) on all s columns of B at once (x0 = 0).

    One Krylov space serves the whole block; the step "scalars" are s x s matrices:
        gamma = Z^T R,  alpha = (P^T A P)^{-1} gamma,  X += P alpha,  R -= (A P) alpha,
        Z = M^{-1} R,  beta = gamma_old^{-1} gamma_new,  P = Z + P beta.
    The block stops when every column meets ``||r_j|| <= tol ||b_j||`` (or after
    ``fixed_iters`` iterations).  With s = 1 this is ``pcg``.  Returns
    ``(X, iterations, relres)``.
    """
    B = _as64(B)
    Xs = np.zeros_like(B)
    R = B.copy()
    bn = np.linalg.norm(B, axis=0)
    Z = apply_M(R)
    P = Z.copy()
    gam = Z.T @ R
    nsteps = fixed_iters if fixed_iters is not None else maxit
    it = 0
    for _ in range(nsteps):
        if fixed_iters is None and np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            break
        Q = apply_A(P)
        alpha = np.linalg.solve(P.T @ Q, gam)
        Xs += P @ alpha
        R -= Q @ alpha
        Z = apply_M(R)
        gam_new = Z.T @ R
        beta = np.linalg.solve(gam, gam_new)
        P = Z + P @ beta
        gam = gam_new
        it += 1
    relres = np.linalg.norm(B - apply_A(Xs), axis=0) / np.where(bn > 0, bn, 1.0)
    return Xs, it, relres


# ----------------------------------------------------------------------------------------
# Hutchinson estimates (eq. 11) and the objective
# ----------------------------------------------------------------------------------------

def quad_forms(X, h, A, B):
    """``q_i = (1/s) sum_j a_j^T H_i b_j`` for every point, via Lemma 1.

    ``a_j^T H_i b_j = sum_k (A_j^T x_i)_k * [((B_j^T x_i) - (B_j^T x_i).h_i) * h_i]_k``.
    """
    X, h, A, B = _as64(X), _as64(h), _as64(A), _as64(B)
    n, d = X.shape
    c = h.shape[1]
    s = A.shape[1]
    Am, Bm = A.reshape(c, d, s), B.reshape(c, d, s)
    q = np.zeros(n)
    for j in range(s):
        ga = X @ Am[:, :, j].T                       # a_j^T x_i components
        gb = X @ Bm[:, :, j].T
        gb = (gb - np.sum(gb * h, axis=1)[:, None]) * h   # Lemma 1 steps 2-3 on b_j
        q += np.sum(ga * gb, axis=1)
    return q / s


def grad_hutchinson(X, h, V, W):
    """Paper estimator, eq. 11: ``g_i = -(1/s) sum_j v_j^T H_i w_j``,
    ``w_j = Sigma^{-1} H_p Sigma^{-1} v_j``."""
    return -quad_forms(X, h, V, W)


def objective_estimate(V, HpU):
    """``f^ = (1/s) sum_j <v_j, H_p Sigma^{-1} v_j>`` (Hutchinson on eq. 4)."""
    return float(np.sum(_as64(V) * _as64(HpU)) / V.shape[1])


# ----------------------------------------------------------------------------------------
# Mirror descent and Relax (Algorithm 2)
# ----------------------------------------------------------------------------------------

def md_step(z, g, b, beta0=1.0):
    """``z <- z exp(-beta g)``, ``z <- b z / sum(z)`` with ``beta = beta0/||g||_inf``."""
    z, g = _as64(z), _as64(g)
    gmax = np.max(np.abs(g))
    beta = beta0 / gmax if gmax > 0 else 0.0
    z = z * np.exp(-beta * g)
    return b * z / np.sum(z)


def _solver(ops, z, solve, tol, maxit, fixed_iters):
    if solve == "direct":
        S = ops.sigma_dense(z)
        L = np.linalg.cholesky(S)
        return lambda R: (np.linalg.solve(L.T, np.linalg.solve(L, R)), None)
    chol = block_cholesky(ops.precond_blocks(z))
    return lambda R: pcg(lambda P: ops.sigma_apply(z, P), R, lambda Rr: block_solve(chol, Rr),
                         tol, maxit, fixed_iters)[:2]


def relax(prob, b, s, T, seed, *, beta0=1.0, z0=None, solve="cg", tol=0.1, maxit=100,
          fixed_iters=None, estimator="paper", chunk=None, record=False):
    """Fast Relax solve (Algorithm 2) on the budget simplex.

    Per MD iteration t (0-based): probes V_t; U = Sigma_z^{-1} V (PCG); HU = H_p U;
    f^ = <V, HU>/s; second solve W = Sigma_z^{-1} HU (``estimator="paper"``,
    eq. 11) or Y = Sigma_z^{-1} H_p V (``estimator="autograd"``: the exact
    derivative of f^ for fixed probes); gradient; MD step.  ``solve="direct"``
    replaces PCG by a dense Cholesky of Sigma_z (small d~ only).
    Returns ``(z, info)`` with per-iteration ``fhat`` (and, if ``record``, the
    probes, solves and gradients).
    """
    ops = Operators(prob, chunk)
    z = np.full(ops.n, b / ops.n) if z0 is None else _as64(z0).copy()
    info = dict(fhat=[], cg_iters=[], g=[], z=[], V=[], U=[], W=[])
    for t in range(T):
        V = rademacher(seed, t, s, ops.D)
        sol = _solver(ops, z, solve, tol, maxit, fixed_iters)
        U, it1 = sol(V)
        HU = ops.hp_apply(U)
        info["fhat"].append(objective_estimate(V, HU))
        if estimator == "paper":
            W, it2 = sol(HU)
            g = grad_hutchinson(ops.X, ops.h, V, W)
        else:
            W, it2 = sol(ops.hp_apply(V))
            g = -quad_forms(ops.X, ops.h, U, W)
        info["cg_iters"].append((it1, it2))
        if record:
            info["g"].append(g)
            info["z"].append(z.copy())
            info["V"].append(V)
            info["U"].append(U)
            info["W"].append(W)
        z = md_step(z, g, b, beta0)
    return z, info


# ----------------------------------------------------------------------------------------
# Round (Algorithm 3)
# ----------------------------------------------------------------------------------------

def nu_bisect(mu, rel=1e-15, maxit=400):
    """The unique ``nu > -min(mu)`` with ``sum_j (nu + mu_j)^{-2} = 1`` (eq. 10).

    The sum decreases monotonically on ``(-min mu, inf)`` and is at most 1 at
    ``sqrt(len(mu)) - min(mu)``, which brackets the root; plain bisection.
    """
    mu = _as64(mu).ravel()
    m0 = mu.min()
    lo, hi = -m0, np.sqrt(mu.size) - m0
    f = lambda nu: np.sum((nu + mu) ** -2.0) - 1.0
    for _ in range(maxit):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= rel * max(abs(hi), 1.0):
            break
    return 0.5 * (lo + hi)


def sherman_morrison_block(Ainv_k, x, gamma_k):
    """Lemma 2 for one block: ``(A_k + gamma_k x x^T)^{-1}``."""
    u = Ainv_k @ x
    return Ainv_k - gamma_k * np.outer(u, u) / (1.0 + gamma_k * x @ u)


def round_scores(X, wk, Binv, Sig, eta, numerator="derived"):
    """Proposition 1 score of every point (eq. 14), (n,).

    ``score_i = sum_k w_ik (x_i^T M1_k x_i) / (1 + eta w_ik x_i^T B_k^{-1} x_i)`` with
    ``w_ik = h_ik (1 - h_ik)`` and ``M1_k = B_k^{-1} Sigma_k B_k^{-1}`` (the form the proof
    derives; ``numerator="printed"`` uses ``B^{-1} Sigma^{-1} B^{-1}`` as eq. 14 is printed).
    """
    X = _as64(X)
    c = Binv.shape[0]
    out = np.zeros(X.shape[0])
    for k in range(c):
        mid = Sig[k] if numerator == "derived" else np.linalg.inv(Sig[k])
        M1 = Binv[k] @ mid @ Binv[k]
        num = np.sum((X @ M1) * X, axis=1)
        den = 1.0 + eta * wk[:, k] * np.sum((X @ Binv[k]) * X, axis=1)
        out += wk[:, k] * num / den
    return out


def tilde_eigvals(L, H):
    """Eigenvalues of ``L^{-1} H L^{-T}`` (similar to ``Sigma^{-1/2} H Sigma^{-1/2}``), per block."""
    out = []
    for k in range(H.shape[0]):
        Y = np.linalg.solve(L[k], H[k])
        M = np.linalg.solve(L[k], Y.T)
        out.append(np.linalg.eigvalsh(0.5 * (M + M.T)))
    return np.stack(out)


def round_select(prob, z_diamond, b, eta=None, exclude_selected=True, numerator="derived",
                 record=False):
    """Diagonal Round step (Algorithm 3).

    ``Sigma_k = B_k(H_o) + sum_pool z_i w_ik x_i x_i^T`` (block diagonal of
    ``H_o + H_{z_diamond}``), ``B_1 = sqrt(d~) Sigma + (eta/b) B(H_o)``; then for
    t = 1..b: pick the best eq. 14 score, ``H_k += B_k(H_o)/b + w_{i_t k} x x^T``,
    eigenvalues of ``H~_k``, ``nu`` from eq. 10, ``B = nu Sigma + eta H + (eta/b) B(H_o)``.
    Returns the selected indices (and, if ``record``, nu and score gaps).
    """
    ops = Operators(prob)
    X, h = ops.X, ops.h
    n, d, c = ops.n, ops.d, ops.c
    D = d * c
    eta = 8.0 * np.sqrt(D) if eta is None else float(eta)
    wk = h * (1.0 - h)
    Ho = ops.ho_blocks()
    Sig = Ho + np.einsum("ik,ie,if->kef", _as64(z_diamond)[:, None] * wk, X, X)
    L = np.linalg.cholesky(Sig)
    Binv = np.linalg.inv(np.sqrt(D) * Sig + (eta / b) * Ho)
    H = np.zeros((c, d, d))
    chosen, nus, gaps, scores = [], [], [], []
    mask = np.zeros(n, dtype=bool)
    for _ in range(b):
        sc = round_scores(X, wk, Binv, Sig, eta, numerator)
        if exclude_selected:
            sc = np.where(mask, -np.inf, sc)
        it = int(np.argmax(sc))
        if record:
            scores.append(sc.copy())
            top = np.sort(sc[np.isfinite(sc)])[::-1]
            gaps.append((top[0] - top[1]) / abs(top[0]) if top.size > 1 else np.inf)
        chosen.append(it)
        mask[it] = True
        H = H + Ho / b + wk[it][:, None, None] * np.outer(X[it], X[it])[None]
        lam = tilde_eigvals(L, H)
        nu = nu_bisect(eta * lam)
        nus.append(nu)
        Binv = np.linalg.inv(nu * Sig + eta * H + (eta / b) * Ho)
    if record:
        return chosen, dict(nu=nus, gap=gaps, H=H, Sig=Sig, scores=scores)
    return chosen


# ----------------------------------------------------------------------------------------
# Choosing eta (Section 5): Round for several eta, keep the one whose selected set has the
# best-conditioned Fisher blocks
# ----------------------------------------------------------------------------------------

def selected_min_eig(prob, selected):
    """``min_k lambda_min(H_k)`` with ``H = sum_{i in selected} H_i`` in its block-diagonal
    form, ``H_k = sum_i h_ik (1 - h_ik) x_i x_i^T`` (the Hessian sum of the selected points;
    the labelled set is not part of it)."""
    X, h = _as64(prob.X), _as64(prob.h)
    sel = np.asarray(selected, dtype=np.int64)
    blocks = block_diag(X[sel], h[sel], np.ones(sel.size))
    return float(min(np.linalg.eigvalsh(B)[0] for B in blocks))


def eta_sweep(prob, z_diamond, b, etas):
    """Run Round (Algorithm 3) once per eta and pick the eta maximising
    ``min_k lambda_min(H_k)`` of its selection (first on ties).  Returns
    ``(best_index, criteria, selections)``."""
    sels = [round_select(prob, z_diamond, b, eta=e) for e in etas]
    crit = [selected_min_eig(prob, s) for s in sels]
    return int(np.argmax(crit)), crit, sels
