"""Pins of the oracle's Round pieces: Lemma 2, Proposition 1, nu, eigenvalues -- no GPU."""
import json
import os

import numpy as np
import pytest

from oracle import approx, exact
from paper_2409_07392_gb300.synth import make_problem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tiny(n=10, d=3, c=3, seed=0, **kw):
    return make_problem(n, d, c, seed=seed, x_dtype="float64", h_dtype="float64", **kw)


def test_lemma2_block_sherman_morrison():
    rng = np.random.default_rng(0)
    c, d = 3, 4
    blocks = [np.eye(d) + (lambda a: a @ a.T)(rng.standard_normal((d, d))) for _ in range(c)]
    x = rng.standard_normal(d)
    gamma = rng.uniform(0.1, 2.0, c)
    for k in range(c):
        ref = np.linalg.inv(blocks[k] + gamma[k] * np.outer(x, x))
        got = approx.sherman_morrison_block(np.linalg.inv(blocks[k]), x, gamma[k])
        np.testing.assert_allclose(got, ref, atol=1e-12)
    # and the dense statement: the inverse of A + diag(gamma) (x) x x^T is block diagonal
    A = np.zeros((c * d, c * d))
    for k in range(c):
        A[k * d:(k + 1) * d, k * d:(k + 1) * d] = blocks[k]
    full = np.linalg.inv(A + np.kron(np.diag(gamma), np.outer(x, x)))
    for k in range(c):
        np.testing.assert_allclose(approx.block_of(full, k, d),
                                   approx.sherman_morrison_block(np.linalg.inv(blocks[k]), x,
                                                                 gamma[k]), atol=1e-12)


def test_nu_closed_forms():
    g = json.load(open(os.path.join(GOLD, "nu_closed_form.json")))
    for case in g["cases"]:
        assert abs(approx.nu_bisect(np.array(case["mu"], float)) - case["nu"]) < 1e-13


def test_nu_residual_random():
    rng = np.random.default_rng(1)
    mu = rng.exponential(3.0, 200)
    nu = approx.nu_bisect(mu)
    assert abs(np.sum((nu + mu) ** -2.0) - 1.0) < 1e-12
    assert nu > -mu.min()


def _jacobi_eigvals(M, sweeps=50):
    """Cyclic Jacobi (independent of LAPACK's method) for the eigenvalue pin."""
    A = M.copy()
    n = A.shape[0]
    for _ in range(sweeps):
        off = np.sqrt(np.sum(A ** 2) - np.sum(np.diag(A) ** 2))
        if off < 1e-15 * np.linalg.norm(A):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if abs(A[p, q]) < 1e-300:
                    continue
                th = (A[q, q] - A[p, p]) / (2 * A[p, q])
                t = np.sign(th) / (abs(th) + np.sqrt(th * th + 1)) if th != 0 else 1.0
                cs = 1 / np.sqrt(t * t + 1)
                sn = t * cs
                R = np.eye(n)
                R[p, p] = R[q, q] = cs
                R[p, q] = sn
                R[q, p] = -sn
                A = R.T @ A @ R
    return np.sort(np.diag(A))


def test_tilde_eigvals_trace_and_jacobi():
    rng = np.random.default_rng(2)
    c, d = 2, 5
    Sig = np.stack([np.eye(d) + (lambda a: a @ a.T)(rng.standard_normal((d, d))) for _ in range(c)])
    H = np.stack([(lambda a: a @ a.T)(rng.standard_normal((d, 3))) for _ in range(c)])
    L = np.linalg.cholesky(Sig)
    lam = approx.tilde_eigvals(L, H)
    for k in range(c):
        M = np.linalg.solve(L[k], np.linalg.solve(L[k], H[k]).T)
        assert abs(lam[k].sum() - np.trace(M)) < 1e-12 * abs(np.trace(M))
        # Sigma^{-1/2} H Sigma^{-1/2} has the same spectrum
        ev, Q = np.linalg.eigh(Sig[k])
        S12 = (Q / np.sqrt(ev)) @ Q.T
        np.testing.assert_allclose(np.sort(lam[k]), _jacobi_eigvals(S12 @ H[k] @ S12), atol=1e-12)


def test_prop1_round_equals_exact_round_on_block_diagonal_hessians():
    """Algorithm 3 (eq. 14 + Lemma 2) selects exactly what Algorithm 1's Round selects when
    every Hessian is replaced by its block diagonal (the premise of Proposition 1)."""
    for seed in range(3):
        p = tiny(n=12, d=2, c=3, seed=seed)
        z = np.full(p.n, 4.0 / p.n)
        sel_a = approx.round_select(p, z, 4)
        sel_e = exact.round_exact(p, z, 4, block_diag=True)
        assert sel_a == sel_e


def test_prop1_derived_numerator_is_the_consistent_one():
    """The score with B^{-1} Sigma B^{-1} (as derived in the proof) ranks points exactly as the
    block-diagonal eq. 9 trace; the printed Sigma^{-1} numerator is checked for comparison."""
    p = tiny(n=15, d=2, c=3, seed=4)
    X, h = p.X, p.h
    d, c = 2, 3
    D = d * c
    eta, b = 8 * np.sqrt(D), 5
    wk = h * (1 - h)
    ops = approx.Operators(p)
    Ho = ops.ho_blocks()
    z = np.full(p.n, 5.0 / p.n)
    Sig = Ho + np.einsum("ik,ie,if->kef", z[:, None] * wk, X, X)
    Binv = np.linalg.inv(np.sqrt(D) * Sig + (eta / b) * Ho)
    derived = approx.round_scores(X, wk, Binv, Sig, eta, "derived")
    # dense block-diagonal trace r_i = Tr[(B + eta B(H_i))^{-1} Sigma] (proof of Prop. 1)
    r = []
    for i in range(p.n):
        tot = 0.0
        for k in range(c):
            Bk = np.linalg.inv(Binv[k]) + eta * wk[i, k] * np.outer(X[i], X[i])
            tot += np.trace(np.linalg.solve(Bk, Sig[k]))
        r.append(tot)
    r = np.array(r)
    const = sum(np.trace(Binv[k] @ Sig[k]) for k in range(c))
    np.testing.assert_allclose(const - eta * derived, r, rtol=1e-10)
    assert np.argmax(derived) == np.argmin(r)


def test_round_first_pick_nu_and_simplex_facts():
    p = tiny(n=20, d=2, c=3, seed=5)
    z = np.full(p.n, 3.0 / p.n)
    sel, info = approx.round_select(p, z, 3, record=True)
    assert len(set(sel)) == 3
    D = 6
    # all nu satisfy eq. 10 with the recorded H after the last step
    L = np.linalg.cholesky(info["Sig"])
    lam = approx.tilde_eigvals(L, info["H"])
    eta = 8 * np.sqrt(D)
    assert abs(np.sum((info["nu"][-1] + eta * lam) ** -2.0) - 1) < 1e-12


def test_round_beats_random_subsets():
    """Relax + Round lands below the 5th percentile of random size-b subsets on f (eq. 4)."""
    for seed in range(3):
        p = tiny(n=40, d=3, c=3, seed=seed)
        b = 4
        Ho, Hp = exact.h_o(p), exact.h_p(p)
        z, _ = exact.relax(p, b, 20)
        sel = approx.round_select(p, z, b)
        f_round = exact.subset_objective(p, sel, Ho, Hp)
        rng = np.random.default_rng(seed)
        rand = [exact.subset_objective(p, rng.choice(p.n, b, replace=False), Ho, Hp)
                for _ in range(200)]
        assert f_round < np.percentile(rand, 5)


def test_round_vs_brute_force_tiny():
    """Report f(Round)/f* on tiny pools (a heuristic: ratio >= 1, bounded)."""
    p = tiny(n=10, d=2, c=2, seed=6)
    b = 3
    fstar, Sstar = exact.brute_force_best(p, b)
    z, _ = exact.relax(p, b, 30)
    sel = approx.round_select(p, z, b)
    ratio = exact.subset_objective(p, sel) / fstar
    assert 1.0 - 1e-12 <= ratio < 2.0


def test_selected_min_eig_matches_dense_hessian_sum():
    """The eta-sweep criterion equals the smallest eigenvalue over the diagonal d x d blocks of
    the dense sum of the selected points' Hessians (eq. 2, Kronecker form)."""
    p = make_problem(40, 4, 3, seed=2, x_dtype="float64", h_dtype="float64")
    sel = [3, 17, 25, 31, 8]
    Hs = exact.hessian_sum(p.X[sel], p.h[sel], np.ones(len(sel)))
    ref = min(np.linalg.eigvalsh(approx.block_of(Hs, k, p.d))[0] for k in range(p.c))
    assert abs(approx.selected_min_eig(p, sel) - ref) < 1e-12 * max(1.0, abs(ref))


def test_eta_sweep_picks_the_best_conditioned_selection():
    p = make_problem(300, 3, 3, seed=4, x_dtype="float64", h_dtype="float64")
    z = np.full(p.n, 6.0 / p.n)
    etas = [0.5, 4.0, 30.0]
    best, crit, sels = approx.eta_sweep(p, z, 6, etas)
    assert len(crit) == 3 and all(len(s) == 6 for s in sels)
    assert crit[best] == max(crit)
    for e, s, cr in zip(etas, sels, crit):
        assert s == approx.round_select(p, z, 6, eta=e)
        assert abs(cr - approx.selected_min_eig(p, s)) == 0.0
