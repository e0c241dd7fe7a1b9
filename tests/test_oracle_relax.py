"""Pins of the oracle's Relax pieces: PCG, Hutchinson estimates, gradients, MD -- no GPU."""
import numpy as np
import pytest

from oracle import approx, exact
from oracle.probes import rademacher
from paper_2409_07392_gb300.synth import make_problem


def tiny(n=10, d=3, c=3, seed=0, **kw):
    return make_problem(n, d, c, seed=seed, x_dtype="float64", h_dtype="float64", **kw)


# ------------------------------------------------------------------------------ PCG

def test_pcg_converges_to_cholesky_solution():
    p = tiny(n=40, d=4, c=5)
    ops = approx.Operators(p)
    z = np.full(p.n, 5.0 / p.n)
    S = exact.sigma(p, z)
    B = np.random.default_rng(0).standard_normal((20, 3))
    chol = approx.block_cholesky(ops.precond_blocks(z))
    X, it, rr = approx.pcg(lambda P: ops.sigma_apply(z, P), B,
                           lambda R: approx.block_solve(chol, R), tol=1e-12, maxit=500)
    ref = np.linalg.solve(S, B)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-10
    assert (rr < 1e-11).all() and (it > 1).all()


def test_pcg_block_diagonal_system_one_iteration():
    """If Sigma equals its block diagonal, B(Sigma)^{-1} is exact: one iteration."""
    rng = np.random.default_rng(2)
    c, d = 4, 3
    blocks = np.stack([np.eye(d) * 2 + 0.3 * (lambda a: a @ a.T)(rng.standard_normal((d, d)))
                       for _ in range(c)])
    A = np.zeros((c * d, c * d))
    for k in range(c):
        A[k * d:(k + 1) * d, k * d:(k + 1) * d] = blocks[k]
    chol = approx.block_cholesky(blocks)
    B = rng.standard_normal((c * d, 2))
    X, it, rr = approx.pcg(lambda P: A @ P, B, lambda R: approx.block_solve(chol, R),
                           tol=1e-12, maxit=10)
    assert (it == 1).all()
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=1e-12)


def test_pcg_fixed_iterations_and_unpreconditioned_cg_agree_with_textbook():
    """With M = I, one CG step is the steepest-descent step x = (b^T b / b^T A b) b."""
    rng = np.random.default_rng(4)
    G = rng.standard_normal((6, 6))
    A = G @ G.T + 6 * np.eye(6)
    b = rng.standard_normal((6, 1))
    X, it, _ = approx.pcg(lambda P: A @ P, b, lambda R: R, fixed_iters=1)
    np.testing.assert_allclose(X, (b.T @ b) / (b.T @ A @ b) * b, rtol=1e-13)
    X6, it6, _ = approx.pcg(lambda P: A @ P, b, lambda R: R, fixed_iters=6)
    np.testing.assert_allclose(X6, np.linalg.solve(A, b), rtol=1e-8)   # n steps = exact


def test_preconditioner_reduces_condition_number():
    """Shape of Fig. 1: kappa(B(Sigma)^{-1} Sigma) < kappa(Sigma) on a mixture pool."""
    p = make_problem(300, 6, 5, seed=3, x_dtype="float64", h_dtype="float64")
    ops = approx.Operators(p)
    z = np.full(p.n, 10.0 / p.n)
    S = ops.sigma_dense(z)
    L = np.linalg.cholesky(ops.precond_blocks(z))
    Linv = np.zeros_like(S)
    for k in range(5):
        Linv[k * 6:(k + 1) * 6, k * 6:(k + 1) * 6] = np.linalg.inv(L[k])
    kap = lambda M: (lambda e: e.max() / e.min())(np.linalg.eigvalsh(M))
    assert kap(Linv @ S @ Linv.T) < kap(S)


# ------------------------------------------------------------------------ Hutchinson

def test_hutchinson_mean_and_variance_closed_form():
    """E[v^T A v] = Tr A and Var = 2 (||A_sym||_F^2 - sum_q A_qq^2) for Rademacher v."""
    p = tiny(n=30, d=3, c=3)
    ops = approx.Operators(p)
    z = np.full(p.n, 3.0 / p.n)
    A = np.linalg.solve(exact.sigma(p, z), exact.h_p(p))     # Sigma^{-1} H_p
    f = np.trace(A)
    As = 0.5 * (A + A.T)
    var1 = 2.0 * (np.sum(As ** 2) - np.sum(np.diag(A) ** 2))
    L = np.linalg.cholesky(ops.sigma_dense(z))
    samples = []
    for t in range(2000):
        V = rademacher(99, t, 1, 9)
        U = np.linalg.solve(L.T, np.linalg.solve(L, V))
        samples.append(approx.objective_estimate(V, ops.hp_apply(U)))
    samples = np.array(samples)
    assert abs(samples.mean() - f) < 4 * np.sqrt(var1 / samples.size)
    assert abs(samples.var() / var1 - 1.0) < 0.15


def test_exact_gradient_matches_finite_differences():
    """eq. 6 against central differences of f (eq. 4)."""
    p = tiny(n=6, d=3, c=3)
    z = np.linspace(0.2, 0.9, p.n)
    Ho, Hp = exact.h_o(p), exact.h_p(p)
    g = exact.gradient(p, z, Ho, Hp)
    for i in range(p.n):
        e = np.zeros(p.n)
        eps = 1e-6 * z[i]
        e[i] = eps
        fd = (exact.objective(p, z + e, Ho, Hp) - exact.objective(p, z - e, Ho, Hp)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-12


def test_autograd_estimator_is_derivative_of_fhat():
    """g^_i = -(1/s) sum_j u_j^T H_i y_j differentiates f^(z) for fixed probes."""
    p = tiny(n=6, d=3, c=3)
    ops = approx.Operators(p)
    z = np.linspace(0.2, 0.9, p.n)
    V = rademacher(5, 0, 4, 9)

    def fhat(zz):
        S = ops.sigma_dense(zz)
        return approx.objective_estimate(V, ops.hp_apply(np.linalg.solve(S, V)))
    S = ops.sigma_dense(z)
    U = np.linalg.solve(S, V)
    Y = np.linalg.solve(S, ops.hp_apply(V))
    g = -approx.quad_forms(p.X, p.h, U, Y)
    for i in range(p.n):
        e = np.zeros(p.n)
        eps = 1e-6 * z[i]
        e[i] = eps
        fd = (fhat(z + e) - fhat(z - e)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-12


def test_paper_estimator_converges_to_exact_gradient():
    """eq. 11 is unbiased: its mean over many probes approaches eq. 6."""
    p = tiny(n=8, d=3, c=3)
    ops = approx.Operators(p)
    z = np.full(p.n, 2.0 / p.n)
    g_exact = exact.gradient(p, z)
    S = ops.sigma_dense(z)
    V = rademacher(11, 0, 20000, 9)
    W = np.linalg.solve(S, ops.hp_apply(np.linalg.solve(S, V)))
    g_est = approx.grad_hutchinson(p.X, p.h, V, W)
    assert np.linalg.norm(g_est - g_exact) / np.linalg.norm(g_exact) < 0.05


def test_quad_form_matches_dense():
    p = tiny(n=5, d=3, c=4)
    rng = np.random.default_rng(8)
    A, B = rng.standard_normal((12, 3)), rng.standard_normal((12, 3))
    q = approx.quad_forms(p.X, p.h, A, B)
    ref = [np.mean([A[:, j] @ exact.hessian_dense(p.X[i], p.h[i]) @ B[:, j] for j in range(3)])
           for i in range(p.n)]
    np.testing.assert_allclose(q, ref, atol=1e-14)


# ------------------------------------------------------------------------ MD / Relax

def test_md_step_simplex_and_first_order():
    rng = np.random.default_rng(5)
    z = rng.uniform(0.1, 1, 50)
    b = 7.0
    z = b * z / z.sum()
    g = rng.standard_normal(50)
    z1 = approx.md_step(z, g, b, beta0=1.0)
    assert abs(z1.sum() - b) < 1e-12 * b and (z1 > 0).all()
    beta0 = 1e-6
    beta = beta0 / np.abs(g).max()
    z2 = approx.md_step(z, g, b, beta0=beta0)
    first = z - beta * z * (g - (z @ g) / b)
    assert np.abs(z2 - first).max() < 10 * beta ** 2 * np.abs(z).max() * np.abs(g).max() ** 2


def test_relax_direct_many_probes_tracks_exact_relax():
    """Approx Relax with exact solves and many probes approaches Exact Relax (Fig. 4 claim)."""
    p = tiny(n=20, d=3, c=3)
    b, T = 3, 5
    z_ex, f_ex = exact.relax(p, b, T)
    z_ap, info = approx.relax(p, b, s=4000, T=T, seed=1, solve="direct")
    assert np.linalg.norm(z_ap - z_ex) / np.linalg.norm(z_ex) < 0.05
    np.testing.assert_allclose(info["fhat"][0], f_ex[0], rtol=0.05)
    assert abs(z_ap.sum() - b) < 1e-12


def test_relax_cg_matches_direct_at_tight_tolerance():
    p = tiny(n=30, d=3, c=4)
    z_cg, i1 = approx.relax(p, 4, s=3, T=3, seed=2, solve="cg", tol=1e-13, maxit=300)
    z_d, i2 = approx.relax(p, 4, s=3, T=3, seed=2, solve="direct")
    np.testing.assert_allclose(z_cg, z_d, rtol=1e-9)
    np.testing.assert_allclose(i1["fhat"], i2["fhat"], rtol=1e-10)


def test_relax_decreases_objective():
    p = make_problem(200, 4, 4, seed=1, x_dtype="float64", h_dtype="float64")
    z0 = np.full(p.n, 8.0 / p.n)
    z, _ = exact.relax(p, 8, 15, beta0=0.5)
    assert exact.objective(p, z) < exact.objective(p, z0)


def _spd_system(n, s, cond, seed):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Qm * np.geomspace(1.0, cond, n)) @ Qm.T
    Md = np.diag(A).copy()
    return A, (lambda V: A @ V), (lambda V: V / Md[:, None]), rng.standard_normal((n, s))


def test_block_pcg_with_one_column_is_pcg():
    """O'Leary's block CG with s = 1 reduces to preconditioned CG, iterate for iterate."""
    A, app, prec, B = _spd_system(60, 1, 1e3, 1)
    for k in (1, 3, 7):
        Xb, _, _ = approx.block_pcg(app, B, prec, fixed_iters=k)
        Xc, _, _ = approx.pcg(app, B, prec, fixed_iters=k)
        np.testing.assert_allclose(Xb, Xc, rtol=1e-11, atol=1e-13)


def test_block_pcg_reaches_the_direct_solution_in_fewer_iterations():
    """Block CG converges to A^{-1} B, and its shared Krylov space needs no more iterations
    than the slowest independent column (here strictly fewer)."""
    A, app, prec, B = _spd_system(120, 8, 1e5, 2)
    Xb, itb, rb = approx.block_pcg(app, B, prec, tol=1e-10, maxit=500)
    Xc, itc, _ = approx.pcg(app, B, prec, tol=1e-10, maxit=500)
    np.testing.assert_allclose(Xb, np.linalg.solve(A, B), rtol=1e-7, atol=1e-9)
    assert rb.max() < 1e-9
    assert itb < int(np.max(itc))
