"""Pins of the active-learning oracle (oracle/al.py) against closed forms, finite
differences, an independent optimiser and the loop's invariants."""
import numpy as np
import pytest

from oracle import al, approx, exact
from paper_2409_07392_gb300.synth import make_problem


def labelled(p):
    return np.arange(p.Xo.shape[0]) % p.c


def test_softmax_two_classes_is_the_logistic_sigmoid():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((20, 5))
    W = rng.standard_normal((2, 5))
    h = al.softmax_probs(X, W)
    s = 1.0 / (1.0 + np.exp(-(X @ (W[1] - W[0]))))
    np.testing.assert_allclose(h[:, 1], s, rtol=1e-13)
    np.testing.assert_allclose(h.sum(axis=1), 1.0, rtol=1e-14)


def test_gradient_matches_finite_differences():
    p = make_problem(40, 4, 3, seed=1)
    rng = np.random.default_rng(1)
    W = rng.standard_normal((3, 4))
    y = p.labels
    g = al.lr_gradient(p.X, y, W, 0.7)
    eps = 1e-6
    for k in range(3):
        for e in range(4):
            E = np.zeros_like(W)
            E[k, e] = eps
            fd = (al.lr_loss(p.X, y, W + E, 0.7) - al.lr_loss(p.X, y, W - E, 0.7)) / (2 * eps)
            assert abs(fd - g[k, e]) < 1e-6 * max(1.0, abs(fd))


def test_fisher_form_is_the_hessian_of_the_loss():
    """sum_i H_i + gamma I (eq. 2, index k d + e) equals the Jacobian of the gradient."""
    p = make_problem(30, 3, 4, seed=2)
    rng = np.random.default_rng(2)
    W = rng.standard_normal((4, 3))
    y = p.labels
    gamma = 0.3
    Hs = exact.hessian_sum(p.X, al.softmax_probs(p.X, W), np.ones(30)) + gamma * np.eye(12)
    eps = 1e-6
    J = np.empty((12, 12))
    for q in range(12):
        E = np.zeros(12)
        E[q] = eps
        J[:, q] = ((al.lr_gradient(p.X, y, W + E.reshape(4, 3), gamma) -
                    al.lr_gradient(p.X, y, W - E.reshape(4, 3), gamma)) / (2 * eps)).reshape(-1)
    np.testing.assert_allclose(J, Hs, atol=1e-7)


def test_newton_fit_matches_an_independent_optimiser():
    scipy_opt = pytest.importorskip("scipy.optimize")
    p = make_problem(60, 5, 4, seed=3)
    y = p.labels
    gamma = 1.0
    W = al.lr_fit(p.X, y, 4, gamma)
    res = scipy_opt.minimize(lambda w: al.lr_loss(p.X, y, w.reshape(4, 5), gamma),
                             np.zeros(20), jac=lambda w: al.lr_gradient(p.X, y, w.reshape(4, 5),
                                                                        gamma).reshape(-1),
                             method="L-BFGS-B", options=dict(gtol=1e-12, ftol=1e-15,
                                                             maxiter=5000))
    np.testing.assert_allclose(W.reshape(-1), res.x, rtol=1e-5, atol=1e-7)
    assert np.linalg.norm(al.lr_gradient(p.X, y, W, gamma)) < 1e-9


def test_active_learning_loop_invariants():
    p = make_problem(120, 4, 3, seed=4)
    rounds, b = 3, 4
    picks, W = al.active_learning(p.X, p.labels, p.Xo, labelled(p), 3, rounds, b, s=6, T=4,
                                  fixed_iters=12)
    assert picks.shape == (rounds, b)
    flat = picks.reshape(-1)
    assert len(set(flat.tolist())) == rounds * b and flat.min() >= 0 and flat.max() < 120
    # the final classifier is the fit on every label revealed
    Xl = np.vstack([p.Xo, p.X[flat]])
    yl = np.concatenate([labelled(p), p.labels[flat]])
    np.testing.assert_allclose(W, al.lr_fit(Xl, yl, 3, 1.0), rtol=1e-8, atol=1e-10)


def test_first_round_is_relax_then_round_on_the_refit_classifier():
    p = make_problem(100, 4, 3, seed=5)
    picks, _ = al.active_learning(p.X, p.labels, p.Xo, labelled(p), 3, 1, 5, s=6, T=4,
                                  fixed_iters=12)
    W = al.lr_fit(p.Xo, labelled(p), 3, 1.0)
    prob = al._Pool(p.X, al.softmax_probs(p.X, W), p.Xo, al.softmax_probs(p.Xo, W), p.lam)
    z, _ = approx.relax(prob, 5, 6, 4, 1, fixed_iters=12)
    assert picks[0].tolist() == approx.round_select(prob, z, 5)
