"""Pins of the oracle's Hessian algebra (eq. 2, Lemma 1, eq. 13) -- no GPU."""
import json
import os

import numpy as np
import pytest

from oracle import approx, exact
from paper_2409_07392_gb300.synth import make_problem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tiny(n=7, d=4, c=3, seed=0, **kw):
    return make_problem(n, d, c, seed=seed, x_dtype="float64", h_dtype="float64", **kw)


def test_c2_closed_form_fixture():
    g = json.load(open(os.path.join(GOLD, "c2_hessian.json")))
    H = exact.hessian_dense(g["x"], g["h"])
    np.testing.assert_allclose(H, np.array(g["H"]), rtol=0, atol=1e-15)
    Hv = approx.hessian_apply(np.array([g["x"]]), np.array([g["h"]]), np.ones(1),
                              np.array(g["v"])[:, None])[:, 0]
    np.testing.assert_allclose(Hv, np.array(g["Hv"]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("d,c", [(1, 2), (3, 2), (4, 3), (8, 5), (5, 4)])
def test_lemma1_matches_dense_kronecker(d, c):
    rng = np.random.default_rng(d * 10 + c)
    p = tiny(n=9, d=d, c=c, seed=d + c)
    w = rng.uniform(0.1, 2.0, size=p.n)
    V = rng.standard_normal((d * c, 3))
    dense = exact.hessian_sum(p.X, p.h, w) @ V
    mf = approx.hessian_apply(p.X, p.h, w, V)
    np.testing.assert_allclose(mf, dense, rtol=0, atol=1e-13 * np.abs(dense).max())
    # chunking the sum over points regroups eq. 3 only
    np.testing.assert_allclose(approx.hessian_apply(p.X, p.h, w, V, chunk=2), mf, atol=1e-14)


def test_c2_reduces_to_scalar_logistic():
    """c = 2: [diag(h) - h h^T] = p(1-p)[[1,-1],[-1,1]] -- the binary logistic Hessian."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(5)
    p = 0.3
    H = exact.hessian_dense(x, [p, 1 - p])
    ref = p * (1 - p) * np.kron(np.array([[1.0, -1.0], [-1.0, 1.0]]), np.outer(x, x))
    np.testing.assert_allclose(H, ref, atol=1e-15)


def test_null_space_and_psd():
    """H_i (1_c (x) u) = 0 when sum_k h_ik = 1; H_i PSD of rank c - 1."""
    p = tiny(n=5, d=4, c=5)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(4)
    v = np.kron(np.ones(5), u)
    for i in range(p.n):
        H = exact.hessian_dense(p.X[i], p.h[i])
        assert np.abs(H @ v).max() < 1e-14
        ev = np.linalg.eigvalsh(H)
        assert ev.min() > -1e-12
        assert np.sum(ev > 1e-10 * ev.max()) == 5 - 1
    out = approx.hessian_apply(p.X, p.h, np.ones(p.n), v[:, None])
    assert np.abs(out).max() < 1e-13


def test_block_diag_eq13_equals_dense_blocks():
    p = tiny(n=8, d=3, c=4)
    w = np.linspace(0.2, 1.7, p.n)
    dense = exact.hessian_sum(p.X, p.h, w)
    blocks = approx.block_diag(p.X, p.h, w)
    np.testing.assert_allclose(blocks, exact.block_diag_of(dense, 3, 4), atol=1e-15)


def test_sigma_two_routes_agree():
    """Sigma_z from Lemma-1 columns equals the Kronecker-sum definition (eqs. 3, 7)."""
    p = tiny(n=6, d=3, c=3, m_o=3)
    z = np.linspace(0.1, 1.0, p.n)
    ops = approx.Operators(p)
    np.testing.assert_allclose(ops.sigma_dense(z), exact.sigma(p, z), atol=1e-14)
    np.testing.assert_allclose(ops.hp_apply(np.eye(9)), exact.h_p(p), atol=1e-14)
    np.testing.assert_allclose(ops.precond_blocks(z),
                               exact.block_diag_of(exact.sigma(p, z), 3, 3), atol=1e-14)


def test_planted_mistake_in_lemma1_is_caught(monkeypatch):
    """A dropped alpha term (a plausible slip) must fail the dense pin."""
    def wrong(X, h, w, V, chunk=None):
        X, h, w, V = map(np.asarray, (X, h, w, V))
        c, d, s = h.shape[1], X.shape[1], V.shape[1]
        out = np.zeros((c, d, s))
        for j in range(s):
            g = (X @ V.reshape(c, d, s)[:, :, j].T) * h
            out[:, :, j] = (X.T @ (w[:, None] * g)).T
        return out.reshape(c * d, s)
    p = tiny(n=5, d=3, c=3)
    V = np.random.default_rng(0).standard_normal((9, 2))
    dense = exact.hessian_sum(p.X, p.h, np.ones(5)) @ V
    assert np.abs(wrong(p.X, p.h, np.ones(5), V) - dense).max() > 1e-3
    # and a transposed vec convention (index e*c + k) fails too
    Vt = V.reshape(3, 3, 2).transpose(1, 0, 2).reshape(9, 2)
    assert np.abs(approx.hessian_apply(p.X, p.h, np.ones(5), Vt) - dense).max() > 1e-3
