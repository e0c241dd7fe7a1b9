"""Active-learning outer loop on the GPU against the FP64 oracle (oracle/al.py): classifier
probabilities (eq. 1), the ridge logistic-regression refit, and the picks of several rounds
of refit -> Relax -> Round.  Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import al  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2409_07392_gb300 import api, build
    build.build()
    return api


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)


@pytest.mark.parametrize("precision,dt,tol", [("fp64", torch.float64, 1e-12),
                                              ("fp32", torch.float32, 2e-6)])
def test_probs_vs_oracle(api, precision, dt, tol):
    p = make_problem(3001, 37, 23, seed=0)             # ragged against every tile
    W = np.random.default_rng(0).standard_normal((23, 37))
    h = api.lr_probs(dev(p.X, dt), dev(W, dt), precision=precision).double().cpu().numpy()
    ref = al.softmax_probs(p.X, W)
    assert np.max(np.abs(h - ref)) < tol


@pytest.mark.parametrize("precision,dt,tol", [("fp64", torch.float64, 1e-8),
                                              ("fp32", torch.float32, 2e-4)])
@pytest.mark.parametrize("m,d,c", [(100, 20, 10), (50, 50, 50)])
def test_lr_fit_vs_oracle(api, precision, dt, tol, m, d, c):
    p = make_problem(m, d, c, seed=1)
    y = p.labels
    W_ref = al.lr_fit(p.X, y, c, 1.0)
    W, steps, gn = api.lr_fit(dev(p.X, dt), torch.from_numpy(y).cuda(), c, 1.0,
                              precision=precision)
    W = W.double().cpu().numpy()
    err = np.linalg.norm(W - W_ref) / np.linalg.norm(W_ref)
    print(f"{precision} m={m} d~={d * c}: {steps} Newton steps, |g| {gn:.2e}, W err {err:.2e}")
    assert err < tol


def test_lr_fit_rejects_bad_labels(api):
    from paper_2409_07392_gb300 import _lib as L
    p = make_problem(30, 4, 3, seed=2)
    y = torch.from_numpy(p.labels).cuda()
    y[5] = 3                                            # outside [0, c)
    with pytest.raises(L.FiralError) as ei:
        api.lr_fit(dev(p.X, torch.float32), y, 3, 1.0)
    assert ei.value.code == L.FIRAL_ERR_ARG


@pytest.mark.parametrize("n,d,c,rounds,b,seed", [(300, 6, 4, 3, 5, 0), (500, 10, 5, 3, 6, 3)])
def test_active_learning_vs_oracle_fp64(api, n, d, c, rounds, b, seed):
    p = make_problem(n, d, c, seed=seed)
    yl = np.arange(p.Xo.shape[0]) % c
    kw = dict(s=6, T=5)
    picks_ref, W_ref = al.active_learning(p.X, p.labels, p.Xo, yl, c, rounds, b, fixed_iters=40,
                                          **kw)
    sel, W, fh = api.active_learning(dev(p.X, torch.float64), torch.from_numpy(p.labels).cuda(),
                                     dev(p.Xo, torch.float64), torch.from_numpy(yl).cuda(), c,
                                     rounds, b, precision="fp64", fixed_iters=40, **kw)
    sel = sel.cpu().numpy()
    print("gpu", sel.tolist(), "oracle", picks_ref.tolist())
    np.testing.assert_array_equal(sel, picks_ref)
    W = W.cpu().numpy()
    assert np.linalg.norm(W - W_ref) / np.linalg.norm(W_ref) < 1e-8
    assert all(np.isfinite(fh))


def test_active_learning_mixed_precision_runs(api):
    """The mixed-precision loop at a CIFAR-like shape: valid, distinct picks every round."""
    p = make_problem(20000, 50, 10, seed=6)
    yl = np.arange(p.Xo.shape[0]) % 10
    rounds, b = 3, 10
    sel, W, fh = api.active_learning(dev(p.X, torch.float32), torch.from_numpy(p.labels).cuda(),
                                     dev(p.Xo, torch.float32), torch.from_numpy(yl).cuda(), 10,
                                     rounds, b, precision="mixed_fast", s=10, T=10)
    flat = sel.reshape(-1).cpu().numpy()
    assert len(set(flat.tolist())) == rounds * b and flat.min() >= 0 and flat.max() < 20000
    assert np.isfinite(W.cpu().numpy()).all() and all(np.isfinite(fh))
