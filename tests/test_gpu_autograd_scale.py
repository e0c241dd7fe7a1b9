"""Autograd Function of the Relax objective at the CIFAR-10-shaped size (n = 50,000, d = 50,
c = 10, s = 20), in the mixed precisions: the backward (the same-probe derivative of f^,
recomputing the probe solves) against

  * central finite differences of the same-probe objective f^(z) = (1/s) tr(V^T H_p S_z^-1 V)
    with exact FP64 solves, on 256 random coordinates, and
  * the exact FP64 gradient -(1/s) sum_j u_j^T H_i y_j with U = S^-1 V, Y = S^-1 H_p V
    (dense Cholesky solves in the oracle, same probes).

Target: 1e-3 relative.  Needs a GPU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import approx, exact  # noqa: E402
from oracle.probes import rademacher  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

N, D, C, S, B = 50000, 50, 10, 20, 100.0


@pytest.fixture(scope="module")
def setup():
    from paper_2409_07392_gb300 import api, build
    build.build()
    p = make_problem(N, D, C, seed=21, x_dtype="bf16", h_dtype="float32")
    rng = np.random.default_rng(5)
    z = rng.gamma(2.0, 1.0, N)
    z *= B / z.sum()                          # a non-uniform point of the budget simplex
    ops = approx.Operators(p)
    Sig = ops.sigma_dense(z)
    V = rademacher(7, 0, S, D * C)
    L = np.linalg.cholesky(Sig)
    U = np.linalg.solve(L.T, np.linalg.solve(L, V))
    HpV = ops.hp_apply(V)
    Y = np.linalg.solve(L.T, np.linalg.solve(L, HpV))
    g_ref = -approx.quad_forms(p.X, p.h, U, Y)          # d f^ / dz, exact solves
    return api, p, z, ops, Sig, V, HpV, g_ref


def fhat(Sig, V, HpV):
    """f^ = (1/s) sum_j v_j^T H_p S^-1 v_j with a dense solve (H_p symmetric)."""
    L = np.linalg.cholesky(Sig)
    return float(np.sum(HpV * np.linalg.solve(L.T, np.linalg.solve(L, V)))) / V.shape[1]


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
def test_mixed_backward_vs_fd_and_exact_gradient(setup, precision):
    api, p, z, ops, Sig, V, HpV, g_ref = setup
    from paper_2409_07392_gb300.autograd import firal_objective
    H = api.Handle()
    X = torch.from_numpy(p.X).cuda().to(torch.bfloat16)
    Xo = torch.from_numpy(p.Xo).cuda().to(torch.bfloat16)
    prob = api.Problem(H, X, torch.from_numpy(p.h).cuda(), Xo, torch.from_numpy(p.ho).cuda(),
                       p.lam, precision=precision)
    zt = torch.from_numpy(z.astype(np.float32)).cuda().requires_grad_(True)
    f = firal_objective(zt, prob, seed=7, t=0, s=S, tol=1e-5, maxit=500, recompute=True)
    f.backward()
    g = zt.grad.double().cpu().numpy()
    f_ref = fhat(Sig, V, HpV)
    e_f = abs(float(f) - f_ref) / abs(f_ref)
    e_g = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    # central differences of the exact same-probe objective on 256 coordinates
    rng = np.random.default_rng(11)
    idx = rng.choice(N, 256, replace=False)
    fd = np.empty(256)
    for q, i in enumerate(idx):
        Hi = exact.hessian_dense(p.X[i].astype(np.float64), p.h[i].astype(np.float64))
        eps = 1e-2 * z[i]
        fd[q] = (fhat(Sig + eps * Hi, V, HpV) - fhat(Sig - eps * Hi, V, HpV)) / (2 * eps)
    e_fd = np.linalg.norm(g[idx] - fd) / np.linalg.norm(fd)
    e_fd_ref = np.linalg.norm(g_ref[idx] - fd) / np.linalg.norm(fd)
    print(f"{precision}: f^ {e_f:.2e}  grad vs exact {e_g:.2e}  grad vs FD(256) {e_fd:.2e}  "
          f"(oracle gradient vs FD {e_fd_ref:.2e})")
    assert e_fd_ref < 1e-4          # the finite differences pin the oracle's derivative
    assert e_f < 1e-3 and e_g < 1e-3 and e_fd < 1e-3
    prob.close()
