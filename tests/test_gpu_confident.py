"""Confident classifiers: the CUDA path vs the FP64 oracle when h is close to one-hot
(needs a GPU).

The classifier weights are scaled by 20 (``make_problem(w_scale=20)``), so the softmax
logits have a standard deviation of about 20: half of the points have ``1 - max_k h_ik``
below 1e-3 and a tenth are one-hot to float precision.  Each per-point Hessian
``H_i = (diag(h_i) - h_i h_i^T) (x) x_i x_i^T`` (Lemma 1) is then a small difference of two
large terms, in the per-point form (``gamma - alpha`` with ``alpha = h_i . gamma``) as in
any regrouping of it: rounding h_m ~ 1 to bf16 errs in the same direction on every confident
row, by as much as the Hessian itself.  This is what active-learning rounds after the first
one see, since a classifier trained on labels is confident on most of the pool.

The tensor-core path therefore takes every row with ``max_k h_ik > 1/2`` centred at its top
class (``h = e_m + u``, every term of the size of u) and the labelled rows on CUDA cores; what
remains are per-element bf16 roundings (2^-9) that average over the points a class's output
is made of, about n / c of them when h is confident (all n when it is flat).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import approx  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

W_SCALE = 20.0


@pytest.fixture(scope="module")
def api():
    from paper_2409_07392_gb300 import api as a, build
    build.build()
    return a


@pytest.fixture(scope="module")
def handle(api):
    return api.Handle()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(api, handle, p, precision):
    X = dev(p.X).to(torch.bfloat16) if p.x_bf16 else dev(p.X)
    Xo = dev(p.Xo).to(torch.bfloat16) if p.x_bf16 else dev(p.Xo)
    return api.Problem(handle, X, dev(p.h), Xo, dev(p.ho), p.lam, precision=precision)


def cancellation_ratio(p, V):
    """|sum_i w_i h_ik x_i x_i^T V_k| / |H_p V| with w = 1/n: how much larger the diagonal
    term of the apply is than the result."""
    X, h = p.X.astype(np.float64), p.h.astype(np.float64)
    n, d = X.shape
    c = h.shape[1]
    Vm = V.reshape(c, d, -1)
    diag = np.stack([((X.T * (h[:, k] / n)) @ X) @ Vm[k] for k in range(c)])
    return np.linalg.norm(diag) / np.linalg.norm(approx.hessian_apply(X, h, np.full(n, 1.0 / n), V))


# (n, d, c, s): the generic SIMT/tensor-core kernels (d = 16), the feature-contracted
# gradient (d = 64, c a multiple of 4), several class tiles with a ragged class tail (c = 130)
SHAPES = [(20000, 16, 10, 8), (12000, 64, 12, 8), (8000, 64, 130, 4)]


@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_fast"])
@pytest.mark.parametrize("n,d,c,s", SHAPES)
def test_confident_hessian_apply(api, handle, n, d, c, s, precision):
    p = make_problem(n, d, c, seed=3, x_dtype="bf16", h_dtype="float32", w_scale=W_SCALE)
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((d * c, s))
    z = rng.uniform(0.5, 1.5, n) * (20.0 / n)
    ops = approx.Operators(p)
    ref_sig, ref_hp = ops.sigma_apply(z, V), ops.hp_apply(V)
    Vd = dev(V.T.astype(np.float32))
    got_sig = prob.hessian_apply(Vd, dev(z.astype(np.float32)), op=0).cpu().numpy().T
    got_hp = prob.hessian_apply(Vd, op=1).cpu().numpy().T
    e1, e2 = relerr(got_sig, ref_sig), relerr(got_hp, ref_hp)
    ratio = cancellation_ratio(p, V)   # how large the apply's cancelling terms are
    print(f"confident {precision} apply n={n} d={d} c={c}: sigma {e1:.2e}  H_p {e2:.2e} "
          f"(cancellation ratio {ratio:.1f})")
    if precision == "fp32":
        tol = 2e-5 * ratio
    else:
        # per-element bf16 roundings (2^-9) averaged over the ~n/c points each class's output
        # is made of (the bound of the flat-h tests with n replaced by n / c)
        tol = 6.0 * 2.0 ** -9 / np.sqrt(n / c) + 2e-6
    assert e1 < tol and e2 < tol


@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_fast"])
@pytest.mark.parametrize("n,d,c,s", SHAPES)
def test_confident_quad_forms(api, handle, n, d, c, s, precision):
    """Per-point gradient forms (eq. 11) on confident h: the two terms of each form cancel to
    1 - max h."""
    p = make_problem(n, d, c, seed=5, x_dtype="bf16", h_dtype="float32", w_scale=W_SCALE)
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((d * c, s)), rng.standard_normal((d * c, s))
    ref = -approx.quad_forms(p.X, p.h, A, B)
    got = prob.quad_forms(dev(A.T.astype(np.float32)), dev(B.T.astype(np.float32))).cpu().numpy()
    e = relerr(got, ref)
    print(f"confident {precision} quad n={n} d={d} c={c} s={s}: {e:.2e}")
    assert e < 1e-4 if precision != "fp32" else e < 1e-5


@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_fast"])
@pytest.mark.parametrize("d,c", [(16, 10), (64, 12)])
def test_confident_relax_fhat_z_and_gradient(api, handle, precision, d, c):
    """Two MD iterations (10 PCG iterations per solve, the timing configuration) and the
    autograd gradient d f^/d z at the uniform start, against the oracle running the same
    recurrences with the same probes.  f^ and z meet 1e-3 in every precision.  The per-point
    derivative is a quadratic form in the two probe solves U, Y, whose deviation from the
    oracle's iterates is the apply's bf16 noise (~1e-4 here) amplified about 30-fold by the
    ill-conditioned Sigma_z of a confident classifier (lambda = 1e-3 on the directions the
    pool barely covers): the mixed modes reach 3.3e-3 there (bound 5e-3), FP32 2e-5."""
    p = make_problem(20000, d, c, seed=3, x_dtype="bf16", h_dtype="float32", w_scale=W_SCALE)
    prob = make(api, handle, p, precision)
    b, s, T, it = 20.0, 8, 2, 10
    z_ref, info = approx.relax(p, b, s=s, T=T, seed=4, fixed_iters=it)
    _, ainfo = approx.relax(p, b, s=s, T=1, seed=4, fixed_iters=it, estimator="autograd",
                            record=True)
    z = torch.full((p.n,), b / p.n, dtype=torch.float32, device="cuda")
    z0 = z.clone()
    opts = prob.relax_opts(s=s, T=T, fixed_iters=it, seed=4)
    fh = [prob.relax_step(opts, t, b, z)["fhat"] for t in range(T)]
    g = prob.objective_bwd(z0, 4, 0, s, fixed_iters=it).cpu().numpy()
    ef = relerr(fh, np.array(info["fhat"]))
    ez = relerr(z.cpu().numpy(), z_ref)
    eg = relerr(g, ainfo["g"][0])
    print(f"confident {precision} relax d={d} c={c}: fhat {ef:.2e}  z {ez:.2e}  dfdz {eg:.2e}")
    assert ef < 1e-3 and ez < 1e-3
    assert eg < (1e-3 if precision == "fp32" else 5e-3)
