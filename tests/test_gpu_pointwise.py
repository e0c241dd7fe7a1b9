"""The fused per-point kernels (at most 32 classes per pool, d <= 64) against the FP64 oracle,
at the accuracy of their hi + lo operands (needs a GPU).

The Hessian apply runs Lemma 1 row by row: a = x . P~ (MMA1), psi = w h (a - alpha) in f32,
out += psi x (MMA2).  P~ and psi enter as bf16 hi + lo, the quadratic forms' A~ and B~ too,
so every operand carries at most 2^-17 relative rounding and x is exact in bf16.  TMEM
accumulates in f32 over chains of at most 256 adds (16 row tiles x 16 MMAs per segment); the
biased rounding of those adds stays below 256 * 2^-25 = 7.6e-6 of the running sum.  Nothing
cancels in the per-point form, so the apply is within ~1e-5 of the oracle whether h is flat or
confident, labelled rows included.

Shapes: cpad = 8 / 16 / 32 columns per probe; s not a multiple of 8 (padded probes); s above
256 / cpad (probe groups of 8 or 16: two or three launches).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import approx  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

# (n, d, c, s)
SHAPES = [(5000, 16, 5, 8), (3001, 32, 10, 3), (4000, 64, 20, 12), (2500, 48, 32, 16),
          (1500, 64, 17, 20)]


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
    X = dev(p.X).to(torch.bfloat16)
    Xo = dev(p.Xo).to(torch.bfloat16)
    return api.Problem(handle, X, dev(p.h), Xo, dev(p.ho), p.lam, precision=precision)


@pytest.mark.parametrize("w_scale", [1.0, 20.0])
@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
@pytest.mark.parametrize("n,d,c,s", SHAPES)
def test_pointwise_hessian_apply(api, handle, n, d, c, s, precision, w_scale):
    p = make_problem(n, d, c, seed=n + c, x_dtype="bf16", h_dtype="float32", m_o=2 * c,
                     w_scale=w_scale)
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(1)
    V = rng.standard_normal((d * c, s))
    z = rng.uniform(0.5, 1.5, n) * (20.0 / n)
    ops = approx.Operators(p)
    ref_sig, ref_hp = ops.sigma_apply(z, V), ops.hp_apply(V)
    Vd = dev(V.T.astype(np.float32))
    got_sig = prob.hessian_apply(Vd, dev(z.astype(np.float32)), op=0).cpu().numpy().T
    got_hp = prob.hessian_apply(Vd, op=1).cpu().numpy().T
    e1, e2 = relerr(got_sig, ref_sig), relerr(got_hp, ref_hp)
    print(f"pointwise {precision} apply n={n} d={d} c={c} s={s} w x{w_scale:g}: "
          f"sigma {e1:.2e}  H_p {e2:.2e}")
    assert e1 < 2e-5 and e2 < 2e-5
    prob.close()


@pytest.mark.parametrize("w_scale", [1.0, 20.0])
@pytest.mark.parametrize("n,d,c,s", SHAPES)
def test_pointwise_quad_forms(api, handle, n, d, c, s, w_scale):
    """Per-point forms sum_j a_j^T H_i b_j (eq. 11).  Their two terms cancel to O(1 - max h) on
    confident rows, so the norm-wise error there is that of the flat rows' terms: 1e-4."""
    p = make_problem(n, d, c, seed=n + 5, x_dtype="bf16", h_dtype="float32", m_o=c,
                     w_scale=w_scale)
    prob = make(api, handle, p, "mixed")
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((d * c, s)), rng.standard_normal((d * c, s))
    ref = -approx.quad_forms(p.X, p.h, A, B)
    got = prob.quad_forms(dev(A.T.astype(np.float32)), dev(B.T.astype(np.float32))).cpu().numpy()
    e = relerr(got, ref)
    print(f"pointwise quad n={n} d={d} c={c} s={s} w x{w_scale:g}: {e:.2e}")
    assert e < (2e-5 if w_scale == 1.0 else 1e-4)
    prob.close()
