"""Mixed-precision (bf16 tcgen05) path vs the FP64 oracle, through the C-ABI (needs a GPU).

Error budget of one Hessian apply: the diagonal part is FP32 on CUDA cores; the low-rank
part rounds h and x (x exact when stored bf16) and walpha x to bf16 with independent
per-element errors (2^-9) that average over the point sums, and feeds the CG direction as
bf16 hi + lo (2^-17).  The relative error in norm shrinks like 1/sqrt(n); the bound asserted is 6 * 2^-9 / sqrt(n).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import approx  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu


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
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def make(api, handle, p, precision="mixed"):
    X = dev(p.X).to(torch.bfloat16) if p.x_bf16 else dev(p.X)
    Xo = dev(p.Xo).to(torch.bfloat16) if p.x_bf16 else dev(p.Xo)
    return api.Problem(handle, X, dev(p.h), Xo, dev(p.ho), p.lam, precision=precision)


MIXED_SHAPES = [(300, 20, 10, 3), (1000, 50, 10, 5), (517, 64, 37, 4), (260, 128, 4, 3),
                (2049, 16, 17, 8), (2049, 33, 17, 20), (2049, 16, 17, 20), (4100, 64, 130, 16)]


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
@pytest.mark.parametrize("n,d,c,s", MIXED_SHAPES)
def test_mixed_hessian_apply(api, handle, n, d, c, s, precision):
    p = make_problem(n, d, c, seed=n + c, x_dtype="bf16", h_dtype="float32", m_o=c)
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((d * c, s))
    z = rng.uniform(0.1, 1.0, n)
    ops = approx.Operators(p)
    ref_sig = ops.sigma_apply(z, V)
    ref_hp = ops.hp_apply(V)
    got_sig = prob.hessian_apply(dev(V.T.astype(np.float32)), dev(z.astype(np.float32)),
                                 op=0).cpu().numpy().T
    got_hp = prob.hessian_apply(dev(V.T.astype(np.float32)), op=1).cpu().numpy().T
    for name, g in (("sigma", got_sig), ("H_p", got_hp)):
        bad = np.argwhere(~np.isfinite(g))
        if bad.size:
            q, j = bad[:, 0], bad[:, 1]
            print(f"{name}: {bad.shape[0]} non-finite; probes {sorted(set(j.tolist()))[:20]} "
                  f"classes {sorted(set((q // d).tolist()))[:20]} "
                  f"features {sorted(set((q % d).tolist()))[:20]}")
    e1, e2 = relerr(got_sig, ref_sig), relerr(got_hp, ref_hp)
    print(f"{precision} apply n={n} d={d} c={c} s={s}: sigma {e1:.2e}  H_p {e2:.2e}")
    # per-element bf16 rounding (2^-9) of h and of walpha x averages over the n-point sums
    tol = 6.0 * 2.0 ** -9 / np.sqrt(n) + 2e-6
    if precision == "mixed_fast":
        # plus the rounding of V itself (2^-9 per entry, shared by every point): the
        # low-rank term is a linear map of V, so its relative error is at most 2^-9
        tol += 2.0 ** -9
    assert e1 < tol and e2 < tol


def test_mixed_apply_keeps_the_softmax_null_space(api, handle):
    """Sigma_z (1_c (x) u) = lambda (1_c (x) u) and H_p (1_c (x) u) = 0 (rows of h sum to 1)."""
    p = make_problem(3000, 32, 12, seed=5, x_dtype="bf16", h_dtype="float64", m_o=12)
    p.h = p.h.astype(np.float32)
    p.ho = p.ho.astype(np.float32)
    prob = make(api, handle, p)
    u = np.random.default_rng(1).standard_normal((3, 32))
    V = np.concatenate([np.tile(u[j], 12)[None] for j in range(3)]).astype(np.float32)
    z = np.full(p.n, 0.01, np.float32)
    sig = prob.hessian_apply(dev(V), dev(z), op=0).cpu().numpy()
    hp = prob.hessian_apply(dev(V), op=1).cpu().numpy()
    assert relerr(sig, p.lam * V.astype(np.float64)) < 1e-4
    assert np.abs(hp).max() < 1e-6 * np.abs(V).max()


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
@pytest.mark.parametrize("d,c", [(16, 10), (64, 12)])
def test_mixed_relax_fhat_and_z_vs_exact_solve_oracle(api, handle, precision, d, c):
    """Mixed Relax (CG to 1e-5) vs the oracle with dense solves and the same probes:
    f^ and z within 1e-3 relative (the stated accuracy target).  d = 64, c = 12 takes the
    feature-contracted gradient."""
    p = make_problem(20000, d, c, seed=3, x_dtype="bf16", h_dtype="float32")
    prob = make(api, handle, p, precision)
    b, s, T = 20.0, 8, 3
    z = torch.full((p.n,), b / p.n, dtype=torch.float32, device="cuda")
    opts = prob.relax_opts(s=s, T=T, tol=1e-5, maxit=300, seed=4)
    fh = [prob.relax_step(opts, t, b, z)["fhat"] for t in range(T)]
    z_ref, info = approx.relax(p, b, s=s, T=T, seed=4, solve="direct")
    ef, ez = relerr(fh, np.array(info["fhat"])), relerr(z.cpu().numpy(), z_ref)
    print(f"{precision} relax: fhat {ef:.2e}  z {ez:.2e}")
    assert ef < 1e-3 and ez < 1e-3


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
@pytest.mark.parametrize("n,d,c,s", [(3000, 20, 10, 4), (2049, 64, 37, 8), (1500, 128, 5, 3),
                                     (4100, 16, 130, 16), (2049, 64, 36, 8), (1500, 128, 8, 3),
                                     (3000, 50, 12, 5), (2049, 64, 36, 20), (1000, 128, 8, 17),
                                     (2049, 64, 36, 1), (1300, 96, 40, 15), (2300, 64, 64, 16)])
def test_mixed_quad_forms(api, handle, n, d, c, s, precision):
    """Tensor-core per-point quadratic forms (eq. 11) vs the oracle; a large N-component added
    to A must not change the result (H_i vanishes on N = {1_c (x) u}).  At most 32 classes
    with d <= 64 take the fused per-point kernel (c = 10, 12 here); otherwise d >= 64 with c a
    multiple of 4 takes the feature-contracted kernel: class-chunk-major for s <= 16 (its two
    epilogue groups split the probes by parity: s = 1, odd s = 3, 15 and s = 16 included),
    probe-major for s = 17, 20."""
    p = make_problem(n, d, c, seed=n + 7, x_dtype="bf16", h_dtype="float64", m_o=c)
    p.h = p.h.astype(np.float32).astype(np.float64)
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((d * c, s)), rng.standard_normal((d * c, s))
    ref = -approx.quad_forms(p.X, p.h, A, B)
    got = prob.quad_forms(dev(A.T.astype(np.float32)), dev(B.T.astype(np.float32))).cpu().numpy()
    e1 = relerr(got, ref)
    u = rng.standard_normal((d, s))
    An = A + 1e3 * np.tile(u, (c, 1))
    got_n = prob.quad_forms(dev(An.T.astype(np.float32)), dev(B.T.astype(np.float32))).cpu().numpy()
    e2 = relerr(got_n, ref)
    print(f"{precision} quad n={n} d={d} c={c} s={s}: {e1:.2e}  with N-component {e2:.2e}")
    # both mixed modes take the same gradient kernels: h enters as bf16 hi + lo (pair form)
    # or exact f32 (feature-contracted form), and the coefficients M~ / [A; B] as bf16
    # hi + lo; the per-point errors are ~2^-16 (the fast mode differs only in the Hessian
    # apply's CG-direction operand)
    assert e1 < 1e-4 and e2 < 2e-4


def test_fixed_iteration_relax_mixed_and_fp32_vs_oracle(api, handle):
    """Two MD iterations with exactly 10 PCG iterations per solve (the timing configuration):
    z from the mixed and the FP32 paths against the oracle running the same recurrences."""
    p = make_problem(20000, 16, 10, seed=11, x_dtype="bf16", h_dtype="float32")
    b, s, T = 20.0, 8, 2
    z_ref, info = approx.relax(p, b, s=s, T=T, seed=4, fixed_iters=10)
    errs = {}
    for prec in ("mixed", "mixed_fast", "fp32"):
        X = dev(p.X).to(torch.bfloat16)
        Xo = dev(p.Xo).to(torch.bfloat16)
        prob = api.Problem(handle, X, dev(p.h), Xo, dev(p.ho), p.lam, precision=prec)
        z = torch.full((p.n,), b / p.n, dtype=torch.float32, device="cuda")
        opts = prob.relax_opts(s=s, T=T, fixed_iters=10, seed=4)
        fh = [prob.relax_step(opts, t, b, z)["fhat"] for t in range(T)]
        errs[prec] = (relerr(fh, np.array(info["fhat"])), relerr(z.cpu().numpy(), z_ref))
        prob.close()
    print("fixed-iteration relax vs oracle (fhat, z):", errs)
    assert errs["mixed"][0] < 1e-3 and errs["mixed"][1] < 1e-3
    assert errs["mixed_fast"][0] < 1e-3 and errs["mixed_fast"][1] < 1e-3


@pytest.mark.parametrize("n,d,c,b", [(3000, 20, 10, 10), (6000, 64, 37, 12), (2500, 128, 5, 8),
                                     (4000, 16, 150, 10)])
def test_mixed_round_matches_oracle_while_gaps_are_clear(api, handle, n, d, c, b):
    """Round (Alg. 3) with tensor-core eq. 14 scores against the FP64 oracle.  While the two
    histories agree, every pick must equal the oracle's when its top-1/top-2 gap exceeds 1e-3,
    and otherwise must be a valid near-tie (oracle score within 1e-3 of the best); comparison
    stops at the first valid divergence (the histories differ from there on)."""
    p = make_problem(n, d, c, seed=d + c, x_dtype="bf16", h_dtype="float32")
    prob = make(api, handle, p)
    z = np.full(p.n, float(b) / p.n)
    ref, info = approx.round_select(p, z, b, record=True)
    sel, st = prob.round(dev(z.astype(np.float32)), b)
    sel = sel.cpu().tolist()
    compared = 0
    for t in range(b):
        if sel[t] == ref[t]:
            compared += 1
            continue
        sc = info["scores"][t]
        assert info["gap"][t] <= 1e-3, (t, sel[:t + 1], ref[:t + 1])
        assert sc[sel[t]] >= sc[ref[t]] - 1e-3 * abs(sc[ref[t]]), (t, sc[sel[t]], sc[ref[t]])
        break
    print(f"mixed round n={n} d={d} c={c} b={b}: {compared} of {b} picks identical, "
          f"first gaps {np.round(info['gap'][:4], 4).tolist()}")


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_round_full_pipeline_shapes_vs_oracle(api, handle, precision):
    """Round at the full-pipeline shapes (d = 128, c = 100, anisotropic clusters, Zipf 1.1
    priors) on a 2000-point pool, from a non-uniform relaxed z: picks equal the oracle's while
    its top-1/top-2 gap exceeds 1e-3, otherwise they are valid near-ties."""
    # seed 4: every oracle top-1/top-2 gap exceeds 1e-3, so all picks must agree
    p = make_problem(2000, 128, 100, seed=4, x_dtype="bf16", h_dtype="float32",
                     anisotropic=True, zipf=1.1)
    prob = make(api, handle, p, precision)
    b = 6
    z = np.random.default_rng(2).gamma(2.0, 1.0, p.n)
    z *= b / z.sum()
    ref, info = approx.round_select(p, z, b, record=True)
    sel, _ = prob.round(dev(z.astype(np.float32)), b)
    sel = sel.cpu().tolist()
    same = 0
    for t in range(b):
        if sel[t] == ref[t]:
            same += 1
            continue
        sc = info["scores"][t]
        assert info["gap"][t] <= 1e-3, (t, sel[:t + 1], ref[:t + 1])
        assert sc[sel[t]] >= sc[ref[t]] - 1e-3 * abs(sc[ref[t]])
        break
    print(f"{precision} round d=128 c=100: {same} of {b} picks identical, "
          f"gaps {np.round(info['gap'], 4).tolist()}")


def test_tuning_round_trip_chain_bound_and_numerics(api, handle, tmp_path):
    """Per-problem launch tuning: the values used are reported, the D-GEMM split count is held
    at the accumulation-chain bound, other split counts reorder sums only, and the autotuner
    stores its pick in the cache."""
    from paper_2409_07392_gb300 import autotune
    p = make_problem(100_000, 64, 40, seed=31, x_dtype="bf16", h_dtype="float32", m_o=40)
    prob = make(api, handle, p, "mixed_fast")
    rng = np.random.default_rng(2)
    V = dev(rng.standard_normal((8, 64 * 40)).astype(np.float32))
    z = dev(rng.uniform(0.1, 1.0, p.n).astype(np.float32))
    ref = prob.hessian_apply(V, z, op=0).cpu().numpy()
    used = prob.get_tuning()
    assert used["dterm_splits"] >= 4 and used["bsum_splits"] >= 1 and used["sm_budget"] > 0
    prob.set_tuning(dterm_splits=1, bsum_splits=3)
    got = prob.hessian_apply(V, z, op=0).cpu().numpy()
    t = prob.get_tuning()
    # 100,000 points = 1,563 K-steps: the chain bound (512 K-steps per split) needs 4 splits
    assert t["dterm_splits"] == 4 and t["bsum_splits"] == 3
    # other split counts only regroup the f32 partial sums (chains of <= 512 K-steps)
    assert relerr(got, ref) < 2e-4
    prob.set_tuning(dterm_splits=2 * used["dterm_splits"])
    got2 = prob.hessian_apply(V, z, op=0).cpu().numpy()
    assert relerr(got2, ref) < 2e-4
    cache = autotune.TuneCache(str(tmp_path / "tune.json"))
    rec = autotune.tune_problem(prob, 8, cg_iters=2, reps=1, cache=cache)
    assert rec["ms"] <= rec["default_ms"] and rec["candidates"] >= 2
    assert cache.get(autotune.shape_key("mixed_fast", p.n, 64, 40, 8)) is not None
    prob.close()
