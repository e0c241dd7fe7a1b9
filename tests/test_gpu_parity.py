"""CUDA path vs the FP64 oracle, element by element, through the C-ABI (needs a GPU).

FP64 runs must agree to rounding (1e-9 relative or tighter); FP32 runs carry float
rounding of the contractions (tolerances below are derived from the float epsilon and the
sum lengths, and are stated per test).  Shapes span several tiles (128-row CTAs, 64-wide
tiles, 16-class chunks) and ragged tails.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import approx  # noqa: E402
from oracle.probes import rademacher  # noqa: E402
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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def make(api, handle, p, precision):
    if p.x_bf16 and precision != "fp64":
        X, Xo = dev(p.X).to(torch.bfloat16), dev(p.Xo).to(torch.bfloat16)
    else:
        X, Xo = dev(p.X), dev(p.Xo)
    return api.Problem(handle, X, dev(p.h), Xo, dev(p.ho), p.lam, precision=precision)


def relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SHAPES = [(1, 1, 2), (7, 3, 2), (130, 5, 3), (300, 20, 10), (1000, 50, 10), (517, 64, 37),
          (260, 128, 4), (2049, 33, 17)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_probes_bit_exact(api, handle, precision):
    p = make_problem(50, 7, 5, seed=1, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, precision)
    for t in (0, 3):
        V = prob.probes(17, t, 6).cpu().numpy()
        np.testing.assert_array_equal(V.T, rademacher(17, t, 6, 35))


@pytest.mark.parametrize("n,d,c", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hessian_apply(api, handle, n, d, c, precision):
    p = make_problem(n, d, c, seed=n + d, x_dtype="float64", h_dtype="float64", m_o=c)
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(0)
    s = 3
    V = rng.standard_normal((d * c, s))
    z = rng.uniform(0.1, 1.0, n)
    ops = approx.Operators(p)
    ref_sig = ops.sigma_apply(z, V)
    ref_hp = ops.hp_apply(V)
    got_sig = prob.hessian_apply(dev(V.T), dev(z), op=0).cpu().numpy().T
    got_hp = prob.hessian_apply(dev(V.T), op=1).cpu().numpy().T
    # fp32: ~ sqrt(n) * 2^-24 growth on O(1) sums; 2e-5 relative in norm
    tol = 1e-11 if precision == "fp64" else 2e-5
    assert relerr(got_sig, ref_sig) < tol
    assert relerr(got_hp, ref_hp) < tol


@pytest.mark.parametrize("n,d,c", [(300, 20, 10), (517, 64, 37), (260, 128, 4)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_precond_blocks(api, handle, n, d, c, precision):
    p = make_problem(n, d, c, seed=3, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, precision)
    z = np.linspace(0.1, 2.0, n)
    ref = approx.Operators(p).precond_blocks(z)
    got = prob.precond_blocks(dev(z)).cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert relerr(got, ref) < tol
    np.testing.assert_allclose(prob.precond_blocks(None).cpu().numpy(),
                               approx.Operators(p).ho_blocks(), rtol=tol, atol=tol)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pcg_matches_direct_solution(api, handle, precision):
    p = make_problem(800, 10, 6, seed=4, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, precision)
    z = np.full(p.n, 5.0 / p.n)
    ops = approx.Operators(p)
    S = ops.sigma_dense(z)
    B = rademacher(2, 0, 4, 60)
    ref = np.linalg.solve(S, B)
    # FP32 recurrences stall near the float rounding of the residual: ask for 1e-5
    tol_cg = 1e-12 if precision == "fp64" else 1e-5
    X, iters, rr = prob.pcg(dev(z), dev(B.T), tol=tol_cg, maxit=400, check=False)
    X = X.cpu().numpy().T
    assert relerr(X, ref) < (1e-10 if precision == "fp64" else 1e-4)
    # same recurrences as the oracle's PCG: identical per-column iteration counts in FP64 at a
    # tolerance well above rounding (near 1e-12 the summation order can shift a count)
    if precision == "fp64":
        _, it_o, _ = approx.pcg(lambda P: ops.sigma_apply(z, P), B,
                                lambda R: approx.block_solve(
                                    approx.block_cholesky(ops.precond_blocks(z)), R),
                                tol=1e-8, maxit=400)
        _, it_g, _ = prob.pcg(dev(z), dev(B.T), tol=1e-8, maxit=400)
        # a column whose residual lands within rounding of the threshold may differ by one
        assert all(abs(int(a) - int(b)) <= 1 for a, b in zip(it_g, it_o))
        assert sum(int(a) == int(b) for a, b in zip(it_g, it_o)) >= len(it_o) - 1


def test_pcg_fixed_iterations_match_oracle_fp64(api, handle):
    p = make_problem(600, 8, 5, seed=5, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, "fp64")
    z = np.linspace(0.2, 1.0, p.n)
    ops = approx.Operators(p)
    chol = approx.block_cholesky(ops.precond_blocks(z))
    B = rademacher(9, 1, 3, 40)
    ref, _, _ = approx.pcg(lambda P: ops.sigma_apply(z, P), B,
                           lambda R: approx.block_solve(chol, R), fixed_iters=7)
    X, iters, _ = prob.pcg(dev(z), dev(B.T), fixed_iters=7)
    assert relerr(X.cpu().numpy().T, ref) < 1e-11
    assert iters == [7, 7, 7]


@pytest.mark.parametrize("n,d,c", [(130, 5, 3), (1000, 50, 10), (517, 64, 37), (260, 128, 4)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_quad_forms(api, handle, n, d, c, precision):
    p = make_problem(n, d, c, seed=7, x_dtype="float64", h_dtype="float64", m_o=2)
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(1)
    A, B = rng.standard_normal((d * c, 4)), rng.standard_normal((d * c, 4))
    ref = -approx.quad_forms(p.X, p.h, A, B)
    got = prob.quad_forms(dev(A.T), dev(B.T)).cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 3e-5
    assert relerr(got, ref) < tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_md_step(api, handle, precision):
    p = make_problem(3000, 4, 3, seed=8, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, precision)
    rng = np.random.default_rng(2)
    z = rng.uniform(0.1, 1, p.n)
    z = 10 * z / z.sum()
    g = rng.standard_normal(p.n)
    ref = approx.md_step(z, g, 10.0, 0.7)
    got = prob.md_step(dev(z), dev(g), 10.0, 0.7).cpu().numpy()
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert relerr(got, ref) < tol
    assert abs(got.sum() - 10.0) < (1e-11 if precision == "fp64" else 1e-4)


def test_relax_fp64_config1_shapes_match_oracle(api, handle):
    """FP64 Relax at the fp64_small workload (n=3000, d=20, c=10, s=10, T=20, b=10)."""
    p = make_problem(3000, 20, 10, seed=0, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, "fp64")
    b, s, T = 10.0, 10, 20
    z = torch.full((p.n,), b / p.n, dtype=torch.float64, device="cuda")
    opts = prob.relax_opts(s=s, T=T, fixed_iters=15, seed=1)
    fh = []
    for t in range(T):
        fh.append(prob.relax_step(opts, t, b, z)["fhat"])
    z_ref, info = approx.relax(p, b, s=s, T=T, seed=1, fixed_iters=15)
    np.testing.assert_allclose(fh, info["fhat"], rtol=1e-9)
    assert relerr(z.cpu().numpy(), z_ref) < 1e-8
    assert abs(z.sum().item() - b) < 1e-9


def test_relax_entry_point_tolerance_mode_fp64(api, handle):
    from paper_2409_07392_gb300.api import relax
    p = make_problem(700, 6, 4, seed=2, x_dtype="float64", h_dtype="float64")
    z, fh = relax(dev(p.X), dev(p.h), dev(p.Xo), dev(p.ho), p.lam, 5.0, s=4, T=4, tol=1e-3,
                  seed=5, precision="fp64", handle=handle)
    z_ref, info = approx.relax(p, 5.0, s=4, T=4, seed=5, tol=1e-3)
    np.testing.assert_allclose(fh, info["fhat"], rtol=1e-9)
    assert relerr(z.cpu().numpy(), z_ref) < 1e-8


def test_relax_fp32_vs_exact_solve_oracle(api, handle):
    """FP32 CG converged to 1e-6 vs the oracle with dense Cholesky solves: f^ and the
    per-step gradient within 1e-3 relative (the stated target)."""
    p = make_problem(5000, 10, 10, seed=3, x_dtype="float32", h_dtype="float32")
    prob = make(api, handle, p, "fp32")
    b, s, T = 20.0, 8, 3
    z = torch.full((p.n,), b / p.n, dtype=torch.float32, device="cuda")
    opts = prob.relax_opts(s=s, T=T, tol=1e-6, maxit=300, seed=4)
    fh = [prob.relax_step(opts, t, b, z)["fhat"] for t in range(T)]
    z_ref, info = approx.relax(p, b, s=s, T=T, seed=4, solve="direct")
    assert relerr(fh, info["fhat"]) < 1e-3
    assert relerr(z.cpu().numpy(), z_ref) < 1e-3


def test_round_fp64_matches_oracle(api, handle):
    p = make_problem(3000, 20, 10, seed=0, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, "fp64")
    z_ref, _ = approx.relax(p, 10.0, s=10, T=5, seed=1, fixed_iters=10)
    sel, st = prob.round(dev(z_ref), 10)
    ref, info = approx.round_select(p, z_ref, 10, record=True)
    assert sel.cpu().tolist() == ref
    assert abs(st["nu_last"] - info["nu"][-1]) < 1e-9 * abs(info["nu"][-1])


def test_round_fp32_selection_matches_when_gaps_are_clear(api, handle):
    p = make_problem(2000, 16, 6, seed=9, x_dtype="float32", h_dtype="float32")
    prob = make(api, handle, p, "fp32")
    z = np.full(p.n, 12.0 / p.n)
    ref, info = approx.round_select(p, z, 12, record=True)
    sel, _ = prob.round(dev(z, torch.float32), 12)
    sel = sel.cpu().tolist()
    # identical while every oracle top-1/top-2 gap exceeds 1e-3 (ties are reported)
    for t, g in enumerate(info["gap"]):
        if g <= 1e-3:
            break
        assert sel[t] == ref[t]


def test_block_eigvals_and_nu(api, handle):
    rng = np.random.default_rng(3)
    c, d = 5, 24
    Sig = np.stack([np.eye(d) + (lambda a: a @ a.T / d)(rng.standard_normal((d, d)))
                    for _ in range(c)])
    H = np.stack([(lambda a: a @ a.T)(rng.standard_normal((d, 5))) for _ in range(c)])
    got = handle.block_eigvals(dev(Sig), dev(H)).cpu().numpy()
    ref = approx.tilde_eigvals(np.linalg.cholesky(Sig), H)
    np.testing.assert_allclose(got, ref, atol=1e-10 * np.abs(ref).max())
    mu = 3.0 * ref.ravel()
    assert abs(handle.nu_bisect(dev(mu)) - approx.nu_bisect(mu)) < 1e-12 * approx.nu_bisect(mu)


def test_autograd_backward_fd_and_oracle(api, handle):
    """FiralObjective: backward vs central differences of its own forward (256 coordinates)
    and vs the oracle's same-probe exact derivative."""
    from paper_2409_07392_gb300.autograd import firal_objective
    p = make_problem(1500, 6, 5, seed=6, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, "fp64")
    z = torch.full((p.n,), 8.0 / p.n, dtype=torch.float64, device="cuda", requires_grad=True)
    f = firal_objective(z, prob, seed=3, t=0, s=6, tol=1e-13, maxit=400)
    f.backward()
    g = z.grad.cpu().numpy()
    for recompute in (True,):
        z2 = z.detach().clone().requires_grad_(True)
        firal_objective(z2, prob, seed=3, t=0, s=6, tol=1e-13, maxit=400,
                        recompute=recompute).backward()
        np.testing.assert_allclose(z2.grad.cpu().numpy(), g, rtol=1e-10, atol=1e-14)
    rng = np.random.default_rng(0)
    idx = rng.choice(p.n, 256, replace=False)
    zc = z.detach()
    for i in idx[:256]:
        eps = 1e-4 * zc[i].item()
        zp, zm = zc.clone(), zc.clone()
        zp[i] += eps
        zm[i] -= eps
        fp = prob.objective_fwd(zp, 3, 0, 6, tol=1e-13, maxit=400, keep=False)[0]
        fm = prob.objective_fwd(zm, 3, 0, 6, tol=1e-13, maxit=400, keep=False)[0]
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * np.abs(g).max()
    # oracle: same probes, exact solves
    ops = approx.Operators(p)
    S = ops.sigma_dense(zc.cpu().numpy())
    V = rademacher(3, 0, 6, p.d * p.c)
    U = np.linalg.solve(S, V)
    Y = np.linalg.solve(S, ops.hp_apply(V))
    ref = -approx.quad_forms(p.X, p.h, U, Y)
    assert relerr(g, ref) < 1e-9


def test_edge_cases(api, handle):
    # n = 1, c = 2, d = 1, no labelled set (lambda only)
    p = make_problem(1, 1, 2, seed=0, x_dtype="float64", h_dtype="float64", m_o=0)
    prob = api.Problem(handle, dev(p.X), dev(p.h), None, None, 1e-3, precision="fp64")
    V = np.array([[1.0, -1.0]])
    out = prob.hessian_apply(dev(V), dev(np.array([2.0])), op=0).cpu().numpy()
    ref = approx.Operators(p).sigma_apply(np.array([2.0]), V.T).T
    np.testing.assert_allclose(out, ref, rtol=1e-14)
    # invalid arguments are rejected, not run
    with pytest.raises(Exception):
        api.Problem(handle, dev(np.zeros((4, 129))), dev(np.full((4, 3), 1 / 3)), None, None,
                    1e-3, precision="fp32")
    with pytest.raises(Exception):
        prob.round(dev(np.array([1.0])), 2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_round_eta_sweep_vs_oracle(api, handle, precision):
    """Choosing eta (Section 5): Round per eta and the criterion min_k lambda_min(H_k) of the
    selected points' block-diagonal Hessian sum, against the oracle.  Picks agree while the
    oracle's gaps are clear; criteria agree to rounding; the chosen eta agrees."""
    p = make_problem(1500, 8, 4, seed=14, x_dtype="bf16" if precision == "mixed" else "float64",
                     h_dtype="float32" if precision == "mixed" else "float64")
    prob = make(api, handle, p, precision)
    b, etas = 8, [2.0, 12.0, 60.0]
    z = np.random.default_rng(3).gamma(2.0, 1.0, p.n)
    z *= b / z.sum()
    best_ref, crit_ref, sels_ref = approx.eta_sweep(p, z, b, etas)
    vdt = torch.float64 if precision == "fp64" else torch.float32
    sel, crit, best = prob.round_sweep(torch.from_numpy(z).to(vdt).cuda(), b, etas)
    sel = sel.cpu().numpy()
    for e in range(len(etas)):
        if list(sel[e]) == list(sels_ref[e]):
            # an eigenvalue moves by at most the perturbation's norm (Weyl): the tolerance
            # scales with the blocks (FP32 block sums in the mixed precision), not with the
            # possibly tiny smallest eigenvalue
            tol = 1e-9 if precision == "fp64" else 1e-5
            assert abs(crit[e] - crit_ref[e]) <= tol * max(crit_ref)
    print(f"{precision} eta sweep: criteria {np.round(crit, 6).tolist()} "
          f"(oracle {np.round(crit_ref, 6).tolist()}), best {best} (oracle {best_ref}), "
          f"selections equal {[list(sel[e]) == list(sels_ref[e]) for e in range(len(etas))]}")
    assert all(list(sel[e]) == list(sels_ref[e]) for e in range(len(etas)))
    assert best == best_ref


def test_block_pcg_fixed_iterations_match_oracle_fp64(api, handle):
    """Block PCG (O'Leary) through firal_pcg: the FP64 iterate after k steps equals the
    oracle's block_pcg iterate (same s x s recurrences).  k stays below d~/s, where the block
    Krylov space is exhausted and the s x s systems become singular (the GPU then freezes
    the iterate; there is no unique iterate to compare)."""
    p = make_problem(600, 10, 6, seed=5, x_dtype="float64", h_dtype="float64")
    prob = make(api, handle, p, "fp64")
    z = np.linspace(0.2, 1.0, p.n)
    ops = approx.Operators(p)
    chol = approx.block_cholesky(ops.precond_blocks(z))
    B = rademacher(9, 1, 6, 60)
    for k in (1, 4, 7):
        ref, _, _ = approx.block_pcg(lambda P: ops.sigma_apply(z, P), B,
                                     lambda R: approx.block_solve(chol, R), fixed_iters=k)
        X, iters, _ = prob.pcg(dev(z), dev(B.T), fixed_iters=k, block=True)
        assert relerr(X.cpu().numpy().T, ref) < 1e-10, k
        assert iters == [k] * 6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_pcg_converges_in_fewer_iterations(api, handle, precision):
    """Block PCG to a tight tolerance reaches the direct solution and needs no more iterations
    than the slowest of the s independent PCG recurrences (one shared Krylov space)."""
    p = make_problem(3000, 16, 10, seed=8, x_dtype="bf16" if precision == "mixed" else "float64",
                     h_dtype="float32" if precision == "mixed" else "float64")
    prob = make(api, handle, p, precision)
    z = np.full(p.n, 8.0 / p.n)
    ops = approx.Operators(p)
    B = rademacher(4, 0, 8, p.d * p.c)
    ref = np.linalg.solve(ops.sigma_dense(z), B)
    vdt = torch.float64 if precision == "fp64" else torch.float32
    zt, Bt = torch.from_numpy(z).to(vdt).cuda(), torch.from_numpy(B.T.copy()).to(vdt).cuda()
    tol = 1e-10 if precision == "fp64" else 1e-5
    Xb, itb, _ = prob.pcg(zt, Bt, tol=tol, maxit=500, block=True, check=False)
    Xc, itc, _ = prob.pcg(zt, Bt, tol=tol, maxit=500, check=False)
    eb = relerr(Xb.cpu().numpy().T, ref)
    ec = relerr(Xc.cpu().numpy().T, ref)
    print(f"{precision} block PCG: {itb[0]} iterations (independent: max {max(itc)}), "
          f"error {eb:.2e} (independent {ec:.2e})")
    assert eb < (1e-8 if precision == "fp64" else 2e-3)
    assert itb[0] <= max(itc)
