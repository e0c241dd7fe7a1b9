"""Exact-FIRAL (Algorithm 1) on the GPU against the FP64 oracle: the objective f(z) and the
exact gradient (eqs. 4-7), the Relax iterates, and the Round picks with their traces and nu
(eqs. 8-10).  Sizes span several 64-wide factorisation panels and 128-wide GEMM tiles with
ragged tails (d c = 299, 1200).  Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import exact  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4, "mixed_fast": 1e-4}


@pytest.fixture(scope="module")
def api():
    from paper_2409_07392_gb300 import api, build
    build.build()
    return api


def make(api, p, precision):
    H = api.Handle()
    dt = torch.float64 if precision == "fp64" else torch.float32
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)
    return api.Problem(H, t(p.X), t(p.h), t(p.Xo), t(p.ho), p.lam, precision=precision)


def simplex_point(n, b, seed):
    z = np.random.default_rng(seed).gamma(2.0, 1.0, n)
    return z * (b / z.sum())


@pytest.mark.parametrize("precision,n,d,c,seed", [
    ("fp64", 300, 6, 4, 0),        # d~ = 24: one tile
    ("fp64", 200, 13, 23, 1),      # d~ = 299: ragged panels and tiles
    ("fp32", 3000, 20, 10, 2),     # the small Gaussian-mixture workload (d~ = 200)
    ("fp32", 400, 13, 23, 3),
    ("fp32", 300, 40, 30, 4),      # d~ = 1200: 19 panels, five doubling levels
    ("mixed_fast", 500, 20, 10, 5),
])
def test_exact_objective_and_gradient_vs_oracle(api, precision, n, d, c, seed):
    p = make_problem(n, d, c, seed=seed)
    z = simplex_point(n, 10.0, seed + 100)
    Ho, Hp = exact.h_o(p), exact.h_p(p)
    f_ref = exact.objective(p, z, Ho, Hp)
    g_ref = exact.gradient(p, z, Ho, Hp)
    prob = make(api, p, precision)
    f, g = prob.exact_objective(torch.from_numpy(z))
    g = g.double().cpu().numpy()
    e_f = abs(f - f_ref) / abs(f_ref)
    e_g = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    e_gmax = np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))
    print(f"{precision} d~={d * c}: f {e_f:.2e} g {e_g:.2e} (max {e_gmax:.2e})")
    tol = TOL[precision]
    assert e_f < tol and e_g < tol and e_gmax < 10 * tol
    prob.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exact_relax_vs_oracle(api, precision):
    n, d, c, b, T = 1000, 20, 10, 10.0, 5
    p = make_problem(n, d, c, seed=6)
    z_ref, hist_ref = exact.relax(p, b, T)
    prob = make(api, p, precision)
    z, hist = prob.exact_relax(b, T)
    z = z.double().cpu().numpy()
    assert abs(z.sum() - b) < 1e-6 * b and (z >= 0).all()
    e_z = np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref)
    e_h = np.max(np.abs(np.array(hist) - hist_ref) / np.abs(hist_ref))
    print(f"{precision}: z {e_z:.2e} f history {e_h:.2e}")
    tol = TOL[precision]
    assert e_z < 10 * tol and e_h < tol
    # the objective decreases along the iterates (the MD steps are descent steps here)
    assert hist[-1] < hist[0]
    prob.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,d,c,b,seed", [
    (200, 6, 4, 6, 3),
    (150, 13, 9, 5, 7),
    (100, 13, 23, 4, 4),     # d~ = 299
    (400, 20, 10, 5, 1),
])
def test_exact_round_vs_oracle(api, precision, n, d, c, b, seed):
    p = make_problem(n, d, c, seed=seed)
    z, _ = exact.relax(p, b, 3)
    sel_ref, r_ref, nu_ref = exact.round_exact(p, z, b, details=True)
    prob = make(api, p, precision)
    sel, r, nu = prob.exact_round(torch.from_numpy(z), b)
    sel = sel.cpu().tolist()
    e_r = np.max(np.abs(np.array(r) - r_ref) / np.abs(r_ref))
    e_nu = np.max(np.abs(np.array(nu) - nu_ref) / np.abs(nu_ref))
    print(f"{precision} d~={d * c}: picks {sel} vs {sel_ref}; trace {e_r:.2e} nu {e_nu:.2e}")
    assert sel == sel_ref
    tol = TOL[precision]
    assert e_r < tol and e_nu < tol
    prob.close()


def test_exact_round_repeats_allowed_when_not_excluded(api):
    n, d, c, b = 60, 5, 3, 8
    p = make_problem(n, d, c, seed=9)
    z, _ = exact.relax(p, b, 3)
    sel_ref = exact.round_exact(p, z, b, exclude_selected=False)
    prob = make(api, p, "fp64")
    sel, _, _ = prob.exact_round(torch.from_numpy(z), b, exclude_selected=False)
    assert sel.cpu().tolist() == sel_ref
    prob.close()


def test_exact_round_matches_brute_force_quality_tiny(api):
    """On this 12-point pool the oracle's picks attain the brute-force optimum of f(1_S); the
    GPU picks equal them."""
    n, d, c, b = 12, 3, 3, 3
    p = make_problem(n, d, c, seed=0)
    z, _ = exact.relax(p, b, 20)
    prob = make(api, p, "fp64")
    sel, _, _ = prob.exact_round(torch.from_numpy(z), b)
    sel = sel.cpu().tolist()
    assert sel == exact.round_exact(p, z, b)
    Ho, Hp = exact.h_o(p), exact.h_p(p)
    fstar, _ = exact.brute_force_best(p, b)
    assert exact.subset_objective(p, sel, Ho, Hp) <= fstar * (1 + 1e-12)
    prob.close()


def test_exact_errors(api):
    from paper_2409_07392_gb300 import _lib as L
    # d~ above the dense limit
    p = make_problem(20, 128, 129, seed=0)
    prob = make(api, p, "fp32")
    with pytest.raises(L.FiralError) as ei:
        prob.exact_objective(torch.ones(20))
    assert ei.value.code == L.FIRAL_ERR_UNSUPPORTED
    prob.close()
    # Round limited to c <= 112
    p = make_problem(30, 2, 113, seed=0)
    prob = make(api, p, "fp32")
    with pytest.raises(L.FiralError) as ei:
        prob.exact_round(torch.full((30,), 0.1), 3)
    assert ei.value.code == L.FIRAL_ERR_UNSUPPORTED
    prob.close()
    # negative weights make Sigma_z = H_o - sum_i H_i indefinite: no Cholesky factor
    p = make_problem(50, 4, 3, seed=0)
    prob = make(api, p, "fp64")
    with pytest.raises(L.FiralError) as ei:
        prob.exact_objective(torch.full((50,), -1.0))
    assert ei.value.code == L.FIRAL_ERR_NOT_SPD
    prob.close()
