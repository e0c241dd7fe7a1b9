"""CUDA-graph replay of MD iterations and the batched Relax entry point (needs a GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_07392_gb300.synth import batched_problems, make_problem  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2409_07392_gb300 import api as a, build
    build.build()
    return a


def dev(a, bf16=False):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t.to(torch.bfloat16) if bf16 else t


def prob_dict(p, budget):
    return dict(X=dev(p.X, p.x_bf16), h=dev(p.h), Xo=dev(p.Xo, p.x_bf16), ho=dev(p.ho),
                lam=p.lam, budget=budget)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_graph_replay_equals_eager_steps(api, precision):
    """firal_relax with fixed CG iterations replays a captured iteration; the result must equal
    T eager firal_relax_step calls bit for bit (same kernels, same order)."""
    p = make_problem(3000, 20, 10, seed=1, x_dtype="bf16" if precision == "mixed" else "float64",
                     h_dtype="float32" if precision == "mixed" else "float64")
    d = prob_dict(p, 10.0)
    H = api.Handle()
    z_graph, _ = api.relax(d["X"], d["h"], d["Xo"], d["ho"], p.lam, 10.0, s=6, T=5,
                           fixed_iters=6, seed=3, precision=precision, handle=H)
    prob = api.Problem(H, d["X"], d["h"], d["Xo"], d["ho"], p.lam, precision=precision)
    z = torch.full((p.n,), 10.0 / p.n, dtype=prob.vdt, device="cuda")
    opts = prob.relax_opts(s=6, T=5, fixed_iters=6, seed=3)
    for t in range(5):
        prob.relax_step(opts, t, 10.0, z, stats=False)
    torch.cuda.synchronize()
    assert torch.equal(z_graph, z)


def test_batched_relax_equals_individual_solves(api):
    shapes = batched_problems(6, seed=0)
    probs = [make_problem(min(sh["n"], 6000), sh["d"], sh["c"], seed=i, x_dtype="bf16",
                          h_dtype="float32") for i, sh in enumerate(shapes)]
    dicts = [prob_dict(p, float(sh["b"])) for p, sh in zip(probs, shapes)]
    H = api.Handle()
    zs = api.batched_relax(dicts, s=8, T=4, fixed_iters=5, seed=2, precision="mixed", handle=H)
    for dct, z in zip(dicts, zs):
        z1, _ = api.relax(dct["X"], dct["h"], dct["Xo"], dct["ho"], dct["lam"], dct["budget"],
                          s=8, T=4, fixed_iters=5, seed=2, precision="mixed", handle=H)
        assert torch.equal(z, z1)
        assert abs(z.double().sum().item() - dct["budget"]) < 1e-3 * dct["budget"]
