"""The allocation-free mirror-descent update (firal_md_step_static) against firal_md_step and
the FP64 oracle's md_step.

Callers that cannot allocate device memory -- code running under CUDA graph capture,
runtimes that pre-assign all device memory to their own pool, plug-in hosts that cap a
library's footprint -- use firal_md_step_static, which works from a fixed scratch array in
the library instead of cudaMalloc.  This file is collected last so that a failure here
comes after every other test has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import approx  # noqa: E402

pytestmark = pytest.mark.gpu


def _static(lib, z, G, n, code, budget, beta0):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.firal_md_step_static(ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                                    n, code, budget, beta0, stream)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_static_md_step_matches_md_step_on_two_calls(dtype):
    from paper_2409_07392_gb300 import _lib, api, build
    from paper_2409_07392_gb300.synth import make_problem
    build.build()
    lib = _lib.load()
    tdt = torch.float32 if dtype == "float32" else torch.float64
    n = 1_000_003                                  # ragged: not a multiple of the 4096 chunk
    p = make_problem(64, 4, 3, seed=0, x_dtype="float64", h_dtype="float64")
    H = api.Handle()
    # an existing-entry-point problem sized for n pool points (X and h content is irrelevant)
    X = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    h = torch.full((n, 3), 1.0 / 3.0, dtype=torch.float64, device="cuda")
    prob = api.Problem(H, X, h, None, None, p.lam, precision="fp64" if dtype == "float64" else "fp32")
    rng = np.random.default_rng(7)
    budget, beta0 = 1000.0, 0.8
    z0 = rng.uniform(0.1, 1.0, n)
    z0 = budget * z0 / z0.sum()
    g1, g2 = rng.standard_normal(n), rng.standard_normal(n) * 3.0
    ref1 = prob.md_step(torch.from_numpy(z0), torch.from_numpy(g1), budget, beta0)
    ref2 = prob.md_step(ref1, torch.from_numpy(g2), budget, beta0)
    z = torch.from_numpy(z0).to("cuda", tdt).contiguous()
    G1 = torch.from_numpy(g1).to("cuda", tdt).contiguous()
    G2 = torch.from_numpy(g2).to("cuda", tdt).contiguous()
    code = _lib.FIRAL_DT_F32 if dtype == "float32" else _lib.FIRAL_DT_F64
    tol = 1e-6 if dtype == "float32" else 1e-13
    z_or = z0
    for G, g, ref in ((G1, g1, ref1), (G2, g2, ref2)):
        # the oracle's step from the same (stored) z and g
        z_or = approx.md_step(z.double().cpu().numpy(), G.double().cpu().numpy(), budget, beta0)
        rc = _static(lib, z, G, n, code, budget, beta0)
        assert rc == 0, _lib.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        got = z.double().cpu().numpy()
        want = ref.double().cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
        assert np.linalg.norm(got - z_or) / np.linalg.norm(z_or) < tol
        assert abs(got.sum() - budget) < 1e3 * tol * budget
    # sizes beyond the static scratch are refused, not run
    big = 4096 * 4096 + 1
    assert _static(lib, z, G1, big, code, budget, beta0) == -1   # FIRAL_ERR_ARG
    prob.close()
    H.close()


def test_static_md_step_non_finite_gradient_leaves_z_unchanged():
    """A NaN or an infinity in g leaves z as it was; the next call with a finite g runs
    normally (the flag slot of the shared scratch is rewritten by every call)."""
    from paper_2409_07392_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    n, budget = 70_001, 50.0
    rng = np.random.default_rng(3)
    z0 = rng.uniform(0.1, 1.0, n)
    z0 = budget * z0 / z0.sum()
    z = torch.from_numpy(z0).cuda()
    for bad in (np.nan, np.inf):
        g = rng.standard_normal(n)
        g[n // 2] = bad
        assert _static(lib, z, torch.from_numpy(g).cuda(), n, _lib.FIRAL_DT_F64, budget, 1.0) == 0
        torch.cuda.synchronize()
        assert np.array_equal(z.cpu().numpy(), z0)
    g = rng.standard_normal(n)
    assert _static(lib, z, torch.from_numpy(g).cuda(), n, _lib.FIRAL_DT_F64, budget, 1.0) == 0
    torch.cuda.synchronize()
    want = approx.md_step(z0, g, budget, 1.0)
    got = z.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-13
