"""Device block cache: a destroyed problem's buffers are parked, a problem of the same shape
takes them back, results are unchanged, and trim empties the cache.  Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def test_park_reuse_trim_and_identical_results():
    from paper_2409_07392_gb300 import _lib as L, api, build
    build.build()
    lib = L.load()
    lib.firal_cache_trim()
    assert lib.firal_cache_bytes() == 0
    H = api.Handle()
    p = make_problem(30000, 32, 24, seed=8, x_dtype="bf16", h_dtype="float32")
    X = torch.from_numpy(p.X).cuda().to(torch.bfloat16)
    Xo = torch.from_numpy(p.Xo).cuda().to(torch.bfloat16)
    h, ho = torch.from_numpy(p.h).cuda(), torch.from_numpy(p.ho).cuda()
    V = torch.from_numpy(np.random.default_rng(1).standard_normal((4, 32 * 24))
                         .astype(np.float32)).cuda()
    z = torch.full((p.n,), 0.5, device="cuda")
    out = []
    for rep in range(2):
        prob = api.Problem(H, X, h, Xo, ho, p.lam, precision="mixed")
        out.append(prob.hessian_apply(V, z, op=0).cpu().numpy())
        prob.close()
        parked = lib.firal_cache_bytes()
        assert parked > 0
        if rep == 0:
            first = parked
    # the second problem took the first one's blocks and parked them again
    assert parked == first
    np.testing.assert_array_equal(out[0], out[1])
    assert lib.firal_cache_trim() == 0 and lib.firal_cache_bytes() == 0
