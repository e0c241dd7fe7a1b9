"""Row partition of the pool (the paper's data decomposition, Section 3.3) emulated on one GPU:
the split-K partitions of the point sums play the role of p ranks.  Results for p in
{1, 2, 4, 7} must agree to rounding (FP64: 1e-13; mixed: 1e-6)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, %r)
from paper_2409_07392_gb300 import api, build
from paper_2409_07392_gb300.synth import make_problem
build.build()
H = api.Handle()
out = {}
for prec in ("fp64", "mixed"):
    p = make_problem(5000, 24, 9, seed=2, x_dtype="bf16", h_dtype="float32")
    X = torch.from_numpy(p.X).cuda()
    Xo = torch.from_numpy(p.Xo).cuda()
    if prec == "mixed":
        X, Xo = X.to(torch.bfloat16), Xo.to(torch.bfloat16)
    prob = api.Problem(H, X, torch.from_numpy(p.h).cuda(), Xo, torch.from_numpy(p.ho).cuda(),
                       p.lam, precision=prec)
    rng = np.random.default_rng(0)
    V = torch.from_numpy(rng.standard_normal((4, 24 * 9))).cuda()
    z = torch.from_numpy(rng.uniform(0.1, 1, 5000)).cuda()
    out[prec] = prob.hessian_apply(V, z, op=0).double().cpu().numpy().tolist()
    prob.close()
print(json.dumps(out))
"""


def run(p):
    env = dict(os.environ, FIRAL_SPLITS=str(p))
    r = subprocess.run([sys.executable, "-c", CHILD % ROOT], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_virtual_shards_agree():
    res = {p: run(p) for p in (1, 2, 4, 7)}
    for prec, tol in (("fp64", 1e-13), ("mixed", 1e-6)):
        ref = np.array(res[1][prec])
        for p in (2, 4, 7):
            got = np.array(res[p][prec])
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, (prec, p)


CHILD_CHAIN = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, %r)
from paper_2409_07392_gb300 import api, build
from paper_2409_07392_gb300.synth import make_problem
build.build()
H = api.Handle()
p = make_problem(120000, 16, 10, seed=9, x_dtype="bf16", h_dtype="float32")
rng = np.random.default_rng(1)
V = torch.from_numpy(rng.standard_normal((4, 160))).cuda()
z = torch.from_numpy(rng.uniform(0.1, 1, p.n)).cuda()
out = {}
for prec in ("fp64", "mixed"):
    X, Xo = torch.from_numpy(p.X).cuda(), torch.from_numpy(p.Xo).cuda()
    if prec == "mixed":
        X, Xo = X.to(torch.bfloat16), Xo.to(torch.bfloat16)
    prob = api.Problem(H, X, torch.from_numpy(p.h).cuda(), Xo, torch.from_numpy(p.ho).cuda(),
                       p.lam, precision=prec)
    out[prec] = prob.hessian_apply(V, z, op=0).double().cpu().numpy()
    prob.close()
print(json.dumps(float(np.linalg.norm(out["mixed"] - out["fp64"]) / np.linalg.norm(out["fp64"]))))
"""


def test_one_split_over_all_points_stays_unbiased():
    """With one split the tensor-core block sums run over all 120,000 points (1,875 K-steps).
    Accumulating them in a single TMEM chain loses about 2^-25 of the sum per add, a bias of
    several 1e-4; the kernel folds short chains into an f32 accumulator instead, so the mixed
    apply stays at its rounding error (6 * 2^-9 / sqrt(n) ~ 3e-5)."""
    env = dict(os.environ, FIRAL_SPLITS="1")
    r = subprocess.run([sys.executable, "-c", CHILD_CHAIN % ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    err = json.loads(r.stdout.strip().splitlines()[-1])
    print(f"one split, n=120000: mixed apply vs fp64 {err:.2e}")
    assert err < 6.0 * 2.0 ** -9 / np.sqrt(120000) + 2e-5
