"""Row-sharded Relax (the paper's data decomposition, Section 3.3) against the same problem
in one process (needs a GPU).

Two processes each hold half of the pool's rows on the one GPU and add their partial sums
over points through a gloo allreduce staged in host memory (no kernel of one process waits
for the other's).  After T mirror-descent iterations the concatenated z and the f^ history
must equal the single-process run: to double rounding in FP64 (the sums are only regrouped),
to float regrouping noise in FP32; in the mixed precisions both runs must be equally close to
the FP64 oracle.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import approx  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = dict(n=3001, d=16, c=10, s=6, T=2, iters=8, budget=20.0, seed=0)
TOL = {"fp64": 1e-11, "fp32": 2e-5}


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem(precision):
    mixed = precision.startswith("mixed")
    return make_problem(CASE["n"], CASE["d"], CASE["c"], seed=CASE["seed"],
                        x_dtype="bf16" if mixed else "float64",
                        h_dtype="float32" if mixed else "float64")


def single(precision):
    from paper_2409_07392_gb300 import api, build
    build.build()
    mixed = precision.startswith("mixed")
    p = problem(precision)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    X, Xo = dev(p.X), dev(p.Xo)
    if mixed:
        X, Xo = X.to(torch.bfloat16), Xo.to(torch.bfloat16)
    prob = api.Problem(api.Handle(), X, dev(p.h), Xo, dev(p.ho), p.lam, precision=precision)
    z = torch.full((p.n,), CASE["budget"] / p.n, dtype=prob.vdt, device="cuda")
    opts = prob.relax_opts(s=CASE["s"], T=CASE["T"], fixed_iters=CASE["iters"], seed=3)
    fh = [prob.relax_step(opts, t, CASE["budget"], z)["fhat"] for t in range(CASE["T"])]
    out = z.double().cpu().numpy(), np.array(fh)
    prob.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed", "mixed_fast"])
def test_two_process_row_shards_equal_one_process(tmp_path, precision):
    z_ref, f_ref = single(precision)
    port, world = free_port(), 2
    args = [f"--{k}={v}" for k, v in CASE.items()] + [f"--precision={precision}"]
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen(
            [sys.executable, os.path.join(ROOT, "tests", "shard_worker.py"), "--mode", "gpu",
             "--out", str(tmp_path / f"r{r}.npz"), *args], env=env, cwd=ROOT,
            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for pr in procs:
        out, err = pr.communicate(timeout=600)
        assert pr.returncode == 0, err[-3000:]
    res = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    assert res[0]["rows"][0] == 0 and res[-1]["rows"][1] == CASE["n"]
    z = np.concatenate([r["z"] for r in res])
    ez = np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref)
    ef = np.max(np.abs(res[0]["fhat"] - f_ref) / np.abs(f_ref))
    print(f"{precision} sharded x{world}: z {ez:.2e}  fhat {ef:.2e}")
    np.testing.assert_array_equal(res[0]["fhat"], res[1]["fhat"])   # every rank sees one f^
    assert abs(z.sum() - CASE["budget"]) < 1e-6 * CASE["budget"]
    if precision in TOL:
        assert ez < TOL[precision] and ef < TOL[precision]
    else:
        # the bf16 CG direction of this mode rounds the direction at every apply: a regrouped
        # f32 sum that moves an entry across a bf16 rounding boundary changes it by 2^-9, so
        # the two runs differ by this precision's own noise.  Both must be as close to the
        # FP64 oracle (same recurrences and probes) as each other.
        z_or, info = approx.relax(problem(precision), CASE["budget"], s=CASE["s"], T=CASE["T"],
                                  seed=3, fixed_iters=CASE["iters"])
        e_sh = np.linalg.norm(z - z_or) / np.linalg.norm(z_or)
        e_one = np.linalg.norm(z_ref - z_or) / np.linalg.norm(z_or)
        print(f"  vs oracle: sharded {e_sh:.2e}, one process {e_one:.2e}")
        assert e_sh < 1.5 * e_one + 1e-5 and e_sh < 1e-2


def test_bench_row_sharded_two_ranks(tmp_path):
    """bench.py's multi-rank path (one pool row-sharded over the ranks, strong scaling) runs
    end to end: two ranks on the one GPU, allreduces staged through host memory (gloo), a
    small pool.  A functional check of the launch, sharding and JSON line, not a measurement."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--gpus", "2", "--steps", "2", "--warmup", "3", "--workload", "cifar_like",
           "--data-backend", "gloo"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    import json
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["scaling"] == "strong" and line["value"] > 0
    assert line["setup"]["parallelism"].startswith("rows2")
    assert line["e2e"]["value"] > 0 and line["gpu_launches"] > 0
