"""One process of a row-sharded group, for the sharding tests (started by them as a
subprocess with RANK, WORLD_SIZE, MASTER_ADDR and MASTER_PORT in its environment).

``--mode cpu``: checks ``api.torch_allreduce`` on host tensors over gloo (no GPU).
``--mode gpu``: holds its slice of a seeded pool (the paper's row partition, Section 3.3),
joins the group through ``Problem.set_comm`` (gloo, host-staged) and runs T mirror-descent
iterations; writes its z slice and the f^ history to ``--out``.
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", choices=["cpu", "gpu"], required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--n", type=int, default=3000)
    ap.add_argument("--d", type=int, default=16)
    ap.add_argument("--c", type=int, default=10)
    ap.add_argument("--s", type=int, default=6)
    ap.add_argument("--T", type=int, default=2)
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--budget", type=float, default=20.0)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    import torch
    import torch.distributed as dist
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2409_07392_gb300 import api
    if a.mode == "cpu":
        red = api.torch_allreduce()
        t = torch.arange(4, dtype=torch.float64) + 10.0 * rank
        red(t, "sum")
        u = torch.tensor([float(rank), -float(rank)], dtype=torch.float32)
        red(u, "max")
        np.savez(a.out, sum=t.numpy(), max=u.numpy(),
                 rows=np.array(api.shard_rows(a.n, world, rank)))
    else:
        from paper_2409_07392_gb300 import build
        from paper_2409_07392_gb300.synth import make_problem
        build.build()
        torch.cuda.set_device(0)
        mixed = a.precision.startswith("mixed")
        p = make_problem(a.n, a.d, a.c, seed=a.seed, x_dtype="bf16" if mixed else "float64",
                         h_dtype="float32" if mixed else "float64")
        lo, hi = api.shard_rows(a.n, world, rank)
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        X, Xo = dev(p.X[lo:hi]), dev(p.Xo)
        if mixed:
            X, Xo = X.to(torch.bfloat16), Xo.to(torch.bfloat16)
        H = api.Handle()
        prob = api.Problem(H, X, dev(p.h[lo:hi]), Xo, dev(p.ho), p.lam, precision=a.precision)
        prob.set_comm(rank, world, api.torch_allreduce())
        z = torch.full((hi - lo,), a.budget / a.n, dtype=prob.vdt, device="cuda")
        opts = prob.relax_opts(s=a.s, T=a.T, fixed_iters=a.iters, seed=3)
        fh = [prob.relax_step(opts, t, a.budget, z)["fhat"] for t in range(a.T)]
        np.savez(a.out, z=z.double().cpu().numpy(), fhat=np.array(fh), rows=np.array([lo, hi]))
        prob.close()
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
