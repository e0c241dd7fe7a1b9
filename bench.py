#!/usr/bin/env python
"""Throughput of the Approx-FIRAL Relax mirror-descent iteration (Algorithm 2) on GB300.

One step = one MD iteration over the whole pool: probes, preconditioner blocks and their
FP64 factorisation, two block-Jacobi PCG solves of s columns with a fixed number of CG
iterations, the H_p apply and f^, the per-point gradient and the MD update.  The default
workload is the ImageNet-shaped pool (n = 1,000,000, d = 64, c = 1000, s = 16, X bf16,
h f32, 10 CG iterations per solve) in the mixed bf16 tensor-core precision.

Printed: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead
(on host cores, on a bounded subsample scaled to the full pool).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Relax MD iters/s at n=1M,c=1000 (mixed vs FP32 @≤1e-3 rel err); % TC peak"
UNIT = "MD iters/s"
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="imagenet_like")
    ap.add_argument("--n", type=int, default=None, help="pool size override (smaller runs)")
    ap.add_argument("--cg-iters", type=int, default=10)
    ap.add_argument("--precision", default="mixed_fast",
                    choices=["mixed", "mixed_fast", "fp32", "fp64"])
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the m=50, cg_tol=0.1 and hi/lo-direction sub-measurements")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="--impl reference: oracle work over all warm-up and timed steps")
    ap.add_argument("--no-round", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-exact", action="store_true")
    ap.add_argument("--no-al", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--round-selections", type=int, default=20)
    ap.add_argument("--batched-iters", type=int, default=5,
                    help="timed batched MD iterations (the batched sub-measurement)")
    ap.add_argument("--batched-pools", type=int, default=64,
                    help="pools of the batched workload (64; fewer for small profiling runs)")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: N independent problems instead of one row-sharded problem")
    ap.add_argument("--only", default=None, choices=["round", "batched", "exact", "al"],
                    help="run one sub-measurement alone and print its record (profiling runs)")
    ap.add_argument("--data-backend", default="nccl", choices=["nccl", "gloo"],
                    help="row-sharded runs: device allreduces over NCCL, or staged through host "
                         "memory over gloo (several ranks may then share one GPU: a functional "
                         "check, not a measurement)")
    return ap.parse_args()


def workload(args):
    from paper_2409_07392_gb300.synth import CONFIGS
    cfg = dict(CONFIGS[args.workload])
    if args.n is not None:
        cfg["n"] = args.n
    return cfg


def describe(cfg, args):
    return (f"{args.workload}: n={cfg['n']} d={cfg['d']} c={cfg['c']} s={cfg['s']} "
            f"cg_iters/solve={args.cg_iters} X={cfg['x_dtype']} h={cfg['h_dtype']}")


def config_of(cfg, args):
    """The ``config`` object of both arms' lines: the workload, and how the timed steps meet
    L2 (every input larger than the 129 MB L2; no flush needed)."""
    h_bytes = cfg["n"] * cfg["c"] * (8 if cfg["h_dtype"] == "float64" else 4)
    l2 = ("inputs larger than L2 (h alone is %.1f GB)" % (h_bytes / 1e9) if h_bytes > 129e6
          else "inputs smaller than L2 (h is %.1f MB): timed steps run warm" % (h_bytes / 1e6))
    return {"workload": describe(cfg, args), "l2": l2}


# ------------------------------------------------------------------------------ distributed
def dist_setup(args, data_backend=False):
    """Join the job's process group.  Host tensors (barrier, max over ranks) go over gloo;
    with ``data_backend`` device tensors (the row-sharded MD iteration's allreduces) go over
    NCCL, unless --data-backend gloo stages them through host memory."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        nccl = data_backend and getattr(args, "data_backend", "nccl") == "nccl"
        dist.init_process_group("cpu:gloo,cuda:nccl" if nccl else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ roofline
def algorithmic_flops(kind, cfg, n_all, s):
    """Algorithmic flops of one timed group of a kernel class: 2 N c d s for each GEMM of the
    Hessian apply, 2 N c d (d + 1) for the block sums, 4 n c d s for the gradient."""
    n, d, c = cfg["n"], cfg["d"], cfg["c"]
    if kind in ("apply_alpha", "apply_dterm"):
        return 2.0 * n_all * c * d * s
    if kind == "syrk_blocks":
        return 2 * 1.0 * n_all * c * d * (d + 1)    # S_k and B_k(Sigma_z), symmetric pairs
    if kind == "quad_forms":
        return 4.0 * n * c * d * s
    return None


def kernel_source_hash(path, fn):
    """First 16 hex digits of the SHA-256 of one kernel's source text: from the line that
    opens the template (or signature) of ``fn``'s definition to the closing brace in column 0.
    A traffic record stays valid while that text is unchanged."""
    import hashlib
    src = open(path).read()
    key = f" {fn}("
    i = src.find(key)
    while i >= 0 and "__global__" not in src[max(0, src.rfind("\n\n", 0, i)):i]:
        i = src.find(key, i + 1)
    if i < 0:
        return None
    start = src.rfind("\n\n", 0, i) + 2
    end = src.find("\n}\n", i)
    return hashlib.sha256(src[start:end + 3].encode()).hexdigest()[:16]


def dram_traffic(kind, n_rows_padded, precision):
    """DRAM bytes per launch of a kernel class from the committed ncu capture (small case):
    reads and row-proportional writes scale with the padded row count, split-K partial
    writes are fixed per launch.  None when the kernel's source changed since the capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
        k = rec["kernels"].get(f"{kind}/{precision}") or rec["kernels"].get(kind)
        if k is None:
            return None
        if kernel_source_hash(os.path.join(ROOT, rec["source"]), k["source_fn"]) != \
                k["source_sha256_16"]:
            return None
        return (k["read_bytes_per_padded_row"] + k["write_bytes_per_padded_row"]) * \
            n_rows_padded + k["write_bytes_fixed"]
    except Exception:
        return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


# ------------------------------------------------------------------------------ oracle timing
def _oracle_iteration_seconds(cfg, cg_iters, n1, seed=0):
    """Seconds of one oracle MD iteration (fixed CG iterations) on an n1-point pool."""
    from oracle import approx
    from paper_2409_07392_gb300.synth import make_problem
    n_full, d, c, s = cfg["n"], cfg["d"], cfg["c"], cfg["s"]
    p1 = make_problem(n1, d, c, seed=seed, x_dtype=cfg["x_dtype"], h_dtype=cfg["h_dtype"])
    t0 = time.perf_counter()
    approx.relax(p1, float(cfg["b"]) * n1 / n_full if n1 < n_full else float(cfg["b"]), s=s,
                 T=1, seed=1, fixed_iters=cg_iters)
    return time.perf_counter() - t0


def oracle_md_iteration_rate(cfg, cg_iters, seconds, seed=0):
    """The FP64 oracle's MD iterations/s at the full pool size, from two bounded samples.

    One MD iteration has per-point work (the Hessian applies, block sums and gradient, linear
    in n) and per-problem work (the c block factorisations and the d c x s CG vector updates,
    independent of n).  The oracle is timed on two subsamples, n1 and n1 / 2 points, sized
    for about ``seconds`` of work in all; the fit t(n) = a + b n through the two times is
    evaluated at the full n.  Returns a dict (value in MD iters/s, the fit, the sample)."""
    from oracle import approx
    from paper_2409_07392_gb300.synth import make_problem
    n_full, d, c, s = cfg["n"], cfg["d"], cfg["c"], cfg["s"]
    # calibrate on a small pool: one Sigma apply
    n0 = max(200, min(2000, n_full))
    p0 = make_problem(n0, d, c, seed=seed, x_dtype=cfg["x_dtype"], h_dtype=cfg["h_dtype"])
    ops = approx.Operators(p0)
    V = np.ones((d * c, s))
    t0 = time.perf_counter()
    ops.sigma_apply(np.full(n0, 1.0 / n0), V)
    t_apply = time.perf_counter() - t0
    per_iter_est = t_apply * (2 * cg_iters + 4) * 1.3
    n1 = int(max(2 * n0, min(n_full, n0 * (seconds / 1.5) / max(per_iter_est, 1e-3))))
    n2 = n1 // 2
    t1 = _oracle_iteration_seconds(cfg, cg_iters, n1, seed)
    t2 = _oracle_iteration_seconds(cfg, cg_iters, n2, seed)
    b = max((t1 - t2) / (n1 - n2), 0.0)
    a = max(t1 - b * n1, 0.0)
    if b == 0.0:                       # timing noise: fall back to proportional scaling
        a, b = 0.0, t1 / n1
    t_full = a + b * n_full
    return {"value": 1.0 / t_full,
            "sample": f"one MD iteration ({cg_iters} CG iterations per solve) timed on n={n1} "
                      f"and n={n2} of {n_full} points ({t1:.2f} s, {t2:.2f} s); "
                      f"extrapolated with t(n) = a + b n",
            "fit": {"a_s": a, "b_s_per_point": b, "n_samples": [n1, n2],
                    "seconds": [t1, t2]},
            "extrapolated": n1 < n_full}


def oracle_rate_one_core(cfg, cg_iters, seconds):
    """The same measurement in a child process limited to one thread (BLAS, OpenMP) and, where
    the OS allows, pinned to one core."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_md_iteration_rate(%r, %d, %f)))"
            % (ROOT, cfg, cg_iters, seconds))
    pre = []
    if hasattr(os, "sched_getaffinity"):
        try:
            core = sorted(os.sched_getaffinity(0))[0]
            pre = ["taskset", "-c", str(core)] if subprocess.run(
                ["taskset", "-c", str(core), "true"], capture_output=True).returncode == 0 else []
        except Exception:
            pre = []
    r = subprocess.run(pre + [sys.executable, "-c", code], env=env, capture_output=True,
                       text=True, timeout=max(120.0, 8 * seconds))
    if r.returncode != 0:
        return {"error": (r.stderr or r.stdout)[-300:]}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["cores"] = 1
    out["pinned"] = bool(pre)
    return out


def cpu_baseline(cfg, cg_iters, seconds, one_core=True):
    """The oracle baseline on all host cores (value) and on one core (beside it)."""
    rec = oracle_md_iteration_rate(cfg, cg_iters, seconds)
    out = {"value": rec["value"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": rec["sample"], "fit": rec["fit"], "extrapolated": rec["extrapolated"],
           "threads_note": "numpy with its BLAS on all host cores; elementwise work on one"}
    if one_core:
        one = oracle_rate_one_core(cfg, cg_iters, seconds)
        out["one_core"] = ({"value": one["value"], "unit": UNIT, "cores": 1,
                            "pinned": one.get("pinned"), "sample": one["sample"],
                            "fit": one["fit"]} if "value" in one else one)
    return out


def round_measure(args, H):
    """Per-selection time of the Round scan (eq. 14 scores, block update, eigenvalues, nu,
    B^-1) on the full_pipeline pool (n = 1M, d = 128, c = 100), mixed and plain FP32."""
    import torch

    from paper_2409_07392_gb300 import api
    from paper_2409_07392_gb300.synth import CONFIGS, config_problem
    cfg = CONFIGS["full_pipeline"]
    p = config_problem("full_pipeline")
    X = torch.from_numpy(p.X).cuda().to(torch.bfloat16)
    Xo = torch.from_numpy(p.Xo).cuda().to(torch.bfloat16)
    h, ho = torch.from_numpy(p.h).cuda(), torch.from_numpy(p.ho).cuda()
    out = {"workload": f"full_pipeline: n={p.n} d={p.d} c={p.c} (anisotropic, Zipf 1.1)",
           "unit": "selections/s"}
    b = float(cfg["b"])
    mixed = args.precision if args.precision.startswith("mixed") else "mixed"
    relax = {"unit": UNIT, "cg_iters/solve": args.cg_iters, "s": cfg["s"]}
    sels = {}
    nover = 4
    for prec, nsel in ((mixed, args.round_selections), ("fp32", 2)):
        prob = api.Problem(H, X, h, Xo, ho, p.lam, precision=prec)
        # Relax at this workload: one MD iteration from the uniform z (same probes for both
        # precisions), then the time per MD iteration
        z = torch.full((p.n,), b / p.n, dtype=torch.float32, device="cuda")
        o = prob.relax_opts(s=cfg["s"], T=8, fixed_iters=args.cg_iters, seed=1)
        st = prob.relax_step(o, 0, b, z)
        k = 3 if prec != "fp32" else 1
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        zt = z.clone()
        e0.record()
        for t in range(1, 1 + k):
            prob.relax_step(o, t, b, zt, stats=False)
        e1.record()
        torch.cuda.synchronize()
        relax[prec] = {"value": 1000.0 * k / e0.elapsed_time(e1), "fhat": st["fhat"], "z": z}
        # Round: per-selection time
        zr = torch.full((p.n,), b / p.n, dtype=torch.float32, device="cuda")
        prob.round(zr, 1)                       # warm-up (and set-up cost)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.round(zr, 1)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sel, _ = prob.round(zr, max(1 + nsel, nover))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        per = ((t2 - t1) - (t1 - t0)) / (max(1 + nsel, nover) - 1)
        sels[prec] = sel[:nover].cpu().tolist()
        if prec != "fp32" and not args.no_variants:
            # choosing eta (Section 5): Round per eta on the same z, keep the best-conditioned
            eta0 = 8.0 * (p.d * p.c) ** 0.5
            etas = [0.25 * eta0, eta0, 4.0 * eta0]
            bs = 10
            torch.cuda.synchronize()
            ts = time.perf_counter()
            _, crit, best = prob.round_sweep(zr, bs, etas)
            torch.cuda.synchronize()
            t_sweep = time.perf_counter() - ts
            # the same chains one after another (one Round call per eta) for comparison
            ts = time.perf_counter()
            for e in etas:
                prob.round(zr, bs, eta=e)
            torch.cuda.synchronize()
            t_seq = time.perf_counter() - ts
            out["eta_sweep"] = {"etas": etas, "budget": bs, "criteria_min_lambda_min": crit,
                                "best": best, "seconds": t_sweep,
                                "seconds_one_round_per_eta": t_seq,
                                "note": "the chains of all eta side by side (one score launch "
                                        "per pick for all of them, set-up shared), criterion "
                                        "min_k lambda_min of the selected points' Hessian "
                                        "blocks; beside it, one Round call per eta"}
        out["fp32" if prec == "fp32" else "mixed"] = {
            "precision": prec, "value": 1.0 / per, "ms_per_selection": 1000.0 * per,
            "selections": max(1 + nsel, nover), "setup_ms": 1000.0 * (t1 - t0)}
        prob.close()
    out["speedup_mixed_over_fp32"] = out["mixed"]["value"] / out["fp32"]["value"]
    prefix = 0
    while prefix < nover and sels[mixed][prefix] == sels["fp32"][prefix]:
        prefix += 1
    out["selection_prefix_equal_mixed_vs_fp32"] = f"{prefix}/{nover}"
    out["selection_note"] = ("with 1M candidates the eq. 14 maxima are near-ties and the "
                             "histories diverge after the first differing pick; the parity test "
                             "at d=128, c=100 with clear gaps agrees 6/6 with the oracle")
    zm, z32 = relax[mixed].pop("z"), relax["fp32"].pop("z")
    relax["fhat_rel_diff_mixed_vs_fp32"] = abs(relax[mixed]["fhat"] - relax["fp32"]["fhat"]) / \
        abs(relax["fp32"]["fhat"])
    relax["z_rel_diff_mixed_vs_fp32"] = float((zm.double() - z32.double()).norm() /
                                              z32.double().norm())
    out["relax"] = relax
    return out


def exact_measure(args, H):
    """Exact-FIRAL (Algorithm 1, dense d~ x d~, FP32) against Approx-FIRAL on the same pools,
    shaped like the paper's Table 5 workloads: ImageNet-50 (n = 5,000, d = 50, c = 50,
    b = 50) and Caltech-101 (n = 1,715, d = 100, c = 101, b = 101), synthetic Gaussian-mixture
    embeddings.  Relax is timed per MD iteration (approx: s = 10 probes, CG to tol 0.1 as in
    Section 5), Round per pick (difference of two budgets, so the set-up cancels)."""
    import torch

    from paper_2409_07392_gb300 import api
    from paper_2409_07392_gb300.synth import make_problem
    paper = {"imagenet50": {"exact_relax_s": 33.6, "exact_round_s": 34.8, "approx_relax_s": 1.3,
                            "approx_round_s": 1.1},
             "caltech101": {"exact_relax_s": 172.3, "exact_round_s": 945.3,
                            "approx_relax_s": 1.9, "approx_round_s": 4.4}}
    out = {"note": "Table 5 of the paper, same shapes on synthetic data; paper figures are whole "
                   "solves on one A100 (context, not a target)"}
    for name, (n, d, c, b, k_rel, picks) in (("imagenet50", (5000, 50, 50, 50, 3, (2, 6))),
                                             ("caltech101", (1715, 100, 101, 101, 1, (1, 3)))):
        p = make_problem(n, d, c, seed=0)
        t = lambda a: torch.from_numpy(a).cuda().float()
        rec = {"n": n, "d": d, "c": c, "d_tilde": d * c, "b": b, "paper_a100": paper[name]}
        for kind, prec in (("exact", "fp32"), ("approx", "mixed_fast")):
            prob = api.Problem(H, t(p.X), t(p.h), t(p.Xo), t(p.ho), p.lam, precision=prec)
            z = torch.full((n,), b / n, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            if kind == "exact":
                prob.exact_relax(b, 1, z0=z)                      # warm-up (workspace)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                zr, hist = prob.exact_relax(b, k_rel, z0=z)
                torch.cuda.synchronize()
                relax_s = (time.perf_counter() - t0) / k_rel
                rnd = lambda bb: prob.exact_round(zr, bb)
            else:
                o = prob.relax_opts(s=10, T=k_rel + 1, tol=0.1, maxit=100, seed=1)
                prob.relax_step(o, 0, b, z)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for it in range(1, 1 + 3 * k_rel):
                    prob.relax_step(o, it, b, z, stats=False)
                torch.cuda.synchronize()
                relax_s = (time.perf_counter() - t0) / (3 * k_rel)
                zr = z
                rnd = lambda bb: prob.round(zr, bb)
            rnd(1)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rnd(picks[0])
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            rnd(picks[1])
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            per_pick = ((t3 - t2) - (t2 - t1)) / (picks[1] - picks[0])
            setup = max(0.0, (t2 - t1) - picks[0] * per_pick)
            rec[kind] = {"precision": prec, "relax_ms_per_md_iter": 1000.0 * relax_s,
                         "round_ms_per_pick": 1000.0 * per_pick, "round_setup_ms": 1000.0 * setup,
                         "round_total_s_at_b": setup + b * per_pick}
            prob.close()
            torch.cuda.empty_cache()
        rec["exact_over_approx_relax_per_iter"] = rec["exact"]["relax_ms_per_md_iter"] / \
            rec["approx"]["relax_ms_per_md_iter"]
        rec["exact_over_approx_round"] = rec["exact"]["round_total_s_at_b"] / \
            rec["approx"]["round_total_s_at_b"]
        out[name] = rec
    return out


def al_measure(args, H):
    """The active-learning outer loop (Section 5) on the ImageNet-50 shape: n = 5,000 pool
    points, d = 50, c = 50, one labelled point per class, 6 rounds of b = 50, each round a
    classifier refit, Relax (s = 10 probes, CG to tol 0.1, MD until the relative change of f^
    is below 1e-4, at most 100 iterations, as in Section 5) and Round; synthetic mixture
    labels."""
    import torch

    from paper_2409_07392_gb300 import api
    from paper_2409_07392_gb300.synth import make_problem
    n, d, c, rounds, b = 5000, 50, 50, 6, 50
    p = make_problem(n, d, c, seed=0)
    X = torch.from_numpy(p.X).cuda()
    Xo = torch.from_numpy(p.Xo).cuda()
    y = torch.from_numpy(p.labels).cuda()
    yo = torch.arange(p.Xo.shape[0], device="cuda") % c
    kw = dict(precision=args.precision if args.precision.startswith("mixed") else "mixed_fast",
              s=10, T=100, tol=0.1, maxit=100, md_tol=1e-4, handle=H)
    api.active_learning(X, y, Xo, yo, c, 1, b, **kw)                 # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sel, W, fh = api.active_learning(X, y, Xo, yo, c, rounds, b, **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # pool accuracy of the final classifier (a sanity figure, not a claim)
    pred = api.lr_probs(X, W, precision="fp32", handle=H).argmax(dim=1)
    acc = float((pred == y).float().mean())
    return {"workload": f"imagenet50 shape: n={n} d={d} c={c}, {rounds} rounds x b={b}",
            "precision": kw["precision"], "seconds_total": dt, "seconds_per_round": dt / rounds,
            "fhat_last_per_round": fh, "final_pool_accuracy": acc,
            "note": "refit + Relax (md_tol 1e-4) + Round per round; synthetic mixture labels"}


def cg_variants(prob, s, b, n):
    """MD iterations/s at m = 50 CG iterations per solve (the paper's timing setting), in
    tolerance mode (cg_tol = 0.1, the paper's default) and at cg_tol = 1e-3 with independent
    and with block PCG, each with the iterations reached."""
    import torch
    out = {}
    for label, kw in (("cg_iters_50", dict(fixed_iters=50)), ("cg_tol_0.1", dict(tol=0.1)),
                      ("cg_tol_1e-3", dict(tol=1e-3)),
                      ("cg_tol_1e-3_block", dict(tol=1e-3, block_cg=True))):
        z = torch.full((n,), b / n, dtype=prob.vdt, device="cuda")
        o = prob.relax_opts(s=s, T=3, seed=1, **kw)
        prob.relax_step(o, 0, b, z, stats=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        e0.record()
        for t in (1, 2):
            its.append(prob.relax_step(o, t, b, z)["cg_iters"])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        out[label] = {"value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms,
                      "cg_iters_per_solve": its}
    return out


def batched_measure(args, H):
    """Batched Relax on the batched_uneven workload (64 pools, n ~ U[2000, 40000], d in
    {16,32,48,64}, c in {5,10,20}, s = 8): batched MD iterations per second (one iteration of
    every pool, replayed from a CUDA graph), with HBM and tensor fractions on algorithmic work."""
    import torch

    from paper_2409_07392_gb300 import api
    from paper_2409_07392_gb300.synth import batched_problems, make_problem
    shapes = batched_problems(args.batched_pools, seed=0)
    dicts, npts, flops_apply, bytes_apply = [], 0, 0.0, 0.0
    s = 8
    for i, sh in enumerate(shapes):
        p = make_problem(sh["n"], sh["d"], sh["c"], seed=i, x_dtype="bf16", h_dtype="float32")
        dicts.append(dict(X=torch.from_numpy(p.X).cuda().to(torch.bfloat16),
                          h=torch.from_numpy(p.h).cuda(),
                          Xo=torch.from_numpy(p.Xo).cuda().to(torch.bfloat16),
                          ho=torch.from_numpy(p.ho).cuda(), lam=p.lam, budget=float(sh["b"])))
        n, d, c = sh["n"], sh["d"], sh["c"]
        npts += n
        flops_apply += 4.0 * n * c * d * s
        bytes_apply += n * (2 * d + 4 * c + 4) + 8.0 * d * c * s
    cg = args.cg_iters
    K = max(1, args.batched_iters)
    bprec = args.precision if args.precision.startswith("mixed") else "mixed_fast"

    def run(T):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.batched_relax(dicts, s=s, T=T, fixed_iters=cg, seed=1, precision=bprec, handle=H)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    run(2)                                   # warm-up (module loading, attributes)
    tuned = None
    if not args.no_autotune:
        from paper_2409_07392_gb300 import autotune

        def one_iter_ms():
            a = run(2)
            return 1000.0 * (run(4) - a) / 2
        tuned = autotune.tune_handle(H, one_iter_ms)
    t1 = run(2)
    tk = run(2 + K)
    per = (tk - t1) / K
    H.set_default_tuning(0, 0, 0)
    applies = 2 * cg + 1
    pk, _ = peaks()
    return {"workload": f"batched_uneven: {len(shapes)} pools, {npts} points in all, s={s}, "
                        f"cg_iters/solve={cg}", "precision": bprec,
            "value": 1.0 / per, "unit": "batched MD iters/s", "ms_per_iteration": 1000 * per,
            "hbm_frac_of_measured": applies * bytes_apply / per / 1e9 / pk["hbm_gbs"],
            "tensor_frac_of_measured": applies * flops_apply / per / 1e12 /
            pk["bf16_tflops_sustained"],
            "tuning": tuned,
            "note": "fractions on algorithmic Sigma-apply work only (bytes n(2d+4c+4) per apply)"}


def run_reference(args):
    """The FP64 oracle timed on the host cores, on this workload.  The first step fits
    t(n) = a + b n from two bounded samples (about --ref-seconds / 8 of estimated work, at
    most 15 s); every later step times one oracle MD iteration on a 250-point sample and
    extrapolates it to the full n with the fitted slope b, so a run of many steps stays
    within minutes."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    cfg = workload(args)
    n_full = cfg["n"]
    rates = []
    rec = oracle_md_iteration_rate(cfg, args.cg_iters,
                                   seconds=max(1.0, min(15.0, args.ref_seconds / 8)))
    fit = rec["fit"]
    n_s = min(n_full, 250)
    step_times = []
    for i in range(args.warmup + args.steps):
        if i == 0:
            v = rec["value"]
        else:
            t = _oracle_iteration_seconds(cfg, args.cg_iters, n_s)
            step_times.append(t)
            v = 1.0 / (t + fit["b_s_per_point"] * (n_full - n_s))
        if i >= args.warmup:
            rates.append(v)
    v = float(np.mean(rates))
    cores = os.cpu_count()
    extrap = n_s < n_full or rec["extrapolated"]
    sample = (rec["sample"] + (f"; each later step: one MD iteration on n={n_s} points "
                               f"(mean {np.mean(step_times):.2f} s), extrapolated with the "
                               f"fitted slope" if step_times else ""))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(cfg, args),
            "extrapolated": ("every step times the FP64 oracle on a sample of the pool and "
                             "extrapolates t(n) = a + b n to the full n; ms_per_step is that "
                             "extrapolated time" if extrap else False),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "fit": fit},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    from paper_2409_07392_gb300 import _lib, api, build
    from paper_2409_07392_gb300.synth import make_problem

    world0 = int(os.environ.get("WORLD_SIZE", "1"))
    # N > 1: one pool row-sharded over the ranks (the paper's decomposition; strong scaling),
    # unless --replicas asks for N independent problems (weak scaling)
    shard = world0 > 1 and not args.replicas
    world, rank, local = dist_setup(args, data_backend=shard)
    torch.cuda.set_device(local % torch.cuda.device_count())
    build.build()
    lib = _lib.load()
    cfg = workload(args)
    n, d, c, s, b = cfg["n"], cfg["d"], cfg["c"], cfg["s"], float(cfg["b"])
    p = make_problem(n, d, c, seed=0 if shard else rank, x_dtype=cfg["x_dtype"],
                     h_dtype=cfg["h_dtype"], anisotropic=cfg.get("anisotropic", False),
                     zipf=cfg.get("zipf"))
    lo, hi = api.shard_rows(n, world, rank) if shard else (0, n)
    n_loc = hi - lo
    xdt = torch.bfloat16 if p.x_bf16 else torch.float32

    def host(a, dt=None):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return (t.to(dt) if dt is not None else t).pin_memory()

    Xh, hh, Xoh, hoh = host(p.X[lo:hi], xdt), host(p.h[lo:hi]), host(p.Xo, xdt), host(p.ho)
    X, h, Xo, ho = (t.cuda(non_blocking=True) for t in (Xh, hh, Xoh, hoh))
    H = api.Handle()
    prob = api.Problem(H, X, h, Xo, ho, p.lam, precision=args.precision)
    if shard:
        prob.set_comm(rank, world, api.torch_allreduce())
    # launch tuning: the autotuner times split-count candidates on MD iterations (outside the
    # timed region) and leaves the fastest set on the problem (not on a sharded problem: every
    # rank must make the same allreduce calls)
    tuning = None
    if args.precision.startswith("mixed") and not args.no_autotune and not shard:
        from paper_2409_07392_gb300 import autotune
        tuning = autotune.tune_problem(prob, s, cg_iters=args.cg_iters, budget=b, reps=2)
    z = torch.full((n_loc,), b / n, dtype=prob.vdt, device="cuda")
    opts = prob.relax_opts(s=s, T=args.warmup + args.steps, fixed_iters=args.cg_iters, seed=1)
    for t in range(args.warmup):
        prob.relax_step(opts, t, b, z, stats=False)
    torch.cuda.synchronize()

    # ---------------- timed region (device events on the library's stream = torch's current)
    lib.firal_profile(1)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = lib.firal_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(args.steps):
        prob.relax_step(opts, args.warmup + t, b, z, stats=False)
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    launches = lib.firal_launch_count() - launches0
    clk = clocks.stop()
    ms_ev = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms_ev, world)
    nk = _lib.FiralStepStats  # noqa: F841
    ncls = 13
    ms_k = (ctypes_arr := __import__("ctypes").c_double * ncls)()
    calls_k = (__import__("ctypes").c_int64 * ncls)()
    lib.firal_profile_read(ms_k, calls_k, ncls)
    lib.firal_profile(0)
    kernels = {lib.firal_profile_name(i).decode(): {"ms_per_step": ms_k[i] / args.steps,
                                                   "groups_per_step": calls_k[i] / args.steps}
               for i in range(ncls) if calls_k[i] > 0}
    # replicas: every rank ran its own problem; sharded: the ranks ran one problem together
    value = (1 if shard else world) * args.steps / (ms_max / 1000.0)

    # ---------------- roofline of the dominant kernel class
    pk, pk_src = peaks()
    top = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    n_all = n_loc + p.Xo.shape[0]          # rows this rank's kernels run over
    cfg_loc = dict(cfg, n=n_loc)
    fl = algorithmic_flops(top, cfg_loc, n_all, s)
    roof = None
    if fl is not None:
        per_launch_ms = kernels[top]["ms_per_step"] / kernels[top]["groups_per_step"]
        achieved = fl / (per_launch_ms / 1000.0) / 1e12
        tensor = args.precision.startswith("mixed") and top in ("apply_alpha", "apply_dterm",
                                                                 "syrk_blocks", "quad_forms")
        peak = pk["bf16_tflops_sustained"] if tensor else FP32_ALU_PEAK_TFLOPS
        n_pad = (n_all + 127) // 128 * 128
        # executed tensor flops: the hi/lo direction doubles the alpha-GEMM's MMA work
        execd = achieved * (2.0 if (top == "apply_alpha" and args.precision == "mixed") else 1.0)
        roof = {"kernel": top, "bound": "tensor" if tensor else "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": dram_traffic(top, n_pad, args.precision) if tensor else None,
                "executed_tflops": execd,
                "peak_source": (("measured bf16 sustained (of measured)" if pk_src == "measured"
                                 else "fallback bf16 sustained (of fallback)") if tensor else
                                "derived FP32 FMA peak: 152 SMs x 128 lanes x 2 x 2.07 GHz")}
        if tensor:
            roof["frac_of_burst"] = achieved / pk["bf16_tflops"]
            # per-clock efficiency: the sustained peak was measured at a lower SM clock than
            # this run's, so compare work per SM cycle (time x median SM MHz)
            peak_mhz = (pk.get("clocks_under_load") or {}).get("sm_mhz_median")
            if peak_mhz and clk and clk.get("sm_mhz"):
                roof["frac_clock_normalized"] = (achieved / clk["sm_mhz"]) / (peak / peak_mhz)
                roof["clock_note"] = (f"sustained peak at a median {peak_mhz:.0f} MHz, this run "
                                      f"at {clk['sm_mhz']:.0f} MHz")
    # every tensor-core class against the same peak: algorithmic flops per MD iteration (one
    # unit per Hessian apply for the two apply GEMMs; one block-sum pass and one gradient per
    # iteration) over the class's time per iteration, with DRAM traffic per launch where
    # captured
    if args.precision.startswith("mixed"):
        n_pad = (n_all + 127) // 128 * 128
        for k in ("apply_alpha", "apply_dterm", "syrk_blocks", "quad_forms"):
            kk = kernels.get(k)
            f_k = algorithmic_flops(k, cfg_loc, n_all, s)
            if not kk or f_k is None or kk["ms_per_step"] <= 0:
                continue
            units = kk["groups_per_step"] if k.startswith("apply_") else 1.0
            a_k = f_k * units / (kk["ms_per_step"] / 1000.0) / 1e12
            kk.update({"tflops_algorithmic": a_k,
                       "frac_of_bf16_sustained": a_k / pk["bf16_tflops_sustained"],
                       "traffic_bytes_per_launch": dram_traffic(k, n_pad, args.precision)})
    # the Hessian apply as a whole (alpha + D + combine), the operation the metric counts
    apply_ms = sum(kernels.get(k, {}).get("ms_per_step", 0.0)
                   for k in ("apply_alpha", "apply_dterm", "apply_combine"))
    applies_per_step = 2 * args.cg_iters + 1
    apply_tflops = (4.0 * n_all * c * d * s * applies_per_step) / (apply_ms / 1000.0) / 1e12 \
        if apply_ms > 0 else None

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "strong" if shard else "weak",
            "vs_baseline": None,
            "dtype": {"mixed": "bf16", "mixed_fast": "bf16", "fp32": "f32",
                      "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": config_of(cfg, args),
            "setup": {"precision": args.precision,
                      "parallelism": (f"rows{world} (pool rows sharded, allreduce per apply)"
                                      if shard else "replicas" if world > 1 else "single"),
                      "tuning": ({k: tuning[k] for k in ("dterm_splits", "bsum_splits",
                                                         "sm_budget", "ms", "default_ms",
                                                         "candidates")}
                                 if tuning else None),
                      "tuning_used": prob.get_tuning()},
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk,
            "kernels": kernels,
            "hessian_apply": {"tflops_algorithmic": apply_tflops,
                              "frac_of_bf16_sustained": (apply_tflops / pk["bf16_tflops_sustained"]
                                                         if apply_tflops else None)}}

    # ---------------- end to end through the public API with host (pinned) buffers
    if not args.no_e2e:
        zh = torch.full((n_loc,), b / n, dtype=prob.vdt).pin_memory()
        k_e2e = max(1, min(args.steps, 10))   # every call timed and listed in ms_per_step

        def e2e_step(t):
            if not shard:
                zout, _ = api.relax(Xh, hh, Xoh, hoh, p.lam, b, s=s, T=1,
                                    fixed_iters=args.cg_iters, seed=1 + t,
                                    precision=args.precision, z0=zh, handle=H)
                zh.copy_(zout)
                return
            # row-sharded: this rank's slice to the device, a problem joined to the group, one
            # MD iteration, its z slice back
            tX, th = Xh.to("cuda", non_blocking=True), hh.to("cuda", non_blocking=True)
            tXo, tho = Xoh.to("cuda", non_blocking=True), hoh.to("cuda", non_blocking=True)
            pr = api.Problem(H, tX, th, tXo, tho, p.lam, precision=args.precision)
            pr.set_comm(rank, world, api.torch_allreduce())
            zd = zh.to("cuda", non_blocking=True)
            pr.relax_step(pr.relax_opts(s=s, T=1, fixed_iters=args.cg_iters, seed=1 + t), 0, b,
                          zd, stats=False)
            zh.copy_(zd.cpu())
            pr.close()
        e2e_step(0)                                  # untimed warm-up call
        barrier(world)
        t0 = time.perf_counter()
        per_step = []
        for t in range(k_e2e):
            ts = time.perf_counter()
            e2e_step(1 + t)
            per_step.append(1000.0 * (time.perf_counter() - ts))
        dt = max_over_ranks(time.perf_counter() - t0, world)
        bi = sum(t.numel() * t.element_size() for t in (Xh, hh, Xoh, hoh, zh))
        line["e2e"] = {"value": (1 if shard else world) * k_e2e / dt, "unit": UNIT,
                       "h2d_bytes_per_step": bi,
                       "d2h_bytes_per_step": zh.numel() * zh.element_size(), "steps": k_e2e,
                       "warmup": 1, "ms_per_step": per_step,
                       "note": "each step is one api.relax(T=1) call on pinned host tensors: "
                               "H2D copies, problem preparation, one MD iteration, D2H of z"}
        # diagnostic only (not the e2e value): the same call split into its H2D copies, the
        # library call on the device copies and the D2H of z, with the collector's counts
        try:
            if shard:
                raise RuntimeError("not measured on a row-sharded run")
            import gc
            parts = []
            for t in range(3):
                gc0 = gc.get_count()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                dX, dh = Xh.to("cuda", non_blocking=True), hh.to("cuda", non_blocking=True)
                dXo, dho = Xoh.to("cuda", non_blocking=True), hoh.to("cuda", non_blocking=True)
                dz0 = zh.to("cuda", non_blocking=True)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                zd, _ = api.relax(dX, dh, dXo, dho, p.lam, b, s=s, T=1, fixed_iters=args.cg_iters,
                                  seed=100 + t, precision=args.precision, z0=dz0, handle=H)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                zh.copy_(zd.cpu())
                t3 = time.perf_counter()
                del dX, dh, dXo, dho, dz0, zd
                parts.append({"h2d_ms": 1e3 * (t1 - t0), "call_ms": 1e3 * (t2 - t1),
                              "d2h_ms": 1e3 * (t3 - t2), "gc_counts": list(gc0)})
            line["e2e_breakdown"] = parts
        except Exception as exc:
            line["e2e_breakdown"] = {"error": str(exc)[:300]}

    if rank == 0 and world == 1:
        # ---------------- the paper's timing setting (m = 50) and the tolerance mode
        if not args.no_variants:
            try:
                line["cg_variants"] = cg_variants(prob, s, b, n)
            except Exception as exc:
                line["cg_variants"] = {"error": str(exc)[:300]}
        # ---------------- plain FP32 form on the same GPU and its agreement with the mixed
        # forms (the timed precision, and the hi/lo-direction variant when it is not timed)
        if not args.no_fp32 and args.precision.startswith("mixed"):
            del prob
            torch.cuda.empty_cache()
            p32 = api.Problem(H, X, h, Xo, ho, p.lam, precision="fp32")
            z32 = torch.full((n,), b / n, dtype=torch.float32, device="cuda")
            o = p32.relax_opts(s=s, T=8, fixed_iters=args.cg_iters, seed=1)
            st32 = p32.relax_step(o, 0, b, z32)
            precs = [args.precision] + (["mixed"] if args.precision == "mixed_fast" and
                                        not args.no_variants else [])
            agree = {}
            for prec in precs:
                pm = api.Problem(H, X, h, Xo, ho, p.lam, precision=prec)
                zm = torch.full((n,), b / n, dtype=torch.float32, device="cuda")
                stm = pm.relax_step(o, 0, b, zm)
                rec = {"fhat_rel_diff_vs_fp32": abs(stm["fhat"] - st32["fhat"]) / abs(st32["fhat"]),
                       "z_rel_diff_vs_fp32": float((zm.double() - z32.double()).norm() /
                                                   z32.double().norm())}
                if prec != args.precision:
                    # time the variant: 3 MD iterations between events
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for t in range(1, 4):
                        pm.relax_step(o, t, b, zm, stats=False)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / 3
                    rec.update({"value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms,
                                "note": "CG direction as bf16 hi + lo in the alpha-GEMM "
                                        "(twice its tensor work)"})
                agree[prec] = rec
                pm.close()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p32.relax_step(o, 1, b, z32, stats=False)
            torch.cuda.synchronize()
            dt32 = time.perf_counter() - t0
            line["fp32"] = {"value": 1.0 / dt32, "unit": UNIT, "steps": 1, "warmup": 1,
                            "fhat_rel_diff_mixed_vs_fp32": agree[args.precision]["fhat_rel_diff_vs_fp32"],
                            "z_rel_diff_mixed_vs_fp32": agree[args.precision]["z_rel_diff_vs_fp32"],
                            "compared": "one MD iteration from the uniform z, same probes",
                            "speedup_mixed_over_fp32": value / world * dt32}
            if "mixed" in agree and args.precision != "mixed":
                line["mixed_hilo"] = agree["mixed"]
            del p32
        # ---------------- Round (Algorithm 3) on the full-pipeline workload
        if not args.no_round:
            try:
                line["round"] = round_measure(args, H)
            except Exception as exc:   # reported in the line; the Relax metric stands
                line["round"] = {"error": str(exc)[:300]}
        if not args.no_batched:
            try:
                line["batched"] = batched_measure(args, H)
            except Exception as exc:
                line["batched"] = {"error": str(exc)[:300]}
        if not args.no_exact:
            try:
                line["exact_vs_approx"] = exact_measure(args, H)
            except Exception as exc:
                line["exact_vs_approx"] = {"error": str(exc)[:300]}
        if not args.no_al:
            try:
                line["active_learning"] = al_measure(args, H)
            except Exception as exc:
                line["active_learning"] = {"error": str(exc)[:300]}
        # ---------------- CPU oracle baseline
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(cfg, args.cg_iters, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_only(args):
    """One sub-measurement on its own (the launch lists under profiles/ come from these)."""
    import torch

    from paper_2409_07392_gb300 import api, build
    build.build()
    torch.cuda.set_device(0)
    H = api.Handle()
    fn = {"round": round_measure, "batched": batched_measure, "exact": exact_measure,
          "al": al_measure}[args.only]
    print(json.dumps({"only": args.only, "record": fn(args, H)}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.only:
        run_only(a)
    else:
        run_ours(a)
