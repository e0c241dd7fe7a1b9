"""Autotuner of the tensor-core path's launch parameters.

The tunable parameters (``firal_tuning`` in the C-ABI) are the point-range split counts of the
Hessian apply's D-GEMM and of the block sums -- the K extent of each CTA's tile -- and the SM
budget of a problem's grids.  The built-in rule picks them from the shape; the autotuner times
candidates around that choice on the real MD iteration (CUDA events on the library's stream,
fixed CG iterations) and keeps the fastest.  Results persist in a JSON cache keyed by
(precision, n rounded to a power of two, d, c, s); ``apply_cached`` reuses them for later
problems of the same key.  For the batched workload the handle-level default (which the pooled
problems of ``firal_batched_relax`` inherit) is tuned the same way.

The D-GEMM split count never drops below the accumulation-chain bound (the library raises it),
so no candidate changes the numerics beyond the usual reordering of sums.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

FIELDS = ("dterm_splits", "bsum_splits", "sm_budget")


def shape_key(precision: str, n: int, d: int, c: int, s: int) -> str:
    """Cache key: n rounded to the nearest power of two."""
    nb = int(round(math.log2(max(int(n), 1))))
    return f"{precision}:n2^{nb}:d{int(d)}:c{int(c)}:s{int(s)}"


def default_cache_path() -> str:
    env = os.environ.get("FIRAL_TUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")


class TuneCache:
    """A JSON file of ``{key: {dterm_splits, bsum_splits, sm_budget, ms, default_ms}}``."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self.data = {}
        try:
            with open(self.path) as f:
                loaded = json.load(f)
            if isinstance(loaded, dict):
                self.data = loaded
        except (OSError, ValueError):
            self.data = {}

    def get(self, key: str):
        v = self.data.get(key)
        if isinstance(v, dict) and all(isinstance(v.get(k), int) and v[k] >= 0 for k in FIELDS):
            return {k: v[k] for k in FIELDS}
        return None

    def put(self, key: str, value: dict) -> None:
        self.data[key] = dict(value)
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=os.path.dirname(self.path) or ".", suffix=".tmp")
        with os.fdopen(fd, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def candidates(used: dict, factors=(0.5, 0.75, 1.0, 1.5, 2.0), bfactors=(0.5, 1.0, 2.0)):
    """Split counts around the rule's choice (``used``: what the default launch used)."""
    d0 = max(1, int(used.get("dterm_splits", 0) or 1))
    b0 = max(1, int(used.get("bsum_splits", 0) or 1))
    ds = sorted({max(1, int(round(d0 * f))) for f in factors})
    bs = sorted({max(1, int(round(b0 * f))) for f in bfactors})
    return [dict(dterm_splits=x, bsum_splits=y, sm_budget=0) for x in ds for y in bs]


def pick_best(timings: list[tuple[dict, float]]):
    """The fastest (tuning, ms); ties keep the earlier (the rule's choice comes first)."""
    best = None
    for cand, ms in timings:
        if best is None or ms < best[1]:
            best = (cand, ms)
    return best


def _time_steps(prob, opts, budget, z0, reps):
    import torch
    z = z0.clone()
    prob.relax_step(opts, 0, budget, z, stats=False)           # warm-up at this tuning
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(1, 1 + reps):
        prob.relax_step(opts, t, budget, z, stats=False)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_problem(prob, s: int, *, cg_iters: int = 10, budget: float | None = None,
                 reps: int = 2, cache: TuneCache | None = None, seed: int = 1) -> dict:
    """Time the rule's tuning and the candidates around it on MD iterations of ``prob``; set
    the fastest on the problem, store it in the cache, and return the record."""
    import torch
    cache = cache or TuneCache()
    b = float(budget) if budget is not None else max(1.0, prob.n / 1000.0)
    opts = prob.relax_opts(s=s, T=1 + reps, fixed_iters=cg_iters, seed=seed)
    z0 = torch.full((prob.n,), b / prob.n, dtype=prob.vdt, device=prob.device)
    prob.set_tuning(0, 0, 0)
    default_ms = _time_steps(prob, opts, b, z0, reps)
    used = prob.get_tuning()
    timings = [(dict(dterm_splits=0, bsum_splits=0, sm_budget=0), default_ms)]
    for cand in candidates(used):
        prob.set_tuning(**cand)
        timings.append((cand, _time_steps(prob, opts, b, z0, reps)))
    best, ms = pick_best(timings)
    prob.set_tuning(**best)
    rec = dict(best, ms=ms, default_ms=default_ms, default_used=used,
               candidates=len(timings))
    cache.put(shape_key(prob.precision, prob.n, prob.d, prob.c, s), rec)
    return rec


def apply_cached(prob, s: int, cache: TuneCache | None = None) -> bool:
    """Set the cached tuning of the problem's key, if any; True when one was applied."""
    cache = cache or TuneCache()
    t = cache.get(shape_key(prob.precision, prob.n, prob.d, prob.c, s))
    if t is None:
        return False
    prob.set_tuning(**t)
    return True


def tune_handle(handle, run, budgets=(0, 114, 76, 38), key: str | None = None,
                cache: TuneCache | None = None) -> dict:
    """Tune the handle-level SM budget for a workload run by ``run()`` (which must create its
    problems on ``handle`` and return its time in ms, e.g. one batched MD iteration)."""
    timings = []
    for sb in budgets:
        handle.set_default_tuning(0, 0, sb)
        timings.append((dict(dterm_splits=0, bsum_splits=0, sm_budget=sb), float(run())))
    best, ms = pick_best(timings)
    handle.set_default_tuning(**best)
    rec = dict(best, ms=ms, default_ms=timings[0][1], candidates=len(timings))
    if key is not None:
        (cache or TuneCache()).put(key, rec)
    return rec
