"""Writes ``imagenet_classes_n20k.npz``: FP64 oracle values for the parity test of the
ImageNet class count (d = 64, c = 1000, s = 16) on a reduced pool.

It calls only ``oracle/`` (and the seeded input generator), never the CUDA path.  The
oracle needs several minutes for this size, more than a GPU test should spend, so its
outputs are stored:

* ``fhat`` and ``z`` of two mirror-descent iterations of Algorithm 2 with the paper's
  gradient estimator (eq. 11), 10 PCG iterations per solve, probe seed 1;
* ``g_autograd``: the exact derivative of the same-probe objective estimate at the uniform
  start, ``-(1/s) sum_j u_j^T H_i y_j`` with ``U = Sigma^{-1} V``, ``Y = Sigma^{-1} H_p V``
  (10 PCG iterations per column), and its ``fhat``;
* a fingerprint of the inputs (float64 sums), which the test compares with the inputs it
  regenerates from the same seed.

Run from the repository root:  python tests/golden/make_imagenet_classes.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import approx  # noqa: E402
from paper_2409_07392_gb300.synth import make_problem  # noqa: E402

N, D, C, S, T, ITERS = 20_000, 64, 1000, 16, 2, 10
BUDGET = 20.0          # z_i = 1e-3 at the start, as budget 1000 over 10^6 points
DATA_SEED, PROBE_SEED = 0, 1
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "imagenet_classes_n20k.npz")


def problem():
    return make_problem(N, D, C, seed=DATA_SEED, x_dtype="bf16", h_dtype="float32", m_o=C)


def fingerprint(p):
    return np.array([p.X.astype(np.float64).sum(), p.h.astype(np.float64).sum(),
                     p.Xo.astype(np.float64).sum(), p.ho.astype(np.float64).sum(),
                     (p.h.astype(np.float64) ** 2).sum()])


def main():
    p = problem()
    z, info = approx.relax(p, BUDGET, s=S, T=T, seed=PROBE_SEED, fixed_iters=ITERS)
    _, ainfo = approx.relax(p, BUDGET, s=S, T=1, seed=PROBE_SEED, fixed_iters=ITERS,
                            estimator="autograd", record=True)
    np.savez_compressed(OUT, fhat=np.array(info["fhat"]), z=z, g_autograd=ainfo["g"][0],
                        fhat_autograd=np.array(ainfo["fhat"]), fingerprint=fingerprint(p),
                        shape=np.array([N, D, C, S, T, ITERS]), budget=BUDGET,
                        seeds=np.array([DATA_SEED, PROBE_SEED]))
    print("wrote", OUT, "fhat", info["fhat"], "autograd fhat", ainfo["fhat"])


if __name__ == "__main__":
    main()
