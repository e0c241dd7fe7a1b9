"""Seeded synthetic inputs shaped like the workloads of Approx-FIRAL's experiments.

This module holds only the input model: Gaussian-mixture embeddings and the
class probabilities of a fixed multinomial logistic-regression classifier
(eq. 1, full c-class softmax).  It contains none of the method's arithmetic
(no Hessian, no solve, no gradient), so both the CUDA path and the FP64 CPU
oracle take their inputs from here.

Recipe (stands in for the MNIST / CIFAR-10 / ImageNet features of Section 5,
which are not available):

* mixture means ``mu_k ~ N(0, 4 I_d)``, one component per class;
* points ``x = mu_k + eps`` with ``eps ~ N(0, I_d)``, or, for the anisotropic
  variant, ``eps ~ N(0, Q_k diag(l) Q_k^T)`` with ``l`` log-uniform in
  ``[1e-2, 1]`` and ``Q_k`` Haar-orthogonal (QR of a Gaussian matrix);
* rows L2-normalised;
* component priors uniform, or Zipf ``p_k ~ k^-a``;
* classifier weights ``W ~ N(0, 1)^{c x d}``; ``h = softmax(W x)`` computed in
  float64 from the stored (possibly bf16-rounded) ``x`` and stored in the
  requested dtype;
* labelled set ``X_o``: one fresh draw per mixture component;
* ``lambda = 1e-3`` regularises ``H_o`` (the softmax Hessian has the null
  space ``1_c (x) v``).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["Problem", "make_problem", "bf16_round", "CONFIGS", "config_problem",
           "batched_problems"]


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returns float32."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@dataclasses.dataclass
class Problem:
    """One active-learning instance: pool (X, h), labelled set (Xo, ho), lambda."""
    X: np.ndarray        # (n, d) pool embeddings (float32 / float64; bf16-representable if x_bf16)
    h: np.ndarray        # (n, c) class probabilities of the pool points
    Xo: np.ndarray       # (m, d) labelled embeddings
    ho: np.ndarray       # (m, c) class probabilities of the labelled points
    lam: float           # ridge added to H_o
    x_bf16: bool = False  # True when X / Xo hold bf16-representable values (stored as bf16 on device)
    labels: np.ndarray | None = None  # (n,) mixture component of each pool point

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def d(self):
        return self.X.shape[1]

    @property
    def c(self):
        return self.h.shape[1]


def _softmax_rows(logits: np.ndarray) -> np.ndarray:
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    return e / e.sum(axis=1, keepdims=True)


def make_problem(n: int, d: int, c: int, *, seed: int = 0, m_o: int | None = None,
                 x_dtype: str = "float32", h_dtype: str = "float32",
                 anisotropic: bool = False, zipf: float | None = None,
                 lam: float = 1e-3, w_scale: float = 1.0, mean_scale: float = 2.0,
                 chunk: int = 1 << 16) -> Problem:
    """Draw one seeded Gaussian-mixture problem.

    ``x_dtype`` is "float64", "float32" or "bf16" (float32 array holding
    bf16-representable values).  ``w_scale`` multiplies the classifier weights
    (large values give confident, near one-hot ``h``).  ``chunk`` bounds the
    memory of the softmax pass; it does not change any value.
    """
    rng = np.random.default_rng(seed)
    k_comp = c
    means = mean_scale * rng.standard_normal((k_comp, d))
    if zipf is None:
        prior = np.full(k_comp, 1.0 / k_comp)
    else:
        prior = np.arange(1, k_comp + 1, dtype=np.float64) ** (-zipf)
        prior /= prior.sum()
    W = w_scale * rng.standard_normal((c, d))
    if anisotropic:
        Qs = np.empty((k_comp, d, d))
        ls = np.empty((k_comp, d))
        for k in range(k_comp):
            q, r = np.linalg.qr(rng.standard_normal((d, d)))
            Qs[k] = q * np.sign(np.diag(r))[None, :]
            ls[k] = np.exp(rng.uniform(np.log(1e-2), np.log(1.0), size=d))

    def draw(count, comp):
        eps = rng.standard_normal((count, d))
        if anisotropic:
            out = np.empty((count, d))
            for k in np.unique(comp):
                sel = comp == k
                out[sel] = means[k] + (eps[sel] * np.sqrt(ls[k])[None, :]) @ Qs[k].T
        else:
            out = means[comp] + eps
        out /= np.linalg.norm(out, axis=1, keepdims=True)
        return out

    comp = rng.choice(k_comp, size=n, p=prior)
    X64 = draw(n, comp)
    m = k_comp if m_o is None else m_o
    comp_o = np.arange(m) % k_comp
    Xo64 = draw(m, comp_o)

    def store_x(a):
        if x_dtype == "float64":
            return a
        if x_dtype == "float32":
            return a.astype(np.float32)
        if x_dtype == "bf16":
            return bf16_round(a.astype(np.float32))
        raise ValueError(x_dtype)

    X = store_x(X64)
    Xo = store_x(Xo64)
    hdt = np.float64 if h_dtype == "float64" else np.float32

    def probs(Xs):
        out = np.empty((Xs.shape[0], c), dtype=hdt)
        for a in range(0, Xs.shape[0], chunk):
            xb = Xs[a:a + chunk].astype(np.float64)
            out[a:a + chunk] = _softmax_rows(xb @ W.T)
        return out

    return Problem(X=X, h=probs(X), Xo=Xo, ho=probs(Xo), lam=lam,
                   x_bf16=(x_dtype == "bf16"), labels=comp)


# The five workload shapes the benchmarks and parity tests use.  Fields: pool
# size n, feature dimension d, classes c, probes s, mirror-descent iterations T,
# budget b and the storage dtypes.
CONFIGS = {
    "fp64_small": dict(n=3000, d=20, c=10, s=10, T=20, b=10, x_dtype="float64",
                       h_dtype="float64"),
    "cifar_like": dict(n=50_000, d=50, c=10, s=20, T=50, b=100, x_dtype="float32",
                       h_dtype="float32"),
    "imagenet_like": dict(n=1_000_000, d=64, c=1000, s=16, T=30, b=1000, x_dtype="bf16",
                          h_dtype="float32"),
    "batched_uneven": dict(nproblems=64, s=8),
    "full_pipeline": dict(n=1_000_000, d=128, c=100, s=16, T=30, b=2000, x_dtype="bf16",
                          h_dtype="float32", anisotropic=True, zipf=1.1),
}


def config_problem(name: str, *, seed: int = 0, n: int | None = None) -> Problem:
    """The seeded problem of one named workload (``n`` overrides the pool size)."""
    cfg = CONFIGS[name]
    return make_problem(n if n is not None else cfg["n"], cfg["d"], cfg["c"], seed=seed,
                        x_dtype=cfg["x_dtype"], h_dtype=cfg["h_dtype"],
                        anisotropic=cfg.get("anisotropic", False), zipf=cfg.get("zipf"))


def batched_problems(nproblems: int = 64, *, seed: int = 0, n_range=(2000, 40000),
                     ds=(16, 32, 48, 64), cs=(5, 10, 20), b_range=(10, 200)):
    """Shapes (n, d, c, b) of the uneven batched workload, drawn with ``seed``."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nproblems):
        out.append(dict(n=int(rng.integers(n_range[0], n_range[1] + 1)),
                        d=int(rng.choice(ds)), c=int(rng.choice(cs)),
                        b=int(rng.integers(b_range[0], b_range[1] + 1))))
    return out
