"""Rademacher probe vectors for the Hutchinson estimator (eq. 11, Algorithm 2).

The paper draws ``s`` fresh Rademacher vectors of length ``d~ = d c`` every
mirror-descent iteration but does not say how.  This package fixes a
counter-based rule so the oracle and the GPU produce the same probes without
sharing code:

    v[t][j][q] = +1  if the top bit of  splitmix64(seed XOR splitmix64((t*s + j)*d~ + q))  is 0
               = -1  otherwise,

where ``splitmix64(x)`` is the output of SplitMix64 (Steele, Lea, Flood,
OOPSLA 2014) whose state before the call is ``x``: add the golden gamma
0x9E3779B97F4A7C15, then apply the variant-13 mixing function.  Index
``q = k d + e`` follows ``vec`` stacking the columns of the d x c matrix.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output for state ``x`` (uint64 array or scalar), wrapping mod 2^64."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def rademacher(seed: int, t: int, s: int, dtil: int) -> np.ndarray:
    """Probe block of MD iteration ``t``: float64 array (dtil, s) of +-1, column j = v_j."""
    j = np.arange(s, dtype=np.uint64)[None, :]
    q = np.arange(dtil, dtype=np.uint64)[:, None]
    with np.errstate(over="ignore"):
        ctr = (np.uint64(t) * np.uint64(s) + j) * np.uint64(dtil) + q
        bits = splitmix64(np.uint64(seed) ^ splitmix64(ctr))
    top = (bits >> np.uint64(63)).astype(np.int64)
    return np.where(top == 0, 1.0, -1.0)
