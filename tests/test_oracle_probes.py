"""Pins of the counter-based Rademacher probes -- no GPU."""
import numpy as np

from oracle import probes

MASK = (1 << 64) - 1


def test_splitmix64_known_answers():
    # SplitMix64 seeded with 0: its first two outputs (published reference values).
    assert int(probes.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    assert int(probes.splitmix64(np.uint64(0x9E3779B97F4A7C15))) == 0x6E789E6AA1B965F4


def _scalar(seed, t, s, D, j, q):
    def sm(x):
        z = (x + 0x9E3779B97F4A7C15) & MASK
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)
    ctr = ((t * s + j) * D + q) & MASK
    return 1.0 if (sm(seed ^ sm(ctr)) >> 63) == 0 else -1.0


def test_vectorised_matches_bigint_counter_rule():
    seed, t, s, D = 12345, 7, 5, 37
    V = probes.rademacher(seed, t, s, D)
    assert V.shape == (D, s)
    for j in range(s):
        for q in (0, 1, 17, D - 1):
            assert V[q, j] == _scalar(seed, t, s, D, j, q)


def test_probes_balanced_and_fresh():
    V = probes.rademacher(1, 0, 16, 64000)
    assert set(np.unique(V)) == {-1.0, 1.0}
    # mean of 1.024e6 fair signs: |mean| < 4 / sqrt(N)
    assert abs(V.mean()) < 4 / np.sqrt(V.size)
    V2 = probes.rademacher(1, 1, 16, 64000)
    assert abs(np.mean(V * V2)) < 4 / np.sqrt(V.size)      # iterations independent
    assert abs(np.mean(V[:, 0] * V[:, 1])) < 4 / np.sqrt(64000)
