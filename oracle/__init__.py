"""FP64 CPU oracle for Approx-FIRAL (Chen, Wen, Biros, SC24) -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously correct statement of what the
GPU path computes.  It is written from the paper (equations, lemmas and
algorithms cited in each function) in float64 numpy, with no blocking,
fusion or reordering beyond what those statements give.  It shares no code
with the CUDA library and imports nothing from it.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline leg and its ``--impl reference`` arm) may import this package; the
product path never does.

Modules
  probes  -- the counter-based Rademacher probes (SplitMix64).
  exact   -- Exact-FIRAL (Algorithm 1): dense dc x dc Hessians on tiny inputs.
  approx  -- Approx-FIRAL (Algorithms 2 and 3): matrix-free Relax and
             block-diagonal Round.
  al      -- the active-learning outer loop of Section 5: classifier refit
             (ridge multinomial logistic regression by Newton) and the rounds.

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, an invariant, an
independent method or brute force; no function is "parity unpinned".
"""
