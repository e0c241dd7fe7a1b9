"""GB300 (sm_103a) implementation of the Approx-FIRAL hot path (Chen, Wen, Biros, SC24).

Submodules:
  build     -- compiles the CUDA library in-tree (``_build/libfiral.so``)
  api       -- Python binding of the C-ABI in ``include/firal.h`` (torch tensors in and out)
  autograd  -- ``FiralObjective``: f^(z) as a torch.autograd.Function
  synth     -- seeded Gaussian-mixture inputs shaped like the paper's workloads

Importing the package does not load the CUDA library; ``api`` does, on first use.
"""

__all__ = ["build", "api", "autograd", "synth"]
