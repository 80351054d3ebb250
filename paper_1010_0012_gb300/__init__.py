"""bpgrid: exact O(mM) belief propagation with truncated (robust) pairwise
potentials on 4-connected grids, for GB300 (sm_103a).

  workload  seeded synthetic random-dot stereo inputs (no BP arithmetic)
  build     compiles the CUDA library in-tree (nvcc, sm_103a)
  bp        ctypes binding of the C ABI in include/bp.h (imports fail loudly
            when the library is not built)
  autograd  torch.autograd.Function around the log-domain forward / adjoint
"""

__all__ = ["workload", "build", "bp", "autograd"]
