"""TNVAN (arXiv 2504.12037) hot path for one GB300 GPU (sm_103a).

  workloads  seeded synthetic inputs (graphs, couplings, width sets, initial
             network parameters)
  tnvan      ctypes binding of the C-ABI library libtnvan.so (include/tnvan.h)
  model      multi-instance training / estimation driver built on the binding
  build      in-tree nvcc build of libtnvan.so
"""
__all__ = ["workloads", "tnvan", "model", "build"]
