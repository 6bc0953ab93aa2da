"""GB300-native HEOM-2DVS hot path (arXiv 2601.20550).

The compute runs in ``libheom2dvs.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in include/heom2dvs.h).  ``paper_2601_20550_gb300.heom`` is the thin
ctypes binding with the same entry-point names; it raises if the library is
missing - there is no CPU fallback.  ``shard`` splits the t1 rows of a 2D scan
over torch.distributed ranks; ``autograd`` wraps the misfit gradient
(heom_response_2d_grad) as a torch.autograd.Function.
"""
__all__ = ["heom", "shard", "autograd"]
