"""GB300 (sm_103a) direction-reuse path tracer after "Generate Coherent Rays Directly"
(Liu et al., arXiv 2310.07182).

The compute path is the C-ABI library ``libcr.so`` (include/cr.h), hand-written CUDA for
sm_103a; ``binding`` is its thin ctypes binding and ``scenes`` generates the seeded
synthetic inputs.  Importing this package loads nothing; ``binding.lib()`` loads the
library and raises if it has not been built.
"""
__all__ = ["binding", "scenes", "build"]
