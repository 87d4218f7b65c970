"""GB300 matrix-free high-order Poisson operator and multigrid solver
(Kronbichler & Wall, arXiv:1611.03029, Sec. 2-4) behind the C ABI of
include/mfpoisson.h.

``build.build()`` compiles the CUDA library in-tree; ``mfpoisson`` is the
ctypes binding (imported lazily, it raises when the library is missing).
"""
__all__ = ["build", "mfpoisson", "synthetic"]
