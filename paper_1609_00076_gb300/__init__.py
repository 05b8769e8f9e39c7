"""GB300-native double-precision GEMM (C := alpha*op(A)*op(B) + beta*C).

The compute path is the CUDA library libgbdgemm.so (include/gbdgemm.h); this
package holds its thin ctypes binding (``gbdgemm``), its build script
(``build``), the seeded synthetic inputs (``synth``) and the request-serving
loop (``serving``).  Importing the package does not load the library; the first
call does, and fails loudly if it cannot.
"""

__all__ = ["gbdgemm", "synth", "build"]
