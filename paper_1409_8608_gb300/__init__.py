"""tc: a tensor-contraction engine for GB300 (sm_103a).

Every algorithm is a loop nest around one BLAS-level kernel (dot, axpy,
gemv, ger, gemm) as in Peise, Fabregat-Traver and Bientinesi, "On the
Performance Prediction of BLAS-based Tensor Contractions" (Section 2), plus
a fused GETT kernel; a planner ranks them by cache-context micro-benchmarks
(Section 3).  The compute runs in hand-written CUDA behind a C ABI
(include/tc.h); ``paper_1409_8608_gb300.tc`` is the thin ctypes binding.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
