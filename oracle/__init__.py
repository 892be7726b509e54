"""CPU oracle for the blocked randUTV factorization (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library.
"""
from .oracle import (  # noqa: F401
    build,
    gaussian,
    gemm,
    householder_qr,
    jacobi_svd,
    larft,
    num_threads,
    philox4x64_10,
    randutv,
    randutv_qrfirst,
)
