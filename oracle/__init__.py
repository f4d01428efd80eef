"""CPU oracle for the mixed-precision recursive Gram-Schmidt QR least-squares path.

TEST INFRASTRUCTURE ONLY. Nothing in the GPU library imports this package;
only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it. It shares no code with the CUDA path.

Contents
--------
direct   : plain FP64 Householder QR least squares (Alg. 1), in C (householder.c)
lowprec  : the rounding operations the low-precision GEMMs apply (FP16/BF16 RN-even,
           power-of-two column scales)
rgsqrf   : recursive Gram-Schmidt QR (Alg. 2) with the CAQR/TSQR panel (Eq. caqr)
           and CGS2 / MGS (Alg. 4) leaves, in FP64 with the GEMM inputs rounded
krylov   : R-preconditioned CGLS (Alg. 5, with its typos corrected) and LSQR
metrics  : QR accuracy (Sec. 3.2.1), least-squares residual and backward errors
adjoint  : closed-form gradient of x*(A, b) for the differentiable solve

Parity status: every function here is pinned by tests in tests/test_oracle_*.py
against closed forms, exact rational arithmetic, invariants or library routines.
"""
