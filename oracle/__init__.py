"""FP64 CPU oracle for the TLR Cholesky / LDL^T method (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only `tests/`, `__graft_entry__.smoke()`
and the CPU-baseline leg of `bench.py` may import it.  It shares no code with
the CUDA path (`paper_2108_11932_gb300`), and the CUDA path never calls it.

Every function follows a passage of the paper (Boukaram, Zampini, Turkiyyah,
Keyes, "H2OPUS-TLR: High Performance Tile Low Rank Symmetric Factorizations
using Adaptive Randomized Approximation", arXiv 2108.11932), cited by section,
equation, algorithm or table.  It is written for clarity, not speed: plain
numpy loops in float64, with library primitives (matmul, SVD, Cholesky) used
as single steps only.

Modules
  kdtree    KD-tree point ordering (Section 6).
  kernel    exponential covariance tiles (Section 6).
  philox    Philox4x32-10 counter-based generator + Box-Muller Gaussians (the
            ARA random blocks, Algorithm 1 / Algorithm 5 batchRandn).
  dense     dense Cholesky / unpivoted LDL^T and triangular solves (Section 3.2,
            Section 5.3).
  compress  truncated-SVD compression and ARA (Algorithm 1) with BCGS2 +
            Cholesky-QR orthogonalization.
  tlr       left-looking TLR Cholesky (Algorithm 6), its tile-pivoted form
            (Algorithm 9) and LDL^T (Algorithm 10), TLR triangular solve
            (Algorithm 7), log-determinant, matvec.
  measures  backward error by power iteration and solve residual (Section 6).
  cmatvec   the exact kernel product in plain C with OpenMP (kernel_matvec.c), for the
            power iterations at full size.
  pcg       preconditioned CG with a TLR factor as the preconditioner (Section 6).
"""
