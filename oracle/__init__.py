"""CPU oracle for the FlashEigen hot path (arXiv 1602.01421).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU legs (the
CPU baseline and the reference arm) may import this package; bench.py's large-graph legs also
use its SpMM to check the residuals of the eigenpairs they report, after the timed solves.  The
CUDA library never calls it, and it shares no code with the CUDA library: it is a plain, slow,
FP64 restatement of what the method computes.

Contents (each function cites the passage it follows):
  core.spmm / core.spmm_rows   Y = A X, Section 3.3 (plain C, FP64 accumulate)
  core.jacobi                  projected m x m eigenproblem, Algorithm 1 step (2)
  blockops                     the dense operations of Table 1 (MvTransMv, MvTimesMatAddMv, ...)
  bks.block_krylov_schur       the Block Krylov-Schur eigensolver (Sections 3.1, 1, 4.3)
  svd.svds / svd.transpose     singular triplets of a directed graph via A^T A (Section 4.3.2)
  rng                          the counter-based start/replacement block generator
  mlp                          the learned start block's network (forward, backward)
"""
