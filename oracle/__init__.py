"""Plain, slow, FP64 CPU oracle for the STROM hot path (TEST INFRASTRUCTURE).

This package exists only to check the CUDA path. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product library never calls it and shares no code with it.

Contents, each following the paper directly:
  relax      sparse second-order moment relaxation (Prop. 1) converted to the
             PSD-only standard SDP {C, A, b} (Sec. 2.3, eq. standardsdp)
  sgs_admm   Algorithm 1 (sGS-ADMM) with the stopping rule of
             eq. (kkt-residual); PSD projection Pi(X) = Q max(0, W) Q^T
             (Sec. 4, parallel PSD cone projection)
  jacobi     the same projection with a LAPACK-free cyclic-by-row Jacobi
             eigensolver (Golub & Van Loan, Sec. 8.5), the reference of the
             PSD-projection microbench
  certify    rank-1 test (Theorem 1 iii), extraction heuristic (Sec. 2.2),
             valid lower bound (eq. valid-lowerbound), suboptimality gap
             (eq. suboptimality-gap), R_beta (Theorem of App. C)
  warm       nearest-neighbour warm start from stored solutions (Sec. 5,
             inverted pendulum)

Parity status: every function is pinned by tests under tests/ against the
paper's worked identities, closed forms, invariants or brute force, except
where a docstring says "parity unpinned".
"""
