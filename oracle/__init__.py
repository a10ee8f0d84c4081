"""Plain FP64 CPU oracle for the sampled limited-memory row-action method (slimLS).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import, call or run it.  It shares no code with the CUDA library
(`paper_1912_07962_gb300`); the two meet only in the seeded input generators
of `workloads`, which hold none of the method's arithmetic.

Everything here is written for a reader checking it against the paper by eye:
numpy / scipy primitives (sparse matmul, Cholesky, QR) as steps, no blocking,
no fusion, float64 throughout.

Modules
  rng      counter-based SplitMix64 and the block sampler (Sec. 1: i.i.d. uniform W_k)
  joseph   the Joseph ray-driven rows of the parallel-beam forward model
  slim     one slimLS step, Eq. (ram)/(B_k), in Woodbury and direct form; runs
  targets  reference solutions: x_LS (Eq. LS), Tikhonov x_tik, CGLS
  theory   Sec. 3 quantities for r = 0: B_k(alpha), B, x_hat (Eq. xhat), bounds
  lsqr     LSQR for the damped least-squares step of Eq. (slimLSstep)
  tik      one slimTik step, Eq. (slimTik) (C_k = L^T L), direct and Woodbury form
  comparators  sg (B_k = alpha_k I), olbfgs (two-loop L-BFGS), decaying damping

Parity status: every function is pinned by tests in `tests/test_oracle_*.py`
against closed forms, special cases and the paper's theorems, except the
absolute reconstruction quality on the synthetic phantoms (parity unpinned:
the paper prints no number for these inputs).
"""
