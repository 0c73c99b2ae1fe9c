"""FP64 CPU oracle for shearlet-regularised multi-label segmentation.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product library never imports it.

The arithmetic lives in ``shearseg_oracle.cpp`` (plain C++17, FP64, its own
FFT); this module compiles it with g++ on first use and wraps it with ctypes.
Each wrapper names the passage of Haeuser & Steidl (arXiv:1112.1805) it
follows.  Parity status per function:

* windows v, b, psi1_hat, psi2_hat, varphi -- pinned (Lemma partitions, the
  overlap identity, the supports of Fig. 1, v(x)+v(1-x)=1);
* filters -- pinned (Theorem: partition of unity at every grid frequency;
  eta = 61 at four scales, Remark 1; evenness);
* fft2 -- pinned (brute-force DFT, numpy.fft);
* analyze / synthesize -- pinned (S^T S = I, isometry, adjointness, direct
  inner products with the translated atoms of eq. wichtig);
* data_term -- pinned (eq. computationOfs on hand values);
* soft_shrink, project_simplex -- pinned (prox optimality by brute force,
  all-support enumeration and KKT);
* admm_iterate -- pinned through its invariants: u-subproblem stationarity,
  fixed-point residual monotonicity, KKT stationarity at convergence, the
  Lambda = 0 and constant-image special cases;
* energy, labels -- pinned (hand values);
* tv_grad, tv_grad_adj -- pinned (hand values, adjointness, constants);
* tv_solve -- pinned (the explicit periodic 5-point stencil applied to the
  solution returns the right-hand side);
* tv_shrink -- pinned (prox optimality by brute force, closed form);
* tv_admm_iterate -- pinned through its invariants (u-subproblem
  stationarity, fixed-point residual monotonicity, KKT at convergence, the
  lambda = 0 and constant-image special cases); tv_energy by hand values of
  a stripe image.
"""

from .oracle import *  # noqa: F401,F403
