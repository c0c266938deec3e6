"""FP64 CPU oracle for the direct inverse NFFT of Kircheis & Potts.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct numpy code that
states what the method computes, written from the paper:

* ``fourier``  -- the nonequispaced Fourier matrix A and the exact sums
  f = A fhat (eq. nfft) and h = A^* f (eq. nfft*), Section 2.
* ``windows``  -- window functions w, their Fourier transforms w^ and the
  truncated periodised window (Section 2.1, Remark 2.2, eq. window_bspline,
  eq. kernel_Dirichlet_asym).
* ``nfft``     -- Algorithm 2.1 (NFFT) and Algorithm 2.4 (adjoint NFFT) step by
  step, and the factor matrices B, F, D of eq. matrix_B / matrix_F / matrix_D.
* ``weights``  -- the density compensation weights of Corollary 3.4 /
  Algorithm 3.6 as the (minimum-norm) least-squares solution of
  A_{2M}^T w = e_0, their residual (eq. residual_lgs) and the
  reconstruction of Algorithm 3.7.
* ``bopt``     -- Algorithm 4.3 column by column from the definition
  (explicit H_l, explicit right side, dense least squares), the closed forms
  of Remark 4.2 and the reconstruction of Algorithm 4.4.

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library and never imports it.
"""
