"""GB300 (sm_103a) direct inverse NFFT: Python binding of libinfft.so.

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``);
this package only marshals arguments.  Importing it does not load the library;
the first call does, and raises if it has not been built.
"""
from .api import (BOPT_PATTERN_2M2, BOPT_PATTERN_PAPER, BOPT_REAL, ECUDA, EINVAL, ENOMEM, ENOTCONV, ESTATE,
                  EUNSUPPORTED, EXPORTED, FP32, FP64, MODE_BOPT,
                  MODE_DCF, MODE_PLAIN, OK, WIN_BSPLINE, WIN_DIRICHLET, WIN_KB, Batch, InfftError, Plan,
                  adjoint_batched, adjoint_batched_timed, infft_adjoint, infft_adjoint_batched, infft_destroy, infft_forward,
                  infft_optimize_B, infft_plan, infft_weights, last_error, launch_count, launch_count_reset, load, wait_timeouts,
                  WEIGHTS_AUTO, WEIGHTS_NFFT, WEIGHTS_TOEPLITZ, POOLED, inject_faults)

__all__ = [n for n in dir() if not n.startswith("_")]
