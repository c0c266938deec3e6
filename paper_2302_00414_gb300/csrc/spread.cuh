// Kernels with a compile-time window width, each family in its own translation unit:
// spreading for d = 2 and d = 3 (Algorithm 2.4 step 1 and its forms in Algorithms 3.7 / 4.4)
// and interpolation for d = 2, 3 (Algorithm 2.1 step 3).
#pragma once

#include "internal.h"
#include "jobset.cuh"

namespace infft {

// Launch the d = 2 register-row spread when every job qualifies (same m in 2..8, P <= 32,
// all window modes or all B_opt); *used tells whether it did.
template <class R>
infft_status spread2d_try(JobSet<R>& js, cudaStream_t st, bool* used);

// Launch the d = 3 spread when every job qualifies (window modes, same m, tiles of 8^3);
// *used tells whether it did.
template <class R>
infft_status spread3d_try(JobSet<R>& js, cudaStream_t st, bool* used);

// Launch the fixed-m interpolation for d = 2 (m <= 8) or d = 3 (m <= 6) when every job has
// the same m and power-of-two tiles and grids; *used tells whether it did.  The FFT passes
// must have filled the grids.
template <class R>
infft_status interp2d_try(JobSet<R>& js, cudaStream_t st, bool* used);
template <class R>
infft_status interp3d_try(JobSet<R>& js, cudaStream_t st, bool* used);

}  // namespace infft
