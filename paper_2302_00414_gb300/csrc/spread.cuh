// Kernels with a compile-time window width, each family in its own translation unit:
// spreading for d = 2 and d = 3 (Algorithm 2.4 step 1 and its forms in Algorithms 3.7 / 4.4)
// and interpolation for d = 2, 3 (Algorithm 2.1 step 3).
#pragma once

#include <cstdlib>
#include <vector>

#include "internal.h"
#include "jobset.cuh"

namespace infft {

// cp.async of one aligned element of B bytes (4, 8 or 16) from global to shared memory
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// the environment's choice of a kernel form: 0 or 1 from the variable's first character,
// -1 when it is unset or says neither
inline int env_form(const char* name) {
    const char* e = getenv(name);
    return (e && e[0] == '0') ? 0 : (e && e[0] == '1') ? 1 : -1;
}

// Launch the d = 2 register-row spread when every job qualifies (same m in 2..8, P <= 32,
// all window modes or all B_opt); *used tells whether it did.
template <class R>
infft_status spread2d_try(JobSet<R>& js, cudaStream_t st, bool* used);

// Launch the d = 3 spread when every job qualifies (window modes, same m, tiles of 8^3);
// *used tells whether it did.
template <class R>
infft_status spread3d_try(JobSet<R>& js, cudaStream_t st, bool* used);

// The persistent batched d = 2 adjoint (spread, merging pass along x and pass along y as work
// units of one launch) when every job qualifies; *used tells whether it ran.  Prefixes filled.
infft_status persist2d_try(JobSet<float>& js, cudaStream_t st, bool* used);

// Halo merge and both pruned FFT passes (with deconvolution) of d = 2 adjoint jobs as one
// thread-block-cluster kernel per grid size, for the jobs whose grid it takes; `rest`
// receives the indices of the jobs left to the two-kernel form.
template <class R>
infft_status mergefft2d_try(const JobSet<R>& js, cudaStream_t st, std::vector<int>& rest);

// Launch the fixed-m interpolation for d = 2 (m <= 8) or d = 3 (m <= 6) when every job has
// the same m and power-of-two tiles and grids; *used tells whether it did.  The FFT passes
// must have filled the grids.
template <class R>
infft_status interp2d_try(JobSet<R>& js, cudaStream_t st, bool* used);
template <class R>
infft_status interp3d_try(JobSet<R>& js, cudaStream_t st, bool* used);

}  // namespace infft
