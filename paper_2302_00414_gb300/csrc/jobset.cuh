// Kernel-parameter block holding up to MAXJ transform descriptors.
//
// Every transform kernel takes one JobSet by value as a __grid_constant__
// parameter, so that a single call and a batch of independent transforms use the
// same kernels, blocks find their job by binary search over a prefix array, and a
// CUDA graph captures the launch with no device-side tables.
#pragma once

#include "common.cuh"

namespace infft {

constexpr int MAXJ = 96;

template <class R>
struct JobSet {
    int njobs;
    int wpb;                    // warps (items) per block of the spread / interpolation kernels
    int smem_per_warp;          // bytes of shared memory per warp (spread / interpolation)
    int L;                      // lines per block of the FFT passes
    // one explicit adjoint FFT pass (axA > 0): J.grid as an (axA, Ms, axB) tensor -> J.out as
    // (axA, M, axB) in axblk blocks along the middle index (see run_fft_axis)
    long long axA, axB;
    int axblk;
    int pre_items[MAXJ + 1];    // prefix of work items
    int pre_merge[MAXJ + 1];    // prefix of merge blocks
    int pre_fft[3][MAXJ + 1];   // prefix of FFT blocks per pass
    // the float32 window polynomial of every job, when all jobs share one (wtab_ok): read by
    // the unrolled tap evaluation straight from the parameter block, no shared-memory loads
    int wtab_ok;
    alignas(16) float wtab[(WPOLY_DEG + 1) * 12];
    Job<R> job[MAXJ];
};

static_assert(sizeof(JobSet<double>) <= 30000, "JobSet exceeds the kernel parameter limit");

}  // namespace infft
