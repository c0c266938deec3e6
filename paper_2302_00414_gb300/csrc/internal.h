// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <array>
#include <vector>

#include "common.cuh"

struct infft_plan_s {
    int d, M, Ms, m;
    int64_t N;
    double sigma;
    unsigned flags;
    bool fp64;
    int window;               // infft::WindowKind
    int T, ntile, P, nitems, S;
    infft_tune_t tune = {0, 0, 0, 0, 0};   // caller's tuning (0 = library default)
    int logMs;
    double beta;

    // sorted points (device)
    int* perm = nullptr;
    uint32_t* cell = nullptr;
    void* u = nullptr;        // float or double, N*d
    double* x64 = nullptr;    // wrapped points in sorted order, N*d (B_opt, weights residual)
    int4* items = nullptr;
    int* tile_items = nullptr;
    int* cell_start = nullptr;  // key range + 1 prefix (tile-major cell order)
    size_t nkeys = 0;

    // tables (device)
    void* dinv = nullptr;     // M entries
    void* tw = nullptr;       // Ms/2 complex
    void* dinv_win = nullptr; // M entries for the B_opt window (may alias dinv)
    float* wpoly = nullptr;   // window polynomial table (float32 Kaiser-Bessel plans)
    std::vector<float> wpoly_host;   // host copy of that table

    // weights (device): caller order float64 master + sorted copy in plan precision
    void* w_master = nullptr; // N complex128, caller order
    void* w_sorted = nullptr; // N complex (plan precision), sorted
    bool has_weights = false;

    // B_opt (device)
    void* coef = nullptr;     // N*S^d complex (plan precision), sorted
    double* coef64 = nullptr; // N*S^d complex128, sorted
    bool has_bopt = false;
    int bopt_window = 0;

    // scratch (device)
    void* padded = nullptr;
    void* grid = nullptr;
    void* tmp1 = nullptr;
    void* tmp2 = nullptr;
    size_t scratch_bytes[4] = {0, 0, 0, 0};   // sizes of padded, grid, tmp1, tmp2
    // further scratch sets, used when one batched call names the plan more than once
    // (slot k >= 1 is extra[k - 1]); allocated on first need and kept
    std::vector<std::array<void*, 4>> extra;
    void* io_in = nullptr;    // staging for host inputs / outputs
    void* io_out = nullptr;

    size_t device_bytes = 0;
    // plans made inside the library (the weights' degree-2M plan) allocate from the
    // library's stream-ordered pool on this stream and free the same way
    bool pooled = false;
    cudaStream_t pool_stream = nullptr;
};

struct infft_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* jobs_dev = nullptr;
    int* prefix_dev = nullptr;
    void* stage_in = nullptr;    // device staging of host inputs / outputs (host-buffer batches)
    void* stage_out = nullptr;
};

namespace infft {

// Stream-ordered device memory from a pool the library owns per device (up to 1 GiB of
// freed blocks is kept for reuse).  Neither call synchronises
// the device, unlike cudaMalloc / cudaFree, so a thread building plans or weights does not
// hold up other threads' launches.  Memory is usable in stream order on `st`.
infft_status pool_alloc(void** ptr, size_t bytes, cudaStream_t st);
void pool_free(void* ptr, cudaStream_t st);

// Copy device -> pageable host memory after the stream has drained: a pageable copy
// waits for the stream's earlier work inside the driver and holds up the other host
// threads' CUDA calls meanwhile; synchronising first leaves only the short copy.
infft_status read_back(void* dst, const void* src, size_t bytes, cudaStream_t st);

// create a plan (argument checks of infft_plan); pooled plans use pool_alloc on `stream`
infft_status plan_create(int d, int M, int64_t N, const double* x, double sigma, int m, unsigned flags,
                         cudaStream_t stream, bool pooled, infft_plan_s** out, const infft_tune_t* tune = nullptr);
// free a plan's memory without a device-wide synchronisation (pooled plans: in stream order)
void plan_release(infft_plan_s* p);

// thread-local error message and launch counter
void set_error(const char* fmt, ...);
void count_launch(int n = 1);

// host-side fault injection (infft_inject_faults / INFFT_FAULT): true when `bit` is set
enum { FAULT_ALLOC = 1, FAULT_LAUNCH = 2, FAULT_CG = 4 };
bool fault(unsigned bit);

#define INFFT_CUDA(call)                                                                   \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess) {                                                          \
            infft::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e__),     \
                             __FILE__, __LINE__);                                          \
            return INFFT_ECUDA;                                                            \
        }                                                                                  \
    } while (0)

#define INFFT_LAUNCHED()                                                                   \
    do {                                                                                   \
        infft::count_launch();                                                             \
        if (infft::fault(infft::FAULT_LAUNCH)) {                                           \
            infft::set_error("injected launch failure (%s:%d)", __FILE__, __LINE__);       \
            return INFFT_ECUDA;                                                            \
        }                                                                                  \
        cudaError_t e__ = cudaGetLastError();                                              \
        if (e__ != cudaSuccess) {                                                          \
            infft::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e__),  \
                             __FILE__, __LINE__);                                          \
            return INFFT_ECUDA;                                                            \
        }                                                                                  \
    } while (0)

#define INFFT_TRY(expr)                                                                    \
    do {                                                                                   \
        infft_status s__ = (expr);                                                         \
        if (s__ != INFFT_OK) return s__;                                                   \
    } while (0)

infft_status dev_alloc(infft_plan_s* p, void** ptr, size_t bytes);
// in-place exclusive prefix sum of n ints on the device (stream ordered)
infft_status scan_exclusive(int* data, long long n, cudaStream_t st);
bool is_device_pointer(const void* ptr);
// the preconditions of a reconstruction mode on a plan (INFFT_EINVAL for an unknown mode,
// INFFT_ESTATE for DCF without weights, BOPT without B_opt, or a window mode on a
// Dirichlet-window plan); shared by every entry point that takes a mode
infft_status check_mode(const infft_plan_s* p, int mode);

// Build the Job descriptors of a list of plans for one transform each.
template <class R>
Job<R> make_job(const infft_plan_s* p, int mode, const void* in, void* out, int slot = 0);

// Execute transforms for jobs of one d and precision: the adjoint (spread -> merge ->
// FFT passes with crop and deconvolution) or the forward NFFT (FFT passes with
// padding -> interpolation); batches larger than the parameter block are chunked.
// With `ev` (5 events) the adjoint of the first chunk records an event before the
// spread and after the spread, the merge and each FFT pass.
template <class R>
infft_status run_jobs(const std::vector<Job<R>>& jobs, cudaStream_t st, bool forward, cudaEvent_t* ev = nullptr);
template <class R>
infft_status run_jobs(const Job<R>* jobs, size_t count, cudaStream_t st, bool forward, cudaEvent_t* ev = nullptr);

// Spreading and halo merge of one job into J.grid (the oversampled grid, Ms^d cells), no FFT.
template <class R>
infft_status run_spread_grid(const Job<R>& J, cudaStream_t st);

// One adjoint FFT pass with crop and deconvolution along the middle index of J.grid viewed
// as an (A, Ms, B) tensor, into J.out as nblk blocks along the middle index, block c holding
// the (A, M/nblk, B) tensor of the indices c M/nblk .. (c+1) M/nblk - 1.
template <class R>
infft_status run_fft_axis(const Job<R>& J, long long A, long long B, int nblk, cudaStream_t st);

// The d FFT passes of one job alone (no spreading, merge or interpolation): forward = true
// maps J.in (M^d over I_M, times J.dinv per axis) to J.grid (Ms^d) with sign +; forward =
// false maps J.grid to J.out (M^d, times J.dinv per axis) with sign -.  Uses J.tw, J.tmp1,
// J.tmp2 (each large enough for the intermediate tensors) and J.d, J.M, J.Ms.
template <class R>
infft_status run_fft_passes(const Job<R>& J, cudaStream_t st, bool forward);

// bounded waits of the persistent d = 2 kernel that gave up since the library was loaded
unsigned int persist_wait_timeouts();

}  // namespace infft
