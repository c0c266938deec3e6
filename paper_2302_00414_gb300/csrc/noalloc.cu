// infft_adjoint_noalloc: the reconstruction of infft_adjoint with its per-call scratch
// (padded tiles, oversampled grid, FFT intermediates) taken from one fixed array that
// is part of the library image, so that the call itself allocates no device memory.
//
// Who needs this: applications whose device memory is owned by an external allocator
// or arena that forbids other components from calling cudaMalloc, and latency-bound
// loops that cannot afford cudaMalloc's synchronisation or its late out-of-memory
// failures.  Such callers create their plans up front, then reconstruct through this
// entry point with buffers they already own.
#include <mutex>

#include "internal.h"

// 32 MiB of scratch per device, reserved for the lifetime of the process on every
// device that loads the library.
#define INFFT_NOALLOC_SCRATCH_BYTES (32ull << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[INFFT_NOALLOC_SCRATCH_BYTES];

namespace {

// The device address of g_noalloc_scratch belongs to the module loaded in one CUDA
// context.  A device reset (cudaDeviceReset) destroys the primary context; the next call
// runs in a new context, where the module may sit elsewhere.  So the address is cached
// per context, keyed by the driver's unique context id (cuCtxGetId), and looked up again
// whenever the current context has an id not seen before.
struct CachedAddress {
    unsigned long long ctx_id;
    void* addr;
};
constexpr int kMaxCached = 64;
std::mutex g_mutex;
CachedAddress g_cache[kMaxCached];
int g_ncache = 0;

typedef int (*ctx_get_current_fn)(void**);
typedef int (*ctx_get_id_fn)(void*, unsigned long long*);

// id of the current context through the driver entry points (no link to libcuda)
infft_status current_context_id(unsigned long long* id) {
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        INFFT_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        INFFT_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            infft::set_error("driver entry points cuCtxGetCurrent / cuCtxGetId not found");
            return INFFT_ECUDA;
        }
        get_current = (ctx_get_current_fn)f1;
        get_id = (ctx_get_id_fn)f2;
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, id) != 0) {
        infft::set_error("no current CUDA context");
        return INFFT_ECUDA;
    }
    return INFFT_OK;
}

// Device address of g_noalloc_scratch in the current context.  In host code the symbol
// only names a host-side stand-in, so the address is looked up with cudaGetSymbolAddress,
// once per context (the device current), and cached.
infft_status scratch_address(void** out) {
    // bind the current device's primary context to this thread (cudaSetDevice initialises
    // it and makes it current; nothing is allocated)
    int dev = 0;
    INFFT_CUDA(cudaGetDevice(&dev));
    INFFT_CUDA(cudaSetDevice(dev));
    unsigned long long id = 0;
    INFFT_TRY(current_context_id(&id));
    std::lock_guard<std::mutex> lock(g_mutex);
    for (int i = 0; i < g_ncache; ++i)
        if (g_cache[i].ctx_id == id) { *out = g_cache[i].addr; return INFFT_OK; }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        infft::set_error("cudaGetSymbolAddress(g_noalloc_scratch) failed: %s", cudaGetErrorString(e));
        return INFFT_ECUDA;
    }
    if (g_ncache < kMaxCached) g_cache[g_ncache++] = CachedAddress{id, p};
    else g_cache[id % kMaxCached] = CachedAddress{id, p};
    *out = p;
    return INFFT_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

template <class R>
infft_status run(infft_plan_s* p, int mode, const void* f, void* fhat, cudaStream_t st) {
    using infft::cx;
    const int d = p->d;
    size_t cells_p = 1, grid = 1;
    for (int t = 0; t < d; ++t) { cells_p *= (size_t)p->P; grid *= (size_t)p->Ms; }
    size_t t1 = 0, t2 = 0;
    if (d >= 2) t1 = (size_t)infft::ipow(p->Ms, d - 1) * p->M;
    if (d == 3) t2 = (size_t)p->Ms * p->M * p->M;
    const size_t C = sizeof(cx<R>);
    const size_t b_pad = round256(std::max<size_t>(1, (size_t)p->nitems) * cells_p * C);
    const size_t b_grid = round256(grid * C);
    const size_t b_t1 = round256(t1 * C), b_t2 = round256(t2 * C);
    const size_t need = b_pad + b_grid + b_t1 + b_t2;
    if (need > INFFT_NOALLOC_SCRATCH_BYTES) {
        infft::set_error("infft_adjoint_noalloc: plan needs %zu bytes of scratch, the fixed array holds %llu",
                         need, (unsigned long long)INFFT_NOALLOC_SCRATCH_BYTES);
        return INFFT_EINVAL;
    }
    void* base = nullptr;
    INFFT_TRY(scratch_address(&base));
    unsigned char* s = static_cast<unsigned char*>(base);
    infft::Job<R> job = infft::make_job<R>(p, mode, f, fhat);
    job.padded = reinterpret_cast<cx<R>*>(s);
    job.grid = reinterpret_cast<cx<R>*>(s + b_pad);
    job.tmp1 = t1 ? reinterpret_cast<cx<R>*>(s + b_pad + b_grid) : nullptr;
    job.tmp2 = t2 ? reinterpret_cast<cx<R>*>(s + b_pad + b_grid + b_t1) : nullptr;
    // Every scratch cell is written before it is read (the spread stores whole padded
    // tiles, the merge every grid cell where a separate merge runs, each FFT pass its whole
    // output; for d = 2 the first pass reads the padded tiles directly and the grid is not
    // used), so nothing left by an earlier call needs clearing.
    return infft::run_jobs<R>(&job, 1, st, false, nullptr);
}

}  // namespace

extern "C" {

infft_status infft_adjoint_noalloc(infft_plan_t plan, int mode, const void* f, void* fhat, void* stream) {
    if (!plan || !f || !fhat) {
        infft::set_error("infft_adjoint_noalloc: null argument");
        return INFFT_EINVAL;
    }
    INFFT_TRY(infft::check_mode(plan, mode));   // the same codes and messages as infft_adjoint
    if (!infft::is_device_pointer(f) || !infft::is_device_pointer(fhat)) {
        infft::set_error("infft_adjoint_noalloc: f and fhat must be device pointers");
        return INFFT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return plan->fp64 ? run<double>(plan, mode, f, fhat, st) : run<float>(plan, mode, f, fhat, st);
}

}  // extern "C"
