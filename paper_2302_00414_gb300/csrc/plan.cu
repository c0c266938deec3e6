// Plan creation (point binning, tables) and the C-ABI entry points of the
// transforms (Algorithms 2.1, 2.4, 3.7, 4.4).
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <vector>

#include "internal.h"
#include "jobset.cuh"

namespace infft {


// ----------------------------------------------------------------------------------------
// error state and launch counter
static thread_local char g_err[512] = "";
static thread_local uint64_t g_launches = 0;

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void count_launch(int n) { g_launches += (uint64_t)n; }

// injected faults: the mask set by infft_inject_faults, initially from INFFT_FAULT
// (a comma-separated list of alloc, launch, cg)
static std::atomic<int> g_fault_mask{-1};

static unsigned fault_mask_from_env() {
    const char* e = getenv("INFFT_FAULT");
    unsigned m = 0;
    if (e) {
        if (strstr(e, "alloc")) m |= FAULT_ALLOC;
        if (strstr(e, "launch")) m |= FAULT_LAUNCH;
        if (strstr(e, "cg")) m |= FAULT_CG;
    }
    return m;
}

bool fault(unsigned bit) {
    int m = g_fault_mask.load(std::memory_order_relaxed);
    if (m < 0) {
        m = (int)fault_mask_from_env();
        g_fault_mask.store(m, std::memory_order_relaxed);
    }
    return (m & (int)bit) != 0;
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

infft_status pool_alloc(void** ptr, size_t bytes, cudaStream_t st) {
    *ptr = nullptr;
    int dev = 0;
    INFFT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device %d out of range", dev); return INFFT_EINVAL; }
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            INFFT_CUDA(cudaMemPoolCreate(&g_pool[dev], &props));
            // keep up to 1 GiB of freed blocks for reuse; the rest goes back to the device
            // at the next synchronisation (a weights solve frees several GB of temporaries)
            uint64_t keep = 1ull << 30;
            INFFT_CUDA(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        }
        pool = g_pool[dev];
    }
    cudaError_t e = cudaMallocFromPoolAsync(ptr, std::max<size_t>(bytes, 16), pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        set_error("pool allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return INFFT_ENOMEM;
    }
    return INFFT_OK;
}

infft_status read_back(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    INFFT_CUDA(cudaStreamSynchronize(st));
    INFFT_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
    INFFT_CUDA(cudaStreamSynchronize(st));
    return INFFT_OK;
}

void pool_free(void* ptr, cudaStream_t st) {
    if (ptr) cudaFreeAsync(ptr, st);
}

infft_status dev_alloc(infft_plan_s* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return INFFT_OK;
    if (fault(FAULT_ALLOC)) {
        set_error("injected allocation failure (%zu bytes)", bytes);
        return INFFT_ENOMEM;
    }
    if (p && p->pooled) {
        INFFT_TRY(pool_alloc(ptr, bytes, p->pool_stream));
        p->device_bytes += bytes;
        return INFFT_OK;
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return INFFT_ENOMEM;
    }
    if (p) p->device_bytes += bytes;
    return INFFT_OK;
}

// page-locked host memory (cudaHostAlloc / cudaHostRegister): copies from and to it can be
// captured into a CUDA graph
static bool is_pinned_host_pointer(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

bool is_device_pointer(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ----------------------------------------------------------------------------------------
// binning kernels

// Wrap x into [-1/2, 1/2), split M_sigma x into base cell and fractional offset, and
// compute the tile-major cell key.  The arithmetic mirrors x - floor(x + 1/2),
// M_sigma * x, floor, with correctly rounded operations and no contraction.
__global__ void k_prep(const double* __restrict__ x, int N, int d, int Ms, int T, int nt,
                       uint32_t* __restrict__ key, uint32_t* __restrict__ cellrm,
                       double* __restrict__ u, double* __restrict__ xw_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    uint32_t tile = 0, intile = 0, rm = 0;
    for (int t = 0; t < d; ++t) {
        const double xv = x[(size_t)j * d + t];
        const double xw = __dsub_rn(xv, floor(__dadd_rn(xv, 0.5)));
        const double y = __dmul_rn((double)Ms, xw);
        const double bf = floor(y);
        u[(size_t)j * d + t] = __dsub_rn(y, bf);
        xw_out[(size_t)j * d + t] = xw;
        int c = (int)bf % Ms;
        if (c < 0) c += Ms;
        tile = tile * nt + c / T;
        intile = intile * T + c % T;
        rm = rm * Ms + c;
    }
    uint32_t tpow = 1;
    for (int t = 0; t < d; ++t) tpow *= T;
    key[j] = tile * tpow + intile;
    cellrm[j] = rm;
}

__global__ void k_hist(const uint32_t* __restrict__ key, int N, int* __restrict__ count) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) atomicAdd(count + key[j], 1);
}

// exclusive scan, 1024 elements per block
__global__ void k_scan_block(int* __restrict__ data, long long n, int* __restrict__ block_sums) {
    __shared__ int wsum[32];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    int v = (i < n) ? data[i] : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;  // inclusive scan of warp sums
    }
    __syncthreads();
    const int before = (wid > 0) ? wsum[wid - 1] : 0;
    if (i < n) data[i] = before + incl - v;
    if (threadIdx.x == 1023 && block_sums) block_sums[blockIdx.x] = wsum[31];
}

__global__ void k_scan_add(int* __restrict__ data, long long n, const int* __restrict__ block_off) {
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) data[i] += block_off[blockIdx.x];
}

infft_status scan_exclusive(int* data, long long n, cudaStream_t st) {
    const long long nb = (n + 1023) / 1024;
    if (nb == 1) {
        k_scan_block<<<1, 1024, 0, st>>>(data, n, nullptr);
        INFFT_LAUNCHED();
        return INFFT_OK;
    }
    int* sums = nullptr;
    INFFT_CUDA(cudaMallocAsync((void**)&sums, nb * sizeof(int), st));
    k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(data, n, sums);
    INFFT_LAUNCHED();
    infft_status s = scan_exclusive(sums, nb, st);
    if (s != INFFT_OK) { cudaFreeAsync(sums, st); return s; }
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(data, n, sums);
    INFFT_LAUNCHED();
    INFFT_CUDA(cudaFreeAsync(sums, st));
    return INFFT_OK;
}

__global__ void k_scatter(const uint32_t* __restrict__ key, int N, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ order) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const uint32_t k = key[j];
    order[start[k] + atomicAdd(fill + k, 1)] = j;
}

// points of one cell in ascending caller index: makes the order (and therefore every
// floating-point summation order downstream) independent of the scatter's atomics.
__global__ void k_cell_sort(const int* __restrict__ start, long long nkeys, int* __restrict__ order) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    const int a = start[k], b = start[k + 1];
    for (int i = a + 1; i < b; ++i) {
        const int v = order[i];
        int p = i - 1;
        while (p >= a && order[p] > v) { order[p + 1] = order[p]; --p; }
        order[p + 1] = v;
    }
}

template <class R>
__global__ void k_gather(const int* __restrict__ order, int N, int d, const uint32_t* __restrict__ cellrm,
                         const double* __restrict__ u, const double* __restrict__ xw, uint32_t* __restrict__ cell_s,
                         R* __restrict__ u_s, double* __restrict__ x_s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int j = order[i];
    cell_s[i] = cellrm[j];
    for (int t = 0; t < d; ++t) {
        u_s[(size_t)i * d + t] = (R)u[(size_t)j * d + t];
        x_s[(size_t)i * d + t] = xw[(size_t)j * d + t];
    }
}

// 1/(M_sigma w^(k)) for k in I_M (one axis of eq. matrix_D) and FFT twiddles exp(-2 pi i k/Ms).
template <class R>
__global__ void k_tables(int M, int Ms, int m, int window, double beta, R* __restrict__ dinv,
                         cx<R>* __restrict__ tw, double* __restrict__ dinv64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) {
        const double k = (double)(i - M / 2);
        double wh;
        if (window == WK_KB) {
            const double a = 2.0 * M_PI * m * k / Ms;
            const double r = beta * beta - a * a;
            double q;
            if (r > 0) { const double s = sqrt(r); q = sinh(s) / s; }
            else if (r < 0) { const double s = sqrt(-r); q = sin(s) / s; }
            else q = 1.0;
            wh = (2.0 * m / Ms) * q;
        } else if (window == WK_BSPLINE) {
            const double t = k / Ms;
            const double s = (k == 0) ? 1.0 : sinpi(t) / (M_PI * t);
            wh = pow(s, 2 * m) / Ms;
        } else {
            wh = 1.0;
        }
        const double v = 1.0 / (Ms * wh);
        dinv[i] = (R)v;
        if (dinv64) dinv64[i] = v;
    }
    if (i < Ms / 2) {
        double s, c;
        sincospi(2.0 * i / Ms, &s, &c);
        tw[i] = mk<R>((R)c, (R)(-s));
    }
}

// Window polynomials for float32 Kaiser-Bessel plans: one thread per tap s = 1..2m
// interpolates phi(u + m - s), u in [0,1], at the WPOLY_DEG+1 Chebyshev points of
// v = 2u - 1 and rewrites the Chebyshev series in powers of v (float64 throughout).
__global__ void k_wpoly(int m, double beta, float* __restrict__ coef) {
    constexpr int P1 = WPOLY_DEG + 1;
    const int W = 2 * m + 1;
    const int WP = wpoly_stride(W);
    const int s = threadIdx.x;
    if (s >= WP) return;
    if (s == 0 || s >= W) {  // tap 0 keeps the exact rule; padding slots are zero
        for (int k = 0; k < P1; ++k) coef[k * WP + s] = 0.f;
        return;
    }
    double fv[P1], c[P1], a[P1], tp[P1], tc[P1], tn[P1];
    for (int k = 0; k < P1; ++k) {
        const double v = cospi((k + 0.5) / P1);
        const double u = 0.5 * (v + 1.0);
        fv[k] = kb_phi<double>(u + (double)(m - s), 1.0 / m, beta);
    }
    for (int j = 0; j < P1; ++j) {
        double acc = 0;
        for (int k = 0; k < P1; ++k) acc += fv[k] * cospi(j * (k + 0.5) / P1);
        c[j] = acc * 2.0 / P1;
    }
    c[0] *= 0.5;
    for (int k = 0; k < P1; ++k) { a[k] = 0; tp[k] = 0; tc[k] = 0; }
    tp[0] = 1.0;          // T_0
    tc[1] = 1.0;          // T_1
    for (int k = 0; k < P1; ++k) a[k] += c[0] * tp[k] + c[1] * tc[k];
    for (int j = 2; j < P1; ++j) {
        // T_j = 2 v T_{j-1} - T_{j-2}
        for (int k = 0; k < P1; ++k) tn[k] = -tp[k] + ((k > 0) ? 2.0 * tc[k - 1] : 0.0);
        for (int k = 0; k < P1; ++k) { a[k] += c[j] * tn[k]; tp[k] = tc[k]; tc[k] = tn[k]; }
    }
    for (int k = 0; k < P1; ++k) coef[k * WP + s] = (float)a[k];
}

// ----------------------------------------------------------------------------------------
template <class R>
Job<R> make_job(const infft_plan_s* p, int mode, const void* in, void* out, int slot) {
    Job<R> J;
    memset(&J, 0, sizeof(J));
    J.d = p->d; J.M = p->M; J.Ms = p->Ms; J.m = p->m;
    J.N = (int)p->N; J.T = p->T; J.ntile = p->ntile;
    // padded edge: the window's 2m+1 taps need T + 2m, the 2m+2 slots of B_opt T + 2m + 1
    // (the plan's P, which sizes the scratch)
    J.P = (mode == INFFT_MODE_BOPT) ? p->P : p->T + 2 * p->m;
    J.nitems = p->nitems; J.window = p->window; J.mode = mode; J.S = p->S;
    J.prefetch = p->tune.prefetch; J.fused_fft = p->tune.fused_fft;
    J.beta = (R)p->beta; J.inv_m = (R)(1.0 / p->m);
    J.perm = p->perm; J.cell = p->cell; J.u = (const R*)p->u;
    J.w = (const cx<R>*)p->w_sorted; J.coef = (const cx<R>*)p->coef;
    J.items = p->items; J.tile_items = p->tile_items;
    J.dinv = (mode == INFFT_MODE_BOPT && p->dinv_win) ? (const R*)p->dinv_win : (const R*)p->dinv;
    J.tw = (const cx<R>*)p->tw;
    J.wpoly = p->wpoly;
    J.wpoly_h = p->wpoly_host.empty() ? nullptr : p->wpoly_host.data();
    if (slot == 0) {
        J.padded = (cx<R>*)p->padded; J.grid = (cx<R>*)p->grid;
        J.tmp1 = (cx<R>*)p->tmp1; J.tmp2 = (cx<R>*)p->tmp2;
    } else {
        const std::array<void*, 4>& e = p->extra[slot - 1];
        J.padded = (cx<R>*)e[0]; J.grid = (cx<R>*)e[1];
        J.tmp1 = (cx<R>*)e[2]; J.tmp2 = (cx<R>*)e[3];
    }
    J.in = (const cx<R>*)in; J.out = (cx<R>*)out;
    return J;
}
template Job<float> make_job<float>(const infft_plan_s*, int, const void*, void*, int);
template Job<double> make_job<double>(const infft_plan_s*, int, const void*, void*, int);

static void free_plan(infft_plan_s* p) {
    if (!p) return;
    void* ptrs[] = {p->perm, p->cell, p->u, p->x64, p->items, p->tile_items, p->cell_start, p->dinv, p->tw,
                    p->dinv_win, p->w_master, p->w_sorted, p->coef, p->coef64, p->padded, p->grid, p->tmp1,
                    p->tmp2, p->io_in, p->io_out, p->wpoly};
    for (void* q : ptrs)
        if (q) { if (p->pooled) pool_free(q, p->pool_stream); else cudaFree(q); }
    for (const auto& e : p->extra)
        for (void* q : e)
            if (q) { if (p->pooled) pool_free(q, p->pool_stream); else cudaFree(q); }
    delete p;
}

void plan_release(infft_plan_s* p) { free_plan(p); }

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static infft_status build_plan(infft_plan_s* p, const double* x_in, cudaStream_t st) {
    const int d = p->d, Ms = p->Ms, m = p->m;
    const int N = (int)p->N;
    const size_t R_sz = p->fp64 ? sizeof(double) : sizeof(float);
    const size_t C_sz = 2 * R_sz;

    // tiles: T^d cells, T > m
    const int Tdef = d == 1 ? 256 : (d == 2 ? 16 : 8);
    p->T = p->tune.tile > 0 ? p->tune.tile : std::min(Tdef, Ms);
    if (p->T > Ms || (p->T & (p->T - 1))) {
        set_error("tile edge %d must be a power of two <= M_sigma = %d", p->T, Ms);
        return INFFT_EINVAL;
    }
    if (p->T <= m) {
        set_error("tile edge %d must exceed m = %d", p->T, m);
        return INFFT_EUNSUPPORTED;
    }
    p->ntile = (Ms + p->T - 1) / p->T;
    p->P = p->T + 2 * m + 1;
    p->S = 2 * m + 2;
    long long nkeys = 1;
    for (int t = 0; t < d; ++t) nkeys *= (long long)p->ntile * p->T;
    p->nkeys = (size_t)nkeys;
    long long msd = 1;
    for (int t = 0; t < d; ++t) msd *= Ms;
    if (nkeys >= (1ll << 31) || msd >= (1ll << 31)) {
        set_error("grid too large");
        return INFFT_EUNSUPPORTED;
    }

    // points to the device
    double* x_dev = nullptr;
    const bool x_on_dev = is_device_pointer(x_in);
    // temporaries of the build, returned to the pool in stream order on every exit path
    struct Temps {
        cudaStream_t st;
        std::vector<void*> v;
        ~Temps() { for (void* q : v) pool_free(q, st); }
    } temps{st, {}};
    INFFT_TRY(pool_alloc((void**)&x_dev, (size_t)N * d * sizeof(double), st));
    temps.v.push_back(x_dev);
    INFFT_CUDA(cudaMemcpyAsync(x_dev, x_in, (size_t)N * d * sizeof(double),
                               x_on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    uint32_t *key = nullptr, *cellrm = nullptr;
    double *u64 = nullptr, *xw = nullptr;
    int *count = nullptr, *fill = nullptr, *order = nullptr;
    INFFT_TRY(pool_alloc((void**)&key, (size_t)N * 4, st));
    temps.v.push_back(key);
    INFFT_TRY(pool_alloc((void**)&cellrm, (size_t)N * 4, st));
    temps.v.push_back(cellrm);
    INFFT_TRY(pool_alloc((void**)&u64, (size_t)N * d * 8, st));
    temps.v.push_back(u64);
    INFFT_TRY(pool_alloc((void**)&xw, (size_t)N * d * 8, st));
    temps.v.push_back(xw);
    INFFT_TRY(pool_alloc((void**)&fill, (size_t)(nkeys + 1) * 4, st));
    temps.v.push_back(fill);
    INFFT_TRY(pool_alloc((void**)&order, (size_t)N * 4, st));
    temps.v.push_back(order);
    INFFT_TRY(dev_alloc(p, (void**)&p->cell_start, (size_t)(nkeys + 1) * 4));
    count = p->cell_start;
    INFFT_CUDA(cudaMemsetAsync(count, 0, (size_t)(nkeys + 1) * 4, st));
    INFFT_CUDA(cudaMemsetAsync(fill, 0, (size_t)(nkeys + 1) * 4, st));

    const int tb = 256;
    const int gb = (N + tb - 1) / tb;
    k_prep<<<gb, tb, 0, st>>>(x_dev, N, d, Ms, p->T, p->ntile, key, cellrm, u64, xw);
    INFFT_LAUNCHED();
    k_hist<<<gb, tb, 0, st>>>(key, N, count);
    INFFT_LAUNCHED();
    INFFT_TRY(scan_exclusive(count, nkeys + 1, st));
    k_scatter<<<gb, tb, 0, st>>>(key, N, count, fill, order);
    INFFT_LAUNCHED();
    k_cell_sort<<<(unsigned)((nkeys + 255) / 256), 256, 0, st>>>(count, nkeys, order);
    INFFT_LAUNCHED();

    INFFT_TRY(dev_alloc(p, (void**)&p->perm, (size_t)N * 4));
    INFFT_TRY(dev_alloc(p, (void**)&p->cell, (size_t)N * 4));
    INFFT_TRY(dev_alloc(p, &p->u, (size_t)N * d * R_sz));
    INFFT_TRY(dev_alloc(p, (void**)&p->x64, (size_t)N * d * 8));
    INFFT_CUDA(cudaMemcpyAsync(p->perm, order, (size_t)N * 4, cudaMemcpyDeviceToDevice, st));
    if (p->fp64)
        k_gather<double><<<gb, tb, 0, st>>>(order, N, d, cellrm, u64, xw, p->cell, (double*)p->u, p->x64);
    else
        k_gather<float><<<gb, tb, 0, st>>>(order, N, d, cellrm, u64, xw, p->cell, (float*)p->u, p->x64);
    INFFT_LAUNCHED();

    // work items: split each tile's points into chunks of at most `cap`
    long long tpow = 1, ntl = 1;
    for (int t = 0; t < d; ++t) { tpow *= p->T; ntl *= p->ntile; }
    const int ntiles = (int)ntl;  // nkeys = ntiles * tpow
    std::vector<int> cs(nkeys + 1);
    INFFT_TRY(read_back(cs.data(), count, (size_t)(nkeys + 1) * 4, st));
    INFFT_CUDA(cudaStreamSynchronize(st));
    // d = 1: short items so that a few hundred points still spread on several warps
    const int cap = p->tune.item_cap > 0 ? p->tune.item_cap : (d == 1 ? 32 : 512);
    std::vector<int4> items;
    std::vector<int> tile_items(ntiles + 1, 0);
    for (int tl = 0; tl < ntiles; ++tl) {
        tile_items[tl] = (int)items.size();
        const int a = cs[(size_t)tl * tpow], b = cs[(size_t)(tl + 1) * tpow];
        for (int s = a; s < b; s += cap) items.push_back(make_int4(tl, s, std::min(cap, b - s), 0));
    }
    tile_items[ntiles] = (int)items.size();
    p->nitems = (int)items.size();
    INFFT_TRY(dev_alloc(p, (void**)&p->items, std::max<size_t>(1, items.size()) * sizeof(int4)));
    INFFT_TRY(dev_alloc(p, (void**)&p->tile_items, (size_t)(ntiles + 1) * 4));
    if (!items.empty())
        INFFT_CUDA(cudaMemcpyAsync(p->items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    INFFT_CUDA(cudaMemcpyAsync(p->tile_items, tile_items.data(), (size_t)(ntiles + 1) * 4, cudaMemcpyHostToDevice,
                               st));



    // tables
    INFFT_TRY(dev_alloc(p, &p->dinv, (size_t)p->M * R_sz));
    INFFT_TRY(dev_alloc(p, &p->tw, (size_t)(Ms / 2) * C_sz));
    const int nt = std::max(p->M, Ms / 2);
    if (p->fp64)
        k_tables<double><<<(nt + 255) / 256, 256, 0, st>>>(p->M, Ms, m, p->window, p->beta, (double*)p->dinv,
                                                          (cx<double>*)p->tw, nullptr);
    else
        k_tables<float><<<(nt + 255) / 256, 256, 0, st>>>(p->M, Ms, m, p->window, p->beta, (float*)p->dinv,
                                                         (cx<float>*)p->tw, nullptr);
    INFFT_LAUNCHED();

    // window polynomials (float32 Kaiser-Bessel plans)
    if (!p->fp64 && p->window == WK_KB && 2 * m + 1 <= 32) {
        INFFT_TRY(dev_alloc(p, (void**)&p->wpoly, (size_t)(WPOLY_DEG + 1) * wpoly_stride(2 * m + 1) * sizeof(float)));
        k_wpoly<<<1, 32, 0, st>>>(m, p->beta, p->wpoly);
        INFFT_LAUNCHED();
        p->wpoly_host.resize((size_t)(WPOLY_DEG + 1) * wpoly_stride(2 * m + 1));
        INFFT_CUDA(cudaMemcpyAsync(p->wpoly_host.data(), p->wpoly, p->wpoly_host.size() * sizeof(float),
                                   cudaMemcpyDeviceToHost, st));
    }

    // scratch
    long long pd = 1, msd_ = 1;
    for (int t = 0; t < d; ++t) { pd *= p->P; msd_ *= Ms; }
    p->scratch_bytes[0] = std::max<size_t>(1, (size_t)p->nitems) * pd * C_sz;
    p->scratch_bytes[1] = (size_t)msd_ * C_sz;
    INFFT_TRY(dev_alloc(p, &p->padded, p->scratch_bytes[0]));
    INFFT_TRY(dev_alloc(p, &p->grid, p->scratch_bytes[1]));
    size_t t1 = 0, t2 = 0;
    if (d >= 2) t1 = (size_t)ipow(Ms, d - 1) * p->M;
    if (d == 3) t2 = (size_t)Ms * p->M * p->M;
    // forward direction uses (M, M, Ms)... sizes: pass0 out Ms*M^(d-1), pass1 out Ms^2*M^(d-2)
    if (d >= 2) t1 = std::max(t1, (size_t)Ms * (size_t)ipow(p->M, d - 1));
    if (d == 3) t2 = std::max(t2, (size_t)Ms * Ms * p->M);
    p->scratch_bytes[2] = t1 * C_sz;
    p->scratch_bytes[3] = t2 * C_sz;
    if (t1) INFFT_TRY(dev_alloc(p, &p->tmp1, t1 * C_sz));
    if (t2) INFFT_TRY(dev_alloc(p, &p->tmp2, t2 * C_sz));
    INFFT_CUDA(cudaStreamSynchronize(st));
    return INFFT_OK;
}

infft_status plan_create(int d, int M, int64_t N, const double* x, double sigma, int m, unsigned flags,
                         cudaStream_t stream, bool pooled, infft_plan_s** out, const infft_tune_t* tune) {
    if (!out) { set_error("out is NULL"); return INFFT_EINVAL; }
    *out = nullptr;
    if (tune && (tune->tile < 0 || tune->item_cap < 0 || tune->branches < 0 || tune->branches > 8 ||
                 tune->prefetch < 0 || tune->prefetch > 2 || tune->fused_fft < 0 || tune->fused_fft > 2)) {
        set_error("invalid tuning (tile %d, item_cap %d, branches %d, prefetch %d, fused_fft %d)", tune->tile,
                  tune->item_cap, tune->branches, tune->prefetch, tune->fused_fft);
        return INFFT_EINVAL;
    }
    if (d < 1 || d > 3 || M < 2 || (M & 1) || N < 1 || N >= (1ll << 31) || !x || !(sigma >= 1.0) || m < 1) {
        set_error("invalid plan arguments (d=%d M=%d N=%lld sigma=%g m=%d)", d, M, (long long)N, sigma, m);
        return INFFT_EINVAL;
    }
    const bool fp64 = (flags & INFFT_FP64) != 0;
    if (((flags & INFFT_FP32) != 0) == fp64) { set_error("exactly one of INFFT_FP32 / INFFT_FP64"); return INFFT_EINVAL; }
    const int Ms = 2 * (int)std::ceil(std::ceil(sigma * M) / 2.0);
    if (2 * m + 2 > Ms) { set_error("2m+2 = %d exceeds M_sigma = %d", 2 * m + 2, Ms); return INFFT_EINVAL; }
    if (!is_pow2(Ms) || Ms > 4096) { set_error("M_sigma = %d must be a power of two <= 4096", Ms); return INFFT_EUNSUPPORTED; }
    if (2 * m > 16 && (flags & INFFT_WIN_BSPLINE)) { set_error("B-spline order 2m > 16"); return INFFT_EUNSUPPORTED; }
    infft_plan_s* p = new infft_plan_s();
    p->d = d; p->M = M; p->Ms = Ms; p->m = m; p->N = N; p->sigma = sigma; p->flags = flags; p->fp64 = fp64;
    p->window = (flags & INFFT_WIN_BSPLINE) ? WK_BSPLINE : ((flags & INFFT_WIN_DIRICHLET) ? WK_DIRICHLET : WK_KB);
    p->beta = M_PI * m * (2.0 - (double)M / Ms);
    int l = 0;
    while ((1 << l) < Ms) ++l;
    p->logMs = l;
    p->pooled = pooled || (flags & INFFT_POOLED) != 0;
    if (tune) p->tune = *tune;
    if (p->tune.tile > 0 && p->tune.tile <= m) {
        set_error("tile edge %d must exceed m = %d", p->tune.tile, m);
        delete p;
        return INFFT_EINVAL;
    }
    p->pool_stream = stream;
    infft_status s = build_plan(p, x, stream);
    if (s != INFFT_OK) { free_plan(p); return s; }
    *out = p;
    return INFFT_OK;
}

}  // namespace infft

using namespace infft;

extern "C" {

const char* infft_last_error(void) { return g_err; }
unsigned int infft_wait_timeouts(void) { return persist_wait_timeouts(); }
uint64_t infft_launch_count(void) { return g_launches; }
void infft_launch_count_reset(void) { g_launches = 0; }

infft_status infft_plan(int d, int M, int64_t N, const double* x, double sigma, int m, unsigned flags, void* stream,
                        infft_plan_t* out) {
    return plan_create(d, M, N, x, sigma, m, flags, (cudaStream_t)stream, false, out);
}

infft_status infft_plan_tuned(int d, int M, int64_t N, const double* x, double sigma, int m, unsigned flags,
                              const infft_tune_t* tune, void* stream, infft_plan_t* out) {
    return plan_create(d, M, N, x, sigma, m, flags, (cudaStream_t)stream, false, out, tune);
}

void infft_inject_faults(unsigned mask) { g_fault_mask.store((int)(mask & 7u), std::memory_order_relaxed); }

void infft_destroy(infft_plan_t p) {
    if (!p) return;
    cudaDeviceSynchronize();
    p->pool_stream = 0;   // pooled memory goes back to the pool; every use has completed
    free_plan(p);
}

#ifdef INFFT_DEBUG
// debug builds only: copy an internal buffer of the plan to host memory
infft_status infft_debug_copy(infft_plan_t p, int which, void* host, size_t bytes) {
    const void* src[] = {p->padded, p->grid, p->items, p->tile_items, p->perm, p->cell, p->u, p->dinv, p->tw,
                         p->cell_start, p->tmp1};
    if (which < 0 || which > 10 || !src[which]) return INFFT_EINVAL;
    cudaDeviceSynchronize();
    INFFT_CUDA(cudaMemcpy(host, src[which], bytes, cudaMemcpyDeviceToHost));
    return INFFT_OK;
}
int infft_debug_info(infft_plan_t p, int which) {
    int v[] = {p->T, p->ntile, p->P, p->nitems, p->S, (int)p->nkeys};
    return v[which];
}
#endif

int64_t infft_plan_N(infft_plan_t p) { return p ? p->N : -1; }
int infft_plan_Msigma(infft_plan_t p) { return p ? p->Ms : -1; }
int infft_plan_work_items(infft_plan_t p) { return p ? p->nitems : -1; }
size_t infft_plan_device_bytes(infft_plan_t p) { return p ? p->device_bytes : 0; }

}  // extern "C"

namespace infft {

infft_status check_mode(const infft_plan_s* p, int mode) {
    if (mode == INFFT_MODE_DCF && !p->has_weights) { set_error("DCF mode needs weights"); return INFFT_ESTATE; }
    if (mode == INFFT_MODE_BOPT && !p->has_bopt) { set_error("BOPT mode needs infft_optimize_B"); return INFFT_ESTATE; }
    if (mode < 0 || mode > 2) { set_error("bad mode %d", mode); return INFFT_EINVAL; }
    if (mode != INFFT_MODE_BOPT && p->window == WK_DIRICHLET) {
        set_error("the Dirichlet window only serves B_opt");
        return INFFT_ESTATE;
    }
    return INFFT_OK;
}

}  // namespace infft

extern "C" {

static size_t coeff_count(const infft_plan_s* p) {
    size_t k = 1;
    for (int t = 0; t < p->d; ++t) k *= (size_t)p->M;
    return k;
}

static infft_status ensure_io(infft_plan_s* p) {
    const size_t C = p->fp64 ? 16 : 8;
    if (!p->io_in) INFFT_TRY(dev_alloc(p, &p->io_in, std::max((size_t)p->N, coeff_count(p)) * C));
    if (!p->io_out) INFFT_TRY(dev_alloc(p, &p->io_out, std::max((size_t)p->N, coeff_count(p)) * C));
    return INFFT_OK;
}

static infft_status transform(infft_plan_t p, int mode, const void* in, void* out, void* stream, bool forward) {
    if (!p || !in || !out) { set_error("null argument"); return INFFT_EINVAL; }
    if (!forward || mode == INFFT_MODE_BOPT) INFFT_TRY(check_mode(p, mode));
    else if (p->window == WK_DIRICHLET) { set_error("no forward NFFT with the Dirichlet window"); return INFFT_ESTATE; }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t C = p->fp64 ? 16 : 8;
    const size_t nin = forward ? coeff_count(p) : (size_t)p->N;
    const size_t nout = forward ? (size_t)p->N : coeff_count(p);
    const bool in_dev = is_device_pointer(in), out_dev = is_device_pointer(out);
    const void* din = in;
    void* dout = out;
    p->pool_stream = st;
    if (!in_dev || !out_dev) INFFT_TRY(ensure_io(p));
    if (!in_dev) {
        INFFT_CUDA(cudaMemcpyAsync(p->io_in, in, nin * C, cudaMemcpyHostToDevice, st));
        din = p->io_in;
    }
    if (!out_dev) dout = p->io_out;
    infft_status s;
    if (p->fp64) {
        std::vector<Job<double>> jobs{make_job<double>(p, mode, din, dout)};
        s = run_jobs<double>(jobs, st, forward);
    } else {
        std::vector<Job<float>> jobs{make_job<float>(p, mode, din, dout)};
        s = run_jobs<float>(jobs, st, forward);
    }
    if (s != INFFT_OK) return s;
    if (!out_dev) {
        INFFT_CUDA(cudaMemcpyAsync(out, dout, nout * C, cudaMemcpyDeviceToHost, st));
        INFFT_CUDA(cudaStreamSynchronize(st));
    }
    return INFFT_OK;
}

infft_status infft_spread_grid(infft_plan_t p, int mode, const void* f, void* grid, void* stream) {
    if (!p || !f || !grid) { set_error("null argument"); return INFFT_EINVAL; }
    INFFT_TRY(check_mode(p, mode));
    if (!is_device_pointer(f) || !is_device_pointer(grid)) {
        set_error("infft_spread_grid: f and grid must be device pointers");
        return INFFT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    p->pool_stream = st;
    if (p->fp64) {
        Job<double> J = make_job<double>(p, mode, f, nullptr);
        J.grid = (cx<double>*)grid;
        return run_spread_grid<double>(J, st);
    }
    Job<float> J = make_job<float>(p, mode, f, nullptr);
    J.grid = (cx<float>*)grid;
    return run_spread_grid<float>(J, st);
}

infft_status infft_fft_axis(infft_plan_t p, int mode, int64_t A, int64_t B, int nblk, const void* in, void* out,
                            void* stream) {
    if (!p || !in || !out) { set_error("null argument"); return INFFT_EINVAL; }
    if (A < 1 || B < 1 || nblk < 1 || p->M % nblk) {
        set_error("infft_fft_axis: A = %lld, B = %lld, nblk = %d (M = %d)", (long long)A, (long long)B, nblk, p->M);
        return INFFT_EINVAL;
    }
    INFFT_TRY(check_mode(p, mode));
    if (!is_device_pointer(in) || !is_device_pointer(out)) {
        set_error("infft_fft_axis: in and out must be device pointers");
        return INFFT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->fp64) {
        Job<double> J = make_job<double>(p, mode, nullptr, out);
        J.grid = (cx<double>*)in;
        return run_fft_axis<double>(J, A, B, nblk, st);
    }
    Job<float> J = make_job<float>(p, mode, nullptr, out);
    J.grid = (cx<float>*)in;
    return run_fft_axis<float>(J, A, B, nblk, st);
}

infft_status infft_adjoint(infft_plan_t p, int mode, const void* f, void* fhat, void* stream) {
    return transform(p, mode, f, fhat, stream, false);
}

infft_status infft_forward(infft_plan_t p, const void* fhat, void* f, void* stream) {
    return transform(p, INFFT_MODE_PLAIN, fhat, f, stream, true);
}

infft_status infft_inverse_adjoint(infft_plan_t p, const void* h, void* f, void* stream) {
    return transform(p, INFFT_MODE_BOPT, h, f, stream, true);
}

static infft_status batched_jobs_check(const infft_plan_t* plans, int count, int mode) {
    if (!plans || count < 1) { set_error("empty batch"); return INFFT_EINVAL; }
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) { set_error("null plan %d", i); return INFFT_EINVAL; }
        if (plans[i]->d != plans[0]->d || plans[i]->fp64 != plans[0]->fp64) {
            set_error("batched plans must share d and precision");
            return INFFT_EINVAL;
        }
        INFFT_TRY(check_mode(plans[i], mode));
    }
    return INFFT_OK;
}

// Scratch slot of every job: the k-th occurrence of a plan in the batch uses slot k
// (slot 0 is the plan's own scratch, slots k >= 1 are allocated here on first need).
// Host buffers are staged through the plan's I/O buffers, so a plan given a host
// pointer may appear only once.  Allocates, so it runs before a graph capture begins.
static infft_status prepare_batched(const infft_plan_t* plans, int count, const void* const* f,
                                    void* const* fhat, const int* slots_in, std::vector<int>& slot,
                                    cudaStream_t st) {
    for (int i = 0; i < count; ++i) plans[i]->pool_stream = st;   // pooled plans allocate in this order
    slot.assign(count, 0);
    for (int i = 0; i < count; ++i) {
        if (slots_in) {
            slot[i] = slots_in[i];
            if (slot[i] < 0 || slot[i] > INFFT_MAX_SCRATCH_SLOT) {
                set_error("scratch slot %d of job %d outside [0, %d]", slot[i], i, INFFT_MAX_SCRATCH_SLOT);
                return INFFT_EINVAL;
            }
            for (int j = 0; j < i; ++j)
                if (plans[j] == plans[i] && slot[j] == slot[i]) {
                    set_error("jobs %d and %d share a plan and scratch slot %d", j, i, slot[i]);
                    return INFFT_EINVAL;
                }
        } else {
            for (int j = 0; j < i; ++j)
                if (plans[j] == plans[i]) slot[i] = std::max(slot[i], slot[j] + 1);
        }
        const bool host = !is_device_pointer(f[i]) || !is_device_pointer(fhat[i]);
        if (host) {
            for (int j = 0; j < count; ++j)
                if (j != i && plans[j] == plans[i]) {
                    set_error("plan of job %d appears more than once and has host buffers", i);
                    return INFFT_EINVAL;
                }
            INFFT_TRY(ensure_io(plans[i]));
        }
        infft_plan_s* p = plans[i];
        if (slot[i] > 0) {   // allocate only the sets that are used
            if ((int)p->extra.size() < slot[i])
                p->extra.resize(slot[i], std::array<void*, 4>{nullptr, nullptr, nullptr, nullptr});
            std::array<void*, 4>& e = p->extra[slot[i] - 1];
            for (int q = 0; q < 4; ++q)
                if (p->scratch_bytes[q] && !e[q]) INFFT_TRY(dev_alloc(p, &e[q], p->scratch_bytes[q]));
        }
    }
    return INFFT_OK;
}

static infft_status run_batched(const infft_plan_t* plans, int count, int mode, const void* const* f,
                                void* const* fhat, cudaStream_t st, cudaEvent_t* ev = nullptr,
                                const int* slots_in = nullptr, bool sync_host = true) {
    std::vector<int> slot;
    INFFT_TRY(prepare_batched(plans, count, f, fhat, slots_in, slot, st));
    std::vector<const void*> fin(count);
    std::vector<void*> fout(count);
    bool any_host_out = false;
    for (int i = 0; i < count; ++i) {
        infft_plan_s* p = plans[i];
        const size_t C = p->fp64 ? 16 : 8;
        fin[i] = f[i];
        fout[i] = fhat[i];
        const bool in_dev = is_device_pointer(f[i]), out_dev = is_device_pointer(fhat[i]);
        if (!in_dev) {
            INFFT_CUDA(cudaMemcpyAsync(p->io_in, f[i], (size_t)p->N * C, cudaMemcpyHostToDevice, st));
            fin[i] = p->io_in;
        }
        if (!out_dev) { fout[i] = p->io_out; any_host_out = true; }
    }
    infft_status s;
    if (plans[0]->fp64) {
        std::vector<Job<double>> jobs;
        for (int i = 0; i < count; ++i) jobs.push_back(make_job<double>(plans[i], mode, fin[i], fout[i], slot[i]));
        s = run_jobs<double>(jobs, st, false, ev);
    } else {
        std::vector<Job<float>> jobs;
        for (int i = 0; i < count; ++i) jobs.push_back(make_job<float>(plans[i], mode, fin[i], fout[i], slot[i]));
        s = run_jobs<float>(jobs, st, false, ev);
    }
    if (s != INFFT_OK) return s;
    if (any_host_out) {
        for (int i = 0; i < count; ++i) {
            if (fout[i] == fhat[i]) continue;
            const size_t C = plans[i]->fp64 ? 16 : 8;
            INFFT_CUDA(cudaMemcpyAsync(fhat[i], fout[i], coeff_count(plans[i]) * C, cudaMemcpyDeviceToHost, st));
        }
        if (sync_host) INFFT_CUDA(cudaStreamSynchronize(st));
    }
    return INFFT_OK;
}

// ----------------------------------------------------------------------------------------
// Branches of a batch.  The jobs are split into G groups of unequal work (shares 1, 2, ..,
// G) that run concurrently on forked streams, so that the latency-bound merge and FFT
// passes (and, with host buffers, the copies) of the smaller groups overlap the spreading
// of the larger ones and the spreads fill each other's tails.  Measured on the batched
// d = 2 workload (graph replay): 1, 2, 3, 4 branches give 71.3k, 76.5k, 77.3k, 76.9k
// reconstructions/s; serialising the spreads across equal groups was slower.  With host
// buffers the copies gain from more branches (end to end 1 / 3 / 6 / 8 branches: 39.8k /
// 53.8k / 57.4k / 63.4k reconstructions/s before later kernel changes), so those calls take 8.
// The environment variable INFFT_BATCH_BRANCHES (1..8) overrides both.
static int branch_count(const infft_plan_t* plans, int count, bool host_buffers = false) {
    int G = host_buffers ? 8 : 3;
    // a plan's tuned count is for device buffers (the copies of host-buffer batches gain from
    // more branches than the kernels alone)
    if (!host_buffers && plans[0]->tune.branches > 0) G = plans[0]->tune.branches;
    else if (const char* env = getenv("INFFT_BATCH_BRANCHES")) G = std::max(1, std::min(8, atoi(env)));
    return std::max(1, std::min(G, count));
}

// Batches that the persistent d = 2 kernel takes (on request, INFFT_PERSISTENT=1) run as a
// whole in one branch: the kernel overlaps the jobs' stages itself (float32, window modes,
// m <= 4, device buffers).  The kernel's launcher makes the final decision and otherwise falls
// back to the staged kernels.
static bool persistent_candidate(const infft_plan_t* plans, int count, int mode) {
    if (mode == INFFT_MODE_BOPT || count > MAXJ) return false;
    const char* e = getenv("INFFT_PERSISTENT");
    if (!e || e[0] != '1') return false;
    for (int i = 0; i < count; ++i) {
        const infft_plan_s* p = plans[i];
        if (p->d != 2 || p->fp64 || p->m > 4 || p->tune.fused_fft == 1) return false;
    }
    return true;
}

static std::vector<std::vector<int>> split_groups(const infft_plan_t* plans, int count, int G) {
    std::vector<std::vector<int>> grp(G);
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int c) { return plans[a]->N > plans[c]->N; });
    std::vector<double> load(G, 0.0);
    for (int i : order) {   // to the group furthest below its share
        int best = 0;
        double bestv = 1e300;
        for (int g = 0; g < G; ++g) {
            const double v = load[g] / (g + 1);
            if (v < bestv) { bestv = v; best = g; }
        }
        grp[best].push_back(i);
        load[best] += (double)plans[i]->N;
    }
    return grp;
}

// forked streams (at the caller's stream priority) and events, kept per host thread
struct BranchSet {
    int dev = -1, prio = 0;
    cudaStream_t s[8] = {};
    cudaEvent_t e[9] = {};
    cudaStream_t cs = nullptr;     // host-input copies
    cudaEvent_t r[9] = {};         // a branch's inputs have arrived; r[8]: all copies issued
};

// Host inputs of a branched batch are copied to the plans' I/O buffers on one copy stream in
// branch order, the smallest branch first, each branch waiting for its own copies only: the
// first branches start computing while the later ones' samples are still arriving (copying
// every branch's inputs at once delayed all of them).  fin[i] becomes the device input of
// job i.  The copy stream is joined back into st.
static infft_status stage_inputs(const infft_plan_t* plans, const std::vector<std::vector<int>>& grp,
                                 const void* const* f, std::vector<const void*>& fin, cudaStream_t st,
                                 cudaStream_t cs, cudaEvent_t fork, const cudaEvent_t* ready, cudaEvent_t done,
                                 const cudaStream_t* br) {
    INFFT_CUDA(cudaStreamWaitEvent(cs, fork, 0));
    for (size_t g = 0; g < grp.size(); ++g) {
        for (int i : grp[g]) {
            if (is_device_pointer(f[i])) continue;
            const size_t C = plans[i]->fp64 ? 16 : 8;
            INFFT_CUDA(cudaMemcpyAsync(plans[i]->io_in, f[i], (size_t)plans[i]->N * C, cudaMemcpyHostToDevice, cs));
            fin[i] = plans[i]->io_in;
        }
        INFFT_CUDA(cudaEventRecord(ready[g], cs));
        INFFT_CUDA(cudaStreamWaitEvent(br[g], ready[g], 0));
    }
    INFFT_CUDA(cudaEventRecord(done, cs));
    INFFT_CUDA(cudaStreamWaitEvent(st, done, 0));
    return INFFT_OK;
}

static infft_status branch_set(cudaStream_t st, BranchSet** out) {
    static thread_local std::vector<BranchSet> sets;
    int dev = 0, prio = 0;
    INFFT_CUDA(cudaGetDevice(&dev));
    if (st) INFFT_CUDA(cudaStreamGetPriority(st, &prio));
    for (auto& b : sets)
        if (b.dev == dev && b.prio == prio) { *out = &b; return INFFT_OK; }
    BranchSet b;
    b.dev = dev;
    b.prio = prio;
    for (int g = 0; g < 8; ++g) INFFT_CUDA(cudaStreamCreateWithPriority(&b.s[g], cudaStreamNonBlocking, prio));
    for (int g = 0; g < 9; ++g) INFFT_CUDA(cudaEventCreateWithFlags(&b.e[g], cudaEventDisableTiming));
    INFFT_CUDA(cudaStreamCreateWithPriority(&b.cs, cudaStreamNonBlocking, prio));
    for (int g = 0; g < 9; ++g) INFFT_CUDA(cudaEventCreateWithFlags(&b.r[g], cudaEventDisableTiming));
    sets.push_back(b);
    *out = &sets.back();
    return INFFT_OK;
}

// one batched adjoint on `st`, its groups on forked branch streams
static infft_status run_branched(const infft_plan_t* plans, int count, int mode, const void* const* f,
                                 void* const* fhat, cudaStream_t st, const int* slots_in) {
    std::vector<int> slot;
    INFFT_TRY(prepare_batched(plans, count, f, fhat, slots_in, slot, st));
    bool host_out = false, host_in = false;
    for (int i = 0; i < count; ++i) {
        host_out = host_out || !is_device_pointer(fhat[i]);
        host_in = host_in || !is_device_pointer(f[i]);
    }
    const bool one = !host_in && !host_out && persistent_candidate(plans, count, mode);
    const int G = one ? 1 : branch_count(plans, count, host_in || host_out);
    if (G == 1 && one) {   // the jobs largest first: the persistent queue's tail is then short
        const std::vector<int> ord = split_groups(plans, count, 1)[0];
        std::vector<infft_plan_t> P;
        std::vector<const void*> F;
        std::vector<void*> H;
        std::vector<int> S;
        for (int i : ord) { P.push_back(plans[i]); F.push_back(f[i]); H.push_back(fhat[i]); S.push_back(slot[i]); }
        return run_batched(P.data(), count, mode, F.data(), H.data(), st, nullptr, S.data());
    }
    if (G == 1) return run_batched(plans, count, mode, f, fhat, st, nullptr, slot.data());
    BranchSet* b = nullptr;
    INFFT_TRY(branch_set(st, &b));
    const std::vector<std::vector<int>> grp = split_groups(plans, count, G);
    INFFT_CUDA(cudaEventRecord(b->e[8], st));
    for (int g = 0; g < G; ++g) INFFT_CUDA(cudaStreamWaitEvent(b->s[g], b->e[8], 0));
    std::vector<const void*> fin(f, f + count);
    if (host_in) INFFT_TRY(stage_inputs(plans, grp, f, fin, st, b->cs, b->e[8], b->r, b->r[8], b->s));
    infft_status s = INFFT_OK;
    for (int g = 0; g < G; ++g) {
        std::vector<infft_plan_t> P;
        std::vector<const void*> F;
        std::vector<void*> H;
        std::vector<int> S;
        for (int i : grp[g]) { P.push_back(plans[i]); F.push_back(fin[i]); H.push_back(fhat[i]); S.push_back(slot[i]); }
        if (!P.empty() && s == INFFT_OK)
            s = run_batched(P.data(), (int)P.size(), mode, F.data(), H.data(), b->s[g], nullptr, S.data(), false);
        INFFT_CUDA(cudaEventRecord(b->e[g], b->s[g]));
        INFFT_CUDA(cudaStreamWaitEvent(st, b->e[g], 0));   // joined even after a failure
    }
    if (s != INFFT_OK) return s;
    if (host_out) INFFT_CUDA(cudaStreamSynchronize(st));
    return INFFT_OK;
}

infft_status infft_adjoint_batched_timed(const infft_plan_t* plans, int count, int mode, const void* const* f,
                                         void* const* fhat, void* stream, float* stage_ms) {
    INFFT_TRY(batched_jobs_check(plans, count, mode));
    if (!f || !fhat || !stage_ms) { set_error("null buffers"); return INFFT_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; ++i) INFFT_CUDA(cudaEventCreate(&ev[i]));
    infft_status s = run_batched(plans, count, mode, f, fhat, st, ev);
    if (s == INFFT_OK) {
        cudaError_t e = cudaEventSynchronize(ev[2 + plans[0]->d]);
        if (e != cudaSuccess) { set_error("event sync: %s", cudaGetErrorString(e)); s = INFFT_ECUDA; }
    }
    if (s == INFFT_OK) {
        for (int k = 0; k < 5; ++k) stage_ms[k] = 0.f;
        cudaEventElapsedTime(&stage_ms[0], ev[0], ev[1]);
        cudaEventElapsedTime(&stage_ms[1], ev[1], ev[2]);
        for (int p = 0; p < plans[0]->d; ++p) cudaEventElapsedTime(&stage_ms[2 + p], ev[2 + p], ev[3 + p]);
    }
    for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
    return s;
}

infft_status infft_adjoint_batched(const infft_plan_t* plans, int count, int mode, const void* const* f,
                                   void* const* fhat, void* stream) {
    INFFT_TRY(batched_jobs_check(plans, count, mode));
    if (!f || !fhat) { set_error("null buffers"); return INFFT_EINVAL; }
    return run_branched(plans, count, mode, f, fhat, (cudaStream_t)stream, nullptr);
}

infft_status infft_adjoint_batched_slots(const infft_plan_t* plans, int count, int mode, const void* const* f,
                                         void* const* fhat, const int* slots, void* stream) {
    INFFT_TRY(batched_jobs_check(plans, count, mode));
    if (!f || !fhat) { set_error("null buffers"); return INFFT_EINVAL; }
    return run_branched(plans, count, mode, f, fhat, (cudaStream_t)stream, slots);
}

}  // extern "C"

// Graph batch over host buffers.  The jobs are ordered by the address of their host input and
// cut into G branches of contiguous runs with work shares 1 : 2 : .. : G (smallest first); each
// branch's inputs are staged into one batch-owned device buffer with one copy per run of
// adjacent host ranges (one per branch when the caller's buffers are slices of one allocation),
// on a copy stream in branch order, and its results come back the same way on the branch's
// stream.  Per-job copies cost a few microseconds each on the copy engines: 128 of them per step
// of the 64-set batch took longer than the transfer itself.
static infft_status batch_create_host(const infft_plan_t* plans, int count, int mode, const void* const* f,
                                      void* const* fhat, const std::vector<int>& slot, int G, infft_batch_t* out) {
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    auto key = [&](int i) -> uintptr_t { return is_device_pointer(f[i]) ? UINTPTR_MAX : (uintptr_t)f[i]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return key(a) < key(c); });
    double total = 0;
    for (int i = 0; i < count; ++i) total += (double)plans[i]->N;
    std::vector<std::vector<int>> grp(G);
    {
        double acc = 0, share = 0;
        int g = 0;
        const double units = (double)G * (G + 1) / 2;
        for (int i : order) {
            while (g < G - 1 && acc >= total * (share + (g + 1)) / units - 1e-9) { share += g + 1; ++g; }
            grp[g].push_back(i);
            acc += (double)plans[i]->N;
        }
    }
    // staging offsets in branch order
    std::vector<size_t> off_in(count, 0), off_out(count, 0);
    size_t bytes_in = 0, bytes_out = 0;
    for (int g = 0; g < G; ++g)
        for (int i : grp[g]) {
            const size_t C = plans[i]->fp64 ? 16 : 8;
            if (!is_device_pointer(f[i])) { off_in[i] = bytes_in; bytes_in += (size_t)plans[i]->N * C; }
            if (!is_device_pointer(fhat[i])) { off_out[i] = bytes_out; bytes_out += coeff_count(plans[i]) * C; }
        }
    infft_batch_s* b = new infft_batch_s();
    if ((bytes_in && cudaMalloc(&b->stage_in, bytes_in) != cudaSuccess) ||
        (bytes_out && cudaMalloc(&b->stage_out, bytes_out) != cudaSuccess)) {
        cudaGetLastError();
        infft_batch_destroy(b);
        set_error("graph batch: out of device memory for %zu + %zu staging bytes", bytes_in, bytes_out);
        return INFFT_ENOMEM;
    }
    unsigned char* sin = (unsigned char*)b->stage_in;
    unsigned char* sout = (unsigned char*)b->stage_out;
    std::vector<const void*> fin(count);
    std::vector<void*> fo(count);
    for (int i = 0; i < count; ++i) {
        fin[i] = is_device_pointer(f[i]) ? f[i] : (const void*)(sin + off_in[i]);
        fo[i] = is_device_pointer(fhat[i]) ? fhat[i] : (void*)(sout + off_out[i]);
    }
    cudaStream_t cap = nullptr, cs = nullptr;
    std::vector<cudaStream_t> br(G, nullptr);
    std::vector<cudaEvent_t> ev(G + 1, nullptr), rd(G + 1, nullptr);
    infft_status s = INFFT_OK;
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && s == INFFT_OK) { set_error("%s: %s", what, cudaGetErrorString(e)); s = INFFT_ECUDA; }
    };
    ck(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "stream");
    ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
    for (int g = 0; g < G; ++g) ck(cudaStreamCreateWithFlags(&br[g], cudaStreamNonBlocking), "stream");
    for (int g = 0; g <= G; ++g) {
        ck(cudaEventCreateWithFlags(&ev[g], cudaEventDisableTiming), "event");
        ck(cudaEventCreateWithFlags(&rd[g], cudaEventDisableTiming), "event");
    }
    cudaError_t e = cudaSuccess;
    if (s == INFFT_OK) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    ck(e, "begin capture");
    if (s == INFFT_OK) {
        ck(cudaEventRecord(ev[G], cap), "record");
        ck(cudaStreamWaitEvent(cs, ev[G], 0), "wait");
        for (int g = 0; g < G; ++g) ck(cudaStreamWaitEvent(br[g], ev[G], 0), "wait");
        // inputs: one copy per run of adjacent host ranges, branch by branch
        for (int g = 0; g < G; ++g) {
            size_t k = 0;
            while (k < grp[g].size()) {
                const int i0 = grp[g][k];
                if (is_device_pointer(f[i0])) { ++k; continue; }
                size_t bytes = (size_t)plans[i0]->N * (plans[i0]->fp64 ? 16 : 8);
                size_t k1 = k + 1;
                while (k1 < grp[g].size()) {
                    const int j = grp[g][k1];
                    if (is_device_pointer(f[j]) || (const unsigned char*)f[j] != (const unsigned char*)f[i0] + bytes ||
                        off_in[j] != off_in[i0] + bytes)
                        break;
                    bytes += (size_t)plans[j]->N * (plans[j]->fp64 ? 16 : 8);
                    ++k1;
                }
                ck(cudaMemcpyAsync(sin + off_in[i0], f[i0], bytes, cudaMemcpyHostToDevice, cs), "input copy");
                k = k1;
            }
            ck(cudaEventRecord(rd[g], cs), "record");
            ck(cudaStreamWaitEvent(br[g], rd[g], 0), "wait");
        }
        ck(cudaEventRecord(rd[G], cs), "record");
        ck(cudaStreamWaitEvent(cap, rd[G], 0), "wait");
        for (int g = 0; g < G; ++g) {
            std::vector<infft_plan_t> P;
            std::vector<const void*> F;
            std::vector<void*> H;
            std::vector<int> S;
            for (int i : grp[g]) { P.push_back(plans[i]); F.push_back(fin[i]); H.push_back(fo[i]); S.push_back(slot[i]); }
            if (!P.empty() && s == INFFT_OK) {
                const infft_status r = run_batched(P.data(), (int)P.size(), mode, F.data(), H.data(), br[g], nullptr,
                                                   S.data(), false);
                if (r != INFFT_OK) s = r;
            }
            // results: one copy per run of adjacent host ranges
            size_t k = 0;
            while (k < grp[g].size() && s == INFFT_OK) {
                const int i0 = grp[g][k];
                if (is_device_pointer(fhat[i0])) { ++k; continue; }
                size_t bytes = coeff_count(plans[i0]) * (plans[i0]->fp64 ? 16 : 8);
                size_t k1 = k + 1;
                while (k1 < grp[g].size()) {
                    const int j = grp[g][k1];
                    if (is_device_pointer(fhat[j]) || (unsigned char*)fhat[j] != (unsigned char*)fhat[i0] + bytes ||
                        off_out[j] != off_out[i0] + bytes)
                        break;
                    bytes += coeff_count(plans[j]) * (plans[j]->fp64 ? 16 : 8);
                    ++k1;
                }
                ck(cudaMemcpyAsync(fhat[i0], sout + off_out[i0], bytes, cudaMemcpyDeviceToHost, br[g]), "result copy");
                k = k1;
            }
            ck(cudaEventRecord(ev[g], br[g]), "record");
            ck(cudaStreamWaitEvent(cap, ev[g], 0), "wait");   // joined even after a failure
        }
        const cudaError_t ee = cudaStreamEndCapture(cap, &b->graph);
        ck(ee, "end capture");
    }
    if (cap) cudaStreamDestroy(cap);
    if (cs) cudaStreamDestroy(cs);
    for (int g = 0; g < G; ++g)
        if (br[g]) cudaStreamDestroy(br[g]);
    for (int g = 0; g <= G; ++g) {
        if (ev[g]) cudaEventDestroy(ev[g]);
        if (rd[g]) cudaEventDestroy(rd[g]);
    }
    if (s == INFFT_OK) ck(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
    if (s != INFFT_OK) {
        infft_batch_destroy(b);
        return s;
    }
    *out = b;
    return INFFT_OK;
}

extern "C" {

infft_status infft_batch_create(const infft_plan_t* plans, int count, int mode, const void* const* f,
                                void* const* fhat, void* stream, infft_batch_t* out) {
    if (!out) { set_error("out is NULL"); return INFFT_EINVAL; }
    *out = nullptr;
    INFFT_TRY(batched_jobs_check(plans, count, mode));
    if (!f || !fhat) { set_error("null buffers"); return INFFT_EINVAL; }
    // scratch sets over the whole batch, allocated outside the capture
    std::vector<int> slot;
    INFFT_TRY(prepare_batched(plans, count, f, fhat, nullptr, slot, (cudaStream_t)stream));
    // device buffers, or page-locked host buffers whose copies the graph then holds
    bool host = false;
    for (int i = 0; i < count; ++i) {
        const bool hi = !is_device_pointer(f[i]), ho = !is_device_pointer(fhat[i]);
        if ((hi && !is_pinned_host_pointer(f[i])) || (ho && !is_pinned_host_pointer(fhat[i]))) {
            set_error("graph batches need device or page-locked host buffers (job %d)", i);
            return INFFT_EINVAL;
        }
        host = host || hi || ho;
    }
    // the jobs in concurrent branches of unequal work, as in run_branched
    const int G = (!host && persistent_candidate(plans, count, mode)) ? 1 : branch_count(plans, count, host);
    if (host) return batch_create_host(plans, count, mode, f, fhat, slot, G, out);
    const std::vector<std::vector<int>> grp = split_groups(plans, count, G);
    bool host_in = false;
    for (int i = 0; i < count; ++i) host_in = host_in || !is_device_pointer(f[i]);
    cudaStream_t cap, cs;
    INFFT_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    INFFT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    std::vector<cudaStream_t> br(G, nullptr);
    std::vector<cudaEvent_t> ev(G + 1, nullptr);       // branch ends, fork
    std::vector<cudaEvent_t> rd(G + 1, nullptr);       // inputs of a branch arrived; all copies issued
    for (int g = 0; g < G; ++g) INFFT_CUDA(cudaStreamCreateWithFlags(&br[g], cudaStreamNonBlocking));
    for (int g = 0; g <= G; ++g) INFFT_CUDA(cudaEventCreateWithFlags(&ev[g], cudaEventDisableTiming));
    for (int g = 0; g <= G; ++g) INFFT_CUDA(cudaEventCreateWithFlags(&rd[g], cudaEventDisableTiming));
    infft_batch_s* b = new infft_batch_s();
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    infft_status s = INFFT_OK;
    if (e != cudaSuccess) {
        set_error("begin capture: %s", cudaGetErrorString(e));
        s = INFFT_ECUDA;
    } else {
        cudaEventRecord(ev[G], cap);
        for (int g = 0; g < G; ++g) cudaStreamWaitEvent(br[g], ev[G], 0);
        std::vector<const void*> fin(f, f + count);
        if (host_in) s = stage_inputs(plans, grp, f, fin, cap, cs, ev[G], rd.data(), rd[G], br.data());
        for (int g = 0; g < G && s == INFFT_OK; ++g) {
            std::vector<infft_plan_t> P;
            std::vector<const void*> F;
            std::vector<void*> H;
            std::vector<int> S;
            for (int i : grp[g]) { P.push_back(plans[i]); F.push_back(fin[i]); H.push_back(fhat[i]); S.push_back(slot[i]); }
            if (!P.empty())
                s = run_batched(P.data(), (int)P.size(), mode, F.data(), H.data(), br[g], nullptr, S.data(), false);
            cudaEventRecord(ev[g], br[g]);
            cudaStreamWaitEvent(cap, ev[g], 0);
        }
        e = cudaStreamEndCapture(cap, &b->graph);
    }
    cudaStreamDestroy(cap);
    cudaStreamDestroy(cs);
    for (int g = 0; g < G; ++g) cudaStreamDestroy(br[g]);
    for (int g = 0; g <= G; ++g) cudaEventDestroy(ev[g]);
    for (int g = 0; g <= G; ++g) cudaEventDestroy(rd[g]);
    if (s != INFFT_OK || e != cudaSuccess) {
        if (s == INFFT_OK) set_error("end capture: %s", cudaGetErrorString(e));
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return s != INFFT_OK ? s : INFFT_ECUDA;
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        set_error("graph instantiate: %s", cudaGetErrorString(e));
        cudaGraphDestroy(b->graph);
        delete b;
        return INFFT_ECUDA;
    }
    (void)stream;
    *out = b;
    return INFFT_OK;
}

infft_status infft_batch_run(infft_batch_t b, void* stream) {
    if (!b) { set_error("null batch"); return INFFT_EINVAL; }
    INFFT_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    count_launch();
    return INFFT_OK;
}

void infft_batch_destroy(infft_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->stage_in) cudaFree(b->stage_in);
    if (b->stage_out) cudaFree(b->stage_out);
    delete b;
}

}  // extern "C"
