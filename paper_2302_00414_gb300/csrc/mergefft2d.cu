// Halo merge and the pruned two-dimensional FFT with deconvolution (Algorithm 2.4 steps
// 2 and 3, d = 2) fused into one thread-block-cluster kernel per grid size.
//
// One cluster of CS CTAs reconstructs one job.  CTA `rank` owns the band of Ms/CS grid
// rows starting at rank * Ms/CS (a whole number of tile rows):
//   1. it sums the padded tiles written by the spread straight into its rows in shared
//      memory, at bit-reversed positions along x (no grid in global memory); the tiles
//      are taken in four phases by the parity of their tile row and column, so that
//      tiles added at the same time never overlap and every cell receives its
//      contributions in one fixed order (deterministic sums);
//   2. it transforms its rows (forward DFT along x), keeps the M frequencies of I_M and
//      multiplies by 1/(Ms w^(k_1)), into a compact M-wide copy of its rows;
//   3. after a cluster barrier it reads its M/CS columns of that compact array from all
//      CTAs of the cluster through distributed shared memory, transforms them along y,
//      keeps I_M, multiplies by 1/(Ms w^(k_0)) and writes its columns of fhat.
// Global memory sees the padded tiles once and fhat once: the grid and the intermediate
// of the two-pass form never leave the chip.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <vector>

#include "internal.h"
#include "jobset.cuh"
#include "spread.cuh"

namespace cg = cooperative_groups;

namespace infft {

struct JobSel {
    int n;
    int job[MAXJ];
};

constexpr int MF_THREADS = 512;

__device__ __forceinline__ int mf_skew(int i) { return i + (i >> 4); }

// In-place decimation-in-time FFT (sign -) of nl lines of length n = 2^logn held in shared
// memory in bit-reversed order: line l at buf + l * ls, element i at mf_skew(i).  Radix-4
// steps (two radix-2 stages per thread in registers), one radix-2 stage first when logn is
// odd.  tws: the n/2 twiddles exp(-2 pi i k / n).  Ends with a block barrier.
template <class R>
__device__ void mf_fft_lines(cx<R>* buf, int nl, int ls, int n, int logn, const cx<R>* tws) {
    const int tid = threadIdx.x, nth = blockDim.x;
    int lh = 0;
    if (logn & 1) {
        const int half_n = n >> 1, loghn = logn - 1;
        for (int e = tid; e < nl * half_n; e += nth) {
            const int l = e >> loghn, jj = e & (half_n - 1);
            cx<R>* row = buf + (size_t)l * ls;
            const cx<R> a = row[mf_skew(2 * jj)], b = row[mf_skew(2 * jj + 1)];
            row[mf_skew(2 * jj)] = add(a, b);
            row[mf_skew(2 * jj + 1)] = sub(a, b);
        }
        __syncthreads();
        lh = 1;
    }
    const int quarter_n = n >> 2, logqn = logn - 2;
    for (; lh < logn; lh += 2) {
        const int q = 1 << lh;
        for (int e = tid; e < nl * quarter_n; e += nth) {
            const int l = e >> logqn, jj = e & (quarter_n - 1);
            const int grp = jj >> lh, pos = jj & (q - 1);
            const int base = grp * (q << 2) + pos;
            cx<R>* row = buf + (size_t)l * ls;
            const cx<R> a0 = row[mf_skew(base)], a1 = row[mf_skew(base + q)];
            const cx<R> a2 = row[mf_skew(base + 2 * q)], a3 = row[mf_skew(base + 3 * q)];
            const cx<R> w1 = tws[pos << (logn - 1 - lh)];
            const cx<R> w2 = tws[pos << (logn - 2 - lh)];
            const cx<R> w3 = tws[(pos + q) << (logn - 2 - lh)];
            cx<R> t = mul(w1, a1);
            const cx<R> b0 = add(a0, t), b1 = sub(a0, t);
            t = mul(w1, a3);
            const cx<R> b2 = add(a2, t), b3 = sub(a2, t);
            t = mul(w2, b2);
            row[mf_skew(base)] = add(b0, t);
            row[mf_skew(base + 2 * q)] = sub(b0, t);
            t = mul(w3, b3);
            row[mf_skew(base + q)] = add(b1, t);
            row[mf_skew(base + 3 * q)] = sub(b1, t);
        }
        __syncthreads();
    }
}

// shared-memory layout of one CTA (sizes in elements)
struct MfLayout {
    int RB, ns, CW, cs;          // rows per CTA, row stride, columns per CTA, column stride
    size_t rc, cmp, tw;          // row / column region, compact rows, twiddles (complex)
    int NR;                      // contributing tile rows
    size_t bytes;
};

template <class R>
__host__ __device__ inline MfLayout mf_layout(int Ms, int M, int nt, int T, int CS) {
    MfLayout L;
    L.RB = Ms / CS;
    L.ns = Ms + (Ms >> 4);
    L.CW = M / CS;
    L.cs = L.ns + 1;             // odd stride in 8-byte words: column gathers spread over banks
    const size_t rows = (size_t)L.RB * L.ns, cols = (size_t)L.CW * L.cs;
    L.rc = rows > cols ? rows : cols;
    L.cmp = (size_t)L.RB * M;
    L.tw = (size_t)(Ms / 2);
    L.NR = CS == 1 ? nt : L.RB / T + 2;
    L.bytes = (L.rc + L.cmp + L.tw) * sizeof(cx<R>) + (size_t)M * sizeof(R) + (size_t)L.NR * (nt + 1) * sizeof(int) +
              64;
    return L;
}

template <class R, int CS>
__global__ void __launch_bounds__(MF_THREADS, 1) k_mergefft2d(const __grid_constant__ JobSet<R> js,
                                                              const __grid_constant__ JobSel sel) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rank = CS == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const Job<R>& J = js.job[sel.job[blockIdx.x / CS]];
    const int Ms = J.Ms, M = J.M, T = J.T, m = J.m, P = J.P, nt = J.ntile;
    const int logn = 31 - __clz(Ms);
    const MfLayout Lo = mf_layout<R>(Ms, M, nt, T, CS);
    const int RB = Lo.RB, ns = Lo.ns, CW = Lo.CW, cs = Lo.cs, NR = Lo.NR;
    const int y0 = rank * RB, c0 = rank * CW;
    cx<R>* rc = reinterpret_cast<cx<R>*>(smem_raw);       // rows RB x ns, later columns CW x cs
    cx<R>* cmp = rc + Lo.rc;                               // compact rows RB x M
    cx<R>* tws = cmp + Lo.cmp;                             // Ms/2 twiddles
    R* dv = reinterpret_cast<R*>(tws + Lo.tw);             // M deconvolution factors
    int* titem = reinterpret_cast<int*>(dv + M);           // NR x (nt + 1) item prefix per tile row
    const int tid = threadIdx.x, nth = blockDim.x;
    const int ty_first = CS == 1 ? 0 : y0 / T - 1;        // unwrapped tile row of contributing row 0

    for (int k = tid; k < (Ms >> 1); k += nth) tws[k] = J.tw[k];
    for (int k = tid; k < M; k += nth) dv[k] = J.dinv[k];
    for (int e = tid; e < NR * (nt + 1); e += nth) {
        const int r = e / (nt + 1), tx = e - r * (nt + 1);
        const int ty = mod_pos(ty_first + r, nt);
        titem[e] = J.tile_items[ty * nt + tx];   // tiles are numbered row-major: a row's prefix is contiguous
    }
    __syncthreads();

    // 1. every cell of the band: the sum of the padded-tile cells that map onto it, taken in
    //    the order of the two-kernel form's merge (along y the own tile, then the neighbour
    //    whose padded edge reaches the cell; the same along x; a tile's work items in order),
    //    stored at its bit-reversed position along x.  Along an axis a cell at offset r of
    //    tile t lies in tile t at r + m, and in tile t - 1 at r + T + m when that is < P or
    //    in tile t + 1 at r - T + m when that is >= 0 (at most one neighbour, as P <= 2T).
    //    Each thread takes four cells at a time and issues the loads of their first items
    //    together.
    const size_t PP = (size_t)P * P;
    const int logT = 31 - __clz(T);
    const int ncell = RB * Ms;
    constexpr int U = 4;
    for (int e0 = tid; e0 < ncell; e0 += U * nth) {
        int it0[U][4], offn[U][4];     // per cell and source: first work item; offset | count << 12
        cx<R> v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nth;
#pragma unroll
            for (int q = 0; q < 4; ++q) { it0[u][q] = 0; offn[u][q] = 0; }
            if (e >= ncell) continue;
            const int y = y0 + (e >> logn), x = e & (Ms - 1);
            const int ry = y & (T - 1), rx = x & (T - 1);
            int yr[2], yo[2], xt[2], xo[2];
            int ny = 1, nx = 1;
            yr[0] = (y >> logT) - ty_first;            // contributing tile row (unwrapped index)
            yo[0] = ry + m;
            if (ry + T + m < P) { yr[1] = yr[0] - 1; yo[1] = ry + T + m; ny = 2; }
            else if (ry - T + m >= 0) { yr[1] = yr[0] + 1; yo[1] = ry - T + m; ny = 2; }
            xt[0] = x >> logT;
            xo[0] = rx + m;
            if (rx + T + m < P) { xt[1] = mod_pos(xt[0] - 1, nt); xo[1] = rx + T + m; nx = 2; }
            else if (rx - T + m >= 0) { xt[1] = mod_pos(xt[0] + 1, nt); xo[1] = rx - T + m; nx = 2; }
#pragma unroll
            for (int a = 0; a < 2; ++a) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    if (a >= ny || b >= nx) continue;
                    const int r = CS == 1 ? mod_pos(yr[a], nt) : yr[a];
                    const int* ti = titem + r * (nt + 1) + xt[b];
                    it0[u][2 * a + b] = ti[0];
                    offn[u][2 * a + b] = (yo[a] * P + xo[b]) | ((ti[1] - ti[0]) << 12);
                }
            }
        }
        // the first work item of every source of the four cells, loads issued together
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[u][q] = (offn[u][q] >> 12) > 0 ? J.padded[(size_t)it0[u][q] * PP + (offn[u][q] & 4095)] : mk<R>(0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nth;
            if (e >= ncell) continue;
            cx<R> acc = mk<R>(0, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int n = offn[u][q] >> 12;
                if (n <= 0) continue;
                acc = add(acc, v[u][q]);
                for (int k = 1; k < n; ++k)     // further work items of a tile with many points
                    acc = add(acc, J.padded[(size_t)(it0[u][q] + k) * PP + (offn[u][q] & 4095)]);
            }
            rc[(e >> logn) * ns + mf_skew(bitrev(e & (Ms - 1), logn))] = acc;
        }
    }
    __syncthreads();

    // 2. row FFTs, crop to I_M, deconvolve along x, into the compact rows
    mf_fft_lines<R>(rc, RB, ns, Ms, logn, tws);
    for (int e = tid; e < RB * M; e += nth) {
        const int yl = e / M, i = e - yl * M;
        cmp[e] = scale(rc[yl * ns + mf_skew(mod_pos(i - M / 2, Ms))], dv[i]);
    }

    // 3. gather this CTA's columns from every CTA of the cluster, column FFTs, crop, deconvolve
    if constexpr (CS > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        for (int e = tid; e < Ms * CW; e += nth) {
            const int y = e / CW, kk = e - y * CW;
            const cx<R>* src = cl.map_shared_rank(cmp, y / RB);
            rc[kk * cs + mf_skew(bitrev(y, logn))] = src[(y % RB) * M + c0 + kk];
        }
        cl.sync();   // every remote read is done before any CTA goes on (or exits)
    } else {
        __syncthreads();
        for (int e = tid; e < Ms * CW; e += nth) {
            const int y = e / CW, kk = e - y * CW;
            rc[kk * cs + mf_skew(bitrev(y, logn))] = cmp[y * M + kk];
        }
        __syncthreads();
    }
    mf_fft_lines<R>(rc, CW, cs, Ms, logn, tws);
    for (int e = tid; e < M * CW; e += nth) {
        const int k0 = e / CW, kk = e - k0 * CW;
        J.out[(size_t)k0 * M + c0 + kk] = scale(rc[kk * cs + mf_skew(mod_pos(k0 - M / 2, Ms))], dv[k0]);
    }
}

// cluster size for a grid: the smallest power of two whose per-CTA share fits in shared
// memory (two CTAs per SM where a cluster of at most 8 allows it), the band a whole
// number of 16-row tile rows, at most 16 CTAs; 0 when the grid is not taken
template <class R>
static int mf_cluster_size(const Job<R>& J, size_t smem_cap) {
    if (J.d != 2 || (J.T != 16 && J.T != 8) || J.Ms < 64 || J.ntile < 4 || J.P > 2 * J.T ||
        J.ntile * J.T != J.Ms)
        return 0;
    for (int CS = 1; CS <= 16; CS *= 2) {
        if (J.Ms / CS < J.T || (J.Ms / CS) % J.T || J.M % CS) return 0;
        const MfLayout Lo = mf_layout<R>(J.Ms, J.M, J.ntile, J.T, CS);
        const size_t b = Lo.bytes;
        if (b <= smem_cap / 2 || (b <= smem_cap && CS >= 8) || (b <= smem_cap && CS == 16)) return CS;
    }
    return 0;
}

template <class R, int CS>
static infft_status mf_launch(const JobSet<R>& js, const JobSel& sel, size_t smem, cudaStream_t st, bool* ok) {
    *ok = false;
    auto kern = k_mergefft2d<R, CS>;
    INFFT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (CS > 8) INFFT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sel.n * CS));
    cfg.blockDim = dim3(MF_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return INFFT_OK;   // not schedulable here: the caller keeps the two-kernel form
    }
    INFFT_CUDA(cudaLaunchKernelEx(&cfg, kern, js, sel));
    INFFT_LAUNCHED();
    *ok = true;
    return INFFT_OK;
}

// forked streams (at the caller's stream priority) and events for the grid-size groups,
// kept per host thread
struct MfStreams {
    int dev = -1, prio = 0;
    cudaStream_t s[8] = {};
    cudaEvent_t e[9] = {};
};

static infft_status mf_streams(cudaStream_t st, MfStreams** out) {
    static thread_local std::vector<MfStreams> sets;
    int dev = 0, prio = 0;
    INFFT_CUDA(cudaGetDevice(&dev));
    if (st) INFFT_CUDA(cudaStreamGetPriority(st, &prio));
    for (auto& b : sets)
        if (b.dev == dev && b.prio == prio) { *out = &b; return INFFT_OK; }
    MfStreams b;
    b.dev = dev;
    b.prio = prio;
    for (int g = 0; g < 8; ++g) INFFT_CUDA(cudaStreamCreateWithPriority(&b.s[g], cudaStreamNonBlocking, prio));
    for (int g = 0; g < 9; ++g) INFFT_CUDA(cudaEventCreateWithFlags(&b.e[g], cudaEventDisableTiming));
    sets.push_back(b);
    *out = &sets.back();
    return INFFT_OK;
}

// Launch the fused merge + FFT for every job of js whose grid it takes (grouped by grid
// size, one launch per group); `rest` receives the indices of the other jobs.
// Off by default: a plan's tuning (fused_fft = 1) or INFFT_FUSED_MERGE_FFT=1 turns it on.
template <class R>
infft_status mergefft2d_try(const JobSet<R>& js, cudaStream_t st, std::vector<int>& rest) {
    rest.clear();
    const int env = env_form("INFFT_FUSED_MERGE_FFT");
    int dev = 0, optin = 0;
    INFFT_CUDA(cudaGetDevice(&dev));
    INFFT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    std::map<long long, std::vector<int>> groups;   // (cluster size, tile, Ms) -> jobs
    for (int j = 0; j < js.njobs; ++j) {
        // off unless the plan's tuning or the environment turns it on
        const int want = js.job[j].fused_fft == 1 ? 1 : js.job[j].fused_fft == 2 ? 0 : (env == 1 ? 1 : 0);
        const int CS = want == 0 ? 0 : mf_cluster_size<R>(js.job[j], (size_t)optin);
        if (CS == 0) rest.push_back(j);
        else groups[((long long)CS * 64 + js.job[j].T) * 65536 + js.job[j].Ms].push_back(j);
    }
    // the groups run concurrently on streams forked from st (a group of small grids alone
    // fills few SMs); up to eight groups, any further ones on the eighth stream
    MfStreams* fs = nullptr;
    const bool fork = groups.size() > 1;
    if (fork) {
        INFFT_TRY(mf_streams(st, &fs));
        INFFT_CUDA(cudaEventRecord(fs->e[8], st));
        for (int g = 0; g < 8; ++g) INFFT_CUDA(cudaStreamWaitEvent(fs->s[g], fs->e[8], 0));
    }
    int gi = 0;
    infft_status status = INFFT_OK;
    for (auto& g : groups) {
        const int CS = (int)(g.first / 65536 / 64);
        cudaStream_t gs = fork ? fs->s[std::min(gi, 7)] : st;
        ++gi;
        JobSel sel;
        sel.n = (int)g.second.size();
        for (int i = 0; i < sel.n; ++i) sel.job[i] = g.second[i];
        const Job<R>& J0 = js.job[g.second[0]];
        const size_t smem = mf_layout<R>(J0.Ms, J0.M, J0.ntile, J0.T, CS).bytes;
        bool ok = false;
        switch (CS) {
            case 1: status = mf_launch<R, 1>(js, sel, smem, gs, &ok); break;
            case 2: status = mf_launch<R, 2>(js, sel, smem, gs, &ok); break;
            case 4: status = mf_launch<R, 4>(js, sel, smem, gs, &ok); break;
            case 8: status = mf_launch<R, 8>(js, sel, smem, gs, &ok); break;
            default: status = mf_launch<R, 16>(js, sel, smem, gs, &ok); break;
        }
        if (status != INFFT_OK) break;
        if (!ok) rest.insert(rest.end(), g.second.begin(), g.second.end());
    }
    if (fork) {   // joined even after a failure
        for (int g = 0; g < 8; ++g) {
            INFFT_CUDA(cudaEventRecord(fs->e[g], fs->s[g]));
            INFFT_CUDA(cudaStreamWaitEvent(st, fs->e[g], 0));
        }
    }
    if (status != INFFT_OK) return status;
    std::sort(rest.begin(), rest.end());
    return INFFT_OK;
}

template infft_status mergefft2d_try<float>(const JobSet<float>&, cudaStream_t, std::vector<int>&);
template infft_status mergefft2d_try<double>(const JobSet<double>&, cudaStream_t, std::vector<int>&);

}  // namespace infft
