// NFFT kernels: tile-sorted spreading (Algorithm 2.4 step 1, and its modified
// forms of Algorithm 3.7 / 4.4), halo merge, d-variate FFT passes with pruned
// output and per-axis deconvolution (Algorithm 2.4 steps 2-3), zero-padded
// inverse FFT passes (Algorithm 2.1 steps 1-2) and tile-sorted interpolation
// (Algorithm 2.1 step 3).
#include <algorithm>
#include <memory>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "jobset.cuh"
#include "spread.cuh"
#include "fft.cuh"

namespace infft {

// ---------------------------------------------------------------------------------------
// spreading: one warp per work item (a tile of T^d grid cells and up to a fixed number of
// its points).  The warp accumulates into a private padded tile of P^d cells in shared
// memory (P = T + 2m + 1 covers every tap of every point whose base cell lies in the
// tile), one point at a time with the lanes over the point's taps, so that no two lanes
// touch the same cell in one step: no atomics, fixed summation order.  The padded tile
// is then written out for the merge.
template <class R, int D>
__global__ void __launch_bounds__(128) k_spread(const __grid_constant__ JobSet<R> js) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gitem = blockIdx.x * js.wpb + warp;
    if (gitem >= js.pre_items[js.njobs]) return;
    const int jb = find_job(js.pre_items, js.njobs, gitem);
    const Job<R>& J = js.job[jb];
    const int it = gitem - js.pre_items[jb];
    const int4 item = J.items[it];
    const int P = J.P, m = J.m, Ms = J.Ms, T = J.T;
    const int W = 2 * m + 1;
    const bool bopt = (J.mode == INFFT_MODE_BOPT);
    const int S = bopt ? J.S : W;           // taps per axis
    const int cells = ipow(P, D);

    unsigned char* base = smem_raw + (size_t)warp * js.smem_per_warp;
    cx<R>* pad = reinterpret_cast<cx<R>*>(base);
    R* psi = reinterpret_cast<R*>(pad + cells);           // [32][D][W]
    cx<R>* cst = reinterpret_cast<cx<R>*>(psi + 32 * D * W);  // [32]
    int* ost = reinterpret_cast<int*>(cst + 32);          // [32][D+1]

    for (int e = lane; e < cells; e += 32) pad[e] = mk<R>(0, 0);

    int tt[D];
    {
        int rem = item.x;
        for (int t = D - 1; t >= 0; --t) { tt[t] = rem % J.ntile; rem /= J.ntile; }
    }
    int pstride[D];
    pstride[D - 1] = 1;
    for (int t = D - 2; t >= 0; --t) pstride[t] = pstride[t + 1] * P;
    int ntap = ipow(S, D);
    __syncwarp();

    for (int c0 = 0; c0 < item.z; c0 += 32) {
        const int np = min(32, item.z - c0);
        if (lane < np) {
            const int i = item.y + c0 + lane;
            const int j = __ldg(J.perm + i);
            cx<R> fv = J.in[j];
            if (J.mode == INFFT_MODE_DCF) fv = mul(J.w[i], fv);
            uint32_t rem = __ldg(J.cell + i);
            for (int t = D - 1; t >= 0; --t) {
                int c = (int)(rem % (uint32_t)Ms);
                rem /= (uint32_t)Ms;
                ost[lane * (D + 1) + t] = c - tt[t] * T;
            }
            ost[lane * (D + 1) + D] = i;
            cst[lane] = fv;
            if (!bopt) {
                for (int t = 0; t < D; ++t) {
                    const R u = J.u[(size_t)i * D + t];
                    for (int s = 0; s < W; ++s)
                        psi[(lane * D + t) * W + s] = tap_weight<R>(J.window, u, s, m, J.inv_m, J.beta);
                }
            }
        }
        __syncwarp();
        for (int p = 0; p < np; ++p) {
            const cx<R> cv = cst[p];
            int o[D];
            for (int t = 0; t < D; ++t) o[t] = ost[p * (D + 1) + t];
            const int i = ost[p * (D + 1) + D];
            const R* ps = psi + p * D * W;
            for (int q = lane; q < ntap; q += 32) {
                int rem = q, idx = 0;
                R wgt = R(1);
                for (int t = D - 1; t >= 0; --t) {
                    const int s = rem % S;
                    rem /= S;
                    idx += (o[t] + s) * pstride[t];
                    if (!bopt) wgt *= ps[t * W + s];
                }
                cx<R> add_v;
                if (bopt) add_v = mulconj(J.coef[(size_t)i * ntap + q], cv);  // conj(b_{j,l}) f_j
                else add_v = scale(cv, wgt);
                pad[idx] = add(pad[idx], add_v);
            }
            __syncwarp();
        }
    }
    cx<R>* dst = J.padded + (size_t)it * cells;
    for (int e = lane; e < cells; e += 32) dst[e] = pad[e];
}

template <class R, int D>
__device__ __forceinline__ cx<R> merged_cell(const Job<R>& J, long long cidx);

// ---------------------------------------------------------------------------------------
// Two-dimensional merge, one block per tile of T x T cells (T <= 16, T > m, Ms a multiple
// of T), one thread per cell.  Along an axis, the cell at offset r in tile t lies in the
// padded tile of t at r + m, of t - 1 at r + T + m when that is < P, and of t + 1 at
// r - T + m when that is >= 0 (tile indices mod ntile): with 2m < T at most two sources
// per axis.
template <class R>
__global__ void __launch_bounds__(256) k_merge2d(const __grid_constant__ JobSet<R> js) {
    const int gblk = blockIdx.x;
    const int jb = find_job(js.pre_merge, js.njobs, gblk);
    const Job<R>& J = js.job[jb];
    const int T = J.T, m = J.m, P = J.P, nt = J.ntile, Ms = J.Ms;
    const int tile = gblk - js.pre_merge[jb];
    const int ty = tile / nt, tx = tile - ty * nt;
    // work-item ranges of the 3 x 3 tiles around this one, read once per block, so that each
    // thread's loads of the padded cells do not wait on a load of the item prefix
    __shared__ int s_i0[9], s_i1[9];
    if (threadIdx.x < 9) {
        const int dy = (int)threadIdx.x / 3 - 1, dx = (int)threadIdx.x % 3 - 1;
        const int tl = mod_pos(ty + dy, nt) * nt + mod_pos(tx + dx, nt);
        s_i0[threadIdx.x] = J.tile_items[tl];
        s_i1[threadIdx.x] = J.tile_items[tl + 1];
    }
    __syncthreads();
    const int r = threadIdx.x >> 4, c = threadIdx.x & 15;
    if (r >= T || c >= T) return;
    int yd[2], yo[2], xd[2], xo[2];   // tile offsets (-1, 0, +1) and padded offsets per axis
    int ny = 1, nx = 1;
    yd[0] = 0; yo[0] = r + m;
    xd[0] = 0; xo[0] = c + m;
    if (r + T + m < P) { yd[1] = -1; yo[1] = r + T + m; ny = 2; }
    else if (r - T + m >= 0) { yd[1] = 1; yo[1] = r - T + m; ny = 2; }
    if (c + T + m < P) { xd[1] = -1; xo[1] = c + T + m; nx = 2; }
    else if (c - T + m >= 0) { xd[1] = 1; xo[1] = c - T + m; nx = 2; }
    const size_t cells = (size_t)P * P;
    // the first item of every source, loaded together; then the sum in source order
    int i0[4], n[4];
    size_t off[4];
    cx<R> v[4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int q = 2 * a + b;
            n[q] = 0;
            off[q] = 0;
            i0[q] = 0;
            if (a < ny && b < nx) {
                const int k = (yd[a] + 1) * 3 + xd[b] + 1;
                i0[q] = s_i0[k];
                n[q] = s_i1[k] - s_i0[k];
                off[q] = (size_t)yo[a] * P + xo[b];
            }
        }
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = n[q] > 0 ? J.padded[(size_t)i0[q] * cells + off[q]] : mk<R>(0, 0);
    cx<R> acc = mk<R>(0, 0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (n[q] <= 0) continue;
        acc = add(acc, v[q]);
        for (int k = 1; k < n[q]; ++k) acc = add(acc, J.padded[(size_t)(i0[q] + k) * cells + off[q]]);
    }
    J.grid[(size_t)(ty * T + r) * Ms + tx * T + c] = acc;
}

// ---------------------------------------------------------------------------------------
// Three-dimensional merge, one block per tile of T^3 cells (T a power of two, m < T),
// threads striding over the tile's cells.  Along an axis the cell at offset r of tile t
// lies in the padded tile of t at r + m, of t - 1 at r + T + m when that is < P, and of
// t + 1 at r - T + m when that is >= 0; with T <= 2m both neighbours can hold it.  Work items of
// a source tile are summed in item order, sources in a fixed order: deterministic.
template <class R>
__global__ void __launch_bounds__(256) k_merge3d(const __grid_constant__ JobSet<R> js) {
    const int gblk = blockIdx.x;
    const int jb = find_job(js.pre_merge, js.njobs, gblk);
    const Job<R>& J = js.job[jb];
    const int T = J.T, m = J.m, P = J.P, nt = J.ntile, Ms = J.Ms;
    const int tile = gblk - js.pre_merge[jb];
    const int tz = tile / (nt * nt), ty = (tile / nt) % nt, tx = tile % nt;
    const int logT = 31 - __clz(T);
    const size_t cells = (size_t)P * P * P;
    for (int e = threadIdx.x; e < T * T * T; e += blockDim.x) {
        const int rz = e >> (2 * logT), ry = (e >> logT) & (T - 1), rx = e & (T - 1);
        const int rr[3] = {rz, ry, rx}, tt[3] = {tz, ty, tx};
        int st[3][3], so[3][3], ns[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int r = rr[a], t = tt[a];
            st[a][0] = t; so[a][0] = r + m; ns[a] = 1;
            if (r + T + m < P) { st[a][ns[a]] = (t - 1 + nt) % nt; so[a][ns[a]] = r + T + m; ++ns[a]; }
            if (r - T + m >= 0) { st[a][ns[a]] = (t + 1) % nt; so[a][ns[a]] = r - T + m; ++ns[a]; }
        }
        cx<R> acc = mk<R>(0, 0);
        for (int a = 0; a < ns[0]; ++a)
            for (int b = 0; b < ns[1]; ++b)
                for (int c = 0; c < ns[2]; ++c) {
                    const int tl = (st[0][a] * nt + st[1][b]) * nt + st[2][c];
                    const int i0 = __ldg(J.tile_items + tl), i1 = __ldg(J.tile_items + tl + 1);
                    const size_t off = ((size_t)so[0][a] * P + so[1][b]) * P + so[2][c];
#pragma unroll 4
                    for (int itm = i0; itm < i1; ++itm) acc = add(acc, J.padded[(size_t)itm * cells + off]);
                }
        J.grid[((size_t)(tz * T + rz) * Ms + ty * T + ry) * Ms + tx * T + rx] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// merge: grid cell c receives the sum of every padded-tile cell that maps onto it
// (padded cell o of tile tl along an axis sits at (tl T - m + o) mod Ms).  One thread per
// grid cell, work items of a tile summed in item order: deterministic.
template <class R, int D>
__global__ void __launch_bounds__(256) k_merge(const __grid_constant__ JobSet<R> js) {
    const int gblk = blockIdx.x;
    const int jb = find_job(js.pre_merge, js.njobs, gblk);
    const Job<R>& J = js.job[jb];
    const int Ms = J.Ms, T = J.T, m = J.m, P = J.P, nt = J.ntile;
    const long long total = (long long)ipow(Ms, D);
    const long long cidx = (long long)(gblk - js.pre_merge[jb]) * blockDim.x + threadIdx.x;
    if (cidx >= total) return;
    J.grid[cidx] = merged_cell<R, D>(J, cidx);
}

// Sum of every padded-tile cell that maps onto grid cell `cidx` (row-major over Ms^D).
template <class R, int D>
__device__ __forceinline__ cx<R> merged_cell(const Job<R>& J, long long cidx) {
    const int Ms = J.Ms, T = J.T, m = J.m, P = J.P, nt = J.ntile;
    int c[D];
    {
        long long rem = cidx;
        for (int t = D - 1; t >= 0; --t) { c[t] = (int)(rem % Ms); rem /= Ms; }
    }
    int cnt[D], tl[D][8], of[D][8];
    for (int t = 0; t < D; ++t) {
        cnt[t] = 0;
        const int own = c[t] / T;
        const int ncand = nt >= 3 ? 3 : nt;
        for (int k = 0; k < ncand; ++k) {
            const int tile = (nt >= 3) ? mod_pos(own - 1 + k, nt) : k;
            int o = mod_pos(c[t] - tile * T + m, Ms);
            for (; o < P && cnt[t] < 8; o += Ms) {
                tl[t][cnt[t]] = tile;
                of[t][cnt[t]] = o;
                ++cnt[t];
            }
        }
    }
    const int cells = ipow(P, D);
    cx<R> acc = mk<R>(0, 0);
    int idx[D];
    for (int t = 0; t < D; ++t) idx[t] = 0;
    bool any = true;
    for (int t = 0; t < D; ++t) any = any && cnt[t] > 0;
    while (any) {
        int tile_lin = 0, pidx = 0;
        for (int t = 0; t < D; ++t) {
            tile_lin = tile_lin * nt + tl[t][idx[t]];
            pidx = pidx * P + of[t][idx[t]];
        }
        const int i0 = __ldg(J.tile_items + tile_lin), i1 = __ldg(J.tile_items + tile_lin + 1);
        for (int itm = i0; itm < i1; ++itm) acc = add(acc, J.padded[(size_t)itm * cells + pidx]);
        int t = D - 1;
        while (t >= 0) {
            if (++idx[t] < cnt[t]) break;
            idx[t] = 0;
            --t;
        }
        if (t < 0) break;
    }
    return acc;
}

// ---------------------------------------------------------------------------------------
// float32 forms bounded to the register counts they reach unbounded as separate kernels (40,
// 48): six (five merging) 256-thread blocks per SM; float64 forms unbounded
template <class R, int D, bool FWD, bool MRG = false>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? (MRG ? 5 : 6) : 1)
    k_fft(const __grid_constant__ JobSet<R> js, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_block<R, D, FWD, MRG, 256>(js, pass, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------
// interpolation (Algorithm 2.1 step 3): one warp per work item; the warp copies the
// padded tile of the grid around its tile into shared memory, then every lane sums the
// taps of one point and writes f_j in the caller's order.
template <class R, int D>
__global__ void __launch_bounds__(128) k_interp(const __grid_constant__ JobSet<R> js) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gitem = blockIdx.x * js.wpb + warp;
    if (gitem >= js.pre_items[js.njobs]) return;
    const int jb = find_job(js.pre_items, js.njobs, gitem);
    const Job<R>& J = js.job[jb];
    const int4 item = J.items[gitem - js.pre_items[jb]];
    const int P = J.P, m = J.m, Ms = J.Ms, T = J.T;
    const int W = 2 * m + 1;
    const bool bopt = (J.mode == INFFT_MODE_BOPT);   // f = B_opt F D h (Remark 4.6)
    const int S = bopt ? J.S : W;                     // slots per axis
    const int cells = ipow(P, D);
    unsigned char* base = smem_raw + (size_t)warp * js.smem_per_warp;
    cx<R>* pad = reinterpret_cast<cx<R>*>(base);
    R* psi = reinterpret_cast<R*>(pad + cells);  // [32][D][W]

    int tt[D];
    {
        int rem = item.x;
        for (int t = D - 1; t >= 0; --t) { tt[t] = rem % J.ntile; rem /= J.ntile; }
    }
    for (int e = lane; e < cells; e += 32) {
        int rem = e;
        long long g = 0;
        for (int t = 0; t < D; ++t) {
            const int div = ipow(P, D - 1 - t);
            const int o = rem / div;
            rem -= o * div;
            g = g * Ms + mod_pos(tt[t] * T - m + o, Ms);
        }
        pad[e] = J.grid[g];
    }
    int pstride[D];
    pstride[D - 1] = 1;
    for (int t = D - 2; t >= 0; --t) pstride[t] = pstride[t + 1] * P;
    const int ntap = ipow(S, D);
    __syncwarp();

    for (int c0 = 0; c0 < item.z; c0 += 32) {
        const int np = min(32, item.z - c0);
        if (lane < np) {
            const int i = item.y + c0 + lane;
            uint32_t rem = __ldg(J.cell + i);
            int o[D];
            for (int t = D - 1; t >= 0; --t) {
                const int c = (int)(rem % (uint32_t)Ms);
                rem /= (uint32_t)Ms;
                o[t] = c - tt[t] * T;
            }
            R* ps = psi + lane * D * W;
            if (!bopt) {
                for (int t = 0; t < D; ++t) {
                    const R u = J.u[(size_t)i * D + t];
                    for (int s = 0; s < W; ++s) ps[t * W + s] = tap_weight<R>(J.window, u, s, m, J.inv_m, J.beta);
                }
            }
            const cx<R>* cf = bopt ? J.coef + (size_t)i * ntap : nullptr;
            cx<R> acc = mk<R>(0, 0);
            for (int q = 0; q < ntap; ++q) {
                int r2 = q, idx = 0;
                R wgt = R(1);
                for (int t = D - 1; t >= 0; --t) {
                    const int s = r2 % S;
                    r2 /= S;
                    idx += (o[t] + s) * pstride[t];
                    if (!bopt) wgt *= ps[t * W + s];
                }
                const cx<R> g = pad[idx];
                if (bopt) {
                    acc = add(acc, mul(cf[q], g));   // B_opt[j, l] g_l
                } else {
                    acc.re += wgt * g.re;
                    acc.im += wgt * g.im;
                }
            }
            J.out[__ldg(J.perm + i)] = acc;
        }
    }
}

// ---------------------------------------------------------------------------------------
// host drivers

static int pick_lines(int n, size_t elem) { return fft_lines(n, (int)elem); }

template <class R>
static void fill_prefixes(JobSet<R>& js, int D, bool forward) {
    js.pre_items[0] = 0;
    js.pre_merge[0] = 0;
    for (int p = 0; p < 3; ++p) js.pre_fft[p][0] = 0;
    int maxMs = 0;
    for (int j = 0; j < js.njobs; ++j) maxMs = std::max(maxMs, js.job[j].Ms);
    js.L = pick_lines(maxMs, sizeof(cx<R>));
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        js.pre_items[j + 1] = js.pre_items[j] + J.nitems;
        const long long cells = (long long)ipow(J.Ms, D);
        js.pre_merge[j + 1] = js.pre_merge[j] + (int)((cells + 255) / 256);
        for (int p = 0; p < 3; ++p) {
            int blocks = 0;
            if (p < D) {
                const int t = forward ? p : D - 1 - p;
                const long long lines = (long long)ipow(J.Ms, t) * ipow(J.M, D - 1 - t);
                const int Lj = pick_lines(J.Ms, sizeof(cx<R>));
                blocks = (int)((lines + Lj - 1) / Lj);
            }
            js.pre_fft[p][j + 1] = js.pre_fft[p][j] + blocks;
        }
    }
}

template <class R>
static size_t spread_smem_per_warp(const JobSet<R>& js, int D) {
    size_t mx = 0;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        const int W = 2 * J.m + 1;
        size_t b = (size_t)ipow(J.P, D) * sizeof(cx<R>) + 32 * D * W * sizeof(R) + 32 * sizeof(cx<R>) +
                   32 * (D + 1) * sizeof(int);
        b = (b + 15) & ~(size_t)15;
        mx = std::max(mx, b);
    }
    return mx;
}

// a JobSet of the listed jobs of js (prefixes not yet filled), on the heap
template <class R>
static JobSet<R>* new_subset(const JobSet<R>& js, const std::vector<int>& idx) {
    JobSet<R>* s = new JobSet<R>();
    memset(s, 0, sizeof(*s));
    s->njobs = (int)idx.size();
    for (int i = 0; i < s->njobs; ++i) s->job[i] = js.job[idx[i]];
    return s;
}

// pruned FFT passes with deconvolution, common to every spreading variant
template <class R, int D>
static infft_status launch_fft_adjoint(JobSet<R>& js, cudaStream_t st, cudaEvent_t* ev) {
    const size_t fsmem = fft_smem(js);
    INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    for (int p = 0; p < D; ++p) {
        k_fft<R, D, false><<<js.pre_fft[p][js.njobs], 256, fsmem, st>>>(js, p);
        INFFT_LAUNCHED();
        if (ev) INFFT_CUDA(cudaEventRecord(ev[3 + p], st));
    }
    return INFFT_OK;
}

template <class R>
static infft_status launch_fft_adjoint_mrg(JobSet<R>& js, cudaStream_t st, cudaEvent_t* ev) {
    const size_t msmem = fft_smem_mrg(js);
    INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, 2, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem));
    k_fft<R, 2, false, true><<<js.pre_fft[0][js.njobs], 256, msmem, st>>>(js, 0);
    INFFT_LAUNCHED();
    if (ev) INFFT_CUDA(cudaEventRecord(ev[3], st));
    const size_t fsmem = fft_smem(js);
    INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    k_fft<R, 2, false><<<js.pre_fft[1][js.njobs], 256, fsmem, st>>>(js, 1);
    INFFT_LAUNCHED();
    if (ev) INFFT_CUDA(cudaEventRecord(ev[4], st));
    return INFFT_OK;
}

template <class R, int D>
static infft_status launch_adjoint(JobSet<R>& js, cudaStream_t st, cudaEvent_t* ev, bool grid_only = false) {
    fill_prefixes(js, D, false);
    if (ev) INFFT_CUDA(cudaEventRecord(ev[0], st));
    bool used = false;
    if constexpr (D == 2 && std::is_same<R, float>::value) {
        // one persistent launch where it applies (untimed: the stages are not separable)
        if (!grid_only && !ev) {
            INFFT_TRY(persist2d_try(js, st, &used));
            if (used) return INFFT_OK;
        }
    }
    if (D == 2) INFFT_TRY(spread2d_try<R>(js, st, &used));
    if (used) {
        if (ev) INFFT_CUDA(cudaEventRecord(ev[1], st));
        // merge and FFT passes fused in one cluster kernel per grid size where it applies
        std::vector<int> rest;
        if (grid_only) {
            for (int j = 0; j < js.njobs; ++j) rest.push_back(j);
        } else {
            INFFT_TRY(mergefft2d_try<R>(js, st, rest));
        }
        if (rest.empty()) {
            if (ev)
                for (int k = 2; k < 3 + D; ++k) INFFT_CUDA(cudaEventRecord(ev[k], st));
            return INFFT_OK;
        }
        // the other jobs: merge (one block per tile), then the FFT passes
        JobSet<R>& jr = (int)rest.size() == js.njobs ? js : *new_subset(js, rest);
        std::unique_ptr<JobSet<R>> own(&jr == &js ? nullptr : &jr);
        if (own) fill_prefixes(jr, D, false);
        if constexpr (D == 2) {
            if (!grid_only && merge_on_load_ok(jr)) {
                if (ev) INFFT_CUDA(cudaEventRecord(ev[2], st));   // the merge is timed with pass 0
                return launch_fft_adjoint_mrg<R>(jr, st, ev);
            }
        }
        jr.pre_merge[0] = 0;
        for (int j = 0; j < jr.njobs; ++j) jr.pre_merge[j + 1] = jr.pre_merge[j] + jr.job[j].ntile * jr.job[j].ntile;
        k_merge2d<R><<<jr.pre_merge[jr.njobs], 256, 0, st>>>(jr);
        INFFT_LAUNCHED();
        if (ev) INFFT_CUDA(cudaEventRecord(ev[2], st));
        if (grid_only) return INFFT_OK;
        return launch_fft_adjoint<R, D>(jr, st, ev);
    }
    if (D == 3) INFFT_TRY(spread3d_try<R>(js, st, &used));
    if (used) {
        if (ev) INFFT_CUDA(cudaEventRecord(ev[1], st));
        js.pre_merge[0] = 0;
        for (int j = 0; j < js.njobs; ++j) {
            const int nt = js.job[j].ntile;
            js.pre_merge[j + 1] = js.pre_merge[j] + nt * nt * nt;
        }
        k_merge3d<R><<<js.pre_merge[js.njobs], 256, 0, st>>>(js);
        INFFT_LAUNCHED();
        if (ev) INFFT_CUDA(cudaEventRecord(ev[2], st));
        if (grid_only) return INFFT_OK;
        return launch_fft_adjoint<R, D>(js, st, ev);
    }
    const size_t spw = spread_smem_per_warp(js, D);
    const size_t smem_cap = 200 * 1024;
    if (spw > smem_cap) {
        set_error("padded tile needs %zu bytes of shared memory", spw);
        return INFFT_EUNSUPPORTED;
    }
    js.smem_per_warp = (int)spw;
    js.wpb = (int)std::max<size_t>(1, std::min<size_t>(4, smem_cap / spw));
    const int nitems = js.pre_items[js.njobs];
    if (nitems > 0) {
        const size_t smem = spw * js.wpb;
        INFFT_CUDA(cudaFuncSetAttribute(k_spread<R, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_spread<R, D><<<(nitems + js.wpb - 1) / js.wpb, 32 * js.wpb, smem, st>>>(js);
        INFFT_LAUNCHED();
    }
    if (ev) INFFT_CUDA(cudaEventRecord(ev[1], st));
    k_merge<R, D><<<js.pre_merge[js.njobs], 256, 0, st>>>(js);
    INFFT_LAUNCHED();
    if (ev) INFFT_CUDA(cudaEventRecord(ev[2], st));
    if (grid_only) return INFFT_OK;
    return launch_fft_adjoint<R, D>(js, st, ev);
}

template <class R, int D>
static infft_status launch_forward(JobSet<R>& js, cudaStream_t st) {
    fill_prefixes(js, D, true);
    const size_t fsmem = fft_smem(js);
    INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    for (int p = 0; p < D; ++p) {
        k_fft<R, D, true><<<js.pre_fft[p][js.njobs], 256, fsmem, st>>>(js, p);
        INFFT_LAUNCHED();
    }
    if constexpr (D >= 2) {
        bool used = false;
        if (D == 2) INFFT_TRY(interp2d_try<R>(js, st, &used));
        else INFFT_TRY(interp3d_try<R>(js, st, &used));
        if (used) return INFFT_OK;
    }
    size_t spw = 0;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        size_t b = (size_t)ipow(J.P, D) * sizeof(cx<R>) + 32 * D * (2 * J.m + 1) * sizeof(R);
        spw = std::max(spw, (b + 15) & ~(size_t)15);
    }
    const size_t smem_cap = 200 * 1024;
    if (spw > smem_cap) {
        set_error("padded tile needs %zu bytes of shared memory", spw);
        return INFFT_EUNSUPPORTED;
    }
    js.smem_per_warp = (int)spw;
    js.wpb = (int)std::max<size_t>(1, std::min<size_t>(4, smem_cap / spw));
    const int nitems = js.pre_items[js.njobs];
    if (nitems > 0) {
        const size_t smem = spw * js.wpb;
        INFFT_CUDA(cudaFuncSetAttribute(k_interp<R, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_interp<R, D><<<(nitems + js.wpb - 1) / js.wpb, 32 * js.wpb, smem, st>>>(js);
        INFFT_LAUNCHED();
    }
    return INFFT_OK;
}

template <class R>
infft_status run_jobs(const std::vector<Job<R>>& jobs, cudaStream_t st, bool forward, cudaEvent_t* ev) {
    return run_jobs<R>(jobs.data(), jobs.size(), st, forward, ev);
}

template <class R>
infft_status run_jobs(const Job<R>* jobs, size_t count, cudaStream_t st, bool forward, cudaEvent_t* ev) {
    if (count == 0) return INFFT_OK;
    const int D = jobs[0].d;
    for (size_t s = 0; s < count; s += MAXJ) {
        JobSet<R> js;
        memset(&js, 0, sizeof(js));
        js.njobs = (int)std::min<size_t>(MAXJ, count - s);
        for (int j = 0; j < js.njobs; ++j) js.job[j] = jobs[s + j];
        infft_status r;
        if (!forward) {
            cudaEvent_t* e = (s == 0) ? ev : nullptr;
            r = D == 1 ? launch_adjoint<R, 1>(js, st, e) : D == 2 ? launch_adjoint<R, 2>(js, st, e) : launch_adjoint<R, 3>(js, st, e);
        } else {
            r = D == 1 ? launch_forward<R, 1>(js, st) : D == 2 ? launch_forward<R, 2>(js, st) : launch_forward<R, 3>(js, st);
        }
        if (r != INFFT_OK) return r;
    }
    return INFFT_OK;
}

template <class R, int D>
static infft_status fft_passes_d(JobSet<R>& js, cudaStream_t st, bool forward) {
    fill_prefixes(js, D, forward);
    const int n = js.job[0].Ms;
    const size_t fsmem = fft_smem(js);
    if (forward) {
        INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
        for (int p = 0; p < D; ++p) {
            k_fft<R, D, true><<<js.pre_fft[p][1], 256, fsmem, st>>>(js, p);
            INFFT_LAUNCHED();
        }
    } else {
        INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
        for (int p = 0; p < D; ++p) {
            k_fft<R, D, false><<<js.pre_fft[p][1], 256, fsmem, st>>>(js, p);
            INFFT_LAUNCHED();
        }
    }
    return INFFT_OK;
}

template <class R>
infft_status run_spread_grid(const Job<R>& J, cudaStream_t st) {
    JobSet<R> js;
    memset(&js, 0, sizeof(js));
    js.njobs = 1;
    js.job[0] = J;
    switch (J.d) {
        case 1: return launch_adjoint<R, 1>(js, st, nullptr, true);
        case 2: return launch_adjoint<R, 2>(js, st, nullptr, true);
        default: return launch_adjoint<R, 3>(js, st, nullptr, true);
    }
}

template <class R>
infft_status run_fft_axis(const Job<R>& J, long long A, long long B, int nblk, cudaStream_t st) {
    JobSet<R> js;
    memset(&js, 0, sizeof(js));
    js.njobs = 1;
    js.job[0] = J;
    js.axA = A;
    js.axB = B;
    js.axblk = nblk;
    const int n = J.Ms;
    js.L = pick_lines(n, sizeof(cx<R>));
    const long long lines = A * B;
    if ((lines + js.L - 1) / js.L >= (1ll << 31)) {
        set_error("too many FFT lines");
        return INFFT_EUNSUPPORTED;
    }
    js.pre_fft[0][1] = (int)((lines + js.L - 1) / js.L);
    const size_t fsmem = fft_smem(js);
    INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    k_fft<R, 2, false><<<js.pre_fft[0][1], 256, fsmem, st>>>(js, 0);
    INFFT_LAUNCHED();
    return INFFT_OK;
}
template infft_status run_spread_grid<float>(const Job<float>&, cudaStream_t);
template infft_status run_spread_grid<double>(const Job<double>&, cudaStream_t);
template infft_status run_fft_axis<float>(const Job<float>&, long long, long long, int, cudaStream_t);
template infft_status run_fft_axis<double>(const Job<double>&, long long, long long, int, cudaStream_t);

template <class R>
infft_status run_fft_passes(const Job<R>& J, cudaStream_t st, bool forward) {
    JobSet<R> js;
    memset(&js, 0, sizeof(js));
    js.njobs = 1;
    js.job[0] = J;
    switch (J.d) {
        case 1: return fft_passes_d<R, 1>(js, st, forward);
        case 2: return fft_passes_d<R, 2>(js, st, forward);
        default: return fft_passes_d<R, 3>(js, st, forward);
    }
}

template infft_status run_fft_passes<double>(const Job<double>&, cudaStream_t, bool);
template infft_status run_jobs<float>(const std::vector<Job<float>>&, cudaStream_t, bool, cudaEvent_t*);
template infft_status run_jobs<double>(const std::vector<Job<double>>&, cudaStream_t, bool, cudaEvent_t*);
template infft_status run_jobs<float>(const Job<float>*, size_t, cudaStream_t, bool, cudaEvent_t*);
template infft_status run_jobs<double>(const Job<double>*, size_t, cudaStream_t, bool, cudaEvent_t*);

}  // namespace infft
