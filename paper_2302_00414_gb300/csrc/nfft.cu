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
// FFT pass along one axis for a batch of lines held in shared memory: radix-2
// decimation in time after a bit-reversed load.  Adjoint direction (FWD = false):
// forward DFT (sign -) of length Ms, keep the M outputs k in I_M, multiply by
// 1/(Ms w^(k)) of this axis.  Forward direction (FWD = true): the M inputs of I_M times
// 1/(Ms w^(k)) are placed at k mod Ms, the rest is zero, inverse DFT (sign +).
// A pass sees a tensor (A, n_in, B): lines run along the middle index with stride B.
// Shared-memory position of element i of a line: one padding slot every 16 elements,
// so that the bit-reversed scatter and the short butterfly strides spread over banks.
__device__ __forceinline__ int skew(int i) { return i + (i >> 4); }

// e / M for 0 <= e < 2^22 through a float32 reciprocal rM ~ 1/M and one correction step (the
// estimate is off by at most one there): a few instructions instead of an integer division
__device__ __forceinline__ int div_small(int e, int M, float rM) {
    int q = __float2int_rz((float)e * rM);
    const int r = e - q * M;
    if (r < 0) --q;
    else if (r >= M) ++q;
    return q;
}

// lines of length n per FFT block: a 16 KB budget of complex elements, at most 32 lines (more,
// smaller blocks hide the passes' load latency better: batched d = 2, n = 512: 64 / 32 / 16 / 8 KB
// of lines per block gave FFT passes of 0.140 / 0.109 / 0.100 / 0.104 ms).  Per job, so that the
// blocks of small grids are as full as those of large ones.
__host__ __device__ inline int fft_lines(int n, int elem) {
    int L = 1;
    while (L < 32 && 2 * L * n * elem <= 16 * 1024) L *= 2;
    return L;
}

// rows of tiles whose item ranges a merge-on-load block of L lines (grid rows) consults: its
// own one or L / T, and one above and below
__host__ __device__ inline int mrg_tile_rows(int L, int T) { return (L <= T ? 1 : L / T) + 2; }

// With MRG (d = 2 adjoint, pass 0 only) the block's lines are grid rows whose cells are summed
// from the padded tiles as they are loaded: the halo merge of k_merge2d in the same order per
// cell, with no grid written or read in between.  The item ranges of the tiles the block's
// rows draw on are staged in shared memory after the twiddles first.
template <class R, int D, bool FWD, bool MRG = false>
__global__ void __launch_bounds__(256) k_fft(const __grid_constant__ JobSet<R> js, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
    const int gblk = blockIdx.x;
    const int jb = find_job(js.pre_fft[pass], js.njobs, gblk);
    const Job<R>& J = js.job[jb];
    const int lb = gblk - js.pre_fft[pass][jb];
    const int Ms = J.Ms, M = J.M, L = fft_lines(J.Ms, (int)sizeof(cx<R>));
    const int t = FWD ? pass : D - 1 - pass;
    const bool expl = !FWD && js.axA > 0;   // one explicit pass over an (A, Ms, B) tensor
    const long long A = expl ? js.axA : ipow(Ms, t);
    const long long B = expl ? js.axB : ipow(M, D - 1 - t);
    const int MB = expl ? M / js.axblk : M;   // output block along the middle index
    const int n = Ms;
    const int ns = n + (n >> 4);    // skewed line stride
    const int logn = 31 - __clz(n);
    const long long nlines = A * B;
    const long long q0 = (long long)lb * L;
    const bool lanes_b = (B >= L);  // consecutive lines are consecutive b: coalesce along b

    cx<R>* tws = buf + L * ns;      // the n/2 twiddles after the lines
    for (int k = threadIdx.x; k < (Ms >> 1); k += blockDim.x) tws[k] = J.tw[k];
    // then (merging pass only) the table of tile item ranges, then the M deconvolution factors
    const int nrng = (MRG && pass == 0) ? mrg_tile_rows(L, J.T) * J.ntile : 0;
    R* dvs = reinterpret_cast<R*>(reinterpret_cast<int2*>(tws + (Ms >> 1)) + nrng);
    for (int k = threadIdx.x; k < M; k += blockDim.x) dvs[k] = J.dinv[k];

    const cx<R>* src;
    cx<R>* dst;
    if (expl) {
        src = J.grid;
        dst = J.out;
    } else if (!FWD) {
        src = (pass == 0) ? J.grid : (pass == 1 ? J.tmp1 : J.tmp2);
        dst = (pass == D - 1) ? J.out : (pass == 0 ? J.tmp1 : J.tmp2);
    } else {
        src = (pass == 0) ? J.in : (pass == 1 ? J.tmp1 : J.tmp2);
        dst = (pass == D - 1) ? J.grid : (pass == 0 ? J.tmp1 : J.tmp2);
    }
    const int tid = threadIdx.x, nth = blockDim.x;
    const int logL = 31 - __clz(L);   // L is a power of two

    // offsets of each line's first element in the source and destination tensors (line l of
    // the block is (a, b) = divmod(q0 + l, B); element i sits i * B further), or -1 past the end
    __shared__ long long s_in[32], s_out[32];
    if (tid < L) {
        const long long q = q0 + tid;
        long long bi = -1, bo = -1;
        if (q < nlines) {
            // a 32-bit division where the counts allow (a 64-bit one is a long software routine
            // that the whole block would wait for)
            long long a;
            if (nlines <= 0x7fffffffLL && B <= 0x7fffffffLL) a = (long long)((unsigned)q / (unsigned)B);
            else a = q / B;
            const long long b = q - a * B;
            bi = (a * (FWD ? M : n)) * B + b;
            bo = (a * (FWD ? n : MB)) * B + b;
        }
        s_in[tid] = bi;
        s_out[tid] = bo;
    }
    __syncthreads();

    if (MRG && pass == 0) {
        const int T = J.T, m = J.m, P = J.P, nt = J.ntile;
        const int logT = 31 - __clz(T), lognt = 31 - __clz(nt);
        const int ty0 = (int)(q0 >> logT);
        const int ntr = mrg_tile_rows(L, T);
        int2* rng = reinterpret_cast<int2*>(tws + (n >> 1));   // [ntr][nt] first item, count
        for (int k = tid; k < ntr * nt; k += nth) {
            const int tyw = (ty0 - 1 + (k >> lognt)) & (nt - 1), tx = k & (nt - 1);
            const int a = __ldg(J.tile_items + tyw * nt + tx), b = __ldg(J.tile_items + tyw * nt + tx + 1);
            rng[k] = make_int2(a, b - a);
        }
        __syncthreads();
        const size_t cells = (size_t)P * P;
#pragma unroll 2
        for (int e = tid; e < L * n; e += nth) {
            int l, i;
            if (lanes_b) { l = e & (L - 1); i = e >> logL; } else { i = e & (n - 1); l = e >> logn; }
            const long long y = q0 + l;
            cx<R> acc = mk<R>(0, 0);
            if (y < nlines) {
                const int r = (int)y & (T - 1), ty = (int)(y >> logT), c = i & (T - 1), tx = i >> logT;
                int yd[2], yo[2], xd[2], xo[2], ny = 1, nx = 1;
                yd[0] = 0; yo[0] = r + m;
                xd[0] = 0; xo[0] = c + m;
                if (r + T + m < P) { yd[1] = -1; yo[1] = r + T + m; ny = 2; }
                else if (r - T + m >= 0) { yd[1] = 1; yo[1] = r - T + m; ny = 2; }
                if (c + T + m < P) { xd[1] = -1; xo[1] = c + T + m; nx = 2; }
                else if (c - T + m >= 0) { xd[1] = 1; xo[1] = c - T + m; nx = 2; }
                // the first item of every source, loaded together; then the sum in source order
                size_t src0[4];
                int cnt[4];
                cx<R> v[4];
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int q = 2 * a + b;
                        cnt[q] = 0;
                        src0[q] = 0;
                        if (a < ny && b < nx) {
                            const int2 g = rng[((ty + yd[a] - ty0 + 1) << lognt) + ((tx + xd[b]) & (nt - 1))];
                            cnt[q] = g.y;
                            src0[q] = (size_t)g.x * cells + (size_t)yo[a] * P + xo[b];
                        }
                    }
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = cnt[q] > 0 ? J.padded[src0[q]] : mk<R>(0, 0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (cnt[q] <= 0) continue;
                    acc = add(acc, v[q]);
#pragma unroll 1
                    for (int k = 1; k < cnt[q]; ++k) acc = add(acc, J.padded[src0[q] + (size_t)k * cells]);
                }
            }
            buf[l * ns + skew(bitrev(i, logn))] = acc;
        }
    } else if (!FWD) {
        // each thread issues the loads of up to eight elements before storing any, so that
        // the block waits for one global-load latency rather than eight in a row
        constexpr int KL = 8;
        const int total = L * n;
        for (int e0 = tid; e0 < total; e0 += KL * nth) {
            cx<R> v[KL];
            int pos[KL];
#pragma unroll
            for (int k = 0; k < KL; ++k) {
                const int e = e0 + k * nth;
                pos[k] = -1;
                v[k] = mk<R>(0, 0);
                if (e < total) {
                    int l, i;
                    if (lanes_b) { l = e & (L - 1); i = e >> logL; } else { i = e & (n - 1); l = e >> logn; }
                    const long long g0 = s_in[l];
                    pos[k] = l * ns + skew(bitrev(i, logn));
                    if (g0 >= 0) v[k] = src[g0 + (long long)i * B];
                }
            }
#pragma unroll
            for (int k = 0; k < KL; ++k)
                if (pos[k] >= 0) buf[pos[k]] = v[k];
        }
    } else {
        for (int e = tid; e < L * ns; e += nth) buf[e] = mk<R>(0, 0);
        __syncthreads();
        const float rM = 1.f / (float)M;
        for (int e = tid; e < L * M; e += nth) {
            int l, i;
            if (lanes_b) { l = e & (L - 1); i = e >> logL; } else { l = div_small(e, M, rM); i = e - l * M; }
            const long long g0 = s_in[l];
            if (g0 >= 0) {
                const cx<R> v = scale(src[g0 + (long long)i * B], dvs[i]);
                const int bin = (i - M / 2) & (n - 1);   // n = M_sigma is a power of two
                buf[l * ns + skew(bitrev(bin, logn))] = v;
            }
        }
    }
    __syncthreads();

    // Butterflies in place, two radix-2 stages at a time: one thread takes the four
    // elements j + k q (k = 0..3) of a group of 4q and applies the stage of half-length q
    // (twiddle W_2q^pos) and then that of half-length 2q (W_4q^pos, W_4q^(pos+q)) in
    // registers.  An odd number of stages starts with one radix-2 stage of half-length 1.
    // Twiddles W_n^k = exp(-2 pi i k / n), k < n/2, come from shared memory (conjugated
    // for the inverse direction).
    const int half_n = n >> 1;
    const int loghn = logn - 1;
    int lh = 0;
    if (logn & 1) {
        for (int e = tid; e < L * half_n; e += nth) {
            const int l = e >> loghn, jj = e & (half_n - 1);
            cx<R>* row = buf + l * ns;
            const cx<R> a = row[skew(2 * jj)], b = row[skew(2 * jj + 1)];
            row[skew(2 * jj)] = add(a, b);
            row[skew(2 * jj + 1)] = sub(a, b);
        }
        __syncthreads();
        lh = 1;
    }
    const int quarter_n = n >> 2;
    const int logqn = logn - 2;
    for (; lh < logn; lh += 2) {
        const int q = 1 << lh;
        for (int e = tid; e < L * quarter_n; e += nth) {
            const int l = e >> logqn, jj = e & (quarter_n - 1);
            const int grp = jj >> lh, pos = jj & (q - 1);
            const int base = grp * (q << 2) + pos;
            cx<R>* row = buf + l * ns;
            const cx<R> a0 = row[skew(base)], a1 = row[skew(base + q)];
            const cx<R> a2 = row[skew(base + 2 * q)], a3 = row[skew(base + 3 * q)];
            cx<R> w1 = tws[pos << (logn - 1 - lh)];
            cx<R> w2 = tws[pos << (logn - 2 - lh)];
            cx<R> w3 = tws[(pos + q) << (logn - 2 - lh)];
            if (FWD) { w1.im = -w1.im; w2.im = -w2.im; w3.im = -w3.im; }
            cx<R> t = mul(w1, a1);
            const cx<R> b0 = add(a0, t), b1 = sub(a0, t);
            t = mul(w1, a3);
            const cx<R> b2 = add(a2, t), b3 = sub(a2, t);
            t = mul(w2, b2);
            row[skew(base)] = add(b0, t);
            row[skew(base + 2 * q)] = sub(b0, t);
            t = mul(w3, b3);
            row[skew(base + q)] = add(b1, t);
            row[skew(base + 3 * q)] = sub(b1, t);
        }
        __syncthreads();
    }

    if (!FWD) {
        if (expl) {
            for (int e = tid; e < L * M; e += nth) {
                int l, i;
                if (lanes_b) { l = e & (L - 1); i = e >> logL; } else { i = e % M; l = e / M; }
                const long long g0 = s_out[l];
                if (g0 >= 0) {
                    const int bin = (i - M / 2) & (n - 1);
                    // block i / MB of the middle index holds the (A, MB, B) tensor of its indices
                    const long long o = (long long)(i / MB) * A * MB * B + (long long)(i % MB) * B;
                    dst[g0 + o] = scale(buf[l * ns + skew(bin)], dvs[i]);
                }
            }
        } else if (lanes_b) {
            for (int e = tid; e < L * M; e += nth) {
                const int l = e & (L - 1), i = e >> logL;
                const long long g0 = s_out[l];
                if (g0 >= 0) dst[g0 + (long long)i * B] = scale(buf[l * ns + skew((i - M / 2) & (n - 1))], dvs[i]);
            }
        } else {   // nth / L threads per line (both powers of two), no division per element
            const int tpl = nth >> logL, l = tid / tpl;
            const long long g0 = s_out[l];
            if (g0 >= 0)
                for (int i = tid & (tpl - 1); i < M; i += tpl)
                    dst[g0 + (long long)i * B] = scale(buf[l * ns + skew((i - M / 2) & (n - 1))], dvs[i]);
        }
    } else {
        for (int e = tid; e < L * n; e += nth) {
            int l, i;
            if (lanes_b) { l = e & (L - 1); i = e >> logL; } else { i = e & (n - 1); l = e >> logn; }
            const long long g0 = s_out[l];
            if (g0 >= 0) dst[g0 + (long long)i * B] = buf[l * ns + skew(i)];
        }
    }
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

// shared memory of an FFT launch over the jobs of js: the largest of the jobs' line buffers
// plus twiddles
template <class R>
static size_t fft_smem(const JobSet<R>& js) {
    size_t mx = 0;
    for (int j = 0; j < js.njobs; ++j) {
        const int n = js.job[j].Ms, L = pick_lines(n, sizeof(cx<R>));
        mx = std::max(mx, ((size_t)L * (n + n / 16) + n / 2) * sizeof(cx<R>) + (size_t)js.job[j].M * sizeof(R));
    }
    return mx;
}

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

// The halo merge of the d = 2 register-row path folded into the first FFT pass (k_fft with
// MRG), unless INFFT_FFT_MERGE=0 or a job's table of tile item ranges would pass 16 KB: the
// grid is then neither written nor read between the two.  Both forms give bitwise the same
// result.
template <class R>
static bool merge_on_load_ok(const JobSet<R>& js) {
    if (env_form("INFFT_FFT_MERGE") == 0 || js.axA > 0) return false;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        const int L = pick_lines(J.Ms, sizeof(cx<R>));
        if ((size_t)mrg_tile_rows(L, J.T) * J.ntile * sizeof(int2) > 16 * 1024) return false;
    }
    return true;
}

template <class R>
static infft_status launch_fft_adjoint_mrg(JobSet<R>& js, cudaStream_t st, cudaEvent_t* ev) {
    size_t msmem = 0;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        const int n = J.Ms, L = pick_lines(n, sizeof(cx<R>));
        const size_t b = ((size_t)L * (n + n / 16) + n / 2) * sizeof(cx<R>) +
                         (size_t)mrg_tile_rows(L, J.T) * J.ntile * sizeof(int2) + (size_t)J.M * sizeof(R);
        msmem = std::max(msmem, b);
    }
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
