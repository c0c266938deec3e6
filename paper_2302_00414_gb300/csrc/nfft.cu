// NFFT kernels: tile-sorted spreading (Algorithm 2.4 step 1, and its modified
// forms of Algorithm 3.7 / 4.4), halo merge, d-variate FFT passes with pruned
// output and per-axis deconvolution (Algorithm 2.4 steps 2-3), zero-padded
// inverse FFT passes (Algorithm 2.1 steps 1-2) and tile-sorted interpolation
// (Algorithm 2.1 step 3).
#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "jobset.cuh"

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

// ---------------------------------------------------------------------------------------
// Two-dimensional spreading with the accumulators in registers.  One warp per work
// item; lane l owns column l of the item's P x P padded tile (P = T + 2m + 1 <= 32).
// The item's points are sorted by base row, so the rows a point can touch,
// [oy, oy + 2m] (padded coordinates; one more row for B_opt slots), only move down:
// each lane keeps those rows of its column in registers, adds the point's taps
// (coefficient c_j psi_y[k] broadcast, times psi_x of its column), and when the next
// point starts lower it stores the rows that no later point can reach.  Every padded
// cell is stored exactly once, no shared-memory read-modify-write, no atomics.
// Window values are computed once per point while staging 32 points per warp.
template <class R, int MM, bool BOPT>
__global__ void __launch_bounds__(128) k_spread2d(const __grid_constant__ JobSet<R> js) {
    constexpr int W = 2 * MM + 1;              // window taps per axis
    constexpr int WE = W + 1;                  // even stride of the staged rows (16-byte loads)
    constexpr int WR = BOPT ? W + 1 : W;       // rows held in registers
    constexpr bool F32 = sizeof(R) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gitem = blockIdx.x * js.wpb + warp;
    if (gitem >= js.pre_items[js.njobs]) return;
    const int jb = find_job(js.pre_items, js.njobs, gitem);
    const Job<R>& J = js.job[jb];
    const int it = gitem - js.pre_items[jb];
    const int4 item = J.items[it];
    const int P = J.P, Ms = J.Ms, T = J.T;

    unsigned char* base = smem_raw + (size_t)warp * js.smem_per_warp;
    cx<R>* cy = reinterpret_cast<cx<R>*>(base);            // [32][WE] c_j psi_y (window mode)
    R* psx = reinterpret_cast<R*>(cy + 32 * WE);            // [32][WE] psi_x
    int* meta = reinterpret_cast<int*>(psx + 32 * WE);      // [32][3]  oy, ox, sorted index
    cx<R>* cst = reinterpret_cast<cx<R>*>(meta + 96);       // [32]     c_j (B_opt mode)
    float* poly = reinterpret_cast<float*>(cst + 32);       // [(WPOLY_DEG+1) * WP] window polynomial (16-byte rows)
    const bool use_poly = F32 && !BOPT && J.wpoly != nullptr;
    if (use_poly) {
        for (int e = lane; e < (WPOLY_DEG + 1) * wpoly_stride(W); e += 32) poly[e] = J.wpoly[e];
    }

    const int ty = item.x / J.ntile, tx = item.x % J.ntile;
    using V2 = typename std::conditional<F32, float2, double2>::type;
    V2 acc[WR];  // (re, im) of the rows r0 .. r0 + WR - 1 of this lane's column
#pragma unroll
    for (int k = 0; k < WR; ++k) { acc[k].x = R(0); acc[k].y = R(0); }
    int r0 = 0;  // padded row held in acc[0]
    cx<R>* dst = J.padded + (size_t)it * P * P;
    const bool col_ok = lane < P;
    const int logMs = 31 - __clz(Ms);

    for (int c0 = 0; c0 < item.z; c0 += 32) {
        const int np = min(32, item.z - c0);
        __syncwarp();
        if (lane < np) {
            const int i = item.y + c0 + lane;
            const int j = __ldg(J.perm + i);
            cx<R> fv = J.in[j];
            if (J.mode == INFFT_MODE_DCF) fv = mul(J.w[i], fv);
            const uint32_t cl = __ldg(J.cell + i);
            const int cxl = (int)(cl & (uint32_t)(Ms - 1)), cyl = (int)(cl >> logMs);
            meta[lane * 3 + 0] = cyl - ty * T;
            meta[lane * 3 + 1] = cxl - tx * T;
            meta[lane * 3 + 2] = i;
            if (BOPT) {
                cst[lane] = fv;
            } else {
                const R uy = J.u[(size_t)i * 2 + 0], ux = J.u[(size_t)i * 2 + 1];
                R wy[W], wx[W];
                bool done = false;
                if constexpr (F32) {
                    if (use_poly) {
                        poly_taps2<W>(poly, uy, ux, wy, wx);
                        done = true;
                    }
                }
                if (!done) {
#pragma unroll
                    for (int s = 0; s < W; ++s) {
                        wy[s] = tap_weight<R>(J.window, uy, s, MM, J.inv_m, J.beta);
                        wx[s] = tap_weight<R>(J.window, ux, s, MM, J.inv_m, J.beta);
                    }
                }
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    cy[lane * WE + s] = scale(fv, wy[s]);
                    psx[lane * WE + s] = wx[s];
                }
                cy[lane * WE + W] = mk<R>(0, 0);
            }
        }
        __syncwarp();
        for (int p = 0; p < np; ++p) {
            const int oy = meta[p * 3 + 0], ox = meta[p * 3 + 1];
            // store the rows above oy: no later point reaches them
            while (r0 < oy) {
                if (col_ok) dst[(size_t)r0 * P + lane] = mk<R>(acc[0].x, acc[0].y);
#pragma unroll
                for (int k = 0; k < WR - 1; ++k) acc[k] = acc[k + 1];
                acc[WR - 1].x = R(0);
                acc[WR - 1].y = R(0);
                ++r0;
            }
            const int sx = lane - ox;
            if (BOPT) {
                constexpr int S = W + 1;
                if (sx >= 0 && sx < S) {
                    const int i = meta[p * 3 + 2];
                    const cx<R> cv = cst[p];
                    const cx<R>* cf = J.coef + (size_t)i * S * S + sx;
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        const cx<R> b = cf[k * S];
                        acc[k].x += b.re * cv.re + b.im * cv.im;   // conj(b) f
                        acc[k].y += b.re * cv.im - b.im * cv.re;
                    }
                }
            } else {
                const bool in = (sx >= 0) && (sx < W);
                const R wx = in ? psx[p * WE + (in ? sx : 0)] : R(0);
                const cx<R>* cp = cy + p * WE;
                if constexpr (F32) {
                    // two complex coefficients per 16-byte broadcast load, one packed
                    // two-wide FMA per row
                    const float4* cp4 = reinterpret_cast<const float4*>(cp);
                    const float2 ww = make_float2(wx, wx);
#pragma unroll
                    for (int k2 = 0; k2 < WE / 2; ++k2) {
                        const float4 c = cp4[k2];
                        acc[2 * k2] = __ffma2_rn(make_float2(c.x, c.y), ww, acc[2 * k2]);
                        if (2 * k2 + 1 < W) acc[2 * k2 + 1] = __ffma2_rn(make_float2(c.z, c.w), ww, acc[2 * k2 + 1]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        const cx<R> c = cp[k];
                        acc[k].x += c.re * wx;
                        acc[k].y += c.im * wx;
                    }
                }
            }
        }
    }
    // remaining rows (including rows no point reached)
    while (r0 < P) {
        if (col_ok) dst[(size_t)r0 * P + lane] = mk<R>(acc[0].x, acc[0].y);
#pragma unroll
        for (int k = 0; k < WR - 1; ++k) acc[k] = acc[k + 1];
        acc[WR - 1].x = R(0);
        acc[WR - 1].y = R(0);
        ++r0;
    }
}

// ---------------------------------------------------------------------------------------
// Three-dimensional spreading (window modes), tiles of 8^3 cells.  One warp per work item,
// the item's padded tile of P^3 cells (P = 8 + 2m + 1) in shared memory.  Lane l takes
// the (z, x) tap pairs q = l + 32 r of a point (W^2 pairs, ceil(W^2 / 32) rounds) and
// holds the W cells of each pair along y in registers, adding (c_j psi_y) psi_z psi_x.
// The items' points are sorted by base cell: while consecutive points share their base
// cell the registers keep accumulating; when it changes, the lanes store their cells,
// meet at a __syncwarp and load the cells of the new base.  Each cell is summed in the
// item's point order (deterministic, no atomics) and shared memory is touched once per
// base cell rather than once per point.
// The z-planes of the shared tile are PZ >= P^2 cells apart with PZ = W (mod 16), so the
// cells of 16 consecutive pairs, at q + const (mod 16) in 8-byte units, fall into
// distinct bank pairs: no bank conflicts.  The tile is written out densely (P^3).
__host__ __device__ constexpr int spread3d_plane(int P, int W) { return P * P + (((W - P * P) % 16) + 16) % 16; }
constexpr int SPREAD3D_T = 8;

template <class R, int MM>
__global__ void __launch_bounds__(64) k_spread3d(const __grid_constant__ JobSet<R> js) {
    constexpr int W = 2 * MM + 1;
    constexpr int WE = W + 1;                  // even stride of the staged rows
    constexpr int NR = (W * W + 31) / 32;      // rounds over the (z, x) pairs
    constexpr int T = SPREAD3D_T;
    constexpr int P = T + 2 * MM + 1, P2 = P * P;
    constexpr int PZ = spread3d_plane(P, W), SC = P * PZ;
    constexpr bool F32 = sizeof(R) == 4;
    using V2 = typename std::conditional<F32, float2, double2>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gitem = blockIdx.x * js.wpb + warp;
    if (gitem >= js.pre_items[js.njobs]) return;
    const int jb = find_job(js.pre_items, js.njobs, gitem);
    const Job<R>& J = js.job[jb];
    const int it = gitem - js.pre_items[jb];
    const int4 item = J.items[it];
    const int Ms = J.Ms, nt = J.ntile;

    unsigned char* base = smem_raw + (size_t)warp * js.smem_per_warp;
    V2* pad = reinterpret_cast<V2*>(base);                             // [P][PZ]
    V2* cyv = pad + ((SC + 1) & ~1);                                   // [32][WE] c_j psi_y
    R* psz = reinterpret_cast<R*>(cyv + 32 * WE);                      // [32][WE]
    R* psx = psz + 32 * WE;                                            // [32][WE]
    int* meta = reinterpret_cast<int*>(psx + 32 * WE);                 // [32] base cell in the shared tile
    float* poly = reinterpret_cast<float*>(meta + 32);                 // window polynomial (float32 plans)
    const bool use_poly = F32 && J.wpoly != nullptr;
    if (use_poly) {
        for (int e = lane; e < (WPOLY_DEG + 1) * wpoly_stride(W); e += 32) poly[e] = J.wpoly[e];
    }
    for (int e = lane; e < SC; e += 32) { pad[e].x = R(0); pad[e].y = R(0); }

    const int tz = item.x / (nt * nt), ty = (item.x / nt) % nt, tx = item.x % nt;
    const int logMs = 31 - __clz(Ms);
    int off[NR], sz[NR], sx[NR];
    bool ok[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int q = lane + 32 * r;
        ok[r] = q < W * W;
        sz[r] = ok[r] ? q / W : 0;
        sx[r] = ok[r] ? q % W : 0;
        off[r] = sz[r] * PZ + sx[r];
    }
    V2 v[NR][W];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int s = 0; s < W; ++s) { v[r][s].x = R(0); v[r][s].y = R(0); }
    int cur = -1;

    for (int c0 = 0; c0 < item.z; c0 += 32) {
        const int np = min(32, item.z - c0);
        __syncwarp();
        if (lane < np) {
            const int i = item.y + c0 + lane;
            const int j = __ldg(J.perm + i);
            cx<R> fv = J.in[j];
            if (J.mode == INFFT_MODE_DCF) fv = mul(J.w[i], fv);
            const uint32_t cl = __ldg(J.cell + i);
            const int cxl = (int)(cl & (uint32_t)(Ms - 1));
            const int cyl = (int)((cl >> logMs) & (uint32_t)(Ms - 1));
            const int czl = (int)(cl >> (2 * logMs));
            meta[lane] = (czl - tz * T) * PZ + (cyl - ty * T) * P + (cxl - tx * T);
            const R uz = J.u[(size_t)i * 3 + 0], uy = J.u[(size_t)i * 3 + 1], ux = J.u[(size_t)i * 3 + 2];
            R wz[W], wy[W], wx[W];
            bool done = false;
            if constexpr (F32) {
                if (use_poly) {
                    poly_taps2<W>(poly, uz, uy, wz, wy);
                    poly_taps<W>(poly, ux, wx);
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    wz[s] = tap_weight<R>(J.window, uz, s, MM, J.inv_m, J.beta);
                    wy[s] = tap_weight<R>(J.window, uy, s, MM, J.inv_m, J.beta);
                    wx[s] = tap_weight<R>(J.window, ux, s, MM, J.inv_m, J.beta);
                }
            }
#pragma unroll
            for (int s = 0; s < W; ++s) {
                cyv[lane * WE + s].x = fv.re * wy[s];
                cyv[lane * WE + s].y = fv.im * wy[s];
                psz[lane * WE + s] = wz[s];
                psx[lane * WE + s] = wx[s];
            }
        }
        __syncwarp();
        for (int p = 0; p < np; ++p) {
            const int b0 = meta[p];
            if (b0 != cur) {   // uniform across the warp
                if (cur >= 0) {
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        if (ok[r]) {
#pragma unroll
                            for (int s = 0; s < W; ++s) pad[cur + off[r] + s * P] = v[r][s];
                        }
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if (ok[r]) {
#pragma unroll
                        for (int s = 0; s < W; ++s) v[r][s] = pad[b0 + off[r] + s * P];
                    }
                cur = b0;
            }
            V2 c[W];
#pragma unroll
            for (int s = 0; s < W; ++s) c[s] = cyv[p * WE + s];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const R w = psz[p * WE + sz[r]] * psx[p * WE + sx[r]];
                if constexpr (F32) {
                    const float2 ww = make_float2(w, w);
#pragma unroll
                    for (int s = 0; s < W; ++s) v[r][s] = __ffma2_rn(c[s], ww, v[r][s]);
                } else {
#pragma unroll
                    for (int s = 0; s < W; ++s) { v[r][s].x += c[s].x * w; v[r][s].y += c[s].y * w; }
                }
            }
        }
    }
    if (cur >= 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (ok[r]) {
#pragma unroll
                for (int s = 0; s < W; ++s) pad[cur + off[r] + s * P] = v[r][s];
            }
    }
    __syncwarp();
    V2* dst = reinterpret_cast<V2*>(J.padded) + (size_t)it * P2 * P;
    for (int z = 0; z < P; ++z)
        for (int e = lane; e < P2; e += 32) dst[(size_t)z * P2 + e] = pad[z * PZ + e];
}

template <class R, int D>
__device__ __forceinline__ cx<R> merged_cell(const Job<R>& J, long long cidx);

// ---------------------------------------------------------------------------------------
// Two-dimensional merge, one block per tile of T x T cells (T <= 16, T > m, Ms a multiple
// of T), one thread per cell.  Along an axis, the cell at offset r in tile t lies in the
// padded tile of t at r + m, of t - 1 at r + T + m when r <= m, and of t + 1 at
// r - T + m when r >= T - m (tile indices mod ntile): at most two sources per axis.
template <class R>
__global__ void __launch_bounds__(256) k_merge2d(const __grid_constant__ JobSet<R> js) {
    const int gblk = blockIdx.x;
    const int jb = find_job(js.pre_merge, js.njobs, gblk);
    const Job<R>& J = js.job[jb];
    const int T = J.T, m = J.m, P = J.P, nt = J.ntile, Ms = J.Ms;
    const int tile = gblk - js.pre_merge[jb];
    const int ty = tile / nt, tx = tile - ty * nt;
    const int r = threadIdx.x >> 4, c = threadIdx.x & 15;
    if (r >= T || c >= T) return;
    int yt[2], yo[2], xt[2], xo[2];
    int ny = 1, nx = 1;
    yt[0] = ty; yo[0] = r + m;
    xt[0] = tx; xo[0] = c + m;
    if (r <= m) { yt[1] = (ty - 1 + nt) % nt; yo[1] = r + T + m; ny = 2; }
    else if (r >= T - m) { yt[1] = (ty + 1) % nt; yo[1] = r - T + m; ny = 2; }
    if (c <= m) { xt[1] = (tx - 1 + nt) % nt; xo[1] = c + T + m; nx = 2; }
    else if (c >= T - m) { xt[1] = (tx + 1) % nt; xo[1] = c - T + m; nx = 2; }
    const size_t cells = (size_t)P * P;
    cx<R> acc = mk<R>(0, 0);
    for (int a = 0; a < ny; ++a) {
        for (int b = 0; b < nx; ++b) {
            const int tl = yt[a] * nt + xt[b];
            const int i0 = J.tile_items[tl], i1 = J.tile_items[tl + 1];
            const size_t off = (size_t)yo[a] * P + xo[b];
            for (int itm = i0; itm < i1; ++itm) acc = add(acc, J.padded[(size_t)itm * cells + off]);
        }
    }
    J.grid[(size_t)(ty * T + r) * Ms + tx * T + c] = acc;
}

// ---------------------------------------------------------------------------------------
// Three-dimensional merge, one block per tile of T^3 cells (T a power of two, m < T),
// threads striding over the tile's cells.  Along an axis the cell at offset r of tile t
// lies in the padded tile of t at r + m, of t - 1 at r + T + m when r <= m, and of t + 1
// at r - T + m when r >= T - m; with T <= 2m both neighbours can hold it.  Work items of
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
            if (r <= m) { st[a][ns[a]] = (t - 1 + nt) % nt; so[a][ns[a]] = r + T + m; ++ns[a]; }
            if (r >= T - m) { st[a][ns[a]] = (t + 1) % nt; so[a][ns[a]] = r - T + m; ++ns[a]; }
        }
        cx<R> acc = mk<R>(0, 0);
        for (int a = 0; a < ns[0]; ++a)
            for (int b = 0; b < ns[1]; ++b)
                for (int c = 0; c < ns[2]; ++c) {
                    const int tl = (st[0][a] * nt + st[1][b]) * nt + st[2][c];
                    const int i0 = __ldg(J.tile_items + tl), i1 = __ldg(J.tile_items + tl + 1);
                    const size_t off = ((size_t)so[0][a] * P + so[1][b]) * P + so[2][c];
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

template <class R, int D, bool FWD>
__global__ void __launch_bounds__(256) k_fft(const __grid_constant__ JobSet<R> js, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
    const int gblk = blockIdx.x;
    const int jb = find_job(js.pre_fft[pass], js.njobs, gblk);
    const Job<R>& J = js.job[jb];
    const int lb = gblk - js.pre_fft[pass][jb];
    const int Ms = J.Ms, M = J.M, L = js.L;
    const int t = FWD ? pass : D - 1 - pass;
    const long long A = ipow(Ms, t);
    const long long B = ipow(M, D - 1 - t);
    const int n = Ms;
    const int ns = n + (n >> 4);    // skewed line stride
    const int logn = 31 - __clz(n);
    const long long nlines = A * B;
    const long long q0 = (long long)lb * L;
    const bool lanes_b = (B >= L);  // consecutive lines are consecutive b: coalesce along b

    const cx<R>* src;
    cx<R>* dst;
    if (!FWD) {
        src = (pass == 0) ? J.grid : (pass == 1 ? J.tmp1 : J.tmp2);
        dst = (pass == D - 1) ? J.out : (pass == 0 ? J.tmp1 : J.tmp2);
    } else {
        src = (pass == 0) ? J.in : (pass == 1 ? J.tmp1 : J.tmp2);
        dst = (pass == D - 1) ? J.grid : (pass == 0 ? J.tmp1 : J.tmp2);
    }
    const int tid = threadIdx.x, nth = blockDim.x;

    if (!FWD) {
        for (int e = tid; e < L * n; e += nth) {
            int l, i;
            if (lanes_b) { l = e % L; i = e / L; } else { i = e & (n - 1); l = e >> logn; }
            const long long q = q0 + l;
            cx<R> v = mk<R>(0, 0);
            if (q < nlines) {
                const long long a = q / B, b = q - a * B;
                const long long g = (a * n + i) * B + b;
                v = src[g];
            }
            buf[l * ns + skew(bitrev(i, logn))] = v;
        }
    } else {
        for (int e = tid; e < L * ns; e += nth) buf[e] = mk<R>(0, 0);
        __syncthreads();
        for (int e = tid; e < L * M; e += nth) {
            int l, i;
            if (lanes_b) { l = e % L; i = e / L; } else { i = e % M; l = e / M; }
            const long long q = q0 + l;
            if (q < nlines) {
                const long long a = q / B, b = q - a * B;
                const cx<R> v = scale(src[(a * M + i) * B + b], J.dinv[i]);
                const int bin = mod_pos(i - M / 2, Ms);
                buf[l * ns + skew(bitrev(bin, logn))] = v;
            }
        }
    }
    __syncthreads();

    const int half_n = n >> 1;
    const int loghn = logn - 1;
    for (int lh = 0; lh < logn; ++lh) {   // butterflies of half-length 2^lh
        const int half = 1 << lh;
        for (int e = tid; e < L * half_n; e += nth) {
            const int l = e >> loghn, jj = e & (half_n - 1);
            const int grp = jj >> lh, pos = jj & (half - 1);
            const int i1 = grp * (half << 1) + pos, i2 = i1 + half;
            cx<R> w = J.tw[pos << (loghn - lh)];
            if (FWD) w.im = -w.im;
            cx<R>* row = buf + l * ns;
            const cx<R> a = row[skew(i1)];
            const cx<R> b = mul(w, row[skew(i2)]);
            row[skew(i1)] = add(a, b);
            row[skew(i2)] = sub(a, b);
        }
        __syncthreads();
    }

    if (!FWD) {
        for (int e = tid; e < L * M; e += nth) {
            int l, i;
            if (lanes_b) { l = e % L; i = e / L; } else { i = e % M; l = e / M; }
            const long long q = q0 + l;
            if (q < nlines) {
                const long long a = q / B, b = q - a * B;
                const int bin = mod_pos(i - M / 2, Ms);
                dst[(a * M + i) * B + b] = scale(buf[l * ns + skew(bin)], J.dinv[i]);
            }
        }
    } else {
        for (int e = tid; e < L * n; e += nth) {
            int l, i;
            if (lanes_b) { l = e % L; i = e / L; } else { i = e & (n - 1); l = e >> logn; }
            const long long q = q0 + l;
            if (q < nlines) {
                const long long a = q / B, b = q - a * B;
                dst[(a * n + i) * B + b] = buf[l * ns + skew(i)];
            }
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
    const int ntap = ipow(W, D);
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
            for (int t = 0; t < D; ++t) {
                const R u = J.u[(size_t)i * D + t];
                for (int s = 0; s < W; ++s) ps[t * W + s] = tap_weight<R>(J.window, u, s, m, J.inv_m, J.beta);
            }
            cx<R> acc = mk<R>(0, 0);
            for (int q = 0; q < ntap; ++q) {
                int r2 = q, idx = 0;
                R wgt = R(1);
                for (int t = D - 1; t >= 0; --t) {
                    const int s = r2 % W;
                    r2 /= W;
                    idx += (o[t] + s) * pstride[t];
                    wgt *= ps[t * W + s];
                }
                const cx<R> g = pad[idx];
                acc.re += wgt * g.re;
                acc.im += wgt * g.im;
            }
            J.out[__ldg(J.perm + i)] = acc;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Interpolation for d = 2, 3 with a fixed m: one warp per work item; the warp gathers the
// padded tile of the grid around its tile into shared memory, then every lane sums the
// W^d taps of one point in separable order (x innermost, then y, then z) and writes f_j
// in the caller's order.  Window values come from the float32 polynomial or the exact
// window (float64 plans).
template <class R, int D, int MM>
__global__ void __launch_bounds__(128) k_interp_t(const __grid_constant__ JobSet<R> js) {
    constexpr int W = 2 * MM + 1;
    constexpr bool F32 = sizeof(R) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gitem = blockIdx.x * js.wpb + warp;
    if (gitem >= js.pre_items[js.njobs]) return;
    const int jb = find_job(js.pre_items, js.njobs, gitem);
    const Job<R>& J = js.job[jb];
    const int4 item = J.items[gitem - js.pre_items[jb]];
    const int P = J.P, m = J.m, Ms = J.Ms, T = J.T, nt = J.ntile;
    const int cells = D == 3 ? P * P * P : P * P;
    unsigned char* base = smem_raw + (size_t)warp * js.smem_per_warp;
    cx<R>* pad = reinterpret_cast<cx<R>*>(base);
    float* poly = reinterpret_cast<float*>(pad + ((cells + 1) & ~1));
    const bool use_poly = F32 && J.wpoly != nullptr;
    if (use_poly) {
        for (int e = lane; e < (WPOLY_DEG + 1) * wpoly_stride(W); e += 32) poly[e] = J.wpoly[e];
    }
    int tz = 0, ty, tx;
    if (D == 3) { tz = item.x / (nt * nt); ty = (item.x / nt) % nt; tx = item.x % nt; }
    else { ty = item.x / nt; tx = item.x % nt; }
    const int Mmask = Ms - 1;  // Ms is a power of two
    for (int e = lane; e < cells; e += 32) {
        const int ox = e % P, r1 = e / P;
        const int oy = r1 % P, oz = r1 / P;
        const int gx = (tx * T - m + ox) & Mmask, gy = (ty * T - m + oy) & Mmask;
        size_t g = (size_t)gy * Ms + gx;
        if (D == 3) g += (size_t)((tz * T - m + oz) & Mmask) * Ms * Ms;
        pad[e] = J.grid[g];
    }
    __syncwarp();
    const int logMs = 31 - __clz(Ms);
    for (int c0 = 0; c0 < item.z; c0 += 32) {
        const int np = min(32, item.z - c0);
        if (lane >= np) continue;
        const int i = item.y + c0 + lane;
        const uint32_t cl = __ldg(J.cell + i);
        const int ox = (int)(cl & (uint32_t)Mmask) - tx * T;
        const int oy = (int)((cl >> logMs) & (uint32_t)Mmask) - ty * T;
        const int oz = D == 3 ? (int)(cl >> (2 * logMs)) - tz * T : 0;
        R wz[W], wy[W], wx[W];
        const R uy = J.u[(size_t)i * D + D - 2], ux = J.u[(size_t)i * D + D - 1];
        const R uz = D == 3 ? J.u[(size_t)i * D] : R(0);
        bool done = false;
        if constexpr (F32) {
            if (use_poly) {
                poly_taps2<W>(poly, uy, ux, wy, wx);
                if (D == 3) poly_taps<W>(poly, uz, wz);
                done = true;
            }
        }
        if (!done) {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                wy[s] = tap_weight<R>(J.window, uy, s, MM, J.inv_m, J.beta);
                wx[s] = tap_weight<R>(J.window, ux, s, MM, J.inv_m, J.beta);
                if (D == 3) wz[s] = tap_weight<R>(J.window, uz, s, MM, J.inv_m, J.beta);
            }
        }
        cx<R> acc = mk<R>(0, 0);
        const int NZ = D == 3 ? W : 1;
#pragma unroll 1
        for (int sz = 0; sz < NZ; ++sz) {
            cx<R> accy = mk<R>(0, 0);
            const cx<R>* plane = pad + (size_t)(oz + sz) * P * P;
#pragma unroll
            for (int sy = 0; sy < W; ++sy) {
                const cx<R>* row = plane + (oy + sy) * P + ox;
                cx<R> t = mk<R>(0, 0);
#pragma unroll
                for (int sx = 0; sx < W; ++sx) {
                    const cx<R> g = row[sx];
                    t.re += wx[sx] * g.re;
                    t.im += wx[sx] * g.im;
                }
                accy.re += wy[sy] * t.re;
                accy.im += wy[sy] * t.im;
            }
            const R wzs = D == 3 ? wz[sz] : R(1);
            acc.re += wzs * accy.re;
            acc.im += wzs * accy.im;
        }
        J.out[__ldg(J.perm + i)] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// host drivers

static int pick_lines(int n, size_t elem) {
    const size_t budget = 64 * 1024;
    int L = 1;
    while (L < 32 && (size_t)(2 * L) * n * elem <= budget) L *= 2;
    return L;
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
                blocks = (int)((lines + js.L - 1) / js.L);
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

// register-row spreading for d = 2 when every job has the same m (2..7) and P <= 32
template <class R, int MM, bool BOPT>
static infft_status launch_spread2d_m(JobSet<R>& js, cudaStream_t st) {
    constexpr int W = 2 * MM + 1;
    constexpr int WE = W + 1;
    size_t spw = 32 * WE * sizeof(cx<R>) + 32 * WE * sizeof(R) + 96 * sizeof(int) + 32 * sizeof(cx<R>) +
                 (WPOLY_DEG + 1) * wpoly_stride(W) * sizeof(float);
    spw = (spw + 15) & ~(size_t)15;
    js.smem_per_warp = (int)spw;
    js.wpb = 4;
    const int nitems = js.pre_items[js.njobs];
    if (nitems == 0) return INFFT_OK;
    const size_t smem = spw * js.wpb;
    INFFT_CUDA(cudaFuncSetAttribute(k_spread2d<R, MM, BOPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_spread2d<R, MM, BOPT><<<(nitems + js.wpb - 1) / js.wpb, 32 * js.wpb, smem, st>>>(js);
    INFFT_LAUNCHED();
    return INFFT_OK;
}

template <class R, bool BOPT>
static infft_status launch_spread2d(JobSet<R>& js, cudaStream_t st, int m) {
    switch (m) {
        case 2: return launch_spread2d_m<R, 2, BOPT>(js, st);
        case 3: return launch_spread2d_m<R, 3, BOPT>(js, st);
        case 4: return launch_spread2d_m<R, 4, BOPT>(js, st);
        case 5: return launch_spread2d_m<R, 5, BOPT>(js, st);
        case 6: return launch_spread2d_m<R, 6, BOPT>(js, st);
        default: return launch_spread2d_m<R, 7, BOPT>(js, st);
    }
}

template <class R>
static bool spread2d_eligible(const JobSet<R>& js, int* m_out, bool* bopt_out) {
    if (js.njobs < 1) return false;
    const int m = js.job[0].m;
    const bool bopt = js.job[0].mode == INFFT_MODE_BOPT;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        if (J.d != 2 || J.m != m || (J.mode == INFFT_MODE_BOPT) != bopt || J.P > 32) return false;
    }
    if (m < 2 || m > 7) return false;
    *m_out = m;
    *bopt_out = bopt;
    return true;
}

// three-dimensional spreading in window modes when every job has the same m (1..7)
template <class R, int MM>
static infft_status launch_spread3d_m(JobSet<R>& js, cudaStream_t st) {
    constexpr int W = 2 * MM + 1;
    constexpr int WE = W + 1;
    constexpr int P = SPREAD3D_T + 2 * MM + 1;
    const size_t cells = (size_t)P * spread3d_plane(P, W);
    size_t spw = ((cells + 1) & ~(size_t)1) * sizeof(cx<R>) + 32 * WE * (sizeof(cx<R>) + 2 * sizeof(R)) +
                 32 * sizeof(int) + (WPOLY_DEG + 1) * wpoly_stride(W) * sizeof(float);
    spw = (spw + 15) & ~(size_t)15;
    const size_t smem_cap = 200 * 1024;
    if (spw > smem_cap) {
        set_error("padded tile needs %zu bytes of shared memory", spw);
        return INFFT_EUNSUPPORTED;
    }
    js.smem_per_warp = (int)spw;
    js.wpb = spw > 48 * 1024 ? 1 : 2;
    const int nitems = js.pre_items[js.njobs];
    if (nitems == 0) return INFFT_OK;
    const size_t smem = spw * js.wpb;
    INFFT_CUDA(cudaFuncSetAttribute(k_spread3d<R, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_spread3d<R, MM><<<(nitems + js.wpb - 1) / js.wpb, 32 * js.wpb, smem, st>>>(js);
    INFFT_LAUNCHED();
    return INFFT_OK;
}

template <class R>
static bool spread3d_eligible(const JobSet<R>& js, int* m_out) {
    if (js.njobs < 1) return false;
    const int m = js.job[0].m;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        if (J.d != 3 || J.m != m || J.mode == INFFT_MODE_BOPT || J.T != SPREAD3D_T || J.T <= m) return false;
    }
    // the register-held cells fit without spilling up to m = 6 (float) / m = 5 (double)
    if (m < 1 || m > (sizeof(R) == 4 ? 6 : 5)) return false;
    *m_out = m;
    return true;
}

template <class R>
static infft_status launch_spread3d(JobSet<R>& js, cudaStream_t st, int m) {
    switch (m) {
        case 1: return launch_spread3d_m<R, 1>(js, st);
        case 2: return launch_spread3d_m<R, 2>(js, st);
        case 3: return launch_spread3d_m<R, 3>(js, st);
        case 4: return launch_spread3d_m<R, 4>(js, st);
        case 5: return launch_spread3d_m<R, 5>(js, st);
        default: return launch_spread3d_m<R, 6>(js, st);
    }
}

// pruned FFT passes with deconvolution, common to every spreading variant
template <class R, int D>
static infft_status launch_fft_adjoint(JobSet<R>& js, cudaStream_t st, cudaEvent_t* ev) {
    int maxMs = 0;
    for (int j = 0; j < js.njobs; ++j) maxMs = std::max(maxMs, js.job[j].Ms);
    const size_t fsmem = (size_t)js.L * (maxMs + maxMs / 16) * sizeof(cx<R>);
    INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    for (int p = 0; p < D; ++p) {
        k_fft<R, D, false><<<js.pre_fft[p][js.njobs], 256, fsmem, st>>>(js, p);
        INFFT_LAUNCHED();
        if (ev) INFFT_CUDA(cudaEventRecord(ev[3 + p], st));
    }
    return INFFT_OK;
}

template <class R, int D>
static infft_status launch_adjoint(JobSet<R>& js, cudaStream_t st, cudaEvent_t* ev) {
    fill_prefixes(js, D, false);
    if (ev) INFFT_CUDA(cudaEventRecord(ev[0], st));
    int m2 = 0;
    bool bopt2 = false;
    if (D == 2 && spread2d_eligible(js, &m2, &bopt2)) {
        const infft_status s2 = bopt2 ? launch_spread2d<R, true>(js, st, m2) : launch_spread2d<R, false>(js, st, m2);
        if (s2 != INFFT_OK) return s2;
        if (ev) INFFT_CUDA(cudaEventRecord(ev[1], st));
        // merge: one block per tile
        js.pre_merge[0] = 0;
        for (int j = 0; j < js.njobs; ++j) js.pre_merge[j + 1] = js.pre_merge[j] + js.job[j].ntile * js.job[j].ntile;
        k_merge2d<R><<<js.pre_merge[js.njobs], 256, 0, st>>>(js);
        INFFT_LAUNCHED();
        if (ev) INFFT_CUDA(cudaEventRecord(ev[2], st));
        return launch_fft_adjoint<R, D>(js, st, ev);
    }
    int m3 = 0;
    if (D == 3 && spread3d_eligible(js, &m3)) {
        INFFT_TRY(launch_spread3d<R>(js, st, m3));
        if (ev) INFFT_CUDA(cudaEventRecord(ev[1], st));
        js.pre_merge[0] = 0;
        for (int j = 0; j < js.njobs; ++j) {
            const int nt = js.job[j].ntile;
            js.pre_merge[j + 1] = js.pre_merge[j] + nt * nt * nt;
        }
        k_merge3d<R><<<js.pre_merge[js.njobs], 256, 0, st>>>(js);
        INFFT_LAUNCHED();
        if (ev) INFFT_CUDA(cudaEventRecord(ev[2], st));
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
    return launch_fft_adjoint<R, D>(js, st, ev);
}

template <class R, int D, int MM>
static infft_status launch_interp_t(JobSet<R>& js, cudaStream_t st) {
    int P = 0;
    for (int j = 0; j < js.njobs; ++j) P = std::max(P, js.job[j].P);
    const size_t cells = D == 3 ? (size_t)P * P * P : (size_t)P * P;
    size_t spw = ((cells + 1) & ~(size_t)1) * sizeof(cx<R>) + (WPOLY_DEG + 1) * wpoly_stride(2 * MM + 1) * sizeof(float);
    spw = (spw + 15) & ~(size_t)15;
    const size_t smem_cap = 200 * 1024;
    if (spw > smem_cap) {
        set_error("padded tile needs %zu bytes of shared memory", spw);
        return INFFT_EUNSUPPORTED;
    }
    js.smem_per_warp = (int)spw;
    js.wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (64 * 1024) / spw));
    const int nitems = js.pre_items[js.njobs];
    if (nitems == 0) return INFFT_OK;
    const size_t smem = spw * js.wpb;
    INFFT_CUDA(cudaFuncSetAttribute(k_interp_t<R, D, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_interp_t<R, D, MM><<<(nitems + js.wpb - 1) / js.wpb, 32 * js.wpb, smem, st>>>(js);
    INFFT_LAUNCHED();
    return INFFT_OK;
}

// interpolation with a fixed m for d = 2, 3 (all jobs the same m, tile edge a power of two)
template <class R, int D>
static bool interp_t_eligible(const JobSet<R>& js, int* m_out) {
    if (D < 2 || js.njobs < 1) return false;
    const int m = js.job[0].m;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        if (J.m != m || (J.T & (J.T - 1)) != 0 || (J.Ms & (J.Ms - 1)) != 0) return false;
    }
    if (m < 1 || m > 8) return false;
    *m_out = m;
    return true;
}

template <class R, int D>
static infft_status launch_interp(JobSet<R>& js, cudaStream_t st, int m) {
    switch (m) {
        case 1: return launch_interp_t<R, D, 1>(js, st);
        case 2: return launch_interp_t<R, D, 2>(js, st);
        case 3: return launch_interp_t<R, D, 3>(js, st);
        case 4: return launch_interp_t<R, D, 4>(js, st);
        case 5: return launch_interp_t<R, D, 5>(js, st);
        case 6: return launch_interp_t<R, D, 6>(js, st);
        case 7: return launch_interp_t<R, D, 7>(js, st);
        default: return launch_interp_t<R, D, 8>(js, st);
    }
}

template <class R, int D>
static infft_status launch_forward(JobSet<R>& js, cudaStream_t st) {
    fill_prefixes(js, D, true);
    int maxMs = 0;
    for (int j = 0; j < js.njobs; ++j) maxMs = std::max(maxMs, js.job[j].Ms);
    const size_t fsmem = (size_t)js.L * (maxMs + maxMs / 16) * sizeof(cx<R>);
    INFFT_CUDA(cudaFuncSetAttribute(k_fft<R, D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    for (int p = 0; p < D; ++p) {
        k_fft<R, D, true><<<js.pre_fft[p][js.njobs], 256, fsmem, st>>>(js, p);
        INFFT_LAUNCHED();
    }
    if constexpr (D >= 2) {
        int mi = 0;
        if (interp_t_eligible<R, D>(js, &mi)) return launch_interp<R, D>(js, st, mi);
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

template infft_status run_jobs<float>(const std::vector<Job<float>>&, cudaStream_t, bool, cudaEvent_t*);
template infft_status run_jobs<double>(const std::vector<Job<double>>&, cudaStream_t, bool, cudaEvent_t*);
template infft_status run_jobs<float>(const Job<float>*, size_t, cudaStream_t, bool, cudaEvent_t*);
template infft_status run_jobs<double>(const Job<double>*, size_t, cudaStream_t, bool, cudaEvent_t*);

}  // namespace infft
