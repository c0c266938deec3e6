// Two-dimensional spreading kernel (register rows) and its launcher, instantiated for
// float32 and float64 in their own translation units (compiled in parallel).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "spread.cuh"

namespace infft {

// Float32 window modes with m <= 4 spread two points at a time, one per half-warp: lane l
// owns columns 2 (l mod 16) and 2 (l mod 16) + 1 for the points of its half, and the two
// halves' partial sums of a cell are added when its row is stored.  A 16-byte load of
// broadcast coefficients costs two shared-memory wavefronts either way, so each then
// serves two points; shared-memory wavefronts bound this kernel.
template <class R, int MM, bool BOPT>
__host__ __device__ constexpr bool spread2d_pair() { return sizeof(R) == 4 && !BOPT && MM <= 4; }
template <class R>
constexpr bool spread2d_pair_m(int m) { return sizeof(R) == 4 && m <= 4; }   // window modes
// row pitch of the staged psi_x: odd (33) when each lane reads one column, even (34) for
// the 8-byte column pairs of the paired form
template <class R, int MM, bool BOPT>
__host__ __device__ constexpr int spread2d_pitch() { return spread2d_pair<R, MM, BOPT>() ? 34 : 33; }

// row stride (complex elements) of the staged c_j psi_y: W in the paired form, whose rows are
// read with 8-byte broadcasts (an odd stride of 8-byte words: the staging stores of 32 lanes
// hit distinct banks), W + 1 elsewhere, whose rows are read with 16-byte broadcasts
template <class R, int MM, bool BOPT>
__host__ __device__ constexpr int spread2d_we() { return spread2d_pair<R, MM, BOPT>() ? 2 * MM + 1 : 2 * MM + 2; }

// bytes of the per-warp prefetch slots (w, u pairs, perm, cell of 32 points); a multiple of 16
template <class R, bool PF>
__host__ __device__ constexpr size_t spread2d_slot_bytes() {
    return PF ? 32 * (sizeof(cx<R>) + 2 * sizeof(R) + 2 * sizeof(int)) : 0;
}

// ---------------------------------------------------------------------------------------
// Two-dimensional spreading with the accumulators in registers.  One warp per work
// item; lane l owns column l of the item's P x P padded tile (P = T + 2m, one more for
// B_opt slots; P <= 32), or a column pair in the paired form above.
// The item's points are sorted by base row, so the rows a point can touch,
// [oy, oy + 2m] (padded coordinates; one more row for B_opt slots), only move down:
// each lane keeps those rows of its column in registers, adds the point's taps
// (coefficient c_j psi_y[k] broadcast, times psi_x of its column), and when the next
// point starts lower it stores the rows that no later point can reach.  Every padded
// cell is stored exactly once, no shared-memory read-modify-write, no atomics.
// Window values are computed once per point while staging 32 points per warp.  With PF
// (window modes: the paired form, and grids too small to hide load latency) the sorted
// data of the next 32 points (perm, cell, u, w) are copied to shared memory with cp.async
// while the current ones are spread, so that staging waits only on the gather of the
// samples f.
// One warp spreads work item gitem (global over the JobSet's jobs); `base` is the warp's
// shared memory.  The body of k_spread2d, and the spread units of the persistent d = 2 kernel.
template <class R, int MM, bool BOPT, bool PF>
__device__ __forceinline__ void spread2d_item(const JobSet<R>& js, const int gitem, unsigned char* base) {
    constexpr int W = 2 * MM + 1;              // window taps per axis
    constexpr int WE = spread2d_we<R, MM, BOPT>();   // stride of the staged rows
    constexpr int WR = BOPT ? W + 1 : W;       // rows held in registers
    constexpr bool F32 = sizeof(R) == 4;
    constexpr bool PAIR = spread2d_pair<R, MM, BOPT>();
    constexpr int PX = spread2d_pitch<R, MM, BOPT>();
    constexpr int NC = PAIR ? 2 : 1;           // columns per lane
    const int lane = threadIdx.x & 31;
    const int jb = find_job(js.pre_items, js.njobs, gitem);
    const Job<R>& J = js.job[jb];
    const int it = gitem - js.pre_items[jb];
    const int4 item = J.items[it];
    const int P = J.P, Ms = J.Ms, T = J.T;

    // prefetch slots (PF only): lane l copies, and later reads, the data of its own point only
    cx<R>* pf_w = reinterpret_cast<cx<R>*>(base);               // [32]    w (DCF)
    R* pf_u = reinterpret_cast<R*>(pf_w + 32);                  // [32][2] fractional offsets
    int* pf_perm = reinterpret_cast<int*>(pf_u + 64);           // [32]    caller's index
    uint32_t* pf_cell = reinterpret_cast<uint32_t*>(pf_perm + 32);  // [32] base cell
    cx<R>* cy = reinterpret_cast<cx<R>*>(base + spread2d_slot_bytes<R, PF>());  // [32][WE] c_j psi_y (window mode)
    // psi_x of each staged point laid out by padded column, zero off the point's taps, so
    // that each lane reads its columns' weights directly (conflict-free both ways)
    R* psx = reinterpret_cast<R*>(cy + 32 * WE);            // [32][PX] psi_x by column
    int* meta = reinterpret_cast<int*>(psx + 32 * PX);      // [32][3]  oy, ox, sorted index
    cx<R>* cst = reinterpret_cast<cx<R>*>(meta + 96);       // [32]     c_j (B_opt mode)
    float* poly = reinterpret_cast<float*>(cst + 32);       // [(WPOLY_DEG+1) * WP] window polynomial (16-byte rows)
    // the paired form evaluates the taps from the parameter block when every job shares one
    // window polynomial (js.wtab_ok), else from a copy in shared memory
    const bool tab_param = PAIR && js.wtab_ok;
    const bool use_poly = F32 && !BOPT && J.wpoly != nullptr;
    if (use_poly && !tab_param) {
        for (int e = lane; e < (WPOLY_DEG + 1) * wpoly_stride(W); e += 32) poly[e] = J.wpoly[e];
    }

    const int ty = item.x / J.ntile, tx = item.x % J.ntile;
    using V2 = typename std::conditional<F32, float2, double2>::type;
    // (re, im) of the rows r0 .. r0 + WR - 1 of this lane's columns: acc[NC k + c] is row
    // r0 + k of the lane's column c
    V2 acc[NC * WR];
#pragma unroll
    for (int k = 0; k < NC * WR; ++k) { acc[k].x = R(0); acc[k].y = R(0); }
    int r0 = 0;  // padded row held in acc[0 .. NC - 1]
    int old_ox = -1;   // first column of this lane's taps in its psi_x row, -1: row not zeroed yet
    cx<R>* dst = J.padded + (size_t)it * P * P;
    const bool col_ok = lane < P;
    // store row r0 (no later point reaches it) and move the held rows up by one
    auto flush_row = [&]() {
        if constexpr (PAIR) {
            float4 v = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
            v.x += __shfl_xor_sync(0xffffffffu, v.x, 16);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, 16);
            v.z += __shfl_xor_sync(0xffffffffu, v.z, 16);
            v.w += __shfl_xor_sync(0xffffffffu, v.w, 16);
            // P and the item's base are even: the column pair is 16-byte aligned
            if (lane < 16 && 2 * lane < P) *reinterpret_cast<float4*>(dst + (size_t)r0 * P + 2 * lane) = v;
        } else {
            if (col_ok) dst[(size_t)r0 * P + lane] = mk<R>(acc[0].x, acc[0].y);
        }
#pragma unroll
        for (int k = 0; k < NC * (WR - 1); ++k) acc[k] = acc[k + NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) { acc[NC * (WR - 1) + c].x = R(0); acc[NC * (WR - 1) + c].y = R(0); }
        ++r0;
    };
    const int logMs = 31 - __clz(Ms);
    const bool dcf = J.mode == INFFT_MODE_DCF;
    auto prefetch = [&](int c) {   // the sorted data of points c .. c + 31 of the item
        if (c + lane < item.z) {
            const size_t i = (size_t)item.y + c + lane;
            cp_async<4>(pf_perm + lane, J.perm + i);
            cp_async<4>(pf_cell + lane, J.cell + i);
            if (!BOPT) {
                cp_async<2 * sizeof(R)>(pf_u + 2 * lane, J.u + 2 * i);
                if (dcf) cp_async<sizeof(cx<R>)>(pf_w + lane, J.w + i);
            }
        }
        cp_async_commit();
    };
    if (PF && item.z > 0) prefetch(0);

    for (int c0 = 0; c0 < item.z; c0 += 32) {
        const int np = min(32, item.z - c0);
        __syncwarp();
        if (PF) cp_async_wait_all();
        if (lane < np) {
            const int i = item.y + c0 + lane;
            const int j = PF ? pf_perm[lane] : __ldg(J.perm + i);
            cx<R> fv = J.in[j];
            if (dcf) fv = mul(PF ? pf_w[lane] : J.w[i], fv);
            const uint32_t cl = PF ? pf_cell[lane] : __ldg(J.cell + i);
            const int cxl = (int)(cl & (uint32_t)(Ms - 1)), cyl = (int)(cl >> logMs);
            meta[lane * 3 + 0] = cyl - ty * T;
            meta[lane * 3 + 1] = cxl - tx * T;
            meta[lane * 3 + 2] = i;
            if (BOPT) {
                cst[lane] = fv;
            } else {
                const R uy = PF ? pf_u[2 * lane + 0] : J.u[(size_t)i * 2 + 0];
                const R ux = PF ? pf_u[2 * lane + 1] : J.u[(size_t)i * 2 + 1];
                R wy[W], wx[W];
                bool done = false;
                if constexpr (F32) {
                    if (tab_param) {
                        poly_taps2<W>(js.wtab, uy, ux, wy, wx);
                        done = true;
                    } else if (use_poly) {
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
                R* row = psx + lane * PX;
                // the row is zero off the taps the lane wrote last time: clear those only
                if (old_ox < 0) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) row[c] = R(0);
                } else {
#pragma unroll
                    for (int s = 0; s < W; ++s) row[old_ox + s] = R(0);
                }
                const int oxl = cxl - tx * T;   // ox + s <= T - 1 + 2m = P - 1 < 32
                old_ox = oxl;
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    cy[lane * WE + s] = scale(fv, wy[s]);
                    row[oxl + s] = wx[s];
                }
                if (WE > W) cy[lane * WE + W] = mk<R>(0, 0);   // the pad the 16-byte row loads read
            }
        }
        __syncwarp();   // orders every read of the prefetch slots before their refill
        if (PF && c0 + 32 < item.z) prefetch(c0 + 32);
        // The points are sorted by base row, so the chunk splits into runs of equal oy
        // (found by one ballot): the rows above a run are stored once per run, and the
        // points of a run only add their taps.  A test of the rows held per point cost
        // selects over all the accumulators on every point (batched d = 2, m = 4: spread
        // 0.505 -> 0.428 ms).
        const int my_oy = lane < np ? meta[lane * 3 + 0] : 0x7fffffff;
        int p = 0;
        while (p < np) {
            const int oy = __shfl_sync(0xffffffffu, my_oy, p);
            // store the rows above oy: no later point reaches them
            while (r0 < oy) flush_row();
            const int q = 32 - __clz(__ballot_sync(0xffffffffu, my_oy == oy));
            if constexpr (PAIR) {
                // points p + h of each pair go to half h; at an odd run end the second
                // half adds zeros (the first point's taps times a zero weight)
                const int half = lane >> 4, hl = lane & 15;
#pragma unroll 2
                for (; p < q; p += 2) {
                    const int pp = p + half;
                    const bool act = pp < q;
                    const int pr = act ? pp : p;
                    float2 wv = *reinterpret_cast<const float2*>(psx + pr * PX + 2 * hl);
                    if (!act) wv = make_float2(0.f, 0.f);
                    const float2 wa = make_float2(wv.x, wv.x), wb = make_float2(wv.y, wv.y);
                    // one 8-byte broadcast per row: the two halves read two points' rows in
                    // one wavefront
                    const float2* cp2 = reinterpret_cast<const float2*>(cy + pr * WE);
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        const float2 c = cp2[k];
                        acc[2 * k] = __ffma2_rn(c, wa, acc[2 * k]);
                        acc[2 * k + 1] = __ffma2_rn(c, wb, acc[2 * k + 1]);
                    }
                }
                p = q;
                continue;
            }
            // float32: four points per unrolled step let the loads of the next points
            // overlap the current FMAs (0.573 -> 0.506 ms before the runs); float64 keeps
            // its registers for the accumulators
            constexpr int UNR = F32 ? 4 : 1;
#pragma unroll UNR
            for (; p < q; ++p) {
                if (BOPT) {
                    constexpr int S = W + 1;
                    const int ox = meta[p * 3 + 1];
                    const int sx = lane - ox;
                    // every lane loads (a column of the point's S x S block, clamped), and the
                    // lanes outside the block add zero: with no branch around the loads the
                    // unrolled points' coefficient loads are in flight together
                    const bool act = sx >= 0 && sx < S;
                    const int sxc = min(max(sx, 0), S - 1);
                    const int i = meta[p * 3 + 2];
                    const cx<R> cv = act ? cst[p] : mk<R>(0, 0);
                    const cx<R>* cf = J.coef + (size_t)i * S * S + sxc;
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        const V2 b = __ldg(reinterpret_cast<const V2*>(cf + k * S));
                        acc[k].x += b.x * cv.re + b.y * cv.im;   // conj(b) f
                        acc[k].y += b.x * cv.im - b.y * cv.re;
                    }
                } else {
                    const R wx = psx[p * PX + lane];
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
    }
    // remaining rows (including rows no point reached)
    while (r0 < P) flush_row();
}

template <class R, int MM, bool BOPT, bool PF>
// the paired form holds 2 (2m + 1) complex accumulators: at most 96 registers, so five 4-warp
// blocks (20 warps) share an SM (the one-point form ran six at 80 registers)
__global__ void __launch_bounds__(128, spread2d_pair<R, MM, BOPT>() ? 5 : 1)
    k_spread2d(const __grid_constant__ JobSet<R> js) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int gitem = blockIdx.x * js.wpb + warp;
    if (gitem >= js.pre_items[js.njobs]) return;
    spread2d_item<R, MM, BOPT, PF>(js, gitem, smem_raw + (size_t)warp * js.smem_per_warp);
}

// Per-launch setup of the register-row spread: shared memory per warp (js.smem_per_warp), four
// warps per block (js.wpb), and the jobs' common window polynomial in the parameter block.
template <class R, int MM, bool BOPT, bool PF>
static void spread2d_setup(JobSet<R>& js) {
    constexpr int W = 2 * MM + 1;
    constexpr int WE = spread2d_we<R, MM, BOPT>();
    size_t spw = spread2d_slot_bytes<R, PF>() + 32 * WE * sizeof(cx<R>) + 32 * spread2d_pitch<R, MM, BOPT>() * sizeof(R) + 96 * sizeof(int) + 32 * sizeof(cx<R>) +
                 (WPOLY_DEG + 1) * wpoly_stride(W) * sizeof(float);
    // one window polynomial for every job: into the parameter block
    js.wtab_ok = 0;
    if (spread2d_pair<R, MM, BOPT>() && wpoly_stride(W) <= 12) {
        const size_t n = (size_t)(WPOLY_DEG + 1) * wpoly_stride(W);
        bool same = js.job[0].wpoly_h != nullptr;
        for (int j = 1; j < js.njobs && same; ++j)
            same = js.job[j].wpoly_h && memcmp(js.job[j].wpoly_h, js.job[0].wpoly_h, n * sizeof(float)) == 0;
        if (same) {
            memcpy(js.wtab, js.job[0].wpoly_h, n * sizeof(float));
            js.wtab_ok = 1;
        }
    }
    spw = (spw + 15) & ~(size_t)15;
    js.smem_per_warp = (int)spw;
    js.wpb = 4;
}

// register-row spreading for d = 2 when every job has the same m (2..8) and P <= 32
template <class R, int MM, bool BOPT, bool PF>
static infft_status launch_spread2d_m(JobSet<R>& js, cudaStream_t st) {
    spread2d_setup<R, MM, BOPT, PF>(js);
    const size_t spw = (size_t)js.smem_per_warp;
    const int nitems = js.pre_items[js.njobs];
    if (nitems == 0) return INFFT_OK;
    const size_t smem = spw * js.wpb;
    INFFT_CUDA(cudaFuncSetAttribute(k_spread2d<R, MM, BOPT, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_spread2d<R, MM, BOPT, PF><<<(nitems + js.wpb - 1) / js.wpb, 32 * js.wpb, smem, st>>>(js);
    INFFT_LAUNCHED();
    return INFFT_OK;
}

template <class R, bool BOPT, bool PF>
static infft_status launch_spread2d(JobSet<R>& js, cudaStream_t st, int m) {
    switch (m) {
        case 2: return launch_spread2d_m<R, 2, BOPT, PF>(js, st);
        case 3: return launch_spread2d_m<R, 3, BOPT, PF>(js, st);
        case 4: return launch_spread2d_m<R, 4, BOPT, PF>(js, st);
        case 5: return launch_spread2d_m<R, 5, BOPT, PF>(js, st);
        case 6: return launch_spread2d_m<R, 6, BOPT, PF>(js, st);
        case 7: return launch_spread2d_m<R, 7, BOPT, PF>(js, st);
        default: return launch_spread2d_m<R, 8, BOPT, PF>(js, st);
    }
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// The paired form (float32, m <= 4) always prefetches (batched d = 2, m = 4: spread 0.389 ->
// 0.383 ms); the one-point forms prefetch only when there are fewer work items than eight
// warps per SM (with many items, other warps hide the staging's load latency and the copies
// cost more than they save: 0.428 -> 0.444 ms for the one-point float32 form).  Either way
// the copies must be aligned element by element.  INFFT_SPREAD2D_PREFETCH=0 or 1 picks the
// form regardless (both give the same sums in the same order).
template <class R>
static bool spread2d_prefetch(const JobSet<R>& js, int m) {
    // the first job's plan tuning (1 on, 2 off) comes first, then the environment
    const int env = js.job[0].prefetch == 1 ? 1 : js.job[0].prefetch == 2 ? 0 : env_form("INFFT_SPREAD2D_PREFETCH");
    if (env == 0) return false;
    if (env != 1 && !spread2d_pair_m<R>(m)) {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (js.pre_items[js.njobs] >= 8 * nsm) return false;
    }
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        if (!aligned(J.perm, 4) || !aligned(J.cell, 4) || !aligned(J.u, 2 * sizeof(R)) ||
            (J.mode == INFFT_MODE_DCF && !aligned(J.w, sizeof(cx<R>))))
            return false;
    }
    return true;
}

template <class R>
static bool spread2d_eligible(const JobSet<R>& js, int* m_out, bool* bopt_out) {
    if (js.njobs < 1) return false;
    const int m = js.job[0].m;
    const bool bopt = js.job[0].mode == INFFT_MODE_BOPT;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        if (J.d != 2 || J.m != m || (J.mode == INFFT_MODE_BOPT) != bopt || J.P > 32) return false;
        // the two-source halo merge that follows needs P <= 2T, i.e. 2m <= T (2m + 1 <= T with
        // B_opt's extra slot): a tuned tile of 8 at m >= 5 (m >= 4 with B_opt) puts some cells
        // in three tiles along an axis, which the generic path handles
        if (J.P > 2 * J.T) return false;
        if (!bopt && spread2d_pair_m<R>(m) && (J.P & 1)) return false;   // paired rows: 16-byte stores
    }
    if (m < 2 || m > 8) return false;   // m = 8 with window taps only: P = 16 + 16 <= 32
    *m_out = m;
    *bopt_out = bopt;
    return true;
}

template <class R>
infft_status spread2d_try(JobSet<R>& js, cudaStream_t st, bool* used) {
    int m = 0;
    bool bopt = false;
    *used = false;
    if (!spread2d_eligible(js, &m, &bopt)) return INFFT_OK;
    *used = true;
    if (bopt) return launch_spread2d<R, true, false>(js, st, m);
    return spread2d_prefetch(js, m) ? launch_spread2d<R, false, true>(js, st, m)
                                 : launch_spread2d<R, false, false>(js, st, m);
}

}  // namespace infft
