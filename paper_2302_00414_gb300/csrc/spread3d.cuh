// Three-dimensional spreading kernel (register-held cells per base cell) and its launcher,
// instantiated for float32 and float64 in their own translation units (compiled in parallel).
#pragma once

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "spread.cuh"

namespace infft {

// ---------------------------------------------------------------------------------------
// Three-dimensional spreading (window modes), tiles of 8^3 cells.  One warp per work item,
// the item's padded tile of P^3 cells (P = 8 + 2m, the window's taps) in shared memory.  Lane l takes
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
// With PF the sorted data of the next chunk of points (perm, cell, u, w) are copied to shared
// memory with cp.async while the current ones are spread: with five warps per SM, other
// warps cannot hide the staging's global loads.
__host__ __device__ constexpr int spread3d_plane(int P, int W) { return P * P + (((W - P * P) % 16) + 16) % 16; }
constexpr int SPREAD3D_T = 8;

// points staged per chunk: 16 for float32 with m <= 4, so that a warp's tile and staging fit
// six warps in an SM's shared memory (with 32 they fit five); 32 otherwise
template <class R, int MM>
__host__ __device__ constexpr int spread3d_chunk() { return (sizeof(R) == 4 && MM <= 4) ? 16 : 32; }

// bytes of the per-warp prefetch slots (w, u triples, perm, cell of a chunk); a multiple of 16
template <class R, int MM, bool PF>
__host__ __device__ constexpr size_t spread3d_slot_bytes() {
    return PF ? spread3d_chunk<R, MM>() * (sizeof(cx<R>) + 3 * sizeof(R) + 2 * sizeof(int)) : 0;
}

template <class R, int MM, bool PF>
__global__ void __launch_bounds__(64) k_spread3d(const __grid_constant__ JobSet<R> js) {
    constexpr int W = 2 * MM + 1;
    constexpr int WE = W + 1;                  // even stride of the staged rows
    constexpr int NR = (W * W + 31) / 32;      // rounds over the (z, x) pairs
    constexpr int T = SPREAD3D_T;
    constexpr int P = T + 2 * MM, P2 = P * P;   // the padded edge of window modes
    constexpr int PZ = spread3d_plane(P, W), SC = P * PZ;
    constexpr bool F32 = sizeof(R) == 4;
    constexpr int CH = spread3d_chunk<R, MM>();
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
    // prefetch slots (PF only): lane l copies, and later reads, the data of its own point only
    cx<R>* pf_w = reinterpret_cast<cx<R>*>(base);                      // [CH]    w (DCF)
    R* pf_u = reinterpret_cast<R*>(pf_w + CH);                         // [CH][3] fractional offsets
    int* pf_perm = reinterpret_cast<int*>(pf_u + 3 * CH);              // [CH]    caller's index
    uint32_t* pf_cell = reinterpret_cast<uint32_t*>(pf_perm + CH);     // [CH]    base cell
    V2* pad = reinterpret_cast<V2*>(base + spread3d_slot_bytes<R, MM, PF>());  // [P][PZ]
    V2* cyv = pad + ((SC + 1) & ~1);                                   // [CH][WE] c_j psi_y
    R* psz = reinterpret_cast<R*>(cyv + CH * WE);                      // [CH][WE]
    R* psx = psz + CH * WE;                                            // [CH][WE]
    int* meta = reinterpret_cast<int*>(psx + CH * WE);                 // [CH] base cell in the shared tile
    float* poly = reinterpret_cast<float*>(meta + CH);                 // window polynomial (float32 plans)
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
    const bool dcf = J.mode == INFFT_MODE_DCF;
    auto prefetch = [&](int c) {   // the sorted data of points c .. c + CH - 1 of the item
        if (lane < CH && c + lane < item.z) {
            const size_t i = (size_t)item.y + c + lane;
            cp_async<4>(pf_perm + lane, J.perm + i);
            cp_async<4>(pf_cell + lane, J.cell + i);
#pragma unroll
            for (int a = 0; a < 3; ++a) cp_async<sizeof(R)>(pf_u + 3 * lane + a, J.u + 3 * i + a);
            if (dcf) cp_async<sizeof(cx<R>)>(pf_w + lane, J.w + i);
        }
        cp_async_commit();
    };
    if (PF && item.z > 0) prefetch(0);

    for (int c0 = 0; c0 < item.z; c0 += CH) {
        const int np = min(CH, item.z - c0);
        __syncwarp();
        if (PF) cp_async_wait_all();
        if (lane < np) {
            const int i = item.y + c0 + lane;
            const int j = PF ? pf_perm[lane] : __ldg(J.perm + i);
            cx<R> fv = J.in[j];
            if (dcf) fv = mul(PF ? pf_w[lane] : J.w[i], fv);
            const uint32_t cl = PF ? pf_cell[lane] : __ldg(J.cell + i);
            const int cxl = (int)(cl & (uint32_t)(Ms - 1));
            const int cyl = (int)((cl >> logMs) & (uint32_t)(Ms - 1));
            const int czl = (int)(cl >> (2 * logMs));
            meta[lane] = (czl - tz * T) * PZ + (cyl - ty * T) * P + (cxl - tx * T);
            const R uz = PF ? pf_u[3 * lane + 0] : J.u[(size_t)i * 3 + 0];
            const R uy = PF ? pf_u[3 * lane + 1] : J.u[(size_t)i * 3 + 1];
            const R ux = PF ? pf_u[3 * lane + 2] : J.u[(size_t)i * 3 + 2];
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
        __syncwarp();   // orders every read of the prefetch slots before their refill
        if (PF && c0 + CH < item.z) prefetch(c0 + CH);
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

// three-dimensional spreading in window modes when every job has the same m (1..6)
template <class R, int MM, bool PF>
static infft_status launch_spread3d_m(JobSet<R>& js, cudaStream_t st) {
    constexpr int W = 2 * MM + 1;
    constexpr int WE = W + 1;
    constexpr int P = SPREAD3D_T + 2 * MM;
    const size_t cells = (size_t)P * spread3d_plane(P, W);
    constexpr int CH = spread3d_chunk<R, MM>();
    size_t spw = spread3d_slot_bytes<R, MM, PF>() +
                 ((cells + 1) & ~(size_t)1) * sizeof(cx<R>) + CH * WE * (sizeof(cx<R>) + 2 * sizeof(R)) +
                 CH * sizeof(int) + (WPOLY_DEG + 1) * wpoly_stride(W) * sizeof(float);
    spw = (spw + 15) & ~(size_t)15;
    const size_t smem_cap = 200 * 1024;
    if (spw > smem_cap) {
        set_error("padded tile needs %zu bytes of shared memory", spw);
        return INFFT_EUNSUPPORTED;
    }
    js.smem_per_warp = (int)spw;
    js.wpb = 1;   // one warp per block packs the 34-40 KB tiles tightest: 5 warps per SM at m = 4
    const int nitems = js.pre_items[js.njobs];
    if (nitems == 0) return INFFT_OK;
    const size_t smem = spw * js.wpb;
    INFFT_CUDA(cudaFuncSetAttribute(k_spread3d<R, MM, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the tiles bound the warps per SM: ask for all of the SM's unified memory as shared memory
    INFFT_CUDA(cudaFuncSetAttribute(k_spread3d<R, MM, PF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
    k_spread3d<R, MM, PF><<<(nitems + js.wpb - 1) / js.wpb, 32 * js.wpb, smem, st>>>(js);
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

template <class R, bool PF>
static infft_status launch_spread3d(JobSet<R>& js, cudaStream_t st, int m) {
    switch (m) {
        case 1: return launch_spread3d_m<R, 1, PF>(js, st);
        case 2: return launch_spread3d_m<R, 2, PF>(js, st);
        case 3: return launch_spread3d_m<R, 3, PF>(js, st);
        case 4: return launch_spread3d_m<R, 4, PF>(js, st);
        case 5: return launch_spread3d_m<R, 5, PF>(js, st);
        default: return launch_spread3d_m<R, 6, PF>(js, st);
    }
}

static bool aligned3(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// The prefetching form runs unless INFFT_SPREAD3D_PREFETCH=0 (both forms give the same sums
// in the same order) or a copy it would make is misaligned.
template <class R>
static bool spread3d_prefetch(const JobSet<R>& js) {
    // the first job's plan tuning (1 on, 2 off) comes first, then the environment
    if (js.job[0].prefetch == 2 || (js.job[0].prefetch == 0 && env_form("INFFT_SPREAD3D_PREFETCH") == 0)) return false;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        if (!aligned3(J.perm, 4) || !aligned3(J.cell, 4) || !aligned3(J.u, sizeof(R)) ||
            (J.mode == INFFT_MODE_DCF && !aligned3(J.w, sizeof(cx<R>))))
            return false;
    }
    return true;
}

template <class R>
infft_status spread3d_try(JobSet<R>& js, cudaStream_t st, bool* used) {
    int m = 0;
    *used = false;
    if (!spread3d_eligible(js, &m)) return INFFT_OK;
    *used = true;
    return spread3d_prefetch(js) ? launch_spread3d<R, true>(js, st, m) : launch_spread3d<R, false>(js, st, m);
}

}  // namespace infft
