// Interpolation kernels with a fixed m for d = 2, 3 (Algorithm 2.1 step 3) and their
// launcher, included by one translation unit per dimension.
#pragma once

#include <algorithm>

#include "spread.cuh"

namespace infft {

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
        if (J.m != m || J.mode == INFFT_MODE_BOPT || (J.T & (J.T - 1)) != 0 || (J.Ms & (J.Ms - 1)) != 0) return false;
    }
    // float64 d = 2 up to the CG's m = 8; otherwise m <= 6
    if (m < 1 || m > ((D == 2 && sizeof(R) == 8) ? 8 : 6)) return false;
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
        default:
            if constexpr (D == 2 && sizeof(R) == 8) {
                if (m == 7) return launch_interp_t<R, D, 7>(js, st);
                return launch_interp_t<R, D, 8>(js, st);
            }
            set_error("no fixed-m interpolation for m = %d", m);
            return INFFT_EUNSUPPORTED;
    }
}

template <class R, int D>
infft_status interp_try_d(JobSet<R>& js, cudaStream_t st, bool* used) {
    int m = 0;
    *used = false;
    if (!interp_t_eligible<R, D>(js, &m)) return INFFT_OK;
    *used = true;
    return launch_interp<R, D>(js, st, m);
}

}  // namespace infft
