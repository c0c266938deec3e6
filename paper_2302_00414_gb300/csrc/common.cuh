// Shared device/host definitions of the iNFFT library (sm_103a).
//
// Notation follows Sections 2-4 of Kircheis & Potts: d dimensions, degree M,
// oversampled grid M_sigma ("Ms"), truncation m, points x_j (j = 1..N).
// Grid cells are stored at l mod Ms along every axis, C order (first axis
// slowest); coefficients k in I_M at k + M/2, C order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/infft.h"

namespace infft {

// ----------------------------------------------------------------------------------------
// complex numbers of float or double
template <class R>
struct alignas(2 * sizeof(R)) cx {
    R re, im;
};

template <class R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <class R>
__host__ __device__ __forceinline__ cx<R> add(cx<R> a, cx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> sub(cx<R> a, cx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> mul(cx<R> a, cx<R> b) {
    return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R>
__host__ __device__ __forceinline__ cx<R> mulconj(cx<R> a, cx<R> b) {  // conj(a) * b
    return mk<R>(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <class R>
__host__ __device__ __forceinline__ cx<R> scale(cx<R> a, R s) { return mk<R>(a.re * s, a.im * s); }
template <class R>
__host__ __device__ __forceinline__ cx<R> conjg(cx<R> a) { return mk<R>(a.re, -a.im); }

// ----------------------------------------------------------------------------------------
// Kaiser-Bessel window in grid units (Section 2.1 with the I0 form of the window):
//   phi(delta) = I0(beta sqrt(1 - (delta/m)^2)) for |delta| <= m, 0 otherwise,
// delta = M_sigma x - l, beta = pi m (2 - M/M_sigma).  The closed support is used:
// |delta| = m is inside.
__device__ __forceinline__ float bessel_i0(float z) { return cyl_bessel_i0f(z); }
__device__ __forceinline__ double bessel_i0(double z) { return cyl_bessel_i0(z); }

template <class R>
__device__ __forceinline__ R kb_phi(R delta, R inv_m, R beta) {
    R t = delta * inv_m;
    R s = R(1) - t * t;
    return (s >= R(0)) ? bessel_i0(beta * sqrt(s)) : R(0);
}

// centred cardinal B-spline of order 2m evaluated at delta (grid units), by the
// Cox-de Boor recursion on the uniform knots -m..m; used for the B-spline window
// (eq. window_bspline).  Only small orders are supported (2m <= 16).
template <class R>
__device__ __forceinline__ R bspline_phi(R delta, int m) {
    const int n = 2 * m;
    R y = delta + R(m);  // shift to [0, n)
    if (!(y >= R(0) && y < R(n))) return R(0);
    R b[17];
    int cell = (int)floor(y);
    for (int i = 0; i < n; ++i) b[i] = (i == cell) ? R(1) : R(0);
    for (int k = 1; k < n; ++k) {
        for (int i = 0; i < n - k; ++i) {
            R left = (y - R(i)) / R(k);
            R right = (R(i + k + 1) - y) / R(k);
            b[i] = left * b[i] + right * b[i + 1];
        }
    }
    return b[0];
}

enum WindowKind { WK_KB = 0, WK_BSPLINE = 1, WK_DIRICHLET = 2 };

template <class R>
__device__ __forceinline__ R window_phi(int kind, R delta, int m, R inv_m, R beta) {
    if (kind == WK_BSPLINE) return bspline_phi<R>(delta, m);
    return kb_phi<R>(delta, inv_m, beta);
}

// Window value of tap s = 0..2m of a point with fractional offset u = M_sigma x - b in
// [0, 1] (b = floor(M_sigma x)); the tap sits at l = b - m + s, delta = u + m - s.
// Membership in the index set (eq. indexset_x) is decided exactly: taps 1..2m always
// satisfy |delta| <= m, tap 0 only when u = 0 (the point on a grid node).
template <class R>
__device__ __forceinline__ R tap_weight(int kind, R u, int s, int m, R inv_m, R beta) {
    if (s == 0 && u != R(0)) return R(0);
    return window_phi<R>(kind, u + R(m - s), m, inv_m, beta);
}

// Float32 plans evaluate the Kaiser-Bessel taps s = 1..2m from per-plan polynomials:
// phi(u + m - s) = sum_k c[k][s] v^k, v = 2u - 1, u in [0, 1], degree WPOLY_DEG, obtained
// by Chebyshev interpolation in float64 at plan creation (piecewise-polynomial kernel
// evaluation in the manner of Barnett, Magland and af Klinteberg, SIAM J. Sci. Comput.
// 2019).  Degree 10 reaches the float32 rounding level of the window.  Tap 0 keeps the
// exact membership rule: I0(0) = 1 on a grid node, 0 otherwise.
constexpr int WPOLY_DEG = 10;

// row stride of the coefficient table: taps padded to a multiple of 4 (16-byte rows)
__host__ __device__ constexpr int wpoly_stride(int W) { return (W + 3) & ~3; }

template <int W>
__device__ __forceinline__ void poly_taps(const float* __restrict__ c, float u, float* out) {
    constexpr int WP = wpoly_stride(W);
    const float v = 2.f * u - 1.f;
#pragma unroll
    for (int s = 1; s < W; ++s) out[s] = c[WPOLY_DEG * WP + s];
#pragma unroll
    for (int k = WPOLY_DEG - 1; k >= 0; --k) {
#pragma unroll
        for (int s = 1; s < W; ++s) out[s] = fmaf(out[s], v, c[k * WP + s]);
    }
    out[0] = (u == 0.f) ? 1.f : 0.f;
}

// the taps of two coordinates at once, each coefficient row read with 16-byte loads
// (c must be 16-byte aligned)
template <int W>
__device__ __forceinline__ void poly_taps2(const float* __restrict__ c, float u0, float u1, float* o0, float* o1) {
    constexpr int WP = wpoly_stride(W);
    // Horner on both coordinates at once: one packed two-wide FMA per tap and degree
    const float2 vv = make_float2(2.f * u0 - 1.f, 2.f * u1 - 1.f);
    float2 a[WP];
#pragma unroll
    for (int q = 0; q < WP / 4; ++q) {
        const float4 t = reinterpret_cast<const float4*>(c + WPOLY_DEG * WP)[q];
        a[4 * q] = make_float2(t.x, t.x); a[4 * q + 1] = make_float2(t.y, t.y);
        a[4 * q + 2] = make_float2(t.z, t.z); a[4 * q + 3] = make_float2(t.w, t.w);
    }
#pragma unroll
    for (int k = WPOLY_DEG - 1; k >= 0; --k) {
#pragma unroll
        for (int q = 0; q < WP / 4; ++q) {
            const float4 t = reinterpret_cast<const float4*>(c + k * WP)[q];
            if (4 * q < W) a[4 * q] = __ffma2_rn(a[4 * q], vv, make_float2(t.x, t.x));
            if (4 * q + 1 < W) a[4 * q + 1] = __ffma2_rn(a[4 * q + 1], vv, make_float2(t.y, t.y));
            if (4 * q + 2 < W) a[4 * q + 2] = __ffma2_rn(a[4 * q + 2], vv, make_float2(t.z, t.z));
            if (4 * q + 3 < W) a[4 * q + 3] = __ffma2_rn(a[4 * q + 3], vv, make_float2(t.w, t.w));
        }
    }
#pragma unroll
    for (int s = 1; s < W; ++s) { o0[s] = a[s].x; o1[s] = a[s].y; }
    o0[0] = (u0 == 0.f) ? 1.f : 0.f;
    o1[0] = (u1 == 0.f) ? 1.f : 0.f;
}

// ----------------------------------------------------------------------------------------
// Work descriptors.  One Job describes one transform (one plan, one in/out pair);
// kernels receive an array of Jobs with the same d and precision and map their
// blocks onto the jobs through prefix sums.
template <class R>
struct Job {
    int d, M, Ms, m;
    int N, T, ntile, P;        // T tile edge, ntile tiles per axis, P = T + 2m + 1 padded edge
    int nitems, window;        // work items (tile, start, count); window kind
    int mode;                  // INFFT_MODE_*
    int S;                     // B_opt slots per axis (2m+2)
    int prefetch, fused_fft;   // the plan's tuning of these choices (0 = library default)
    R beta, inv_m;
    const int* perm;           // sorted position -> caller's index
    const uint32_t* cell;      // row-major wrapped base cell of each sorted point
    const R* u;                // N*d fractional offsets M_sigma x - floor(M_sigma x)
    const cx<R>* w;            // weights in sorted order (DCF)
    const cx<R>* coef;         // B_opt coefficients, sorted order, N*S^d (BOPT)
    const int4* items;         // (tile, start, count, 0)
    const int* tile_items;     // ntile^d + 1 prefix of items per tile
    const R* dinv;             // M entries 1/(Ms w^(k)) (per axis)
    const float* wpoly;        // (WPOLY_DEG + 1) x (2m+1) window polynomial (float32 KB plans) or null
    const float* wpoly_h;      // host copy of the same table (read by the launchers only) or null
    const cx<R>* tw;           // Ms/2 twiddles exp(-2 pi i k / Ms)
    cx<R>* padded;             // nitems * P^d
    cx<R>* grid;               // Ms^d
    cx<R>* tmp1;               // FFT intermediates
    cx<R>* tmp2;
    const cx<R>* in;           // adjoint: f (N), forward: fhat (M^d)
    cx<R>* out;                // adjoint: fhat (M^d), forward: f (N)
};

// ----------------------------------------------------------------------------------------
// small helpers
__host__ __device__ __forceinline__ int ipow(int b, int e) {
    int r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

__device__ __forceinline__ int find_job(const int* prefix, int njobs, int idx) {
    // largest j with prefix[j] <= idx (prefix has njobs+1 entries, prefix[0] = 0)
    int lo = 0, hi = njobs;  // invariant prefix[lo] <= idx < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= idx) lo = mid; else hi = mid;
    }
    return lo;
}

__host__ __device__ __forceinline__ int mod_pos(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ int bitrev(int i, int logn) {
    return (int)(__brev((unsigned)i) >> (32 - logn));
}

}  // namespace infft
