// Density compensation weights (Algorithm 3.6, Corollary 3.4) by CG in float64.
//
// With A = A_{2M} (eq. matrix_A at degree 2M):
//  * |I_2M| <= N: the normal equations of the second kind A^T conj(A) v = e_0,
//    w = conj(A) v (eq. normal_equations_second_kind_double).  Writing u = conj(v)
//    they become A^* A u = e_0 and w = conj(A u): CG on the Hermitian operator
//    A^* A (an NFFT followed by an adjoint NFFT).
//  * |I_2M| > N: the normal equations of the first kind conj(A) A^T w = 1_N
//    (eq. normal_equations_first_kind_double).  With q = conj(w) they become
//    A A^* q = 1_N: CG on A A^* (adjoint NFFT followed by NFFT), w = conj(q).
// The products are float64 NFFTs of an internal plan at degree 2M (sigma = 2)
// whose point order is the parent plan's sorted order, so the resulting weights
// are already in the order the spreading kernels read them.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "internal.h"
#include "jobset.cuh"

namespace infft {


constexpr int RED_BLOCKS = 1024;
constexpr int RED_THREADS = 256;

// partial sums of sum_i conj(a_i) b_i over a fixed grid: deterministic
__global__ void __launch_bounds__(RED_THREADS) k_dot_partial(const cx<double>* __restrict__ a,
                                                             const cx<double>* __restrict__ b, long long n,
                                                             double* __restrict__ part) {
    __shared__ double sre[RED_THREADS], sim[RED_THREADS];
    double re = 0, im = 0;
    for (long long i = (long long)blockIdx.x * RED_THREADS + threadIdx.x; i < n; i += (long long)RED_BLOCKS * RED_THREADS) {
        const cx<double> x = a[i], y = b[i];
        re += x.re * y.re + x.im * y.im;
        im += x.re * y.im - x.im * y.re;
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sre[threadIdx.x] += sre[threadIdx.x + s];
            sim[threadIdx.x] += sim[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sre[0];
        part[2 * blockIdx.x + 1] = sim[0];
    }
}

// out[0..1] = sum of the partials (fixed order)
__global__ void k_dot_final(const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sre[RED_THREADS], sim[RED_THREADS];
    double re = 0, im = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) { re += part[2 * i]; im += part[2 * i + 1]; }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) { sre[threadIdx.x] += sre[threadIdx.x + s]; sim[threadIdx.x] += sim[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = sre[0]; out[1] = sim[0]; }
}

// CG scalars, all on the device: s[0] = rr, s[2] = <p, q>, s[4] = rr_new, s[6] = alpha,
// s[7] = beta, s[10] = smallest rr so far, s[11] = state (0 running, 1 converged, 2 NaN,
// 3 max_iter reached), s[12] = iterations taken, s[13] = (rel_tol ||b||)^2, s[14] = max_iter,
// s[15] = this iteration improved on s[10], s[16] = this iteration runs.  Every kernel of an
// iteration is a no-op once the state is no longer 0, so the host may queue several
// iterations between looks at the state.
__global__ void k_cg_begin(double* s) { s[16] = (s[11] == 0.0) ? 1.0 : 0.0; }
__global__ void k_cg_alpha(double* s) {
    if (s[16] == 0.0) return;
    s[6] = (s[2] != 0.0) ? s[0] / s[2] : 0.0;
}
__global__ void k_cg_end(double* s) {
    if (s[16] == 0.0) return;
    const double rn = s[4];
    s[12] += 1.0;
    if (!(rn == rn)) { s[11] = 2.0; s[15] = 0.0; return; }
    s[15] = (rn < s[10]) ? 1.0 : 0.0;
    if (rn < s[10]) s[10] = rn;
    s[7] = (s[0] != 0.0) ? rn / s[0] : 0.0;
    s[0] = rn;
    if (rn <= s[13]) s[11] = 1.0;
    else if (s[12] >= s[14]) s[11] = 3.0;
}

__global__ void k_cg_update_xr(cx<double>* __restrict__ x, cx<double>* __restrict__ r, const cx<double>* __restrict__ p,
                               const cx<double>* __restrict__ q, long long n, const double* __restrict__ s) {
    if (s[16] == 0.0) return;
    const double al = s[6];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] = add(x[i], scale(p[i], al));
        r[i] = sub(r[i], scale(q[i], al));
    }
}

// x_best = x when this iteration's residual is the smallest so far (the weights come from
// the best iterate, so that a capped CG never returns worse weights than an earlier step of
// the same run)
__global__ void k_cg_keep_best(const cx<double>* __restrict__ x, cx<double>* __restrict__ xb, long long n,
                               const double* __restrict__ s) {
    if (s[16] == 0.0 || s[15] == 0.0) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        xb[i] = x[i];
}

__global__ void k_cg_update_p(cx<double>* __restrict__ p, const cx<double>* __restrict__ r, long long n,
                              const double* __restrict__ s) {
    if (s[16] == 0.0 || s[11] != 0.0) return;
    const double be = s[7];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = add(r[i], scale(p[i], be));
}

// the CG's starting scalars: rr = ||b||^2, no best iterate yet (the first iteration always
// becomes the best: x0 = 0 itself is never returned), tolerance and iteration cap
__global__ void k_cg_init(double* s, double rel_tol, int max_iter) {
    s[10] = HUGE_VAL;
    s[11] = 0.0;
    s[12] = 0.0;
    s[13] = rel_tol * rel_tol * s[0];
    s[14] = (double)max_iter;
    s[15] = 0.0;
    s[16] = 1.0;
}

__global__ void k_conj(const cx<double>* __restrict__ a, cx<double>* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = conjg(a[i]);
}

__global__ void k_fill(cx<double>* __restrict__ a, long long n, cx<double> v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

// max_k |conj(r_k) - delta_{0,k}|, partial maxima per block
__global__ void __launch_bounds__(RED_THREADS) k_resid_partial(const cx<double>* __restrict__ r, long long n,
                                                               long long k0, double* __restrict__ part) {
    __shared__ double sm[RED_THREADS];
    double mx = 0;
    for (long long i = (long long)blockIdx.x * RED_THREADS + threadIdx.x; i < n; i += (long long)RED_BLOCKS * RED_THREADS) {
        double re = r[i].re, im = -r[i].im;
        if (i == k0) re -= 1.0;
        mx = fmax(mx, sqrt(re * re + im * im));
    }
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_max_final(const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sm[RED_THREADS];
    double mx = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) mx = fmax(mx, part[i]);
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}

// weights in sorted order -> caller order (complex128) and plan-precision sorted copy
template <class R>
__global__ void k_store_weights(const cx<double>* __restrict__ ws, const int* __restrict__ perm, int N,
                                cx<double>* __restrict__ master, cx<R>* __restrict__ sorted) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const cx<double> v = ws[i];
    master[perm[i]] = v;
    sorted[i] = mk<R>((R)v.re, (R)v.im);
}

template <class R>
__global__ void k_sort_weights(const cx<double>* __restrict__ master, const int* __restrict__ perm, int N,
                               cx<R>* __restrict__ sorted) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const cx<double> v = master[perm[i]];
    sorted[i] = mk<R>((R)v.re, (R)v.im);
}

// ---------------------------------------------------------------------------------------
// Toeplitz form of the second-kind products.  For A = A_2M (N x |I_2M|),
//   [A^* A]_{k,k'} = sum_j exp(-2 pi i (k - k') x_j) = t(k - k'),  k - k' in (-2M, 2M)^d,
// so A^* A u is a d-variate discrete convolution of t with u.  t on I_4M is obtained once
// from 2^d adjoint NFFTs at degree 2M of modulated unit samples,
//   t(s + k) = sum_j exp(-2 pi i s x_j) exp(-2 pi i k x_j),  s in {-M, M}^d, k in I_2M,
// and the convolution is a circular one of period L = 4M (u zero-padded):
//   A^* A u = crop_{I_2M} F_L^- ( c_hat .* F_L^+ u ),  c_hat = L^{-d} F_L^+ t,
// where F_L^+ / F_L^- are the unnormalised DFTs with sign + / - (the pruned FFT passes with
// unit deconvolution factors).  Each CG iteration is then two FFTs of L^d points instead of
// an NFFT and an adjoint NFFT.

// f_j = exp(-2 pi i sum_t s_t x_{j,t}), s_t = -M2/2 or +M2/2 by bit t of `bits`; each
// s_t x_t is exact (M2/2 is a power of two) and is reduced mod 1 before the sum
__global__ void k_modulate(const double* __restrict__ x, int N, int d, int M2, int bits, cx<double>* __restrict__ f) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double ph = 0.0;
    for (int t = 0; t < d; ++t) {
        const double st = ((bits >> t) & 1) ? 0.5 * M2 : -0.5 * M2;
        const double v = st * x[(size_t)j * d + t];
        ph += v - rint(v);
    }
    double sn, cs;
    sincospi(-2.0 * ph, &sn, &cs);
    f[j] = mk<double>(cs, sn);
}

// place the degree-2M result of shift `bits` into I_4M: entry (i_t)_t of h goes to
// (i_t + M2 bit_t)_t of t (C order, 2 M2 per axis)
__global__ void k_scatter_t(const cx<double>* __restrict__ h, int d, int M2, int bits, cx<double>* __restrict__ t) {
    long long K = 1;
    for (int q = 0; q < d; ++q) K *= M2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    long long rem = i, dst = 0, stride = 1;
    for (int q = d - 1; q >= 0; --q) {
        const int it = (int)(rem % M2);
        rem /= M2;
        dst += (long long)(it + (((bits >> q) & 1) ? M2 : 0)) * stride;
        stride *= 2LL * M2;
    }
    t[dst] = h[i];
}

__global__ void k_cmul(cx<double>* __restrict__ a, const cx<double>* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = mul(a[i], b[i]);
}

__global__ void k_fill_real(double* __restrict__ a, int n, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void k_twiddles(int L, cx<double>* __restrict__ tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L / 2) {
        double sn, cs;
        sincospi(2.0 * i / L, &sn, &cs);
        tw[i] = mk<double>(cs, -sn);
    }
}

struct ToeplitzOp {
    Job<double> fwd;     // u (I_2M) -> G (L^d), sign +
    Job<double> adj;     // G -> A^*A u (I_2M), sign -
    cx<double>* G = nullptr;
    const cx<double>* chat = nullptr;
    long long Ld = 0;
};

static infft_status nfft64(infft_plan_s* q, bool forward, const void* in, void* out, cudaStream_t st);

// Build the operator: t by 2^d modulated adjoint NFFTs of the degree-2M sub-plan, then c_hat.
static infft_status toeplitz_setup(const infft_plan_s* p, infft_plan_s* sub, int M2, cudaStream_t st,
                                   const std::function<void*(size_t)>& alloc, ToeplitzOp& op) {
    const int d = p->d, N = (int)p->N, L = 2 * M2;
    long long Ld = 1, K = 1;
    for (int t = 0; t < d; ++t) { Ld *= L; K *= M2; }
    cx<double>* G = (cx<double>*)alloc(Ld * 16);
    cx<double>* chat = (cx<double>*)alloc(Ld * 16);
    cx<double>* t1 = d >= 2 ? (cx<double>*)alloc(Ld * 16) : nullptr;
    cx<double>* t2 = d == 3 ? (cx<double>*)alloc(Ld * 16) : nullptr;
    cx<double>* fm = (cx<double>*)alloc((size_t)N * 16);
    cx<double>* hb = (cx<double>*)alloc(K * 16);
    cx<double>* tw = (cx<double>*)alloc((size_t)(L / 2) * 16);
    double* ones = (double*)alloc((size_t)M2 * 8);
    double* invL = (double*)alloc((size_t)L * 8);
    if (!G || !chat || (d >= 2 && !t1) || (d == 3 && !t2) || !fm || !hb || !tw || !ones || !invL) {
        set_error("Toeplitz buffers: out of device memory");
        return INFFT_ENOMEM;
    }
    k_twiddles<<<(L / 2 + 255) / 256, 256, 0, st>>>(L, tw);
    INFFT_LAUNCHED();
    k_fill_real<<<(M2 + 255) / 256, 256, 0, st>>>(ones, M2, 1.0);
    INFFT_LAUNCHED();
    k_fill_real<<<(L + 255) / 256, 256, 0, st>>>(invL, L, 1.0 / L);
    INFFT_LAUNCHED();
    // t on I_4M, stored in G
    for (int bits = 0; bits < (1 << d); ++bits) {
        k_modulate<<<(N + 255) / 256, 256, 0, st>>>(p->x64, N, d, M2, bits, fm);
        INFFT_LAUNCHED();
        INFFT_TRY(nfft64(sub, false, fm, hb, st));
        k_scatter_t<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(hb, d, M2, bits, G);
        INFFT_LAUNCHED();
    }
    Job<double> J;
    memset(&J, 0, sizeof(J));
    J.d = d; J.tw = tw; J.tmp1 = t1; J.tmp2 = t2;
    // c_hat = L^{-d} F_L^+ t: every frequency of I_4M is an input (M = Ms = L)
    J.M = L; J.Ms = L; J.dinv = invL; J.in = G; J.grid = chat;
    INFFT_TRY(run_fft_passes<double>(J, st, true));
    op.fwd = J;
    op.fwd.M = M2; op.fwd.dinv = ones; op.fwd.grid = G;
    op.adj = op.fwd;
    op.G = G;
    op.chat = chat;
    op.Ld = Ld;
    return INFFT_OK;
}

// q = A^* A p through the Toeplitz operator
static infft_status toeplitz_apply(ToeplitzOp& op, const cx<double>* pin, cx<double>* qout, cudaStream_t st) {
    op.fwd.in = pin;
    INFFT_TRY(run_fft_passes<double>(op.fwd, st, true));
    k_cmul<<<1024, 256, 0, st>>>(op.G, op.chat, op.Ld);
    INFFT_LAUNCHED();
    op.adj.out = qout;
    return run_fft_passes<double>(op.adj, st, false);
}

static infft_status nfft64(infft_plan_s* q, bool forward, const void* in, void* out, cudaStream_t st) {
    std::vector<Job<double>> jobs{make_job<double>(q, INFFT_MODE_PLAIN, in, out)};
    return run_jobs<double>(jobs, st, forward);
}

static infft_status dot(const cx<double>* a, const cx<double>* b, long long n, double* part, double* out,
                        cudaStream_t st) {
    k_dot_partial<<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, n, part);
    INFFT_LAUNCHED();
    k_dot_final<<<1, RED_THREADS, 0, st>>>(part, out);
    INFFT_LAUNCHED();
    return INFFT_OK;
}

static infft_status ensure_weight_buffers(infft_plan_s* p) {
    const size_t R_sz = p->fp64 ? 8 : 4;
    if (!p->w_master) INFFT_TRY(dev_alloc(p, &p->w_master, (size_t)p->N * 16));
    if (!p->w_sorted) INFFT_TRY(dev_alloc(p, &p->w_sorted, (size_t)p->N * 2 * R_sz));
    return INFFT_OK;
}

static infft_status weights_impl(infft_plan_s* p, int max_iter, double rel_tol, int m_cg, unsigned opts,
                                 double* residual_inf, int* iters_out, cudaStream_t st, std::vector<void*>& tmp,
                                 infft_plan_s*& sub) {
    const int d = p->d, M2 = 2 * p->M;
    const int N = (int)p->N;
    if (m_cg <= 0) m_cg = (d <= 2) ? 8 : 4;
    const int Ms2 = 2 * M2;
    m_cg = std::min(m_cg, (Ms2 - 2) / 2);
    INFFT_TRY(plan_create(d, M2, N, p->x64, 2.0, m_cg, INFFT_FP64 | INFFT_WIN_KB, st, true, &sub));
    long long K = 1;
    for (int t = 0; t < d; ++t) K *= M2;
    const bool second_kind = K <= N;
    // Toeplitz products need the second kind and FFT lines of 4M <= 4096 points
    const bool toeplitz_ok = second_kind && 2 * M2 <= 4096;
    if ((opts & INFFT_WEIGHTS_TOEPLITZ) && !toeplitz_ok) {
        set_error("Toeplitz CG needs (2M)^d <= N and 4M <= 4096");
        return INFFT_EUNSUPPORTED;
    }
    const bool toeplitz = toeplitz_ok && !(opts & INFFT_WEIGHTS_NFFT);
    const long long n = second_kind ? K : N;   // CG unknowns
    const long long aux_n = second_kind ? N : K;
    // temporaries from the library's stream-ordered pool: no device-wide synchronisation
    auto alloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (pool_alloc(&q, bytes, st) != INFFT_OK) return nullptr;
        tmp.push_back(q);
        return q;
    };
    cx<double>* x = (cx<double>*)alloc(n * 16);
    cx<double>* xb = (cx<double>*)alloc(n * 16);
    cx<double>* r = (cx<double>*)alloc(n * 16);
    cx<double>* pv = (cx<double>*)alloc(n * 16);
    cx<double>* qv = (cx<double>*)alloc(n * 16);
    cx<double>* aux = (cx<double>*)alloc(std::max(aux_n, (long long)N) * 16);
    cx<double>* ws = (cx<double>*)alloc((size_t)N * 16);
    cx<double>* kv = (cx<double>*)alloc(K * 16);
    double* part = (double*)alloc(2 * RED_BLOCKS * 8);
    double* sc = (double*)alloc(32 * 8);
    if (!x || !xb || !r || !pv || !qv || !aux || !ws || !kv || !part || !sc) {
        set_error("CG buffers: out of device memory");
        return INFFT_ENOMEM;
    }
    const int eb = 1024, et = 256;
    ToeplitzOp top;
    if (toeplitz) INFFT_TRY(toeplitz_setup(p, sub, M2, st, [&](size_t b) { return alloc(b); }, top));
    // x = x_best = 0; r = b; p = b
    INFFT_CUDA(cudaMemsetAsync(x, 0, n * 16, st));
    INFFT_CUDA(cudaMemsetAsync(xb, 0, n * 16, st));
    if (second_kind) {
        INFFT_CUDA(cudaMemsetAsync(r, 0, n * 16, st));
        long long k0 = 0;
        for (int t = 0; t < d; ++t) k0 = k0 * M2 + M2 / 2;
        k_fill<<<1, 1, 0, st>>>(r + k0, 1, mk<double>(1.0, 0.0));
        INFFT_LAUNCHED();
    } else {
        k_fill<<<eb, et, 0, st>>>(r, n, mk<double>(1.0, 0.0));
        INFFT_LAUNCHED();
    }
    INFFT_CUDA(cudaMemcpyAsync(pv, r, n * 16, cudaMemcpyDeviceToDevice, st));
    INFFT_TRY(dot(r, r, n, part, sc + 0, st));  // rr = ||b||^2
    k_cg_init<<<1, 1, 0, st>>>(sc, rel_tol, max_iter);
    INFFT_LAUNCHED();

    // Iterations are queued in chunks of up to eight; the device's state flag makes the
    // queued iterations after convergence no-ops, and the host reads the state once per chunk
    // (no synchronisation inside a chunk).
    int queued = 0;
    double state[3] = {0, 0, 0};   // state, iterations, best rr
    while (queued < max_iter) {
        const int chunk = std::min(8, max_iter - queued);
        for (int c = 0; c < chunk; ++c) {
            k_cg_begin<<<1, 1, 0, st>>>(sc);
            INFFT_LAUNCHED();
            // q = op(p)
            if (toeplitz) {
                INFFT_TRY(toeplitz_apply(top, pv, qv, st));   // A^* A p as a convolution
            } else if (second_kind) {
                INFFT_TRY(nfft64(sub, true, pv, aux, st));    // A p   (K -> N)
                INFFT_TRY(nfft64(sub, false, aux, qv, st));   // A^* (A p)
            } else {
                INFFT_TRY(nfft64(sub, false, pv, aux, st));   // A^* p (N -> K)
                INFFT_TRY(nfft64(sub, true, aux, qv, st));    // A (A^* p)
            }
            INFFT_TRY(dot(pv, qv, n, part, sc + 2, st));
            k_cg_alpha<<<1, 1, 0, st>>>(sc);
            INFFT_LAUNCHED();
            k_cg_update_xr<<<eb, et, 0, st>>>(x, r, pv, qv, n, sc);
            INFFT_LAUNCHED();
            INFFT_TRY(dot(r, r, n, part, sc + 4, st));
            k_cg_end<<<1, 1, 0, st>>>(sc);
            INFFT_LAUNCHED();
            k_cg_keep_best<<<eb, et, 0, st>>>(x, xb, n, sc);
            INFFT_LAUNCHED();
            k_cg_update_p<<<eb, et, 0, st>>>(pv, r, n, sc);
            INFFT_LAUNCHED();
        }
        queued += chunk;
        INFFT_TRY(read_back(state, sc + 10, 3 * 8, st));
        if (state[1] != 0.0) break;
    }
    if (state[1] == 2.0) { set_error("CG breakdown (NaN)"); return INFFT_ENOTCONV; }
    bool conv = state[1] == 1.0;
    const int it = (int)state[2];
    x = xb;   // the weights come from the iterate of smallest residual
    // weights in sorted order
    if (second_kind) {
        INFFT_TRY(nfft64(sub, true, x, aux, st));  // A u
        k_conj<<<eb, et, 0, st>>>(aux, ws, N);
    } else {
        k_conj<<<eb, et, 0, st>>>(x, ws, N);
    }
    INFFT_LAUNCHED();
    INFFT_TRY(ensure_weight_buffers(p));
    if (p->fp64)
        k_store_weights<double><<<(N + 255) / 256, 256, 0, st>>>(ws, p->perm, N, (cx<double>*)p->w_master,
                                                                 (cx<double>*)p->w_sorted);
    else
        k_store_weights<float><<<(N + 255) / 256, 256, 0, st>>>(ws, p->perm, N, (cx<double>*)p->w_master,
                                                                (cx<float>*)p->w_sorted);
    INFFT_LAUNCHED();
    p->has_weights = true;
    if (residual_inf) {
        // A^T w = conj(A^* conj(w)) on I_2M
        k_conj<<<eb, et, 0, st>>>(ws, aux, N);
        INFFT_LAUNCHED();
        INFFT_TRY(nfft64(sub, false, aux, kv, st));
        long long k0 = 0;
        for (int t = 0; t < d; ++t) k0 = k0 * M2 + M2 / 2;
        k_resid_partial<<<RED_BLOCKS, RED_THREADS, 0, st>>>(kv, K, k0, part);
        INFFT_LAUNCHED();
        k_max_final<<<1, RED_THREADS, 0, st>>>(part, sc + 8);
        INFFT_LAUNCHED();
        INFFT_TRY(read_back(residual_inf, sc + 8, 8, st));
    }
    INFFT_CUDA(cudaStreamSynchronize(st));
    if (iters_out) *iters_out = it;
    if (fault(FAULT_CG)) conv = false;   // injected: report non-convergence (weights stored)
    if (!conv) {
        set_error("CG did not reach rel_tol %g in %d iterations", rel_tol, max_iter);
        return INFFT_ENOTCONV;
    }
    return INFFT_OK;
}

}  // namespace infft

using namespace infft;

extern "C" {

infft_status infft_weights_opts(infft_plan_t p, int max_iter, double rel_tol, int m_cg, unsigned opts,
                                double* residual_inf, int* iters, void* stream) {
    if (!p || max_iter < 1 || !(rel_tol >= 0)) { set_error("invalid weights arguments"); return INFFT_EINVAL; }
    if ((opts & ~(unsigned)(INFFT_WEIGHTS_NFFT | INFFT_WEIGHTS_TOEPLITZ)) ||
        ((opts & INFFT_WEIGHTS_NFFT) && (opts & INFFT_WEIGHTS_TOEPLITZ))) {
        set_error("invalid weights options %u", opts);
        return INFFT_EINVAL;
    }
    std::vector<void*> tmp;
    infft_plan_s* sub = nullptr;
    p->pool_stream = (cudaStream_t)stream;
    infft_status s = weights_impl(p, max_iter, rel_tol, m_cg, opts, residual_inf, iters, (cudaStream_t)stream, tmp, sub);
    // temporaries and the degree-2M plan go back to the pool in stream order
    for (void* q : tmp) pool_free(q, (cudaStream_t)stream);
    if (sub) plan_release(sub);
    cudaStreamSynchronize((cudaStream_t)stream);
    return s;
}

infft_status infft_weights(infft_plan_t p, int max_iter, double rel_tol, int m_cg, double* residual_inf, int* iters,
                           void* stream) {
    return infft_weights_opts(p, max_iter, rel_tol, m_cg, 0u, residual_inf, iters, stream);
}

infft_status infft_set_weights(infft_plan_t p, const void* w, void* stream) {
    if (!p || !w) { set_error("null argument"); return INFFT_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    p->pool_stream = st;
    INFFT_TRY(ensure_weight_buffers(p));
    const bool dev = is_device_pointer(w);
    INFFT_CUDA(cudaMemcpyAsync(p->w_master, w, (size_t)p->N * 16, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    const int N = (int)p->N;
    if (p->fp64)
        k_sort_weights<double><<<(N + 255) / 256, 256, 0, st>>>((const cx<double>*)p->w_master, p->perm, N,
                                                                (cx<double>*)p->w_sorted);
    else
        k_sort_weights<float><<<(N + 255) / 256, 256, 0, st>>>((const cx<double>*)p->w_master, p->perm, N,
                                                               (cx<float>*)p->w_sorted);
    INFFT_LAUNCHED();
    INFFT_CUDA(cudaStreamSynchronize(st));
    p->has_weights = true;
    return INFFT_OK;
}

infft_status infft_get_weights(infft_plan_t p, void* w, void* stream) {
    if (!p || !w) { set_error("null argument"); return INFFT_EINVAL; }
    if (!p->has_weights) { set_error("no weights"); return INFFT_ESTATE; }
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = is_device_pointer(w);
    INFFT_CUDA(cudaMemcpyAsync(w, p->w_master, (size_t)p->N * 16, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    INFFT_CUDA(cudaStreamSynchronize(st));
    return INFFT_OK;
}

}  // extern "C"
