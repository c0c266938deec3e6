// Optimisation of the sparse matrix B (Algorithm 4.3) in float64.
//
// For every column l of B (one cell of the oversampled grid) the nonzeros b_l solve
// the least-squares problem of eq. opt_overdet_columnwise through its normal
// equations G_l b_l = v_l (eq. solution_overdet):
//   G_l = H_l^* H_l, entries prod_t (D_{M/2-1}(x_h - x_j) + exp(-M pi i (x_h - x_j)))
//         with D_{M/2-1}(u) = sin((M-1) pi u)/sin(pi u)   (eq. matrix_normal_equations_overdet)
//   v_l = (prod_t V(x_{j,t} - l_t/M_sigma))_j, V(y) = sum_{k in I_M} w^(k) exp(2 pi i k y)
//         (eq. right_side_normal_equations_overdet, the window being a tensor product).
// The members of column l (eq. indexset_l) come from the point-wise tap patterns:
// the 2m+2 slots floor(M_sigma x_t) - m + s, s = 0..2m+1 (default), or the index set of
// eq. indexset_x.  The solve is a Cholesky factorisation; if it breaks down (rank
// deficient G_l: duplicate points, more members than |I_M|) it is repeated with a
// diagonal shift delta = 1e-13, 1e-10, 1e-7 times tr(G_l)/n (a Tikhonov regularised
// least-squares solution, which tends to the minimum-norm one as delta -> 0).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace infft {

struct BoptGeom {
    int d, M, Ms, m, S, NS, N, pattern, real_field;
};

__device__ __forceinline__ double frac_u(double xw, int Ms) {
    const double y = __dmul_rn((double)Ms, xw);
    return __dsub_rn(y, floor(y));
}

// slot s of a coordinate with fractional offset u belongs to the pattern
__device__ __forceinline__ bool slot_ok(int pattern, int s, int m, double u) {
    if (pattern == INFFT_BOPT_PATTERN_PAPER) {
        if (s == 0) return u == 0.0;
        return s <= 2 * m;
    }
    return true;
}

// column of slot tuple q of sorted point i, or -1 if the slot is outside the pattern
__device__ __forceinline__ long long slot_column(const BoptGeom& g, const uint32_t* cell, const double* x64, long long i,
                                                 int q) {
    uint32_t rem = cell[i];
    int b[3];
    for (int t = g.d - 1; t >= 0; --t) { b[t] = (int)(rem % (uint32_t)g.Ms); rem /= (uint32_t)g.Ms; }
    long long col = 0;
    int qq = q;
    int s[3];
    for (int t = g.d - 1; t >= 0; --t) { s[t] = qq % g.S; qq /= g.S; }
    for (int t = 0; t < g.d; ++t) {
        if (!slot_ok(g.pattern, s[t], g.m, frac_u(x64[i * g.d + t], g.Ms))) return -1;
        col = col * g.Ms + mod_pos(b[t] - g.m + s[t], g.Ms);
    }
    return col;
}

__global__ void k_bopt_count(BoptGeom g, const uint32_t* __restrict__ cell, const double* __restrict__ x64,
                             int* __restrict__ count) {
    const long long total = (long long)g.N * g.NS;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long col = slot_column(g, cell, x64, e / g.NS, (int)(e % g.NS));
        if (col >= 0) atomicAdd(count + col, 1);
    }
}

__global__ void k_bopt_fill(BoptGeom g, const uint32_t* __restrict__ cell, const double* __restrict__ x64,
                            const int* __restrict__ start, int* __restrict__ fill, long long* __restrict__ members) {
    const long long total = (long long)g.N * g.NS;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long col = slot_column(g, cell, x64, e / g.NS, (int)(e % g.NS));
        if (col >= 0) members[start[col] + atomicAdd(fill + col, 1)] = e;
    }
}

// members of a column in ascending (point, slot) order: deterministic
__global__ void k_bopt_sort(const int* __restrict__ start, long long ncols, long long* __restrict__ members) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int a = start[c], b = start[c + 1];
    for (int i = a + 1; i < b; ++i) {
        const long long v = members[i];
        int p = i - 1;
        while (p >= a && members[p] > v) { members[p + 1] = members[p]; --p; }
        members[p + 1] = v;
    }
}

// V(y) = sum_{k in I_M} w^(k) exp(2 pi i k y) for y = (u + m - s)/M_sigma, per point,
// coordinate and slot.  exp(2 pi i k y) advances by rotation and is recomputed exactly
// every 16 terms.
__global__ void k_bopt_V(BoptGeom g, const double* __restrict__ x64, const double* __restrict__ what1,
                         cx<double>* __restrict__ V) {
    const long long total = (long long)g.N * g.d * g.S;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e % g.S);
        const long long it = e / g.S;  // i * d + t
        const double u = frac_u(x64[it], g.Ms);
        const double y = (u + (double)(g.m - s)) / (double)g.Ms;
        double sr, cr;
        sincospi(2.0 * y, &sr, &cr);  // one step
        double acc_r = 0, acc_i = 0, zr = 0, zi = 0;
        for (int k0 = 0; k0 < g.M; ++k0) {
            if ((k0 & 15) == 0) sincospi(2.0 * y * (double)(k0 - g.M / 2), &zi, &zr);
            const double wk = what1[k0];
            acc_r += wk * zr;
            acc_i += wk * zi;
            const double nr = zr * cr - zi * sr, ni = zr * sr + zi * cr;
            zr = nr;
            zi = ni;
        }
        V[e] = mk<double>(acc_r, acc_i);
    }
}

// one factor of the Gram entries: D_{M/2-1}(u) + exp(-M pi i u), periodic in u
__device__ __forceinline__ cx<double> gram_factor(double u, int M) {
    u -= rint(u);
    double d;
    if (u == 0.0) d = (double)(M - 1);
    else d = sinpi((double)(M - 1) * u) / sinpi(u);
    double s, c;
    sincospi((double)M * u, &s, &c);
    return mk<double>(d + c, -s);
}

__host__ __device__ __forceinline__ long long tri(long long r, long long c) { return r * (r + 1) / 2 + c; }

constexpr int BOPT_THREADS = 256;

// bytes of the per-column arrays (v, y, current column of L, member points, member ids),
// rounded up to 256 so that consecutive per-block slices keep the 16-byte complex arrays aligned
__host__ __device__ __forceinline__ size_t bopt_fixed_bytes(int n, int d) {
    return ((size_t)n * (16 * 3 + 8 * d + 8) + 255) & ~(size_t)255;
}

// (row, column) of entry e of a packed lower triangle (e = r (r + 1) / 2 + c, c <= r): a
// float estimate of the row, corrected by integer steps
__device__ __forceinline__ void tri_rc(long long e, long long* r_out, long long* c_out) {
    long long r = (long long)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while (r * (r + 1) / 2 > e) --r;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    *r_out = r;
    *c_out = e - r * (r + 1) / 2;
}

// Persistent solver over a list of columns: each block takes the next column of `list`
// from the counter `next`, so blocks that drew large columns do not hold up the others
// (every column's arithmetic is independent of the block that solves it).  G_l lives in
// shared memory when n(n+1)/2 entries fit (n <= n_smem), otherwise in the block's slice
// of `gscratch` (n_max = the largest column of the list).  The per-column
// arrays live in shared memory when the largest column's fit (fix_smem), otherwise in the
// block's slice of `gfix` (columns of thousands of members: the centre of a linogram grid).
__global__ void __launch_bounds__(BOPT_THREADS) k_bopt_solve(BoptGeom g, const int* __restrict__ start,
                                                             const long long* __restrict__ members,
                                                             const double* __restrict__ x64,
                                                             const cx<double>* __restrict__ V, double rhs2,
                                                             const int* __restrict__ list, int nlist,
                                                             int* __restrict__ next, int n_smem, int n_max,
                                                             cx<double>* __restrict__ gscratch,
                                                             int fix_smem, unsigned char* __restrict__ gfix,
                                                             cx<double>* __restrict__ coef, double* __restrict__ eps,
                                                             int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 16-byte aligned complex arrays first, then the 8-byte arrays
    cx<double>* Gs = reinterpret_cast<cx<double>*>(smem_raw);     // packed lower, tri(n_smem + 1)
    unsigned char* fix = fix_smem ? reinterpret_cast<unsigned char*>(Gs + tri(n_smem + 1, 0))
                                  : gfix + (size_t)blockIdx.x * bopt_fixed_bytes(n_max, g.d);
    cx<double>* vv = reinterpret_cast<cx<double>*>(fix);          // n_max: right side v_l
    cx<double>* yy = vv + n_max;                                  // n_max: solution in place
    cx<double>* colk = yy + n_max;                                // n_max: current column of L
    double* xs = reinterpret_cast<double*>(colk + n_max);         // n_max * d
    long long* mem = reinterpret_cast<long long*>(xs + (size_t)n_max * g.d);  // n_max
    __shared__ double s_diag;
    __shared__ int s_fail;
    __shared__ double s_trace;
    const int tid = threadIdx.x, nth = blockDim.x;
    __shared__ int s_item;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(next, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();   // every thread has read s_item before thread 0 draws again
        if (item >= nlist) break;
        const long long col = list[item];
        const int a = start[col];
        const int n = start[col + 1] - a;
        if (n == 0) {
            if (tid == 0) eps[col] = rhs2;
            continue;
        }
        cx<double>* G = (n <= n_smem) ? Gs : gscratch + (size_t)blockIdx.x * ((size_t)n_max * (n_max + 1) / 2);
        for (int j = tid; j < n; j += nth) {
            const long long e = members[a + j];
            mem[j] = e;
            const long long i = e / g.NS;
            int qq = (int)(e % g.NS);
            int s[3];
            for (int t = g.d - 1; t >= 0; --t) { s[t] = qq % g.S; qq /= g.S; }
            cx<double> v = mk<double>(1.0, 0.0);
            for (int t = 0; t < g.d; ++t) {
                xs[j * g.d + t] = x64[i * g.d + t];
                v = mul(v, V[(i * g.d + t) * g.S + s[t]]);
            }
            if (g.real_field) v.im = 0.0;
            vv[j] = v;
        }
        __syncthreads();
        bool done = false;
        for (int attempt = 0; attempt < 4 && !done; ++attempt) {
            // G_l (lower triangle) from the Dirichlet closed form, plus the diagonal shift
            const long long ne = tri(n, 0);
            for (long long e = tid; e < ne; e += nth) {
                long long rr, c;
                tri_rc(e, &rr, &c);
                cx<double> v = mk<double>(1.0, 0.0);
                for (int t = 0; t < g.d; ++t) v = mul(v, gram_factor(xs[rr * g.d + t] - xs[c * g.d + t], g.M));
                if (g.real_field) v.im = 0.0;
                G[e] = v;
            }
            __syncthreads();
            if (tid == 0) {
                double tr = 0;
                for (int j = 0; j < n; ++j) tr += G[tri(j, j)].re;
                s_trace = tr;
                s_fail = 0;
            }
            __syncthreads();
            if (attempt > 0) {
                const double shift = s_trace / n * (attempt == 1 ? 1e-13 : attempt == 2 ? 1e-10 : 1e-7);
                for (int j = tid; j < n; j += nth) G[tri(j, j)].re += shift;
                __syncthreads();
            }
            // Cholesky G = L L^*, L in place
            for (int k = 0; k < n; ++k) {
                if (tid == 0) {
                    const double dk = G[tri(k, k)].re;
                    if (!(dk > 0.0)) s_fail = 1;
                    s_diag = (dk > 0.0) ? sqrt(dk) : 1.0;
                    G[tri(k, k)] = mk<double>(s_diag, 0.0);
                }
                __syncthreads();
                if (s_fail) break;
                const double inv = 1.0 / s_diag;
                for (int i = k + 1 + tid; i < n; i += nth) {
                    const cx<double> l = scale(G[tri(i, k)], inv);
                    G[tri(i, k)] = l;
                    colk[i] = l;
                }
                __syncthreads();
                const int w = n - k - 1;
                const long long sq = (long long)w * (w + 1) / 2;   // the trailing lower triangle
                for (long long e = tid; e < sq; e += nth) {
                    long long ii, jj;
                    tri_rc(e, &ii, &jj);
                    const int i = k + 1 + (int)ii, j = k + 1 + (int)jj;
                    const cx<double> li = colk[i], lj = colk[j];
                    cx<double> gij = G[tri(i, j)];
                    gij.re -= li.re * lj.re + li.im * lj.im;  // l_i conj(l_j)
                    gij.im -= li.im * lj.re - li.re * lj.im;
                    G[tri(i, j)] = gij;
                }
                __syncthreads();
            }
            if (!s_fail) done = true;
            __syncthreads();
        }
        if (!done) {
            if (tid == 0) { eps[col] = rhs2; atomicAdd(status, 1); }
            for (int j = tid; j < n; j += nth) coef[mem[j]] = mk<double>(0, 0);
            __syncthreads();
            continue;
        }
        // L y = v (forward), L^* b = y (backward)
        for (int j = tid; j < n; j += nth) yy[j] = vv[j];
        __syncthreads();
        for (int c = 0; c < n; ++c) {
            const double lcc = G[tri(c, c)].re;
            const cx<double> yc = scale(yy[c], 1.0 / lcc);
            __syncthreads();
            if (tid == 0) yy[c] = yc;
            for (int r = c + 1 + tid; r < n; r += nth) yy[r] = sub(yy[r], mul(G[tri(r, c)], yc));
            __syncthreads();
        }
        for (int c = n - 1; c >= 0; --c) {
            const double lcc = G[tri(c, c)].re;
            const cx<double> bc = scale(yy[c], 1.0 / lcc);
            __syncthreads();
            if (tid == 0) yy[c] = bc;
            for (int r = tid; r < c; r += nth) yy[r] = sub(yy[r], mulconj(G[tri(c, r)], bc));  // conj(L_cr) b_c
            __syncthreads();
        }
        // scatter b and the residual ||rhs||^2 - Re(b^* v)
        for (int j = tid; j < n; j += nth) coef[mem[j]] = yy[j];
        if (tid == 0) {
            double re = 0;
            for (int j = 0; j < n; ++j) re += yy[j].re * vv[j].re + yy[j].im * vv[j].im;
            eps[col] = rhs2 - re;
        }
        __syncthreads();
    }
}

__global__ void k_bopt_what(int M, int Ms, int m, int window, double beta, double* __restrict__ what1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
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
    what1[i] = wh;
}

__global__ void k_max(const double* __restrict__ a, long long n, double* __restrict__ out) {
    __shared__ double sm[256];
    double mx = 0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, a[i]);
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}

template <class R>
__global__ void k_bopt_convert(const cx<double>* __restrict__ a, long long n, cx<R>* __restrict__ b) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = mk<R>((R)a[i].re, (R)a[i].im);
}

__global__ void k_bopt_unsort(const cx<double>* __restrict__ a, const int* __restrict__ perm, long long N, int NS,
                              cx<double>* __restrict__ out) {
    const long long total = N * NS;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / NS;
        out[(long long)perm[i] * NS + e % NS] = a[e];
    }
}

// caller order -> sorted order (the inverse of k_bopt_unsort)
__global__ void k_bopt_sort_in(const cx<double>* __restrict__ in, const int* __restrict__ perm, long long N, int NS,
                               cx<double>* __restrict__ a) {
    const long long total = N * NS;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / NS;
        a[e] = in[(long long)perm[i] * NS + e % NS];
    }
}

static infft_status optimize_impl(infft_plan_s* p, unsigned opts, double* max_res, cudaStream_t st,
                                  std::vector<void*>& tmp) {
    BoptGeom g;
    g.d = p->d; g.M = p->M; g.Ms = p->Ms; g.m = p->m; g.S = 2 * p->m + 2;
    g.NS = ipow(g.S, g.d); g.N = (int)p->N;
    g.pattern = (opts & INFFT_BOPT_PATTERN_PAPER) ? INFFT_BOPT_PATTERN_PAPER : INFFT_BOPT_PATTERN_2M2;
    g.real_field = (opts & INFFT_BOPT_REAL) ? 1 : 0;
    const long long ncols = ipow(g.Ms, g.d);
    const long long nent = (long long)g.N * g.NS;
    // temporaries from the library's stream-ordered pool: unlike cudaMalloc / cudaFree they do
    // not synchronise the device, so a server's reconstructions on other streams go on while a
    // new point set's B_opt is computed
    auto alloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (pool_alloc(&q, std::max<size_t>(bytes, 16), st) != INFFT_OK) return nullptr;
        tmp.push_back(q);
        return q;
    };
    int* start = (int*)alloc((ncols + 1) * 4);
    int* fill = (int*)alloc((ncols + 1) * 4);
    long long* members = (long long*)alloc(nent * 8);
    cx<double>* V = (cx<double>*)alloc((size_t)g.N * g.d * g.S * 16);
    double* what1 = (double*)alloc((size_t)g.M * 8);
    double* eps = (double*)alloc(ncols * 8);
    double* scal = (double*)alloc(64);
    int* status = (int*)alloc(16);
    if (!start || !fill || !members || !V || !what1 || !eps || !scal || !status) {
        set_error("optimize_B: out of device memory");
        return INFFT_ENOMEM;
    }
    if (!p->coef64) INFFT_TRY(dev_alloc(p, (void**)&p->coef64, (size_t)nent * 16));
    if (!p->coef) INFFT_TRY(dev_alloc(p, &p->coef, (size_t)nent * (p->fp64 ? 16 : 8)));
    INFFT_CUDA(cudaMemsetAsync(p->coef64, 0, (size_t)nent * 16, st));
    INFFT_CUDA(cudaMemsetAsync(start, 0, (ncols + 1) * 4, st));
    INFFT_CUDA(cudaMemsetAsync(fill, 0, (ncols + 1) * 4, st));
    INFFT_CUDA(cudaMemsetAsync(status, 0, 16, st));
    const int tb = 256;
    const int gb = (int)std::min<long long>((nent + tb - 1) / tb, 65535LL * 16);
    k_bopt_count<<<gb, tb, 0, st>>>(g, p->cell, p->x64, start);
    INFFT_LAUNCHED();
    INFFT_TRY(scan_exclusive(start, ncols + 1, st));
    k_bopt_fill<<<gb, tb, 0, st>>>(g, p->cell, p->x64, start, fill, members);
    INFFT_LAUNCHED();
    k_bopt_sort<<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(start, ncols, members);
    INFFT_LAUNCHED();
    k_bopt_what<<<(g.M + 255) / 256, 256, 0, st>>>(g.M, g.Ms, g.m, p->window, p->beta, what1);
    INFFT_LAUNCHED();
    const long long nv = (long long)g.N * g.d * g.S;
    k_bopt_V<<<(int)std::min<long long>((nv + tb - 1) / tb, 65535LL * 16), tb, 0, st>>>(g, p->x64, what1, V);
    INFFT_LAUNCHED();

    // largest column, ||rhs||^2 = sum_k w^(k)^2 = prod_t sum_{k_t} w^(k_t)^2
    std::vector<int> hs(ncols + 1);
    std::vector<double> hw(g.M);
    INFFT_TRY(read_back(hs.data(), start, (ncols + 1) * 4, st));
    INFFT_TRY(read_back(hw.data(), what1, g.M * 8, st));
    INFFT_CUDA(cudaStreamSynchronize(st));
    int n_max = 1;
    for (long long c = 0; c < ncols; ++c) n_max = std::max(n_max, hs[c + 1] - hs[c]);
    double s1 = 0;
    for (double w : hw) s1 += w * w;
    const double rhs2 = std::pow(s1, g.d);

    int dev = 0, nsm = 0;
    INFFT_CUDA(cudaGetDevice(&dev));
    INFFT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // Two launches.  Columns whose Gram matrix fits in shared memory (with the per-column
    // arrays) run first, several blocks per SM.  Larger columns (the centre of a linogram
    // grid holds thousands of members) keep G in global memory; they run largest first on
    // as many blocks as a share of the free device memory allows.
    const size_t cap = 200 * 1024;
    long long n_smem = 0;
    while (n_smem < n_max && bopt_fixed_bytes((int)n_smem + 1, g.d) + (size_t)tri(n_smem + 2, 0) * 16 + 64 <= cap)
        ++n_smem;
    std::vector<int> small, big;
    int n_small = 0, n_big = 0;
    for (long long c = 0; c < ncols; ++c) {
        const int n = hs[c + 1] - hs[c];
        if (n <= n_smem) { small.push_back((int)c); n_small = std::max(n_small, n); }
        else { big.push_back((int)c); n_big = std::max(n_big, n); }
    }
    std::stable_sort(big.begin(), big.end(), [&](int a, int b) { return hs[a + 1] - hs[a] > hs[b + 1] - hs[b]; });
    // The solve goes out in launches of about sixteen columns per block (tens of milliseconds
    // each), so that the blocks leave the SMs regularly and work of higher-priority streams (a
    // server's reconstructions while a new point set is admitted) is scheduled in between;
    // each launch has its own work counter.  (Two columns per block made the tails of the
    // launches cost half again the solve's time.)
    int* list = (int*)alloc((small.size() + big.size()) * 4);
    if (!list) { set_error("optimize_B: out of device memory (column lists)"); return INFFT_ENOMEM; }
    if (!small.empty())
        INFFT_CUDA(cudaMemcpyAsync(list, small.data(), small.size() * 4, cudaMemcpyHostToDevice, st));
    if (!big.empty())
        INFFT_CUDA(cudaMemcpyAsync(list + small.size(), big.data(), big.size() * 4, cudaMemcpyHostToDevice, st));
    if (!small.empty()) {
        const size_t smem = bopt_fixed_bytes(std::max(n_small, 1), g.d) + (size_t)tri(n_small + 1, 0) * 16 + 64;
        int per_sm = 0;
        INFFT_CUDA(cudaFuncSetAttribute(k_bopt_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        INFFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bopt_solve, BOPT_THREADS, smem));
        const int blocks = nsm * std::max(1, per_sm);
        const long long chunk = 16LL * blocks;
        const long long nchunk = ((long long)small.size() + chunk - 1) / chunk;
        int* next = (int*)alloc((size_t)nchunk * 4);   // one work counter per launch
        if (!next) { set_error("optimize_B: out of device memory (work counters)"); return INFFT_ENOMEM; }
        INFFT_CUDA(cudaMemsetAsync(next, 0, (size_t)nchunk * 4, st));
        for (long long c = 0; c < nchunk; ++c) {
            const long long c0 = c * chunk;
            const int n = (int)std::min<long long>(chunk, (long long)small.size() - c0);
            k_bopt_solve<<<std::min(blocks, n), BOPT_THREADS, smem, st>>>(
                g, start, members, p->x64, V, rhs2, list + c0, n, next + c, n_small, std::max(n_small, 1), nullptr, 1,
                nullptr, (cx<double>*)p->coef64, eps, status);
            INFFT_LAUNCHED();
        }
    }
    if (!big.empty()) {
        const bool fix_smem = bopt_fixed_bytes(n_big, g.d) + 64 <= cap;
        const size_t per_block = (size_t)tri(n_big + 1, 0) * 16 + (fix_smem ? 0 : bopt_fixed_bytes(n_big, g.d));
        size_t free_b = 0, total_b = 0;
        INFFT_CUDA(cudaMemGetInfo(&free_b, &total_b));
        const long long fit = (long long)((double)free_b * 0.6 / (double)per_block);
        const int blocks = (int)std::min<long long>(std::min<long long>(nsm, (long long)big.size()), fit);
        if (blocks < 1) {
            set_error("optimize_B: a column of %d members needs %zu bytes of Gram scratch, %zu bytes are free",
                      n_big, per_block, free_b);
            return INFFT_ENOMEM;
        }
        cx<double>* gscr = (cx<double>*)alloc((size_t)blocks * tri(n_big + 1, 0) * 16);
        unsigned char* gfix = fix_smem ? nullptr : (unsigned char*)alloc((size_t)blocks * bopt_fixed_bytes(n_big, g.d));
        if (!gscr || (!fix_smem && !gfix)) {
            set_error("optimize_B: out of device memory (Gram scratch for columns of %d members)", n_big);
            return INFFT_ENOMEM;
        }
        const size_t smem = (fix_smem ? bopt_fixed_bytes(n_big, g.d) : 0) + 16 + 64;
        INFFT_CUDA(cudaFuncSetAttribute(k_bopt_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // one column per block per launch (largest first)
        const size_t nchunk = (big.size() + (size_t)blocks - 1) / (size_t)blocks;
        int* next = (int*)alloc(nchunk * 4);   // one work counter per launch
        if (!next) { set_error("optimize_B: out of device memory (work counters)"); return INFFT_ENOMEM; }
        INFFT_CUDA(cudaMemsetAsync(next, 0, nchunk * 4, st));
        for (size_t c = 0; c < nchunk; ++c) {
            const size_t c0 = c * (size_t)blocks;
            const int n = (int)std::min<size_t>((size_t)blocks, big.size() - c0);
            k_bopt_solve<<<n, BOPT_THREADS, smem, st>>>(g, start, members, p->x64, V, rhs2, list + small.size() + c0, n,
                                                         next + c, 0, n_big, gscr, fix_smem ? 1 : 0, gfix,
                                                         (cx<double>*)p->coef64, eps, status);
            INFFT_LAUNCHED();
        }
    }
    const int cb = (int)std::min<long long>((nent + 255) / 256, 65535LL * 16);
    if (p->fp64) k_bopt_convert<double><<<cb, 256, 0, st>>>((cx<double>*)p->coef64, nent, (cx<double>*)p->coef);
    else k_bopt_convert<float><<<cb, 256, 0, st>>>((cx<double>*)p->coef64, nent, (cx<float>*)p->coef);
    INFFT_LAUNCHED();
    k_max<<<1, 256, 0, st>>>(eps, ncols, scal);
    INFFT_LAUNCHED();
    double mres = 0;
    int nfail = 0;
    INFFT_TRY(read_back(&mres, scal, 8, st));
    INFFT_TRY(read_back(&nfail, status, 4, st));
    INFFT_CUDA(cudaStreamSynchronize(st));
    if (max_res) *max_res = mres;
    p->has_bopt = true;
    p->bopt_window = p->window;
    if (nfail) {
        set_error("%d columns without a stable factorisation were left empty", nfail);
        return INFFT_ENOTCONV;
    }
    return INFFT_OK;
}

}  // namespace infft

using namespace infft;

extern "C" {

infft_status infft_optimize_B(infft_plan_t p, unsigned opts, double* max_col_residual, void* stream) {
    if (!p) { set_error("null plan"); return INFFT_EINVAL; }
    if (opts & ~3u) { set_error("unknown options %u", opts); return INFFT_EINVAL; }
    std::vector<void*> tmp;
    p->pool_stream = (cudaStream_t)stream;
    infft_status s = optimize_impl(p, opts, max_col_residual, (cudaStream_t)stream, tmp);
    for (void* q : tmp) pool_free(q, (cudaStream_t)stream);   // in stream order, after the solve
    cudaStreamSynchronize((cudaStream_t)stream);
    return s;
}

infft_status infft_set_bopt(infft_plan_t p, const void* coeff, void* stream) {
    if (!p || !coeff) { set_error("null argument"); return INFFT_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    p->pool_stream = st;
    const int NS = ipow(2 * p->m + 2, p->d);
    const long long nent = (long long)p->N * NS;
    const size_t bytes = (size_t)nent * 16;
    if (!p->coef64) INFFT_TRY(dev_alloc(p, (void**)&p->coef64, bytes));
    if (!p->coef) INFFT_TRY(dev_alloc(p, &p->coef, (size_t)nent * (p->fp64 ? 16 : 8)));
    const bool dev = is_device_pointer(coeff);
    const void* src = coeff;
    void* staged = nullptr;
    if (!dev) {
        INFFT_CUDA(cudaMalloc(&staged, bytes));
        INFFT_CUDA(cudaMemcpyAsync(staged, coeff, bytes, cudaMemcpyHostToDevice, st));
        src = staged;
    }
    k_bopt_sort_in<<<1024, 256, 0, st>>>((const cx<double>*)src, p->perm, p->N, NS, (cx<double>*)p->coef64);
    INFFT_LAUNCHED();
    const int cb = (int)std::min<long long>((nent + 255) / 256, 65535LL * 16);
    if (p->fp64) k_bopt_convert<double><<<cb, 256, 0, st>>>((cx<double>*)p->coef64, nent, (cx<double>*)p->coef);
    else k_bopt_convert<float><<<cb, 256, 0, st>>>((cx<double>*)p->coef64, nent, (cx<float>*)p->coef);
    INFFT_LAUNCHED();
    INFFT_CUDA(cudaStreamSynchronize(st));
    if (staged) cudaFree(staged);
    p->has_bopt = true;
    p->bopt_window = p->window;
    return INFFT_OK;
}

infft_status infft_get_bopt(infft_plan_t p, void* coeff, void* stream) {
    if (!p || !coeff) { set_error("null argument"); return INFFT_EINVAL; }
    if (!p->has_bopt || !p->coef64) { set_error("no B_opt"); return INFFT_ESTATE; }
    cudaStream_t st = (cudaStream_t)stream;
    const int NS = ipow(2 * p->m + 2, p->d);
    const size_t bytes = (size_t)p->N * NS * 16;
    const bool dev = is_device_pointer(coeff);
    void* dst = coeff;
    if (!dev) INFFT_CUDA(cudaMalloc(&dst, bytes));
    k_bopt_unsort<<<1024, 256, 0, st>>>((const cx<double>*)p->coef64, p->perm, p->N, NS, (cx<double>*)dst);
    INFFT_LAUNCHED();
    if (!dev) {
        INFFT_CUDA(cudaMemcpyAsync(coeff, dst, bytes, cudaMemcpyDeviceToHost, st));
        INFFT_CUDA(cudaStreamSynchronize(st));
        cudaFree(dst);
    }
    INFFT_CUDA(cudaStreamSynchronize(st));
    return INFFT_OK;
}

}  // extern "C"
