// FFT passes over lines held in shared memory (Algorithm 2.4 steps 2-3, Algorithm 2.1 steps
// 1-2): the block body shared by the FFT kernels of nfft.cu and the persistent d = 2 adjoint.
#pragma once

#include <algorithm>

#include "jobset.cuh"
#include "spread.cuh"

namespace infft {

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
//
// One block's lines of FFT pass `pass` (block gblk of the pass, global over the JobSet's jobs),
// with the block's dynamic shared memory at smem_raw: the body of k_fft, and the FFT units of the
// persistent d = 2 kernel.  Generic in the block size (a power of two, >= 32).
template <class R, int D, bool FWD, bool MRG, int NTH>
__device__ __forceinline__ void fft_block(const JobSet<R>& js, const int pass, const int gblk,
                                          unsigned char* smem_raw) {
    cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
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
    // skewed line stride, odd in 8-byte words: the same element of 16 consecutive lines (the
    // loads and stores of the passes along y and z) falls into 16 distinct bank pairs
    const int ns = n + (n >> 4) + 1;
    const int logn = 31 - __clz(n);
    const long long nlines = A * B;
    const long long q0 = (long long)lb * L;
    const bool lanes_b = (B >= L);  // consecutive lines are consecutive b: coalesce along b

    cx<R>* tws = buf + L * ns;      // the n/2 twiddles after the lines
    for (int k = threadIdx.x; k < (Ms >> 1); k += NTH) tws[k] = J.tw[k];
    // then (merging pass only) the table of tile item ranges, then the M deconvolution factors
    const int nrng = (MRG && pass == 0) ? mrg_tile_rows(L, J.T) * J.ntile : 0;
    R* dvs = reinterpret_cast<R*>(reinterpret_cast<int2*>(tws + (Ms >> 1)) + nrng);
    for (int k = threadIdx.x; k < M; k += NTH) dvs[k] = J.dinv[k];

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
    const int tid = threadIdx.x;
    constexpr int nth = NTH;
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
        // Thread columns: i = tid + nth kc for n >= nth (every line), else i = tid mod n on lines
        // l = tid / n + (nth / n) k.  The x-sources of a column and the y-sources of a line are
        // found once each; an element then looks up its (at most four) tiles' item ranges.
        const unsigned cells = (unsigned)(P * P);
        const int ncol = n >= nth ? n / nth : 1, dl = n >= nth ? 1 : nth / n;
        const int i0 = n >= nth ? tid : (tid & (n - 1)), l0 = n >= nth ? 0 : (tid >> logn);
        for (int kc = 0; kc < ncol; ++kc) {
            const int i = i0 + kc * nth;
            const int c = i & (T - 1), tx = i >> logT;
            int xcol[2], xoff[2], nx = 1;
            xcol[0] = tx; xoff[0] = c + m;
            xcol[1] = 0; xoff[1] = 0;
            if (c + T + m < P) { xcol[1] = (tx - 1) & (nt - 1); xoff[1] = c + T + m; nx = 2; }
            else if (c - T + m >= 0) { xcol[1] = (tx + 1) & (nt - 1); xoff[1] = c - T + m; nx = 2; }
            const int pos = skew(bitrev(i, logn));
#pragma unroll 2
            for (int l = l0; l < L; l += dl) {
                const long long y = q0 + l;
                cx<R> acc = mk<R>(0, 0);
                if (y < nlines) {
                    const int r = (int)y & (T - 1), trow = (int)(y >> logT) - ty0 + 1;
                    int yrow[2], yoff[2], ny = 1;
                    yrow[0] = trow << lognt; yoff[0] = (r + m) * P;
                    yrow[1] = 0; yoff[1] = 0;
                    if (r + T + m < P) { yrow[1] = (trow - 1) << lognt; yoff[1] = (r + T + m) * P; ny = 2; }
                    else if (r - T + m >= 0) { yrow[1] = (trow + 1) << lognt; yoff[1] = (r - T + m) * P; ny = 2; }
                    // the first item of every source, loaded together; then the sum in
                    // k_merge2d's order (y-source major, x-source minor, items in order)
                    size_t src0[4];
                    int cnt[4];
                    cx<R> v[4];
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 2; ++b) {
                            const int q = 2 * a + b;
                            const bool has = a < ny && b < nx;
                            const int2 g = has ? rng[yrow[a] + xcol[b]] : make_int2(0, 0);
                            cnt[q] = g.y;
                            src0[q] = (size_t)(unsigned)g.x * cells + (unsigned)(yoff[a] + xoff[b]);
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
                buf[l * ns + pos] = acc;
            }
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


// The halo merge of the d = 2 register-row path folded into the first FFT pass (fft_block with
// MRG), unless INFFT_FFT_MERGE=0 or a job's table of tile item ranges would pass 16 KB: the
// grid is then neither written nor read between the two.  Both forms give bitwise the same
// result.
template <class R>
inline bool merge_on_load_ok(const JobSet<R>& js) {
    if (env_form("INFFT_FFT_MERGE") == 0 || js.axA > 0) return false;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        const int L = fft_lines(J.Ms, (int)sizeof(cx<R>));
        if ((size_t)mrg_tile_rows(L, J.T) * J.ntile * sizeof(int2) > 16 * 1024) return false;
    }
    return true;
}

// dynamic shared memory of a merging first pass (MRG) over the jobs of js
template <class R>
inline size_t fft_smem_mrg(const JobSet<R>& js) {
    size_t mx = 0;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<R>& J = js.job[j];
        const int n = J.Ms, L = fft_lines(n, (int)sizeof(cx<R>));
        mx = std::max(mx, ((size_t)L * (n + n / 16 + 1) + n / 2) * sizeof(cx<R>) +
                              (size_t)mrg_tile_rows(L, J.T) * J.ntile * sizeof(int2) + (size_t)J.M * sizeof(R));
    }
    return mx;
}

// dynamic shared memory of an FFT pass over the jobs of js: the largest of the jobs' line
// buffers plus twiddles and deconvolution factors
template <class R>
inline size_t fft_smem(const JobSet<R>& js) {
    size_t mx = 0;
    for (int j = 0; j < js.njobs; ++j) {
        const int n = js.job[j].Ms, L = fft_lines(n, (int)sizeof(cx<R>));
        mx = std::max(mx, ((size_t)L * (n + n / 16 + 1) + n / 2) * sizeof(cx<R>) + (size_t)js.job[j].M * sizeof(R));
    }
    return mx;
}

}  // namespace infft
