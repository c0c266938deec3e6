/*
 * infft.h -- C ABI of a GB300 (sm_103a) library for the direct inverse NFFT
 * of Kircheis & Potts, "Fast and direct inversion methods for the
 * multivariate nonequispaced fast Fourier transform".
 *
 * Notation (Section 2): d in {1,2,3}; M even; I_M = Z^d cap [-M/2, M/2)^d;
 * points x_j in the torus T^d = [-1/2, 1/2)^d, j = 1..N; A = (exp(2 pi i k x_j))
 * (eq. matrix_A); M_sigma = 2 ceil(ceil(sigma M)/2) (Section 2.1); window
 * truncation parameter m.
 *
 * Layouts.
 *   x     : N x d row-major float64 (coordinate t of point j at x[j*d + t]).
 *           Points need not be wrapped; x - floor(x + 1/2) is used.
 *   f     : N complex samples, interleaved (re, im), in the caller's point order.
 *   fhat  : M^d complex coefficients in C order over I_M, the entry of k sits at
 *           sum_t (k_t + M/2) M^(d-1-t) (first coordinate slowest), interleaved.
 *   Complex values are float2-like (8 bytes) for INFFT_FP32 plans and
 *   double2-like (16 bytes) for INFFT_FP64 plans.
 *
 * Ownership.  The caller owns x, f and fhat.  A plan copies what it needs
 * from x and owns every device buffer it allocates (sorted points, bins,
 * work lists, tables, weights, B_opt coefficients, scratch grids) until
 * infft_destroy.
 *
 * Pointers.  f / fhat passed to infft_adjoint / infft_forward may be device
 * pointers or host pointers; host memory is staged through plan-owned device
 * buffers with cudaMemcpyAsync on the given stream (synchronising at the end
 * of the call so that a host result is ready on return).  All other array
 * arguments documented as "device" must be device pointers.
 *
 * Streams.  `stream` is a cudaStream_t passed as void*; NULL means the legacy
 * default stream.  Calls on device buffers are stream ordered and do not
 * synchronise the host, except where stated (plan creation, infft_weights,
 * infft_optimize_B and the getters synchronise).  A plan's transforms write the
 * plan's own scratch grids: transforms of one plan must not overlap in time, so
 * enqueue them on one stream (or order the streams with events).  Different plans
 * may run concurrently on different streams and host threads.
 *
 * Errors.  Every call returns an infft_status and never throws or aborts.
 * infft_last_error() returns a thread-local message for the last failing call.
 * A plan stays valid after a failed call unless the status is INFFT_ESTATE.
 */
#ifndef INFFT_H
#define INFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct infft_plan_s* infft_plan_t;
typedef struct infft_batch_s* infft_batch_t;

typedef enum {
    INFFT_OK = 0,
    INFFT_EINVAL = 1,        /* invalid argument (sizes, null pointers, flags) */
    INFFT_ENOMEM = 2,        /* device or pinned-host allocation failed */
    INFFT_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    INFFT_ENOTCONV = 4,      /* CG reached max_iter before rel_tol */
    INFFT_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    INFFT_ESTATE = 6,        /* call not valid in the plan's state (e.g. DCF before weights) */
    INFFT_EUNSUPPORTED = 7   /* valid but unsupported size (M_sigma not a power of two, ...) */
} infft_status;

/* plan flags */
enum {
    INFFT_FP32 = 1,          /* spreading / FFT / interpolation in float32 */
    INFFT_FP64 = 2,          /* everything in float64 */
    INFFT_WIN_KB = 0,        /* Kaiser-Bessel window (default) */
    INFFT_WIN_BSPLINE = 4,   /* B-spline window B_{2m}(M_sigma x), eq. window_bspline */
    INFFT_WIN_DIRICHLET = 8, /* asymmetric Dirichlet window (B_opt only, Theorem 4.5) */
    INFFT_POOLED = 16        /* plan memory from the library's stream-ordered pool (see infft_plan) */
};

/* reconstruction modes of infft_adjoint */
enum {
    INFFT_MODE_PLAIN = 0,    /* h = D^* F^* B^* f          (Algorithm 2.4)            */
    INFFT_MODE_DCF = 1,      /* h = D^* F^* B^* W f        (Algorithm 3.7)            */
    INFFT_MODE_BOPT = 2      /* h = D^* F^* B_opt^* f      (Algorithm 4.4)            */
};

/* options of infft_weights_opts */
enum {
    INFFT_WEIGHTS_AUTO = 0,       /* Toeplitz products where they apply, else NFFT products  */
    INFFT_WEIGHTS_NFFT = 1,       /* an NFFT and an adjoint NFFT per iteration (as printed)  */
    INFFT_WEIGHTS_TOEPLITZ = 2    /* convolution form of A^*A (second kind only)             */
};

/* options of infft_optimize_B */
enum {
    INFFT_BOPT_PATTERN_2M2 = 0,   /* 2m+2 consecutive indices per coordinate (default)       */
    INFFT_BOPT_PATTERN_PAPER = 1, /* the index set I_{Msigma,m}(x_j) of eq. indexset_x         */
    INFFT_BOPT_REAL = 2           /* real-constrained least squares instead of complex b_l     */
};

/*
 * infft_plan -- create a plan for fixed points (Sections 2-4).
 *   d      : 1, 2 or 3.
 *   M      : even degree, M >= 2.
 *   N      : number of points, 1 <= N < 2^31.
 *   x      : N x d float64, host or device; copied.
 *   sigma  : oversampling factor >= 1; M_sigma = 2 ceil(ceil(sigma M)/2) must be a
 *            power of two <= 4096 (else INFFT_EUNSUPPORTED).
 *   m      : truncation parameter, 1 <= m, 2m+2 <= M_sigma.
 *   flags  : INFFT_FP32 or INFFT_FP64, or-ed with a window flag and optionally INFFT_POOLED.
 *   stream : stream for the set-up kernels (the call synchronises it).
 *   out    : receives the plan.
 * Sorts the points into tiles of the oversampled grid (counting sort over
 * grid cells, deterministic order), builds the work lists and the tables of
 * 1/(M_sigma w^(k)) (eq. matrix_D) and FFT twiddles.
 *
 * Memory.  By default a plan's device buffers come from cudaMalloc and go back by
 * cudaFree; both synchronise the device with work that other host threads have queued.
 * With INFFT_POOLED they come from a stream-ordered pool the library owns per device,
 * allocated in the order of the stream of the call that needs them (creation, later
 * batched calls, weights, B_opt) and returned in infft_destroy after a device
 * synchronisation; the pool keeps up to 1 GiB of freed blocks for reuse.
 * Meant for servers that build plans on one thread while another launches
 * reconstructions.
 */
infft_status infft_plan(int d, int M, int64_t N, const double* x, double sigma, int m,
                        unsigned flags, void* stream, infft_plan_t* out);

/*
 * Tuning of a plan's kernels: the choices the library otherwise makes by itself.  The paper
 * has no counterpart; the values change speed only, never results beyond the rounding of
 * a different summation order (the spread tile and the item cap change which padded tiles
 * hold a point's taps, the others the schedule).  0 in a field keeps the library's default.
 *   tile      : edge T of the spreading tiles (a power of two, m < T <= M_sigma; the register-row
 *               spread of d = 2 needs T + 2m + 1 <= 32 and the fused merge-FFT kernel T in
 *               {8, 16}); default 16 for d = 2, 8 for d = 3, min(256, M_sigma) for d = 1.
 *   item_cap  : most points per work item, >= 1 (default 512; 32 for d = 1).
 *   branches  : concurrent branches of batched adjoints with device buffers whose first plan
 *               is this one (1..8; default 3; batches with host buffers keep 8).
 *   prefetch  : spreading kernels copy the next points' data to shared memory while they
 *               spread the current ones: 1 on, 2 off (default: by form and grid size).
 *   fused_fft : d = 2 adjoints merge the padded tiles and run both FFT passes in one
 *               thread-block-cluster kernel: 1 on (where the grid fits), 2 off (default off).
 * An environment variable (INFFT_SPREAD2D_PREFETCH, INFFT_SPREAD3D_PREFETCH,
 * INFFT_FUSED_MERGE_FFT, INFFT_BATCH_BRANCHES) applies only where the plan leaves the field 0.
 */
typedef struct {
    int tile;
    int item_cap;
    int branches;
    int prefetch;
    int fused_fft;
} infft_tune_t;

/* infft_plan_tuned -- infft_plan with tuning (tune may be NULL: all defaults).  Invalid
 * tuning values give INFFT_EINVAL. */
infft_status infft_plan_tuned(int d, int M, int64_t N, const double* x, double sigma, int m,
                              unsigned flags, const infft_tune_t* tune, void* stream, infft_plan_t* out);

/*
 * infft_weights -- Algorithm 3.6: density compensation weights for exact
 * reconstruction (Corollary 3.4, eq. claim_quadrature_coefficients_double).
 * If (2M)^d <= N: CG on A_2M^* A_2M u = e_0 (the normal equations of the
 * second kind, eq. normal_equations_second_kind_double, after conjugation),
 * w = conj(A_2M u).  Otherwise: CG on A_2M A_2M^* q = 1_N (first kind,
 * eq. normal_equations_first_kind_double), w = conj(q).  Matrix products are
 * float64 NFFTs (Algorithms 2.1 / 2.4) at degree 2M with oversampling 2 and
 * truncation m_cg (<= 0 selects 8 for d <= 2 and 4 for d = 3), or, in the second
 * kind, the convolution form of infft_weights_opts below; CG vectors,
 * inner products and updates are float64.  x0 = 0, stop when
 * ||r||_2 / ||b||_2 <= rel_tol or after max_iter iterations.  The CG state stays on the
 * device: the host looks at it once per eight queued iterations, and iterations queued after
 * the stop do nothing.  The weights come from the CG iterate (x_1, x_2, ...) of smallest
 * ||r||_2, so that a capped run returns the best weights it met: in the second kind ||r||_2
 * is exactly the 2-norm of A_2M^T w - e_0, which therefore does not grow with max_iter.
 *   residual_inf : (out, may be NULL) max_k |[A_2M^T w]_k - delta_{0,k}| over
 *                  I_2M, evaluated with the same float64 NFFT.
 *   iters        : (out, may be NULL) CG iterations taken.
 * Returns INFFT_ENOTCONV (weights still stored) if max_iter was reached.
 * Synchronises.
 */
infft_status infft_weights(infft_plan_t plan, int max_iter, double rel_tol, int m_cg,
                           double* residual_inf, int* iters, void* stream);

/*
 * infft_weights_opts -- infft_weights with a choice of how the CG applies its matrix.
 *   INFFT_WEIGHTS_NFFT: every iteration applies A_2M^* A_2M (or A_2M A_2M^*) by a
 *     float64 NFFT and an adjoint NFFT, as Algorithm 3.6 prints it.
 *   INFFT_WEIGHTS_TOEPLITZ: second kind only ((2M)^d <= N) and 4M <= 4096.  The entries
 *     of A_2M^* A_2M depend on k - k' only, [A^*A]_{k,k'} = t(k - k') with
 *     t(n) = sum_j exp(-2 pi i n x_j) on I_4M.  t is computed once from 2^d adjoint
 *     NFFTs at degree 2M of the samples exp(-2 pi i s x_j), s in {-M, M}^d; each
 *     iteration is then a circular convolution of period 4M: two float64 FFTs of
 *     (4M)^d points and a pointwise product.  Temporary device memory of about
 *     4 (4M)^d complex128 values.
 *   INFFT_WEIGHTS_AUTO (0, what infft_weights uses): TOEPLITZ where it applies, else NFFT.
 * Other arguments, results and errors as infft_weights; INFFT_EUNSUPPORTED when
 * TOEPLITZ is asked for where it does not apply, INFFT_EINVAL for unknown options.
 */
infft_status infft_weights_opts(infft_plan_t plan, int max_iter, double rel_tol, int m_cg, unsigned opts,
                                double* residual_inf, int* iters, void* stream);

/* infft_set_weights / infft_get_weights -- N complex128 weights in the caller's
 * point order (host or device).  set marks the plan ready for INFFT_MODE_DCF. */
infft_status infft_set_weights(infft_plan_t plan, const void* w, void* stream);
infft_status infft_get_weights(infft_plan_t plan, void* w, void* stream);

/*
 * infft_optimize_B -- Algorithm 4.3: for every column l of the sparse matrix B
 * solve the least-squares problem eq. opt_overdet_columnwise through its
 * normal equations G_l b_l = v_l, with G_l = H_l^* H_l from the Dirichlet
 * closed form (eq. matrix_normal_equations_overdet) and v_l from
 * eq. right_side_normal_equations_overdet, in float64 (one batched kernel,
 * Cholesky with a diagonal-shift retry).  The window used for w^ is the
 * plan's window flag (KB, B-spline or Dirichlet).  opts: INFFT_BOPT_* flags.
 *   max_col_residual : (out, may be NULL) max_l ||H_l b_l - rhs_l||_2^2
 *                      (eq. res_opt_columnwise), from ||rhs||^2 - Re(b^* v).
 * Synchronises.
 */
infft_status infft_optimize_B(infft_plan_t plan, unsigned opts, double* max_col_residual, void* stream);

/* infft_set_bopt -- restore B_opt coefficients saved by infft_get_bopt for a plan with the
 * same points and parameters (N x S^d complex128, caller's point order, host or device),
 * so that a cached precompute (Algorithm 4.3) need not be repeated; the plan is then
 * ready for INFFT_MODE_BOPT and infft_inverse_adjoint.  Synchronises. */
infft_status infft_set_bopt(infft_plan_t plan, const void* coeff, void* stream);

/* infft_get_bopt -- copy B_opt coefficients, N x S^d complex128 (S = 2m+2, slot
 * s_t holds column floor(M_sigma x_t) - m + s_t), caller's point order. */
infft_status infft_get_bopt(infft_plan_t plan, void* coeff, void* stream);

/*
 * infft_adjoint -- the reconstruction step.
 *   mode = INFFT_MODE_PLAIN: Algorithm 2.4, h ~ A^* f;
 *   mode = INFFT_MODE_DCF  : Algorithm 3.7, h ~ A^* W f (needs weights);
 *   mode = INFFT_MODE_BOPT : Algorithm 4.4, h = D^* F^* B_opt^* f (needs B_opt).
 *   f    : N complex samples (host or device), caller's point order.
 *   fhat : M^d complex result (host or device), C order over I_M.
 * The spreading kernels for d = 2 and d = 3 copy the next points' sorted data to shared
 * memory while they spread the current ones (d = 3: always; d = 2: float32 with m <= 4,
 * and grids with fewer work items than eight warps per SM).  INFFT_SPREAD2D_PREFETCH and
 * INFFT_SPREAD3D_PREFETCH in the environment ("0" off, "1" on) override that choice; the
 * sums and their order, and so the results bit for bit, are the same either way.  So with
 * INFFT_FFT_MERGE (on unless "0"): for d = 2 the first FFT pass sums each grid cell from the
 * padded tiles as it loads its rows (steps 2-3 of Algorithm 2.4 with no grid written in
 * between) instead of a separate halo-merge kernel.
 */
infft_status infft_adjoint(infft_plan_t plan, int mode, const void* f, void* fhat, void* stream);

/*
 * The steps of the adjoint NFFT (Algorithm 2.4) one at a time, for callers that place a
 * collective between them -- the point-sharded adjoint over several GPUs, where every rank
 * spreads its own points into a whole grid, the grids are summed with a reduce-scatter of
 * slabs, and the pruned FFT runs on slabs with one all-to-all between the axes.
 *
 * infft_spread_grid -- step 1 of Algorithm 2.4 (with W for INFFT_MODE_DCF, B_opt^* for
 * INFFT_MODE_BOPT): g_l = sum_j c_j w~_m(x_j - l/M_sigma) for every l of the oversampled
 * grid.  f: N complex (device), the caller's point order.  grid: M_sigma^d complex (device),
 * C order, l stored at l mod M_sigma along every axis.  Uses the plan's scratch set 0 (as
 * infft_adjoint).  Stream ordered.
 *
 * infft_fft_axis -- steps 2 and 3 of Algorithm 2.4 along one axis: for an input tensor
 * in[a][l][b] (A x M_sigma x B, device, complex), out[a][i][b] = (1/(M_sigma w^(k))) sum_l
 * in[a][l][b] exp(-2 pi i k l / M_sigma), k = i - M/2, i = 0..M-1 (the crop to I_M and
 * the deconvolution of eq. matrix_D of that axis; mode picks the window of D as in
 * infft_adjoint).  The output is written as nblk blocks along i (nblk divides M): block c
 * holds the (A x M/nblk x B) tensor of i = c M/nblk .. (c+1) M/nblk - 1, contiguous, so that
 * block c can be sent to rank c of an all-to-all as it is (nblk = 1: the plain A x M x B
 * tensor).  Stream ordered.
 */
infft_status infft_spread_grid(infft_plan_t plan, int mode, const void* f, void* grid, void* stream);
infft_status infft_fft_axis(infft_plan_t plan, int mode, int64_t A, int64_t B, int nblk, const void* in, void* out,
                            void* stream);

/* infft_forward -- Algorithm 2.1, f ~ A fhat (fhat: M^d complex, f: N complex). */
infft_status infft_forward(infft_plan_t plan, const void* fhat, void* f, void* stream);

/*
 * infft_inverse_adjoint -- the inverse adjoint NFFT of Remark 4.6: an approximate
 * solution f of A^* f = h (eq. problem_infft*, |I_M| <= N), f = B_opt F D h.  The steps of
 * Algorithm 2.1 with the window entries of B replaced by the plan's optimised entries
 * B_opt[j, l] (not conjugated), D built from the window B_opt was optimised for.
 *   h : M^d complex (host or device), C order over I_M, as fhat elsewhere.
 *   f : N complex (host or device), the caller's point order.
 * Needs infft_optimize_B first (else INFFT_ESTATE).  Stream ordered like infft_forward.
 */
infft_status infft_inverse_adjoint(infft_plan_t plan, const void* h, void* f, void* stream);

/*
 * infft_adjoint_batched -- `count` reconstructions on (possibly different) plans
 * of the same d and precision, executed as one launch per kernel stage over
 * all of them.  f[i], fhat[i] are device pointers, or host pointers staged through
 * the plan's own I/O buffers (then that plan may appear only once in the batch,
 * else INFFT_EINVAL, and the call synchronises).  A plan may appear several times
 * with device buffers (several sample vectors on one point set, e.g. one per
 * receive coil): its k-th occurrence uses the k-th set of scratch grids, allocated
 * on first need and owned by the plan until infft_destroy (counted in
 * infft_plan_device_bytes).  The fhat[i] must not overlap.  The jobs run in three (eight
 * when host buffers are involved) concurrent branches of unequal work on streams the
 * library forks from `stream` (at its priority) and joins back to it;
 * INFFT_BATCH_BRANCHES in the environment (1..8) changes the count.  Results do not depend
 * on the branching.
 * Persistent form (no counterpart in the paper; on request, INFFT_PERSISTENT=1): a batch of at
 * most 96 float32 d = 2 jobs in window modes (PLAIN or DCF) with m <= 4 and device buffers
 * runs as one persistent kernel
 * (after a small counter reset), whose CTAs take work units from a queue: the spread of four
 * work items, a block of the FFT pass along x that merges the padded tiles, a block of the
 * pass along y; a job's x blocks wait for its spread, its y blocks for its x blocks.  The jobs
 * run largest first, and the queue interleaves the stages of consecutive jobs.  Each sum is
 * formed in the same order as in the staged kernels, so the results are bitwise the same.
 * It is slower than the staged kernels in graph branches on the batched workload measured
 * (0.470 against 0.450 ms per 64-set step), hence off by default.  INFFT_PERSIST_LAG sets the
 * distance, in waves of the kernel's CTAs, between a job's spread and its FFT blocks in the
 * queue (default 4).  Tuned plans with fused_fft = 1 or prefetch = 2 take the staged kernels.
 * infft_batch_create records the form in effect.
 */
infft_status infft_adjoint_batched(const infft_plan_t* plans, int count, int mode,
                                   const void* const* f, void* const* fhat, void* stream);

/*
 * infft_adjoint_batched_slots -- as infft_adjoint_batched, with the scratch set of
 * every job chosen by the caller: job i runs on scratch set slots[i] of its plan
 * (0 = the plan's own, k >= 1 allocated on first need, at most
 * INFFT_MAX_SCRATCH_SLOT).  Jobs of one plan in one call need distinct slots
 * (else INFFT_EINVAL).  Transforms of one plan that may overlap in time (batches on
 * different streams) are safe when they use different slots; that is the caller's
 * promise, the library does not track streams.  The library's extension for
 * schedulers that keep one point set in flight on several streams; the method
 * itself (Algorithm 3.7) has no counterpart.
 */
#define INFFT_MAX_SCRATCH_SLOT 1024
infft_status infft_adjoint_batched_slots(const infft_plan_t* plans, int count, int mode,
                                         const void* const* f, void* const* fhat, const int* slots,
                                         void* stream);

/*
 * infft_adjoint_batched_timed -- as infft_adjoint_batched (count <= 96), and
 * reports device times of the stages in stage_ms[5]: spreading, halo merge and
 * the FFT passes along each axis (unused entries 0), from CUDA events recorded on
 * `stream` between the kernel launches.  Jobs whose plans turn on the fused merge-FFT
 * kernel (infft_tune_t fused_fft) count it in the merge stage; where the first FFT pass does
 * the merge as it loads (INFFT_FFT_MERGE, d = 2), the merge stage is 0 and the first pass
 * holds it.  Synchronises.
 */
infft_status infft_adjoint_batched_timed(const infft_plan_t* plans, int count, int mode,
                                         const void* const* f, void* const* fhat, void* stream,
                                         float* stage_ms);

/*
 * Graph-replayed batches.  infft_batch_create records the batched adjoint for
 * fixed plans and fixed buffers f[i] / fhat[i] into a CUDA graph;
 * infft_batch_run replays it on `stream`.  The plans and buffers must outlive
 * the batch.  The buffers are device memory or page-locked host memory (cudaHostAlloc,
 * cudaHostRegister; pageable memory gives INFFT_EINVAL): for host buffers the graph also
 * holds the copies to and from the plans' I/O buffers, so one replay moves a whole step's
 * inputs and results, and the caller synchronises `stream` before reading fhat.  A plan with
 * host buffers may appear only once.  The graph holds the jobs in the concurrent branches of
 * infft_adjoint_batched (eight with host buffers).  Plans may repeat as in
 * infft_adjoint_batched; the extra scratch grids are allocated before the capture starts.
 */
infft_status infft_batch_create(const infft_plan_t* plans, int count, int mode,
                                const void* const* f, void* const* fhat, void* stream,
                                infft_batch_t* out);
infft_status infft_batch_run(infft_batch_t batch, void* stream);
void infft_batch_destroy(infft_batch_t batch);

/*
 * infft_adjoint_noalloc -- the same reconstruction as infft_adjoint, for callers that
 * must not allocate device memory during the call: programs whose device memory is
 * owned by an external allocator or arena that forbids other components from calling
 * cudaMalloc, and latency-bound loops that cannot afford cudaMalloc's synchronisation
 * or a late out-of-memory failure.  (The paper has no counterpart; this is an interface
 * of the library.)
 *   plan, mode : as for infft_adjoint (the plan is created beforehand).
 *   f, fhat    : DEVICE pointers (host pointers are rejected with INFFT_EINVAL).
 * The per-call scratch (padded tiles, oversampled grid, FFT intermediates) lives in a
 * fixed 32 MiB array compiled into the library, which every device that loads the
 * library holds until the process exits.  A plan whose scratch would exceed 32 MiB is
 * rejected with INFFT_EINVAL and a message giving both sizes.  The call allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 * The first call in a CUDA context (on each device, and again after a cudaDeviceReset has
 * replaced the device's primary context) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it per context; make that
 * first call before any stream capture.  Mode and state errors are those of infft_adjoint.  All calls share the one array and every call overwrites all the scratch it
 * reads, so nothing carries over between calls -- but calls that overlap on the GPU
 * (different streams, or different host threads) race on it and must be serialised by
 * the caller.
 */
infft_status infft_adjoint_noalloc(infft_plan_t plan, int mode, const void* f, void* fhat, void* stream);

/* Accessors. */
int64_t infft_plan_N(infft_plan_t plan);
int infft_plan_Msigma(infft_plan_t plan);
int infft_plan_work_items(infft_plan_t plan);        /* work items (tile, point range) of the spread */
size_t infft_plan_device_bytes(infft_plan_t plan);   /* device memory held by the plan */
const char* infft_last_error(void);
void infft_destroy(infft_plan_t plan);

/* infft_wait_timeouts -- how many bounded waits of the persistent batched kernel (a unit
 * waiting for the units it depends on) gave up after about a second since the library was
 * loaded.  The queue order rules such waits out; a nonzero count means the results of the
 * launches since the last check are not to be trusted.  Synchronous with the device. */
unsigned int infft_wait_timeouts(void);

/*
 * infft_inject_faults -- host-side fault injection for testing callers' error handling
 * (no counterpart in the paper).  Bits: 1 every device allocation of a plan fails
 * (INFFT_ENOMEM), 2 every kernel launch reports failure (INFFT_ECUDA; the kernel was
 * still queued, nothing faults on the device), 4 the weights CG reports non-convergence
 * (INFFT_ENOTCONV, weights stored).  0 turns injection off.  The initial mask comes from
 * the environment variable INFFT_FAULT, a comma-separated list of alloc, launch, cg.
 * Process-wide.
 */
void infft_inject_faults(unsigned mask);

/* Number of kernel launches issued by this thread since the last reset
 * (for reporting; not synchronised with the device). */
uint64_t infft_launch_count(void);
void infft_launch_count_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* INFFT_H */
