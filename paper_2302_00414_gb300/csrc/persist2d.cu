// Persistent batched d = 2 adjoint (Algorithm 3.7 / 2.4 over many point sets in one launch):
// one kernel whose CTAs take work units from a queue until it is empty.  Units are the spread
// of four work items (Algorithm 2.4 step 1, the register-row form of spread2d.cuh), a block of
// the FFT pass along x that merges the padded tiles as it loads (steps 2-3), and a block of the
// pass along y.  The spread units run in job order; the x blocks of job j enter the queue `lag`
// spread units after job j's last spread unit, its y blocks `lag` spread units after that
// (lag = four waves of the launch's CTAs, so that a job's spreads are done when its FFT blocks
// are taken).  The latency-bound FFT blocks of earlier jobs thus share the SMs with the
// issue-bound spreads of later ones, and the last jobs' FFT blocks run after the spreads.  The
// queue is a list of segments (a run of spread units, or one job's x or y blocks) in the kernel
// parameters.
//
// Measured on the batched d = 2 workload (64 sets): 0.456 ms per step against 0.439 ms for the
// staged kernels in graph branches.  The FFT blocks run as four-warp CTAs at the spread's
// occupancy (five per SM), where the staged passes run eight-warp blocks at six per SM, and
// the overlap does not make up for it.  The form is therefore taken only on request
// (INFFT_PERSISTENT=1).
//
// Dependencies: an x unit of job j needs every work item of job j spread; a y unit needs every
// x block of job j.  Each finished item or block adds one to its job's counter (after a fence);
// the unit that depends on it waits on the counter.  A unit depends only on units earlier in
// the queue, and a CTA takes a unit only while it runs, so the earliest unfinished unit never
// waits: no CTA can wait forever.  Every wait is still bounded (about a second of clock
// cycles); a wait that gives up counts a timeout (read by infft_wait_timeouts), marks the
// launch aborted so that no later wait of it blocks, and carries on, so the kernel ends.
//
// The counters of job j live in the first bytes of its grid buffer, which the merging pass
// leaves unused; the queue head and the abort mark of the launch in job 0's.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "fft.cuh"
#include "spread2d.cuh"

namespace infft {

constexpr int PERSIST_THREADS = 128;   // four warps: the spread's block, and the FFT units' size
constexpr int MAXSEG = 4 * MAXJ + 1;   // 2 groups per job, a spread run before each, one after

struct PersistQueue {
    int nseg;
    int pre[MAXSEG + 1];       // units before segment s
    int kind[MAXSEG];          // 0 spread run, 1 x blocks of a job, 2 y blocks of a job
    int arg[MAXSEG];           // spread run: its first spread unit; x / y: the job
    int su_pre[MAXJ + 1];      // spread units before job j (four work items each)
};

static_assert(sizeof(JobSet<float>) + sizeof(PersistQueue) <= 32000, "kernel parameters exceed the limit");

__device__ unsigned int g_wait_timeouts;

__device__ __forceinline__ int* job_counters(const Job<float>& J) { return reinterpret_cast<int*>(J.grid); }

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0 of the CTA waits until *ctr >= target (or the launch is aborted / the wait times out)
__device__ void wait_at_least(const int* ctr, int target, int* abort_flag) {
    if (load_acquire(ctr) >= target) return;
    const long long t0 = clock64();
    for (;;) {
        if (load_acquire(ctr) >= target) return;
        if (load_acquire(abort_flag) != 0) return;
        if (clock64() - t0 > (1LL << 31)) {
            atomicAdd(&g_wait_timeouts, 1u);
            atomicExch(abort_flag, 1);
            return;
        }
        __nanosleep(100);
    }
}

__global__ void k_persist_reset(const __grid_constant__ JobSet<float> js) {
    for (int j = threadIdx.x; j < js.njobs; j += blockDim.x) {
        int* c = job_counters(js.job[j]);
        c[0] = 0;   // work items spread
        c[1] = 0;   // x blocks done
    }
    if (threadIdx.x == 0) {
        int* c = job_counters(js.job[0]);
        c[2] = 0;   // queue head
        c[3] = 0;   // abort mark
    }
}

template <int MM>
__global__ void __launch_bounds__(PERSIST_THREADS, 5)
    k_adjoint2d_persistent(const __grid_constant__ JobSet<float> js, const __grid_constant__ PersistQueue pq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_unit;
    int* head = job_counters(js.job[0]) + 2;
    int* abort_flag = job_counters(js.job[0]) + 3;
    const int total = pq.pre[pq.nseg];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        __syncthreads();   // the previous unit is done with shared memory and s_unit
        if (threadIdx.x == 0) s_unit = atomicAdd(head, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= total) return;
        const int sg = find_job(pq.pre, pq.nseg, u);
        const int o = u - pq.pre[sg];
        if (pq.kind[sg] == 0) {   // spread unit: four work items of one job
            const int su = pq.arg[sg] + o;
            const int j = find_job(pq.su_pre, js.njobs, su);
            const Job<float>& J = js.job[j];
            const int li = 4 * (su - pq.su_pre[j]) + warp;
            if (li < J.nitems) {
                spread2d_item<float, MM, false, true>(js, js.pre_items[j] + li,
                                                      smem_raw + (size_t)warp * js.smem_per_warp);
                __threadfence();
                __syncwarp();
                if (lane == 0) atomicAdd(job_counters(J), 1);
            }
        } else if (pq.kind[sg] == 1) {   // block of the merging pass along x
            const int j = pq.arg[sg];
            const Job<float>& J = js.job[j];
            if (threadIdx.x == 0) wait_at_least(job_counters(J), J.nitems, abort_flag);
            __threadfence();
            __syncthreads();
            fft_block<float, 2, false, true, PERSIST_THREADS>(js, 0, js.pre_fft[0][j] + o, smem_raw);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(job_counters(J) + 1, 1);
        } else {   // block of the pass along y
            const int j = pq.arg[sg];
            const Job<float>& J = js.job[j];
            if (threadIdx.x == 0)
                wait_at_least(job_counters(J) + 1, js.pre_fft[0][j + 1] - js.pre_fft[0][j], abort_flag);
            __threadfence();
            __syncthreads();
            fft_block<float, 2, false, false, PERSIST_THREADS>(js, 1, js.pre_fft[1][j] + o, smem_raw);
        }
    }
}

unsigned int persist_wait_timeouts() {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0xffffffffu;
    }
    return v;
}

// The queue: spread units in job order; job j's x blocks at spread position e_j + lag (e_j: one
// past its last spread unit), its y blocks at e_j + 2 lag, positions past the end clamped to the
// end; at one position the FFT groups come before the spread unit there, x before y, in job
// order.  Every unit's dependencies therefore lie earlier in the queue.
static void build_queue(const JobSet<float>& js, int lag, PersistQueue& pq) {
    memset(&pq, 0, sizeof(pq));
    const int nj = js.njobs;
    pq.su_pre[0] = 0;
    for (int j = 0; j < nj; ++j) pq.su_pre[j + 1] = pq.su_pre[j] + (js.job[j].nitems + 3) / 4;
    const int S = pq.su_pre[nj];
    struct Ev { int pos, kind, job; };
    std::vector<Ev> ev;
    for (int j = 0; j < nj; ++j) {
        const int px = std::min(S, pq.su_pre[j + 1] + lag);
        ev.push_back({px, 1, j});
        ev.push_back({std::min(S, px + lag), 2, j});
    }
    std::stable_sort(ev.begin(), ev.end(), [](const Ev& a, const Ev& b) {
        return a.pos != b.pos ? a.pos < b.pos : (a.kind != b.kind ? a.kind < b.kind : a.job < b.job);
    });
    int n = 0, pos = 0, units = 0;
    auto add = [&](int kind, int arg, int count) {
        if (count <= 0) return;
        pq.pre[n] = units;
        pq.kind[n] = kind;
        pq.arg[n] = arg;
        units += count;
        ++n;
    };
    for (const Ev& e : ev) {
        add(0, pos, e.pos - pos);   // the spread units before this group
        pos = e.pos;
        const int p = e.kind == 1 ? 0 : 1;
        add(e.kind, e.job, js.pre_fft[p][e.job + 1] - js.pre_fft[p][e.job]);
    }
    add(0, pos, S - pos);
    pq.nseg = n;
    pq.pre[n] = units;
}

template <int MM>
static infft_status launch_persist2d(JobSet<float>& js, cudaStream_t st) {
    spread2d_setup<float, MM, false, true>(js);
    const size_t smem = std::max({(size_t)4 * js.smem_per_warp, fft_smem_mrg(js), fft_smem(js)});
    auto kern = k_adjoint2d_persistent<MM>;
    INFFT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, nsm = 0, per_sm = 0;
    INFFT_CUDA(cudaGetDevice(&dev));
    INFFT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    INFFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PERSIST_THREADS, smem));
    const int ctas = std::max(1, per_sm) * nsm;
    PersistQueue pq;
    // the lag in waves of the launch's CTAs (INFFT_PERSIST_LAG, default 4: on the batched d = 2
    // workload 0.25 / 0.5 / 1 / 2 / 4 waves gave 0.610 / 0.543 / 0.486 / 0.478 / 0.470 ms per
    // step; a shorter lag makes FFT blocks wait for spreads still running)
    double waves = 4.0;
    if (const char* e = getenv("INFFT_PERSIST_LAG")) waves = std::max(0.0, std::min(16.0, atof(e)));
    build_queue(js, (int)(waves * ctas), pq);
    const int grid = std::max(1, std::min(pq.pre[pq.nseg], ctas));
    k_persist_reset<<<1, PERSIST_THREADS, 0, st>>>(js);
    INFFT_LAUNCHED();
    kern<<<grid, PERSIST_THREADS, smem, st>>>(js, pq);
    INFFT_LAUNCHED();
    return INFFT_OK;
}

// The persistent form for a JobSet (prefixes filled) when INFFT_PERSISTENT=1 and every job
// takes the paired register-row spread (float32 window modes, m <= 4) with the prefetching
// copies and the merging first pass; *used tells whether it ran.
infft_status persist2d_try(JobSet<float>& js, cudaStream_t st, bool* used) {
    *used = false;
    if (env_form("INFFT_PERSISTENT") != 1 || js.njobs < 1 || js.axA > 0) return INFFT_OK;
    int m = 0;
    bool bopt = false;
    if (!spread2d_eligible(js, &m, &bopt) || bopt || !spread2d_pair_m<float>(m)) return INFFT_OK;
    if (!spread2d_prefetch(js, m) || !merge_on_load_ok(js)) return INFFT_OK;
    for (int j = 0; j < js.njobs; ++j) {
        const Job<float>& J = js.job[j];
        if (J.fused_fft == 1 || (J.fused_fft == 0 && env_form("INFFT_FUSED_MERGE_FFT") == 1)) return INFFT_OK;
        if ((size_t)J.Ms * J.Ms * sizeof(cx<float>) < 4 * sizeof(int)) return INFFT_OK;
    }
    *used = true;
    switch (m) {
        case 2: return launch_persist2d<2>(js, st);
        case 3: return launch_persist2d<3>(js, st);
        default: return launch_persist2d<4>(js, st);
    }
}

}  // namespace infft
