// Batched estimates: many (pattern, eps) jobs share one persistent sampler
// launch per convergence round, and the rounds run as a captured CUDA graph.
//
// Every job is Algorithm 3 on its own sample stream (RNG slot = job index
// plus the configured slot): round r of a job covers its samples
// [r W, (r+1) W).  One launch hands out (job, chunk) pairs of all active jobs
// from one dispenser; each chunk writes its partial; a reduce-and-check kernel
// (one block per job) folds the job's partials in chunk order into its running
// totals and evaluates Eq. equ:error on the device, retiring jobs with
// eps_hat <= eps or n >= n_max; a one-thread kernel lays out the next round's
// chunks over the jobs still active.  R rounds (sampler, check, relayout) are
// captured once into a CUDA graph and replayed until no job is active; rounds
// after the last job retires find no chunks and return at once.  The chunk
// size and the reduction tree are those of the single-job path, so every job's
// result equals a separate gpm_estimate of its pattern with the same slot.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "sampler.cuh"

namespace gpm {

struct BatchJob {
    double sum, sumsq;      // running totals of X and X^2
    uint64_t hits, n;
    double eps, mu, half, eps_hat;
    uint64_t n_min, n_max, rounds;
    uint32_t slot, active, converged, chunk_off, nchunks, single;   // single: plan has single-list steps
};

struct BatchCtl {
    uint32_t counter;        // chunk dispenser of the current round
    uint32_t total_chunks;   // chunks of the current round over active jobs
    uint32_t active;         // jobs still running
    uint32_t rounds;         // rounds laid out so far
    uint32_t any_single;     // some active job needs the single-list sampler variant
    uint32_t pad;
};

struct BatchArgs {
    uint64_t seed, window;
    double z;
    uint32_t njobs, cap, chunk, chunks_per_job;
    gpm_mlp mlp;
    uint32_t mlp_tc;
};

// static shared memory of ns_batch_kernel: one StepPlan per warp
constexpr size_t kBatchStaticSmem = 8 * sizeof(StepPlan);

template <int MODE, bool COMPACT>
__global__ void __launch_bounds__(256, (MODE == MODE_LEARNED) ? 2 : GPM_MIN_BLOCKS)
    ns_batch_kernel(const DGraph g, const Plan *__restrict__ plans, const BatchJob *jobs, BatchCtl *ctl,
                    const BatchArgs ba, Partial *partials) {
    extern __shared__ __align__(16) uint64_t smem64[];
    __shared__ StepPlan splan[8];
    const unsigned lane = lane_id();
    WarpMem wm = warp_mem<MODE>(smem64, ba.cap, ba.mlp);
    StepPlan *sp = &splan[threadIdx.x >> 5];
    uint32_t cur_job = 0xFFFFFFFFu;
    const uint32_t total = ctl->total_chunks;
    RunArgs a;
    a.seed = ba.seed;
    a.cap = ba.cap;
    a.trace = nullptr;
    a.mlp_tc = ba.mlp_tc;
    for (;;) {
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(&ctl->counter, 1u);
        c = __shfl_sync(kFull, c, 0);
        if (c >= total) break;
        uint32_t job = 0;
        for (uint32_t q = 0; q < ba.njobs; q++) {
            if (jobs[q].active && c >= jobs[q].chunk_off && c < jobs[q].chunk_off + jobs[q].nchunks) {
                job = q;
                break;
            }
        }
        const BatchJob &J = jobs[job];
        const uint64_t first = J.rounds * ba.window;
        const uint64_t end = first + ba.window;
        const uint64_t s0 = first + (uint64_t)(c - J.chunk_off) * ba.chunk;
        const uint64_t s1 = (s0 + ba.chunk < end) ? s0 + ba.chunk : end;
        a.slot = J.slot;
        if (job != cur_job) {
            load_step_plan(plans[job], sp);
            cur_job = job;
        }
        const StepPlan &p = *sp;
        double sum = 0.0, sumsq = 0.0;
        uint64_t hits = 0;
        for (uint64_t s = s0; s < s1; s++) {
            __syncwarp();
            const SampleOut r = sample_one<MODE, StepPlan, COMPACT>(g, p, a, s, wm);
            if (r.hit) {
                sum = __dadd_rn(sum, r.w);
                sumsq = __dadd_rn(sumsq, __dmul_rn(r.w, r.w));
                hits++;
            }
        }
        if (lane == 0) {
            Partial q;
            q.sum = sum;
            q.sumsq = sumsq;
            q.hits = hits;
            q.n = s1 - s0;
            partials[c] = q;
        }
    }
}

// One block per job: the job's partials in chunk order (same tree as the
// single-job reduction), then the end-of-window test of Algorithm 3.
__global__ void __launch_bounds__(1024) batch_reduce_check(const Partial *__restrict__ parts, BatchJob *jobs,
                                                           const BatchArgs ba) {
    __shared__ double s_sum[1024], s_sq[1024];
    __shared__ unsigned long long s_hits[1024], s_n[1024];
    BatchJob &J = jobs[blockIdx.x];
    if (!J.active) return;
    const unsigned t = threadIdx.x;
    const Partial *pp = parts + J.chunk_off;
    const uint32_t n = J.nchunks;
    const uint32_t per = (n + 1023) / 1024;
    const uint64_t b = (uint64_t)t * per;
    const uint64_t e = (b + per < n) ? b + per : n;
    double sum = 0.0, sq = 0.0;
    unsigned long long hits = 0, cnt = 0;
    for (uint64_t i = b; i < e; i++) {
        sum = __dadd_rn(sum, pp[i].sum);
        sq = __dadd_rn(sq, pp[i].sumsq);
        hits += pp[i].hits;
        cnt += pp[i].n;
    }
    s_sum[t] = sum;
    s_sq[t] = sq;
    s_hits[t] = hits;
    s_n[t] = cnt;
    __syncthreads();
    for (unsigned h = 512; h; h >>= 1) {
        if (t < h) {
            s_sum[t] = __dadd_rn(s_sum[t], s_sum[t + h]);
            s_sq[t] = __dadd_rn(s_sq[t], s_sq[t + h]);
            s_hits[t] += s_hits[t + h];
            s_n[t] += s_n[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        if (J.rounds == 0) {
            J.sum = s_sum[0];
            J.sumsq = s_sq[0];
        } else {
            J.sum = __dadd_rn(J.sum, s_sum[0]);
            J.sumsq = __dadd_rn(J.sumsq, s_sq[0]);
        }
        J.hits += s_hits[0];
        J.n += s_n[0];
        J.rounds += 1;
        window_test(J.sum, J.sumsq, J.n, ba.z, J.eps, J.n_min, J.n_max, &J.mu, &J.half, &J.eps_hat, &J.converged,
                    &J.active);
    }
}

__global__ void batch_relayout(BatchJob *jobs, BatchCtl *ctl, const BatchArgs ba) {
    if (threadIdx.x != 0) return;
    uint32_t off = 0, act = 0, single = 0;
    for (uint32_t q = 0; q < ba.njobs; q++) {
        if (jobs[q].active) {
            jobs[q].chunk_off = off;
            jobs[q].nchunks = ba.chunks_per_job;
            off += ba.chunks_per_job;
            act++;
            single |= jobs[q].single;
        } else {
            jobs[q].nchunks = 0;
        }
    }
    ctl->total_chunks = off;
    ctl->active = act;
    ctl->any_single = single;
    ctl->counter = 0;
    ctl->rounds += 1;
}

template <int MODE, bool COMPACT>
static cudaError_t batch_grid(gpm_graph *h, const Shape &sh, uint32_t *blocks) {
    auto kern = ns_batch_kernel<MODE, COMPACT>;
    const size_t smem = smem_bytes(sh, MODE);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (sh.blocks) {
        *blocks = sh.blocks;
        return cudaSuccess;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)(sh.warps * 32), smem);
    *blocks = (uint32_t)((per_sm > 0 ? per_sm : 1) * h->sm_count);
    return e;
}

// Runs the batch to completion; results[q] for job q.
gpm_status batch_estimate(gpm_graph *h, const std::vector<Plan> &plans, const double *eps, double delta,
                          uint64_t seed, const gpm_config *cfg, gpm_result *results, int mode) {
    const auto t0 = std::chrono::steady_clock::now();
    const uint32_t nj = (uint32_t)plans.size();
    const uint64_t W = (cfg && cfg->window) ? cfg->window : (1ull << 20);
    const uint64_t n_min = (cfg && cfg->n_min) ? cfg->n_min : W;
    const uint64_t n_max = (cfg && cfg->n_max) ? cfg->n_max : (1ull << 40);
    const double max_s = cfg ? cfg->max_seconds : 0.0;
    if (!(delta > 0.0 && delta < 1.0)) {
        set_error("delta must be in (0, 1)");
        return GPM_ERR_ARG;
    }
    for (uint32_t q = 0; q < nj; q++)
        if (!(eps[q] > 0.0)) {
            set_error("every eps must be > 0");
            return GPM_ERR_ARG;
        }
    Shape sh = pick_shape(h, cfg, W);
    bool single = false;
    for (const Plan &pl : plans) single = single || plan_single_steps(pl);
    const int kmode = kernel_mode(mode, single);
    bool induced = false;
    for (const Plan &pl : plans) induced = induced || pl.induced;
    // the compact step-2 loop for edge-induced batches (see sample_one)
    const bool compact = !induced && (kmode == MODE_INTERSECT || kmode == MODE_INTERSECT_SINGLE);
    if (sh.cap == 0) sh.cap = default_cap(h, kBatchStaticSmem, sh.warps, mode, induced);
    if (mode == MODE_LEARNED && sh.cap < kLearnedMax) sh.cap = kLearnedMax;
    const uint64_t cpj = (W + sh.chunk - 1) / sh.chunk;
    if (cpj * nj >= (1ull << 31)) {
        set_error("batch too large for one launch");
        return GPM_ERR_ARG;
    }
    BatchArgs ba;
    ba.seed = seed;
    ba.window = W;
    ba.z = normal_quantile(1.0 - delta / 2.0);
    ba.njobs = nj;
    ba.cap = sh.cap;
    ba.chunk = sh.chunk;
    ba.chunks_per_job = (uint32_t)cpj;
    std::memset(&ba.mlp, 0, sizeof(ba.mlp));
    if (mode == MODE_LEARNED) ba.mlp = *cfg->mlp;
    ba.mlp_tc = (mode == MODE_LEARNED && cfg->mlp_tensor) ? 1u : 0u;

    std::vector<BatchJob> jobs(nj);
    for (uint32_t q = 0; q < nj; q++) {
        BatchJob &J = jobs[q];
        std::memset(&J, 0, sizeof(J));
        J.eps = eps[q];
        J.n_min = n_min;
        J.n_max = n_max;
        J.slot = (cfg ? cfg->slot : 0) + q;
        J.active = 1;
        J.chunk_off = (uint32_t)(q * cpj);
        J.nchunks = (uint32_t)cpj;
        J.eps_hat = INFINITY;
        J.single = plan_single_steps(plans[q]) ? 1u : 0u;
    }
    BatchCtl ctl{0u, (uint32_t)(cpj * nj), nj, 0u, 1u, 0u};

    Plan *d_plans = nullptr;
    BatchJob *d_jobs = nullptr;
    BatchCtl *d_ctl = nullptr;
    Partial *d_parts = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr, graph_plain = nullptr;
    cudaGraphExec_t exec = nullptr, exec_plain = nullptr;
    cudaEvent_t ev_in = nullptr, ev_a = nullptr, ev_b = nullptr;
    const int R = 4;   // rounds per graph launch
    cudaEvent_t ev_k[2 * R] = {};
    gpm_status status = GPM_OK;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (exec_plain) cudaGraphExecDestroy(exec_plain);
        if (graph_plain) cudaGraphDestroy(graph_plain);
        // stream-ordered frees after the batch's own work
        cudaStream_t fs = cs ? cs : h->stream;
        pool_free(d_plans, fs);
        pool_free(d_jobs, fs);
        pool_free(d_ctl, fs);
        pool_free(d_parts, fs);
        if (cs) cudaStreamDestroy(cs);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_a) cudaEventDestroy(ev_a);
        if (ev_b) cudaEventDestroy(ev_b);
        for (int i = 0; i < 2 * R; i++)
            if (ev_k[i]) cudaEventDestroy(ev_k[i]);
    };
    // allocated on the handle's stream, which the batch stream waits for below
    if (pool_alloc((void **)&d_plans, sizeof(Plan) * nj, h->stream) != cudaSuccess ||
        pool_alloc((void **)&d_jobs, sizeof(BatchJob) * nj, h->stream) != cudaSuccess ||
        pool_alloc((void **)&d_ctl, sizeof(BatchCtl), h->stream) != cudaSuccess ||
        pool_alloc((void **)&d_parts, sizeof(Partial) * cpj * nj, h->stream) != cudaSuccess) {
        cleanup();
        set_error("batch: device allocation failed");
        return GPM_ERR_OOM;
    }
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&ev_a);
    if (e == cudaSuccess) e = cudaEventCreate(&ev_b);
    for (int i = 0; i < 2 * R && e == cudaSuccess; i++) e = cudaEventCreate(&ev_k[i]);
    // inputs are ordered after the caller's work on the handle's stream
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_plans, plans.data(), sizeof(Plan) * nj, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(BatchJob) * nj, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ctl, &ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    // R rounds (sampler, reduce-and-check, relayout) of one compiled sampler
    // variant captured into a graph
    auto capture = [&](int km, cudaGraph_t *gr, cudaGraphExec_t *ex) -> cudaError_t {
        uint32_t blocks = 0;
        cudaError_t ce = (km == MODE_CHECK)     ? batch_grid<MODE_CHECK, false>(h, sh, &blocks)
                         : (km == MODE_LAZY)    ? batch_grid<MODE_LAZY, false>(h, sh, &blocks)
                         : (km == MODE_LEARNED) ? batch_grid<MODE_LEARNED, false>(h, sh, &blocks)
                         : (km == MODE_INTERSECT_SINGLE)
                             ? (compact ? batch_grid<MODE_INTERSECT_SINGLE, true>(h, sh, &blocks)
                                        : batch_grid<MODE_INTERSECT_SINGLE, false>(h, sh, &blocks))
                             : (compact ? batch_grid<MODE_INTERSECT, true>(h, sh, &blocks)
                                        : batch_grid<MODE_INTERSECT, false>(h, sh, &blocks));
        if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return ce;
        const size_t smem = smem_bytes(sh, mode);
        const dim3 grid(blocks), block(sh.warps * 32);
        for (int r = 0; r < R; r++) {
            // event nodes around each sampler launch time the sampler alone
            cudaEventRecordWithFlags(ev_k[2 * r], cs, cudaEventRecordExternal);
            if (km == MODE_CHECK)
                ns_batch_kernel<MODE_CHECK, false><<<grid, block, smem, cs>>>(h->d, d_plans, d_jobs, d_ctl, ba, d_parts);
            else if (km == MODE_LAZY)
                ns_batch_kernel<MODE_LAZY, false><<<grid, block, smem, cs>>>(h->d, d_plans, d_jobs, d_ctl, ba, d_parts);
            else if (km == MODE_LEARNED)
                ns_batch_kernel<MODE_LEARNED, false>
                    <<<grid, block, smem, cs>>>(h->d, d_plans, d_jobs, d_ctl, ba, d_parts);
            else if (km == MODE_INTERSECT_SINGLE && compact)
                ns_batch_kernel<MODE_INTERSECT_SINGLE, true>
                    <<<grid, block, smem, cs>>>(h->d, d_plans, d_jobs, d_ctl, ba, d_parts);
            else if (km == MODE_INTERSECT_SINGLE)
                ns_batch_kernel<MODE_INTERSECT_SINGLE, false>
                    <<<grid, block, smem, cs>>>(h->d, d_plans, d_jobs, d_ctl, ba, d_parts);
            else if (compact)
                ns_batch_kernel<MODE_INTERSECT, true>
                    <<<grid, block, smem, cs>>>(h->d, d_plans, d_jobs, d_ctl, ba, d_parts);
            else
                ns_batch_kernel<MODE_INTERSECT, false>
                    <<<grid, block, smem, cs>>>(h->d, d_plans, d_jobs, d_ctl, ba, d_parts);
            cudaEventRecordWithFlags(ev_k[2 * r + 1], cs, cudaEventRecordExternal);
            batch_reduce_check<<<nj, 1024, 0, cs>>>(d_parts, d_jobs, ba);
            batch_relayout<<<1, 32, 0, cs>>>(d_jobs, d_ctl, ba);
        }
        ce = cudaStreamEndCapture(cs, gr);
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(ex, *gr, 0);
        return ce;
    };
    if (e == cudaSuccess) e = capture(kmode, &graph, &exec);
    // a batch that mixes plans with and without single-list steps switches to
    // the smaller plain variant once no job that needs the other is running
    if (e == cudaSuccess && kmode == MODE_INTERSECT_SINGLE) {
        bool all_single = true;
        for (const Plan &pl : plans) all_single = all_single && plan_single_steps(pl);
        if (!all_single) e = capture(MODE_INTERSECT, &graph_plain, &exec_plain);
    }
    std::vector<float> round_ms;
    uint64_t launches = 0;
    cudaGraphExec_t cur = exec;
    while (e == cudaSuccess) {
        e = cudaEventRecord(ev_a, cs);
        if (e == cudaSuccess) e = cudaGraphLaunch(cur, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_b, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) break;
        for (int r = 0; r < R; r++) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev_k[2 * r], ev_k[2 * r + 1]);
            round_ms.push_back(ms);
        }
        launches += 3 * R;
        if (ctl.active == 0) break;
        if (exec_plain && !ctl.any_single) cur = exec_plain;
        if (h->abort_flag) {
            status = GPM_ERR_ABORTED;
            set_error("aborted");
            break;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (max_s > 0.0 && el >= max_s) {
            status = GPM_ERR_NOT_CONVERGED;
            set_error("max_seconds reached before eps_hat <= eps");
            break;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(jobs.data(), d_jobs, sizeof(BatchJob) * nj, cudaMemcpyDeviceToHost);
    // the caller's stream sees the batch as finished
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, ev_in, 0);
    if (e != cudaSuccess) {
        cleanup();
        set_error(std::string("batch: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    const double t_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // sampler time of the rounds that had work (later rounds of a graph launch are empty)
    uint64_t work_rounds = 0;
    for (uint32_t q = 0; q < nj; q++) work_rounds = jobs[q].rounds > work_rounds ? jobs[q].rounds : work_rounds;
    double t_kernel = 0.0;
    for (uint64_t r = 0; r < work_rounds && r < round_ms.size(); r++) t_kernel += round_ms[r] * 1e-3;
    bool all = true;
    for (uint32_t q = 0; q < nj; q++) {
        const BatchJob &J = jobs[q];
        gpm_result &o = results[q];
        std::memset(&o, 0, sizeof(o));
        o.estimate = J.mu;
        o.ci_half_width = J.half;
        o.eps_hat = J.eps_hat;
        o.sum = J.sum;
        o.sumsq = J.sumsq;
        o.samples = J.n;
        o.hits = J.hits;
        o.rounds = J.rounds;
        o.scheme_used = GPM_NS;
        o.converged = (int32_t)J.converged;
        o.t_total_s = t_total;
        o.t_sample_s = t_kernel;
        o.kernel_launches = launches;
        all = all && J.converged;
    }
    cleanup();
    if (cfg && cfg->bytes_sample && (status == GPM_OK || status == GPM_ERR_NOT_CONVERGED)) {
        for (uint32_t q = 0; q < nj; q++) {
            const gpm_status sb = algo_bytes_mean(h, plans[q], mode, seed, jobs[q].slot, cfg, cfg->bytes_sample,
                                                  &results[q].algo_bytes_per_sample);
            if (sb != GPM_OK) return sb;
        }
    }
    if (status == GPM_OK && !all) {
        status = GPM_ERR_NOT_CONVERGED;
        set_error("n_max reached before eps_hat <= eps for at least one job");
    }
    return status;
}

}  // namespace gpm

using namespace gpm;

extern "C" gpm_status gpm_estimate_batch(gpm_graph *h, uint32_t count, const gpm_pattern *patterns, const double *eps,
                                         double delta, uint64_t seed, const gpm_config *cfg, gpm_result *out) {
    if (!h || !patterns || !eps || !out || count == 0) {
        set_error("gpm_estimate_batch: null argument or empty batch");
        return GPM_ERR_ARG;
    }
    if (count > 1024) {
        set_error("gpm_estimate_batch: at most 1024 jobs");
        return GPM_ERR_ARG;
    }
    std::vector<Plan> plans(count);
    for (uint32_t q = 0; q < count; q++) {
        std::string why = build_plan(patterns[q], &plans[q]);
        if (!why.empty()) {
            set_error("pattern rejected: " + why);
            return GPM_ERR_ARG;
        }
    }
    h->abort_flag = 0;
    return batch_estimate(h, plans, eps, delta, seed, cfg, out, verify_mode(cfg));
}

extern "C" gpm_status gpm_autotune(gpm_graph *h, uint32_t count, const gpm_pattern *patterns, uint64_t seed,
                                   gpm_config *io) {
    if (!h || !patterns || !io || count == 0 || count > 1024) {
        set_error("gpm_autotune: null argument or bad batch size");
        return GPM_ERR_ARG;
    }
    std::vector<Plan> plans(count);
    for (uint32_t q = 0; q < count; q++) {
        std::string why = build_plan(patterns[q], &plans[q]);
        if (!why.empty()) {
            set_error("pattern rejected: " + why);
            return GPM_ERR_ARG;
        }
    }
    // the default shape first (cap 0 = the default buffer: 512 entries with a
    // vertex-induced plan, else the largest at full residency), then the
    // others; each shape is timed over 3 rounds, and another shape replaces
    // the default only when it is more than 2% faster
    static const uint32_t kShapes[][2] = {{8, 0}, {8, 256}, {8, 512}, {4, 256}, {4, 512}, {4, 0}};
    std::vector<double> eps(count, 1e-300);
    std::vector<gpm_result> res(count);
    bool induced = false;
    for (const Plan &pl : plans) induced = induced || pl.induced;
    double best = INFINITY, t_default = INFINITY;
    uint32_t bw = 8, bc = 0;
    for (const auto &shape : kShapes) {
        gpm_config t = *io;
        t.block_warps = shape[0];
        t.cap = shape[1];
        t.grid_blocks = 0;
        t.window = io->window ? io->window : (1ull << 18);
        t.n_min = t.window;
        t.n_max = 3 * t.window;
        const int mode = verify_mode(&t);
        gpm_status st = batch_estimate(h, plans, eps.data(), 0.01, seed, &t, res.data(), mode);
        if (st != GPM_OK && st != GPM_ERR_NOT_CONVERGED) return st;
        const double ts = res[0].t_sample_s;
        if (shape[0] == 8 && shape[1] == 0) t_default = ts;
        if (ts < best && (ts < 0.98 * t_default || (shape[0] == 8 && shape[1] == 0))) {
            best = ts;
            bw = shape[0];
            bc = shape[1];
        }
    }
    io->block_warps = bw;
    io->cap = bc ? bc : default_cap(h, kBatchStaticSmem, bw, verify_mode(io), induced);
    set_error("");
    return GPM_OK;
}
