// Neighbour sampling with eager verify (Sec. 4.2, Algorithm 4, Lemma 1) and
// online convergence detection (Sec. 4.1, Algorithm 3, Eq. equ:error).
//
// One warp draws one sample at a time.  Sample s takes its random words from
// Philox4x32-10 with counter (s_lo, s_hi, block, slot << 8) and key = seed;
// choice t is the 64-bit word pair (t mod 2) of block t / 2, and an index in
// [0, N) is floor(r * N / 2^64).
//
// Step j of a sample builds the candidate set
//   S_j = { x : x in N(v_i) for every pattern edge (i, j), i < j;
//               x not in N(v_i) for every pattern non-edge (i, j) if induced;
//               x distinct from v_0..v_{j-1}; x > v_a for each restriction a < j }
// in ascending order, draws x = S_j[floor(r * |S_j| / 2^64)], and multiplies
// the weight by |S_j|; an empty set ends the sample as a miss (weight 0).
// The weight starts at M = m (oriented first edge) or 2m.
//
// Layout: the warp keeps the partial match, the per-step factors and two
// candidate buffers of `cap` entries in shared memory; lane i holds the row
// start, degree and first-upper-neighbour offset of v_i (offsets inside a
// list are 32-bit).  S_j is built by streaming the shortest back-neighbour
// list (coalesced 128-byte warp loads) and testing each element against the
// other lists with per-lane binary searches, the next shortest list (its part
// above the bound) copied on chip by cp.async, whole or, when longer than
// `cap`, window by window, compacting survivors with ballots.  When S_j
// extends S_{j-1} by one more adjacency (cliques and similar), it is built
// from S_{j-1} on chip and only N(v_{j-1}) is read.  A set larger than `cap`
// is counted in one pass and its drawn element found in a second pass.  A step
// with a single back-neighbour (paths, stars, cycles) never builds S_j: its
// size and drawn element follow from positions in that neighbour's list, of
// the matched vertices (edge-induced) or also of the non-neighbours' entries
// (vertex-induced) (the MODE_INTERSECT_SINGLE variant).
//
// CHECK mode draws x from the single list L_j = N(v_p) above the lower bound
// (p the last back-neighbour), weighs |L_j|, and verifies the remaining
// conditions of S_j with one binary search per lane.
//
// Each warp accumulates sum X and sum X^2 (FP64, sample-index order) over a
// chunk of consecutive samples into a per-chunk partial; chunks are handed out
// by an atomic counter, and a single-block kernel adds the partials in chunk
// order, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "sampler.cuh"

namespace gpm {

// Algorithmic 32-byte sectors of a finished sample (trace mode only): the
// graph data the candidate-set definition of Sec. 4.2 references on the path
// the sample took, independent of how the kernel actually read it.  All
// lanes call it; v[] holds the matched vertices, fac[] the step factors.
//   first edge: 1 sector;
//   step j (every step taken; a miss at j ends after step j):
//     INTERSECT: per referenced list L (the back-neighbours of j, and every
//       earlier position when vertex-induced; only N(v_{j-1}) when S_j is
//       S_{j-1} cut by N(v_{j-1}): same earlier neighbours plus j-1, and every
//       lower bound of j-1 also bounds j), 1 sector for its row_ptr pair plus
//       the sectors spanned by its entries above the step's lower bound;
//     CHECK: 1 for the row_ptr pair of the drawn-from list N(v_p), a bound
//       search of ceil(log2(d + 1)) sectors when bounded, and when L_j is not
//       empty 1 for the drawn entry plus 1 + ceil(log2(d + 1)) per other
//       referenced list (its membership search).
__device__ __forceinline__ uint32_t log2_ceil_plus1(uint64_t d) { return 64u - (uint32_t)__clzll((long long)d); }

template <int MODE>
__device__ uint32_t algo_sectors(const DGraph &g, const Plan &p, const uint32_t *v, const uint64_t *fac, int depth,
                                 bool hit) {
    uint32_t sec = 1;
    if (MODE == MODE_LAZY) {
        // NS-base: whole back-neighbour lists per step, one search per checked pair
        if (depth < p.k) return sec;
        for (int j = 2; j < p.k; j++)
            for (int i = 0; i < j; i++)
                if ((p.back[j] >> i) & 1u) {
                    const uint64_t rb = __ldg(g.row_ptr + v[i]), re = __ldg(g.row_ptr + v[i] + 1);
                    sec += 1u + (re > rb ? (uint32_t)((re * 4 + 31) / 32 - (rb * 4) / 32) : 0u);
                }
        for (int j = 1; j < p.k; j++)
            for (int i = 0; i < j; i++)
                if (((p.back[j] >> i) & 1u) || p.induced)
                    sec += 1u + log2_ceil_plus1(__ldg(g.row_ptr + v[i] + 1) - __ldg(g.row_ptr + v[i]));
        return sec;
    }
    const int steps = hit ? p.k : depth + 1;
    for (int j = 2; j < steps && j < p.k; j++) {
        const uint32_t lm = p.lower[j];
        uint32_t lo = 0;
        for (int i = 0; i < j; i++)
            if ((lm >> i) & 1u) lo = v[i] > lo ? v[i] : lo;
        if (MODE == MODE_CHECK) {
            const int pb = (int)p.last_back[j];
            const uint64_t dpb = __ldg(g.row_ptr + v[pb] + 1) - __ldg(g.row_ptr + v[pb]);
            sec += 1u + (lm ? log2_ceil_plus1(dpb) : 0u);
            if (fac[j] == 0) continue;
            sec += 1u;
            for (int i = 0; i < j; i++) {
                const bool edge = (p.back[j] >> i) & 1u;
                if (i == pb || (!edge && !p.induced)) continue;
                const uint64_t di = __ldg(g.row_ptr + v[i] + 1) - __ldg(g.row_ptr + v[i]);
                sec += 1u + log2_ceil_plus1(di);
            }
            continue;
        }
        const uint32_t below = (1u << (j - 1)) - 1u;
        const bool reuse = j >= 3 && (p.back[j] & below) == p.back[j - 1] && ((p.back[j] >> (j - 1)) & 1u) &&
                           (p.lower[j - 1] & ~lm) == 0;
        for (int i = 0; i < j; i++) {
            const bool edge = (p.back[j] >> i) & 1u;
            if (!edge && !p.induced) continue;
            if (reuse && i != j - 1) continue;
            const uint64_t rb = __ldg(g.row_ptr + v[i]), re = __ldg(g.row_ptr + v[i] + 1);
            const uint64_t b = lm ? rb + warp_upper_bound(g.col + rb, re - rb, lo) : rb;
            if (re > b) sec += 1u + (uint32_t)((re * 4 + 31) / 32 - (b * 4) / 32);
            else sec += 1u;
        }
    }
    return sec;
}

template <int MODE, bool TRACE>
__global__ void __launch_bounds__(256, (MODE == MODE_LEARNED) ? 2 : GPM_MIN_BLOCKS) ns_kernel(const DGraph g, const Plan p, const RunArgs a) {
    extern __shared__ __align__(16) uint64_t smem64[];
    const unsigned lane = lane_id();
    WarpMem wm = warp_mem<MODE>(smem64, a.cap, a.mlp);
    const uint64_t end = a.first + a.count;
    for (;;) {
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(a.counter, 1u);
        c = __shfl_sync(kFull, c, 0);
        if (c >= a.nchunks) break;
        const uint64_t s0 = a.first + (uint64_t)c * a.stride * a.chunk;
        const uint64_t s1 = (s0 + a.chunk < end) ? s0 + a.chunk : end;
        double sum = 0.0, sumsq = 0.0;
        uint64_t hits = 0;
        for (uint64_t s = s0; s < s1; s++) {
            if (TRACE && lane < kMaxK) {
                wm.fac[lane] = 0;
                wm.aux[lane] = 0;
            }
            __syncwarp();
            const SampleOut r = sample_one<MODE>(g, p, a, s, wm);
            if (r.hit) {
                sum = __dadd_rn(sum, r.w);
                sumsq = __dadd_rn(sumsq, __dmul_rn(r.w, r.w));
                hits++;
            }
            if (TRACE) {
                __syncwarp();
                const uint32_t sectors = algo_sectors<(MODE == MODE_CHECK || MODE == MODE_LAZY) ? MODE : MODE_INTERSECT>(
                    g, p, wm.v, wm.fac, r.hit ? p.k : r.depth, r.hit);
                gpm_sample_record *rec = a.trace + (s - a.first);
                if (lane < kMaxK) {
                    rec->factor[lane] = wm.fac[lane];
                    rec->vert[lane] = ((int)lane < r.depth && (int)lane < p.k) ? wm.v[lane] : 0xFFFFFFFFu;
                    rec->aux[lane] = wm.aux[lane];
                }
                if (lane == 0) {
                    rec->w_u64 = r.hit ? r.wu : 0;
                    rec->w_f64 = r.hit ? r.w : 0.0;
                    rec->hit = r.hit;
                    rec->depth = (uint8_t)(r.hit ? p.k : r.depth);
                    rec->overflow = r.overflow;
                    rec->pad = 0;
                    rec->sectors = sectors;
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            Partial q;
            q.sum = sum;
            q.sumsq = sumsq;
            q.hits = hits;
            q.n = s1 - s0;
            a.partials[c] = q;
        }
    }
}

// Adds the partials in chunk order (each thread a contiguous run, then a
// fixed-shape tree) and folds them into the running totals.
__global__ void __launch_bounds__(1024) reduce_partials(const Partial *__restrict__ parts, uint32_t n, Totals *tot,
                                                        int accumulate) {
    __shared__ double s_sum[1024], s_sq[1024];
    __shared__ unsigned long long s_hits[1024], s_n[1024];
    const unsigned t = threadIdx.x;
    const uint32_t per = (n + 1023) / 1024;
    const uint64_t b = (uint64_t)t * per;
    const uint64_t e = (b + per < n) ? b + per : n;
    double sum = 0.0, sq = 0.0;
    unsigned long long hits = 0, cnt = 0;
    for (uint64_t i = b; i < e; i++) {
        sum = __dadd_rn(sum, parts[i].sum);
        sq = __dadd_rn(sq, parts[i].sumsq);
        hits += parts[i].hits;
        cnt += parts[i].n;
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
        if (accumulate) {
            tot->sum = __dadd_rn(tot->sum, s_sum[0]);
            tot->sumsq = __dadd_rn(tot->sumsq, s_sq[0]);
            tot->hits += s_hits[0];
            tot->n += s_n[0];
        } else {
            tot->sum = s_sum[0];
            tot->sumsq = s_sq[0];
            tot->hits = s_hits[0];
            tot->n = s_n[0];
        }
    }
}

template <int MODE, bool TRACE>
static cudaError_t launch_ns(gpm_graph *h, const Plan &p, const Shape &sh, const RunArgs &a) {
    auto kern = ns_kernel<MODE, TRACE>;
    const size_t smem = smem_bytes(sh, MODE);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    uint32_t blocks = sh.blocks;
    if (blocks == 0) {
        // persistent grid: as many blocks as stay resident on every SM
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)(sh.warps * 32), smem);
        if (e != cudaSuccess) return e;
        blocks = (uint32_t)((per_sm > 0 ? per_sm : 1) * h->sm_count);
    }
    kern<<<blocks, sh.warps * 32, smem, h->stream>>>(h->d, p, a);
    return cudaGetLastError();
}

// The compiled sampler variant for a kernel mode (kernel_mode's result).
template <bool TRACE>
static cudaError_t launch_mode(gpm_graph *h, const Plan &p, const Shape &sh, const RunArgs &a, int kmode) {
    switch (kmode) {
        case MODE_CHECK: return launch_ns<MODE_CHECK, TRACE>(h, p, sh, a);
        case MODE_LEARNED: return launch_ns<MODE_LEARNED, TRACE>(h, p, sh, a);
        case MODE_INTERSECT_SINGLE: return launch_ns<MODE_INTERSECT_SINGLE, TRACE>(h, p, sh, a);
        case MODE_LAZY: return launch_ns<MODE_LAZY, TRACE>(h, p, sh, a);
        default: return launch_ns<MODE_INTERSECT, TRACE>(h, p, sh, a);
    }
}

static gpm_status ensure_partials(gpm_graph *h, uint64_t n) {
    if (h->partials_cap >= n) return GPM_OK;
    pool_free(h->partials, h->stream);
    h->partials = nullptr;
    h->partials_cap = 0;
    if (pool_alloc((void **)&h->partials, sizeof(Partial) * n, h->stream) != cudaSuccess) {
        set_error("device allocation of the per-chunk partials failed");
        return GPM_ERR_OOM;
    }
    h->partials_cap = n;
    return GPM_OK;
}

// One sampling launch over [first, first + count) plus the chunk-order
// reduction into h->totals[0] (accumulate = fold into the running totals).
// With world > 1 only the chunks c = rank (mod world) of the range are drawn
// (h->partials then holds them in that order).
static gpm_status run_block(gpm_graph *h, const Plan &p, int mode, uint64_t seed, uint32_t slot, uint64_t first,
                            uint64_t count, const gpm_config *cfg, int accumulate, gpm_sample_record *trace,
                            float *kernel_ms, uint32_t rank = 0, uint32_t world = 1, uint64_t *nchunks_out = nullptr) {
    Shape sh = pick_shape(h, cfg, count);
    if (sh.cap == 0) sh.cap = default_cap(h, 0, sh.warps, mode, p.induced);   // ns_kernel: no static shared memory
    if (mode == MODE_LEARNED && sh.cap < kLearnedMax) sh.cap = kLearnedMax;
    const uint64_t all_chunks = (count + sh.chunk - 1) / sh.chunk;
    const uint64_t nchunks = (rank < all_chunks) ? (all_chunks - rank + world - 1) / world : 0;
    if (nchunks_out) *nchunks_out = nchunks;
    first += (uint64_t)rank * sh.chunk;
    count = (nchunks > 0) ? count - (uint64_t)rank * sh.chunk : 0;
    if (nchunks >= (1ull << 31)) {
        set_error("too many samples in one launch");
        return GPM_ERR_ARG;
    }
    gpm_status st = ensure_partials(h, nchunks ? nchunks : 1);
    if (st != GPM_OK) return st;
    RunArgs a;
    a.seed = seed;
    a.first = first;
    a.count = count;
    a.partials = h->partials;
    a.counter = h->counter;
    a.trace = trace;
    a.slot = slot;
    a.cap = sh.cap;
    a.chunk = sh.chunk;
    a.nchunks = (uint32_t)nchunks;
    a.stride = world;
    std::memset(&a.mlp, 0, sizeof(a.mlp));
    if (mode == MODE_LEARNED) a.mlp = *cfg->mlp;
    a.mlp_tc = (mode == MODE_LEARNED && cfg->mlp_tensor) ? 1u : 0u;
    if (cudaMemsetAsync(h->counter, 0, sizeof(unsigned int), h->stream) != cudaSuccess) {
        set_error("cudaMemsetAsync failed");
        return GPM_ERR_CUDA;
    }
    if (kernel_ms) cudaEventRecord(h->ev0, h->stream);
    const int kmode = kernel_mode(mode, plan_single_steps(p));
    cudaError_t e = trace ? launch_mode<true>(h, p, sh, a, kmode) : launch_mode<false>(h, p, sh, a, kmode);
    if (kernel_ms) cudaEventRecord(h->ev1, h->stream);
    if (e != cudaSuccess) {
        set_error(std::string("sampler launch: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    reduce_partials<<<1, 1024, 0, h->stream>>>(h->partials, (uint32_t)nchunks, h->totals, accumulate);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->totals_host, h->totals, sizeof(Totals), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        set_error(std::string("sampling round: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    if (kernel_ms) cudaEventElapsedTime(kernel_ms, h->ev0, h->ev1);
    return GPM_OK;
}

static gpm_status plan_or_error(const gpm_pattern *pat, Plan *p) {
    if (!pat) {
        set_error("null pattern");
        return GPM_ERR_ARG;
    }
    std::string why = build_plan(*pat, p);
    if (!why.empty()) {
        set_error("pattern rejected: " + why);
        return GPM_ERR_ARG;
    }
    return GPM_OK;
}

// gpm_sample_sums / gpm_trace: weights in cfg->mlp select the learned proposal
static int mode_of(const gpm_config *cfg) {
    if (cfg && cfg->mlp) return MODE_LEARNED;
    return verify_mode(cfg);
}

// Phi^-1 by Newton iteration on the complementary error function, solved in
// the lower tail (where erfc keeps full relative accuracy) and mirrored:
// Phi(x) = erfc(-x / sqrt 2) / 2 and Phi'(x) = exp(-x^2 / 2) / sqrt(2 pi);
// a bisection bracket on [-40, 0] gives the starting point.
double normal_quantile(double p) {
    if (!(p > 0.0 && p < 1.0)) return std::nan("");
    const bool upper = p > 0.5;
    const double q = upper ? 1.0 - p : p;
    if (q == 0.5) return 0.0;
    const double rs2 = 0.70710678118654752440;
    double lo = -40.0, hi = 0.0;
    for (int i = 0; i < 80 && hi - lo > 1e-3; i++) {
        const double mid = 0.5 * (lo + hi);
        if (0.5 * std::erfc(-mid * rs2) < q) lo = mid;
        else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    const double inv_sqrt_2pi = 0.39894228040143267794;
    for (int i = 0; i < 60; i++) {
        const double c = 0.5 * std::erfc(-x * rs2);
        const double d = inv_sqrt_2pi * std::exp(-0.5 * x * x);
        if (d == 0.0) break;
        const double step = (c - q) / d;
        x -= step;
        if (std::fabs(step) <= 1e-16 * std::fabs(x)) break;
    }
    return upper ? -x : x;
}

// A single NS estimate is a batch of one job (rounds in a captured CUDA
// graph, Eq. equ:error evaluated on the device after each round).
gpm_status ns_estimate(gpm_graph *h, const Plan &p, double eps, double delta, uint64_t seed,
                       const gpm_config *cfg, gpm_result *out) {
    if (!(eps > 0.0) || !(delta > 0.0 && delta < 1.0)) {
        set_error("eps must be > 0 and delta in (0, 1)");
        return GPM_ERR_ARG;
    }
    h->abort_flag = 0;
    std::vector<Plan> plans(1, p);
    return batch_estimate(h, plans, &eps, delta, seed, cfg, out, verify_mode(cfg));
}

// NS with the learned proposal: the same rounds, candidates drawn by score.
gpm_status learned_estimate(gpm_graph *h, const Plan &p, double eps, double delta, uint64_t seed,
                            const gpm_config *cfg, gpm_result *out) {
    if (!cfg || !cfg->mlp || !cfg->mlp->w1 || !cfg->mlp->b1 || !cfg->mlp->w2 || !cfg->mlp->b2 || !cfg->mlp->w3 ||
        !cfg->mlp->b3) {
        set_error("GPM_NS_LEARNED needs cfg->mlp with all six device weight arrays");
        return GPM_ERR_ARG;
    }
    if (!(eps > 0.0) || !(delta > 0.0 && delta < 1.0)) {
        set_error("eps must be > 0 and delta in (0, 1)");
        return GPM_ERR_ARG;
    }
    h->abort_flag = 0;
    std::vector<Plan> plans(1, p);
    gpm_status st = batch_estimate(h, plans, &eps, delta, seed, cfg, out, MODE_LEARNED);
    out->scheme_used = GPM_NS_LEARNED;
    return st;
}

}  // namespace gpm

using namespace gpm;

namespace gpm {
// Records of samples [first, first + count) into a device buffer.
gpm_status trace_device(gpm_graph *h, const Plan &p, uint64_t seed, uint64_t first, uint64_t count,
                        const gpm_config *cfg, gpm_sample_record *d_out) {
    return run_block(h, p, mode_of(cfg), seed, cfg ? cfg->slot : 0, first, count, cfg, 0, d_out, nullptr);
}
// Mean of the records' algorithmic bytes over samples [0, count) of a run's
// stream (seed, slot, mode as the run), for gpm_result.algo_bytes_per_sample.
gpm_status algo_bytes_mean(gpm_graph *h, const Plan &p, int mode, uint64_t seed, uint32_t slot,
                           const gpm_config *cfg, uint64_t count, double *out) {
    *out = 0.0;
    if (count == 0) return GPM_OK;
    gpm_sample_record *d = nullptr;
    if (cudaMalloc((void **)&d, sizeof(gpm_sample_record) * count) != cudaSuccess) {
        set_error("algorithmic bytes: device allocation of the trace failed");
        return GPM_ERR_OOM;
    }
    std::vector<gpm_sample_record> rec(count);
    gpm_status st = run_block(h, p, mode, seed, slot, 0, count, cfg, 0, d, nullptr);
    if (st == GPM_OK && cudaMemcpy(rec.data(), d, sizeof(gpm_sample_record) * count, cudaMemcpyDeviceToHost) !=
                            cudaSuccess) {
        set_error("algorithmic bytes: copy back failed");
        st = GPM_ERR_CUDA;
    }
    cudaFree(d);
    if (st != GPM_OK) return st;
    uint64_t sec = 0;
    for (const auto &r : rec) sec += r.sectors;
    *out = 32.0 * (double)sec / (double)count;
    return GPM_OK;
}

}  // namespace gpm

extern "C" gpm_status gpm_sample_sums(gpm_graph *h, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                                      uint64_t count, const gpm_config *cfg, gpm_sums *out) {
    if (!h || !out) {
        set_error("gpm_sample_sums: null argument");
        return GPM_ERR_ARG;
    }
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    std::memset(out, 0, sizeof(*out));
    if (count == 0) return GPM_OK;
    st = run_block(h, p, mode_of(cfg), seed, cfg ? cfg->slot : 0, first, count, cfg, 0, nullptr, nullptr);
    if (st != GPM_OK) return st;
    out->n = h->totals_host->n;
    out->hits = h->totals_host->hits;
    out->sum = h->totals_host->sum;
    out->sumsq = h->totals_host->sumsq;
    return GPM_OK;
}

extern "C" gpm_status gpm_sample_partials(gpm_graph *h, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                                          uint64_t count, uint32_t rank, uint32_t world, const gpm_config *cfg,
                                          gpm_partial *out, uint64_t *n_out) {
    if (!h || !n_out || world == 0 || rank >= world) {
        set_error("gpm_sample_partials: null argument or rank >= world");
        return GPM_ERR_ARG;
    }
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    *n_out = 0;
    const uint64_t mine = (count + kChunk - 1) / kChunk > rank ? ((count + kChunk - 1) / kChunk - rank + world - 1) / world : 0;
    if (mine == 0) return GPM_OK;
    if (!out) {
        set_error("gpm_sample_partials: null output array");
        return GPM_ERR_ARG;
    }
    uint64_t n = 0;
    st = run_block(h, p, mode_of(cfg), seed, cfg ? cfg->slot : 0, first, count, cfg, 0, nullptr, nullptr, rank, world,
                   &n);
    if (st != GPM_OK) return st;
    static_assert(sizeof(gpm_partial) == sizeof(Partial), "partial layout");
    if (cudaMemcpy(out, h->partials, sizeof(Partial) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("gpm_sample_partials: copy back failed");
        return GPM_ERR_CUDA;
    }
    *n_out = n;
    return GPM_OK;
}

// ------------------------------------------------------------------ run blocks (multi-GPU rounds)
// The chunk-order reduction of a round (reduce_partials) adds 1024 contiguous
// runs of ceil(nchunks / 1024) chunks left to right and then folds the runs
// pairwise.  Rank r of `world` takes the runs [r B, (r + 1) B), B =
// ceil(1024 / world): one contiguous range of chunks, hence of samples, whose
// run sums it computes on its GPU exactly as the single-GPU reduction would.
namespace gpm {

constexpr uint32_t kRuns = 1024;

// Run sums of a rank's chunks: run t adds partials [t per, min((t + 1) per, n))
// left to right (one thread per run).
__global__ void reduce_runs(const Partial *__restrict__ parts, uint32_t n, uint32_t per, uint32_t nruns,
                            Partial *out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nruns) return;
    const uint64_t b = (uint64_t)t * per;
    const uint64_t e = (b + per < n) ? b + per : n;
    Partial q;
    q.sum = 0.0;
    q.sumsq = 0.0;
    q.hits = 0;
    q.n = 0;
    for (uint64_t i = b; i < e; i++) {
        q.sum = __dadd_rn(q.sum, parts[i].sum);
        q.sumsq = __dadd_rn(q.sumsq, parts[i].sumsq);
        q.hits += parts[i].hits;
        q.n += parts[i].n;
    }
    out[t] = q;
}

// This rank's run sums of samples [first, first + count) into host out[B].
static gpm_status sample_runs(gpm_graph *h, const Plan &p, int mode, uint64_t seed, uint32_t slot, uint64_t first,
                              uint64_t count, uint32_t rank, uint32_t world, const gpm_config *cfg, gpm_partial *out) {
    const uint32_t B = (kRuns + world - 1) / world;
    std::memset(out, 0, sizeof(gpm_partial) * B);
    const uint64_t nch = (count + kChunk - 1) / kChunk;
    const uint64_t per = (nch + kRuns - 1) / kRuns;
    const uint64_t run_lo = (uint64_t)rank * B;
    const uint64_t run_hi = std::min<uint64_t>(run_lo + B, kRuns);
    const uint64_t c_lo = std::min<uint64_t>(run_lo * per, nch), c_hi = std::min<uint64_t>(run_hi * per, nch);
    if (run_lo >= run_hi || c_lo >= c_hi) return GPM_OK;
    const uint64_t s_lo = c_lo * kChunk, s_hi = std::min<uint64_t>(c_hi * kChunk, count);
    const uint64_t nloc = c_hi - c_lo;
    const uint32_t nruns = (uint32_t)(run_hi - run_lo);
    // room for the chunk partials and, after them, the run sums (before sampling:
    // growing the array later would drop the partials)
    gpm_status st = ensure_partials(h, nloc + nruns);
    if (st != GPM_OK) return st;
    st = run_block(h, p, mode, seed, slot, first + s_lo, s_hi - s_lo, cfg, 0, nullptr, nullptr);
    if (st != GPM_OK) return st;
    Partial *d_runs = h->partials + nloc;
    reduce_runs<<<(nruns + 127) / 128, 128, 0, h->stream>>>(h->partials, (uint32_t)nloc, (uint32_t)per, nruns,
                                                            d_runs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_runs, sizeof(Partial) * nruns, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        set_error(std::string("run sums: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    return GPM_OK;
}

// The pairwise tree over 1024 run sums (the second half of reduce_partials).
static void merge_runs(const gpm_partial *runs, gpm_sums *out) {
    std::vector<double> s_sum(kRuns), s_sq(kRuns);
    std::vector<uint64_t> s_hits(kRuns), s_n(kRuns);
    for (uint32_t t = 0; t < kRuns; t++) {
        s_sum[t] = runs[t].sum;
        s_sq[t] = runs[t].sumsq;
        s_hits[t] = runs[t].hits;
        s_n[t] = runs[t].n;
    }
    for (uint32_t hh = kRuns / 2; hh; hh >>= 1)
        for (uint32_t t = 0; t < hh; t++) {
            s_sum[t] = rn_add(s_sum[t], s_sum[t + hh]);
            s_sq[t] = rn_add(s_sq[t], s_sq[t + hh]);
            s_hits[t] += s_hits[t + hh];
            s_n[t] += s_n[t + hh];
        }
    out->n = s_n[0];
    out->hits = s_hits[0];
    out->sum = s_sum[0];
    out->sumsq = s_sq[0];
}

}  // namespace gpm

extern "C" gpm_status gpm_sample_runs(gpm_graph *h, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                                      uint64_t count, uint32_t rank, uint32_t world, const gpm_config *cfg,
                                      gpm_partial *out) {
    if (!h || !out || world == 0 || world > kRuns || rank >= world) {
        set_error("gpm_sample_runs: null argument, world outside 1..1024 or rank >= world");
        return GPM_ERR_ARG;
    }
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    return sample_runs(h, p, mode_of(cfg), seed, cfg ? cfg->slot : 0, first, count, rank, world, cfg, out);
}

extern "C" gpm_status gpm_merge_runs(const gpm_partial *runs, gpm_sums *out) {
    if (!runs || !out) {
        set_error("gpm_merge_runs: null argument");
        return GPM_ERR_ARG;
    }
    merge_runs(runs, out);
    return GPM_OK;
}

extern "C" gpm_status gpm_estimate_sharded(gpm_graph *h, const gpm_pattern *pattern, double eps, double delta,
                                           uint64_t seed, uint32_t rank, uint32_t world, const gpm_config *cfg,
                                           gpm_allgather_fn gather, void *ctx, gpm_window *state,
                                           uint64_t max_rounds, gpm_result *out) {
    if (!h || !out || !gather || world == 0 || world > kRuns || rank >= world) {
        set_error("gpm_estimate_sharded: null argument, world outside 1..1024 or rank >= world");
        return GPM_ERR_ARG;
    }
    if (!(eps > 0.0) || !(delta > 0.0 && delta < 1.0)) {
        set_error("eps must be > 0 and delta in (0, 1)");
        return GPM_ERR_ARG;
    }
    std::memset(out, 0, sizeof(*out));
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    const uint64_t W = (cfg && cfg->window) ? cfg->window : (1ull << 20);
    const uint64_t n_min = (cfg && cfg->n_min) ? cfg->n_min : W;
    const uint64_t n_max = (cfg && cfg->n_max) ? cfg->n_max : (1ull << 40);
    const double max_s = cfg ? cfg->max_seconds : 0.0;
    const double z = normal_quantile(1.0 - delta / 2.0);
    const int mode = mode_of(cfg);
    const uint32_t B = (kRuns + world - 1) / world;
    gpm_window w;
    if (state) {
        w = *state;
    } else {
        std::memset(&w, 0, sizeof(w));
        w.active = 1;
    }
    std::vector<gpm_partial> mine(B), all((size_t)B * world);
    h->abort_flag = 0;
    uint64_t done = 0, launches = 0;
    double t_sample = 0.0;
    while (w.active && (max_rounds == 0 || done < max_rounds)) {
        const auto ta = std::chrono::steady_clock::now();
        st = sample_runs(h, p, mode, seed, cfg ? cfg->slot : 0, w.rounds * W, W, rank, world, cfg, mine.data());
        if (st != GPM_OK) return st;
        t_sample += std::chrono::duration<double>(std::chrono::steady_clock::now() - ta).count();
        launches += 3;
        if (gather(ctx, mine.data(), all.data(), sizeof(gpm_partial) * B) != 0) {
            set_error("gpm_estimate_sharded: the gather callback failed");
            return GPM_ERR_COMM;
        }
        gpm_sums win;
        merge_runs(all.data(), &win);
        gpm_window_update(&w, &win, z, eps, n_min, n_max);
        done++;
        if (h->abort_flag) {
            st = GPM_ERR_ABORTED;
            set_error("aborted");
            break;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (w.active && max_s > 0.0 && el >= max_s) {
            st = GPM_ERR_NOT_CONVERGED;
            set_error("max_seconds reached before eps_hat <= eps");
            break;
        }
    }
    if (state) *state = w;
    out->estimate = w.mu;
    out->ci_half_width = w.half;
    out->eps_hat = w.eps_hat;
    out->sum = w.sum;
    out->sumsq = w.sumsq;
    out->samples = w.n;
    out->hits = w.hits;
    out->rounds = w.rounds;
    out->scheme_used = (mode == MODE_LEARNED) ? GPM_NS_LEARNED : GPM_NS;
    out->converged = (int32_t)w.converged;
    out->t_sample_s = t_sample;
    out->kernel_launches = launches;
    out->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (st == GPM_OK && !w.converged && !w.active) {
        st = GPM_ERR_NOT_CONVERGED;
        set_error("n_max reached before eps_hat <= eps");
    }
    return st;
}

extern "C" gpm_status gpm_merge_partials(const gpm_partial *parts, uint64_t n, gpm_sums *out) {
    if (!out || (n && !parts) || n >= (1ull << 32)) {
        set_error("gpm_merge_partials: null argument or n >= 2^32");
        return GPM_ERR_ARG;
    }
    // the reduction of reduce_partials / batch_reduce_check, written out on the host
    std::vector<double> s_sum(1024), s_sq(1024);
    std::vector<uint64_t> s_hits(1024), s_n(1024);
    const uint32_t per = (uint32_t)((n + 1023) / 1024);
    for (uint32_t t = 0; t < 1024; t++) {
        const uint64_t b = (uint64_t)t * per;
        const uint64_t e = (b + per < n) ? b + per : n;
        double sum = 0.0, sq = 0.0;
        uint64_t hits = 0, cnt = 0;
        for (uint64_t i = b; i < e; i++) {
            sum = rn_add(sum, parts[i].sum);
            sq = rn_add(sq, parts[i].sumsq);
            hits += parts[i].hits;
            cnt += parts[i].n;
        }
        s_sum[t] = sum;
        s_sq[t] = sq;
        s_hits[t] = hits;
        s_n[t] = cnt;
    }
    for (uint32_t hh = 512; hh; hh >>= 1)
        for (uint32_t t = 0; t < hh; t++) {
            s_sum[t] = rn_add(s_sum[t], s_sum[t + hh]);
            s_sq[t] = rn_add(s_sq[t], s_sq[t + hh]);
            s_hits[t] += s_hits[t + hh];
            s_n[t] += s_n[t + hh];
        }
    out->n = s_n[0];
    out->hits = s_hits[0];
    out->sum = s_sum[0];
    out->sumsq = s_sq[0];
    return GPM_OK;
}

extern "C" gpm_status gpm_window_update(gpm_window *w, const gpm_sums *win, double z, double eps, uint64_t n_min,
                                       uint64_t n_max) {
    if (!w || !win || !(eps > 0.0) || !(z > 0.0)) {
        set_error("gpm_window_update: null argument, eps <= 0 or z <= 0");
        return GPM_ERR_ARG;
    }
    if (!w->active) {
        set_error("gpm_window_update: the run has stopped");
        return GPM_ERR_ARG;
    }
    // as batch_reduce_check: the first window is assigned, later ones added
    if (w->rounds == 0) {
        w->sum = win->sum;
        w->sumsq = win->sumsq;
    } else {
        w->sum = rn_add(w->sum, win->sum);
        w->sumsq = rn_add(w->sumsq, win->sumsq);
    }
    w->hits += win->hits;
    w->n += win->n;
    w->rounds += 1;
    window_test(w->sum, w->sumsq, w->n, z, eps, n_min, n_max, &w->mu, &w->half, &w->eps_hat, &w->converged, &w->active);
    return GPM_OK;
}

extern "C" gpm_status gpm_trace(gpm_graph *h, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                                uint64_t count, const gpm_config *cfg, gpm_sample_record *out) {
    if (!h || (!out && count)) {
        set_error("gpm_trace: null argument");
        return GPM_ERR_ARG;
    }
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    if (count == 0) return GPM_OK;
    gpm_sample_record *d = nullptr;
    if (cudaMalloc((void **)&d, sizeof(gpm_sample_record) * count) != cudaSuccess) {
        set_error("gpm_trace: device allocation failed");
        return GPM_ERR_OOM;
    }
    st = run_block(h, p, mode_of(cfg), seed, cfg ? cfg->slot : 0, first, count, cfg, 0, d, nullptr);
    if (st == GPM_OK) {
        cudaError_t e = cudaMemcpy(out, d, sizeof(gpm_sample_record) * count, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error(std::string("gpm_trace: copy back: ") + cudaGetErrorString(e));
            st = GPM_ERR_CUDA;
        }
    }
    cudaFree(d);
    return st;
}

extern "C" gpm_status gpm_plan(const gpm_pattern *pattern, int32_t *order, int32_t *res_lo, int32_t *res_hi,
                               int32_t *nres, int32_t *oriented) {
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    if (order)
        for (int j = 0; j < p.k; j++) order[j] = p.order[j];
    if (res_lo && res_hi)
        for (int r = 0; r < p.nres; r++) {
            res_lo[r] = p.res_lo[r];
            res_hi[r] = p.res_hi[r];
        }
    if (nres) *nres = p.nres;
    if (oriented) *oriented = p.oriented;
    return GPM_OK;
}

extern "C" double gpm_normal_quantile(double p) { return normal_quantile(p); }

// ------------------------------------------------------------------ hybrid
namespace gpm {

// Loose mode (Sec. 5.1): a pilot NS round on G gives the per-sample mean and
// variance, the hit rate and the device time per sample; the NS cost model
// (Sec. 4.3) turns them into a cone [t_lo, t_hi] = N_s * c_step * [1, k - 2]
// with N_s = (z * sd / (eps * mu))^2 samples and c_step the pilot's time per
// candidate-set step (the lower edge is every sample breaking at its first
// set, the upper edge none breaking).  The GS model (Sec. 4.4) adds the
// sparsification pass |E| (w1 + p w2) at streaming bandwidth and the nested
// loops of the exact search, whose level sizes follow the GraphPi estimates
// on the sparsified graph (|V'| = |V|, |E'| = p|E|, T' = p^2 T): an extension
// by one neighbour costs the mean degree 2|E'|/|V|, an intersection of b
// lists |V| p1 p2^(b-1) with p1 = 2|E'|/|V|^2 and p2 = T|V| / (2|E|^2) (the
// substitution leaves p2 unchanged).  T comes from a short NS triangle pilot.
// GS runs only if its prediction lies below the whole cone and its error
// bound (below) allows the target; otherwise NS (the confidence-preserving
// choice).
struct HybridModel {
    double n_s, t_lo, t_hi, t_gs, t_pre, t_search, c_step, triangles;
    double gs_err_lb;   // lower bound on GS's relative error at 1 - delta
    int choose_gs;
};

gpm_status mlp_score_rows(gpm_graph *h, const gpm_mlp *mlp, const float *feat_host, uint64_t n, uint32_t *out_host);

static float clamp64(double x) {
    if (!(x == x)) return 0.f;
    return (float)(x > 64.0 ? 64.0 : (x < -64.0 ? -64.0 : x));
}

// Selector features: log2(t_gs / t_lo), log2(t_hi / t_lo), log2(n_s).
static void selector_features(const HybridModel &hm, float f[3]) {
    f[0] = clamp64(std::log2(hm.t_gs / hm.t_lo));
    f[1] = clamp64(std::log2(hm.t_hi / hm.t_lo));
    f[2] = clamp64(std::log2(hm.n_s));
}

static gpm_status hybrid_model(gpm_graph *h, const Plan &p, double eps, double delta, uint64_t seed,
                               const gpm_config *cfg, HybridModel *hm) {
    const uint64_t Wp = (cfg && cfg->window) ? cfg->window : (1ull << 20);
    const uint32_t slot = cfg ? cfg->slot : 0;
    const double z = normal_quantile(1.0 - delta / 2.0);
    float ms = 0.f;
    gpm_status st = run_block(h, p, MODE_INTERSECT, seed ^ 0x9E3779B97F4A7C15ull, slot, 0, Wp, cfg, 0, nullptr, &ms);
    if (st != GPM_OK) return st;
    Totals t = *h->totals_host;
    const double mu = t.sum / (double)t.n;
    const double var = std::max(0.0, t.sumsq / (double)t.n - mu * mu);
    const double t_sample = ms * 1e-3 / (double)t.n;
    // steps per sample from a traced slice of the pilot stream
    const uint64_t nt = 4096;
    gpm_sample_record *d = nullptr;
    std::vector<gpm_sample_record> rec(nt);
    if (cudaMalloc((void **)&d, sizeof(gpm_sample_record) * nt) != cudaSuccess) {
        set_error("hybrid: device allocation failed");
        return GPM_ERR_OOM;
    }
    st = run_block(h, p, MODE_INTERSECT, seed ^ 0x9E3779B97F4A7C15ull, slot, 0, nt, cfg, 0, d, nullptr);
    if (st == GPM_OK && cudaMemcpy(rec.data(), d, sizeof(gpm_sample_record) * nt, cudaMemcpyDeviceToHost) != cudaSuccess)
        st = GPM_ERR_CUDA;
    cudaFree(d);
    if (st != GPM_OK) return st;
    double steps = 0.0;
    for (const auto &r : rec) {
        int s_i = r.hit ? p.k - 2 : (r.depth >= 2 ? r.depth - 1 : 1);
        steps += s_i < 1 ? 1 : s_i;
    }
    steps /= (double)nt;
    const double c_step = t_sample / std::max(steps, 1.0);
    hm->c_step = c_step;
    hm->n_s = (mu > 0.0) ? std::ceil(z * z * var / (eps * eps * mu * mu)) : INFINITY;
    if (hm->n_s < (double)Wp) hm->n_s = (double)Wp;
    hm->t_lo = hm->n_s * c_step;
    hm->t_hi = hm->n_s * c_step * std::max(1, p.k - 2);

    // triangle count of G for the GraphPi estimate
    Plan tri;
    gpm_pattern tp;
    std::memset(&tp, 0, sizeof(tp));
    tp.k = 3;
    tp.adj[0] = 6;
    tp.adj[1] = 5;
    tp.adj[2] = 3;
    build_plan(tp, &tri);
    st = run_block(h, tri, MODE_INTERSECT, seed ^ 0x5851F42D4C957F2Dull, slot, 0, 1ull << 18, cfg, 0, nullptr, nullptr);
    if (st != GPM_OK) return st;
    const double T = h->totals_host->sum / (double)h->totals_host->n;
    hm->triangles = T;

    const double c = (cfg && cfg->colors) ? cfg->colors : 8;
    const double pk = 1.0 / c;
    const double V = (double)h->d.n, E = (double)h->d.m;
    const double Ep = E * pk;
    const double d_avg = V > 0 ? 2.0 * E / V : 0.0;
    const double d_sp = V > 0 ? 2.0 * Ep / V : 0.0;
    const double p1 = V > 0 ? 2.0 * Ep / (V * V) : 0.0;
    const double p2 = E > 0 ? T * V / (2.0 * E * E) : 0.0;
    // nested loops: iterations reaching level j times the set-op cost there,
    // in units of one sampler step (which scans about d_avg entries)
    double iters = p.oriented ? Ep : 2.0 * Ep;
    double work = 0.0;
    for (int j = 2; j < p.k; j++) {
        const int b = __builtin_popcount(p.back[j]);
        work += iters * (d_sp / std::max(d_avg, 1.0));
        const double z_j = (b <= 1) ? d_sp : V * p1 * std::pow(p2, (double)(b - 1));
        iters *= z_j;
    }
    const double bytes_pre = 4.0 * 2.0 * E * 2.0 + 4.0 * 2.0 * E * pk + 8.0 * V * 3.0;
    const double bw = 2.0e12;   // effective sparsification bandwidth (B/s), measured on GB300
    // a match survives the sparsification with probability P = c^-(k-1)
    // (Bernoulli edges: p^l, l pattern edges); R samplers are averaged
    const double R = (cfg && cfg->samplers > 1) ? (double)cfg->samplers : 1.0;
    double inv_p = std::pow(c, (double)(p.k - 1));
    if (cfg && cfg->edge_p > 0.0) {
        int l = 0;
        for (int j = 0; j < p.k; j++) l += __builtin_popcount(p.back[j]);
        inv_p = std::pow(1.0 / std::min(cfg->edge_p, 1.0), (double)l);
    }
    hm->t_pre = bytes_pre / bw;
    // the exact search visits every match of the sparsified graphs, R C P of
    // them by the pilot's C, each at least one sampler step's work: a floor
    // under the average-degree model, which a hub core makes far too low
    hm->t_search = std::max(work * c_step, (mu > 0.0 ? R * mu / inv_p : 0.0) * c_step);
    hm->t_gs = hm->t_pre + hm->t_search;
    // GS can only be chosen when its own error can meet the target (Sec. 5.2,
    // corrected): no two matches covary negatively, so Var(C_hat) >= C (1/P - 1)
    // and the relative error of R averaged samplers is at least
    // z sqrt((1/P - 1) / (R C)), C from the pilot's mean
    hm->gs_err_lb = (mu > 0.0) ? z * std::sqrt((inv_p - 1.0) / (R * mu)) : INFINITY;
    hm->choose_gs = hm->gs_err_lb <= eps && hm->t_gs < hm->t_lo;
    return GPM_OK;
}

// The decision: the selector head's score (GS iff a >= 2049, i.e. the logit
// is >= 0) when one is configured, else the cost-model rule.
static gpm_status hybrid_decide(gpm_graph *h, const Plan &p, double eps, double delta, uint64_t seed,
                                const gpm_config *cfg, HybridModel *hm, gpm_hybrid_info *info) {
    gpm_status st = hybrid_model(h, p, eps, delta, seed, cfg, hm);
    if (st != GPM_OK) return st;
    float f[3];
    selector_features(*hm, f);
    int sel = -1;
    if (cfg && cfg->selector) {
        uint32_t a = 0;
        st = mlp_score_rows(h, cfg->selector, f, 1, &a);
        if (st != GPM_OK) return st;
        sel = a >= 2049 ? 1 : 0;
    }
    if (info) {
        info->n_s = hm->n_s;
        info->t_lo = hm->t_lo;
        info->t_hi = hm->t_hi;
        info->t_gs = hm->t_gs;
        info->t_pre = hm->t_pre;
        info->t_search = hm->t_search;
        info->c_step = hm->c_step;
        info->triangles = hm->triangles;
        for (int i = 0; i < 3; i++) info->features[i] = f[i];
        info->cost_model_gs = hm->choose_gs;
        info->selector_gs = sel;
    }
    if (sel >= 0) hm->choose_gs = sel && hm->gs_err_lb <= eps;
    return GPM_OK;
}

static gpm_status hybrid_estimate(gpm_graph *h, const Plan &p, double eps, double delta, uint64_t seed,
                                  const gpm_config *cfg, gpm_result *out) {
    const auto t0 = std::chrono::steady_clock::now();
    HybridModel hm;
    gpm_status st = hybrid_decide(h, p, eps, delta, seed, cfg, &hm, nullptr);
    if (st != GPM_OK) return st;
    const double t_pilot = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (hm.choose_gs) st = gs_estimate(h, p, seed, delta, cfg, out);
    else st = ns_estimate(h, p, eps, delta, seed, cfg, out);
    out->t_pilot_s = t_pilot;
    out->kernel_launches += 6;
    out->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

}  // namespace gpm

namespace gpm {

// ------------------------------------------------------------------ sample-count profilers
// Two predictions of N_s, the samples NS needs for eps at 1 - delta (the NS
// cost model's input, Sec. 4.3), for comparison:
//  PILOT (this library's reading): CV^2 = var / mu^2 from one window of
//    samples on G itself, N_s = (z CV / eps)^2;
//  SPARSIFIED (Sec. 5.3's fast profiler): G' keeps each edge of G with
//    probability p (10% in the paper), NS-online runs on G' to an internal
//    error of 50% at the same confidence and stops after N_o samples with a
//    final predicted error eps_o; with per-sample CV^2 about 1 / rho for the
//    hit rate rho, CV'^2 = N_o (eps_o / z)^2 on G' transfers to G as
//    N_s = N_o (eps_o / eps)^2 rho(P, G') / rho(P, G), rho(P, G) from a short
//    hit-rate run on G.  The printed formula has eps_o unsquared and the
//    ratio of rho the other way round (neither is dimensionally consistent);
//    this is the reading that is.
gpm_status profile_samples(gpm_graph *h, const Plan &p, int kind, double frac, double eps, double delta,
                           uint64_t seed, const gpm_config *cfg, gpm_profile_info *out) {
    const auto t0 = std::chrono::steady_clock::now();
    std::memset(out, 0, sizeof(*out));
    out->kind = kind;
    const double z = normal_quantile(1.0 - delta / 2.0);
    const uint32_t slot = cfg ? cfg->slot : 0;
    if (kind == GPM_PROFILE_PILOT) {
        const uint64_t Wp = (cfg && cfg->window) ? cfg->window : (1ull << 20);
        gpm_status st = run_block(h, p, MODE_INTERSECT, seed ^ 0x9E3779B97F4A7C15ull, slot, 0, Wp, cfg, 0, nullptr,
                                  nullptr);
        if (st != GPM_OK) return st;
        const Totals t = *h->totals_host;
        const double mu = t.sum / (double)t.n;
        const double var = std::max(0.0, t.sumsq / (double)t.n - mu * mu);
        out->samples_used = t.n;
        out->rho_g = (double)t.hits / (double)t.n;
        out->n_s = mu > 0.0 ? z * z * var / (eps * eps * mu * mu) : INFINITY;
    } else if (kind == GPM_PROFILE_SPARSIFIED) {
        if (!(frac > 0.0 && frac <= 1.0)) {
            set_error("gpm_profile: the sparsified profiler needs 0 < frac <= 1");
            return GPM_ERR_ARG;
        }
        // G': every edge kept with probability frac (Algorithm 2's Bernoulli sampler)
        const uint64_t t_keep = frac >= 1.0 ? (1ull << 32) : (uint64_t)std::floor(frac * 4294967296.0);
        uint64_t *row = nullptr, kept = 0;
        uint32_t *col = nullptr;
        gpm_status st = sparsify_alloc(h, 1, seed ^ 0xD1B54A32D192ED03ull, 0, slot, &row, &col, &kept, nullptr,
                                       nullptr, t_keep ? t_keep : 1);
        if (st != GPM_OK) return st;
        gpm_graph *gp = nullptr;
        st = gpm_load_csr(h->d.n, row, col, GPM_DEVICE_PTRS, h->stream, &gp);
        gpm_result r;
        std::memset(&r, 0, sizeof(r));
        if (st == GPM_OK) {
            gpm_config c2;
            std::memset(&c2, 0, sizeof(c2));
            c2.window = 1ull << 14;
            c2.n_max = 1ull << 26;
            c2.slot = slot;
            c2.max_seconds = cfg ? cfg->max_seconds : 0.0;
            st = ns_estimate(gp, p, 0.5, delta, seed, &c2, &r);
            if (st == GPM_ERR_NOT_CONVERGED) st = GPM_OK;
        }
        if (gp) gpm_free_graph(gp);
        cudaFreeAsync(row, h->stream);
        cudaFreeAsync(col, h->stream);
        if (st != GPM_OK) return st;
        out->samples_used = r.samples;
        out->n_o = (double)r.samples;
        out->eps_o = r.eps_hat;
        out->rho_gp = r.samples ? (double)r.hits / (double)r.samples : 0.0;
        // rho(P, G) from a short run on G
        const uint64_t nh = 1ull << 16;
        st = run_block(h, p, MODE_INTERSECT, seed ^ 0x5851F42D4C957F2Dull, slot, 0, nh, cfg, 0, nullptr, nullptr);
        if (st != GPM_OK) return st;
        out->samples_used += nh;
        out->rho_g = (double)h->totals_host->hits / (double)h->totals_host->n;
        out->n_s = (out->rho_g > 0.0 && r.converged && out->eps_o > 0.0)
                       ? out->n_o * (out->eps_o / eps) * (out->eps_o / eps) * out->rho_gp / out->rho_g
                       : INFINITY;
    } else {
        set_error("gpm_profile: unknown profiler kind");
        return GPM_ERR_ARG;
    }
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return GPM_OK;
}

}  // namespace gpm

extern "C" gpm_status gpm_profile(gpm_graph *h, const gpm_pattern *pattern, int32_t kind, double frac, double eps,
                                  double delta, uint64_t seed, const gpm_config *cfg, gpm_profile_info *out) {
    if (!h || !out || !(eps > 0.0) || !(delta > 0.0 && delta < 1.0)) {
        set_error("gpm_profile: null argument, eps <= 0 or delta outside (0, 1)");
        return GPM_ERR_ARG;
    }
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    return profile_samples(h, p, kind, frac, eps, delta, seed, cfg, out);
}

extern "C" gpm_status gpm_hybrid_model(gpm_graph *h, const gpm_pattern *pattern, double eps, double delta,
                                       uint64_t seed, const gpm_config *cfg, gpm_hybrid_info *out) {
    if (!h || !out) {
        set_error("gpm_hybrid_model: null argument");
        return GPM_ERR_ARG;
    }
    if (!(eps > 0.0) || !(delta > 0.0 && delta < 1.0)) {
        set_error("eps must be > 0 and delta in (0, 1)");
        return GPM_ERR_ARG;
    }
    std::memset(out, 0, sizeof(*out));
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    HybridModel hm;
    return hybrid_decide(h, p, eps, delta, seed, cfg, &hm, out);
}

extern "C" gpm_status gpm_estimate(gpm_graph *h, const gpm_pattern *pattern, gpm_scheme scheme, double eps,
                                   double delta, uint64_t seed, const gpm_config *cfg, gpm_result *out) {
    if (!h || !out) {
        set_error("gpm_estimate: null argument");
        return GPM_ERR_ARG;
    }
    std::memset(out, 0, sizeof(*out));
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    switch (scheme) {
        case GPM_NS:
            return ns_estimate(h, p, eps, delta, seed, cfg, out);
        case GPM_GS:
            if (!(delta > 0.0 && delta < 1.0)) {
                set_error("delta must be in (0, 1)");
                return GPM_ERR_ARG;
            }
            return gs_estimate(h, p, seed, delta, cfg, out);
        case GPM_NS_LEARNED:
            return learned_estimate(h, p, eps, delta, seed, cfg, out);
        case GPM_HYBRID:
            if (!(eps > 0.0) || !(delta > 0.0 && delta < 1.0)) {
                set_error("eps must be > 0 and delta in (0, 1)");
                return GPM_ERR_ARG;
            }
            return hybrid_estimate(h, p, eps, delta, seed, cfg, out);
        case GPM_EXACT: {
            const auto t0 = std::chrono::steady_clock::now();
            uint64_t c = 0;
            float ms = 0.f;
            st = exact_count_plan(h, p, &c, &ms, cfg ? cfg->max_seconds : 0.0);
            if (st != GPM_OK && st != GPM_ERR_NOT_CONVERGED) return st;
            out->estimate = (double)c;
            out->exact_count = c;
            out->ci_half_width = 0.0;
            out->eps_hat = 0.0;
            out->converged = st == GPM_OK ? 1 : 0;
            out->scheme_used = GPM_EXACT;
            out->t_sample_s = ms * 1e-3;
            out->kernel_launches = 1;
            out->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            return st;
        }
        default:
            set_error("gpm_estimate: scheme not available in this build");
            return GPM_ERR_UNSUPPORTED;
    }
}

// ------------------------------------------------------------------ static-scratch variant
// gpm_sample_sums_static: the same sampler and chunk-order reduction as
// gpm_sample_sums, with every scratch word (per-chunk partials, the chunk
// counter, the totals) in one file-scope device array instead of memory the
// handle allocates, so the call itself allocates no device or pinned memory.
// The chunk size stays the fixed 64 samples of every other path, so the
// array's 65,536 partials bound a call to 2^22 samples and the totals equal
// gpm_sample_sums's bit for bit.
namespace gpm {

constexpr uint32_t kStaticMaxChunks = 1u << 16;                          // partials per call
constexpr uint64_t kStaticMaxSamples = (uint64_t)kStaticMaxChunks * kChunk;   // 2^22 samples per call
constexpr size_t kStaticPartialBytes = sizeof(Partial) * kStaticMaxChunks;
constexpr size_t kStaticScratchBytes = kStaticPartialBytes + 256 + 256;   // partials | totals | counter

// About 2 MiB; every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void *g_static_addr[256];

// Device address of g_static_scratch for the current device, looked up once
// per device (the array's name in host code is only a host-side stand-in).
static gpm_status static_scratch_addr(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        set_error("gpm_sample_sums_static: no current CUDA device");
        return GPM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("gpm_sample_sums_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return GPM_ERR_CUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_static_addr[dev]);
    return GPM_OK;
}

}  // namespace gpm

extern "C" gpm_status gpm_sample_sums_static(gpm_graph *h, const gpm_pattern *pattern, uint64_t seed,
                                             uint64_t first, uint64_t count, const gpm_config *cfg,
                                             gpm_sums *out) {
    if (!h || !out) {
        set_error("gpm_sample_sums_static: null argument");
        return GPM_ERR_ARG;
    }
    if (count > kStaticMaxSamples) {
        set_error("gpm_sample_sums_static: count exceeds the static scratch limit of 2^22 samples per call");
        return GPM_ERR_ARG;
    }
    Plan p;
    gpm_status st = plan_or_error(pattern, &p);
    if (st != GPM_OK) return st;
    std::memset(out, 0, sizeof(*out));
    if (count == 0) return GPM_OK;
    unsigned char *base = nullptr;
    st = static_scratch_addr(&base);
    if (st != GPM_OK) return st;
    Partial *parts = reinterpret_cast<Partial *>(base);
    Totals *tot = reinterpret_cast<Totals *>(base + kStaticPartialBytes);
    unsigned int *ctr = reinterpret_cast<unsigned int *>(base + kStaticPartialBytes + 256);

    Shape sh = pick_shape(h, cfg, count);
    const int mode = mode_of(cfg);
    if (sh.cap == 0) sh.cap = default_cap(h, 0, sh.warps, mode, p.induced);
    if (mode == MODE_LEARNED && sh.cap < kLearnedMax) sh.cap = kLearnedMax;
    const uint64_t nchunks = (count + sh.chunk - 1) / sh.chunk;   // <= kStaticMaxChunks
    RunArgs a;
    a.seed = seed;
    a.first = first;
    a.count = count;
    a.partials = parts;
    a.counter = ctr;
    a.trace = nullptr;
    a.slot = cfg ? cfg->slot : 0;
    a.cap = sh.cap;
    a.chunk = sh.chunk;
    a.nchunks = (uint32_t)nchunks;
    a.stride = 1;
    std::memset(&a.mlp, 0, sizeof(a.mlp));
    if (mode == MODE_LEARNED) a.mlp = *cfg->mlp;
    a.mlp_tc = (mode == MODE_LEARNED && cfg->mlp_tensor) ? 1u : 0u;
    cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess)
        e = launch_mode<false>(h, p, sh, a, kernel_mode(mode, plan_single_steps(p)));
    if (e == cudaSuccess) {
        reduce_partials<<<1, 1024, 0, h->stream>>>(parts, (uint32_t)nchunks, tot, 0);
        e = cudaGetLastError();
    }
    Totals t;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&t, tot, sizeof(Totals), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        set_error(std::string("gpm_sample_sums_static: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    out->n = t.n;
    out->hits = t.hits;
    out->sum = t.sum;
    out->sumsq = t.sumsq;
    return GPM_OK;
}
