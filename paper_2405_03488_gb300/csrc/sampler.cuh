// Per-sample device code of the NS sampler, shared by the single-run and the
// batched kernels.  See ns.cu for the method and the layout.
#pragma once

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"

namespace gpm {

enum { MODE_INTERSECT = 0, MODE_CHECK = 1, MODE_LEARNED = 2, MODE_INTERSECT_SINGLE = 3, MODE_LAZY = 4 };
// MODE_LAZY is NS-base (Sec. 2.2.1, Algorithm 1; the lazy verify Sec. 4.2
// contrasts with eager verify): x is drawn from the union U_j of the
// back-neighbours' lists and every constraint waits for the closure check
// after the last draw.
// MODE_INTERSECT_SINGLE is MODE_INTERSECT compiled with the position form of
// single-list steps (below); plans without such steps run the plain variant,
// whose code stays as small as before.

// resident 256-thread blocks per SM the plain sampler kernels are compiled for
#ifndef GPM_MIN_BLOCKS
#define GPM_MIN_BLOCKS 4
#endif

constexpr uint32_t kLearnedMax = 256;   // larger candidate sets are drawn uniformly
// S_j = S_{j-1} cut by N(v_{j-1}): stream the list through on-chip searches
// while |list| <= FACTOR * |usable part of S_{j-1}| + BIAS, else search the
// list for each element of S_{j-1}
#ifndef GPM_REUSE_STREAM_FACTOR
#define GPM_REUSE_STREAM_FACTOR 4
#endif
#ifndef GPM_REUSE_STREAM_BIAS
#define GPM_REUSE_STREAM_BIAS 0
#endif
// a partner list longer than the on-chip buffer is staged window by window
// instead of being searched in global memory
#ifndef GPM_PARTNER_WINDOWS
#define GPM_PARTNER_WINDOWS 1
#endif
// ... while the partner is at most this many times longer than the driver
// (a much longer partner is cheaper to search per driver entry; 8, 16, 32 and
// unbounded measured 1.55, 1.66, 1.72 and 1.65 times the global search on the
// R-MAT 27 5-clique / 4-cycle batch)
#ifndef GPM_WINDOW_RATIO
#define GPM_WINDOW_RATIO 32
#endif
// staging copies: cp.async, all of a list's copies in flight at once and no
// register round trip (1), or four loads per lane then stores (0)
// vertex-induced steps with one back-neighbour: counted and drawn from the
// positions of the removed entries when the non-neighbour lists are short
#ifndef GPM_INDUCED_POSITIONS
#define GPM_INDUCED_POSITIONS 1
#endif
// ... used when the back-neighbour's list (above the bound) is this many times
// longer than the non-neighbours' lists together
#ifndef GPM_INDUCED_RATIO
#define GPM_INDUCED_RATIO 2
#endif
#ifndef GPM_STAGE_ASYNC
#define GPM_STAGE_ASYNC 1
#endif

constexpr int kMlpFloats = 4481;        // 3->64->64->1 weights and biases
constexpr int kW2Stride = 72;           // BF16 W2 rows and hidden tiles, padded against bank conflicts
// the FP32 weights (padded to 8 bytes), then W2 as raw BF16, 64 rows of kW2Stride
constexpr int kMlpSmemFloats = 4482 + 64 * kW2Stride / 2;
// the BF16 hidden tile of 16 candidates (tensor-core scoring), scores, and
// each candidate's CSR offsets (u64 row start, u32 degree, u32 offset of its
// first neighbour above itself)
constexpr int kHTileWords = 16 * kW2Stride / 2;
constexpr int kLearnedWarpWords = kHTileWords + kLearnedMax + 4 * kLearnedMax;

struct RunArgs {
    uint64_t seed;
    uint64_t first;               // first sample index of this launch
    uint64_t count;               // samples in this launch
    Partial *partials;            // one per chunk
    unsigned int *counter;        // chunk dispenser
    gpm_sample_record *trace;     // optional per-sample records (device)
    uint32_t slot;
    uint32_t cap;                 // entries per on-chip candidate buffer
    uint32_t chunk;               // samples per chunk
    uint32_t nchunks;
    uint32_t stride;              // chunks of the range between consecutive chunks of this launch
    gpm_mlp mlp;                  // learned proposal weights (device, BF16)
    uint32_t mlp_tc;              // learned: score on the tensor cores (mma.sync BF16)
};

// The fields of a Plan the sampler reads, for an on-chip copy per warp.
struct StepPlan {
    int32_t k, induced, oriented, pad;
    uint32_t back[kMaxK], lower[kMaxK], reuse[kMaxK], last_back[kMaxK];
};

// Copies plan fields into a warp's StepPlan (all lanes call it).
__device__ __forceinline__ void load_step_plan(const Plan &src, StepPlan *dst) {
    const unsigned lane = threadIdx.x & 31u;
    if (lane == 0) {
        dst->k = src.k;
        dst->induced = src.induced;
        dst->oriented = src.oriented;
        dst->pad = 0;
    }
    if (lane < (unsigned)kMaxK) {
        dst->back[lane] = src.back[lane];
        dst->lower[lane] = src.lower[lane];
        dst->reuse[lane] = src.reuse[lane];
        dst->last_back[lane] = src.last_back[lane];
    }
    __syncwarp();
}

// 12 u64 factors + 16 u32 vertices + 12 u32 scores, then the step-2 test table:
// 9 u64 list starts, 9 u32 lengths (top bit: the list must not hold y), 9 u32
// vertices y must differ from
constexpr int kWarpHeaderWords = 88;
constexpr int kTestSlots = 9;   // positions before the last of a 10-vertex pattern

// Words per warp slice, rounded up to an even count so that every warp's
// 8-byte fields (factors, test-table pointers, learned row starts) stay
// 8-byte aligned for any buffer sizes.
__host__ __device__ inline uint32_t warp_words(uint32_t cap, bool learned) {
    return (kWarpHeaderWords + 2 * cap + (learned ? kLearnedWarpWords : 0) + 1u) & ~1u;
}

struct WarpMem {
    uint64_t *fac;
    uint32_t *v;
    uint32_t *aux;
    uint64_t *tptr;        // step-2 test table (see kWarpHeaderWords)
    uint32_t *tlen, *tneq;
    uint32_t *S0, *S1;
    uint16_t *htile;       // learned, tensor cores: BF16 layer-1 outputs of 16 candidates
    uint32_t *score;       // learned: a_x of each candidate
    const float *W;        // learned: block copy of the weights (FP32, gpm_mlp order)
    const uint16_t *W2b;   // learned: W2 as raw BF16, rows of kW2Stride
};

// Block-level setup: the learned weights (BF16 -> FP32, in the gpm_mlp order;
// every lane reads the same weight at once, a broadcast) and each warp's slices.
template <int MODE>
__device__ __forceinline__ WarpMem warp_mem(uint64_t *smem64, uint32_t cap, const gpm_mlp &mlp) {
    uint32_t *smem = reinterpret_cast<uint32_t *>(smem64);
    float *W = reinterpret_cast<float *>(smem);
    if (MODE == MODE_LEARNED) {
        auto bf = [](const uint16_t *p, int i) { return __uint_as_float((uint32_t)p[i] << 16); };
        for (int i = threadIdx.x; i < kMlpFloats; i += blockDim.x) {
            if (i < 192) W[i] = bf(mlp.w1, i);
            else if (i < 256) W[i] = bf(mlp.b1, i - 192);
            else if (i < 4352) W[i] = bf(mlp.w2, i - 256);
            else if (i < 4416) W[i] = bf(mlp.b2, i - 4352);
            else if (i < 4480) W[i] = bf(mlp.w3, i - 4416);
            else W[i] = bf(mlp.b3, 0);
        }
        uint16_t *W2b = reinterpret_cast<uint16_t *>(W + 4482);
        for (int i = threadIdx.x; i < 64 * kW2Stride; i += blockDim.x) {
            const int o = i / kW2Stride, in = i % kW2Stride;
            W2b[i] = in < 64 ? mlp.w2[o * 64 + in] : (uint16_t)0;
        }
        __syncthreads();
        smem += kMlpSmemFloats;
    }
    const unsigned warp = threadIdx.x >> 5;
    const uint32_t per = warp_words(cap, MODE == MODE_LEARNED);
    uint32_t *base = smem + warp * per;
    WarpMem wm;
    wm.fac = reinterpret_cast<uint64_t *>(base);
    wm.v = base + 24;
    wm.aux = base + 40;
    wm.tptr = reinterpret_cast<uint64_t *>(base + 52);
    wm.tlen = base + 70;
    wm.tneq = base + 79;
    wm.S0 = base + kWarpHeaderWords;
    wm.S1 = wm.S0 + cap;
    wm.htile = reinterpret_cast<uint16_t *>(wm.S1 + cap);
    wm.score = wm.S1 + cap + kHTileWords;
    wm.W = W;
    wm.W2b = reinterpret_cast<const uint16_t *>(W + 4482);
    return wm;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        uint64_t t = __shfl_xor_sync(kFull, x, o);
        x = t < x ? t : x;
    }
    return x;
}

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Copies src[0, n) (global) to dst[0, n) (the warp's shared-memory buffer);
// all lanes call it, and the caller's __syncwarp publishes the copy.
__device__ __forceinline__ void stage_list(const uint32_t *__restrict__ src, uint32_t n, uint32_t *dst) {
    const unsigned lane = lane_id();
#if GPM_STAGE_ASYNC
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(dst);
    for (uint32_t idx = lane; idx < n; idx += 32)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d0 + 4u * idx), "l"(src + idx) : "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
#else
    for (uint32_t base = 0; base < n; base += 128) {
        uint32_t y[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t idx = base + 32 * u + lane;
            y[u] = idx < n ? __ldg(src + idx) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t idx = base + 32 * u + lane;
            if (idx < n) dst[idx] = y[u];
        }
    }
#endif
}

}  // namespace gpm

// The learned proposal's device code (features, MLP score, lookahead, draw).
#include "learned.cuh"

namespace gpm {

// Result of one sample, uniform across the warp.
struct SampleOut {
    double w;
    uint64_t wu;
    int depth;
    bool hit, overflow;
};

// COMPACT: evaluate the step-2 predicate from one inlined copy (the element
// picked by selects) instead of four unrolled copies.  Fewer instruction-fetch
// stalls make it faster in the batched kernel for edge-induced plans; the
// unrolled copies overlap the global searches of vertex-induced plans and
// suit the single-run kernel.
template <int MODE, typename PlanT, bool COMPACT = false>
__device__ SampleOut sample_one(const DGraph &g, const PlanT &p, const RunArgs &a, uint64_t s, WarpMem &wm) {
    constexpr bool kCompact = COMPACT;
    const unsigned lane = lane_id();
    const int k = p.k;
    SampleOut out;
    out.w = 0.0;
    out.wu = 0;
    out.depth = 0;
    out.hit = false;
    out.overflow = false;

    const int nb = k / 2;  // Philox blocks for the k-1 choices
    Philox4 o = {0u, 0u, 0u, 0u};
    if ((int)lane < nb)
        o = philox10((uint32_t)s, (uint32_t)(s >> 32), lane, a.slot << 8, (uint32_t)a.seed,
                     (uint32_t)(a.seed >> 32));
    auto word = [&](int t) -> uint64_t {
        uint32_t lo = (t & 1) ? o.z : o.x;
        uint32_t hi = (t & 1) ? o.w : o.y;
        lo = __shfl_sync(kFull, lo, t >> 1);
        hi = __shfl_sync(kFull, hi, t >> 1);
        return ((uint64_t)hi << 32) | lo;
    };

    // NS-base draws from all 2m directed entries: its restrictions wait for the closure
    const bool orient = (MODE != MODE_LAZY) && p.oriented;
    const uint64_t M = orient ? g.m : g.nnz;
    if (lane == 0) wm.fac[0] = M;
    if (M == 0) return out;
    const uint64_t e = index_map(word(0), M);
    uint32_t v0, v1;
    uint64_t pos01a = ~0ull;  // index of v1 inside N(v0) in col, when known
    if (orient && g.edges) {
        const uint64_t pr = __ldg(g.edges + e);
        v0 = (uint32_t)pr;
        v1 = (uint32_t)(pr >> 32);
    } else if (orient) {
        const uint64_t u = warp_upper_bound(g.uoff, g.n + 1, e) - 1;
        v0 = (uint32_t)u;
        pos01a = __ldg(g.up + u) + (e - __ldg(g.uoff + u));
        v1 = __ldg(g.col + pos01a);
    } else {
        const uint64_t u = warp_upper_bound(g.row_ptr, g.n + 1, e) - 1;
        v0 = (uint32_t)u;
        pos01a = e;
        v1 = __ldg(g.col + e);
    }
    // lane i: row start rb of v_i in col, its degree rn, and ru, the offset of
    // its first neighbour above v_i (degrees are below 2^31, so offsets inside a
    // list are 32-bit)
    uint64_t rb = 0;
    uint32_t rn = 0, ru = 0;
    if (lane == 0) {
        rb = __ldg(g.row_ptr + v0);
        rn = (uint32_t)(__ldg(g.row_ptr + v0 + 1) - rb);
        ru = (uint32_t)(__ldg(g.up + v0) - rb);
        wm.v[0] = v0;
        wm.v[1] = v1;
    } else if (lane == 1) {
        rb = __ldg(g.row_ptr + v1);
        rn = (uint32_t)(__ldg(g.row_ptr + v1 + 1) - rb);
        ru = (uint32_t)(__ldg(g.up + v1) - rb);
    }
    // offset of v1 inside N(v0), when known
    uint32_t pos01 = 0xFFFFFFFFu;
    if (pos01a != ~0ull) pos01 = (uint32_t)(pos01a - __shfl_sync(kFull, rb, 0));
    __syncwarp();
    // list of position i, as a pointer to its first entry and its length
    auto row = [&](int i) -> const uint32_t * { return g.col + __shfl_sync(kFull, rb, i); };
    auto deg = [&](int i) -> uint32_t { return __shfl_sync(kFull, rn, i); };
    out.depth = 2;
    double w = (double)M;
    uint64_t wu = M;
    bool ovf = false;
    uint32_t prev_size = 0;
    uint32_t prev_off = 0;   // 1 + index of v_{j-1} in the on-chip S_{j-1} (0: unknown)
    bool prev_mat = false;

    for (int j = 2; j < k; j++) {
        const uint32_t lm = p.lower[j];
        const bool has_lo = lm != 0;
        uint32_t lo = 0;
        for (int i = 0; i < j; i++)
            if ((lm >> i) & 1u) lo = wm.v[i] > lo ? wm.v[i] : lo;
        const uint64_t r = word(j - 1);
        // offset of the first entry of position i's list L (n entries) above
        // the lower bound; the split at ru and the known slot of v1 in N(v0)
        // shorten or skip the search
        auto above = [&](int i, const uint32_t *L, uint32_t n) -> uint32_t {
            const uint32_t ui = __shfl_sync(kFull, ru, i);
            if (!has_lo) return 0u;
            const uint32_t vi = wm.v[i];
            if (lo == vi) return ui;
            if (i == 0 && lo == wm.v[1] && pos01 != 0xFFFFFFFFu) return pos01 + 1u;
            if (lo > vi) return ui + warp_upper_bound32(L + ui, n - ui, lo);
            return warp_upper_bound32(L, ui, lo);
        };
        uint64_t size = 0;
        uint32_t x = 0;
        uint32_t pick = 0;   // 1 + index of x in the on-chip S_j (0: not drawn from it)
        bool learned_step = false;
        double lfac = 1.0;
        if (MODE == MODE_LAZY) {
            // U_j in list order: the first back-neighbour's list whole, then
            // each later back-neighbour's entries that no earlier one holds
            const uint32_t back = p.back[j];
            auto fresh = [&](uint32_t y, int i) -> bool {
                bool ok = true;
                for (int q = 0; q < i; q++) {
                    if (!((back >> q) & 1u)) continue;
                    const uint32_t *Lq = row(q);
                    const uint32_t nq = deg(q);
                    ok = ok && !lane_contains32(Lq, nq, y);
                }
                return ok;
            };
            uint32_t my_kept = 0;   // lane i: entries back-neighbour i adds to U_j
            for (int i = 0; i < j; i++) {
                if (!((back >> i) & 1u)) continue;
                const uint32_t *L = row(i);
                const uint32_t n = deg(i);
                uint32_t c = 0;
                if ((back & ((1u << i) - 1u)) == 0) {
                    c = n;
                } else {
                    for (uint32_t base = 0; base < n; base += 32) {
                        const uint32_t idx = base + lane;
                        const bool valid = idx < n;
                        const uint32_t y = valid ? __ldg(L + idx) : 0u;
                        const bool ok = fresh(y, i) && valid;
                        c += (uint32_t)__popc(__ballot_sync(kFull, ok));
                    }
                }
                if ((int)lane == i) my_kept = c;
                size += c;
            }
            if (lane == 0) wm.fac[j] = size;
            if (size == 0) {
                out.depth = j;
                return out;
            }
            uint64_t t = index_map(r, size);
            for (int i = 0; i < j; i++) {
                if (!((back >> i) & 1u)) continue;
                const uint64_t c = __shfl_sync(kFull, my_kept, i);
                if (t >= c) {
                    t -= c;
                    continue;
                }
                const uint32_t *L = row(i);
                const uint32_t n = deg(i);
                if ((back & ((1u << i) - 1u)) == 0) {
                    x = __ldg(L + t);
                } else {
                    uint64_t seen = 0;
                    for (uint32_t base = 0; base < n; base += 32) {
                        const uint32_t idx = base + lane;
                        const bool valid = idx < n;
                        const uint32_t y = valid ? __ldg(L + idx) : 0u;
                        const bool ok = fresh(y, i) && valid;
                        const unsigned m = __ballot_sync(kFull, ok);
                        const uint64_t cm = __popc(m);
                        if (seen + cm > t) {
                            const uint32_t rank = (uint32_t)(t - seen);
                            const bool mine = ok && (uint32_t)__popc(m & lanemask_lt()) == rank;
                            x = __shfl_sync(kFull, y, __ffs(__ballot_sync(kFull, mine)) - 1);
                            break;
                        }
                        seen += cm;
                    }
                }
                break;
            }
        } else if (MODE == MODE_CHECK) {
            const int pb = (int)p.last_back[j];
            const uint32_t *L = row(pb);
            const uint32_t n = deg(pb);
            const uint32_t start = above(pb, L, n);
            size = n - start;
            if (lane == 0) wm.fac[j] = size;
            if (size == 0) {
                out.depth = j;
                return out;
            }
            x = __ldg(L + start + (uint32_t)index_map(r, size));
            bool okl = true;
            if ((int)lane < j) {
                okl = (x != wm.v[lane]);
                const bool edge = (p.back[j] >> lane) & 1u;
                if (edge) {
                    if ((int)lane != pb) okl = okl && lane_contains32(g.col + rb, rn, x);
                } else if (p.induced) {
                    okl = okl && !lane_contains32(g.col + rb, rn, x);
                }
            }
            if (!__all_sync(kFull, okl)) {
                out.depth = j;
                return out;
            }
        } else {
            uint32_t *Sc = (j & 1) ? wm.S1 : wm.S0;
            uint32_t *Sp = (j & 1) ? wm.S0 : wm.S1;
            uint32_t count = 0;
            bool mat = true;
            const uint32_t back = p.back[j];
            bool done = false;
            // (batches with vertex-induced plans run the unrolled variant)
            if constexpr (MODE == MODE_INTERSECT_SINGLE && !kCompact) {
                if (GPM_INDUCED_POSITIONS && p.induced && (back & (back - 1)) == 0 &&
                    !(p.reuse[j] >= 1 && prev_mat)) {
                    // one back-neighbour v_d, vertex-induced: S_j is A = N(v_d) above
                    // the bound without the entries that lie in a non-neighbour's
                    // list or are matched vertices.  When the non-neighbours' lists
                    // are short against A, each is walked once and the positions in A
                    // of its entries (one ascending run per list, an entry counted in
                    // the first list that holds it) give |S_j| and the drawn entry, as
                    // in the edge-induced position form; A itself is never streamed.
                    const int d = __ffs(back) - 1;
                    const uint32_t *DL = row(d);
                    const uint32_t dn = deg(d);
                    const bool nnl = (int)lane < j && (int)lane != d;
                    const uint32_t sumdeg = __reduce_add_sync(kFull, nnl ? (rn < (1u << 26) ? rn : (1u << 26)) : 0u);
                    const uint32_t ds = above(d, DL, dn);
                    const uint32_t *S = DL + ds;
                    const uint32_t L = dn - ds;
                    if (L >= 64 && (uint64_t)sumdeg * GPM_INDUCED_RATIO < (uint64_t)L) {
                        const uint32_t amax = __ldg(S + L - 1);
                        uint32_t nr = 0, run0 = 0, runn = 0;   // lane i: its run in Sc
                        bool over = false;
                        for (int i = 0; i < j && !over; i++) {
                            if (i == d) continue;
                            const uint32_t *B = row(i);
                            const uint32_t bn = deg(i);
                            const uint32_t bs = above(i, B, bn);
                            const uint32_t start = nr;
                            for (uint32_t base = bs; base < bn; base += 32) {
                                const uint32_t idx = base + lane;
                                const uint32_t y = idx < bn ? __ldg(B + idx) : 0xFFFFFFFFu;
                                const bool in = idx < bn && y <= amax;
                                uint32_t q = in ? lane_find32(S, L, y) : 0xFFFFFFFFu;
                                for (int m = 0; m < j; m++) q = (y == wm.v[m]) ? 0xFFFFFFFFu : q;
                                for (int i2 = 0; i2 < i; i2++) {
                                    if (i2 == d) continue;
                                    const uint32_t *B2 = row(i2);
                                    const uint32_t n2 = deg(i2);
                                    if (q != 0xFFFFFFFFu && lane_contains32(B2, n2, y)) q = 0xFFFFFFFFu;
                                }
                                const unsigned km = __ballot_sync(kFull, q != 0xFFFFFFFFu);
                                const uint32_t pos = nr + __popc(km & lanemask_lt());
                                if (q != 0xFFFFFFFFu && pos < a.cap) Sc[pos] = q;
                                nr += __popc(km);
                                if (nr > a.cap) {
                                    over = true;
                                    break;
                                }
                                // entries past A's last one cannot lie in A
                                if (__ballot_sync(kFull, idx < bn && y > amax)) break;
                            }
                            if ((int)lane == i) {
                                run0 = start;
                                runn = nr - start;
                            }
                        }
                        if (!over) {
                            // matched vertices above the bound that lie in A (lane m);
                            // the runs above leave them out
                            uint32_t qm = 0xFFFFFFFFu;
                            if (nnl && !(has_lo && wm.v[lane] <= lo)) qm = lane_find32(S, L, wm.v[lane]);
                            __syncwarp();
                            count = L - nr - (uint32_t)__popc(__ballot_sync(kFull, qm != 0xFFFFFFFFu));
                            if (count) {
                                // smallest position with t kept entries before it
                                const uint32_t t = (uint32_t)index_map(r, count);
                                uint32_t idx = t;
                                for (;;) {
                                    // removed positions <= idx: lane i counts its run
                                    uint32_t c = 0;
                                    if (nnl && runn) {
                                        uint32_t lo2 = 0, hi2 = runn;
                                        while (lo2 < hi2) {
                                            const uint32_t mid = (lo2 + hi2) >> 1;
                                            if (Sc[run0 + mid] <= idx) lo2 = mid + 1;
                                            else hi2 = mid;
                                        }
                                        c = lo2;
                                    }
                                    c += (qm <= idx) ? 1u : 0u;
                                    const uint32_t nx = t + __reduce_add_sync(kFull, c);
                                    if (nx == idx) break;
                                    idx = nx;
                                }
                                x = __ldg(S + idx);
                            }
                            mat = false;
                            done = true;
                        }
                    }
                }
            }
            if (done) {
            } else if ((MODE == MODE_INTERSECT_SINGLE || (MODE == MODE_LEARNED && j == k - 1)) && !p.induced &&
                (back & (back - 1)) == 0) {
                // one back-neighbour v_d, edge-induced: S_j is N(v_d) above the
                // bound without the matched vertices it holds, so |S_j| and its
                // t-th element follow from their positions in the list alone
                const int d = __ffs(back) - 1;
                const uint32_t *DL = row(d);
                const uint32_t dn = deg(d);
                const uint32_t ds = above(d, DL, dn);
                const uint32_t *S = DL + ds;
                const uint32_t L = dn - ds;
                // a matched vertex at or below the bound cannot lie in the list's
                // part above it: only the others are searched
                const uint32_t q = ((int)lane < j && (int)lane != d && !(has_lo && wm.v[lane] <= lo))
                                       ? lane_find32(S, L, wm.v[lane])
                                       : 0xFFFFFFFFu;
                count = L - (uint32_t)__popc(__ballot_sync(kFull, q != 0xFFFFFFFFu));
                if (count) {
                    // smallest list index with t kept entries before it
                    const uint32_t t = (uint32_t)index_map(r, count);
                    uint32_t idx = t;
                    for (;;) {
                        const uint32_t nx = t + (uint32_t)__popc(__ballot_sync(kFull, q <= idx));
                        if (nx == idx) break;
                        idx = nx;
                    }
                    x = __ldg(S + idx);
                }
                mat = false;
            } else if (p.reuse[j] == 1 && prev_mat) {
                // S_j = S_{j-1} (on chip) cut by N(v_{j-1}) above the bound;
                // when the bound is at least v_{j-1}, only the part of S_{j-1}
                // after v_{j-1} can qualify
                const uint32_t *NL = row(j - 1);
                const uint32_t nn = deg(j - 1);
                const uint32_t start = above(j - 1, NL, nn);
                const uint32_t *A = NL + start;
                const uint32_t L = nn - start;
                const uint32_t off = (has_lo && lo >= wm.v[j - 1]) ? prev_off : 0u;
                const uint32_t P = prev_size;
                if (L <= (uint32_t)GPM_REUSE_STREAM_FACTOR * (P - off) + GPM_REUSE_STREAM_BIAS) {
                    for (uint32_t base = 0; base < L; base += 128) {
                        uint32_t y[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const uint32_t idx = base + 32 * u + lane;
                            y[u] = idx < L ? __ldg(A + idx) : 0u;
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const bool ok = (base + 32 * u + lane < L) && lane_contains_shared(Sp + off, P - off, y[u]);
                            const unsigned m = __ballot_sync(kFull, ok);
                            if (ok) Sc[count + __popc(m & lanemask_lt())] = y[u];
                            count += __popc(m);
                        }
                    }
                } else {
                    for (uint32_t base = off; base < P; base += 32) {
                        const uint32_t idx = base + lane;
                        const bool valid = idx < P;
                        const uint32_t y = valid ? Sp[idx] : 0u;
                        const bool ok = valid && (!has_lo || y > lo) && lane_contains32(A, L, y);
                        const unsigned m = __ballot_sync(kFull, ok);
                        if (ok) Sc[count + __popc(m & lanemask_lt())] = y;
                        count += __popc(m);
                    }
                }
            } else if (p.reuse[j] >= 2 && prev_mat) {
                // S_j = S_{j-1} (on chip) above the bound, without v_{j-1}, and
                // (vertex-induced) without N(v_{j-1})
                const uint32_t *NL = row(j - 1);
                const uint32_t nn = deg(j - 1);
                const uint32_t vj1 = wm.v[j - 1];
                const bool drop = p.reuse[j] == 2;
                const uint32_t P = prev_size;
                const uint32_t off = (has_lo && lo >= vj1) ? prev_off : 0u;
                for (uint32_t base = off; base < P; base += 32) {
                    const uint32_t idx = base + lane;
                    const bool valid = idx < P;
                    const uint32_t y = valid ? Sp[idx] : 0u;
                    bool ok = valid && (!has_lo || y > lo) && y != vj1;
                    if (drop) ok = ok && !lane_contains32(NL, nn, y);
                    const unsigned m = __ballot_sync(kFull, ok);
                    if (ok) Sc[count + __popc(m & lanemask_lt())] = y;
                    count += __popc(m);
                }
            } else {
                // driver: shortest back-neighbour list, streamed; partner: the
                // next shortest, staged on chip when its part above the bound fits
                const bool isback = (int)lane < j && ((back >> lane) & 1u);
                // shortest list first, lowest position on ties
                const uint32_t mylen = isback ? rn : 0xFFFFFFFFu;
                const uint32_t m1 = __reduce_min_sync(kFull, mylen);
                const int driver = __ffs(__ballot_sync(kFull, isback && rn == m1)) - 1;
                const bool other = isback && (int)lane != driver;
                const uint32_t m2 = __reduce_min_sync(kFull, other ? rn : 0xFFFFFFFFu);
                const unsigned pm = __ballot_sync(kFull, other && rn == m2);
                const int partner = pm ? __ffs(pm) - 1 : -1;
                const uint32_t *DL = row(driver);
                const uint32_t dn = deg(driver);
                const uint32_t dstart = above(driver, DL, dn);
                const uint32_t *D = DL + dstart;
                const uint32_t dlen = dn - dstart;
                bool empty = dlen == 0;
                int staged = -1;
                uint32_t plen = 0;
                // the partner's part above the bound; longer than the buffer, it is
                // staged window by window (each window settles the driver entries
                // up to its last element)
                const uint32_t *Q = nullptr;
                uint32_t qn = 0;
                bool windowed = false;
                if (partner >= 0 && !empty) {
                    const uint32_t *PL = row(partner);
                    const uint32_t pn = deg(partner);
                    const uint32_t ps = above(partner, PL, pn);
                    Q = PL + ps;
                    qn = pn - ps;
                    if (ps >= pn) {
                        empty = true;
                    } else if (qn <= a.cap) {
                        stage_list(Q, qn, Sp);
                        staged = partner;
                        plen = qn;
                        __syncwarp();
                    } else if (GPM_PARTNER_WINDOWS &&
                               (uint64_t)qn <= (uint64_t)GPM_WINDOW_RATIO * dlen) {
                        staged = partner;
                        windowed = true;
                    }
                }
                int ntest = 0, nneq = 0;
                // every condition of S_j but membership in the driver list,
                // gathered once per step into the warp's test table: lane i
                // enters its own list when y must (edge, not the driver or the
                // staged partner) or must not (vertex-induced non-edge) lie in
                // it, and its vertex when y could equal it (a non-edge not
                // below the bound y already exceeds; membership in N(v_i)
                // rules out y = v_i, the graph having no loops)
                if constexpr (kCompact) {
                    const bool edge = (int)lane < j && ((back >> lane) & 1u);
                    const bool nonedge = (int)lane < j && !edge;
                    const bool test = (edge && (int)lane != driver && (int)lane != staged) || (nonedge && p.induced);
                    const bool neq = nonedge && !(has_lo && wm.v[lane] <= lo);
                    const unsigned tm = __ballot_sync(kFull, test), nm = __ballot_sync(kFull, neq);
                    if (test) {
                        const int t = __popc(tm & lanemask_lt());
                        wm.tptr[t] = rb;
                        wm.tlen[t] = rn | (nonedge ? 0x80000000u : 0u);
                    }
                    if (neq) wm.tneq[__popc(nm & lanemask_lt())] = wm.v[lane];
                    ntest = __popc(tm);
                    nneq = __popc(nm);
                    __syncwarp();
                }
                // the unrolled variant (vertex-induced batches and single runs)
                // keeps the per-position form: its four inlined copies overlap the
                // global non-edge searches, which the table form measured slower on
                bool gpart = false;   // search the windowed partner in global memory
                // every lane of the warp calls pred (the per-position form
                // shuffles), so it comes first in any short-circuit condition
                auto pred = [&](uint32_t y) -> bool {
                    bool ok = true;
                    if constexpr (kCompact) {
                        for (int t = 0; t < nneq; t++) ok = ok && y != wm.tneq[t];
                        if (staged >= 0)
                            ok = ok && (gpart ? lane_contains32(Q, qn, y) : lane_contains_shared(Sp, plen, y));
                        for (int t = 0; t < ntest; t++) {
                            const uint32_t ln = wm.tlen[t];
                            ok = ok && (lane_contains32(g.col + wm.tptr[t], ln & 0x7FFFFFFFu, y) != (ln >> 31));
                        }
                    } else {
                        for (int i = 0; i < j; i++) {
                            const uint32_t *Li = row(i);
                            const uint32_t ni = deg(i);
                            ok = ok && (y != wm.v[i]);
                            const bool edge = (back >> i) & 1u;
                            if (edge) {
                                if (i == driver) continue;
                                if (i == staged)
                                    ok = ok && (gpart ? lane_contains32(Q, qn, y) : lane_contains_shared(Sp, plen, y));
                                else ok = ok && lane_contains32(Li, ni, y);
                            } else if (p.induced) {
                                ok = ok && !lane_contains32(Li, ni, y);
                            }
                        }
                    }
                    return ok;
                };
                if (!empty) {
                    if constexpr (kCompact) {
                    // one copy of pred (the element picked by selects); the
                    // driver entries are settled window by window, a partner
                    // staged whole (or none) being a single last window
                    uint32_t pw = 0, dcur = 0;
                    for (;;) {
                        bool tail = true;
                        uint32_t wlast = 0u;
                        if (windowed) {
                            const uint32_t wn = (qn - pw < a.cap) ? qn - pw : a.cap;
                            __syncwarp();
                            stage_list(Q + pw, wn, Sp);
                            __syncwarp();
                            plen = wn;
                            pw += wn;
                            tail = pw >= qn;
                            wlast = Sp[wn - 1];
                        }
                        bool stop = false;
                        for (uint32_t base = dcur; base < dlen && !stop; base += 128) {
                            uint32_t y[4];
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                const uint32_t idx = base + 32 * u + lane;
                                y[u] = idx < dlen ? __ldg(D + idx) : 0u;
                            }
#pragma unroll 1
                            for (int u = 0; u < 4; u++) {
                                const uint32_t b = base + 32 * u;
                                if (b >= dlen) break;
                                const uint32_t yu = u == 0 ? y[0] : u == 1 ? y[1] : u == 2 ? y[2] : y[3];
                                const bool in = (b + lane < dlen) && (tail || yu <= wlast);
                                const bool ok = pred(yu) && in;
                                const unsigned m = __ballot_sync(kFull, ok);
                                if (ok) {
                                    const uint32_t pos = count + __popc(m & lanemask_lt());
                                    if (pos < a.cap) Sc[pos] = yu;
                                }
                                count += __popc(m);
                                if (!tail) {
                                    // the entries up to the window's last element form a prefix
                                    const unsigned im = __ballot_sync(kFull, in);
                                    if (im != kFull) {
                                        dcur = b + __popc(im);
                                        stop = true;
                                        break;
                                    }
                                }
                            }
                        }
                        if (tail || !stop) break;
                    }
                    gpart = windowed;
                    } else {
                    // four inlined copies of pred, same windows
                    uint32_t pw = 0, dcur = 0;
                    for (;;) {
                        bool tail = true;
                        uint32_t wlast = 0u;
                        if (windowed) {
                            const uint32_t wn = (qn - pw < a.cap) ? qn - pw : a.cap;
                            __syncwarp();
                            stage_list(Q + pw, wn, Sp);
                            __syncwarp();
                            plen = wn;
                            pw += wn;
                            tail = pw >= qn;
                            wlast = Sp[wn - 1];
                        }
                        bool stop = false;
                        for (uint32_t base = dcur; base < dlen && !stop; base += 128) {
                            uint32_t y[4];
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                const uint32_t idx = base + 32 * u + lane;
                                y[u] = idx < dlen ? __ldg(D + idx) : 0u;
                            }
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                const uint32_t b = base + 32 * u;
                                if (b >= dlen) break;
                                const bool in = (b + lane < dlen) && (tail || y[u] <= wlast);
                                const bool ok = pred(y[u]) && in;
                                const unsigned m = __ballot_sync(kFull, ok);
                                if (ok) {
                                    const uint32_t pos = count + __popc(m & lanemask_lt());
                                    if (pos < a.cap) Sc[pos] = y[u];
                                }
                                count += __popc(m);
                                if (!tail) {
                                    const unsigned im = __ballot_sync(kFull, in);
                                    if (im != kFull) {
                                        dcur = b + __popc(im);
                                        stop = true;
                                        break;
                                    }
                                }
                            }
                        }
                        if (tail || !stop) break;
                    }
                    gpart = windowed;
                    }
                }
                if (!empty) {
                    mat = count <= a.cap;
                    if (!mat) {
                        if constexpr (kCompact) {
                        // second pass: locate the drawn element without storing the set
                            const uint32_t target = (uint32_t)index_map(r, count);
                            uint32_t seen = 0;
                            bool found = false;
                            for (uint32_t base = 0; base < dlen && !found; base += 128) {
                                uint32_t y[4];
    #pragma unroll
                                for (int u = 0; u < 4; u++) {
                                    const uint32_t idx = base + 32 * u + lane;
                                    y[u] = idx < dlen ? __ldg(D + idx) : 0u;
                                }
    #pragma unroll 1
                                for (int u = 0; u < 4; u++) {
                                    if (found || base + 32 * u >= dlen) break;
                                    const uint32_t yu = u == 0 ? y[0] : u == 1 ? y[1] : u == 2 ? y[2] : y[3];
                                    const bool ok = pred(yu) && (base + 32 * u + lane < dlen);
                                    const unsigned m = __ballot_sync(kFull, ok);
                                    const uint32_t c = __popc(m);
                                    if (seen + c > target) {
                                        const uint32_t rank = (uint32_t)(target - seen);
                                        const bool mine = ok && (uint32_t)__popc(m & lanemask_lt()) == rank;
                                        const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
                                        x = __shfl_sync(kFull, yu, src);
                                        found = true;
                                    }
                                    seen += c;
                                }
                            }
                        } else {
                        // second pass: locate the drawn element without storing the set
                            const uint32_t target = (uint32_t)index_map(r, count);
                            uint32_t seen = 0;
                            bool found = false;
                            for (uint32_t base = 0; base < dlen && !found; base += 128) {
                                uint32_t y[4];
    #pragma unroll
                                for (int u = 0; u < 4; u++) {
                                    const uint32_t idx = base + 32 * u + lane;
                                    y[u] = idx < dlen ? __ldg(D + idx) : 0u;
                                }
    #pragma unroll
                                for (int u = 0; u < 4; u++) {
                                    if (found || base + 32 * u >= dlen) break;
                                    const uint32_t yu = y[u];
                                    const bool ok = pred(yu) && (base + 32 * u + lane < dlen);
                                    const unsigned m = __ballot_sync(kFull, ok);
                                    const uint32_t c = __popc(m);
                                    if (seen + c > target) {
                                        const uint32_t rank = (uint32_t)(target - seen);
                                        const bool mine = ok && (uint32_t)__popc(m & lanemask_lt()) == rank;
                                        const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
                                        x = __shfl_sync(kFull, yu, src);
                                        found = true;
                                    }
                                    seen += c;
                                }
                            }
                        }
                    }
                }
            }
            size = count;
            if (lane == 0) wm.fac[j] = size;
            if (size == 0) {
                out.depth = j;
                return out;
            }
            __syncwarp();
            if (MODE == MODE_LEARNED && j <= k - 2 && mat && size <= kLearnedMax) {
                uint64_t A = 0;
                uint32_t ax = 0;
                x = learned_pick(g, p, wm, Sc, (uint32_t)size, j, r, rb, rb + rn, a.mlp_tc != 0, &A, &ax);
                if (lane == 0) {
                    wm.fac[j] = A;
                    wm.aux[j] = ax;
                }
                lfac = __ddiv_rn((double)A, (double)ax);
                learned_step = true;
            } else if (mat) {
                const uint32_t t = (uint32_t)index_map(r, size);
                x = Sc[t];
                pick = t + 1;
            }
            prev_size = (uint32_t)(mat ? size : 0);
            prev_off = pick;
            prev_mat = mat;
        }
        if (lane == 0) wm.v[j] = x;
        if ((int)lane == j && j + 1 < k) {
            rb = __ldg(g.row_ptr + x);
            rn = (uint32_t)(__ldg(g.row_ptr + x + 1) - rb);
            ru = (uint32_t)(__ldg(g.up + x) - rb);
        }
        __syncwarp();
        if (learned_step) {
            w = __dmul_rn(w, lfac);
        } else {
            w = __dmul_rn(w, (double)size);
            if (MODE != MODE_LEARNED) {
                if (__umul64hi(wu, size) != 0) ovf = true;
                wu = wu * size;
            }
        }
        out.depth = j + 1;
    }
    out.depth = k;
    if (MODE == MODE_LAZY) {
        // closure check over every pair i < j: distinct, pattern edges present,
        // pattern non-edges absent when vertex-induced, restrictions hold;
        // pair q = j (j - 1) / 2 + i, one lane per pair
        const int npairs = k * (k - 1) / 2;
        bool ok = true;
        for (int base = 0; base < npairs; base += 32) {
            const int q = base + (int)lane;
            const int qq = q < npairs ? q : 0;
            int jj = 1;
            while ((jj + 1) * jj / 2 <= qq) jj++;
            const int ii = qq - jj * (jj - 1) / 2;
            const uint32_t *Li = row(ii);
            const uint32_t ni = deg(ii);
            if (q < npairs) {
                const uint32_t vi = wm.v[ii], vj = wm.v[jj];
                bool good = vi != vj;
                const bool edge = (p.back[jj] >> ii) & 1u;
                if (good && (edge || p.induced)) {
                    const bool adj = lane_contains32(Li, ni, vj);
                    good = edge ? adj : !adj;
                }
                if ((p.lower[jj] >> ii) & 1u) good = good && vi < vj;
                ok = ok && good;
            }
        }
        if (!__all_sync(kFull, ok)) return out;
    }
    out.hit = true;
    out.w = w;
    out.wu = (MODE == MODE_LEARNED || ovf) ? 0 : wu;
    out.overflow = ovf;
    return out;
}

// True when some step of the plan has one back-neighbour, the steps the
// MODE_INTERSECT_SINGLE variant evaluates by list positions.
inline bool plan_single_steps(const Plan &p) {
    if (p.induced && !GPM_INDUCED_POSITIONS) return false;
    for (int j = 2; j < p.k; j++)
        if ((p.back[j] & (p.back[j] - 1u)) == 0) return true;
    return false;
}

// The uniform-proposal mode a configuration asks for.
inline int verify_mode(const gpm_config *cfg) {
    if (!cfg) return MODE_INTERSECT;
    if (cfg->verify == GPM_VERIFY_CHECK) return MODE_CHECK;
    if (cfg->verify == GPM_VERIFY_LAZY) return MODE_LAZY;
    return MODE_INTERSECT;
}

// The sampler variant a mode runs with for a plan (or a batch of plans).
inline int kernel_mode(int mode, bool single) {
    return (mode == MODE_INTERSECT && single) ? MODE_INTERSECT_SINGLE : mode;
}

// ------------------------------------------------------------------ launch shape
struct Shape {
    uint32_t blocks, warps, cap, chunk;
};

inline size_t smem_bytes(const Shape &sh, int mode) {
    const size_t per = warp_words(sh.cap, mode == MODE_LEARNED);
    return (size_t)sh.warps * per * sizeof(uint32_t) +
           (mode == MODE_LEARNED ? kMlpSmemFloats * sizeof(float) : 0);
}

// Default on-chip buffer: the largest cap (a multiple of 32 entries) at which
// the sampler's target number of resident blocks (4, or 2 for the learned
// proposal) of `warps` warps still fits one SM's shared memory beside the
// kernel's static shared memory.  More of the partner lists of step 2 then
// stay on chip (on R-MAT 22 a list above 512 entries is otherwise searched in
// global memory in 38% of 4-clique samples).
inline uint32_t fit_cap(const gpm_graph *h, size_t static_smem, uint32_t warps, int mode) {
    const bool learned = mode == MODE_LEARNED;
    const long per_sm = learned ? 2 : GPM_MIN_BLOCKS;
    const long budget = (long)h->smem_per_sm / per_sm - h->smem_reserved - (long)static_smem -
                        (learned ? (long)kMlpSmemFloats * 4 : 0);
    const long words = budget / (4L * (long)warps) - kWarpHeaderWords - (learned ? kLearnedWarpWords : 0);
    long cap = (words / 2) & ~31L;
    if (cap < 64) cap = 64;
    if (cap > 2048) cap = 2048;
    return (uint32_t)cap;
}

// Default buffer for a set of plans: vertex-induced plans test non-edges by
// searches in global memory, which want the L1 capacity a larger shared-memory
// carve-out takes, so they keep 512 entries; otherwise fit_cap.
inline uint32_t default_cap(const gpm_graph *h, size_t static_smem, uint32_t warps, int mode, bool induced) {
    if (mode == MODE_LAZY) return 32;   // NS-base builds no candidate set on chip
    const uint32_t fit = fit_cap(h, static_smem, warps, mode);
    return (induced && mode != MODE_LEARNED && fit > 512) ? 512 : fit;
}

// Samples per chunk is fixed, so per-chunk partials (and every FP64 total
// built from them in chunk order) are the same for every launch shape.
constexpr uint32_t kChunk = 64;

inline Shape pick_shape(gpm_graph *h, const gpm_config *cfg, uint64_t count) {
    (void)h;
    (void)count;
    Shape sh;
    sh.warps = (cfg && cfg->block_warps) ? (cfg->block_warps < 8 ? cfg->block_warps : 8) : 8;
    sh.cap = (cfg && cfg->cap) ? cfg->cap : 0;   // 0: fit_cap at launch
    sh.blocks = (cfg && cfg->grid_blocks) ? cfg->grid_blocks : 0;
    sh.chunk = kChunk;
    return sh;
}

}  // namespace gpm
