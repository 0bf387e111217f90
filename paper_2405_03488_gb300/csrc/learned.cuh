// Device code of the learned proposal (not in the paper), used by the sampler
// in MODE_LEARNED and by the scoring and training kernels: the exact FP32
// feature log2(1 + d), the 3 -> 64 -> 64 -> 1 score of a candidate, the
// lookahead size |S_{j+1}(x)| and the score-proportional draw.  Included by
// sampler.cuh after the warp memory layout and the warp helpers.
#pragma once

namespace gpm {

// log2(1 + d) as the chord between powers of two: e + (y - 2^e) / 2^e with
// y = d + 1 and e = floor(log2 y), every operation correctly rounded in FP32.
__device__ __forceinline__ float flog2p1(uint64_t d) {
    const uint64_t y = d + 1;
    const int e = 63 - __clzll((long long)y);
    const uint64_t p2 = 1ull << e;
    const float frac = __fdiv_rn(__ull2float_rn(y - p2), __ull2float_rn(p2));
    return __fadd_rn(__int2float_rn(e), frac);
}

// Score of one candidate, computed by one lane alone: the 3 -> 64 -> 64 -> 1
// ReLU MLP with FP32 fused multiply-adds in input order (hidden layer 2 and
// the output chain walk the units in ascending order, as the oracle does),
// weights read as broadcasts from the block's copy (W2 row-major, rows of 64
// loaded 4 at a time), the output mapped without exp to
// s = clamp(z / 8 + 1/2, 0, 1) and a = 1 + floor(4096 s).
__device__ __forceinline__ uint32_t mlp_score_lane(const float *W, float f0, float f1, float f2) {
    const float *w1 = W, *b1 = W + 192, *w2 = W + 256, *b2 = W + 4352, *w3 = W + 4416, *b3 = W + 4480;
    float h1[64];
#pragma unroll
    for (int o = 0; o < 64; o++) {
        float acc = b1[o];
        acc = __fmaf_rn(w1[o * 3 + 0], f0, acc);
        acc = __fmaf_rn(w1[o * 3 + 1], f1, acc);
        acc = __fmaf_rn(w1[o * 3 + 2], f2, acc);
        h1[o] = acc > 0.f ? acc : 0.f;
    }
    float z = b3[0];
#pragma unroll 1
    for (int o = 0; o < 64; o += 2) {
        // two hidden units at a time: two independent chains, each in input order
        const float4 *ra = reinterpret_cast<const float4 *>(w2 + o * 64);
        const float4 *rb = reinterpret_cast<const float4 *>(w2 + (o + 1) * 64);
        float acc_a = b2[o], acc_b = b2[o + 1];
#pragma unroll
        for (int i4 = 0; i4 < 16; i4++) {
            const float4 wa = ra[i4], wb = rb[i4];
            acc_a = __fmaf_rn(wa.x, h1[4 * i4 + 0], acc_a);
            acc_b = __fmaf_rn(wb.x, h1[4 * i4 + 0], acc_b);
            acc_a = __fmaf_rn(wa.y, h1[4 * i4 + 1], acc_a);
            acc_b = __fmaf_rn(wb.y, h1[4 * i4 + 1], acc_b);
            acc_a = __fmaf_rn(wa.z, h1[4 * i4 + 2], acc_a);
            acc_b = __fmaf_rn(wb.z, h1[4 * i4 + 2], acc_b);
            acc_a = __fmaf_rn(wa.w, h1[4 * i4 + 3], acc_a);
            acc_b = __fmaf_rn(wb.w, h1[4 * i4 + 3], acc_b);
        }
        z = __fmaf_rn(w3[o], acc_a > 0.f ? acc_a : 0.f, z);
        z = __fmaf_rn(w3[o + 1], acc_b > 0.f ? acc_b : 0.f, z);
    }
    float sc = __fmaf_rn(z, 0.125f, 0.5f);
    if (!(sc > 0.f)) sc = 0.f;
    if (sc > 1.f) sc = 1.f;
    return 1u + (uint32_t)floorf(__fmul_rn(sc, 4096.0f));
}

// |S_{j+1}| if candidate Sj[ix] were chosen as v_j.  When S_{j+1} extends S_j
// by one adjacency it is counted from S_j on chip (elements above the new
// bound that lie in N(x)); otherwise every condition is tested on the lists.
template <typename PlanT>
static __device__ __noinline__ uint64_t lookahead_count(const DGraph &g, const PlanT &p, const WarpMem &wm,
                                                 const uint32_t *Sj, uint32_t sz, uint32_t ix, int j, uint64_t lb,
                                                 uint64_t le, uint64_t xb, uint64_t xe, uint64_t xu) {
    const unsigned lane = lane_id();
    const int jj = j + 1;
    const uint32_t x = Sj[ix];
    const uint32_t lm = p.lower[jj];
    const bool has_lo = lm != 0;
    uint32_t lo = 0;
    for (int i = 0; i < jj; i++)
        if ((lm >> i) & 1u) {
            const uint32_t vi = (i == j) ? x : wm.v[i];
            lo = vi > lo ? vi : lo;
        }
    uint64_t cnt = 0;
    if (p.reuse[jj] == 1) {
        // entries of S_j at or below the bound (S_j ascends, so with the bound
        // at x itself they are the first ix + 1)
        uint32_t s0 = 0;
        if (has_lo && lo == x)
            s0 = ix + 1;
        else if (has_lo)
            for (uint32_t base = 0; base < sz; base += 32) {
                const uint32_t idx = base + lane;
                s0 += __popc(__ballot_sync(kFull, idx < sz && Sj[idx] <= lo));
            }
        const uint32_t P = sz - s0;
        if (P == 0) return 0;
        uint64_t ls = xb;
        if (has_lo) {
            if (lo == x) ls = xu;
            else if (lo > x) ls = xu + warp_upper_bound(g.col + xu, xe - xu, lo);
            else ls = xb + warp_upper_bound(g.col + xb, xu - xb, lo);
        }
        const uint64_t L = xe > ls ? xe - ls : 0;
        if (L <= 8ull * P + 32) {
            for (uint64_t base = ls; base < xe; base += 32) {
                const uint64_t idx = base + lane;
                const bool ok = idx < xe && lane_contains_shared(Sj + s0, P, __ldg(g.col + idx));
                cnt += __popc(__ballot_sync(kFull, ok));
            }
        } else {
            for (uint32_t base = 0; base < P; base += 32) {
                const uint32_t idx = base + lane;
                const bool ok = idx < P && lane_contains(g.col + ls, L, Sj[s0 + idx]);
                cnt += __popc(__ballot_sync(kFull, ok));
            }
        }
        return cnt;
    }
    const uint64_t mb = ((int)lane == j) ? xb : lb, me = ((int)lane == j) ? xe : le;
    const uint32_t back = p.back[jj];
    const uint64_t key = ((int)lane < jj && ((back >> lane) & 1u)) ? (((me - mb) << 5) | lane) : ~0ull;
    const int d = (int)(warp_min_u64(key) & 31u);
    const uint64_t db = __shfl_sync(kFull, mb, d), de = __shfl_sync(kFull, me, d);
    const uint64_t start = has_lo ? db + warp_upper_bound(g.col + db, de - db, lo) : db;
    for (uint64_t base = start; base < de; base += 32) {
        const uint64_t idx = base + lane;
        const bool valid = idx < de;
        const uint32_t y = valid ? __ldg(g.col + idx) : 0u;
        bool ok = true;
        for (int i = 0; i < jj; i++) {
            const uint64_t bi = __shfl_sync(kFull, mb, i), ei = __shfl_sync(kFull, me, i);
            const uint32_t vi = (i == j) ? x : wm.v[i];
            ok = ok && (y != vi);
            const bool edge = (back >> i) & 1u;
            if (edge && i != d) ok = ok && lane_contains(g.col + bi, ei - bi, y);
            else if (!edge && p.induced) ok = ok && !lane_contains(g.col + bi, ei - bi, y);
        }
        cnt += __popc(__ballot_sync(kFull, ok && valid));
    }
    return cnt;
}

// Learned draw over the materialised S_j: scores a_x of every candidate, A =
// their sum, t = floor(r A / 2^64), the smallest index whose score prefix
// exceeds t.
template <typename PlanT>
static __device__ __noinline__ uint32_t learned_pick(const DGraph &g, const PlanT &p, const WarpMem &wm, const uint32_t *Sj,
                                              uint32_t sz, int j, uint64_t r, uint64_t lb, uint64_t le,
                                              uint64_t *A_out, uint32_t *a_out) {
    const unsigned lane = lane_id();
    // every candidate's CSR offsets in one pass over the lanes
    uint64_t *cb = reinterpret_cast<uint64_t *>(wm.score + kLearnedMax);
    uint32_t *cd = wm.score + 3 * kLearnedMax, *cu = wm.score + 4 * kLearnedMax;
    for (uint32_t i = lane; i < sz; i += 32) {
        const uint32_t x = Sj[i];
        const uint64_t xb = __ldg(g.row_ptr + x);
        cb[i] = xb;
        cd[i] = (uint32_t)(__ldg(g.row_ptr + x + 1) - xb);
        cu[i] = (uint32_t)(__ldg(g.up + x) - xb);
    }
    __syncwarp();
    // lookahead sizes |S_{j+1}(x)|, one warp-wide count per candidate, into cu
    for (uint32_t i = 0; i < sz; i++) {
        const uint64_t xb = cb[i], dx = cd[i];
        const uint64_t nxt = lookahead_count(g, p, wm, Sj, sz, i, j, lb, le, xb, xb + dx, xb + cu[i]);
        __syncwarp();
        if (lane == 0) cu[i] = (uint32_t)nxt;
    }
    __syncwarp();
    // scores, one candidate per lane
    uint64_t A = 0;
    const float fj = __int2float_rn(j);
    for (uint32_t base = 0; base < sz; base += 32) {
        const uint32_t i = base + lane;
        uint32_t a = 0;
        if (i < sz) {
            a = mlp_score_lane(wm.W, flog2p1(cd[i]), fj, flog2p1(cu[i]));
            wm.score[i] = a;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
        A += a;
    }
    __syncwarp();
    const uint64_t t = index_map(r, A);
    uint64_t run = 0;
    uint32_t chosen = 0;
    for (uint32_t base = 0; base < sz; base += 32) {
        const uint32_t idx = base + lane;
        uint64_t inc = idx < sz ? wm.score[idx] : 0;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const uint64_t t2 = __shfl_up_sync(kFull, inc, dd);
            if ((int)lane >= dd) inc += t2;
        }
        const unsigned m = __ballot_sync(kFull, idx < sz && run + inc > t);
        if (m) {
            chosen = base + __ffs(m) - 1;
            break;
        }
        run += __shfl_sync(kFull, inc, 31);
    }
    *A_out = A;
    *a_out = wm.score[chosen];
    return Sj[chosen];
}

}  // namespace gpm
