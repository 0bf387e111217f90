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

// The score mapping of a logit z: s = clamp(z / 8 + 1/2, 0, 1), a = 1 + floor(4096 s).
__device__ __forceinline__ uint32_t score_of_logit(float z) {
    float sc = __fmaf_rn(z, 0.125f, 0.5f);
    if (!(sc > 0.f)) sc = 0.f;
    if (sc > 1.f) sc = 1.f;
    return 1u + (uint32_t)floorf(__fmul_rn(sc, 4096.0f));
}

__device__ __forceinline__ uint32_t bf16_bits(float x) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)); }

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
    return score_of_logit(z);
}

// D += A B for one m16n8k16 tile: A 16x16 BF16 (row-major), B 16x8 BF16
// (column-major), D 16x8 FP32; fragments in the PTX ISA's register layout.
__device__ __forceinline__ void mma_bf16_16816(float d[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Scores of 16 candidates (rows) with the 64 x 64 layer on the tensor cores
// (the warp calls it together).  feat(c, &f0, &f1, &f2) gives candidate c's
// features.  Layer 1 runs in FP32 (lane l: candidate l mod 16, hidden units
// 32 (l / 16) .. + 31) and is rounded to BF16 into the warp's tile; layer 2
// is 8 x 4 mma.sync m16n8k16 (BF16 products, FP32 accumulation); bias, ReLU
// and the output layer follow in FP32, reduced over the 4 lanes that share a
// row.  Writes score[c] for c < n.  Not bit-identical to the FP32 chain of
// mlp_score_lane: its h1 is rounded to BF16 and the sums run in the tensor
// cores' order.
template <typename Feat>
__device__ __forceinline__ void mlp_scores_tc(const WarpMem &wm, uint32_t n, Feat feat, uint32_t *score) {
    const unsigned lane = lane_id();
    const float *w1 = wm.W, *b1 = wm.W + 192, *b2 = wm.W + 4352, *w3 = wm.W + 4416, *b3 = wm.W + 4480;
    uint16_t *H = wm.htile;
    {
        const uint32_t c = lane & 15u, o0 = (lane >> 4) * 32;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        if (c < n) feat(c, &f0, &f1, &f2);
        uint32_t *row = reinterpret_cast<uint32_t *>(H + c * kW2Stride + o0);
#pragma unroll
        for (int o = 0; o < 32; o += 2) {
            float h[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int u = o0 + o + q;
                float acc = b1[u];
                acc = __fmaf_rn(w1[u * 3 + 0], f0, acc);
                acc = __fmaf_rn(w1[u * 3 + 1], f1, acc);
                acc = __fmaf_rn(w1[u * 3 + 2], f2, acc);
                h[q] = acc > 0.f ? acc : 0.f;
            }
            row[o / 2] = bf16_bits(h[0]) | (bf16_bits(h[1]) << 16);
        }
    }
    __syncwarp();
    const unsigned gq = lane >> 2, tq = lane & 3u;
    float d[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        const uint32_t *r0 = reinterpret_cast<const uint32_t *>(H + gq * kW2Stride + ks * 16 + tq * 2);
        const uint32_t *r1 = reinterpret_cast<const uint32_t *>(H + (gq + 8) * kW2Stride + ks * 16 + tq * 2);
        const uint32_t a0 = r0[0], a1 = r1[0], a2 = r0[4], a3 = r1[4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const uint32_t *bw = reinterpret_cast<const uint32_t *>(wm.W2b + (nt * 8 + gq) * kW2Stride + ks * 16 +
                                                                    tq * 2);
            mma_bf16_16816(d[nt], a0, a1, a2, a3, bw[0], bw[4]);
        }
    }
    float z0 = 0.f, z1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; nt++)
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int o = nt * 8 + tq * 2 + q;
            const float h0 = __fadd_rn(d[nt][q], b2[o]), h1 = __fadd_rn(d[nt][2 + q], b2[o]);
            z0 = __fmaf_rn(w3[o], h0 > 0.f ? h0 : 0.f, z0);
            z1 = __fmaf_rn(w3[o], h1 > 0.f ? h1 : 0.f, z1);
        }
    z0 = __fadd_rn(z0, __shfl_xor_sync(kFull, z0, 1));
    z0 = __fadd_rn(z0, __shfl_xor_sync(kFull, z0, 2));
    z1 = __fadd_rn(z1, __shfl_xor_sync(kFull, z1, 1));
    z1 = __fadd_rn(z1, __shfl_xor_sync(kFull, z1, 2));
    if (tq == 0) {
        if (gq < n) score[gq] = score_of_logit(__fadd_rn(z0, b3[0]));
        if (gq + 8 < n) score[gq + 8] = score_of_logit(__fadd_rn(z1, b3[0]));
    }
    __syncwarp();
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
                                              bool tc, uint64_t *A_out, uint32_t *a_out) {
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
    // (lane-per-candidate forms of this count, walking each candidate's list
    // in its own lane, measured no faster: the count's instructions, not the
    // latency of the list reads, bound it)
    for (uint32_t i = 0; i < sz; i++) {
        const uint64_t xb = cb[i], dx = cd[i];
        const uint64_t nxt = lookahead_count(g, p, wm, Sj, sz, i, j, lb, le, xb, xb + dx, xb + cu[i]);
        __syncwarp();
        if (lane == 0) cu[i] = (uint32_t)nxt;
    }
    __syncwarp();
    uint64_t A = 0;
    const float fj = __int2float_rn(j);
    if (tc) {
        // scores, 16 candidates per tensor-core tile
        for (uint32_t base = 0; base < sz; base += 16) {
            auto feat = [&](uint32_t c, float *f0, float *f1, float *f2) {
                *f0 = flog2p1(cd[base + c]);
                *f1 = fj;
                *f2 = flog2p1(cu[base + c]);
            };
            mlp_scores_tc(wm, sz - base < 16 ? sz - base : 16, feat, wm.score + base);
        }
        for (uint32_t base = 0; base < sz; base += 32) {
            uint32_t a = base + lane < sz ? wm.score[base + lane] : 0u;
#pragma unroll
            for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
            A += a;
        }
    } else {
        // scores, one candidate per lane
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
