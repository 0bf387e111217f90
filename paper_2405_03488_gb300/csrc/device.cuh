// Device helpers of libgpm: the counter-based generator and warp-cooperative
// search primitives over sorted uint32 / uint64 arrays.
#pragma once

#include <stdint.h>

namespace gpm {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Philox4x32-10 (Salmon et al., SC'11): ten rounds; each round forms the
// 64-bit products of counter words 0 and 2 with two odd multipliers and
// crosses their halves with words 1 and 3 and the key; the key advances by
// the two Weyl increments between rounds.
struct Philox4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ Philox4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo_a = 0xD2511F53u * c0;
        const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
        const uint32_t lo_b = 0xCD9E8D57u * c2;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi_b ^ c1 ^ k0;
        const uint32_t n2 = hi_a ^ c3 ^ k1;
        c0 = n0;
        c1 = lo_b;
        c2 = n2;
        c3 = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Philox4{c0, c1, c2, c3};
}

// floor(r * n / 2^64)
__device__ __forceinline__ uint64_t index_map(uint64_t r, uint64_t n) { return __umul64hi(r, n); }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// First index i in [0, len) with a[i] > key (len if none); every lane of the
// warp calls it with the same arguments and gets the same answer.  Each pass
// splits the open range into 32 pieces, so a list of length L costs
// ceil(log32 L) + 1 dependent loads.
template <typename T>
__device__ __forceinline__ uint64_t warp_upper_bound(const T *__restrict__ a, uint64_t len, T key) {
    const unsigned lane = lane_id();
    uint64_t lo = 0, hi = len;
    while (hi - lo > 32) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t pos = lo + lane * step;
        const bool le = (pos < hi) && (__ldg(a + pos) <= key);
        const unsigned m = __ballot_sync(kFull, le);
        const int c = __popc(m);
        if (c == 0) return lo;
        const uint64_t nlo = lo + (uint64_t)(c - 1) * step + 1;
        const uint64_t nhi = lo + (uint64_t)c * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    const uint64_t pos = lo + lane;
    const bool le = (pos < hi) && (__ldg(a + pos) <= key);
    return lo + (uint64_t)__popc(__ballot_sync(kFull, le));
}

// Per-lane membership test in a sorted global list; the iteration count
// depends only on len, so lanes searching one list never diverge.
__device__ __forceinline__ bool lane_contains(const uint32_t *__restrict__ a, uint64_t len, uint32_t x) {
    if (len == 0) return false;
    const uint32_t *b = a;
    uint64_t n = len;
    while (n > 1) {
        const uint64_t half = n >> 1;
        b = (__ldg(b + half) <= x) ? b + half : b;
        n -= half;
    }
    return __ldg(b) == x;
}

// Position of x in the sorted global list a[0, len), or ~0 when absent (one
// lane, the same halving search as lane_contains).
__device__ __forceinline__ uint64_t lane_find(const uint32_t *__restrict__ a, uint64_t len, uint32_t x) {
    if (len == 0) return ~0ull;
    const uint32_t *b = a;
    uint64_t n = len;
    while (n > 1) {
        const uint64_t half = n >> 1;
        b = (__ldg(b + half) <= x) ? b + half : b;
        n -= half;
    }
    return __ldg(b) == x ? (uint64_t)(b - a) : ~0ull;
}

// 32-bit forms of the three searches for one neighbour list (fewer than 2^31
// entries: the load rejects larger degrees).  Same probes in the same order as
// the forms above; positions are offsets from the list's first entry, so index
// arithmetic stays in 32-bit registers.
__device__ __forceinline__ uint32_t warp_upper_bound32(const uint32_t *__restrict__ a, uint32_t len,
                                                       uint32_t key) {
    const unsigned lane = lane_id();
    uint32_t lo = 0, hi = len;
    while (hi - lo > 32) {
        const uint32_t step = ((hi - lo - 1u) >> 5) + 1u;   // ceil((hi - lo) / 32)
        const uint32_t pos = lo + lane * step;
        const bool le = (pos < hi) && (__ldg(a + pos) <= key);
        const unsigned m = __ballot_sync(kFull, le);
        const uint32_t c = (uint32_t)__popc(m);
        if (c == 0) return lo;
        const uint32_t nlo = lo + (c - 1u) * step + 1u;
        const uint32_t nhi = lo + c * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    const uint32_t pos = lo + lane;
    const bool le = (pos < hi) && (__ldg(a + pos) <= key);
    return lo + (uint32_t)__popc(__ballot_sync(kFull, le));
}

__device__ __forceinline__ bool lane_contains32(const uint32_t *__restrict__ a, uint32_t len, uint32_t x) {
    if (len == 0) return false;
    uint32_t b = 0, n = len;
    while (n > 1) {
        const uint32_t half = n >> 1;
        b = (__ldg(a + b + half) <= x) ? b + half : b;
        n -= half;
    }
    return __ldg(a + b) == x;
}

// offset of x in a[0, len), or 0xFFFFFFFF when absent
__device__ __forceinline__ uint32_t lane_find32(const uint32_t *__restrict__ a, uint32_t len, uint32_t x) {
    if (len == 0) return 0xFFFFFFFFu;
    uint32_t b = 0, n = len;
    while (n > 1) {
        const uint32_t half = n >> 1;
        b = (__ldg(a + b + half) <= x) ? b + half : b;
        n -= half;
    }
    return __ldg(a + b) == x ? b : 0xFFFFFFFFu;
}

// Same on a shared-memory list.
__device__ __forceinline__ bool lane_contains_shared(const uint32_t *a, uint32_t len, uint32_t x) {
    if (len == 0) return false;
    uint32_t b = 0, n = len;
    while (n > 1) {
        const uint32_t half = n >> 1;
        b = (a[b + half] <= x) ? b + half : b;
        n -= half;
    }
    return a[b] == x;
}

}  // namespace gpm
