// Colour sparsification (GS) and exact counting.
//
// Colour sparsification (Sec. 2.2.2): every vertex gets a colour in [0, c)
// and only monochromatic edges stay; a match with k vertices survives iff its
// vertices share one colour, with probability c^-(k-1), so the exact count C'
// of the sparsified graph scaled by c^(k-1) is an unbiased estimate of C
// (Sec. 5.2; the paper writes the exponent with the edge count, which only
// agrees for triangles).  colour(v) = floor(w0 * c / 2^32), w0 the first word
// of Philox4x32-10 at counter (v_lo, v_hi, colouring, slot << 8 | 2), key =
// seed, a stream disjoint from the sampling words.
//
// Bernoulli edge sparsification (Algorithm 2) keeps every edge independently
// with probability p = t / 2^32: edge {u, w} stays iff the first word of
// Philox4x32-10 at counter (min(u, w), max(u, w), colouring, slot << 8 | 3) is
// below t, one decision for both CSR entries; a match with l edges survives
// with probability p^l, so C' (2^32 / t)^l estimates C for edge-induced
// counting (removing edges can create vertex-induced occurrences, so that
// case is refused).  Several independent sparsifications ("samplers") are
// averaged; with R >= 2 their sample standard deviation s gives the interval
// half width z s / sqrt(R).
//
// Sparsification reads every edge once and writes the kept ones (the paper's
// preprocessing cost |E| (w1 + p w2), Sec. 4.4): a colour pass, a count pass
// and a compaction pass (one warp per vertex, ballot compaction keeps the
// neighbour order), with the row offsets from the library's prefix scan.
//
// Exact counting runs the same plan as the sampler but follows every branch
// (the nested loops of Sec. 4.4): one warp walks the subtree of one first edge
// depth first; each level keeps its driver-list cursor and one 32-entry chunk
// of candidates on chip, so no level needs more than 32 slots, and the last
// level only counts |S_{k-1}|.  Per-warp totals are added with 64-bit atomics
// (exact integers, order independent).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>

#include "device.cuh"
#include "internal.h"

namespace gpm {

cudaError_t scan_exclusive_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t st);

__global__ void colour_kernel(uint64_t n, uint32_t c, uint64_t seed, uint32_t colouring, uint32_t slot,
                              uint32_t *colours) {
    const uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const Philox4 o = philox10((uint32_t)v, (uint32_t)(v >> 32), colouring, (slot << 8) | 2u, (uint32_t)seed,
                               (uint32_t)(seed >> 32));
    colours[v] = (uint32_t)(((uint64_t)o.x * (uint64_t)c) >> 32);
}

// Sharding by colour class: a vertex whose class c has c mod world != rank
// gets a colour of its own (never below c, never another vertex's), so none
// of its edges survives and only the rank's classes remain.
__global__ void class_mask(uint64_t n, uint32_t rank, uint32_t world, uint32_t *colours) {
    const uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (colours[v] % world != rank) colours[v] = 0xFFFFFFFFu - (uint32_t)v;
}

__global__ void keep_count(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                           const uint32_t *__restrict__ colours, uint64_t n, uint64_t *cnt) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < n; v += nw) {
        const uint64_t b = row_ptr[v], e = row_ptr[v + 1];
        const uint32_t cv = colours[v];
        uint64_t c = 0;
        for (uint64_t i = b + lane; i < e; i += 32) c += (colours[__ldg(col + i)] == cv);
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) cnt[v] = c;
    }
}

__device__ __forceinline__ bool bes_keep(uint64_t seed, uint32_t u, uint32_t w, uint32_t colouring, uint32_t slot,
                                         uint64_t t) {
    const uint32_t lo = u < w ? u : w, hi = u < w ? w : u;
    const Philox4 o = philox10(lo, hi, colouring, (slot << 8) | 3u, (uint32_t)seed, (uint32_t)(seed >> 32));
    return (uint64_t)o.x < t;
}

__global__ void bes_count(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col, uint64_t n,
                          uint64_t seed, uint32_t colouring, uint32_t slot, uint64_t t, uint64_t *cnt) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < n; v += nw) {
        const uint64_t b = row_ptr[v], e = row_ptr[v + 1];
        uint64_t c = 0;
        for (uint64_t i = b + lane; i < e; i += 32) c += bes_keep(seed, (uint32_t)v, __ldg(col + i), colouring, slot, t);
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) cnt[v] = c;
    }
}

__global__ void bes_write(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col, uint64_t n,
                          uint64_t seed, uint32_t colouring, uint32_t slot, uint64_t t,
                          const uint64_t *__restrict__ row_out, uint32_t *col_out) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < n; v += nw) {
        const uint64_t b = row_ptr[v], e = row_ptr[v + 1];
        uint64_t pos = row_out[v];
        for (uint64_t base = b; base < e; base += 32) {
            const uint64_t i = base + lane;
            const uint32_t x = i < e ? __ldg(col + i) : 0u;
            const bool keep = i < e && bes_keep(seed, (uint32_t)v, x, colouring, slot, t);
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) col_out[pos + __popc(m & ((1u << lane) - 1u))] = x;
            pos += __popc(m);
        }
    }
}

__global__ void keep_write(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                           const uint32_t *__restrict__ colours, uint64_t n, const uint64_t *__restrict__ row_out,
                           uint32_t *col_out) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < n; v += nw) {
        const uint64_t b = row_ptr[v], e = row_ptr[v + 1];
        const uint32_t cv = colours[v];
        uint64_t pos = row_out[v];
        for (uint64_t base = b; base < e; base += 32) {
            const uint64_t i = base + lane;
            const uint32_t x = i < e ? __ldg(col + i) : 0u;
            const bool keep = i < e && colours[x] == cv;
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) col_out[pos + __popc(m & ((1u << lane) - 1u))] = x;
            pos += __popc(m);
        }
    }
}

// ------------------------------------------------------------------ exact count
struct Level {
    uint64_t base, end;      // driver cursor and end
    uint32_t mask;           // candidates of the current chunk not yet visited
    int32_t driver;
};

__device__ __forceinline__ bool exact_ok(const DGraph &g, const Plan &p, const uint32_t *v, int j, int driver,
                                         uint64_t lb, uint64_t le, uint32_t x) {
    bool ok = true;
    const uint32_t back = p.back[j];
    for (int i = 0; i < j; i++) {
        const uint64_t b = __shfl_sync(kFull, lb, i);
        const uint64_t e = __shfl_sync(kFull, le, i);
        ok = ok && (x != v[i]);
        const bool edge = (back >> i) & 1u;
        if (edge && i != driver) ok = ok && lane_contains(g.col + b, e - b, x);
        else if (!edge && p.induced) ok = ok && !lane_contains(g.col + b, e - b, x);
    }
    return ok;
}

// Driver (shortest back-neighbour list) and its range above the lower bound.
__device__ __forceinline__ void level_init(const DGraph &g, const Plan &p, const uint32_t *v, int j, uint64_t lb,
                                           uint64_t le, Level *L) {
    const unsigned lane = lane_id();
    const uint32_t back = p.back[j];
    uint64_t key = ((int)lane < j && ((back >> lane) & 1u)) ? (((le - lb) << 5) | lane) : ~0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        uint64_t t = __shfl_xor_sync(kFull, key, o);
        key = t < key ? t : key;
    }
    const int d = (int)(key & 31u);
    const uint64_t b = __shfl_sync(kFull, lb, d);
    const uint64_t e = __shfl_sync(kFull, le, d);
    const uint32_t lm = p.lower[j];
    uint32_t lo = 0;
    for (int i = 0; i < j; i++)
        if ((lm >> i) & 1u) lo = v[i] > lo ? v[i] : lo;
    const uint64_t start = lm ? b + warp_upper_bound(g.col + b, e - b, lo) : b;
    if (lane == 0) {
        L->base = start;
        L->end = e;
        L->mask = 0;
        L->driver = d;
    }
    __syncwarp();
}

// stop (host memory mapped into the device, or null): once the host sets it,
// every warp leaves at its next grab of first edges or within 256 search
// steps and raises *timed_out; the total is then a lower bound.
__global__ void __launch_bounds__(256) exact_kernel(const DGraph g, const Plan p, uint64_t M, unsigned int *counter,
                                                    uint32_t per_grab, unsigned long long *total,
                                                    const volatile int *stop, unsigned int *timed_out) {
    __shared__ Level lev[8][kMaxK];
    __shared__ uint32_t vv[8][kMaxK];
    __shared__ uint32_t buf[8][kMaxK][32];
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    Level *L = lev[warp];
    uint32_t *v = vv[warp];
    const int k = p.k;
    unsigned long long acc = 0;
    bool out_of_time = false;
    uint32_t steps = 0;
    auto stopped = [&]() -> bool {
        int f = 0;
        if (lane == 0) f = *stop;
        return __shfl_sync(kFull, f, 0) != 0;
    };
    for (;;) {
        if (stop && stopped()) out_of_time = true;
        if (out_of_time) break;
        unsigned grab = 0;
        if (lane == 0) grab = atomicAdd(counter, 1u);
        grab = __shfl_sync(kFull, grab, 0);
        const uint64_t e0 = (uint64_t)grab * per_grab;
        if (e0 >= M) break;
        const uint64_t e1 = (e0 + per_grab < M) ? e0 + per_grab : M;
        for (uint64_t e = e0; e < e1; e++) {
            uint32_t v0, v1;
            if (p.oriented && g.edges) {
                const uint64_t pr = __ldg(g.edges + e);
                v0 = (uint32_t)pr;
                v1 = (uint32_t)(pr >> 32);
            } else if (p.oriented) {
                const uint64_t u = warp_upper_bound(g.uoff, g.n + 1, e) - 1;
                v0 = (uint32_t)u;
                v1 = __ldg(g.col + __ldg(g.up + u) + (e - __ldg(g.uoff + u)));
            } else {
                const uint64_t u = warp_upper_bound(g.row_ptr, g.n + 1, e) - 1;
                v0 = (uint32_t)u;
                v1 = __ldg(g.col + e);
            }
            if (k == 2) {
                acc += 1;
                continue;
            }
            uint64_t lb = 0, le = 0;
            if (lane == 0) {
                lb = __ldg(g.row_ptr + v0);
                le = __ldg(g.row_ptr + v0 + 1);
                v[0] = v0;
                v[1] = v1;
            } else if (lane == 1) {
                lb = __ldg(g.row_ptr + v1);
                le = __ldg(g.row_ptr + v1 + 1);
            }
            __syncwarp();
            int j = 2;
            level_init(g, p, v, j, lb, le, &L[j]);
            while (j >= 2) {
                if (stop && ((++steps) & 255u) == 0 && stopped()) {
                    out_of_time = true;
                    break;
                }
                Level &cur = L[j];
                const bool last = (j == k - 1);
                if (cur.mask == 0 || last) {
                    if (cur.base >= cur.end) {
                        j--;
                        continue;
                    }
                    const uint64_t idx = cur.base + lane;
                    const bool valid = idx < cur.end;
                    const uint32_t y = valid ? __ldg(g.col + idx) : 0u;
                    const bool ok = exact_ok(g, p, v, j, cur.driver, lb, le, y) && valid;
                    const unsigned m = __ballot_sync(kFull, ok);
                    if (last) {
                        acc += __popc(m);
                    } else {
                        buf[warp][j][lane] = y;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        cur.base += 32;
                        cur.mask = last ? 0u : m;
                    }
                    __syncwarp();
                    continue;
                }
                const uint32_t m = cur.mask;
                const int bit = __ffs(m) - 1;
                const uint32_t x = buf[warp][j][bit];
                __syncwarp();
                if (lane == 0) {
                    cur.mask = m & (m - 1u);
                    v[j] = x;
                }
                if ((int)lane == j) {
                    lb = __ldg(g.row_ptr + x);
                    le = __ldg(g.row_ptr + x + 1);
                }
                __syncwarp();
                j++;
                level_init(g, p, v, j, lb, le, &L[j]);
            }
            if (out_of_time) break;
        }
    }
    if (lane == 0 && acc) atomicAdd(total, acc);
    if (lane == 0 && out_of_time) atomicExch(timed_out, 1u);
}

}  // namespace gpm

using namespace gpm;

namespace gpm {

gpm_status exact_count_plan(gpm_graph *h, const Plan &p, uint64_t *out, float *kernel_ms, double max_seconds) {
    const uint64_t M = p.oriented ? h->d.m : h->d.nnz;
    unsigned long long *tot = nullptr;
    unsigned int *ctr = nullptr;
    if (cudaMallocAsync((void **)&tot, sizeof(unsigned long long), h->stream) != cudaSuccess ||
        cudaMallocAsync((void **)&ctr, sizeof(unsigned int) * 2, h->stream) != cudaSuccess) {
        set_error("exact count: device allocation failed");
        return GPM_ERR_OOM;
    }
    cudaMemsetAsync(tot, 0, sizeof(unsigned long long), h->stream);
    cudaMemsetAsync(ctr, 0, sizeof(unsigned int) * 2, h->stream);
    // the stop flag lives in pinned host memory mapped into the device
    int *stop_h = nullptr, *stop_d = nullptr;
    if (max_seconds > 0.0) {
        if (cudaHostAlloc((void **)&stop_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&stop_d, stop_h, 0) != cudaSuccess) {
            if (stop_h) cudaFreeHost(stop_h);
            cudaFreeAsync(tot, h->stream);
            cudaFreeAsync(ctr, h->stream);
            set_error("exact count: mapped host allocation failed");
            return GPM_ERR_OOM;
        }
        *(volatile int *)stop_h = 0;
    }
    const auto t_launch = std::chrono::steady_clock::now();
    uint64_t per = M / ((uint64_t)h->sm_count * 8 * 8 * 64) + 1;
    if (per > 64) per = 64;
    if (M / per >= (1ull << 32)) per = M / (1ull << 31) + 1;
    if (kernel_ms) cudaEventRecord(h->ev0, h->stream);
    if (M > 0)
        exact_kernel<<<h->sm_count * 8, 256, 0, h->stream>>>(h->d, p, M, ctr, (uint32_t)per, tot, stop_d, ctr + 1);
    if (kernel_ms) cudaEventRecord(h->ev1, h->stream);
    cudaError_t e = cudaGetLastError();
    // wall-clock watchdog: raise the flag once max_seconds have passed
    while (e == cudaSuccess && stop_h) {
        const cudaError_t q = cudaStreamQuery(h->stream);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) {
            e = q;
            break;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_launch).count();
        if (el >= max_seconds) *(volatile int *)stop_h = 1;
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    unsigned long long r = 0;
    unsigned int late = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, tot, sizeof(r), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&late, ctr + 1, sizeof(late), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(tot, h->stream);
    cudaFreeAsync(ctr, h->stream);
    if (stop_h) cudaFreeHost(stop_h);
    if (e != cudaSuccess) {
        set_error(std::string("exact count: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    if (kernel_ms) cudaEventElapsedTime(kernel_ms, h->ev0, h->ev1);
    *out = r;
    if (late) {
        set_error("exact count: max_seconds reached; the count is a lower bound");
        return GPM_ERR_NOT_CONVERGED;
    }
    return GPM_OK;
}

// Colour + sparsify into freshly allocated device arrays (caller frees).
gpm_status sparsify_alloc(gpm_graph *h, uint32_t c, uint64_t seed, uint32_t colouring, uint32_t slot,
                          uint64_t **row_out, uint32_t **col_out, uint64_t *kept, uint64_t *user_row,
                          uint32_t *user_col, uint64_t bes_t, uint32_t class_rank, uint32_t class_world) {
    const uint64_t n = h->d.n;
    cudaStream_t st = h->stream;
    uint32_t *colours = nullptr;
    uint64_t *cnt = nullptr, *row = user_row;
    uint32_t *col = user_col;
    cudaError_t e = cudaMallocAsync((void **)&colours, sizeof(uint32_t) * (n + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cnt, sizeof(uint64_t) * (n + 1), st);
    if (e == cudaSuccess && !row) e = cudaMallocAsync((void **)&row, sizeof(uint64_t) * (n + 1), st);
    if (e != cudaSuccess) {
        cudaFreeAsync(colours, st);
        cudaFreeAsync(cnt, st);
        set_error("sparsify: device allocation failed");
        return GPM_ERR_OOM;
    }
    const unsigned blocks_v = (unsigned)((n + 255) / 256);
    const uint64_t warps = n < (1ull << 22) ? (n ? n : 1) : (1ull << 22);
    const unsigned blocks_w = (unsigned)((warps * 32 + 255) / 256);
    if (n && bes_t) {
        bes_count<<<blocks_w, 256, 0, st>>>(h->d.row_ptr, h->d.col, n, seed, colouring, slot, bes_t, cnt);
    } else if (n) {
        colour_kernel<<<blocks_v, 256, 0, st>>>(n, c, seed, colouring, slot, colours);
        if (class_world > 1) class_mask<<<blocks_v, 256, 0, st>>>(n, class_rank, class_world, colours);
        keep_count<<<blocks_w, 256, 0, st>>>(h->d.row_ptr, h->d.col, colours, n, cnt);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_exclusive_u64(cnt, row, n, st);
    uint64_t k = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&k, row + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && !col) e = cudaMallocAsync((void **)&col, sizeof(uint32_t) * (k ? k : 1), st);
    if (e == cudaSuccess && n) {
        if (bes_t)
            bes_write<<<blocks_w, 256, 0, st>>>(h->d.row_ptr, h->d.col, n, seed, colouring, slot, bes_t, row, col);
        else
            keep_write<<<blocks_w, 256, 0, st>>>(h->d.row_ptr, h->d.col, colours, n, row, col);
        e = cudaGetLastError();
    }
    cudaFreeAsync(colours, st);
    cudaFreeAsync(cnt, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error(std::string("sparsify: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    *kept = k;
    if (row_out) *row_out = row;
    if (col_out) *col_out = col;
    return GPM_OK;
}

static uint64_t bes_threshold(double p) { return p >= 1.0 ? (1ull << 32) : (uint64_t)std::floor(p * 4294967296.0); }

gpm_status gs_estimate(gpm_graph *h, const Plan &p, uint64_t seed, double delta, const gpm_config *cfg,
                       gpm_result *out) {
    const auto t0 = std::chrono::steady_clock::now();
    const uint32_t c = (cfg && cfg->colors) ? cfg->colors : 8;
    const uint32_t slot = cfg ? cfg->slot : 0;
    const uint32_t R = (cfg && cfg->samplers) ? cfg->samplers : 1;
    const double ep = cfg ? cfg->edge_p : 0.0;
    if (!(ep >= 0.0 && ep <= 1.0)) {
        set_error("GS: edge_p must be in [0, 1]");
        return GPM_ERR_ARG;
    }
    const uint64_t t = ep > 0.0 ? bes_threshold(ep) : 0;
    if (ep > 0.0 && t == 0) {
        set_error("GS: edge_p below 2^-32");
        return GPM_ERR_ARG;
    }
    if (ep > 0.0 && p.induced) {
        set_error("GS: Bernoulli edge sparsification has no unbiased vertex-induced estimator");
        return GPM_ERR_UNSUPPORTED;
    }
    // scale of one sparsified count: c^(k-1) (colours) or (2^32 / t)^l (edges),
    // l = the pattern's edge count, as l multiplications left to right
    double scale = 1.0;
    if (ep > 0.0) {
        int l = 0;
        for (int j = 0; j < p.k; j++) l += __builtin_popcount(p.back[j]);
        for (int q = 0; q < l; q++) scale *= 4294967296.0 / (double)t;
    } else {
        scale = std::pow((double)c, (double)(p.k - 1));
    }
    const double budget = cfg ? cfg->max_seconds : 0.0;
    gpm_status late = GPM_OK;
    double t_pre = 0.0, t_search = 0.0, mean = 0.0;
    uint64_t total = 0;
    std::vector<double> est(R);
    for (uint32_t r = 0; r < R; r++) {
        const auto ta = std::chrono::steady_clock::now();
        uint64_t *row = nullptr;
        uint32_t *col = nullptr;
        uint64_t kept = 0;
        gpm_status st = sparsify_alloc(h, c, seed, r, slot, &row, &col, &kept, nullptr, nullptr, t);
        if (st != GPM_OK) return st;
        gpm_graph *gs = nullptr;
        st = gpm_load_csr(h->d.n, row, col, GPM_DEVICE_PTRS, h->stream, &gs);
        t_pre += std::chrono::duration<double>(std::chrono::steady_clock::now() - ta).count();
        uint64_t cp = 0;
        float ms = 0.f;
        if (st == GPM_OK) {
            st = exact_count_plan(gs, p, &cp, &ms, budget);
            if (st == GPM_ERR_NOT_CONVERGED) {
                late = st;
                st = GPM_OK;
            }
        }
        if (gs) gpm_free_graph(gs);
        cudaFree(row);
        cudaFree(col);
        if (st != GPM_OK) return st;
        t_search += ms * 1e-3;
        total += cp;
        est[r] = (double)cp * scale;
        mean += est[r];
    }
    mean /= (double)R;
    out->exact_count = total;
    out->estimate = mean;
    out->ci_half_width = NAN;
    out->eps_hat = NAN;
    if (R >= 2) {
        double ss = 0.0;
        for (uint32_t r = 0; r < R; r++) ss += (est[r] - mean) * (est[r] - mean);
        const double s = std::sqrt(ss / (double)(R - 1));
        out->ci_half_width = normal_quantile(1.0 - delta / 2.0) * (s / std::sqrt((double)R));
        out->eps_hat = mean > 0.0 ? out->ci_half_width / mean : INFINITY;
    }
    out->samples = R;
    out->scheme_used = GPM_GS;
    out->converged = late == GPM_OK ? 1 : 0;
    out->t_preproc_s = t_pre;
    out->t_sample_s = t_search;
    out->kernel_launches += 7 * (uint64_t)R;
    out->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (late != GPM_OK) set_error("GS: exact count on a sparsified graph hit max_seconds");
    return late;
}

}  // namespace gpm

extern "C" gpm_status gpm_exact_count(gpm_graph *h, const gpm_pattern *pattern, uint64_t *out) {
    if (!h || !pattern || !out) {
        set_error("gpm_exact_count: null argument");
        return GPM_ERR_ARG;
    }
    Plan p;
    std::string why = build_plan(*pattern, &p);
    if (!why.empty()) {
        set_error("pattern rejected: " + why);
        return GPM_ERR_ARG;
    }
    return exact_count_plan(h, p, out, nullptr, 0.0);
}

extern "C" gpm_status gpm_gs_count_classes(gpm_graph *h, const gpm_pattern *pattern, uint32_t colors, uint64_t seed,
                                           uint32_t colouring, uint32_t slot, uint32_t rank, uint32_t world,
                                           double max_seconds, uint64_t *count) {
    if (!h || !pattern || !count || colors == 0 || world == 0 || rank >= world || h->d.n >= 0xFFFFFFFFull - colors) {
        set_error("gpm_gs_count_classes: null argument, zero colours or rank >= world");
        return GPM_ERR_ARG;
    }
    Plan p;
    std::string why = build_plan(*pattern, &p);
    if (!why.empty()) {
        set_error("pattern rejected: " + why);
        return GPM_ERR_ARG;
    }
    uint64_t *row = nullptr;
    uint32_t *col = nullptr;
    uint64_t kept = 0;
    gpm_status st = sparsify_alloc(h, colors, seed, colouring, slot, &row, &col, &kept, nullptr, nullptr, 0, rank, world);
    if (st != GPM_OK) return st;
    gpm_graph *gs = nullptr;
    st = gpm_load_csr(h->d.n, row, col, GPM_DEVICE_PTRS, h->stream, &gs);
    uint64_t cp = 0;
    if (st == GPM_OK) st = exact_count_plan(gs, p, &cp, nullptr, max_seconds);
    if (gs) gpm_free_graph(gs);
    cudaFree(row);
    cudaFree(col);
    *count = cp;
    return st;
}

extern "C" gpm_status gpm_sparsify_edges(gpm_graph *h, double p, uint64_t seed, uint32_t colouring, uint32_t slot,
                                         uint64_t *row_out, uint32_t *col_out, uint64_t *kept) {
    if (!h || !row_out || !col_out || !kept || !(p > 0.0) || bes_threshold(p) == 0) {
        set_error("gpm_sparsify_edges: null argument or p not in (2^-32, 1]");
        return GPM_ERR_ARG;
    }
    return sparsify_alloc(h, 1, seed, colouring, slot, nullptr, nullptr, kept, row_out, col_out, bes_threshold(p));
}

extern "C" gpm_status gpm_sparsify(gpm_graph *h, uint32_t colors, uint64_t seed, uint32_t colouring, uint32_t slot,
                                   uint64_t *row_out, uint32_t *col_out, uint64_t *kept) {
    if (!h || !row_out || !col_out || !kept || colors == 0) {
        set_error("gpm_sparsify: null argument or zero colours");
        return GPM_ERR_ARG;
    }
    return sparsify_alloc(h, colors, seed, colouring, slot, nullptr, nullptr, kept, row_out, col_out);
}
