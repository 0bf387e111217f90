// Graph residency: load a CSR into HBM, validate it on the device, and build
// the oriented-edge index used to draw the first edge of a sample.
//
// The paper stores the data graph as a symmetric CSR without loops or
// duplicate edges (Sec. 6, Table tab:input caption).  For patterns whose first
// two vertices carry a restriction v_0 < v_1 the first edge is drawn from the
// m oriented edges (u < w), enumerated u ascending, then N+(u) ascending; this
// needs up[v] (first neighbour above v) and uoff[v] = sum_{u<v} |N+(u)|.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "device.cuh"
#include "internal.h"

namespace gpm {

static cudaMemPool_t g_pools[64];
static std::once_flag g_pool_once[64];

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
    std::call_once(g_pool_once[dev], [dev]() {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    });
    e = g_pools[dev] ? cudaMallocFromPoolAsync(p, bytes, g_pools[dev], st) : cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        // a refused allocation must not surface later as a launch error
        cudaGetLastError();
        *p = nullptr;
    }
    return e;
}

void pool_free(void *p, cudaStream_t st) {
    if (!p) return;
    // a stream the caller has destroyed cannot order the free: free synchronously
    if (cudaFreeAsync(p, st) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
    }
}

thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

#define GPM_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t err_ = (call);                                                           \
        if (err_ != cudaSuccess) {                                                           \
            set_error(std::string(#call) + ": " + cudaGetErrorString(err_));                 \
            return GPM_ERR_CUDA;                                                             \
        }                                                                                    \
    } while (0)

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of n uint64 values into out[0..n] (out[n] = total).
// Three phases per level: block-local scans of 8192 items, a scan of the
// block totals (recursively), and the block offsets added back.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *warp_tot, uint64_t *total) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t t = __shfl_up_sync(kFull, inc, d);
        if (lane >= (unsigned)d) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint64_t wv = warp_tot[lane];
        uint64_t wi = wv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t t = __shfl_up_sync(kFull, wi, d);
            if (lane >= (unsigned)d) wi += t;
        }
        warp_tot[lane] = wi - wv;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    return inc - v + warp_tot[warp];
}

__global__ void scan_tiles(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *tile_sums) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t total;
    const uint64_t base = blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t local[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        uint64_t idx = base + i;
        local[i] = idx < n ? in[idx] : 0;
        s += local[i];
    }
    uint64_t off = block_exclusive_scan(s, warp_tot, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        uint64_t idx = base + i;
        if (idx < n) out[idx] = off;
        off += local[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void scan_add(uint64_t *out, uint64_t n, const uint64_t *tile_offsets) {
    const uint64_t t = blockIdx.x;
    const uint64_t base = t * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    const uint64_t add = tile_offsets[t];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        uint64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

// out must hold n + 1 values; scratch is allocated per level.
cudaError_t scan_exclusive_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t st) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    uint64_t *sums = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sums, sizeof(uint64_t) * (tiles + 1), st);
    if (e != cudaSuccess) return e;
    scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, sums);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        if (tiles > 1) {
            // sums -> exclusive offsets in place via a second buffer
            uint64_t *offs = nullptr;
            e = cudaMallocAsync((void **)&offs, sizeof(uint64_t) * (tiles + 1), st);
            if (e == cudaSuccess) {
                e = scan_exclusive_u64(sums, offs, tiles, st);
                if (e == cudaSuccess) {
                    scan_add<<<(unsigned)tiles, kScanThreads, 0, st>>>(out, n, offs);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(out + n, offs + tiles, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
                cudaFreeAsync(offs, st);
            }
        } else {
            e = cudaMemcpyAsync(out + n, sums, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
        }
    }
    cudaFreeAsync(sums, st);
    return e;
}

// ------------------------------------------------------------------ index
// Per vertex: up[v] (first neighbour above v, found by binary search in the
// sorted list) and |N+(v)|; one thread per vertex.
__global__ void upper_index(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col, uint64_t n,
                            uint64_t *up, uint64_t *cnt) {
    const uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint64_t lo = row_ptr[v], hi = row_ptr[v + 1];
    const uint64_t end = hi;
    while (lo < hi) {
        uint64_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] <= (uint32_t)v) lo = mid + 1;
        else hi = mid;
    }
    up[v] = lo;
    cnt[v] = end - lo;
}

// Oriented edge e (canonical order: u ascending, then N+(u) ascending) stored
// as (w << 32 | u), so a sample reads its first edge with one 8-byte load.
__global__ void oriented_edges(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                               const uint64_t *__restrict__ up, const uint64_t *__restrict__ uoff, uint64_t n,
                               uint64_t *edges) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = warp; u < n; u += nw) {
        const uint64_t b = up[u], e = row_ptr[u + 1], o = uoff[u];
        for (uint64_t i = b + lane; i < e; i += 32) edges[o + (i - b)] = ((uint64_t)col[i] << 32) | u;
    }
}

__global__ void max_degree_kernel(const uint64_t *__restrict__ row_ptr, uint64_t n, unsigned long long *out) {
    uint64_t best = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t d = row_ptr[v + 1] - row_ptr[v];
        best = d > best ? d : best;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        uint64_t t = __shfl_xor_sync(kFull, best, o);
        best = t > best ? t : best;
    }
    if ((threadIdx.x & 31u) == 0) atomicMax(out, (unsigned long long)best);
}

// Validation, one warp per vertex: offsets monotone, ids in range, no self
// loop, strictly ascending (sorted and duplicate-free), symmetric.
// bad[0] receives the smallest failing code (1 offsets, 2 range, 3 loop,
// 4 order, 5 symmetry) through atomicMin (initialised to 0xFF).
__global__ void validate_kernel(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col, uint64_t n,
                                unsigned int *bad) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nnz = row_ptr[n];
    for (uint64_t v = warp; v < n; v += nw) {
        const uint64_t b = row_ptr[v], e = row_ptr[v + 1];
        if (e < b || e > nnz) {
            if (lane == 0) atomicMin(bad, 1u);
            continue;
        }
        for (uint64_t i = b + lane; i < e; i += 32) {
            const uint32_t x = col[i];
            unsigned code = 0;
            if ((uint64_t)x >= n) code = 2;
            else if (x == (uint32_t)v) code = 3;
            else if (i > b && col[i - 1] >= x) code = 4;
            else {
                uint64_t lo = row_ptr[x], hi = row_ptr[x + 1];
                if (hi < lo || hi > nnz) code = 1;
                else {
                    while (lo < hi) {
                        uint64_t mid = lo + ((hi - lo) >> 1);
                        if (col[mid] < (uint32_t)v) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo >= row_ptr[x + 1] || col[lo] != (uint32_t)v) code = 5;
                }
            }
            if (code) atomicMin(bad, code);
        }
    }
}

}  // namespace gpm

using namespace gpm;

static const char *kValidateMsg[] = {"", "row offsets are not monotone or exceed nnz", "a neighbour id is >= n",
                                     "a vertex lists itself (self loop)",
                                     "a neighbour list is unsorted or has a duplicate",
                                     "the graph is not symmetric"};

extern "C" gpm_status gpm_load_csr(uint64_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t flags,
                                   void *stream, gpm_graph **out) {
    if (!out || !row_ptr || (n > 0 && !col && !(flags & GPM_DEVICE_PTRS))) {
        set_error("gpm_load_csr: null argument");
        return GPM_ERR_ARG;
    }
    if (n >= 0xFFFFFFFFull) {
        set_error("gpm_load_csr: n must be below 2^32 - 1");
        return GPM_ERR_ARG;
    }
    *out = nullptr;
    gpm_graph *g = new (std::nothrow) gpm_graph;
    if (!g) return GPM_ERR_OOM;
    std::memset(g, 0, sizeof(*g));
    g->totals_host = g->totals_buf;
    g->stream = (cudaStream_t)stream;
    cudaStream_t st = g->stream;
    auto fail = [&](gpm_status s) {
        gpm_free_graph(g);
        return s;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
        set_error("gpm_load_csr: no CUDA device");
        return fail(GPM_ERR_CUDA);
    }
    uint64_t nnz = 0;
    if (flags & GPM_DEVICE_PTRS) {
        if (cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("gpm_load_csr: cannot read row_ptr[n] from the device");
            return fail(GPM_ERR_CUDA);
        }
        g->d.row_ptr = row_ptr;
        g->d.col = col;
    } else {
        nnz = row_ptr[n];
        if (pool_alloc((void **)&g->own_row_ptr, sizeof(uint64_t) * (n + 1), st) != cudaSuccess ||
            pool_alloc((void **)&g->own_col, sizeof(uint32_t) * (nnz ? nnz : 1), st) != cudaSuccess) {
            set_error("gpm_load_csr: device allocation failed");
            return fail(GPM_ERR_OOM);
        }
        if (cudaMemcpyAsync(g->own_row_ptr, row_ptr, sizeof(uint64_t) * (n + 1), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            (nnz && cudaMemcpyAsync(g->own_col, col, sizeof(uint32_t) * nnz, cudaMemcpyHostToDevice, st) !=
                        cudaSuccess)) {
            set_error("gpm_load_csr: host to device copy failed");
            return fail(GPM_ERR_CUDA);
        }
        g->d.row_ptr = g->own_row_ptr;
        g->d.col = g->own_col;
    }
    g->d.n = n;
    g->d.nnz = nnz;
    if (pool_alloc((void **)&g->up, sizeof(uint64_t) * (n + 1), st) != cudaSuccess ||
        pool_alloc((void **)&g->uoff, sizeof(uint64_t) * (n + 1), st) != cudaSuccess ||
        pool_alloc((void **)&g->totals, sizeof(Totals) * 2, st) != cudaSuccess ||
        pool_alloc((void **)&g->counter, sizeof(unsigned int) * 64, st) != cudaSuccess) {
        set_error("gpm_load_csr: device allocation failed");
        return fail(GPM_ERR_OOM);
    }
    if (cudaEventCreate(&g->ev0) != cudaSuccess || cudaEventCreate(&g->ev1) != cudaSuccess) {
        set_error("gpm_load_csr: event creation failed");
        return fail(GPM_ERR_CUDA);
    }
    unsigned int *bad = nullptr;
    unsigned long long *maxd = nullptr;
    if (pool_alloc((void **)&bad, sizeof(unsigned int), st) != cudaSuccess ||
        pool_alloc((void **)&maxd, sizeof(unsigned long long), st) != cudaSuccess) {
        pool_free(bad, st);
        set_error("gpm_load_csr: device allocation failed");
        return fail(GPM_ERR_OOM);
    }
    unsigned int bad_h = 0xFF;
    unsigned long long maxd_h = 0;
    cudaError_t e = cudaMemcpyAsync(bad, &bad_h, sizeof(bad_h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(maxd, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && n > 0 && (flags & GPM_VALIDATE)) {
        const uint64_t warps = n < (1ull << 22) ? n : (1ull << 22);
        validate_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(g->d.row_ptr, g->d.col, n, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(bad_h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && bad_h != 0xFF) {
        pool_free(bad, st);
        pool_free(maxd, st);
        set_error(std::string("gpm_load_csr: invalid CSR: ") + kValidateMsg[bad_h < 6 ? bad_h : 0]);
        return fail(GPM_ERR_GRAPH);
    }
    if (e == cudaSuccess && (flags & GPM_RELABEL_DEGREE)) {
        uint64_t *nrp = nullptr;
        uint32_t *ncol = nullptr, *nid = nullptr;
        const gpm_status rs = relabel_by_degree(n, nnz, g->d.row_ptr, g->d.col, st, &nrp, &ncol, &nid);
        if (rs != GPM_OK) {
            pool_free(bad, st);
            pool_free(maxd, st);
            return fail(rs);
        }
        // the handle's own copy is replaced; a borrowed CSR stays the caller's
        pool_free(g->own_row_ptr, st);
        pool_free(g->own_col, st);
        g->own_row_ptr = nrp;
        g->own_col = ncol;
        g->d.row_ptr = nrp;
        g->d.col = ncol;
        g->newid = nid;
    }
    uint64_t *cnt = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cnt, sizeof(uint64_t) * (n + 1), st);
    if (e == cudaSuccess && n > 0) {
        upper_index<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g->d.row_ptr, g->d.col, n, g->up, cnt);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            max_degree_kernel<<<(unsigned)(g->sm_count * 8), 256, 0, st>>>(g->d.row_ptr, n, maxd);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = scan_exclusive_u64(cnt, g->uoff, n, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->up + n, g->d.row_ptr + n, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    uint64_t m = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, g->uoff + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&maxd_h, maxd, sizeof(maxd_h), cudaMemcpyDeviceToHost, st);
    if (cnt) cudaFreeAsync(cnt, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    pool_free(bad, st);
    pool_free(maxd, st);
    if (e != cudaSuccess) {
        set_error(std::string("gpm_load_csr: ") + cudaGetErrorString(e));
        return fail(GPM_ERR_CUDA);
    }
    g->d.up = g->up;
    g->d.uoff = g->uoff;
    g->d.m = m;
    g->max_degree = maxd_h;
    if (maxd_h >= (1ull << 31)) {
        // the sampler addresses entries inside one list with 32-bit offsets
        set_error("gpm_load_csr: a vertex of degree 2^31 or more is not supported");
        return fail(GPM_ERR_GRAPH);
    }
    // optional first-edge table; without memory for it the sampler searches uoff
    g->d.edges = nullptr;
    if (m > 0 && pool_alloc((void **)&g->edges, sizeof(uint64_t) * m, st) == cudaSuccess) {
        const uint64_t warps = n < (1ull << 22) ? n : (1ull << 22);
        oriented_edges<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(g->d.row_ptr, g->d.col, g->up, g->uoff,
                                                                             n, g->edges);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("gpm_load_csr: edge table: ") + cudaGetErrorString(e));
            return fail(GPM_ERR_CUDA);
        }
        g->d.edges = g->edges;
    } else {
        g->edges = nullptr;
        cudaGetLastError();
    }
    *out = g;
    return GPM_OK;
}

extern "C" void gpm_free_graph(gpm_graph *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    pool_free(g->own_row_ptr, g->stream);
    pool_free(g->own_col, g->stream);
    pool_free(g->up, g->stream);
    pool_free(g->uoff, g->stream);
    pool_free(g->edges, g->stream);
    pool_free(g->newid, g->stream);
    pool_free(g->partials, g->stream);
    pool_free(g->totals, g->stream);
    pool_free(g->counter, g->stream);
    g->totals_host = nullptr;
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

extern "C" gpm_status gpm_relabel_map(const gpm_graph *g, uint32_t *new_of_old) {
    if (!g || !new_of_old) {
        set_error("gpm_relabel_map: null argument");
        return GPM_ERR_ARG;
    }
    if (!g->newid) {
        set_error("gpm_relabel_map: the graph was loaded without GPM_RELABEL_DEGREE");
        return GPM_ERR_ARG;
    }
    if (g->d.n == 0) return GPM_OK;
    cudaError_t e = cudaMemcpyAsync(new_of_old, g->newid, sizeof(uint32_t) * g->d.n, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        set_error(std::string("gpm_relabel_map: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    return GPM_OK;
}

extern "C" gpm_status gpm_graph_info(const gpm_graph *g, uint64_t *n, uint64_t *m, uint64_t *nnz,
                                     uint64_t *max_degree) {
    if (!g) {
        set_error("gpm_graph_info: null handle");
        return GPM_ERR_ARG;
    }
    if (n) *n = g->d.n;
    if (m) *m = g->d.m;
    if (nnz) *nnz = g->d.nnz;
    if (max_degree) *max_degree = g->max_degree;
    return GPM_OK;
}

extern "C" gpm_status gpm_abort(gpm_graph *g) {
    if (!g) {
        set_error("gpm_abort: null handle");
        return GPM_ERR_ARG;
    }
    g->abort_flag = 1;
    return GPM_OK;
}

extern "C" const char *gpm_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *gpm_version(void) { return "gpm-gb300 0.1 (sm_103a)"; }
