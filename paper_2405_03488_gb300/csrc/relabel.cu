// Degree relabelling at load time (GPM_RELABEL_DEGREE).
//
// The paper orients clique searches (Table tab:input caption: "orientation is
// applied" for cliques; the ordering is not given).  This library reads that
// as relabelling vertices by (degree, id) ascending before sampling, so that
// the restriction v_0 < v_1 < ... points every oriented edge at the endpoint
// of higher degree.  Vertex v gets the new id rank(deg(v), v); the lists are
// rewritten in new ids and sorted.
//
// Both steps are sorts of 64-bit keys, done by a least-significant-digit radix
// sort written here: 8-bit digits; per pass one warp per tile of 2^16 keys
// counts its digits, an exclusive scan over (digit, tile) gives every tile's
// first slot per digit, and the tile scatters its keys in order (lanes with
// equal digits ranked by __match_any_sync), so each pass is stable.
#include <cuda_runtime.h>

#include <cstring>

#include "device.cuh"
#include "internal.h"

namespace gpm {

cudaError_t scan_exclusive_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t st);

constexpr uint64_t kSortTile = 1ull << 16;   // keys per warp and pass
constexpr int kSortWarps = 8;

__global__ void __launch_bounds__(32 * kSortWarps) radix_count(const uint64_t *__restrict__ keys, uint64_t n,
                                                                int shift, uint64_t ntiles, uint64_t *hist) {
    __shared__ unsigned int cnt[kSortWarps][256];
    const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t t = (uint64_t)blockIdx.x * kSortWarps + warp;
    for (int d = lane; d < 256; d += 32) cnt[warp][d] = 0;
    __syncwarp();
    if (t < ntiles) {
        const uint64_t b = t * kSortTile, e = (b + kSortTile < n) ? b + kSortTile : n;
        for (uint64_t i = b + lane; i < e; i += 32) atomicAdd(&cnt[warp][(keys[i] >> shift) & 255u], 1u);
        __syncwarp();
        for (int d = lane; d < 256; d += 32) hist[(uint64_t)d * ntiles + t] = cnt[warp][d];
    }
}

__global__ void __launch_bounds__(32 * kSortWarps) radix_scatter(const uint64_t *__restrict__ in, uint64_t *out,
                                                                  uint64_t n, int shift, uint64_t ntiles,
                                                                  const uint64_t *__restrict__ offs) {
    __shared__ unsigned long long base[kSortWarps][256];
    const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t t = (uint64_t)blockIdx.x * kSortWarps + warp;
    if (t >= ntiles) return;
    for (int d = lane; d < 256; d += 32) base[warp][d] = offs[(uint64_t)d * ntiles + t];
    __syncwarp();
    const uint64_t b = t * kSortTile, e = (b + kSortTile < n) ? b + kSortTile : n;
    for (uint64_t i0 = b; i0 < e; i0 += 32) {
        const uint64_t i = i0 + lane;
        const bool valid = i < e;
        const uint64_t key = valid ? in[i] : 0;
        const unsigned d = valid ? (unsigned)((key >> shift) & 255u) : 256u + lane;   // past-the-end lanes alone
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        const unsigned long long pos = valid ? base[warp][d] : 0ull;
        __syncwarp();
        if (valid) {
            out[pos + rank] = key;
            if ((int)lane == __ffs(peers) - 1) base[warp][d] = pos + __popc(peers);
        }
        __syncwarp();
    }
}

// Sorts keys[0, n) by their low `bits` bits (stable); tmp holds n keys.  The
// result ends in *result (keys or tmp).
static cudaError_t radix_sort_u64(uint64_t *keys, uint64_t *tmp, uint64_t n, int bits, cudaStream_t st,
                                  uint64_t **result) {
    *result = keys;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
    uint64_t *hist = nullptr, *offs = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&hist, sizeof(uint64_t) * 256 * ntiles, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&offs, sizeof(uint64_t) * (256 * ntiles + 1), st);
    uint64_t *src = keys, *dst = tmp;
    const unsigned blocks = (unsigned)((ntiles + kSortWarps - 1) / kSortWarps);
    for (int shift = 0; shift < bits && e == cudaSuccess; shift += 8) {
        radix_count<<<blocks, 32 * kSortWarps, 0, st>>>(src, n, shift, ntiles, hist);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = scan_exclusive_u64(hist, offs, 256 * ntiles, st);
        if (e == cudaSuccess) {
            radix_scatter<<<blocks, 32 * kSortWarps, 0, st>>>(src, dst, n, shift, ntiles, offs);
            e = cudaGetLastError();
        }
        uint64_t *x = src;
        src = dst;
        dst = x;
    }
    if (hist) cudaFreeAsync(hist, st);
    if (offs) cudaFreeAsync(offs, st);
    *result = src;
    return e;
}

__global__ void degree_keys(const uint64_t *__restrict__ row_ptr, uint64_t n, uint64_t *keys) {
    const uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v < n) keys[v] = ((row_ptr[v + 1] - row_ptr[v]) << 32) | v;
}

// new id of every old vertex, and the degrees in new order
__global__ void ranks_from_keys(const uint64_t *__restrict__ sorted, uint64_t n, uint32_t *newid, uint64_t *ndeg) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        newid[(uint32_t)sorted[i]] = (uint32_t)i;
        ndeg[i] = sorted[i] >> 32;
    }
}

// one warp per old vertex: every entry (v, w) becomes the key newid[v] << B | newid[w]
__global__ void edge_keys(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col, uint64_t n,
                          const uint32_t *__restrict__ newid, int B, uint64_t *keys) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    for (uint64_t v = warp; v < n; v += nw) {
        const uint64_t hi = (uint64_t)newid[v] << B;
        for (uint64_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) keys[e] = hi | newid[col[e]];
    }
}

__global__ void low_bits(const uint64_t *__restrict__ keys, uint64_t nnz, int B, uint32_t *col) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < nnz) col[i] = (uint32_t)(keys[i] & ((1ull << B) - 1ull));
}

static int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

// Relabels the device CSR (row_ptr, col) into freshly allocated row_out (n + 1),
// col_out (nnz) and newid (n): new id = rank of (degree, id).
gpm_status relabel_by_degree(uint64_t n, uint64_t nnz, const uint64_t *row_ptr, const uint32_t *col,
                             cudaStream_t st, uint64_t **row_out, uint32_t **col_out, uint32_t **newid_out) {
    *row_out = nullptr;
    *col_out = nullptr;
    *newid_out = nullptr;
    uint64_t *ka = nullptr, *kb = nullptr, *ndeg = nullptr, *rp = nullptr;
    uint32_t *newid = nullptr, *cc = nullptr;
    const uint64_t big = n > nnz ? n : nnz;
    cudaError_t e = cudaMallocAsync((void **)&ka, sizeof(uint64_t) * (big ? big : 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&kb, sizeof(uint64_t) * (big ? big : 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&ndeg, sizeof(uint64_t) * (n ? n : 1), st);
    if (e == cudaSuccess) e = pool_alloc((void **)&rp, sizeof(uint64_t) * (n + 1), st);
    if (e == cudaSuccess) e = pool_alloc((void **)&newid, sizeof(uint32_t) * (n ? n : 1), st);
    if (e == cudaSuccess) e = pool_alloc((void **)&cc, sizeof(uint32_t) * (nnz ? nnz : 1), st);
    uint64_t *sorted = nullptr;
    if (e == cudaSuccess && n) {
        degree_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(row_ptr, n, ka);
        e = cudaGetLastError();
        // degrees are below n
        if (e == cudaSuccess) e = radix_sort_u64(ka, kb, n, 32 + bit_length(n), st, &sorted);
        if (e == cudaSuccess) {
            ranks_from_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sorted, n, newid, ndeg);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = scan_exclusive_u64(ndeg, rp, n, st);
    const int B = bit_length(n ? n - 1 : 0) > 0 ? bit_length(n - 1) : 1;
    if (e == cudaSuccess && nnz) {
        edge_keys<<<(unsigned)((n * 32 + 255) / 256 < (1u << 20) ? (n * 32 + 255) / 256 : (1u << 20)), 256, 0, st>>>(
            row_ptr, col, n, newid, B, ka);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = radix_sort_u64(ka, kb, nnz, 2 * B, st, &sorted);
        if (e == cudaSuccess) {
            low_bits<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(sorted, nnz, B, cc);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ka) cudaFreeAsync(ka, st);
    if (kb) cudaFreeAsync(kb, st);
    if (ndeg) cudaFreeAsync(ndeg, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        pool_free(rp, st);
        pool_free(newid, st);
        pool_free(cc, st);
        set_error(std::string("relabel by degree: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GPM_ERR_OOM : GPM_ERR_CUDA;
    }
    *row_out = rp;
    *col_out = cc;
    *newid_out = newid;
    return GPM_OK;
}

}  // namespace gpm
