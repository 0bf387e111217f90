// Random-sector gather roofline probe (measurement only; not on the
// estimator's path).  Every thread follows independent pointer chains through
// a buffer of random 64-bit words: each hop reads the first word of one
// 32-byte sector at a random position, and the next position is computed from
// the word just read, so the hops of a chain are dependent loads, as the
// sampler's are (edge -> row offsets -> neighbour lists).  Throughput is
// counted in 32-byte sectors, the unit of the sampler's algorithmic bytes.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>

#include "device.cuh"
#include "internal.h"

namespace gpm {

__global__ void probe_fill(uint64_t *buf, uint64_t words, uint64_t seed) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words; i += stride) {
        const Philox4 o = philox10((uint32_t)i, (uint32_t)(i >> 32), 0u, 7u, (uint32_t)seed, (uint32_t)(seed >> 32));
        buf[i] = ((uint64_t)o.y << 32) | o.x;
    }
}

__global__ void __launch_bounds__(256) probe_chase(const uint64_t *__restrict__ buf, uint64_t sectors, uint32_t chain,
                                                   uint32_t chains, uint64_t seed, unsigned long long *sink) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t acc = 0;
    for (uint32_t c = 0; c < chains; c++) {
        const Philox4 o = philox10((uint32_t)tid, (uint32_t)(tid >> 32), c, 8u, (uint32_t)seed, (uint32_t)(seed >> 32));
        uint64_t s = index_map(((uint64_t)o.y << 32) | o.x, sectors);
        for (uint32_t h = 0; h < chain; h++) {
            const uint64_t v = __ldg(buf + 4 * s);
            acc ^= v;
            s = index_map(v * 0x9E3779B97F4A7C15ull + h, sectors);
        }
    }
    if (acc == 0x5DEECE66Dull) atomicAdd(sink, 1ull);   // keeps the loads live
}

}  // namespace gpm

using namespace gpm;

extern "C" gpm_status gpm_gather_probe(uint64_t bytes, uint32_t chain, uint64_t hops, double *sectors_bytes_per_s) {
    if (!sectors_bytes_per_s || bytes < 4096 || chain == 0 || chain > 64 || hops == 0) {
        set_error("gpm_gather_probe: bytes >= 4096, 1 <= chain <= 64 and hops > 0 are required");
        return GPM_ERR_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        set_error("gpm_gather_probe: no CUDA device");
        return GPM_ERR_CUDA;
    }
    cudaStream_t st = nullptr;
    uint64_t *buf = nullptr;
    unsigned long long *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const uint64_t words = bytes / 8, sectors = bytes / 32;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = pool_alloc((void **)&buf, words * 8, st);
    if (e == cudaSuccess) e = pool_alloc((void **)&sink, sizeof(*sink), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned blocks = (unsigned)sms * 8u;
    const uint64_t threads = (uint64_t)blocks * 256;
    uint64_t chains = (hops + threads * chain - 1) / (threads * chain);
    if (chains == 0) chains = 1;
    float ms = 0.f;
    if (e == cudaSuccess) {
        probe_fill<<<blocks, 256, 0, st>>>(buf, words, 12345);
        e = cudaMemsetAsync(sink, 0, sizeof(*sink), st);
    }
    if (e == cudaSuccess) {
        probe_chase<<<blocks, 256, 0, st>>>(buf, sectors, chain, (uint32_t)chains, 1, sink);   // warm-up
        cudaEventRecord(e0, st);
        probe_chase<<<blocks, 256, 0, st>>>(buf, sectors, chain, (uint32_t)chains, 2, sink);
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    pool_free(buf, st);
    pool_free(sink, st);
    if (st) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        set_error(std::string("gpm_gather_probe: ") + cudaGetErrorString(e));
        return GPM_ERR_CUDA;
    }
    const double total = (double)threads * (double)chains * (double)chain;
    *sectors_bytes_per_s = total * 32.0 / (ms * 1e-3);
    return GPM_OK;
}
