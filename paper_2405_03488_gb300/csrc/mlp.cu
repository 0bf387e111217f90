// Learned proposal: scoring, training data from plain-NS traces, and training.
//
// The proposal (not in the paper) scores each candidate x of a step j <= k-2
// with a 3 -> 64 -> 64 -> 1 ReLU MLP on (log2(1 + d(x)), j, log2(1 +
// |S_{j+1}(x)|)); the sampler draws x with probability a_x / A and weighs
// A / a_x, so Lemma 1's argument (each match's probability is the inverse of
// its weight) still gives an unbiased estimator.
//
// Training rows come from the plain sampler's records: at every step j <= k-2
// a sample passed, the chosen vertex vert[j] with its degree, j and the size
// of the next candidate set factor[j+1] (exactly the lookahead feature), and
// the progress label (d - j - 1) / (k - j - 1), d the depth the sample reached
// (k on a hit): 1 on a hit, 0 when the next step found no candidate, so rare
// hits still leave a dense signal.  The loss is binary cross-entropy on the
// logit z, averaged over rows; the trainer keeps FP32 master weights, updates
// them with Adam, and exports BF16 copies (round to nearest even) for the
// sampler.  Forward and backward run on 64-row tiles: per tile the block forms
// H1 = relu(X W1^T + b1) and A2 = H1 W2^T + b2 in shared memory, the output
// and its gradient per row, and accumulates the weight gradients as small
// tile contractions; per-block partials are summed in block order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "sampler.cuh"

namespace gpm {

cudaError_t scan_exclusive_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t st);
gpm_status trace_device(gpm_graph *h, const Plan &p, uint64_t seed, uint64_t first, uint64_t count,
                        const gpm_config *cfg, gpm_sample_record *d_out);

// offsets of the parameter blocks in the 4481-float layout
constexpr int kW1 = 0, kB1 = 192, kW2 = 256, kB2 = 4352, kW3 = 4416, kB3 = 4480;

// ------------------------------------------------------------------ scoring
__global__ void __launch_bounds__(256) mlp_score_kernel(const gpm_mlp mlp, const float *__restrict__ feat,
                                                        uint64_t n, uint32_t *out) {
    extern __shared__ __align__(16) uint64_t smem64[];
    WarpMem wm = warp_mem<MODE_LEARNED>(smem64, 0, mlp);
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    // one row per thread (the sampler scores one candidate per lane the same way)
    for (uint64_t r = t0; r < n; r += nt) out[r] = mlp_score_lane(wm.W, feat[3 * r], feat[3 * r + 1], feat[3 * r + 2]);
}

// Scores on the tensor cores, 16 rows per warp and tile (the sampler's
// tensor-core scoring, mlp_scores_tc).
__global__ void __launch_bounds__(256) mlp_score_tc_kernel(const gpm_mlp mlp, const float *__restrict__ feat,
                                                           uint64_t n, uint32_t *out) {
    extern __shared__ __align__(16) uint64_t smem64[];
    WarpMem wm = warp_mem<MODE_LEARNED>(smem64, 0, mlp);
    const unsigned lane = lane_id();
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * 16; base < n; base += nw * 16) {
        const uint32_t cnt = (n - base < 16) ? (uint32_t)(n - base) : 16u;
        auto f = [&](uint32_t c, float *f0, float *f1, float *f2) {
            *f0 = feat[3 * (base + c)];
            *f1 = feat[3 * (base + c) + 1];
            *f2 = feat[3 * (base + c) + 2];
        };
        mlp_scores_tc(wm, cnt, f, wm.score);
        if (lane < cnt) out[base + lane] = wm.score[lane];
        __syncwarp();
    }
}

// ------------------------------------------------------------------ features
// rows per record: steps 2 <= j <= k-2 that the sample passed
__global__ void feature_count(const gpm_sample_record *__restrict__ recs, uint64_t n, int k, uint64_t *cnt) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const gpm_sample_record &r = recs[i];
    uint64_t c = 0;
    for (int j = 2; j <= k - 2; j++)
        if (r.hit || r.depth > j) c++;
    cnt[i] = c;
}

__global__ void feature_write(const DGraph g, const gpm_sample_record *__restrict__ recs, uint64_t n, int k,
                              const uint64_t *__restrict__ off, float *feat, float *label) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const gpm_sample_record &r = recs[i];
    uint64_t o = off[i];
    for (int j = 2; j <= k - 2; j++) {
        if (!(r.hit || r.depth > j)) continue;
        const uint32_t x = r.vert[j];
        const uint64_t d = g.row_ptr[x + 1] - g.row_ptr[x];
        feat[3 * o] = flog2p1(d);
        feat[3 * o + 1] = __int2float_rn(j);
        feat[3 * o + 2] = flog2p1(r.factor[j + 1]);
        // progress label: the share of the remaining steps j+1 .. k-1 the
        // sample survived (1 on a hit, 0 when it missed at step j+1)
        const int reached = r.hit ? k : (int)r.depth;
        label[o] = __fdiv_rn(__int2float_rn(reached - j - 1), __int2float_rn(k - j - 1));
        o++;
    }
}

// ------------------------------------------------------------------ forward / backward
constexpr int kTile = 64;
constexpr int kGradFloats = 4481;

// Per block: rows [row0 + blockIdx.x * rows_per_block, ...) of the batch; the
// block's gradient partial (scaled by 1 / total) goes to part[blockIdx.x].
__global__ void __launch_bounds__(256) mlp_fwd_bwd(const float *__restrict__ w, const float *__restrict__ feat,
                                                   const float *__restrict__ label, uint64_t row0, uint64_t rows,
                                                   uint32_t rows_per_block, double inv_total, float *part,
                                                   double *loss_part) {
    extern __shared__ float sW[];   // kGradFloats weights
    __shared__ float sX[kTile * 3], sY[kTile], sDz[kTile];
    __shared__ float sH1[kTile][65];
    __shared__ float sA2[kTile][65];
    __shared__ float gw1[192], gb1[64], gb2[64], gw3[64], gb3s;
    __shared__ double sLoss[256];
    const int t = threadIdx.x;
    for (int i = t; i < kGradFloats; i += 256) sW[i] = w[i];
    for (int i = t; i < 192; i += 256) gw1[i] = 0.f;
    if (t < 64) {
        gb1[t] = 0.f;
        gb2[t] = 0.f;
        gw3[t] = 0.f;
    }
    if (t == 0) gb3s = 0.f;
    // gW2 entries owned by this thread: o = t / 4, inputs i = (t % 4) * 16 .. + 16
    float gw2[16];
#pragma unroll
    for (int q = 0; q < 16; q++) gw2[q] = 0.f;
    double loss = 0.0;
    __syncthreads();
    const uint64_t b0 = row0 + (uint64_t)blockIdx.x * rows_per_block;
    const uint64_t b1 = (b0 + rows_per_block < row0 + rows) ? b0 + rows_per_block : row0 + rows;
    for (uint64_t base = b0; base < b1; base += kTile) {
        const int nr = (int)((b1 - base) < (uint64_t)kTile ? (b1 - base) : kTile);
        for (int i = t; i < kTile * 3; i += 256) sX[i] = (i < nr * 3) ? feat[3 * base + i] : 0.f;
        if (t < kTile) sY[t] = (t < nr) ? label[base + t] : 0.f;
        __syncthreads();
        // H1 = relu(X W1^T + b1): thread t -> row t/4, units (t%4)*16 ..
        {
            const int r = t >> 2, o0 = (t & 3) * 16;
            for (int o = o0; o < o0 + 16; o++) {
                float acc = sW[kB1 + o];
                acc = fmaf(sW[kW1 + o * 3 + 0], sX[r * 3 + 0], acc);
                acc = fmaf(sW[kW1 + o * 3 + 1], sX[r * 3 + 1], acc);
                acc = fmaf(sW[kW1 + o * 3 + 2], sX[r * 3 + 2], acc);
                sH1[r][o] = acc > 0.f ? acc : 0.f;
            }
        }
        __syncthreads();
        // A2 = H1 W2^T + b2
        {
            const int r = t >> 2, o0 = (t & 3) * 16;
            for (int o = o0; o < o0 + 16; o++) {
                float acc = sW[kB2 + o];
                for (int i = 0; i < 64; i++) acc = fmaf(sW[kW2 + o * 64 + i], sH1[r][i], acc);
                sA2[r][o] = acc;
            }
        }
        __syncthreads();
        // z and dz per row (warp w: rows w, w+8, ...)
        {
            const int wp = t >> 5, ln = t & 31;
            for (int r = wp; r < kTile; r += 8) {
                const float h_a = sA2[r][ln] > 0.f ? sA2[r][ln] : 0.f;
                const float h_b = sA2[r][ln + 32] > 0.f ? sA2[r][ln + 32] : 0.f;
                float part_z = sW[kW3 + ln] * h_a + sW[kW3 + ln + 32] * h_b;
#pragma unroll
                for (int o = 16; o; o >>= 1) part_z += __shfl_xor_sync(kFull, part_z, o);
                if (ln == 0) {
                    const float z = part_z + sW[kB3];
                    if (r < nr) {
                        const double zd = z, y = sY[r];
                        loss += (zd > 0 ? zd : 0.0) - y * zd + log1p(exp(-fabs(zd)));
                        sDz[r] = (float)((1.0 / (1.0 + exp(-zd)) - y) * inv_total);
                    } else {
                        sDz[r] = 0.f;
                    }
                }
            }
        }
        __syncthreads();
        // output layer gradients and DA2 = (dz w3) * [A2 > 0] (in place of A2)
        if (t < 64) {
            float g3 = 0.f;
            for (int r = 0; r < kTile; r++) {
                const float h = sA2[r][t] > 0.f ? sA2[r][t] : 0.f;
                g3 = fmaf(sDz[r], h, g3);
            }
            gw3[t] += g3;
        }
        if (t == 64) {
            float gz = 0.f;
            for (int r = 0; r < kTile; r++) gz += sDz[r];
            gb3s += gz;
        }
        __syncthreads();
        {
            const int r = t >> 2, o0 = (t & 3) * 16;
            for (int o = o0; o < o0 + 16; o++) sA2[r][o] = sA2[r][o] > 0.f ? sDz[r] * sW[kW3 + o] : 0.f;
        }
        __syncthreads();
        // gW2[o][i] += sum_r DA2[r][o] H1[r][i]; gb2[o] += sum_r DA2[r][o]
        {
            const int o = t >> 2, i0 = (t & 3) * 16;
            for (int r = 0; r < kTile; r++) {
                const float d = sA2[r][o];
#pragma unroll
                for (int q = 0; q < 16; q++) gw2[q] = fmaf(d, sH1[r][i0 + q], gw2[q]);
            }
            if ((t & 3) == 0) {
                float s = 0.f;
                for (int r = 0; r < kTile; r++) s += sA2[r][o];
                gb2[o] += s;
            }
        }
        __syncthreads();
        // DA1 = (DA2 W2) * [H1 > 0], written over H1 after every thread has read it
        float da1[16];
        {
            const int r = t >> 2, i0 = (t & 3) * 16;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const int i = i0 + q;
                float acc = 0.f;
                for (int o = 0; o < 64; o++) acc = fmaf(sA2[r][o], sW[kW2 + o * 64 + i], acc);
                da1[q] = sH1[r][i] > 0.f ? acc : 0.f;
            }
        }
        __syncthreads();
        {
            const int r = t >> 2, i0 = (t & 3) * 16;
#pragma unroll
            for (int q = 0; q < 16; q++) sH1[r][i0 + q] = da1[q];
        }
        __syncthreads();
        // gW1[o][i] += sum_r DA1[r][o] X[r][i]; gb1[o] += sum_r DA1[r][o]
        if (t < 64) {
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, gb = 0.f;
            for (int r = 0; r < kTile; r++) {
                const float d = sH1[r][t];
                g0 = fmaf(d, sX[r * 3 + 0], g0);
                g1 = fmaf(d, sX[r * 3 + 1], g1);
                g2 = fmaf(d, sX[r * 3 + 2], g2);
                gb += d;
            }
            gw1[t * 3 + 0] += g0;
            gw1[t * 3 + 1] += g1;
            gw1[t * 3 + 2] += g2;
            gb1[t] += gb;
        }
        __syncthreads();
    }
    float *out = part + (uint64_t)blockIdx.x * kGradFloats;
    {
        const int o = t >> 2, i0 = (t & 3) * 16;
#pragma unroll
        for (int q = 0; q < 16; q++) out[kW2 + o * 64 + i0 + q] = gw2[q];
    }
    for (int i = t; i < 192; i += 256) out[kW1 + i] = gw1[i];
    if (t < 64) {
        out[kB1 + t] = gb1[t];
        out[kB2 + t] = gb2[t];
        out[kW3 + t] = gw3[t];
    }
    if (t == 0) out[kB3] = gb3s;
    sLoss[t] = loss;
    __syncthreads();
    for (int hh = 128; hh; hh >>= 1) {
        if (t < hh) sLoss[t] += sLoss[t + hh];
        __syncthreads();
    }
    if (t == 0) loss_part[blockIdx.x] = sLoss[0];
}

// grad[i] = sum over blocks (block order) of part[b][i]
__global__ void grad_reduce(const float *__restrict__ part, uint32_t blocks, float *grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kGradFloats) return;
    float s = 0.f;
    for (uint32_t b = 0; b < blocks; b++) s += part[(uint64_t)b * kGradFloats + i];
    grad[i] = s;
}

__global__ void loss_reduce(const double *__restrict__ lp, uint32_t blocks, double inv_total, double *loss) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (uint32_t b = 0; b < blocks; b++) s += lp[b];
    *loss = s * inv_total;
}

// Adam (Kingma & Ba) with bias correction, then the BF16 copy (round to
// nearest even on the bit pattern).
__global__ void adam_step(float *w, const float *__restrict__ g, float *m, float *v, float lr, float b1, float b2,
                          float epsa, float c1, float c2, uint16_t *w16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kGradFloats) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + epsa);
    w[i] = wi;
    w16[i] = __bfloat16_as_ushort(__float2bfloat16_rn(wi));   // nearest even; NaN stays NaN
}

__global__ void to_bf16(const float *__restrict__ w, uint16_t *w16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kGradFloats) return;
    w16[i] = __bfloat16_as_ushort(__float2bfloat16_rn(w[i]));
}

static gpm_status cuda_fail(const char *where, cudaError_t e) {
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return GPM_ERR_CUDA;
}

// loss and gradient of rows [0, rows) at weights w (device), into grad (device)
static gpm_status loss_grad(cudaStream_t st, int sms, const float *w, const float *feat, const float *label,
                            uint64_t row0, uint64_t rows, uint64_t total, float *grad, double *d_loss,
                            float **part, double **lpart, uint32_t *part_cap) {
    uint32_t rpb = 256;
    uint64_t blocks = (rows + rpb - 1) / rpb;
    const uint64_t max_blocks = (uint64_t)sms * 8;
    if (blocks > max_blocks) {
        rpb = (uint32_t)(((rows + max_blocks - 1) / max_blocks + kTile - 1) / kTile * kTile);
        blocks = (rows + rpb - 1) / rpb;
    }
    if (blocks == 0) blocks = 1;
    if (*part_cap < blocks) {
        cudaFree(*part);
        cudaFree(*lpart);
        *part = nullptr;
        *lpart = nullptr;
        if (cudaMalloc((void **)part, sizeof(float) * kGradFloats * blocks) != cudaSuccess ||
            cudaMalloc((void **)lpart, sizeof(double) * blocks) != cudaSuccess) {
            set_error("mlp: device allocation failed");
            return GPM_ERR_OOM;
        }
        *part_cap = (uint32_t)blocks;
    }
    const double inv = 1.0 / (double)total;
    cudaFuncSetAttribute(mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kGradFloats * sizeof(float)));
    mlp_fwd_bwd<<<(unsigned)blocks, 256, kGradFloats * sizeof(float), st>>>(w, feat, label, row0, rows, rpb, inv, *part, *lpart);
    grad_reduce<<<(kGradFloats + 255) / 256, 256, 0, st>>>(*part, (uint32_t)blocks, grad);
    loss_reduce<<<1, 32, 0, st>>>(*lpart, (uint32_t)blocks, inv, d_loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GPM_OK : cuda_fail("mlp forward/backward", e);
}

}  // namespace gpm

using namespace gpm;

namespace gpm {
// Scores of feature rows given on the host (a handful: the selector head).
gpm_status mlp_score_rows(gpm_graph *h, const gpm_mlp *mlp, const float *feat_host, uint64_t n, uint32_t *out_host) {
    float *f = nullptr;
    uint32_t *o = nullptr;
    if (cudaMalloc((void **)&f, sizeof(float) * 3 * n) != cudaSuccess ||
        cudaMalloc((void **)&o, sizeof(uint32_t) * n) != cudaSuccess) {
        cudaFree(f);
        set_error("selector: device allocation failed");
        return GPM_ERR_OOM;
    }
    gpm_status st = GPM_OK;
    cudaError_t e = cudaMemcpyAsync(f, feat_host, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) st = cuda_fail("selector", e);
    if (st == GPM_OK) st = gpm_mlp_scores(h, mlp, f, n, o);
    if (st == GPM_OK) {
        e = cudaMemcpyAsync(out_host, o, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail("selector", e);
    }
    cudaFree(f);
    cudaFree(o);
    return st;
}
}  // namespace gpm

extern "C" gpm_status gpm_mlp_scores(gpm_graph *h, const gpm_mlp *mlp, const float *feat, uint64_t n,
                                     uint32_t *out) {
    if (!h || !mlp || (n && (!feat || !out))) {
        set_error("gpm_mlp_scores: null argument");
        return GPM_ERR_ARG;
    }
    if (n == 0) return GPM_OK;
    const size_t smem = kMlpSmemFloats * sizeof(float) + 8 * (kWarpHeaderWords + kLearnedWarpWords) * 4;
    cudaFuncSetAttribute(mlp_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint64_t blocks = (n + 7) / 8;
    if (blocks > (uint64_t)h->sm_count * 16) blocks = (uint64_t)h->sm_count * 16;
    mlp_score_kernel<<<(unsigned)blocks, 256, smem, h->stream>>>(*mlp, feat, n, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? GPM_OK : cuda_fail("gpm_mlp_scores", e);
}

extern "C" gpm_status gpm_mlp_scores_tc(gpm_graph *h, const gpm_mlp *mlp, const float *feat, uint64_t n,
                                        uint32_t *out) {
    if (!h || !mlp || (n && (!feat || !out))) {
        set_error("gpm_mlp_scores_tc: null argument");
        return GPM_ERR_ARG;
    }
    if (n == 0) return GPM_OK;
    const size_t smem = kMlpSmemFloats * sizeof(float) + 8 * (kWarpHeaderWords + kLearnedWarpWords) * 4;
    cudaFuncSetAttribute(mlp_score_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint64_t blocks = (n + 127) / 128;
    if (blocks > (uint64_t)h->sm_count * 16) blocks = (uint64_t)h->sm_count * 16;
    mlp_score_tc_kernel<<<(unsigned)blocks, 256, smem, h->stream>>>(*mlp, feat, n, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? GPM_OK : cuda_fail("gpm_mlp_scores_tc", e);
}

extern "C" gpm_status gpm_mlp_loss_grad(gpm_graph *h, const float *w32, const float *feat, const float *label,
                                        uint64_t rows, float *grad, double *loss) {
    if (!h || !w32 || !grad || !loss || (rows && (!feat || !label))) {
        set_error("gpm_mlp_loss_grad: null argument");
        return GPM_ERR_ARG;
    }
    if (rows == 0) {
        set_error("gpm_mlp_loss_grad: no rows");
        return GPM_ERR_ARG;
    }
    float *part = nullptr;
    double *lpart = nullptr, *d_loss = nullptr;
    uint32_t cap = 0;
    if (cudaMalloc((void **)&d_loss, sizeof(double)) != cudaSuccess) {
        set_error("mlp: device allocation failed");
        return GPM_ERR_OOM;
    }
    gpm_status st = loss_grad(h->stream, h->sm_count, w32, feat, label, 0, rows, rows, grad, d_loss, &part, &lpart, &cap);
    if (st == GPM_OK) {
        cudaError_t e = cudaMemcpyAsync(loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail("gpm_mlp_loss_grad", e);
    }
    cudaFree(part);
    cudaFree(lpart);
    cudaFree(d_loss);
    return st;
}

extern "C" gpm_status gpm_proposal_features(gpm_graph *h, const gpm_pattern *pattern, const gpm_sample_record *recs,
                                            uint64_t n, float *feat, float *label, uint64_t *rows) {
    if (!h || !pattern || !rows || (n && (!recs || !feat || !label))) {
        set_error("gpm_proposal_features: null argument");
        return GPM_ERR_ARG;
    }
    Plan p;
    std::string why = build_plan(*pattern, &p);
    if (!why.empty()) {
        set_error("pattern rejected: " + why);
        return GPM_ERR_ARG;
    }
    *rows = 0;
    if (n == 0 || p.k < 4) return GPM_OK;
    uint64_t *cnt = nullptr, *off = nullptr;
    if (cudaMalloc((void **)&cnt, sizeof(uint64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc((void **)&off, sizeof(uint64_t) * (n + 1)) != cudaSuccess) {
        cudaFree(cnt);
        set_error("gpm_proposal_features: device allocation failed");
        return GPM_ERR_OOM;
    }
    const unsigned blocks = (unsigned)((n + 255) / 256);
    feature_count<<<blocks, 256, 0, h->stream>>>(recs, n, p.k, cnt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_exclusive_u64(cnt, off, n, h->stream);
    if (e == cudaSuccess) {
        feature_write<<<blocks, 256, 0, h->stream>>>(h->d, recs, n, p.k, off, feat, label);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(rows, off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(cnt);
    cudaFree(off);
    return e == cudaSuccess ? GPM_OK : cuda_fail("gpm_proposal_features", e);
}

namespace gpm {

// Adam over minibatches of `batch` rows for `epochs` passes, then the loss of
// the final weights over all rows and their BF16 copy.
static gpm_status train_rows(gpm_graph *h, const float *feat, const float *label, uint64_t rows, uint32_t epochs,
                             uint32_t batch, float lr, float *w32, uint16_t *w16, double *final_loss) {
    cudaStream_t st = h->stream;
    float *grad = nullptr, *m = nullptr, *v = nullptr, *part = nullptr;
    double *lpart = nullptr, *d_loss = nullptr;
    uint32_t cap = 0;
    auto cleanup = [&]() {
        cudaFree(grad);
        cudaFree(m);
        cudaFree(v);
        cudaFree(part);
        cudaFree(lpart);
        cudaFree(d_loss);
    };
    if (cudaMalloc((void **)&grad, sizeof(float) * kGradFloats) != cudaSuccess ||
        cudaMalloc((void **)&m, sizeof(float) * kGradFloats) != cudaSuccess ||
        cudaMalloc((void **)&v, sizeof(float) * kGradFloats) != cudaSuccess ||
        cudaMalloc((void **)&d_loss, sizeof(double)) != cudaSuccess) {
        cleanup();
        set_error("mlp training: device allocation failed");
        return GPM_ERR_OOM;
    }
    cudaMemsetAsync(m, 0, sizeof(float) * kGradFloats, st);
    cudaMemsetAsync(v, 0, sizeof(float) * kGradFloats, st);
    gpm_status s = GPM_OK;
    uint64_t step = 0;
    for (uint32_t ep = 0; ep < epochs && s == GPM_OK; ep++) {
        for (uint64_t r0 = 0; r0 < rows && s == GPM_OK; r0 += batch) {
            const uint64_t nr = (r0 + batch < rows) ? batch : rows - r0;
            s = loss_grad(st, h->sm_count, w32, feat, label, r0, nr, nr, grad, d_loss, &part, &lpart, &cap);
            if (s != GPM_OK) break;
            step++;
            const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
            adam_step<<<(kGradFloats + 255) / 256, 256, 0, st>>>(w32, grad, m, v, lr, 0.9f, 0.999f, 1e-8f, c1, c2, w16);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) s = cuda_fail("adam", e);
        }
    }
    if (s == GPM_OK) {
        s = loss_grad(st, h->sm_count, w32, feat, label, 0, rows, rows, grad, d_loss, &part, &lpart, &cap);
        to_bf16<<<(kGradFloats + 255) / 256, 256, 0, st>>>(w32, w16);
        double lh = 0.0;
        cudaError_t e = cudaMemcpyAsync(&lh, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess && s == GPM_OK) s = cuda_fail("mlp training", e);
        if (final_loss) *final_loss = lh;
    }
    cleanup();
    return s;
}

}  // namespace gpm

extern "C" gpm_status gpm_mlp_train(gpm_graph *h, const float *feat, const float *label, uint64_t rows,
                                    uint32_t epochs, uint32_t batch, float lr, float *w32, uint16_t *w16,
                                    double *final_loss) {
    if (!h || !feat || !label || !w32 || !w16 || rows == 0 || epochs == 0 || batch == 0 || !(lr > 0.f)) {
        set_error("gpm_mlp_train: bad argument");
        return GPM_ERR_ARG;
    }
    return train_rows(h, feat, label, rows, epochs, batch, lr, w32, w16, final_loss);
}

extern "C" gpm_status gpm_train_proposal(gpm_graph *h, const gpm_pattern *pattern, uint64_t seed, uint64_t samples,
                                         uint32_t epochs, uint32_t batch, float lr, float *w32, uint16_t *w16,
                                         double *final_loss, uint64_t *rows_used) {
    if (!h || !pattern || !w32 || !w16 || samples == 0 || epochs == 0 || batch == 0 || !(lr > 0.f)) {
        set_error("gpm_train_proposal: bad argument");
        return GPM_ERR_ARG;
    }
    Plan p;
    std::string why = build_plan(*pattern, &p);
    if (!why.empty()) {
        set_error("pattern rejected: " + why);
        return GPM_ERR_ARG;
    }
    if (p.k < 4) {
        set_error("gpm_train_proposal: the learned proposal acts on steps j <= k-2, so k >= 4");
        return GPM_ERR_ARG;
    }
    gpm_sample_record *recs = nullptr;
    float *feat = nullptr, *label = nullptr;
    auto cleanup = [&]() {
        cudaFree(recs);
        cudaFree(feat);
        cudaFree(label);
    };
    const uint64_t max_rows = samples * (uint64_t)(p.k - 3);
    if (cudaMalloc((void **)&recs, sizeof(gpm_sample_record) * samples) != cudaSuccess ||
        cudaMalloc((void **)&feat, sizeof(float) * 3 * max_rows) != cudaSuccess ||
        cudaMalloc((void **)&label, sizeof(float) * max_rows) != cudaSuccess) {
        cleanup();
        set_error("gpm_train_proposal: device allocation failed");
        return GPM_ERR_OOM;
    }
    gpm_config plain;
    std::memset(&plain, 0, sizeof(plain));
    gpm_status s = trace_device(h, p, seed, 0, samples, &plain, recs);
    uint64_t rows = 0;
    if (s == GPM_OK) s = gpm_proposal_features(h, pattern, recs, samples, feat, label, &rows);
    if (s == GPM_OK && rows == 0) {
        s = GPM_ERR_ARG;
        set_error("gpm_train_proposal: no training rows (no sample passed step 2)");
    }
    // the records are not needed during training
    cudaFree(recs);
    recs = nullptr;
    if (s == GPM_OK) s = train_rows(h, feat, label, rows, epochs, batch, lr, w32, w16, final_loss);
    if (s == GPM_OK && rows_used) *rows_used = rows;
    cleanup();
    return s;
}
