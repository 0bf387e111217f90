// Internal declarations of libgpm (host and device).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include <string>
#include <vector>

#include "../../include/gpm.h"

namespace gpm {

constexpr int kMaxK = GPM_MAX_K;

// Pattern compiled for the sampler: everything is indexed by matching
// position j (v_0 .. v_{k-1}).
struct Plan {
    int32_t k, induced, oriented, nres;
    int32_t order[kMaxK];         // pattern vertex placed at position j
    uint32_t back[kMaxK];         // positions i < j adjacent to j in the pattern
    uint32_t nonback[kMaxK];      // positions i < j not adjacent to j
    uint32_t lower[kMaxK];        // positions i < j with the restriction v_i < v_j
    uint32_t reuse[kMaxK];        // S_j from S_{j-1} above the bounds: 1 keep N(v_{j-1}), 2 drop it, 3 neither
    uint32_t last_back[kMaxK];    // largest back-neighbour position of j
    int32_t res_lo[64], res_hi[64];
};

// Builds the plan; returns an empty string on success, else the reason.
std::string build_plan(const gpm_pattern &pat, Plan *out);

// Device view of a resident graph.
struct DGraph {
    const uint64_t *row_ptr;   // n + 1
    const uint32_t *col;       // nnz
    const uint64_t *up;        // n: index of the first neighbour above v
    const uint64_t *uoff;      // n + 1: prefix sum of |N+(u)|
    const uint64_t *edges;     // m oriented edges (w << 32 | u), u < w, or null
    uint64_t n, nnz, m;
};

// Per-chunk partial of a sampling round.
struct Partial {
    double sum, sumsq;
    uint64_t hits, n;
};

// Running totals of a run, updated on the device after each round.
struct Totals {
    double sum, sumsq;
    uint64_t hits, n;
};

void set_error(const std::string &msg);

// Stream-ordered device allocations from the library's pool (one per device,
// memory kept by the pool when freed, so a freed graph's arrays serve the next
// graph loaded in the process without new device mappings).
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st);
void pool_free(void *p, cudaStream_t st);

// Single correctly rounded FP64 operations on host and device (the device
// would otherwise be free to fuse a multiply and an add).
__host__ __device__ inline double rn_add(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ inline double rn_sub(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ inline double rn_mul(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ inline double rn_div(double a, double b) {
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    return a / b;
#endif
}
__host__ __device__ inline double rn_sqrt(double a) {
#ifdef __CUDA_ARCH__
    return __dsqrt_rn(a);
#else
    return std::sqrt(a);
#endif
}

// Algorithm 3's window test on the running totals (Eq. equ:error), shared by
// the device (batch_reduce_check) and the host (gpm_window_update).
__host__ __device__ inline void window_test(double sum, double sumsq, uint64_t n, double z, double eps,
                                            uint64_t n_min, uint64_t n_max, double *mu_out, double *half_out,
                                            double *eps_hat_out, uint32_t *converged, uint32_t *active) {
    const double nn = (double)n;
    const double mu = rn_div(sum, nn);
    double var = rn_sub(rn_div(sumsq, nn), rn_mul(mu, mu));
    if (var < 0.0) var = 0.0;
    const double sigma = rn_sqrt(rn_div(var, nn));
    const double half = rn_mul(z, sigma);
    *mu_out = mu;
    *half_out = half;
    *eps_hat_out = (mu > 0.0) ? rn_div(half, mu) : INFINITY;
    if (n >= n_min && mu > 0.0 && *eps_hat_out <= eps) {
        *converged = 1;
        *active = 0;
    } else if (n >= n_max) {
        *active = 0;
    }
}

}  // namespace gpm

struct gpm_graph;
namespace gpm {
gpm_status exact_count_plan(gpm_graph *h, const Plan &p, uint64_t *out, float *kernel_ms, double max_seconds);
gpm_status gs_estimate(gpm_graph *h, const Plan &p, uint64_t seed, double delta, const gpm_config *cfg,
                       gpm_result *out);
gpm_status sparsify_alloc(gpm_graph *h, uint32_t c, uint64_t seed, uint32_t colouring, uint32_t slot,
                          uint64_t **row_out, uint32_t **col_out, uint64_t *kept, uint64_t *user_row,
                          uint32_t *user_col, uint64_t bes_t = 0, uint32_t class_rank = 0, uint32_t class_world = 1);
double normal_quantile(double p);
gpm_status batch_estimate(gpm_graph *h, const std::vector<Plan> &plans, const double *eps, double delta,
                          uint64_t seed, const gpm_config *cfg, gpm_result *results, int mode);
gpm_status relabel_by_degree(uint64_t n, uint64_t nnz, const uint64_t *row_ptr, const uint32_t *col,
                             cudaStream_t st, uint64_t **row_out, uint32_t **col_out, uint32_t **newid_out);
gpm_status algo_bytes_mean(gpm_graph *h, const Plan &p, int mode, uint64_t seed, uint32_t slot,
                           const gpm_config *cfg, uint64_t count, double *out);
}  // namespace gpm

// The opaque handle.
struct gpm_graph {
    gpm::DGraph d;
    cudaStream_t stream;
    uint64_t max_degree;
    // owned device memory (null when borrowed)
    uint64_t *own_row_ptr;
    uint32_t *own_col;
    uint64_t *up, *uoff;
    uint64_t *edges;              // materialised oriented edges (optional)
    uint32_t *newid;              // GPM_RELABEL_DEGREE: new id of every loaded vertex (else null)
    // sampler scratch
    gpm::Partial *partials;
    uint64_t partials_cap;
    gpm::Totals *totals;          // device
    gpm::Totals *totals_host;     // points at totals_buf (each copy into it is followed by a stream sync)
    gpm::Totals totals_buf[2];
    unsigned int *counter;        // device chunk counter
    volatile int abort_flag;
    int sm_count;
    int smem_per_sm;              // shared memory per SM and reserved per block, bytes
    int smem_reserved;
    cudaEvent_t ev0, ev1;
};
