/*
 * gpm.h -- C ABI of libgpm.so: GPU (sm_103a) approximate graph pattern mining
 * by neighbour sampling with eager verify and online convergence detection,
 * plus colour sparsification and the hybrid choice between the two.
 *
 * Method: "Accurate and Fast Approximate Graph Pattern Mining at Scale"
 * (ScaleGPM).  Every entry point cites the passage that defines what it
 * computes.
 *
 * Conventions that hold for every call:
 *  - Return value: GPM_OK (0) or a negative gpm_status.  On error a
 *    thread-local message is available from gpm_last_error().
 *  - Outputs are caller-allocated; the library never frees caller memory.
 *  - A gpm_graph owns its device copy of the graph (or borrows the caller's
 *    device arrays, see GPM_DEVICE_PTRS) and all device scratch it needs; calls
 *    on one handle run on the handle's CUDA stream and are not thread-safe for
 *    the same handle.  Different handles are independent.
 *  - Vertex ids are uint32; neighbour lists are sorted ascending; the graph is
 *    symmetric without self loops or duplicate edges (the paper's CSR, Sec. 6).
 *  - Sample s of a run draws its random words from Philox4x32-10 keyed by the
 *    run's seed and counted by s, so results do not depend on the launch shape.
 */
#ifndef GPM_H
#define GPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GPM_MAX_K 12          /* size of the per-sample record arrays */
#define GPM_MAX_PATTERN_K 10  /* largest pattern the planner accepts */

typedef struct gpm_graph gpm_graph;   /* opaque handle */

typedef enum {
    GPM_OK = 0,
    GPM_ERR_ARG = -1,             /* bad argument (null pointer, size, pattern) */
    GPM_ERR_GRAPH = -2,           /* CSR failed validation: unsorted, duplicate, loop, asymmetric, out of range */
    GPM_ERR_OOM = -3,             /* device allocation failed */
    GPM_ERR_CUDA = -4,            /* a CUDA runtime call failed */
    GPM_ERR_NOT_CONVERGED = -5,   /* n_max or max_seconds reached; the result is filled */
    GPM_ERR_ABORTED = -6,         /* gpm_abort() was called; the result is filled */
    GPM_ERR_UNSUPPORTED = -8,     /* the combination of options is not implemented */
    GPM_ERR_COMM = -9             /* the caller's gather callback reported a failure */
} gpm_status;

typedef enum {
    GPM_NS = 0,          /* neighbour sampling with eager verify (Sec. 4.1-4.2) */
    GPM_GS = 1,          /* graph sparsification + exact count (Sec. 2.2.2, 5.2; Algorithm 2):
                            colour classes (cfg->colors) or Bernoulli edges (cfg->edge_p);
                            cfg->samplers >= 2 independent sparsifications are averaged and
                            give ci_half_width = z s / sqrt(R), s the sample standard
                            deviation of the R scaled counts, eps_hat = ci / estimate */
    GPM_HYBRID = 2,      /* cost-model choice between NS and GS (Sec. 4.3-4.4, 5.1) */
    GPM_NS_LEARNED = 3,  /* NS with the learned, importance-weighted proposal */
    GPM_EXACT = 4        /* exact count on the full graph */
} gpm_scheme;

typedef enum {
    GPM_VERIFY_INTERSECT = 0,  /* draw from the full candidate set S_j (Algorithm 4) */
    GPM_VERIFY_CHECK = 1,      /* draw from one restricted list L_j, verify S_j membership by binary search */
    GPM_VERIFY_LAZY = 2        /* NS-base, the lazy verify of Sec. 2.2.1 / Algorithm 1 that Sec. 4.2 prunes:
                                  first edge from the 2m directed entries (M = 2m), x drawn from the union
                                  U_j of the back-neighbours' lists (the first one's list whole, then each
                                  later list's entries no earlier list holds, back-neighbours by position,
                                  lists ascending), factor |U_j|; after the last draw the closure check
                                  (distinct vertices, every pattern edge present, every non-edge absent when
                                  vertex-induced, every restriction) decides hit or miss (depth = k) */
} gpm_verify;

/* gpm_load_csr flags */
#define GPM_DEVICE_PTRS 1u   /* row_ptr/col are device pointers, borrowed for the handle's lifetime */
#define GPM_VALIDATE    2u   /* check the CSR invariants on the device (GPM_ERR_GRAPH if violated) */
#define GPM_RELABEL_DEGREE 4u /* relabel vertices by (degree, id) ascending on the device before building the
                                 index (the orientation the paper applies to cliques, Table tab:input caption;
                                 the order is this library's reading), into arrays the handle owns; every
                                 vertex id the library reports afterwards (traces) is a new id, see
                                 gpm_relabel_map */

/* A connected pattern with k vertices; bit j of adj[i] marks the edge i-j
 * (the matrix must be symmetric without diagonal).  induced = 1 counts
 * vertex-induced occurrences (motif counting), 0 edge-induced. */
typedef struct {
    uint8_t k;
    uint8_t induced;
    uint16_t adj[16];
} gpm_pattern;

/* BF16 weights of the learned proposal's 3 -> 64 -> 64 -> 1 ReLU MLP, as raw
 * 16-bit patterns, row-major [out][in], in DEVICE memory (4481 values). */
typedef struct {
    const uint16_t *w1, *b1, *w2, *b2, *w3, *b3;
} gpm_mlp;

/* Options; a zeroed struct (or NULL) selects every default. */
typedef struct {
    uint64_t window;        /* samples per convergence round W (default 2^20) */
    uint64_t n_min;         /* no stop before this many samples (default W) */
    uint64_t n_max;         /* stop unconverged here (default 2^40) */
    double max_seconds;     /* stop unconverged after this wall time (0 = none) */
    uint32_t colors;        /* GS colour count c (default 8) */
    uint32_t slot;          /* pattern slot in the RNG counter (default 0) */
    uint32_t verify;        /* gpm_verify (default INTERSECT) */
    uint32_t grid_blocks;   /* sampler launch shape overrides (0 = tuned default) */
    uint32_t block_warps;
    uint32_t cap;           /* per-warp on-chip candidate buffer, entries (0 = the largest
                               that keeps 4 resident 256-thread blocks per SM, 2 with a
                               learned proposal, 832 at 8 warps on a GB300; at most 512
                               when a pattern is vertex-induced) */
    const gpm_mlp *mlp;     /* learned proposal weights (device); required by GPM_NS_LEARNED and,
                               when set, selects the learned proposal in gpm_sample_sums,
                               gpm_sample_sums_static and gpm_trace */
    const gpm_mlp *selector; /* GPM_HYBRID: learned NS/GS selector head (device weights, same
                               MLP shape); NULL = the cost-model rule decides */
    double edge_p;          /* GS: 0 = colour sparsification with `colors`; in (0, 1] =
                               Bernoulli edge sparsification keeping each edge with this
                               probability (Algorithm 2; edge-induced patterns only) */
    uint32_t samplers;      /* GS: independent sparsifications averaged (default 1) */
    uint32_t bytes_sample;  /* NS, NS_LEARNED, batches: after the run, trace this many samples from
                               the start of the run's stream and report their mean algorithmic
                               bytes in gpm_result.algo_bytes_per_sample (0 = skip; not counted
                               in t_total_s) */
    uint32_t mlp_tensor;    /* learned proposal: 1 = score on the tensor cores (the 64 x 64 layer as
                               BF16 mma.sync tiles of 16 candidates, FP32 accumulation; layer-1
                               outputs rounded to BF16), 0 = the exact FP32 chain (default).  The
                               estimator stays unbiased either way (every score is >= 1) */
    uint32_t pad_;
} gpm_config;

/* What the hybrid choice saw (Sec. 4.3-4.4, 5.1): the pilot's sample count
 * estimate, the NS cone, the GS prediction and its parts, the time per
 * sampler step, the triangle estimate, the selector features
 * (log2(t_gs / t_lo), log2(t_hi / t_lo), log2(n_s), each clamped to +-64) and
 * both decisions (1 = GS).  cost_model_gs is the rule the hybrid applies: GS
 * iff t_gs < t_lo and GS's relative error can meet eps at all, i.e.
 * z sqrt((1/P - 1) / (R C)) <= eps with P = c^-(k-1) (colours) or p^l
 * (Bernoulli edges, l pattern edges), R samplers and C the pilot's estimate
 * (the diagonal term of the Sec. 5.2 variance: no two matches covary
 * negatively).  selector_gs is the head's own output; the hybrid follows it
 * under the same error condition. */
typedef struct {
    double n_s, t_lo, t_hi, t_gs, t_pre, t_search, c_step, triangles;
    float features[3];
    int32_t cost_model_gs, selector_gs;
} gpm_hybrid_info;

typedef struct {
    double estimate;        /* mu, the estimated count */
    double ci_half_width;   /* z * sigma (Algorithm 3), z = Phi^-1(1 - delta/2); GS: z s / sqrt(R)
                               over R >= 2 samplers, NaN for one */
    double eps_hat;         /* predicted relative error z * sigma / mu (Eq. equ:error); GS: the
                               interval over the estimate, NaN for one sampler */
    double sum, sumsq;      /* running sum X_i and sum X_i^2 over all samples */
    uint64_t samples;       /* n at the stop, a multiple of the window; GS: the samplers R */
    uint64_t hits;          /* samples with every candidate set non-empty */
    uint64_t rounds;        /* convergence rounds run */
    int32_t scheme_used;    /* gpm_scheme that produced the estimate */
    int32_t converged;      /* 1 if eps_hat <= eps was reached */
    double t_total_s;       /* wall time of the call */
    double t_pilot_s;       /* hybrid: pilot NS round and cost models */
    double t_preproc_s;     /* GS: colouring and sparsification */
    double t_sample_s;      /* device time of the sampling / counting kernels (CUDA events) */
    uint64_t exact_count;   /* GS: count on the sparsified graph(s), summed over the samplers;
                               EXACT: the count */
    uint64_t kernel_launches; /* kernels this call launched */
    double algo_bytes_per_sample; /* mean of gpm_sample_record.sectors x 32 over the first
                               cfg->bytes_sample samples of the run (0 when not asked for) */
} gpm_result;

/* One sample's path, for parity checks and training traces. */
typedef struct {
    uint64_t factor[GPM_MAX_K]; /* [0] = M (m or 2m), [j] = |S_j| (CHECK: |L_j|; learned: A_j) */
    uint64_t w_u64;             /* exact weight, 0 on a miss or overflow (learned: 0) */
    double w_f64;               /* weight as a left-to-right FP64 product, 0 on a miss */
    uint32_t vert[GPM_MAX_K];   /* matched vertices in matching order, 0xFFFFFFFF past the depth */
    uint32_t aux[GPM_MAX_K];    /* learned: score a_x of the chosen vertex at step j */
    uint8_t hit, depth, overflow, pad;
    uint32_t sectors;           /* algorithmic 32-byte sectors of the sample's path (Sec. 4.2's
                                   per-step set reads): 1 for the first edge; per step j taken and
                                   per list the candidate-set definition references there (every
                                   back-neighbour, and every other earlier vertex when vertex-
                                   induced; only N(v_{j-1}) when S_j extends S_{j-1} by one
                                   adjacency under the same bounds), 1 for its row_ptr pair plus
                                   the sectors its part above the step's lower bound spans; CHECK:
                                   per step 1 + a bound search ceil(log2(d + 1)) when bounded, and
                                   when L_j is not empty 1 for the drawn entry plus, per other
                                   referenced list, 1 + ceil(log2(d + 1)) */
} gpm_sample_record;

/* Totals of a fixed block of samples. */
typedef struct {
    uint64_t n, hits;
    double sum, sumsq;
} gpm_sums;

/* Totals of one 64-sample chunk (the unit every reduction adds in chunk
 * order). */
typedef struct {
    double sum, sumsq;
    uint64_t hits, n;
} gpm_partial;

/* Running state of Algorithm 3 for one estimate: totals over the finished
 * windows and the outcome of the last window test. */
typedef struct {
    double sum, sumsq;            /* running totals of X and X^2 */
    uint64_t hits, n, rounds;
    double mu, half, eps_hat;     /* estimate, z sigma, z sigma / mu */
    uint32_t converged, active;   /* start a run with active = 1, everything else 0 */
} gpm_window;

/* Load a graph (Sec. 6: symmetric CSR without loops or duplicates).
 *  n        vertex count (< 2^32 - 1)
 *  row_ptr  n + 1 offsets into col, row_ptr[0] = 0 (uint64)
 *  col      row_ptr[n] neighbour ids, each list sorted ascending (uint32);
 *           every degree below 2^31 (else GPM_ERR_GRAPH)
 *  flags    GPM_DEVICE_PTRS: both arrays are device pointers the handle borrows
 *           (the caller keeps them alive and unchanged until gpm_free_graph);
 *           otherwise they are host arrays that the call copies.
 *           GPM_VALIDATE: check the invariants on the device.
 *  stream   cudaStream_t for every call on this handle (NULL = legacy default)
 *  out      receives the handle
 * Builds the oriented-edge index (first neighbour above v and the prefix of
 * upper-degree counts) used to draw the first edge of a sample. */
gpm_status gpm_load_csr(uint64_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t flags,
                        void *stream, gpm_graph **out);

/* Release a handle and every device array it owns (borrowed arrays stay the
 * caller's).  Library convenience: the paper has no counterpart.  NULL is a
 * no-op; the handle's stream is synchronised first. */
void gpm_free_graph(gpm_graph *g);

/* For a graph loaded with GPM_RELABEL_DEGREE: new_of_old (HOST, n entries)
 * receives the new id of every vertex as given to gpm_load_csr.  Library
 * convenience: the paper has no counterpart.  GPM_ERR_ARG without the flag. */
gpm_status gpm_relabel_map(const gpm_graph *g, uint32_t *new_of_old);

/* n, m (undirected edges), 2m, maximum degree. Any output may be NULL.
 * Library convenience: the paper has no counterpart. */
gpm_status gpm_graph_info(const gpm_graph *g, uint64_t *n, uint64_t *m, uint64_t *nnz, uint64_t *max_degree);

/* Estimate the pattern's count to relative error eps with confidence 1-delta.
 * GPM_NS / GPM_NS_LEARNED: Algorithm 3 over Algorithm 4-style samples, rounds
 * of cfg->window samples until eps_hat <= eps (Eq. equ:error).
 * GPM_GS: one colouring with cfg->colors colours, exact count on the
 * sparsified graph, scaled by c^(k-1) (eps and delta unused, ci = NaN).
 * GPM_HYBRID: a pilot NS round feeds the cost models of Sec. 4.3-4.4 and the
 * faster engine runs (Sec. 5.1, loose mode); GS only when its error bound
 * allows eps (see gpm_hybrid_info).  GPM_EXACT: exact count.
 * Returns GPM_ERR_NOT_CONVERGED (result filled) if n_max or max_seconds ends
 * the run first; for GPM_GS and GPM_EXACT, max_seconds bounds the exact
 * search on the device, and a search stopped by it leaves a lower bound in
 * exact_count with converged = 0. */
gpm_status gpm_estimate(gpm_graph *g, const gpm_pattern *pattern, gpm_scheme scheme, double eps,
                        double delta, uint64_t seed, const gpm_config *cfg, gpm_result *out);

/* The hybrid choice without running the chosen engine (pilot NS round, cost
 * models, selector if cfg->selector).  eps and delta as for gpm_estimate. */
gpm_status gpm_hybrid_model(gpm_graph *g, const gpm_pattern *pattern, double eps, double delta, uint64_t seed,
                            const gpm_config *cfg, gpm_hybrid_info *out);

/* Sample-count profilers (Sec. 5.3 and this library's pilot reading): the
 * predicted number of NS samples N_s to reach eps at 1 - delta, the input of
 * the NS cost model (Sec. 4.3).  kind GPM_PROFILE_PILOT: one window
 * (cfg->window, default 2^20) of samples on G, N_s = (z sd / (eps mu))^2.
 * kind GPM_PROFILE_SPARSIFIED: the paper's fast profiler: G' keeps each edge
 * with probability frac (0.1 in the paper), NS-online on G' stops at a 50%
 * error (windows of 2^14, at most 2^26 samples) after N_o samples with final
 * predicted error eps_o, and N_s = N_o (eps_o / eps)^2 rho(G') / rho(G), rho
 * the hit rates (rho(G) from 2^16 samples on G; the printed formula is not
 * dimensionally consistent, see gpm_profile_info).  Neither changes any
 * estimate. */
#define GPM_PROFILE_PILOT 0
#define GPM_PROFILE_SPARSIFIED 1
typedef struct {
    double n_s;             /* predicted samples (infinity when the profile saw no hit) */
    double seconds;         /* wall time of the profile */
    double n_o, eps_o;      /* sparsified: samples and final predicted error of the run on G' */
    double rho_g, rho_gp;   /* hit rates on G and (sparsified) on G' */
    uint64_t samples_used;  /* samples drawn by the profile on G and G' together */
    int32_t kind, pad_;
} gpm_profile_info;

gpm_status gpm_profile(gpm_graph *g, const gpm_pattern *pattern, int32_t kind, double frac, double eps,
                       double delta, uint64_t seed, const gpm_config *cfg, gpm_profile_info *out);

/* Trains the MLP on given rows (DEVICE feat [rows][3], label [rows]): `epochs`
 * passes of Adam (lr; beta 0.9, 0.999) over minibatches of `batch` rows of the
 * mean cross-entropy on the logits; w32 (DEVICE, 4481) in/out, w16 (DEVICE,
 * 4481) receives the BF16 copies; *final_loss over all rows.  Used for the
 * NS/GS selector head. */
gpm_status gpm_mlp_train(gpm_graph *g, const float *feat, const float *label, uint64_t rows, uint32_t epochs,
                         uint32_t batch, float lr, float *w32, uint16_t *w16, double *final_loss);

/* Many (pattern, eps) jobs at once: every round is one persistent sampler
 * launch over the chunks of all jobs still running, followed by a per-job
 * reduction and convergence test on the device; rounds run as a captured CUDA
 * graph.  Job i uses RNG slot cfg->slot + i, so its result equals a separate
 * gpm_estimate with that slot.  out has count entries; at most 1024 jobs.
 * GPM_ERR_NOT_CONVERGED if any job hit n_max (all results filled). */
gpm_status gpm_estimate_batch(gpm_graph *g, uint32_t count, const gpm_pattern *patterns,
                              const double *eps, double delta, uint64_t seed, const gpm_config *cfg,
                              gpm_result *out);

/* Times three convergence rounds of the batch under each candidate launch
 * shape (4 or 8 warps per block; on-chip candidate buffers of 256 or 512
 * entries per warp, or the default) and writes the fastest into
 * io->block_warps and io->cap; the default shape (8 warps, default buffers)
 * is kept unless another is more than 2% faster.  The paper has no
 * counterpart (its windows run on CPU threads, Sec. 5.4); library
 * convenience for batched launches.
 * Estimates do not depend on the shape: samples are grouped in fixed chunks of
 * 64 whose partials are reduced in chunk order. */
gpm_status gpm_autotune(gpm_graph *g, uint32_t count, const gpm_pattern *patterns, uint64_t seed, gpm_config *io);

/* Samples [first, first + count) of an NS run (Algorithm 3's inner loop):
 * totals of X_i and X_i^2 in FP64.  cfg selects verify mode, slot and MLP. */
gpm_status gpm_sample_sums(gpm_graph *g, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                           uint64_t count, const gpm_config *cfg, gpm_sums *out);

/* The per-chunk partials of samples [first, first + count) (Algorithm 3's inner
 * loop) that fall to one of `world` ranks when the range's 64-sample chunks are
 * dealt round robin: chunk c (samples first + 64c .. first + 64c + 63, the last
 * chunk possibly shorter) belongs to rank c mod world.  out[i] receives the
 * partial of chunk rank + i * world, for every such chunk in the range;
 * *n_out receives their number, ceil((ceil(count / 64) - rank) / world) when
 * positive, else 0.  out is a host array with room for that many entries.
 * Interleaving the ranks' arrays restores chunk order, and gpm_merge_partials
 * over it gives gpm_sample_sums's totals bit for bit (the multi-GPU form of a
 * round: each rank samples its chunks, the partials are gathered and merged
 * in chunk order).  rank < world, world >= 1; cfg selects verify mode, slot
 * and MLP as for gpm_sample_sums. */
gpm_status gpm_sample_partials(gpm_graph *g, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                               uint64_t count, uint32_t rank, uint32_t world, const gpm_config *cfg,
                               gpm_partial *out, uint64_t *n_out);

/* Host-only: adds n chunk partials (in chunk order) with the fixed-shape
 * reduction the device uses for a round -- 1024 contiguous runs of
 * ceil(n / 1024) partials, each added left to right, then a pairwise tree over
 * the runs (run t += run t + h for h = 512, 256, ..., 1) -- so the result is
 * bit-identical to the device's.  n < 2^32.  Needs no GPU. */
gpm_status gpm_merge_partials(const gpm_partial *parts, uint64_t n, gpm_sums *out);

/* ---- multi-GPU rounds (Algorithm 3 with each window split over ranks) ----
 * A window's chunk-order reduction adds 1024 contiguous runs of
 * per = ceil(ceil(count / 64) / 1024) chunks each, left to right, then folds
 * the runs pairwise (run t += run t + h, h = 512, 256, ..., 1).  Rank r of
 * `world` (1 <= world <= 1024) owns the runs [r B, min((r + 1) B, 1024)),
 * B = ceil(1024 / world): one contiguous range of samples.  Gathering every
 * rank's B run sums in rank order and folding the first 1024 gives the
 * one-GPU totals of the window bit for bit. */

/* This rank's run sums of samples [first, first + count): out (HOST, B entries,
 * zeros for runs past the window's chunks). */
gpm_status gpm_sample_runs(gpm_graph *g, const gpm_pattern *pattern, uint64_t seed, uint64_t first, uint64_t count,
                           uint32_t rank, uint32_t world, const gpm_config *cfg, gpm_partial *out);

/* Host-only: the pairwise fold of 1024 run sums (HOST, in run order) into
 * totals.  Needs no GPU. */
gpm_status gpm_merge_runs(const gpm_partial *runs, gpm_sums *out);

/* All-gather supplied by the caller (NCCL, MPI, torch.distributed, ...):
 * every rank passes `bytes` bytes in `send` and receives all ranks' blocks,
 * in rank order, in `recv` (world x bytes).  Returns 0 on success. */
typedef int (*gpm_allgather_fn)(void *ctx, const void *send, void *recv, size_t bytes);

/* Algorithm 3 over `world` ranks, one call per rank (each on its own GPU and
 * handle of the same graph): every window, this rank samples its run block
 * (gpm_sample_runs), `gather` exchanges B x 32 bytes, and every rank folds the
 * runs and applies the window test (gpm_window_update) identically, so all
 * ranks stop together with the one-GPU gpm_estimate's totals and estimate
 * (same seed, cfg->slot, cfg->window) bit for bit.  cfg as for gpm_estimate
 * (window, n_min, n_max, max_seconds, slot, verify, mlp).  state (nullable):
 * the run's gpm_window, continued and written back, for checkpoint/resume;
 * max_rounds > 0 stops after that many windows of this call (a paused run
 * returns GPM_OK with state->active = 1).  GPM_ERR_COMM if the callback fails;
 * NOT_CONVERGED / ABORTED as for gpm_estimate. */
gpm_status gpm_estimate_sharded(gpm_graph *g, const gpm_pattern *pattern, double eps, double delta, uint64_t seed,
                                uint32_t rank, uint32_t world, const gpm_config *cfg, gpm_allgather_fn gather,
                                void *ctx, gpm_window *state, uint64_t max_rounds, gpm_result *out);

/* Host-only: one window of Algorithm 3 (Eq. equ:error).  Folds the window's
 * totals into w (the first window is assigned, later ones added), then with
 * nn = n: mu = sum / nn, var = max(sumsq / nn - mu^2, 0), sigma = sqrt(var / nn),
 * half = z sigma, eps_hat = z sigma / mu (infinity unless mu > 0); converged
 * when n >= n_min, mu > 0 and eps_hat <= eps, else inactive once n >= n_max.
 * Every step is one correctly rounded FP64 operation in this order, as in the
 * device's window test, so both decide alike.  z = Phi^-1(1 - delta / 2)
 * (gpm_normal_quantile).  Needs no GPU. */
gpm_status gpm_window_update(gpm_window *w, const gpm_sums *window, double z, double eps, uint64_t n_min,
                             uint64_t n_max);

/* Same totals as gpm_sample_sums, bit for bit, for callers that cannot
 * allocate device memory while they run: applications that reserve all their
 * device memory up front in a pool of their own (so a cudaMalloc would fail or
 * fragment that pool), and latency-bound loops that cannot afford the device
 * synchronisation an allocation implies.  The paper has no counterpart: this
 * is a library convenience.  Instead of handle-owned buffers the call keeps
 * its scratch (per-chunk partials, chunk counter, totals) in one fixed array
 * of about 2 MiB that every GPU loading the library holds until the process
 * exits.  It still synchronises the handle's stream to read the totals back.
 * Limits and rules:
 *  - count <= 2^22 samples per call (65,536 chunks of the fixed 64 samples),
 *    else GPM_ERR_ARG with nothing launched; split larger ranges into calls
 *    and add their totals;
 *  - the handle must come from gpm_load_csr (which allocates once, up front);
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current;
 *  - all calls in the process share the one array and leave their contents in
 *    it (each call resets the chunk counter it needs): calls whose work
 *    overlaps on the GPU (other streams, other threads) race and must be
 *    serialised by the caller. */
gpm_status gpm_sample_sums_static(gpm_graph *g, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                                  uint64_t count, const gpm_config *cfg, gpm_sums *out);

/* Per-sample records of samples [first, first + count) into HOST memory: the
 * path each sample of Algorithm 4 / Lemma 1 takes (Sec. 4.2): the first-edge
 * count M, every |S_j|, the matched vertices, the hit flag and the weight
 * M prod |S_j| (0 on a miss), plus the algorithmic sectors of the path.  Used
 * for parity checks and as the learned proposal's training traces. */
gpm_status gpm_trace(gpm_graph *g, const gpm_pattern *pattern, uint64_t seed, uint64_t first,
                     uint64_t count, const gpm_config *cfg, gpm_sample_record *out);

/* Exact count of the pattern: the plan's nested loops over every branch of
 * the candidate sets (the exact GPM count C of Sec. 2.1 that GS runs on the
 * sparsified graph, Sec. 2.2.2 / Algorithm 2; here on the whole graph). */
gpm_status gpm_exact_count(gpm_graph *g, const gpm_pattern *pattern, uint64_t *out);

/* ---- learned proposal (not in the paper; see gpm_scheme GPM_NS_LEARNED) ----
 * At a step j <= k-2 whose candidate set has 1..256 entries, candidate x gets
 * the score a_x = 1 + floor(4096 clamp(z/8 + 1/2, 0, 1)), z the output of a
 * 3 -> 64 -> 64 -> 1 ReLU MLP (BF16 weights, FP32 fused multiply-adds in input
 * order) on the features (log2(1 + deg x), j, log2(1 + |S_{j+1}(x)|)) with
 * log2(1 + d) taken as the chord between powers of two; x is drawn with
 * probability a_x / A (A = sum of scores, integer CDF in candidate order) and
 * the weight takes the factor A / a_x.  Every score is >= 1, so the estimator
 * stays unbiased (Lemma 1's argument); larger sets and the last step are drawn
 * uniformly.  Weights: 4481 values in the order w1 [64][3], b1 [64],
 * w2 [64][64], b2 [64], w3 [64], b3 [1]. */

/* Scores a_x of n feature rows (DEVICE float [n][3]) into DEVICE out [n];
 * bit-identical to the scores the sampler computes. */
gpm_status gpm_mlp_scores(gpm_graph *g, const gpm_mlp *mlp, const float *feat, uint64_t n, uint32_t *out);

/* The same rows scored as the sampler does with cfg->mlp_tensor = 1: the 64 x 64
 * layer as BF16 mma.sync tiles (FP32 accumulation) after rounding the layer-1
 * outputs to BF16.  Close to, not equal to, gpm_mlp_scores: the difference in
 * the logit is bounded by the BF16 rounding of the hidden layer. */
gpm_status gpm_mlp_scores_tc(gpm_graph *g, const gpm_mlp *mlp, const float *feat, uint64_t n, uint32_t *out);

/* Mean binary cross-entropy on the logits over rows (DEVICE feat [rows][3],
 * label [rows] in {0, 1}) at FP32 weights w32 (DEVICE, 4481) and its
 * gradient into DEVICE grad (4481); *loss on the host. */
gpm_status gpm_mlp_loss_grad(gpm_graph *g, const float *w32, const float *feat, const float *label, uint64_t rows,
                             float *grad, double *loss);

/* Training rows from plain-NS records (DEVICE, n): for every step
 * 2 <= j <= k-2 a sample passed, the features of its chosen vertex vert[j]
 * (the lookahead is factor[j+1]) and the progress label
 * (d - j - 1) / (k - j - 1) in FP32, d = depth (k on a hit): 1 on a hit, 0
 * when step j+1 found no candidate; rows in record then step order into
 * DEVICE feat [n (k-3)][3] and label; *rows = rows written. */
gpm_status gpm_proposal_features(gpm_graph *g, const gpm_pattern *pattern, const gpm_sample_record *recs,
                                 uint64_t n, float *feat, float *label, uint64_t *rows);

/* Trains the proposal on the device: records of `samples` plain-NS samples
 * (seed), their feature rows, then `epochs` passes of Adam (lr; beta 0.9,
 * 0.999) over minibatches of `batch` rows of the mean cross-entropy.  w32
 * (DEVICE, 4481) holds the initial FP32 weights and receives the trained
 * ones; w16 (DEVICE, 4481) receives their BF16 copies (round to nearest even)
 * in the gpm_mlp order.  *final_loss: loss of the trained weights over all
 * rows; *rows_used: row count.  Pattern size k >= 4. */
gpm_status gpm_train_proposal(gpm_graph *g, const gpm_pattern *pattern, uint64_t seed, uint64_t samples,
                              uint32_t epochs, uint32_t batch, float lr, float *w32, uint16_t *w16,
                              double *final_loss, uint64_t *rows_used);

/* Colour sparsification (Sec. 2.2.2): colour every vertex with
 * floor(philox_word0 * c / 2^32) and keep monochromatic edges.  Writes the
 * sparsified CSR into caller-provided DEVICE arrays row_out (n + 1) and
 * col_out (capacity 2m); *kept receives its entry count. */
gpm_status gpm_sparsify(gpm_graph *g, uint32_t colors, uint64_t seed, uint32_t colouring, uint32_t slot,
                        uint64_t *row_out, uint32_t *col_out, uint64_t *kept);

/* The multi-GPU form of GS (Sec. 2.2.2, 5.2): the exact count, on the colour-
 * sparsified graph of gpm_sparsify (colors, seed, colouring, slot), of the
 * matches in the colour classes c with c mod world == rank.  A match of the
 * sparsified graph lies inside one class, so the counts of ranks 0..world-1
 * add up to its exact count (one integer all-reduce); times c^(k-1) that is
 * GS's estimate.  max_seconds bounds the search as in gpm_estimate
 * (GPM_ERR_NOT_CONVERGED with a lower bound).  rank < world. */
gpm_status gpm_gs_count_classes(gpm_graph *g, const gpm_pattern *pattern, uint32_t colors, uint64_t seed,
                                uint32_t colouring, uint32_t slot, uint32_t rank, uint32_t world, double max_seconds,
                                uint64_t *count);

/* Bernoulli edge sparsification (Algorithm 2): keep probability p realised as
 * t / 2^32 with t = floor(p * 2^32) (t = 2^32 for p >= 1); edge {u, w} stays
 * iff the first word of Philox4x32-10 at counter (min(u, w), max(u, w),
 * colouring, slot << 8 | 3), key = seed, is below t, one decision for both
 * CSR entries.  Output as gpm_sparsify.  0 < p; t must be positive. */
gpm_status gpm_sparsify_edges(gpm_graph *g, double p, uint64_t seed, uint32_t colouring, uint32_t slot,
                              uint64_t *row_out, uint32_t *col_out, uint64_t *kept);

/* Measurement only (not part of any estimate): the random-access roofline
 * of the sampler's memory pattern.  Threads follow independent chains of
 * `chain` dependent hops through a fresh buffer of `bytes` random words; each
 * hop reads one 32-byte sector at a random position computed from the
 * previous hop's data.  About `hops` hops are timed (after one warm-up pass)
 * and *sectors_bytes_per_s receives 32 bytes x hops / kernel time.  Use a
 * buffer the size of the graph (an L2-resident size gives the L2 figure).
 * bytes >= 4096, 1 <= chain <= 64. */
gpm_status gpm_gather_probe(uint64_t bytes, uint32_t chain, uint64_t hops, double *sectors_bytes_per_s);

/* Ask a running estimate on this handle to stop at its next round boundary
 * (it returns GPM_ERR_ABORTED with the partial result).  Library
 * convenience: the paper has no counterpart.  Safe to call from another host
 * thread while the estimate runs. */
gpm_status gpm_abort(gpm_graph *g);

/* Matching order and symmetry-breaking restrictions of a pattern (for
 * inspection; the pruning of Sec. 4.2: matching order and symmetry breaking,
 * which Algorithm 4 shows for the 4-cycle): order[j] = pattern vertex at
 * position j; restriction r reads
 * v[res_lo[r]] < v[res_hi[r]]; *oriented = 1 if the first edge is drawn from
 * the m oriented edges.  Arrays hold GPM_MAX_K and 64 entries. */
gpm_status gpm_plan(const gpm_pattern *pattern, int32_t *order, int32_t *res_lo, int32_t *res_hi,
                    int32_t *nres, int32_t *oriented);

/* Phi^-1(p), the standard normal quantile of Eq. equ:error (z = Phi^-1(1 - delta/2)). */
double gpm_normal_quantile(double p);

/* The calling thread's message for the last failed call (library convenience). */
const char *gpm_last_error(void);
/* Library version string (library convenience). */
const char *gpm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPM_H */
