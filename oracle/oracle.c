/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for the neighbour-sampling
 * (NS) estimator with eager verify, its online convergence test, colour
 * sparsification (GS) with exact counting, and the learned proposal.
 *
 * TEST INFRASTRUCTURE ONLY.  The product library never links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or helper with the CUDA path.
 *
 * Paper: "Accurate and Fast Approximate Graph Pattern Mining at Scale".
 *   - Sec. 2.2.1 / Algorithm 1: neighbour sampling, weight = m * prod c_j.
 *   - Sec. 4.1 / Eq. (equ:error) / Theorem 1 / Algorithm 3: online convergence
 *     detection with running sum and squared sum, var = sq/n - mu^2,
 *     sigma = sqrt(var/n), eps_hat = Phi^-1(1 - delta/2) * sigma / mu.
 *   - Sec. 2.2.1 / Algorithm 1 and Sec. 4.2: NS-base, lazy verify: each vertex
 *     is drawn from the union of its pattern neighbours' lists with weight
 *     factor |U_j|, and every constraint is checked only after all k draws
 *     (closure check); see og_union and og_closure.
 *   - Sec. 4.2 / Algorithm 4 / Lemma 1: eager verify ("NS-prune"): each vertex
 *     is drawn uniformly from a candidate set that already folds in every
 *     pattern edge to earlier vertices and the symmetry-breaking bounds; the
 *     weight is m * prod |S_j| and a sample with an empty set is a miss (0).
 *   - Sec. 2.2.2: colour sparsification keeps monochromatic edges; a match
 *     with k vertices survives with probability c^-(k-1) (the paper writes the
 *     exponent with the edge count l; for a connected pattern the survival
 *     event is "all k vertices share one colour", so the exponent is k-1).
 *   - Sec. 2.2.2 / Algorithm 2: Bernoulli edge sparsification keeps every edge
 *     independently with probability p; a match with l edges survives with
 *     probability p^l, so the exact count of G' scaled by p^-l is unbiased
 *     (edge-induced counting; removing edges can create vertex-induced
 *     occurrences, so that case has no such estimator).  Several independent
 *     sparsifications ("samplers", Sec. 2.2.2) are averaged.
 *   - Sec. 6 (evaluation setup): vertex-induced (motif) counting uses set
 *     difference for pattern non-edges.
 *
 * Readings where the paper is silent (all pinned the same way in the tests):
 *   - RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = seed,
 *     counter = (s_lo, s_hi, block, slot << 8 | purpose).  Choice t uses the
 *     64-bit word pair (t mod 2) of block t/2.
 *   - Index map: idx = floor(r * N / 2^64) (multiply-high, no rejection).
 *   - Candidate sets are sorted ascending by vertex id; the drawn index refers
 *     to that order.
 *   - Matching order and Grochow-Kellis symmetry breaking, see og_plan_build.
 *   - Misses count in n; var uses the population form of Algorithm 3.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_MAXK 12
#define OG_MAXRES 66
/* learned proposal: candidate sets above this size are drawn uniformly */
#define OG_LEARNED_MAX 256

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, written from its published definition (SC'11).  Each round */
/* multiplies counter words 0 and 2 by two fixed odd constants, takes the    */
/* high and low halves, and mixes them with words 1, 3 and the round key.    */
/* The key is advanced by the two Weyl constants between rounds.             */
/* ------------------------------------------------------------------------- */
void og_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 64-bit uniform word for choice t of sample s (purpose 0 = sampling). */
uint64_t og_choice_word(uint64_t seed, uint64_t s, uint32_t slot, uint32_t purpose, uint32_t t)
{
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), t / 2u, (slot << 8) | purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    og_philox4x32_10(ctr, key, o);
    uint32_t w = (t % 2u) * 2u;
    return (uint64_t)o[w] | ((uint64_t)o[w + 1] << 32);
}

/* floor(r * n / 2^64) */
uint64_t og_index_map(uint64_t r, uint64_t n)
{
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

/* ------------------------------------------------------------------------- */
/* Graph: symmetric CSR without loops or duplicates, sorted neighbour lists. */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint64_t n, nnz;               /* nnz = 2m directed entries */
    const uint64_t *row_ptr;       /* n + 1 */
    const uint32_t *col;           /* nnz */
    uint64_t *up;                  /* up[v] = index of the first neighbour > v */
    uint64_t *uoff;                /* uoff[v] = sum over u < v of |N+(u)|, n + 1 */
} og_graph;

/* Returns 0 if valid, else a negative code naming the first violation. */
int og_validate(uint64_t n, const uint64_t *row_ptr, const uint32_t *col)
{
    if (row_ptr[0] != 0) return -1;
    for (uint64_t v = 0; v < n; v++) {
        if (row_ptr[v + 1] < row_ptr[v]) return -1;
        for (uint64_t i = row_ptr[v]; i < row_ptr[v + 1]; i++) {
            uint32_t x = col[i];
            if (x >= n) return -2;                          /* out of range */
            if (x == v) return -3;                          /* self loop */
            if (i > row_ptr[v] && col[i - 1] >= x) return -4; /* unsorted/dup */
            /* symmetry: v must be in N(x) */
            uint64_t lo = row_ptr[x], hi = row_ptr[x + 1];
            int found = 0;
            while (lo < hi) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (col[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            if (lo < row_ptr[x + 1] && col[lo] == (uint32_t)v) found = 1;
            if (!found) return -5;
        }
    }
    return 0;
}

og_graph *og_graph_new(uint64_t n, const uint64_t *row_ptr, const uint32_t *col)
{
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    g->n = n;
    g->nnz = row_ptr[n];
    g->row_ptr = row_ptr;
    g->col = col;
    g->up = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    g->uoff = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    uint64_t acc = 0;
    for (uint64_t v = 0; v < n; v++) {
        uint64_t i = row_ptr[v];
        while (i < row_ptr[v + 1] && col[i] < v) i++;
        g->up[v] = i;
        g->uoff[v] = acc;
        acc += row_ptr[v + 1] - i;
    }
    g->up[n] = row_ptr[n];
    g->uoff[n] = acc;
    return g;
}

void og_graph_free(og_graph *g)
{
    if (!g) return;
    free(g->up);
    free(g->uoff);
    free(g);
}

uint64_t og_graph_m(const og_graph *g) { return g->uoff[g->n]; }

static uint64_t og_deg(const og_graph *g, uint32_t v) { return g->row_ptr[v + 1] - g->row_ptr[v]; }

static int og_adjacent(const og_graph *g, uint32_t v, uint32_t x)
{
    uint64_t lo = g->row_ptr[v], hi = g->row_ptr[v + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (g->col[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo < g->row_ptr[v + 1] && g->col[lo] == x;
}

/* index of the first element of N(v) greater than x */
static uint64_t og_first_above(const og_graph *g, uint32_t v, uint32_t x)
{
    uint64_t lo = g->row_ptr[v], hi = g->row_ptr[v + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (g->col[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------- */
/* Plan: matching order, symmetry-breaking restrictions, first-edge mode.    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t k, induced, oriented, nres;
    int32_t order[OG_MAXK];          /* order[j] = pattern vertex at position j */
    uint32_t adj[OG_MAXK];           /* bit i of adj[j]: positions i and j adjacent */
    int32_t res_lo[OG_MAXRES];       /* restriction r: v[res_lo[r]] < v[res_hi[r]] */
    int32_t res_hi[OG_MAXRES];
    int64_t aut_size;                /* |Aut(P)| from the orbit-stabiliser chain */
} og_plan;

static int og_popc(uint32_t x)
{
    int c = 0;
    while (x) { c += (int)(x & 1u); x >>= 1; }
    return c;
}

/* Backtracking search: is there an automorphism g of the (reordered) pattern
 * with g(i) = i for every i in 'fixed' and g(a) = b? */
static int og_aut_exists(int k, const uint32_t *adj, uint32_t fixed, int a, int b)
{
    int g[OG_MAXK];
    int used[OG_MAXK];
    int pos = 0;
    for (int i = 0; i < k; i++) { g[i] = -1; used[i] = 0; }
    /* candidate cursor per position */
    int cur[OG_MAXK];
    for (int i = 0; i < k; i++) cur[i] = -1;
    while (pos >= 0) {
        if (pos == k) return 1;
        /* release previous choice at this position */
        if (g[pos] >= 0) { used[g[pos]] = 0; g[pos] = -1; }
        int next = -1;
        for (int c = cur[pos] + 1; c < k; c++) {
            if (used[c]) continue;
            if (((fixed >> pos) & 1u) && c != pos) continue;
            if (pos == a && c != b) continue;
            int ok = 1;
            for (int i = 0; i < pos && ok; i++) {
                int e1 = (int)((adj[pos] >> i) & 1u);
                int e2 = (int)((adj[c] >> g[i]) & 1u);
                if (e1 != e2) ok = 0;
            }
            if (!ok) continue;
            next = c;
            break;
        }
        if (next < 0) {
            cur[pos] = -1;
            pos--;
            continue;
        }
        cur[pos] = next;
        g[pos] = next;
        used[next] = 1;
        pos++;
        if (pos < k) cur[pos] = -1;
    }
    return 0;
}

/* Build the plan for a pattern given by k and pattern adjacency bitmasks.
 * Matching order: start at the vertex of maximum degree (lowest id on ties);
 * then repeatedly append the unplaced vertex with the most edges to placed
 * vertices, ties to higher pattern degree, then lowest id.
 * Restrictions: Grochow-Kellis symmetry breaking (RECOMB 2007).  While some
 * position has a non-trivial orbit under the stabiliser of the positions fixed
 * so far, take the lowest such a, add v_a < v_b for every other b in its orbit,
 * and fix a.  First edge: oriented (m edges, v0 < v1) if a restriction links
 * positions 0 and 1, else directed (2m entries).
 * Returns 0, or -1 for a bad size, -2 for a disconnected pattern. */
int og_plan_build(int k, const uint32_t *pattern_adj, int induced, og_plan *p)
{
    memset(p, 0, sizeof(*p));
    if (k < 2 || k > OG_MAXK) return -1;
    int deg[OG_MAXK];
    for (int i = 0; i < k; i++) deg[i] = og_popc(pattern_adj[i] & ((1u << k) - 1u));
    int placed[OG_MAXK] = {0};
    int order[OG_MAXK];
    int best = 0;
    for (int i = 1; i < k; i++)
        if (deg[i] > deg[best]) best = i;
    order[0] = best;
    placed[best] = 1;
    for (int j = 1; j < k; j++) {
        int pick = -1, pick_links = -1;
        for (int c = 0; c < k; c++) {
            if (placed[c]) continue;
            int links = 0;
            for (int i = 0; i < j; i++) links += (int)((pattern_adj[c] >> order[i]) & 1u);
            if (links == 0) continue;
            if (pick < 0 || links > pick_links ||
                (links == pick_links && deg[c] > deg[pick])) {
                pick = c;
                pick_links = links;
            }
        }
        if (pick < 0) return -2;
        order[j] = pick;
        placed[pick] = 1;
    }
    p->k = k;
    p->induced = induced ? 1 : 0;
    for (int j = 0; j < k; j++) {
        p->order[j] = order[j];
        uint32_t m = 0;
        for (int i = 0; i < k; i++)
            if ((pattern_adj[order[j]] >> order[i]) & 1u) m |= 1u << i;
        p->adj[j] = m;
    }
    uint32_t fixed = 0;
    int64_t aut = 1;
    for (;;) {
        int a_sel = -1;
        for (int a = 0; a < k && a_sel < 0; a++) {
            if ((fixed >> a) & 1u) continue;
            for (int b = 0; b < k; b++) {
                if (b == a) continue;
                if (og_aut_exists(k, p->adj, fixed, a, b)) { a_sel = a; break; }
            }
        }
        if (a_sel < 0) break;
        int orbit = 1;
        for (int b = 0; b < k; b++) {
            if (b == a_sel) continue;
            if (og_aut_exists(k, p->adj, fixed, a_sel, b)) {
                if (b < a_sel || p->nres >= OG_MAXRES) return -3; /* cannot happen */
                p->res_lo[p->nres] = a_sel;
                p->res_hi[p->nres] = b;
                p->nres++;
                orbit++;
            }
        }
        aut *= orbit;
        fixed |= 1u << a_sel;
    }
    p->aut_size = aut;
    p->oriented = 0;
    for (int r = 0; r < p->nres; r++)
        if (p->res_lo[r] == 0 && p->res_hi[r] == 1) p->oriented = 1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sampler (Algorithm 4 generalised; Lemma 1).                              */
/* ------------------------------------------------------------------------- */
enum { OG_INTERSECT = 0, OG_CHECK = 1, OG_LEARNED = 2, OG_LAZY = 3 };

typedef struct {
    uint64_t factor[OG_MAXK];  /* factor[0] = M; factor[j] = |S_j| (|L_j|, or A) */
    uint64_t w_u64;            /* exact weight (uniform modes), 0 on a miss */
    double w_f64;              /* left-to-right FP64 product, 0 on a miss */
    uint32_t vert[OG_MAXK];    /* matched vertices, 0xFFFFFFFF beyond depth */
    uint32_t aux[OG_MAXK];     /* learned mode: a_x of the chosen vertex */
    uint8_t hit, depth, overflow, pad[5];
} og_record;

typedef struct {
    const uint16_t *w1, *b1, *w2, *b2, *w3, *b3;  /* BF16 bit patterns */
} og_mlp;

/* lower bound at position j: x must exceed v[a] for each restriction (a, j) */
static int og_lower(const og_plan *p, const uint32_t *v, int j, uint32_t *lo)
{
    int has = 0;
    for (int r = 0; r < p->nres; r++) {
        if (p->res_hi[r] != j) continue;
        uint32_t b = v[p->res_lo[r]];
        if (!has || b > *lo) *lo = b;
        has = 1;
    }
    return has;
}

/* every condition of S_j (the candidate set) for vertex x */
static int og_member(const og_graph *g, const og_plan *p, const uint32_t *v, int j, uint32_t x)
{
    for (int i = 0; i < j; i++)
        if (v[i] == x) return 0;
    uint32_t lo;
    if (og_lower(p, v, j, &lo) && x <= lo) return 0;
    for (int i = 0; i < j; i++) {
        int edge = (int)((p->adj[j] >> i) & 1u);
        if (edge && !og_adjacent(g, v[i], x)) return 0;
        if (!edge && p->induced && og_adjacent(g, v[i], x)) return 0;
    }
    return 1;
}

static int og_first_back(const og_plan *p, int j)
{
    for (int i = 0; i < j; i++)
        if ((p->adj[j] >> i) & 1u) return i;
    return -1;
}

static int og_last_back(const og_plan *p, int j)
{
    for (int i = j - 1; i >= 0; i--)
        if ((p->adj[j] >> i) & 1u) return i;
    return -1;
}

/* S_j written ascending into out; returns |S_j|. */
static uint64_t og_cand(const og_graph *g, const og_plan *p, const uint32_t *v, int j, uint32_t *out)
{
    int b0 = og_first_back(p, j);
    uint32_t u = v[b0];
    uint64_t cnt = 0;
    for (uint64_t i = g->row_ptr[u]; i < g->row_ptr[u + 1]; i++) {
        uint32_t x = g->col[i];
        if (og_member(g, p, v, j, x)) {
            if (out) out[cnt] = x;
            cnt++;
        }
    }
    return cnt;
}

/* NS-base (Sec. 2.2.1, Algorithm 1; the lazy verify of Sec. 4.2): the
 * candidates of position j are the union of its back-neighbours' lists,
 * U_j = N(v_a) u N(v_b) u ... (the paper's 4-cycle example draws v3 from
 * N(v0) u N(v2)), with no other condition.  Order: the back-neighbours by
 * position ascending; the first one's list in full, then each later list's
 * entries that no earlier list holds, each list in ascending order.
 * Written into out; returns |U_j|. */
static uint64_t og_union(const og_graph *g, const og_plan *p, const uint32_t *v, int j, uint32_t *out)
{
    uint64_t cnt = 0;
    for (int i = 0; i < j; i++) {
        if (!((p->adj[j] >> i) & 1u)) continue;
        for (uint64_t e = g->row_ptr[v[i]]; e < g->row_ptr[v[i] + 1]; e++) {
            uint32_t x = g->col[e];
            int seen = 0;
            for (int q = 0; q < i; q++)
                if (((p->adj[j] >> q) & 1u) && og_adjacent(g, v[q], x)) seen = 1;
            if (seen) continue;
            if (out) out[cnt] = x;
            cnt++;
        }
    }
    return cnt;
}

/* The closure check NS-base defers to the end of a sample: the k drawn
 * vertices are distinct, every pattern edge is a graph edge, every pattern
 * non-edge is a non-edge when vertex-induced, and every symmetry-breaking
 * restriction holds. */
static int og_closure(const og_graph *g, const og_plan *p, const uint32_t *v)
{
    for (int j = 1; j < p->k; j++)
        for (int i = 0; i < j; i++) {
            if (v[i] == v[j]) return 0;
            int edge = (int)((p->adj[j] >> i) & 1u);
            int adj = og_adjacent(g, v[i], v[j]);
            if (edge && !adj) return 0;
            if (!edge && p->induced && adj) return 0;
        }
    for (int r = 0; r < p->nres; r++)
        if (!(v[p->res_lo[r]] < v[p->res_hi[r]])) return 0;
    return 1;
}

/* Map the first-edge index e to (v0, v1). */
static void og_first_edge(const og_graph *g, const og_plan *p, uint64_t e, uint32_t *v0, uint32_t *v1)
{
    if (p->oriented) {
        /* canonical oriented enumeration: u ascending, then N+(u) ascending */
        uint64_t lo = 0, hi = g->n;  /* find u with uoff[u] <= e < uoff[u+1] */
        while (hi - lo > 1) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (g->uoff[mid] <= e) lo = mid;
            else hi = mid;
        }
        uint64_t u = lo;
        while (g->uoff[u + 1] <= e) u++;   /* skip vertices with empty N+ */
        *v0 = (uint32_t)u;
        *v1 = g->col[g->up[u] + (e - g->uoff[u])];
    } else {
        uint64_t lo = 0, hi = g->n;
        while (hi - lo > 1) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (g->row_ptr[mid] <= e) lo = mid;
            else hi = mid;
        }
        uint64_t u = lo;
        while (g->row_ptr[u + 1] <= e) u++;
        *v0 = (uint32_t)u;
        *v1 = g->col[e];
    }
}

/* Feature log2(1 + d), piecewise linear between powers of two, in FP32:
 * e + (y - 2^e) / 2^e with y = d + 1 and e = floor(log2 y). */
float og_flog2p1(uint64_t d)
{
    uint64_t y = d + 1;
    int e = 63;
    while (!((y >> e) & 1u)) e--;
    float base = (float)(1ull << e);
    float frac = (float)(y - (1ull << e)) / base;
    return (float)e + frac;
}

static float og_bf16(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* Learned proposal (not in the paper): at step j <= k-2 with 0 < |S_j| <= 256
 * each candidate x gets the integer score a_x from the MLP below on the
 * features (log2(1 + d(x)), j, log2(1 + |S_{j+1}(x)|)), where S_{j+1}(x) is the
 * next candidate set if x were chosen; x is drawn with probability a_x / A,
 * A = sum of the scores (the integer CDF in candidate order), and the weight
 * takes the factor A / a_x.  Every a_x >= 1, so each match keeps a positive
 * probability whose inverse is its weight (Lemma 1's argument).  Larger sets,
 * and the last step, are drawn uniformly. */

/* MLP 3 -> 64 -> 64 -> 1 with ReLU, BF16 weights, FP32 FMA chains in input
 * order; the output z is mapped to a score without exp: s = clamp(z/8 + 1/2),
 * a = 1 + floor(4096 s) in [1, 4097]. */
float og_mlp_logit(const og_mlp *mlp, const float f[3])
{
    float h1[64], h2[64];
    for (int o = 0; o < 64; o++) {
        float acc = og_bf16(mlp->b1[o]);
        for (int i = 0; i < 3; i++) acc = fmaf(og_bf16(mlp->w1[o * 3 + i]), f[i], acc);
        h1[o] = acc > 0.f ? acc : 0.f;
    }
    for (int o = 0; o < 64; o++) {
        float acc = og_bf16(mlp->b2[o]);
        for (int i = 0; i < 64; i++) acc = fmaf(og_bf16(mlp->w2[o * 64 + i]), h1[i], acc);
        h2[o] = acc > 0.f ? acc : 0.f;
    }
    float z = og_bf16(mlp->b3[0]);
    for (int i = 0; i < 64; i++) z = fmaf(og_bf16(mlp->w3[i]), h2[i], z);
    return z;
}

uint32_t og_score(float z)
{
    float s = fmaf(z, 0.125f, 0.5f);
    if (!(s > 0.f)) s = 0.f;
    if (s > 1.f) s = 1.f;
    return 1u + (uint32_t)floorf(s * 4096.0f);
}

/* One sample from its choice words r[0..k-2].  'buf' must hold OG_MAXK times
 * (max degree + 1) entries (an NS-base union spans up to k - 1 lists), 'buf2'
 * too (learned mode lookahead). */
int og_sample(const og_graph *g, const og_plan *p, const uint64_t *r, int mode,
              const og_mlp *mlp, uint32_t *buf, uint32_t *buf2, og_record *rec)
{
    memset(rec, 0, sizeof(*rec));
    for (int j = 0; j < OG_MAXK; j++) rec->vert[j] = 0xFFFFFFFFu;
    uint32_t v[OG_MAXK];
    /* NS-base draws the first edge from all 2m directed entries: the
     * restriction between v0 and v1, like every other, waits for the closure */
    int oriented = (mode == OG_LAZY) ? 0 : p->oriented;
    uint64_t M = oriented ? og_graph_m(g) : g->nnz;
    rec->factor[0] = M;
    if (M == 0) {
        rec->depth = 0;
        return 0;
    }
    uint64_t e = og_index_map(r[0], M);
    if (oriented) {
        og_first_edge(g, p, e, &v[0], &v[1]);
    } else {
        og_plan q = *p;
        q.oriented = 0;
        og_first_edge(g, &q, e, &v[0], &v[1]);
    }
    rec->vert[0] = v[0];
    rec->vert[1] = v[1];
    double w = (double)M;
    uint64_t wu = M;
    int overflow = 0;
    for (int j = 2; j < p->k; j++) {
        uint64_t size, pick;
        uint32_t x;
        if (mode == OG_LAZY) {
            size = og_union(g, p, v, j, buf);      /* never empty: v_a has a neighbour */
            rec->factor[j] = size;
            pick = og_index_map(r[j - 1], size);
            x = buf[pick];
            w = w * (double)size;
            if (__builtin_mul_overflow(wu, size, &wu)) overflow = 1;
        } else if (mode == OG_CHECK) {
            int pb = og_last_back(p, j);
            uint32_t lo = 0;
            int has = og_lower(p, v, j, &lo);
            uint64_t start = has ? og_first_above(g, v[pb], lo) : g->row_ptr[v[pb]];
            size = g->row_ptr[v[pb] + 1] - start;
            if (size == 0) { rec->depth = (uint8_t)j; return 0; }
            pick = og_index_map(r[j - 1], size);
            x = g->col[start + pick];
            rec->factor[j] = size;
            if (!og_member(g, p, v, j, x)) { rec->depth = (uint8_t)j; return 0; }
            w = w * (double)size;
            if (__builtin_mul_overflow(wu, size, &wu)) overflow = 1;
        } else if (mode == OG_LEARNED && j <= p->k - 2 &&
                   og_cand(g, p, v, j, NULL) <= OG_LEARNED_MAX) {
            size = og_cand(g, p, v, j, buf);
            rec->factor[j] = 0;
            if (size == 0) { rec->depth = (uint8_t)j; return 0; }
            uint64_t A = 0;
            for (uint64_t i = 0; i < size; i++) {
                v[j] = buf[i];
                float f[3];
                f[0] = og_flog2p1(og_deg(g, buf[i]));
                f[1] = (float)j;
                f[2] = og_flog2p1(og_cand(g, p, v, j + 1, NULL));
                buf2[i] = og_score(og_mlp_logit(mlp, f));
                A += buf2[i];
            }
            uint64_t t = og_index_map(r[j - 1], A);
            uint64_t acc = 0;
            pick = 0;
            for (uint64_t i = 0; i < size; i++) {
                acc += buf2[i];
                if (acc > t) { pick = i; break; }
            }
            x = buf[pick];
            rec->factor[j] = A;
            rec->aux[j] = buf2[pick];
            w = w * ((double)A / (double)buf2[pick]);
            wu = 0;
        } else {
            size = og_cand(g, p, v, j, buf);
            rec->factor[j] = size;
            if (size == 0) { rec->depth = (uint8_t)j; return 0; }
            pick = og_index_map(r[j - 1], size);
            x = buf[pick];
            w = w * (double)size;
            if (mode != OG_LEARNED) {
                if (__builtin_mul_overflow(wu, size, &wu)) overflow = 1;
            }
        }
        v[j] = x;
        rec->vert[j] = x;
    }
    rec->depth = (uint8_t)p->k;
    if (mode == OG_LAZY && !og_closure(g, p, v)) return 0;   /* a miss after all k draws */
    rec->hit = 1;
    rec->w_f64 = w;
    rec->w_u64 = (mode == OG_LEARNED) ? 0 : (overflow ? 0 : wu);
    rec->overflow = (uint8_t)overflow;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Algorithmic bytes of one sample: 32-byte sectors of graph data that the   */
/* candidate-set definition references on the path actually taken.          */
/*   first edge: 1 sector; each step j: per referenced list, 1 sector for its */
/*   row_ptr pair plus the sectors spanned by its part above the lower bound. */
/*   A step whose back-neighbours are those of step j-1 plus j-1 (and whose   */
/*   bounds extend those of j-1) reads only N(v_{j-1}), S_{j-1} being on chip. */
/*   CHECK mode: the drawn element's sector plus a binary search (ceil(log2)) */
/*   per other referenced list.                                               */
/* ------------------------------------------------------------------------- */
static int og_step_reuses(const og_plan *p, int j)
{
    if (j < 3) return 0;
    uint32_t below = (1u << (j - 1)) - 1u;
    if ((p->adj[j] & below) != (p->adj[j - 1] & below)) return 0;
    if (!((p->adj[j] >> (j - 1)) & 1u)) return 0;
    /* every lower bound of j-1 must also be a lower bound of j */
    for (int r = 0; r < p->nres; r++) {
        if (p->res_hi[r] != j - 1) continue;
        int found = 0;
        for (int q = 0; q < p->nres; q++)
            if (p->res_hi[q] == j && p->res_lo[q] == p->res_lo[r]) found = 1;
        if (!found) return 0;
    }
    return 1;
}

static double og_sectors(uint64_t begin, uint64_t end)
{
    if (end <= begin) return 0.0;
    uint64_t b = (begin * 4) / 32, e = (end * 4 + 31) / 32;
    return (double)(e - b);
}

static double og_log2ceil(uint64_t n)
{
    int c = 0;
    while ((1ull << c) < n + 1) c++;
    return (double)c;
}

double og_sample_bytes(const og_graph *g, const og_plan *p, int mode, const og_record *rec)
{
    double sec = 1.0;
    if (mode == OG_LAZY) {
        /* NS-base: each step reads its back-neighbours' lists in full; the
         * closure reads one binary search per checked pair (i, j) */
        if (rec->depth < p->k) return 32.0 * sec;
        for (int j = 2; j < p->k; j++)
            for (int i = 0; i < j; i++)
                if ((p->adj[j] >> i) & 1u) sec += 1.0 + og_sectors(g->row_ptr[rec->vert[i]], g->row_ptr[rec->vert[i] + 1]);
        for (int j = 1; j < p->k; j++)
            for (int i = 0; i < j; i++) {
                int edge = (int)((p->adj[j] >> i) & 1u);
                if (edge || p->induced) sec += 1.0 + og_log2ceil(og_deg(g, rec->vert[i]));
            }
        return 32.0 * sec;
    }
    int steps = rec->hit ? p->k : rec->depth + 1;
    uint32_t v[OG_MAXK];
    for (int i = 0; i < OG_MAXK; i++) v[i] = rec->vert[i];
    for (int j = 2; j < steps && j < p->k; j++) {
        uint32_t lo = 0;
        int has = og_lower(p, v, j, &lo);
        if (mode == OG_CHECK) {
            int pb = og_last_back(p, j);
            sec += 1.0;                                       /* row_ptr pair of v_pb */
            if (has) sec += og_log2ceil(og_deg(g, v[pb]));    /* locate the bound */
            if (rec->factor[j] == 0) continue;                /* L_j empty */
            sec += 1.0;                                       /* the drawn element */
            for (int i = 0; i < j; i++) {
                int edge = (int)((p->adj[j] >> i) & 1u);
                if (i == pb || (!edge && !p->induced)) continue;
                sec += 1.0 + og_log2ceil(og_deg(g, v[i]));
            }
            continue;
        }
        for (int i = 0; i < j; i++) {
            int edge = (int)((p->adj[j] >> i) & 1u);
            if (!edge && !p->induced) continue;
            if (og_step_reuses(p, j) && i != j - 1) continue;
            uint64_t b = has ? og_first_above(g, v[i], lo) : g->row_ptr[v[i]];
            sec += 1.0 + og_sectors(b, g->row_ptr[v[i] + 1]);
        }
    }
    return 32.0 * sec;
}

/* ------------------------------------------------------------------------- */
/* Fixed-count runs and traces (Algorithm 3's inner loop).                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint64_t n, hits;
    double sum, sumsq;         /* sum X_i and sum X_i^2, index order, FP64 */
    double bytes;              /* sum of algorithmic bytes */
} og_sums;

static uint64_t og_maxdeg(const og_graph *g)
{
    uint64_t d = 0;
    for (uint64_t v = 0; v < g->n; v++)
        if (og_deg(g, (uint32_t)v) > d) d = og_deg(g, (uint32_t)v);
    return d;
}

int og_ns_run(const og_graph *g, const og_plan *p, int mode, const og_mlp *mlp,
              uint64_t seed, uint32_t slot, uint64_t first, uint64_t count,
              og_sums *acc, og_record *recs, int want_bytes)
{
    uint64_t md = (og_maxdeg(g) + 1) * OG_MAXK;   /* NS-base unions span several lists */
    uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * md);
    uint32_t *buf2 = (uint32_t *)malloc(sizeof(uint32_t) * md);
    if (!buf || !buf2) { free(buf); free(buf2); return -1; }
    for (uint64_t s = first; s < first + count; s++) {
        uint64_t r[OG_MAXK];
        for (int t = 0; t + 1 < p->k; t++) r[t] = og_choice_word(seed, s, slot, 0, (uint32_t)t);
        og_record rec;
        og_sample(g, p, r, mode, mlp, buf, buf2, &rec);
        double x = rec.hit ? rec.w_f64 : 0.0;
        acc->n += 1;
        acc->hits += rec.hit;
        acc->sum += x;
        acc->sumsq += x * x;
        if (want_bytes) acc->bytes += og_sample_bytes(g, p, mode, &rec);
        if (recs) recs[s - first] = rec;
    }
    free(buf);
    free(buf2);
    return 0;
}

/* Mean and M2 (sum of squared deviations) of samples [first, first+count) by
 * Welford's update in sample order (Welford 1962): the numerically stable
 * counterpart of Algorithm 3's running sum and squared sum, for the
 * cross-check var = sumsq / n - mu^2 = M2 / n. */
int og_welford_run(const og_graph *g, const og_plan *p, int mode, const og_mlp *mlp,
                   uint64_t seed, uint32_t slot, uint64_t first, uint64_t count, double *mean, double *m2)
{
    uint64_t md = (og_maxdeg(g) + 1) * OG_MAXK;
    uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * md);
    uint32_t *buf2 = (uint32_t *)malloc(sizeof(uint32_t) * md);
    if (!buf || !buf2) { free(buf); free(buf2); return -1; }
    double mu = 0.0, q = 0.0;
    uint64_t n = 0;
    for (uint64_t s = first; s < first + count; s++) {
        uint64_t r[OG_MAXK];
        for (int t = 0; t + 1 < p->k; t++) r[t] = og_choice_word(seed, s, slot, 0, (uint32_t)t);
        og_record rec;
        og_sample(g, p, r, mode, mlp, buf, buf2, &rec);
        double x = rec.hit ? rec.w_f64 : 0.0;
        n++;
        double d = x - mu;
        mu += d / (double)n;
        q += d * (x - mu);
    }
    free(buf);
    free(buf2);
    *mean = mu;
    *m2 = q;
    return 0;
}

/* Per-sample algorithmic bytes of samples [first, first+count) into out. */
int og_ns_bytes(const og_graph *g, const og_plan *p, int mode, const og_mlp *mlp,
                uint64_t seed, uint32_t slot, uint64_t first, uint64_t count, double *out)
{
    uint64_t md = (og_maxdeg(g) + 1) * OG_MAXK;   /* NS-base unions span several lists */
    uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * md);
    uint32_t *buf2 = (uint32_t *)malloc(sizeof(uint32_t) * md);
    if (!buf || !buf2) { free(buf); free(buf2); return -1; }
    for (uint64_t s = first; s < first + count; s++) {
        uint64_t r[OG_MAXK];
        for (int t = 0; t + 1 < p->k; t++) r[t] = og_choice_word(seed, s, slot, 0, (uint32_t)t);
        og_record rec;
        og_sample(g, p, r, mode, mlp, buf, buf2, &rec);
        out[s - first] = og_sample_bytes(g, p, mode, &rec);
    }
    free(buf);
    free(buf2);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Inverse standard normal CDF: Wichura, Algorithm AS 241 (PPND16),          */
/* Applied Statistics 37(3), 1988.  Rational approximations in three regions. */
/* ------------------------------------------------------------------------- */
static double og_poly(const double *c, int n, double x)
{
    double r = 0.0;
    for (int i = n - 1; i >= 0; i--) r = r * x + c[i];
    return r;
}

double og_phi_inv(double p)
{
    static const double a[8] = {3.3871328727963666080e0, 1.3314166789178437745e2,
                                1.9715909503065514427e3, 1.3731693765509461125e4,
                                4.5921953931549871457e4, 6.7265770927008700853e4,
                                3.3430575583588128105e4, 2.5090809287301226727e3};
    static const double b[8] = {1.0, 4.2313330701600911252e1, 6.8718700749205790830e2,
                                5.3941960214247511077e3, 2.1213794301586595867e4,
                                3.9307895800092710610e4, 2.8729085735721942674e4,
                                5.2264952788528545610e3};
    static const double c[8] = {1.42343711074968357734e0, 4.63033784615654529590e0,
                                5.76949722146069140550e0, 3.64784832476320460504e0,
                                1.27045825245236838258e0, 2.41780725177450611770e-1,
                                2.27238449892691845833e-2, 7.74545014278341407640e-4};
    static const double d[8] = {1.0, 2.05319162663775882187e0, 1.67638483018380384940e0,
                                6.89767334985100004550e-1, 1.48103976427480074590e-1,
                                1.51986665636164571966e-2, 5.47593808499534494600e-4,
                                1.05075007164441684324e-9};
    static const double e[8] = {6.65790464350110377720e0, 5.46378491116411436990e0,
                                1.78482653991729133580e0, 2.96560571828504891230e-1,
                                2.65321895265761230930e-2, 1.24266094738807843860e-3,
                                2.71155556874348757815e-5, 2.01033439929228813265e-7};
    static const double f[8] = {1.0, 5.99832206555887937690e-1, 1.36929880922735805310e-1,
                                1.48753612908506148525e-2, 7.86869131145613259100e-4,
                                1.84631831751005468180e-5, 1.42151175831644588870e-7,
                                2.04426310338993978564e-15};
    if (!(p > 0.0 && p < 1.0)) return NAN;
    double q = p - 0.5;
    if (fabs(q) <= 0.425) {
        double r = 0.180625 - q * q;
        return q * og_poly(a, 8, r) / og_poly(b, 8, r);
    }
    double r = q < 0 ? p : 1.0 - p;
    r = sqrt(-log(r));
    double val;
    if (r <= 5.0) {
        r -= 1.6;
        val = og_poly(c, 8, r) / og_poly(d, 8, r);
    } else {
        r -= 5.0;
        val = og_poly(e, 8, r) / og_poly(f, 8, r);
    }
    return q < 0 ? -val : val;
}

/* ------------------------------------------------------------------------- */
/* Online convergence detection (Algorithm 3, Eq. equ:error).               */
/* ------------------------------------------------------------------------- */
typedef struct {
    double estimate, ci_half_width, eps_hat, sum, sumsq;
    uint64_t samples, hits, rounds;
    int32_t converged, pad;
} og_online;

/* The statistics after n samples (Algorithm 3's end-of-window block). */
void og_error_of(double sum, double sumsq, uint64_t n, double z, double *mu, double *half, double *eps_hat)
{
    double m = sum / (double)n;
    double var = sumsq / (double)n - m * m;
    if (var < 0.0) var = 0.0;
    double sigma = sqrt(var / (double)n);
    *mu = m;
    *half = z * sigma;
    *eps_hat = (m > 0.0) ? z * sigma / m : INFINITY;
}

int og_ns_online(const og_graph *g, const og_plan *p, int mode, const og_mlp *mlp,
                 double eps, double delta, uint64_t seed, uint32_t slot,
                 uint64_t window, uint64_t n_min, uint64_t n_max, og_online *out)
{
    memset(out, 0, sizeof(*out));
    double z = og_phi_inv(1.0 - delta / 2.0);
    og_sums acc;
    memset(&acc, 0, sizeof(acc));
    for (;;) {
        if (og_ns_run(g, p, mode, mlp, seed, slot, acc.n, window, &acc, NULL, 0) != 0) return -1;
        out->rounds++;
        double mu, half, eh;
        og_error_of(acc.sum, acc.sumsq, acc.n, z, &mu, &half, &eh);
        out->estimate = mu;
        out->ci_half_width = half;
        out->eps_hat = eh;
        out->samples = acc.n;
        out->hits = acc.hits;
        out->sum = acc.sum;
        out->sumsq = acc.sumsq;
        if (acc.n >= n_min && mu > 0.0 && eh <= eps) { out->converged = 1; return 0; }
        if (acc.n >= n_max) { out->converged = 0; return 0; }
    }
}

/* ------------------------------------------------------------------------- */
/* GS: colour sparsification (Sec. 2.2.2, Sec. 5.2) and exact counting.      */
/* ------------------------------------------------------------------------- */
uint32_t og_color(uint64_t seed, uint64_t v, uint32_t colouring, uint32_t slot, uint32_t c)
{
    uint32_t ctr[4] = {(uint32_t)v, (uint32_t)(v >> 32), colouring, (slot << 8) | 2u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    og_philox4x32_10(ctr, key, o);
    return (uint32_t)(((uint64_t)o[0] * (uint64_t)c) >> 32);
}

/* Keep edge (u, w) iff colour(u) == colour(w).  row_out has n + 1 entries;
 * col_out must hold nnz entries; returns the kept entry count. */
uint64_t og_sparsify(const og_graph *g, const uint32_t *colors, uint64_t *row_out, uint32_t *col_out)
{
    uint64_t k = 0;
    row_out[0] = 0;
    for (uint64_t v = 0; v < g->n; v++) {
        for (uint64_t i = g->row_ptr[v]; i < g->row_ptr[v + 1]; i++) {
            uint32_t x = g->col[i];
            if (colors[v] == colors[x]) col_out[k++] = x;
        }
        row_out[v + 1] = k;
    }
    return k;
}

/* Bernoulli edge sparsification (Algorithm 2).  The keep probability p is
 * realised as t / 2^32 with t = floor(p * 2^32) (t = 2^32 for p >= 1): edge
 * {u, w} stays iff the first word of Philox4x32-10 at counter (min(u, w),
 * max(u, w), colouring, slot << 8 | 3), key = seed, is below t, so both CSR
 * entries of an edge get one decision. */
uint64_t og_bes_threshold(double p)
{
    if (p >= 1.0) return 1ull << 32;
    return (uint64_t)floor(p * 4294967296.0);
}

int og_bes_keep(uint64_t seed, uint32_t u, uint32_t w, uint32_t colouring, uint32_t slot, uint64_t t)
{
    uint32_t lo = u < w ? u : w, hi = u < w ? w : u;
    uint32_t ctr[4] = {lo, hi, colouring, (slot << 8) | 3u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    og_philox4x32_10(ctr, key, o);
    return (uint64_t)o[0] < t;
}

/* The kept CSR of one Bernoulli sparsification; same layout as og_sparsify. */
uint64_t og_bes_sparsify(const og_graph *g, uint64_t seed, uint32_t colouring, uint32_t slot, uint64_t t,
                         uint64_t *row_out, uint32_t *col_out)
{
    uint64_t k = 0;
    row_out[0] = 0;
    for (uint64_t v = 0; v < g->n; v++) {
        for (uint64_t i = g->row_ptr[v]; i < g->row_ptr[v + 1]; i++) {
            uint32_t x = g->col[i];
            if (og_bes_keep(seed, (uint32_t)v, x, colouring, slot, t)) col_out[k++] = x;
        }
        row_out[v + 1] = k;
    }
    return k;
}

/* Exact count: every branch of the same plan (nested loops over the
 * candidate sets), the last level adding |S_{k-1}|. */
static uint64_t og_exact_rec(const og_graph *g, const og_plan *p, uint32_t *v, int j, uint32_t **bufs)
{
    uint64_t size = og_cand(g, p, v, j, bufs[j]);
    if (j == p->k - 1) return size;
    uint64_t tot = 0;
    for (uint64_t i = 0; i < size; i++) {
        v[j] = bufs[j][i];
        tot += og_exact_rec(g, p, v, j + 1, bufs);
    }
    return tot;
}

uint64_t og_exact_count(const og_graph *g, const og_plan *p)
{
    uint64_t md = og_maxdeg(g) + 1;
    uint32_t *bufs[OG_MAXK];
    for (int j = 0; j < OG_MAXK; j++) bufs[j] = (uint32_t *)malloc(sizeof(uint32_t) * md);
    uint64_t M = p->oriented ? og_graph_m(g) : g->nnz;
    uint64_t tot = 0;
    uint32_t v[OG_MAXK];
    for (uint64_t e = 0; e < M; e++) {
        og_first_edge(g, p, e, &v[0], &v[1]);
        if (p->k == 2) { tot += 1; continue; }
        tot += og_exact_rec(g, p, v, 2, bufs);
    }
    for (int j = 0; j < OG_MAXK; j++) free(bufs[j]);
    return tot;
}

/* ------------------------------------------------------------------------- */
/* Learned proposal training reference: FP32 forward and backward of the     */
/* 3 -> 64 -> 64 -> 1 ReLU MLP with BCE-with-logits loss, mean over rows.    */
/* Weights are FP32 here (the trainer's master copy).                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    float w1[64 * 3], b1[64], w2[64 * 64], b2[64], w3[64], b3[1];
} og_mlp32;

double og_mlp_loss_grad(const og_mlp32 *w, const float *feat, const float *label, uint64_t rows, og_mlp32 *grad)
{
    memset(grad, 0, sizeof(*grad));
    double loss = 0.0;
    for (uint64_t r = 0; r < rows; r++) {
        const float *f = feat + 3 * r;
        float a1[64], h1[64], a2[64], h2[64];
        for (int o = 0; o < 64; o++) {
            float acc = w->b1[o];
            for (int i = 0; i < 3; i++) acc += w->w1[o * 3 + i] * f[i];
            a1[o] = acc;
            h1[o] = acc > 0.f ? acc : 0.f;
        }
        for (int o = 0; o < 64; o++) {
            float acc = w->b2[o];
            for (int i = 0; i < 64; i++) acc += w->w2[o * 64 + i] * h1[i];
            a2[o] = acc;
            h2[o] = acc > 0.f ? acc : 0.f;
        }
        float z = w->b3[0];
        for (int i = 0; i < 64; i++) z += w->w3[i] * h2[i];
        double y = label[r];
        /* softplus(z) - y z, written to avoid overflow */
        double zd = z;
        loss += (zd > 0 ? zd : 0.0) - y * zd + log1p(exp(-fabs(zd)));
        float dz = (float)((1.0 / (1.0 + exp(-zd)) - y) / (double)rows);
        grad->b3[0] += dz;
        float dh2[64], dh1[64];
        for (int i = 0; i < 64; i++) {
            grad->w3[i] += dz * h2[i];
            dh2[i] = dz * w->w3[i];
        }
        for (int i = 0; i < 64; i++) dh1[i] = 0.f;
        for (int o = 0; o < 64; o++) {
            float da = a2[o] > 0.f ? dh2[o] : 0.f;
            grad->b2[o] += da;
            for (int i = 0; i < 64; i++) {
                grad->w2[o * 64 + i] += da * h1[i];
                dh1[i] += da * w->w2[o * 64 + i];
            }
        }
        for (int o = 0; o < 64; o++) {
            float da = a1[o] > 0.f ? dh1[o] : 0.f;
            grad->b1[o] += da;
            for (int i = 0; i < 3; i++) grad->w1[o * 3 + i] += da * f[i];
        }
    }
    return loss / (double)rows;
}

/* sizes for the binding to check its struct mirrors */
uint64_t og_sizeof_plan(void) { return sizeof(og_plan); }
uint64_t og_sizeof_record(void) { return sizeof(og_record); }
uint64_t og_sizeof_online(void) { return sizeof(og_online); }
uint64_t og_sizeof_sums(void) { return sizeof(og_sums); }
