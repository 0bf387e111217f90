// Host-side pattern planner of libgpm: matching order, symmetry-breaking
// restrictions and the first-edge mode.
//
// Eager verify needs a fixed matching order in which every vertex after the
// first has an earlier pattern neighbour, and a restriction set under which
// each match maps to exactly one k-tuple (Sec. 4.2, Lemma 1; the paper uses the
// matching orders and symmetry breaking of GraphZero / G2Miner).
//
// Order rule: begin at the pattern vertex of largest degree (lowest id on
// ties); then keep appending the unplaced vertex with the most edges into the
// placed set, ties to larger pattern degree, then lowest id.
//
// Restrictions: Grochow-Kellis symmetry breaking.  The automorphism group of
// the reordered pattern is enumerated once; while some position has an orbit
// of size > 1 under the current group, the lowest such position a gets
// v_a < v_b for every other b of its orbit and the group shrinks to the
// stabiliser of a.  For a clique this yields v_0 < v_1 < ... < v_{k-1}.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace gpm {

namespace {

struct AutSearch {
    int k;
    uint32_t adj[kMaxK];
    std::vector<std::vector<int8_t>> found;
    int8_t map[kMaxK];
    bool used[kMaxK];

    void run(int pos) {
        if (pos == k) {
            found.emplace_back(map, map + k);
            return;
        }
        for (int c = 0; c < k; c++) {
            if (used[c]) continue;
            bool ok = true;
            for (int i = 0; i < pos && ok; i++) {
                bool e1 = (adj[pos] >> i) & 1u;
                bool e2 = (adj[c] >> map[i]) & 1u;
                ok = (e1 == e2);
            }
            if (!ok) continue;
            used[c] = true;
            map[pos] = (int8_t)c;
            run(pos + 1);
            used[c] = false;
        }
    }
};

}  // namespace

std::string build_plan(const gpm_pattern &pat, Plan *out) {
    std::memset(out, 0, sizeof(*out));
    const int k = pat.k;
    if (k < 2 || k > GPM_MAX_PATTERN_K) return "pattern size k must be in [2, 10]";
    uint32_t full = (1u << k) - 1u;
    for (int i = 0; i < k; i++) {
        if ((pat.adj[i] >> i) & 1u) return "pattern has a self loop";
        if (pat.adj[i] & ~full) return "pattern adjacency names a vertex >= k";
        for (int j = 0; j < k; j++)
            if (((pat.adj[i] >> j) & 1u) != ((pat.adj[j] >> i) & 1u)) return "pattern adjacency is not symmetric";
    }
    int deg[kMaxK];
    for (int i = 0; i < k; i++) deg[i] = __builtin_popcount(pat.adj[i]);

    std::vector<int> order;
    std::vector<bool> placed(k, false);
    int start = 0;
    for (int i = 1; i < k; i++)
        if (deg[i] > deg[start]) start = i;
    order.push_back(start);
    placed[start] = true;
    while ((int)order.size() < k) {
        int best = -1, best_links = 0;
        for (int c = 0; c < k; c++) {
            if (placed[c]) continue;
            int links = 0;
            for (int u : order) links += (pat.adj[c] >> u) & 1u;
            if (links == 0) continue;
            bool better = best < 0 || links > best_links || (links == best_links && deg[c] > deg[best]);
            if (better) {
                best = c;
                best_links = links;
            }
        }
        if (best < 0) return "pattern is not connected";
        order.push_back(best);
        placed[best] = true;
    }

    out->k = k;
    out->induced = pat.induced ? 1 : 0;
    AutSearch as;
    as.k = k;
    for (int j = 0; j < k; j++) {
        out->order[j] = order[j];
        uint32_t m = 0;
        for (int i = 0; i < k; i++)
            if ((pat.adj[order[j]] >> order[i]) & 1u) m |= 1u << i;
        as.adj[j] = m;
        out->back[j] = m & ((1u << j) - 1u);
        out->nonback[j] = (~m) & ((1u << j) - 1u);
        out->last_back[j] = 0;
        for (int i = 0; i < j; i++)
            if ((m >> i) & 1u) out->last_back[j] = (uint32_t)i;
    }
    for (int i = 0; i < k; i++) as.used[i] = false;
    as.run(0);

    std::vector<std::vector<int8_t>> group = as.found;
    int nres = 0;
    for (;;) {
        int a = -1;
        for (int pos = 0; pos < k && a < 0; pos++)
            for (const auto &g : group)
                if (g[pos] != pos) {
                    a = pos;
                    break;
                }
        if (a < 0) break;
        std::vector<bool> in_orbit(k, false);
        for (const auto &g : group) in_orbit[g[a]] = true;
        for (int b = 0; b < k; b++) {
            if (b == a || !in_orbit[b]) continue;
            if (b < a || nres >= 64) return "internal: restriction order";
            out->res_lo[nres] = a;
            out->res_hi[nres] = b;
            out->lower[b] |= 1u << a;
            nres++;
        }
        std::vector<std::vector<int8_t>> stab;
        for (const auto &g : group)
            if (g[a] == a) stab.push_back(g);
        group.swap(stab);
    }
    out->nres = nres;
    out->oriented = (out->lower[1] & 1u) ? 1 : 0;
    for (int j = 0; j < k; j++) {
        out->reuse[j] = 0;
        if (j < 3) continue;
        uint32_t below = (1u << (j - 1)) - 1u;
        bool same = ((as.adj[j] & below) == (as.adj[j - 1] & below));
        bool links = (as.adj[j] >> (j - 1)) & 1u;
        bool bounds = (out->lower[j] & out->lower[j - 1]) == out->lower[j - 1];
        // S_j is S_{j-1} (same adjacency to every earlier position, bounds that
        // only grow) cut by N(v_{j-1}): kept if adjacent (1), removed if the
        // count is vertex-induced (2), else only filtered by the bounds (3)
        if (same && bounds) out->reuse[j] = links ? 1u : (pat.induced ? 2u : 3u);
    }
    return "";
}

}  // namespace gpm
