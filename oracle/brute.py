"""Brute-force subgraph counting on tiny graphs (test infrastructure only).

This is the plain definition of the quantity every estimator targets: the
number of edge-induced (or vertex-induced) subgraphs of G isomorphic to P
(problem statement of Sec. 2.1; vertex-induced counting for motifs, Sec. 6).
It counts injective maps f: V(P) -> V(G) that keep every pattern edge (and,
if induced, every pattern non-edge) and divides by |Aut(P)|.  It uses no plan,
no matching order and no symmetry breaking, so it is independent of the
oracle's sampler.  Pure-Python loops: graphs of at most a dozen vertices.
"""
import itertools


def adjacency_sets(row_ptr, col):
    n = len(row_ptr) - 1
    return [set(int(x) for x in col[row_ptr[v]:row_ptr[v + 1]]) for v in range(n)]


def automorphisms(k, edges):
    es = {frozenset(e) for e in edges}
    count = 0
    for perm in itertools.permutations(range(k)):
        if all(frozenset((perm[a], perm[b])) in es for a, b in edges):
            count += 1
    return count


def count_embeddings(adj, k, edges, induced=False):
    n = len(adj)
    es = {frozenset(e) for e in edges}
    non_edges = [(a, b) for a in range(k) for b in range(a + 1, k) if frozenset((a, b)) not in es]
    total = 0
    for f in itertools.permutations(range(n), k):
        if any(f[b] not in adj[f[a]] for a, b in edges):
            continue
        if induced and any(f[b] in adj[f[a]] for a, b in non_edges):
            continue
        total += 1
    return total


def count(row_ptr, col, k, edges, induced=False):
    adj = adjacency_sets(row_ptr, col)
    emb = count_embeddings(adj, k, edges, induced)
    aut = automorphisms(k, edges)
    assert emb % aut == 0
    return emb // aut


def matches(row_ptr, col, k, edges, induced=False):
    """The set of matches, each as (frozenset of vertices, frozenset of edges)."""
    adj = adjacency_sets(row_ptr, col)
    n = len(adj)
    es = {frozenset(e) for e in edges}
    non_edges = [(a, b) for a in range(k) for b in range(a + 1, k) if frozenset((a, b)) not in es]
    out = set()
    for f in itertools.permutations(range(n), k):
        if any(f[b] not in adj[f[a]] for a, b in edges):
            continue
        if induced and any(f[b] in adj[f[a]] for a, b in non_edges):
            continue
        out.add((frozenset(f), frozenset(frozenset((f[a], f[b])) for a, b in edges)))
    return out
