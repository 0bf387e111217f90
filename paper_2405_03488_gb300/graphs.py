"""Seeded synthetic input graphs.

This module only synthesises data graphs in CSR form; it holds none of the
estimator's arithmetic, and both the CUDA path and the CPU oracle consume its
output.  The paper evaluates on SNAP / LAW / ClueWeb graphs (Table tab:input),
which are not available offline; these generators stand in for them with the
same structure (power-law degrees from R-MAT and Chung-Lu, a uniform G(n, p)
baseline, planted dense regions for the needle-in-the-hay case).

Every graph is returned as a symmetric CSR without self-loops or duplicate
edges, with sorted neighbour lists (the paper's layout, Sec. 6): ``row_ptr``
int64 [n + 1] and ``col`` int32 [2m].  ``relabel_by_degree`` renumbers vertices
by (degree, id) ascending, the orientation used for cliques (Table tab:input
caption: orientation is applied for cliques; the ordering is this project's
reading).

Randomness comes from ``torch.Generator`` seeded with the config's seed on the
device that runs the generator; a given (seed, device) pair always yields the
same graph.
"""
import math

import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


_UNIQUE_LIMIT = 1 << 31


def _unique(keys, n):
    """Sorted unique keys s * n + d; above 2^31 entries (the sort library's
    size limit) the keys are split at source vertices chosen so that every part
    holds about the same number of entries, and each part is made unique."""
    if keys.numel() < _UNIQUE_LIMIT:
        return torch.unique(keys)
    parts = 2 * ((keys.numel() + _UNIQUE_LIMIT - 1) // _UNIQUE_LIMIT)
    per_src = torch.cumsum(torch.bincount(keys // n, minlength=n), 0)
    targets = torch.arange(1, parts, device=keys.device, dtype=per_src.dtype) * (keys.numel() // parts)
    cuts = torch.searchsorted(per_src, targets).tolist()
    bounds = sorted(set([0] + [c * n for c in cuts] + [n * n]))
    del per_src
    out = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        sel = keys[(keys >= a) & (keys < b)]
        if sel.numel():
            out.append(torch.unique(sel))
        del sel
    return torch.cat(out)


def _csr_from_keys(box, n, relabel):
    """CSR from directed keys s * n + d (box = [keys], emptied here so that no
    caller frame keeps the array alive)."""
    keys = _unique(box.pop(), n)
    if relabel:
        s = keys // n
        deg = torch.bincount(s, minlength=n)
        order = torch.sort(deg, stable=True).indices          # new id -> old id
        newid = torch.empty_like(order)
        newid[order] = torch.arange(n, device=order.device)
        del deg, order
        s = newid[s]
        d = newid[keys % n]
        del keys, newid
        s.mul_(n).add_(d)
        del d
        keys = _unique(s, n)
        del s
    s = keys // n
    col = (keys % n).to(torch.int32)
    del keys
    counts = torch.bincount(s, minlength=n)
    del s
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=col.device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr, col


def _symmetric_keys(box, n):
    """box = [src, dst] (emptied): keys of both directions, self-loops dropped."""
    dst = box.pop().to(torch.int64)
    src = box.pop().to(torch.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    del keep
    keys = torch.cat([src * n + dst, dst * n + src])
    del src, dst
    return keys


def csr_from_edges(src, dst, n, relabel=False):
    """Symmetrise, drop loops, deduplicate and sort; optional degree relabel."""
    return _csr_from_keys([_symmetric_keys([src, dst], n)], n, relabel)


def relabel_by_degree(row_ptr, col):
    n = row_ptr.numel() - 1
    src = torch.repeat_interleave(torch.arange(n, device=col.device), row_ptr[1:] - row_ptr[:-1])
    return csr_from_edges(src, col.to(torch.int64), n, relabel=True)


def erdos_renyi(n, p, seed=1, device="cpu", relabel=False):
    """G(n, p): every pair i < j is an edge independently with probability p."""
    g = _gen(seed, device)
    srcs, dsts = [], []
    # row blocks keep the pair mask small
    block = max(1, (1 << 24) // max(n, 1))
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        rows = torch.arange(i0, i1, device=device)
        mask = torch.rand((i1 - i0, n), generator=g, device=device) < p
        mask &= torch.arange(n, device=device)[None, :] > rows[:, None]
        ii, jj = mask.nonzero(as_tuple=True)
        srcs.append(ii + i0)
        dsts.append(jj)
    return csr_from_edges(torch.cat(srcs), torch.cat(dsts), n, relabel=relabel)


def rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=2, device="cpu", relabel=True,
         permute=True):
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004) without noise: 2^scale vertices,
    edge_factor * 2^scale generated edges, quadrant probabilities (a, b, c, d),
    then a seeded random vertex permutation (Graph500 style)."""
    n = 1 << scale
    E = edge_factor * n
    g = _gen(seed, device)
    src = torch.zeros(E, dtype=torch.int64, device=device)
    dst = torch.zeros(E, dtype=torch.int64, device=device)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        u = torch.rand(E, generator=g, device=device)
        sbit = u >= ab
        dbit = ((u >= a) & (u < ab)) | (u >= abc)
        src |= sbit.to(torch.int64) << level
        dst |= dbit.to(torch.int64) << level
        del u, sbit, dbit
    if permute:
        perm = torch.randperm(n, generator=g, device=device)
        src = perm[src]
        dst = perm[dst]
        del perm
    box = [src, dst]
    del src, dst
    box = [_symmetric_keys(box, n)]
    return _csr_from_keys(box, n, relabel)


def chung_lu(n, gamma=2.1, mean_degree=20.0, n_cliques=200, clique_size=12, seed=4,
             device="cpu", relabel=True, offset=10.0, w_max=None):
    """Chung-Lu graph with expected degrees w_i ~ (i + offset)^(-1/(gamma-1)),
    scaled to the mean degree and capped at sqrt(sum w) (or at w_max when given);
    n * mean / 2 endpoint pairs drawn from the weight distribution; plus planted
    cliques on uniformly chosen vertex sets."""
    g = _gen(seed, device)
    i = torch.arange(n, dtype=torch.float64, device=device)
    w = (i + offset).pow(-1.0 / (gamma - 1.0))
    w = w * (n * mean_degree / w.sum())
    w = torch.clamp(w, max=math.sqrt(float(w.sum())) if w_max is None else float(w_max))
    cdf = torch.cumsum(w, 0)
    cdf = cdf / cdf[-1]
    m = int(n * mean_degree / 2)
    src = torch.searchsorted(cdf, torch.rand(m, generator=g, device=device, dtype=torch.float64))
    dst = torch.searchsorted(cdf, torch.rand(m, generator=g, device=device, dtype=torch.float64))
    src = torch.clamp(src, max=n - 1)
    dst = torch.clamp(dst, max=n - 1)
    cs, cd = [], []
    for _ in range(n_cliques):
        verts = torch.randperm(n, generator=g, device=device)[:clique_size]
        ii, jj = torch.triu_indices(clique_size, clique_size, 1, device=device)
        cs.append(verts[ii])
        cd.append(verts[jj])
    if cs:
        src = torch.cat([src] + cs)
        dst = torch.cat([dst] + cd)
    return csr_from_edges(src, dst, n, relabel=relabel)


# ---------------------------------------------------------------- small graphs
def from_edge_list(n, edges, device="cpu"):
    if len(edges) == 0:
        return (torch.zeros(n + 1, dtype=torch.int64, device=device),
                torch.zeros(0, dtype=torch.int32, device=device))
    e = torch.tensor(edges, dtype=torch.int64, device=device)
    return csr_from_edges(e[:, 0], e[:, 1], n)


def complete(n):
    return from_edge_list(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def complete_bipartite(a, b):
    return from_edge_list(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def star(leaves):
    return from_edge_list(leaves + 1, [(0, i) for i in range(1, leaves + 1)])


def cycle(n):
    return from_edge_list(n, [(i, (i + 1) % n) for i in range(n)])


def random_small(n, p, seed):
    return erdos_renyi(n, p, seed=seed, device="cpu")


def to_numpy(row_ptr, col):
    return row_ptr.cpu().numpy().astype("uint64"), col.cpu().numpy().astype("uint32")


# ---------------------------------------------------------------- patterns
# pattern name -> (k, edge list); vertex ids are pattern-local
PATTERNS = {
    "edge": (2, [(0, 1)]),
    "triangle": (3, [(0, 1), (1, 2), (0, 2)]),
    "wedge": (3, [(0, 1), (0, 2)]),
    "3-star": (4, [(0, 1), (0, 2), (0, 3)]),
    "4-path": (4, [(0, 1), (1, 2), (2, 3)]),
    "tailed-triangle": (4, [(0, 1), (1, 2), (0, 2), (2, 3)]),
    "4-cycle": (4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    "diamond": (4, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]),
    "5-path": (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4)]),
    "dumbbell": (6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (2, 3)]),
}


def clique(k):
    return (k, [(i, j) for i in range(k) for j in range(i + 1, k)])


def pattern(name):
    if name.endswith("-clique"):
        return clique(int(name.split("-")[0]))
    return PATTERNS[name]


MOTIFS4 = ["3-star", "4-path", "tailed-triangle", "4-cycle", "diamond", "4-clique"]
