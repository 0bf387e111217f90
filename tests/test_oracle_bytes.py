"""Hand-counted pins of the oracle's algorithmic-byte count (og_sample_bytes).

The count is the memory the candidate-set definition of Sec. 4.2 (Algorithm 4)
references on the path a sample takes, in 32-byte sectors (8 uint32 column
entries): 1 sector for the first edge; per step j and per list the step
references, 1 sector for the list's row_ptr pair plus the sectors spanned by
the list's part above the step's lower bound; a clique-like step that extends
S_{j-1} by one adjacency references only N(v_{j-1}); CHECK mode reads one list
position plus one binary search (ceil(log2(d + 1)) sectors) per other list.

Every expected value below is counted by hand from the column offsets of the
graph drawn here; the arithmetic is in the comments.  Nothing calls the
oracle's formula to get an expected value.  CPU only.
"""
import numpy as np
import pytest

from oracle import oracle as O

# Adjacency lists (sorted, symmetric) and the column offsets they occupy.
# Sector s of col holds entries [8 s, 8 s + 8).
#   N(0)  = 1..11              col[0, 11)
#   N(1)  = 0 2 3 4 6 9        col[11, 17)
#   N(2)  = 0 1                col[17, 19)
#   N(3)  = 0 1 4 5 6 9        col[19, 25)
#   N(4)  = 0 1 3              col[25, 28)
#   N(5)  = 0 3                col[28, 30)
#   N(6)  = 0 1 3 7 8 9        col[30, 36)
#   N(7)  = 0 6                col[36, 38)
#   N(8)  = 0 6                col[38, 40)
#   N(9)  = 0 1 3 6 10 11      col[40, 46)
#   N(10) = 0 9                col[46, 48)
#   N(11) = 0 9                col[48, 50)
LISTS = [
    list(range(1, 12)),
    [0, 2, 3, 4, 6, 9],
    [0, 1],
    [0, 1, 4, 5, 6, 9],
    [0, 1, 3],
    [0, 3],
    [0, 1, 3, 7, 8, 9],
    [0, 6],
    [0, 6],
    [0, 1, 3, 6, 10, 11],
    [0, 9],
    [0, 9],
]
ROW_PTR = [0, 11, 17, 19, 25, 28, 30, 36, 38, 40, 46, 48, 50]

CLIQUE4 = (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
CYCLE4 = (4, [(0, 1), (1, 2), (2, 3), (3, 0)])
WEDGE = (3, [(0, 1), (1, 2)])


@pytest.fixture(scope="module")
def g():
    rp = np.zeros(len(LISTS) + 1, dtype=np.uint64)
    for v, lst in enumerate(LISTS):
        rp[v + 1] = rp[v] + len(lst)
    assert rp.tolist() == ROW_PTR
    col = np.array([x for lst in LISTS for x in lst], dtype=np.uint32)
    assert O.validate(rp, col) == 0
    return O.Graph(rp, col)


def word(i, n):
    """A choice word r with floor(r n / 2^64) = i."""
    return ((i << 64) + n - 1) // n


def run(g, pat, words, mode=O.INTERSECT, induced=False):
    p = O.plan(pat[0], pat[1], induced=induced)
    rec = O.sample(g, p, words, mode=mode)
    return p, rec, O.sample_bytes(g, p, rec, mode=mode)


def verts(rec, k):
    return [rec.vert[i] for i in range(k)]


def test_graph_has_25_edges(g):
    assert g.m == 25 and g.nnz == 50


def test_clique_step_three_reads_only_the_newest_list(g):
    # 4-clique, restrictions v0 < v1 < v2 < v3, first edge from the m = 25
    # oriented edges; (1, 3) is oriented edge 12 (11 edges of vertex 0, then
    # (1,2) = 11, (1,3) = 12).
    # step 2, bound v1 = 3:  N(1) above 3 = {4, 6, 9} = col[14, 17): sectors 1..2 -> 1 + 2
    #                        N(3) above 3 = {4, 5, 6, 9} = col[21, 25): sectors 2..3 -> 1 + 2
    #   S_2 = {4, 6, 9}, index 1 -> 6
    # step 3 extends S_2 by N(6): only N(6) above 6 = {7, 8, 9} = col[33, 36): sector 4 -> 1 + 1
    #   S_3 = {9}
    # total 1 + 3 + 3 + 2 = 9 sectors = 288 bytes
    p, rec, b = run(g, CLIQUE4, [word(12, 25), word(1, 3), word(0, 1)])
    assert rec.hit == 1 and verts(rec, 4) == [1, 3, 6, 9]
    assert [rec.factor[j] for j in range(4)] == [25, 0, 3, 1]
    assert b == 288.0


def test_two_back_neighbours_with_bound_inside_the_lists(g):
    # 4-cycle: order 0-1-2-3, restrictions v0 < v1, v0 < v2, v0 < v3, v1 < v3;
    # step 2 has the single back-neighbour v1 (bound v0), step 3 the back-neighbours
    # v0 and v2 (bound max(v0, v1)); step 3 does not extend step 2's set.
    # first edge (1, 3) = oriented edge 12.
    # step 2, bound 1: N(3) above 1 = {4, 5, 6, 9} = col[21, 25) -> 1 + 2;  S_2 = {4, 5, 6, 9}, index 2 -> 6
    # step 3, bound 3: N(1) above 3 = col[14, 17) -> 1 + 2
    #                  N(6) above 3 = {7, 8, 9} = col[33, 36) -> 1 + 1;   S_3 = {9}
    # total 1 + 3 + 3 + 2 = 9 sectors = 288 bytes
    p, rec, b = run(g, CYCLE4, [word(12, 25), word(2, 4), word(0, 1)])
    assert rec.hit == 1 and verts(rec, 4) == [1, 3, 6, 9]
    assert b == 288.0


def test_miss_at_depth_three_counts_the_empty_list(g):
    # 4-cycle as above with v2 = 4 (index 0 of S_2):
    # step 2: 1 + 2 as above
    # step 3, bound 3: N(1) above 3 = col[14, 17) -> 1 + 2
    #                  N(4) above 3 = col[28, 28), empty -> 1 + 0;  S_3 empty: miss
    # total 1 + 3 + 3 + 1 = 8 sectors = 256 bytes
    p, rec, b = run(g, CYCLE4, [word(12, 25), word(0, 4), word(0, 1)])
    assert rec.hit == 0 and rec.depth == 3 and verts(rec, 3) == [1, 3, 4]
    assert b == 256.0


def test_miss_at_depth_two(g):
    # 4-clique, first edge (0, 5) = oriented edge 4 (N+(0) = 1..11)
    # step 2, bound 5: N(0) above 5 = {6..11} = col[5, 11): sectors 0..1 -> 1 + 2
    #                  N(5) above 5 = col[30, 30), empty -> 1 + 0;  S_2 empty: miss
    # step 3 not taken.  total 1 + 3 + 1 = 5 sectors = 160 bytes
    p, rec, b = run(g, CLIQUE4, [word(4, 25), word(0, 1), word(0, 1)])
    assert rec.hit == 0 and rec.depth == 2 and verts(rec, 2) == [0, 5]
    assert b == 160.0


def test_check_mode_counts_searches(g):
    # 4-clique in CHECK mode, first edge (1, 3).  ceil(log2(6 + 1)) = 3 sectors for a
    # binary search in a list of 6.
    # step 2: L_2 = N(v1 = 3) above 3 = {4, 5, 6, 9}
    #   row_ptr pair 1 + bound search in N(3) 3 + drawn element 1
    #   + other back-neighbour v0 = 1: row_ptr pair 1 + search in N(1) 3  = 9; index 2 -> 6
    # step 3: L_3 = N(v2 = 6) above 6 = {7, 8, 9}
    #   1 + search in N(6) 3 + drawn 1 + N(1): 1 + 3 + N(3): 1 + 3         = 13; index 2 -> 9
    # total 1 + 9 + 13 = 23 sectors = 736 bytes
    p, rec, b = run(g, CLIQUE4, [word(12, 25), word(2, 4), word(2, 3)], mode=O.CHECK)
    assert rec.hit == 1 and verts(rec, 4) == [1, 3, 6, 9]
    assert [rec.factor[j] for j in range(4)] == [25, 0, 4, 3]
    assert b == 736.0


def test_vertex_induced_step_reads_the_non_neighbour(g):
    # vertex-induced wedge: order (centre, leaf, leaf), restriction v1 < v2, first
    # edge from the 2m = 50 directed entries; (3 -> 1) is entry row_ptr[3] + 1 = 20.
    # step 2, bound v1 = 1: edge list N(3) above 1 = col[21, 25) -> 1 + 2
    #                       non-edge list N(1) above 1 = {2, 3, 4, 6, 9} = col[12, 17): sectors 1..2 -> 1 + 2
    #   S_2 = {4, 5, 6, 9} minus N(1) = {5}
    # total 1 + 3 + 3 = 7 sectors = 224 bytes
    p, rec, b = run(g, WEDGE, [word(20, 50), word(0, 1)], induced=True)
    assert rec.hit == 1 and verts(rec, 3) == [3, 1, 5]
    assert rec.factor[0] == 50
    assert b == 224.0
    # edge-induced, the same path does not read N(1):  S_2 = {4, 5, 6, 9}, index 1 -> 5
    # total 1 + 3 = 4 sectors = 128 bytes
    p, rec, b = run(g, WEDGE, [word(20, 50), word(1, 4)], induced=False)
    assert rec.hit == 1 and verts(rec, 3) == [3, 1, 5]
    assert b == 128.0


def test_lazy_mode_reads_whole_lists_and_one_search_per_closing_pair(g):
    # NS-base, triangle: first edge from the 50 directed entries; (1 -> 3) is entry
    # row_ptr[1] + 2 = 13.  U_2 = N(1) then N(3) minus N(1) = [0 2 3 4 6 9 | 1 5], size 8.
    # step 2 reads both lists whole: N(1) = col[11, 17): sectors 1..2 -> 1 + 2
    #                                N(3) = col[19, 25): sectors 2..3 -> 1 + 2
    # closure, one search per pattern edge (i, j), i < j, in N(v_i), ceil(log2(6 + 1)) = 3:
    #   (0, 1) in N(1): 1 + 3;  (0, 2) in N(1): 1 + 3;  (1, 2) in N(3): 1 + 3
    # total 1 + 3 + 3 + 12 = 19 sectors = 608 bytes, hit or miss alike
    TRI = (3, [(0, 1), (1, 2), (0, 2)])
    p, rec, b = run(g, TRI, [word(13, 50), word(4, 8)], mode=O.LAZY)
    assert rec.hit == 1 and verts(rec, 3) == [1, 3, 6] and rec.factor[2] == 8 and rec.w_u64 == 400
    assert b == 608.0
    p, rec, b = run(g, TRI, [word(13, 50), word(6, 8)], mode=O.LAZY)    # x = 1 = v0: closure fails
    assert rec.hit == 0 and rec.depth == 3 and verts(rec, 3) == [1, 3, 1]
    assert b == 608.0
