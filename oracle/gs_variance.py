"""Variance of the GS estimators (Sec. 5.2's variance model, corrected), from
the matches of a small graph (test infrastructure only).

A GS estimate scales the exact count of the sparsified graph G' back up:
colour sparsification with c colours keeps a match iff its k vertices share a
colour (probability c^-(k-1)), Bernoulli edge sparsification keeps it iff its
l edges all stay (probability p^l).  Writing the scaled count as a sum of one
indicator per match, its variance is the sum of the covariances over ordered
pairs of matches (M1, M2):

  colours: two matches sharing z >= 1 vertices both survive iff the 2k - z
           vertices of their union share a colour, so
           Var = sum over pairs with z >= 1 of (c^(z - 1) - 1);
           pairs with no common vertex are independent;
  edges:   two matches sharing e edges both survive with probability
           p^(2l - e), so Var = sum over pairs of (p^-e - 1).

The paper writes the covariance term with p^(1 - z) for pairs sharing z
vertices; for colour sparsification (p = 1/c) that is c^(z - 1), and the
corrected form subtracts the product of the two survival probabilities (the
"- 1").  The pair sums here enumerate the matches (brute force), so they are
for graphs of a dozen vertices or so.
"""
from fractions import Fraction


def colour_variance(matches, k, c):
    """Exact Var of C' c^(k-1) over uniform colourings (matches: brute.matches)."""
    vs = [m[0] for m in matches]
    tot = Fraction(0)
    for a in vs:
        for b in vs:
            z = len(a & b)
            if z >= 1:
                tot += Fraction(c) ** (z - 1) - 1
    return tot


def edge_variance(matches, l, p):
    """Exact Var of C' p^-l when every edge stays independently with probability p."""
    p = Fraction(p)
    es = [m[1] for m in matches]
    tot = Fraction(0)
    for a in es:
        for b in es:
            e = len(a & b)
            tot += p ** (-e) - 1
    return tot
