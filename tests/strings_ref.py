"""Address order of the class string lists, rebuilt in plain Python from the
convention that e2.h documents (test helper; no GPU, no product code)."""
from math import comb

import numpy as np


def _patterns(sizes, count):
    """Occupation patterns (n_1..n_k), sum = count, n_s <= sizes[s], in
    lexicographic order with n_1 most significant."""
    if len(sizes) == 1:
        return [(count,)] if 0 <= count <= sizes[0] else []
    out = []
    for k in range(0, min(sizes[0], count) + 1):
        out += [(k,) + rest for rest in _patterns(sizes[1:], count - k)]
    return out


class ClassStrings:
    """Address order of a class's strings, rebuilt from the documented
    convention: the patterns of N+h-p electrons within two substitutions of a
    P pattern (h + min deficit <= 2; class (0,0) without the P patterns), in
    lexicographic order; inside a pattern a mixed radix over the subspaces,
    subspace 1 fastest, of colex ranks."""

    def __init__(self, prob, h, p):
        sizes, lo, hi = list(prob.das_size), list(prob.das_min), list(prob.das_max)
        ok = lambda pt: all(lo[s] <= pt[s] <= hi[s] for s in range(len(sizes)))
        P = [q for q in _patterns(sizes, prob.n_elec) if ok(q)]
        deficit = lambda pt: min(sum(max(0, q[s] - pt[s]) for s in range(len(sizes))) for q in P)
        self.sizes = sizes
        self.off = [sum(sizes[:s]) for s in range(len(sizes))]
        self.pats, self.start = [], []
        n = 0
        for pt in _patterns(sizes, prob.n_elec + h - p):
            if h + deficit(pt) > 2 or (h == 0 and p == 0 and ok(pt)):
                continue
            self.pats.append(pt)
            self.start.append(n)
            n += int(np.prod([comb(sizes[s], pt[s]) for s in range(len(sizes))]))
        self.n = n

    def __call__(self, r):
        k = max(i for i, s in enumerate(self.start) if s <= r)
        r -= self.start[k]
        bits = 0
        for s, occ in enumerate(self.pats[k]):
            cs = comb(self.sizes[s], occ)
            bits |= _colex_unrank(r % cs, occ) << self.off[s]
            r //= cs
        return bits


def _colex_unrank(r, k):
    """Active-local bitset of the k-subset with colex rank r (sum_j C(t_j, j))."""
    bits = 0
    for j in range(k, 0, -1):
        t = j - 1
        while comb(t + 1, j) <= r:
            t += 1
        r -= comb(t, j)
        bits |= 1 << t
    return bits
