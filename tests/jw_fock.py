"""Brute-force Fock-space reference for tiny systems (test helper).

The Hamiltonian H = sum h_pq a+_p a_q + 1/4 sum <pq||rs> a+_p a+_q a_s a_r is
built as a dense-in-the-sector sparse matrix with Jordan-Wigner operators:
basis state index bit p = occupation of spinor p, and a_p carries the parity
of the occupied spinors below p (creators in ascending order act on the
vacuum).  This shares nothing with the oracle's bitset Slater-Condon code.
"""
from itertools import combinations
from math import comb

import numpy as np
import scipy.sparse as sp


def annihilators(n):
    dim = 1 << n
    idx = np.arange(dim)
    ops = []
    for p in range(n):
        occ = (idx >> p) & 1
        src = idx[occ == 1]
        dst = src ^ (1 << p)
        below = np.array([bin(s & ((1 << p) - 1)).count("1") for s in src])
        sign = np.where(below % 2 == 0, 1.0, -1.0)
        ops.append(sp.csr_matrix((sign, (dst, src)), shape=(dim, dim)))
    return ops


def integrals(prob):
    """(pq|rs) = sum_L w_L B^L_pq B^L_rs and <pq||rs> = (pr|qs) - (ps|qr)."""
    B, w = prob.factors()
    eri = np.einsum("l,lpq,lrs->pqrs", w, B, B)
    asym = eri.transpose(0, 2, 1, 3) - eri.transpose(0, 2, 3, 1)
    return eri, asym


def fock_hamiltonian(prob):
    n = prob.n
    a = annihilators(n)
    ad = [x.T.tocsr() for x in a]
    _, g = integrals(prob)
    H = sp.csr_matrix((1 << n, 1 << n), dtype=complex)
    for p in range(n):
        for q in range(n):
            if prob.h[p, q] != 0:
                H = H + prob.h[p, q] * (ad[p] @ a[q])
    pairs = list(combinations(range(n), 2))
    ann2 = {(r, s): (a[s] @ a[r]) for (r, s) in pairs}        # a_s a_r, r < s
    for (p, q) in pairs:
        acc = sp.csr_matrix((1 << n, 1 << n), dtype=complex)
        for (r, s) in pairs:
            v = g[p, q, r, s]
            if v != 0:
                acc = acc + v * ann2[(r, s)]
        H = H + (ad[p] @ ad[q]) @ acc                           # sum over p<q, r<s
    return H.tocsr()


def p_address(prob, act_bits):
    """Address of an active string in the reference vector (pattern blocks in
    lexicographic order, colex ranks inside, subspace 1 fastest), or -1."""
    sizes, lo, hi, N = prob.das_size, prob.das_min, prob.das_max, prob.n_elec
    pats = []

    def rec(s, left, cur):
        if s == len(sizes):
            if left == 0:
                pats.append(tuple(cur))
            return
        for k in range(lo[s], min(hi[s], sizes[s]) + 1):
            if k <= left:
                rec(s + 1, left - k, cur + [k])

    rec(0, N, [])
    offs, o = {}, 0
    for pt in pats:
        offs[pt] = o
        cnt = 1
        for sz, k in zip(sizes, pt):
            cnt *= comb(sz, k)
        o += cnt
    start = 0
    occ, ranks = [], []
    for sz in sizes:
        bits = [(act_bits >> (start + t)) & 1 for t in range(sz)]
        occ.append(sum(bits))
        r, j = 0, 0
        for t in range(sz):
            if bits[t]:
                j += 1
                r += comb(t, j)
        ranks.append(r)
        start += sz
    pt = tuple(occ)
    if pt not in offs:
        return -1
    addr, stride = offs[pt], 1
    for sz, k, r in zip(sizes, occ, ranks):
        addr += r * stride
        stride *= comb(sz, k)
    return addr


def brute_e2(prob, c, b=0.0, allowed=None):
    """E2 per root and class from the Fock-space matrix: Q = determinants of the
    right electron count, not in P, touching no frozen spinor, within two
    substitutions of some P determinant (and, if given, allowed(K) true for
    the Fock index K)."""
    n, nc, na = prob.n, prob.n_core, prob.n_act
    a0, v0 = nc, nc + na
    ntot = nc + prob.n_elec
    H = fock_hamiltonian(prob)
    dim = 1 << n
    frozen = [p for p in range(n) if prob.frozen[p]]
    fc = [p for p in frozen if p < nc]
    fv = [p for p in frozen if p >= v0]
    core_mask = (1 << nc) - 1
    # P determinants
    Pidx, Paddr = [], []
    for A in combinations(range(na), prob.n_elec):
        bits = sum(1 << t for t in A)
        ad = p_address(prob, bits)
        if ad >= 0:
            Pidx.append(core_mask | (bits << a0))
            Paddr.append(ad)
    Pidx = np.array(Pidx)
    psi = np.zeros((c.shape[0], dim), complex)
    for i, ad in zip(Pidx, Paddr):
        psi[:, i] = c[:, ad]
    Hpsi = np.array([H @ psi[m] for m in range(c.shape[0])])
    E0 = np.array([np.vdot(psi[m], Hpsi[m]).real / np.vdot(psi[m], psi[m]).real for m in range(c.shape[0])])
    diag = H.diagonal().real
    Pset = set(Pidx.tolist())
    e2 = np.zeros((c.shape[0], 9))
    count = np.zeros(9, int)
    for K in range(dim):
        if bin(K).count("1") != ntot or K in Pset:
            continue
        if any(not (K >> p) & 1 for p in fc) or any((K >> p) & 1 for p in fv):
            continue
        rank = min(bin(L & ~K).count("1") for L in Pidx)
        if rank > 2:
            continue
        if allowed is not None and not allowed(K):
            continue
        h = nc - bin(K & core_mask).count("1")
        p = bin(K >> v0).count("1")
        cls = 3 * h + p
        count[cls] += 1
        for m in range(c.shape[0]):
            D = E0[m] - diag[K]
            v2 = abs(Hpsi[m, K]) ** 2
            e2[m, cls] += v2 / D if b == 0 else v2 * D ** 3 / (D ** 4 + b * b)
    return E0, e2, count, H
