"""Determinant enumeration and the two-species product basis (oracle).

Test infrastructure only (see the package docstring).

* A species determinant is the bit string of Sec. II Eq. (mbasis): bit i set
  when m-state i is occupied (App. A, Table I).
* Species determinants are grouped by their 2M and, inside a group, sorted by
  the unsigned value of the bit string.
* The product basis is the factorised form of App. A Eq. (part): a basis state
  is (proton determinant, neutron determinant) with M_A + M_B = M.  Blocks are
  ordered by ascending 2M_A; inside a block the index is iA * N_B + iB.

Pins: Table I (9 determinants), the dimensions printed in the paper (640 for
the 20Ne sd space, 28,503 for 24Mg, 1,963,461 for 48Cr pf), and an
independent generating-function count.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Sequence, Tuple

import numpy as np


def species_determinants(twom: Sequence[int], k: int) -> List[Tuple[int, int]]:
    """All k-particle determinants of one species as (2M, bits), sorted.

    Every k-subset of the m-states is one Slater determinant (Eq. (mbasis)).
    """
    out = []
    for occ in itertools.combinations(range(len(twom)), k):
        bits = 0
        for i in occ:
            bits |= 1 << i
        out.append((sum(twom[i] for i in occ), bits))
    out.sort()
    return out


def table1_order(twom: Sequence[int], orbit: Sequence[int], k: int, twoM: int):
    """Determinants with total 2M in the order of the paper's Table I.

    Groups are occupation-number vectors N = (N_1, N_2, ...) in descending
    lexicographic order (the first orbit's occupation descending), and inside
    a group the occupied-index tuples ascend lexicographically.
    Returns a list of (occupation tuple, occupied-index tuple, bits).
    """
    norb = max(orbit) + 1
    rows = []
    for occ in itertools.combinations(range(len(twom)), k):
        if sum(twom[i] for i in occ) != twoM:
            continue
        N = [0] * norb
        for i in occ:
            N[orbit[i]] += 1
        bits = sum(1 << i for i in occ)
        rows.append((tuple(N), occ, bits))
    rows.sort(key=lambda r: (tuple(-x for x in r[0]), r[1]))
    return rows


class ProductBasis:
    """Two-species M-scheme basis (App. A Eq. (part)).

    Attributes
    ----------
    detsA, detsB: sorted (2M, bits) lists of each species.
    blocks: list of (2M_A, 2M_B, offset, nA_in_block, nB_in_block,
            first index of A group, first index of B group).
    states: list of (bitsA, bitsB) in basis order.
    index: dict (bitsA, bitsB) -> basis index.
    """

    def __init__(self, twomA, kA, twomB, kB, twoM):
        self.twomA, self.twomB = tuple(twomA), tuple(twomB)
        self.kA, self.kB, self.twoM = kA, kB, twoM
        self.nA, self.nB = len(twomA), len(twomB)
        self.detsA = species_determinants(twomA, kA)
        self.detsB = species_determinants(twomB, kB)
        groupsA = _groups(self.detsA)
        groupsB = _groups(self.detsB)
        self.blocks = []
        self.states: List[Tuple[int, int]] = []
        off = 0
        for mA in sorted(groupsA):
            mB = twoM - mA
            if mB not in groupsB:
                continue
            a0, na = groupsA[mA]
            b0, nb = groupsB[mB]
            self.blocks.append((mA, mB, off, na, nb, a0, b0))
            for ia in range(na):
                sa = self.detsA[a0 + ia][1]
                for ib in range(nb):
                    self.states.append((sa, self.detsB[b0 + ib][1]))
            off += na * nb
        self.dim = off
        self.index: Dict[Tuple[int, int], int] = {
            s: i for i, s in enumerate(self.states)}


def partitions(twomA, orbitA, kA, twomB, orbitB, kB, twoM):
    """Partitions Gamma = (N^A, N^B, 2M_A) of App. A: orbit occupation
    vectors of the two species and the first species' 2M for which both
    species have determinants with 2M_A + 2M_B = twoM.  Returns a dict
    Gamma -> number of basis states in it (the product of the two species'
    determinant counts)."""
    def occupations(twom, orbit, k):
        norb = max(orbit) + 1 if len(orbit) else 0
        cnt: Dict[Tuple[Tuple[int, ...], int], int] = {}
        for occ in itertools.combinations(range(len(twom)), k):
            N = [0] * norb
            for i in occ:
                N[orbit[i]] += 1
            key = (tuple(N), sum(twom[i] for i in occ))
            cnt[key] = cnt.get(key, 0) + 1
        return cnt
    PA = occupations(twomA, orbitA, kA)
    PB = occupations(twomB, orbitB, kB)
    return {(NA, NB, mA): cA * cB for (NA, mA), cA in PA.items() for (NB, mB), cB in PB.items()
            if mA + mB == twoM}


def _groups(dets):
    """2M -> (first index, count) for a sorted determinant list."""
    g: Dict[int, List[int]] = {}
    for i, (m, _) in enumerate(dets):
        if m in g:
            g[m][1] += 1
        else:
            g[m] = [i, 1]
    return {m: (v[0], v[1]) for m, v in g.items()}


def dimension_by_generating_function(twomA, kA, twomB, kB, twoM,
                                     parityB=None, want_parity=None) -> int:
    """Count basis states as a coefficient of prod_i (1 + x y^(2m_i)).

    Independent of the enumerator: it multiplies polynomials in (particle
    number, 2M[, parity]) and reads off the coefficient.  ``parityB`` (0/1
    per m-state of species B) with ``want_parity`` restricts species B to a
    total parity; species A then has no parity label.
    """

    def poly(twom, k, par=None):
        # dict (n, 2M, parity) -> count
        P = {(0, 0, 0): 1}
        for i, tm in enumerate(twom):
            pi = par[i] if par is not None else 0
            Q = dict(P)
            for (n, m, p), c in P.items():
                if n < k:
                    key = (n + 1, m + tm, p ^ pi)
                    Q[key] = Q.get(key, 0) + c
            P = Q
        return {(m, p): c for (n, m, p), c in P.items() if n == k}

    PA = poly(twomA, kA)
    PB = poly(twomB, kB, parityB)
    total = 0
    for (mA, pA), cA in PA.items():
        for (mB, pB), cB in PB.items():
            if mA + mB != twoM:
                continue
            if want_parity is not None and (pA ^ pB) != want_parity:
                continue
            total += cA * cB
    return total


def one_body_jump_count(twom: Sequence[int], k: int) -> int:
    """Number of (determinant, a != c) pairs with c occupied and a empty.

    Counted by brute force over determinants (no M restriction): it equals
    N_det * k * (n - k).
    """
    n = len(twom)
    cnt = 0
    for _, bits in species_determinants(twom, k):
        for c in range(n):
            if not bits >> c & 1:
                continue
            for a in range(n):
                if a != c and not bits >> a & 1:
                    cnt += 1
    return cnt


def same_species_targets(twom: Sequence[int], k: int) -> int:
    """Ordered pairs (S, S') of distinct determinants with equal 2M that differ
    in at most two occupied states (popcount(S xor S') <= 4), brute force."""
    dets = species_determinants(twom, k)
    byM: Dict[int, List[int]] = {}
    for m, b in dets:
        byM.setdefault(m, []).append(b)
    cnt = 0
    for m, L in byM.items():
        arr = np.array(L, dtype=np.uint64)
        for b in L:
            x = np.bitwise_xor(arr, np.uint64(b))
            pc = np.array([int(v).bit_count() for v in x])
            cnt += int(np.count_nonzero((pc > 0) & (pc <= 4)))
    return cnt
