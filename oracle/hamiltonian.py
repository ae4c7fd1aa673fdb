"""Explicit M-scheme Hamiltonian by applying every operator term (oracle).

Test infrastructure only (see the package docstring).

The Hamiltonian is the one of Sec. II,
    H = sum_ac h(1)_ac c+_a c_c + sum_{a<b, c<d} h(2)_abcd c+_a c+_b c_d c_c,
written per species as in App. B: like-particle one- and two-body terms for
species A and B (App. B.1, Eq. (twobodybit)) and the cross-species term
    sum_{a,c in A; b,d in B} V^AB_{ab,cd} a+_a b+_b b_d a_c
(App. B.2, Eq. (pntwobodybit)).  Every term is applied to every basis state,
operator by operator from the right, with the fermion sign of the
Jordan-Wigner ordering: modes of species A first, then species B; a basis
state is (A creators ascending)(B creators ascending)|0>.  An operator on
mode x picks up (-1)^(number of occupied modes before x in that ordering).
App. B.1 finds the target index by a binary search; here a dictionary does it.

The matrix element <j|term|i> is accumulated as H[j, i].  Nothing here uses
the factorisation of App. B.2: the cross-species term is applied as a
four-operator string like any other.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from .basis import ProductBasis

# operator = (species 0/1, creation?, mode)
Op = Tuple[int, bool, int]


def apply_string(SA: int, SB: int, ops) -> Tuple[int, int, int]:
    """Apply ops (written left to right) to |SA, SB>; returns (sign, SA', SB').

    sign == 0 means the result vanishes (Pauli blocking).
    """
    sign = 1
    for spc, dag, x in reversed(ops):
        bit = 1 << x
        if spc == 0:
            S = SA
            before = (S & (bit - 1)).bit_count()
        else:
            S = SB
            before = SA.bit_count() + (S & (bit - 1)).bit_count()
        if dag:
            if S & bit:
                return 0, 0, 0
            S |= bit
        else:
            if not S & bit:
                return 0, 0, 0
            S ^= bit
        if before & 1:
            sign = -sign
        if spc == 0:
            SA = S
        else:
            SB = S
    return sign, SA, SB


class TermTables:
    """Nonzero coefficients of each operator family, keyed by the annihilated modes."""

    def __init__(self, inter, tol: float = 0.0):
        h1A, h1B = inter.h1A, inter.h1B
        VAA, VBB, VAB = inter.VAA, inter.VBB, inter.VAB
        nA, nB = h1A.shape[0], h1B.shape[0]
        self.nA, self.nB = nA, nB
        self.oneA = {c: [(a, h1A[a, c]) for a in range(nA) if abs(h1A[a, c]) > tol]
                     for c in range(nA)}
        self.oneB = {d: [(b, h1B[b, d]) for b in range(nB) if abs(h1B[b, d]) > tol]
                     for d in range(nB)}
        self.twoAA = self._like(VAA, tol)
        self.twoBB = self._like(VBB, tol)
        self.pn: Dict[Tuple[int, int], List[Tuple[int, int, float]]] = {}
        for c in range(nA):
            for d in range(nB):
                L = []
                for a in range(nA):
                    for b in range(nB):
                        v = VAB[a, b, c, d]
                        if abs(v) > tol:
                            L.append((a, b, v))
                self.pn[(c, d)] = L

    @staticmethod
    def _like(V, tol):
        n = V.shape[0]
        out = {}
        for c in range(n):
            for d in range(c + 1, n):
                L = []
                for a in range(n):
                    for b in range(a + 1, n):
                        v = V[a, b, c, d]
                        if abs(v) > tol:
                            L.append((a, b, v))
                out[(c, d)] = L
        return out


def column_terms(SA: int, SB: int, T: TermTables):
    """All (sign * coefficient, SA', SB') produced by H acting on |SA, SB>."""
    out = []
    occA = [x for x in range(T.nA) if SA >> x & 1]
    occB = [x for x in range(T.nB) if SB >> x & 1]
    for c in occA:
        for a, h in T.oneA[c]:
            s, A2, B2 = apply_string(SA, SB, ((0, True, a), (0, False, c)))
            if s:
                out.append((s * h, A2, B2))
    for d in occB:
        for b, h in T.oneB[d]:
            s, A2, B2 = apply_string(SA, SB, ((1, True, b), (1, False, d)))
            if s:
                out.append((s * h, A2, B2))
    for i, c in enumerate(occA):
        for d in occA[i + 1:]:
            for a, b, v in T.twoAA[(c, d)]:
                s, A2, B2 = apply_string(
                    SA, SB, ((0, True, a), (0, True, b), (0, False, d), (0, False, c)))
                if s:
                    out.append((s * v, A2, B2))
    for i, c in enumerate(occB):
        for d in occB[i + 1:]:
            for a, b, v in T.twoBB[(c, d)]:
                s, A2, B2 = apply_string(
                    SA, SB, ((1, True, a), (1, True, b), (1, False, d), (1, False, c)))
                if s:
                    out.append((s * v, A2, B2))
    for c in occA:
        for d in occB:
            for a, b, v in T.pn[(c, d)]:
                s, A2, B2 = apply_string(
                    SA, SB, ((0, True, a), (1, True, b), (1, False, d), (0, False, c)))
                if s:
                    out.append((s * v, A2, B2))
    return out


def assemble(basis: ProductBasis, inter) -> sp.csr_matrix:
    """Explicit sparse H (FP64 CSR), H[j, i] = <j|H|i>."""
    T = TermTables(inter)
    rows, cols, vals = [], [], []
    idx = basis.index
    for i, (SA, SB) in enumerate(basis.states):
        for v, A2, B2 in column_terms(SA, SB, T):
            j = idx[(A2, B2)]  # KeyError: a term broke M conservation
            rows.append(j)
            cols.append(i)
            vals.append(v)
    D = basis.dim
    H = sp.coo_matrix((np.array(vals), (np.array(rows, dtype=np.int64),
                                        np.array(cols, dtype=np.int64))), shape=(D, D))
    return H.tocsr()


def structural_pattern(basis: ProductBasis, inter) -> sp.csr_matrix:
    """Boolean pattern of (j, i) pairs reached by any term with a nonzero
    coefficient, counted before numerical cancellation."""
    T = TermTables(inter)
    rows, cols = [], []
    idx = basis.index
    for i, (SA, SB) in enumerate(basis.states):
        for v, A2, B2 in column_terms(SA, SB, T):
            rows.append(idx[(A2, B2)])
            cols.append(i)
    D = basis.dim
    P = sp.coo_matrix((np.ones(len(rows), dtype=np.int8),
                       (np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64))),
                      shape=(D, D)).tocsr()
    P.data[:] = 1
    return P


def column(basis: ProductBasis, inter, i: int, T: TermTables = None) -> Dict[int, float]:
    """Column i of H as {j: H[j, i]}."""
    if T is None:
        T = TermTables(inter)
    SA, SB = basis.states[i]
    out: Dict[int, float] = {}
    for v, A2, B2 in column_terms(SA, SB, T):
        j = basis.index[(A2, B2)]
        out[j] = out.get(j, 0.0) + v
    return out


def hv_rows(basis: ProductBasis, inter, V: np.ndarray, rows, T: TermTables = None) -> np.ndarray:
    """Rows of H @ V for the listed row indices, one row at a time.

    H is real symmetric (the interaction is symmetric), so row r of H equals
    column r, which is what ``column`` generates.
    """
    if T is None:
        T = TermTables(inter)
    out = np.zeros((len(rows), V.shape[1]), dtype=np.float64)
    for k, r in enumerate(rows):
        for j, h in column(basis, inter, int(r), T).items():
            out[k] += h * V[j].astype(np.float64)
    return out


class LazyIndex:
    """Basis index for spaces too large to hold a dict of all states.

    index(SA, SB) = block offset + rank(SA in its 2M group) * N_B + rank(SB).
    Ranks come from a dict per species, built from the sorted determinants.
    """

    def __init__(self, twomA, kA, twomB, kB, twoM):
        from .basis import species_determinants, _groups
        self.detsA = species_determinants(twomA, kA)
        self.detsB = species_determinants(twomB, kB)
        gA, gB = _groups(self.detsA), _groups(self.detsB)
        self.rankA = {b: i - gA[m][0] for i, (m, b) in enumerate(self.detsA)}
        self.rankB = {b: i - gB[m][0] for i, (m, b) in enumerate(self.detsB)}
        self.mA = {b: m for (m, b) in self.detsA}
        self.block = {}
        self.blocks = []
        off = 0
        for mA in sorted(gA):
            mB = twoM - mA
            if mB not in gB:
                continue
            na, nb = gA[mA][1], gB[mB][1]
            self.block[mA] = (off, nb)
            self.blocks.append((mA, mB, off, na, nb, gA[mA][0], gB[mB][0]))
            off += na * nb
        self.dim = off

    def index(self, SA: int, SB: int) -> int:
        off, nb = self.block[self.mA[SA]]
        return off + self.rankA[SA] * nb + self.rankB[SB]

    def state(self, i: int) -> Tuple[int, int]:
        for (mA, mB, off, na, nb, a0, b0) in self.blocks:
            if off <= i < off + na * nb:
                ia, ib = divmod(i - off, nb)
                return self.detsA[a0 + ia][1], self.detsB[b0 + ib][1]
        raise IndexError(i)


def hv_rows_lazy(L: LazyIndex, T: TermTables, V: np.ndarray, rows) -> np.ndarray:
    """Rows of H @ V for large spaces (no full state list), one row at a time."""
    out = np.zeros((len(rows), V.shape[1]), dtype=np.float64)
    for k, r in enumerate(rows):
        SA, SB = L.state(int(r))
        for v, A2, B2 in column_terms(SA, SB, T):
            out[k] += v * V[L.index(A2, B2)].astype(np.float64)
    return out


def one_body_jumps(twom, k: int):
    """Every one-body jump a+_a a_c |S> = sign |S'> of one species (App. B.2,
    the "one-body jumps"), diagonal a = c included, as a set of
    (target index, source index, a, c, sign) with the species' sorted
    determinant indices."""
    from .basis import species_determinants
    dets = species_determinants(twom, k)
    where = {b: i for i, (_, b) in enumerate(dets)}
    n = len(twom)
    out = set()
    for i, (_, S) in enumerate(dets):
        for c in range(n):
            for a in range(n):
                s, A2, _ = apply_string(S, 0, ((0, True, a), (0, False, c)))
                if s:
                    out.add((where[A2], i, a, c, s))
    return out
