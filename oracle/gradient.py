"""Hellmann-Feynman gradient of eigenvalues with respect to every parameter.

Test infrastructure only (see the package docstring).

H of Sec. II is linear in its parameters (one-body h(1)_ac and two-body
h(2)_abcd), so dE_k/dtheta = <v_k| dH/dtheta |v_k> for a normalised,
non-degenerate eigenvector v_k.  For a cluster C of (near-)degenerate levels
the well-defined quantity is the sum over the cluster,
    sum_{k in C} dE_k/dtheta = Tr(P_C dH/dtheta),
which is what this returns when it is given the cluster's vectors.

A parameter theta placed at slot (I, J) with I != J appears in two operator
terms (the term and its Hermitian conjugate); its derivative is the sum of
both terms' expectation values.  Every parameter allowed by M conservation is
listed, including those whose value is zero (off-diagonal one-body terms).
"""
from __future__ import annotations

from typing import Dict

import numpy as np

from .basis import ProductBasis
from .hamiltonian import apply_string


def term_expectations(basis: ProductBasis, twomA, twomB, vecs: np.ndarray) -> Dict[tuple, float]:
    """sum_k <v_k| T |v_k> for every M-allowed operator term T, keyed by term.

    Keys: ("h1A", a, c), ("h1B", b, d), ("VAA", a, b, c, d) with a<b, c<d,
    ("VBB", ...), ("VAB", a, b, c, d).
    """
    nA, nB = len(twomA), len(twomB)
    bins: Dict[tuple, float] = {}
    idx = basis.index
    pairs_like = {}
    for twom, n, key in ((twomA, nA, 0), (twomB, nB, 1)):
        d = {}
        for a in range(n):
            for b in range(a + 1, n):
                d.setdefault(twom[a] + twom[b], []).append((a, b))
        pairs_like[key] = d
    pairs_cross = {}
    for a in range(nA):
        for b in range(nB):
            pairs_cross.setdefault(twomA[a] + twomB[b], []).append((a, b))

    def add(key, s, A2, B2, vi):
        j = idx[(A2, B2)]
        bins[key] = bins.get(key, 0.0) + s * float(vecs[j] @ vi)

    for i, (SA, SB) in enumerate(basis.states):
        vi = vecs[i]
        occA = [x for x in range(nA) if SA >> x & 1]
        occB = [x for x in range(nB) if SB >> x & 1]
        for c in occA:
            for a in range(nA):
                if twomA[a] == twomA[c]:
                    s, A2, B2 = apply_string(SA, SB, ((0, True, a), (0, False, c)))
                    if s:
                        add(("h1A", a, c), s, A2, B2, vi)
        for d in occB:
            for b in range(nB):
                if twomB[b] == twomB[d]:
                    s, A2, B2 = apply_string(SA, SB, ((1, True, b), (1, False, d)))
                    if s:
                        add(("h1B", b, d), s, A2, B2, vi)
        for spc, occ, twom, name in ((0, occA, twomA, "VAA"), (1, occB, twomB, "VBB")):
            for x, c in enumerate(occ):
                for d in occ[x + 1:]:
                    for a, b in pairs_like[spc].get(twom[c] + twom[d], ()):
                        s, A2, B2 = apply_string(
                            SA, SB, ((spc, True, a), (spc, True, b), (spc, False, d), (spc, False, c)))
                        if s:
                            add((name, a, b, c, d), s, A2, B2, vi)
        for c in occA:
            for d in occB:
                for a, b in pairs_cross.get(twomA[c] + twomB[d], ()):
                    s, A2, B2 = apply_string(
                        SA, SB, ((0, True, a), (1, True, b), (1, False, d), (0, False, c)))
                    if s:
                        add(("VAB", a, b, c, d), s, A2, B2, vi)
    return bins


def hf_gradient(basis: ProductBasis, inter, vecs: np.ndarray) -> np.ndarray:
    """sum over the given vectors of dE/dtheta, in the canonical parameter order."""
    bins = term_expectations(basis, inter.spaceA.twom, inter.spaceB.twom, vecs)
    g = np.zeros(len(inter.param_index))
    for p, (name, ix) in enumerate(inter.param_index):
        if name in ("h1A", "h1B"):
            a, c = ix
            val = bins.get((name, a, c), 0.0)
            if a != c:
                val += bins.get((name, c, a), 0.0)
        else:
            i, j, k, l = ix
            val = bins.get((name, i, j, k, l), 0.0)
            if (i, j) != (k, l):
                val += bins.get((name, k, l, i, j), 0.0)
        g[p] = val
    return g


def clusters(evals: np.ndarray, gap: float):
    """Split sorted eigenvalues into clusters whose neighbours differ by < gap."""
    out, cur = [], [0]
    for k in range(1, len(evals)):
        if evals[k] - evals[k - 1] < gap:
            cur.append(k)
        else:
            out.append(cur)
            cur = [k]
    out.append(cur)
    return out
