"""The loop order of the split product's cross-term kernel, checked on the
host against the oracle.

The cross-species term of H (App. B.2, Eq. (pntwobodybit)) is a sum over
pairs of a proton jump pA -> pA' (a+_a a_c, sign s_p) and a neutron jump
nB -> nB' (b+_b b_d, sign s_n) whose 2m transfers cancel, each contributing
s_p s_n V^AB_{ab,cd} at row (pA', nB'), column (pA, nB).  The
source-stationary kernel enumerates these pairs from the source side: for
each proton jump into pA', it walks every neutron row nB of the source slab
and every outgoing neutron jump of nB in the opposite transfer class.  Here
that enumeration is written out in numpy over the library's exported jump
lists (which include the number operators a = c and b = d).  The matrix it
builds must equal the oracle's explicit H for an interaction with only V^AB
(no one-body or like-particle terms), element by element.  No GPU is
needed.
"""
import dataclasses
from collections import defaultdict

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh

trbl = pytest.importorskip("paper_1902_02064_gb300")


def _cross_term_by_source_rows(tb, twomA, twomB, VAB, twoM, index):
    bitsA, mA, bitsB, mB, blocks = tb.export()
    tgtA, srcA, aA, cA, sA = tb.export_jumps(0)
    tgtB, srcB, aB, cB, sB = tb.export_jumps(1)
    out = defaultdict(list)  # (source neutron determinant, transfer) -> outgoing jumps
    for t, s, b, d, sg in zip(tgtB, srcB, aB, cB, sB):
        out[(int(s), twomB[b] - twomB[d])].append((int(t), int(b), int(d), int(sg)))
    rows_of_M = defaultdict(list)
    for n, m in enumerate(mB):
        rows_of_M[int(m)].append(n)
    H = defaultdict(float)
    for pt, ps, a, c, sp in zip(tgtA, srcA, aA, cA, sA):
        dP = twomA[a] - twomA[c]
        for n in rows_of_M.get(twoM - int(mA[ps]), ()):  # the source slab of proton jump (ps -> pt)
            for nt, b, d, sn in out.get((n, -dP), ()):  # outgoing neutron jumps of the opposite class
                i = index[(int(bitsA[ps]), int(bitsB[n]))]
                j = index[(int(bitsA[pt]), int(bitsB[nt]))]
                H[(j, i)] += sp * sn * VAB[a, b, c, d]
    return H


@pytest.mark.parametrize("kA,kB,twoM", [(2, 2, 0), (3, 1, -2), (1, 1, 2), (2, 3, 3)])
def test_source_stationary_cross_term_equals_oracle(kA, kB, twoM):
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 36)
    only_ab = dataclasses.replace(inter, h1A=np.zeros_like(inter.h1A), h1B=np.zeros_like(inter.h1B),
                                  VAA=np.zeros_like(inter.VAA), VBB=np.zeros_like(inter.VBB))
    B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    ref = oh.assemble(B, only_ab).toarray()
    tb = trbl.Basis(sp, kA, sp, kB, twoM)
    assert tb.dim == B.dim
    H = _cross_term_by_source_rows(tb, list(sp.twom), list(sp.twom), inter.VAB, twoM, B.index)
    M = np.zeros_like(ref)
    for (j, i), v in H.items():
        M[j, i] = v
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(M - ref).max() <= 1e-13 * scale
