"""Pins of the oracle's determinant enumeration and product basis.

Sources: Table I (App. A) for the bit representation and its order; the
dimensions printed in the paper for the 20Ne sd space (640, App. C Fig. 8),
24Mg sd space (28,503, App. C Fig. 9), 48Cr pf space (1,963,461, Sec. IV A),
112Sn (6,210,638, Sec. IV C) and 56Ni (1,087,455,228, App. B); the partition
counts of App. C (162 for 20Ne, 1020 for 24Mg); closed forms for the number
of one-body jumps.
"""
import itertools
import os

import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table1():
    rows = []
    for line in open(os.path.join(GOLDEN, "table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        bits = [int(x) for x in parts[1:9]]
        group = tuple(int(x) for x in parts[9].split(",")) if len(parts) > 9 else None
        rows.append((int(parts[0]), bits, group))
    return rows


def test_table1_bit_rows_and_order():
    sp = synth.make_space(synth.TABLE1_SHELLS)
    got = ob.table1_order(sp.twom, sp.orbit, 3, 1)
    want = _read_table1()
    assert len(got) == len(want) == 9
    prev_group = None
    for (N, occ, bits), (serial, wbits, wgroup) in zip(got, want):
        assert [bits >> i & 1 for i in range(8)] == wbits, serial
        if wgroup is not None:
            assert N == wgroup and N != prev_group
        else:
            assert N == prev_group
        prev_group = N


def test_table1_determinants_are_the_M_block():
    sp = synth.make_space(synth.TABLE1_SHELLS)
    dets = [b for (m, b) in ob.species_determinants(sp.twom, 3) if m == 1]
    assert sorted(dets) == sorted(r[2] for r in ob.table1_order(sp.twom, sp.orbit, 3, 1))


@pytest.mark.parametrize("k,want", [(2, 640), (4, 28503)])
def test_paper_dimensions_sd_enumerated(k, want):
    sp = synth.make_space(synth.SPACE12_SHELLS)
    B = ob.ProductBasis(sp.twom, k, sp.twom, k, 0)
    assert B.dim == want
    assert len(set(B.states)) == want
    for (SA, SB) in B.states[:: max(1, want // 200)]:
        mA = sum(sp.twom[i] for i in range(sp.n) if SA >> i & 1)
        mB = sum(sp.twom[i] for i in range(sp.n) if SB >> i & 1)
        assert mA + mB == 0
        assert SA.bit_count() == k and SB.bit_count() == k


def test_paper_dimension_pf_48Cr():
    sp = synth.make_space(synth.SPACE20_SHELLS)
    L = oh.LazyIndex(sp.twom, 4, sp.twom, 4, 0)
    assert L.dim == 1963461
    assert len(L.detsA) == 4845


def test_generating_function_matches_enumeration():
    for shells, k1, k2, twoM in ((synth.SPACE12_SHELLS, 2, 2, 0), (synth.SPACE12_SHELLS, 3, 2, 1),
                                 (synth.SPACE12_SHELLS, 4, 4, 0), (synth.TABLE1_SHELLS, 3, 0, 1),
                                 (synth.SPACE12_SHELLS, 1, 0, 3)):
        sp = synth.make_space(shells)
        B = ob.ProductBasis(sp.twom, k1, sp.twom, k2, twoM)
        assert B.dim == ob.dimension_by_generating_function(sp.twom, k1, sp.twom, k2, twoM)


def test_generating_function_paper_dimensions():
    sp20 = synth.make_space(synth.SPACE20_SHELLS)
    assert ob.dimension_by_generating_function(sp20.twom, 4, sp20.twom, 4, 0) == 1963461
    # 112Sn: 12 neutrons in g7/2 d5/2 d3/2 s1/2 h11/2, M = 0, positive parity.
    sn = synth.make_space(((7, 0), (5, 0), (3, 0), (1, 0), (11, 0)))
    parity = [1 if o == 4 else 0 for o in sn.orbit]
    assert ob.dimension_by_generating_function((), 0, sn.twom, 12, 0, parity, 0) == 6210638


@pytest.mark.parametrize("k,want", [(2, 162), (4, 1020)])
def test_paper_partition_counts_sd(k, want):
    """The sd-shell partitions (N^p, N^n, M^p) the paper counts for 20Ne
    (162) and 24Mg (1020) in App. C; their states add up to the M-scheme
    dimension."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    P = ob.partitions(sp.twom, sp.orbit, k, sp.twom, sp.orbit, k, 0)
    assert len(P) == want
    assert sum(P.values()) == ob.ProductBasis(sp.twom, k, sp.twom, k, 0).dim


def test_generating_function_56Ni():
    """56Ni in the pf shell, 8 + 8 particles, M = 0: 1,087,455,228 states
    (the dimension the paper gives when it motivates the on-the-fly
    product, App. B)."""
    sp20 = synth.make_space(synth.SPACE20_SHELLS)
    assert ob.dimension_by_generating_function(sp20.twom, 8, sp20.twom, 8, 0) == 1087455228


def test_one_body_jump_closed_form():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    for k in (1, 2, 3, 4):
        ndet = len(ob.species_determinants(sp.twom, k))
        assert ob.one_body_jump_count(sp.twom, k) == ndet * k * (sp.n - k)


def _targets_by_moves(twom, k):
    """Like-particle targets counted by explicit moves: from every determinant,
    one particle i -> j with m_i = m_j, or a pair {i, j} -> {a, b} with
    m_i + m_j = m_a + m_b (App. B.1: the states a one- or two-body term
    reaches inside one M block).  Distinct moves reach distinct states."""
    n = len(twom)
    cnt = 0
    for occ in itertools.combinations(range(n), k):
        empty = [x for x in range(n) if x not in occ]
        cnt += sum(1 for i in occ for j in empty if twom[i] == twom[j])
        cnt += sum(1 for i, j in itertools.combinations(occ, 2) for a, b in itertools.combinations(empty, 2)
                   if twom[i] + twom[j] == twom[a] + twom[b])
    return cnt


@pytest.mark.parametrize("shells,k", [(synth.SPACE12_SHELLS, 2), (synth.SPACE12_SHELLS, 4),
                                      (synth.SPACE20_SHELLS, 2), (synth.SPACE20_SHELLS, 3)])
def test_same_species_targets_by_moves(shells, k):
    """The xor-popcount count of the oracle equals the count of explicit
    moves; with 2 particles every other pair state of equal M is a target."""
    sp = synth.make_space(shells)
    assert ob.same_species_targets(sp.twom, k) == _targets_by_moves(sp.twom, k)
    if k == 2 and sp.n == 12:
        dets = ob.species_determinants(sp.twom, 2)
        per_m = {}
        for m, _ in dets:
            per_m[m] = per_m.get(m, 0) + 1
        assert ob.same_species_targets(sp.twom, 2) == sum(c * (c - 1) for c in per_m.values())


def test_species_order_is_M_then_value():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    dets = ob.species_determinants(sp.twom, 3)
    keys = [(m, b) for m, b in dets]
    assert keys == sorted(keys)
    for m, b in dets:
        assert m == sum(sp.twom[i] for i in range(sp.n) if b >> i & 1)
