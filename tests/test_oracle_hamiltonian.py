"""Pins of the oracle's explicit Hamiltonian (Sec. II; App. B Eqs. (twobodybit),
(pntwobodybit)).

* Element-by-element equality with an independent Jordan-Wigner Kronecker
  construction on tiny spaces (signs of every term type, with spectators).
* Special cases with a closed form: 1 particle (H = one-body matrix), 2 like
  particles (H = pair-space two-body block plus energies), 1+1 (H = the
  cross-species block plus energies).
* Trace identity and Frobenius norm against the spectrum; symmetry.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh
from oracle import jw

SMALL_SHELLS = ((1, 0.3), (3, -0.7))  # 6 m-states per species


def _with_offdiag_one_body(inter, seed):
    """Add random symmetric M-conserving off-diagonal one-body terms."""
    rng = np.random.default_rng(seed)
    for h1, sp in ((inter.h1A, inter.spaceA), (inter.h1B, inter.spaceB)):
        for a in range(sp.n):
            for c in range(a + 1, sp.n):
                if sp.twom[a] == sp.twom[c]:
                    x = rng.standard_normal()
                    h1[a, c] = h1[c, a] = x
    return inter


@pytest.mark.parametrize("kA,kB,twoM", [(1, 1, 0), (2, 1, 1), (2, 2, 0), (3, 2, -1), (3, 3, 2), (2, 0, 0), (0, 3, 1)])
def test_bitstring_equals_jordan_wigner(kA, kB, twoM):
    sp = synth.make_space(SMALL_SHELLS)
    inter = _with_offdiag_one_body(synth.draw_interaction(sp, sp, 7 + kA + kB), 3)
    B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    H = oh.assemble(B, inter).toarray()
    HJ = jw.restrict(jw.hamiltonian(inter), B.states, sp.n, sp.n)
    assert np.abs(H - HJ).max() < 1e-12


def test_one_body_jumps_match_jordan_wigner_and_count():
    """The oracle's one-body jump list of one species (App. B.2): every entry
    (S', S, a, c, sign) equals the Jordan-Wigner matrix element
    <S'|c+_a c_c|S>, and there are N_det k (n - k + 1) of them (c occupied,
    a empty or a = c)."""
    sp = synth.make_space(SMALL_SHELLS)
    n = sp.n
    c = jw.annihilators(n)
    cd = [x.T.tocsr() for x in c]
    for k in (1, 2, 3):
        dets = ob.species_determinants(sp.twom, k)
        J = oh.one_body_jumps(sp.twom, k)
        assert len(J) == len(dets) * k * (n - k + 1)
        rows = [jw.occupation_index([b >> j & 1 for j in range(n)], n) for _, b in dets]
        ops = {}
        for t, src, a, cc, sign in J:
            if (a, cc) not in ops:
                ops[(a, cc)] = (cd[a] @ c[cc]).tocsr()
            assert ops[(a, cc)][rows[t], rows[src]] == sign


def test_jordan_wigner_anticommutation():
    c = jw.annihilators(4)
    for i in range(4):
        for j in range(4):
            ac = (c[i] @ c[j].T + c[j].T @ c[i]).toarray()
            assert np.allclose(ac, np.eye(16) * (i == j))
            assert np.allclose((c[i] @ c[j] + c[j] @ c[i]).toarray(), 0)


def test_one_particle_is_one_body_matrix():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = _with_offdiag_one_body(synth.draw_interaction(sp, sp, 11), 5)
    for twoM in (-3, 1, 5):
        B = ob.ProductBasis(sp.twom, 1, sp.twom, 0, twoM)
        H = oh.assemble(B, inter).toarray()
        modes = [next(i for i in range(sp.n) if SA >> i & 1) for SA, _ in B.states]
        assert np.allclose(H, inter.h1A[np.ix_(modes, modes)], atol=1e-14)


def test_two_like_particles_is_pair_block():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 13)
    for twoM in (0, 2, -4):
        B = ob.ProductBasis(sp.twom, 0, sp.twom, 2, twoM)
        H = oh.assemble(B, inter).toarray()
        pairs = []
        for _, SB in B.states:
            occ = [i for i in range(sp.n) if SB >> i & 1]
            pairs.append(tuple(occ))
        want = np.array([[inter.VBB[a, b, c, d] for (c, d) in pairs] for (a, b) in pairs])
        want += np.diag([sp.eps[a] + sp.eps[b] for (a, b) in pairs])
        assert np.allclose(H, want, atol=1e-14)


def test_one_plus_one_is_cross_block():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 17)
    for twoM in (0, 4):
        B = ob.ProductBasis(sp.twom, 1, sp.twom, 1, twoM)
        H = oh.assemble(B, inter).toarray()
        st = []
        for SA, SB in B.states:
            st.append((SA.bit_length() - 1, SB.bit_length() - 1))
        want = np.array([[inter.VAB[a, b, c, d] for (c, d) in st] for (a, b) in st])
        want += np.diag([sp.eps[a] + sp.eps[b] for (a, b) in st])
        assert np.allclose(H, want, atol=1e-14)


def _count_occ(B, spc, modes):
    n = 0
    for SA, SB in B.states:
        S = SA if spc == 0 else SB
        if all(S >> m & 1 for m in modes):
            n += 1
    return n


def _count_cross(B, a, b):
    return sum(1 for SA, SB in B.states if SA >> a & 1 and SB >> b & 1)


def test_trace_and_frobenius_identities():
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    ev = np.linalg.eigvalsh(H.toarray())
    n = sa.n
    tr = 0.0
    for a in range(n):
        tr += inter.h1A[a, a] * _count_occ(B, 0, [a]) + inter.h1B[a, a] * _count_occ(B, 1, [a])
    for a, b in itertools.combinations(range(n), 2):
        tr += inter.VAA[a, b, a, b] * _count_occ(B, 0, [a, b])
        tr += inter.VBB[a, b, a, b] * _count_occ(B, 1, [a, b])
    for a in range(n):
        for b in range(n):
            tr += inter.VAB[a, b, a, b] * _count_cross(B, a, b)
    assert abs(tr - ev.sum()) < 1e-9 * max(1.0, abs(tr))
    assert abs(H.diagonal().sum() - tr) < 1e-9 * max(1.0, abs(tr))
    fro2 = (H.multiply(H)).sum()
    assert abs(fro2 - (ev ** 2).sum()) < 1e-9 * fro2
    assert abs(H - H.T).max() == 0.0


def test_single_energy_term_spectrum():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 0)
    for arr in (inter.h1A, inter.h1B, inter.VAA, inter.VBB, inter.VAB):
        arr[...] = 0.0
    a0 = 5
    inter.h1A[a0, a0] = 1.0
    B = ob.ProductBasis(sp.twom, 2, sp.twom, 2, 0)
    ev = np.linalg.eigvalsh(oh.assemble(B, inter).toarray())
    n1 = _count_occ(B, 0, [a0])
    assert np.allclose(ev[-n1:], 1.0) and np.allclose(ev[:-n1], 0.0)


def test_sampled_rows_match_assembled():
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    V = synth.random_block(B.dim, 3, 5)
    rows = [0, 17, 320, 639]
    assert np.allclose(oh.hv_rows(B, inter, V, rows), (H @ V)[rows], atol=1e-13)
    L = oh.LazyIndex(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    for i in (0, 5, 333, 639):
        assert L.index(*L.state(i)) == i
        assert B.index[L.state(i)] == i
    T = oh.TermTables(inter)
    assert np.allclose(oh.hv_rows_lazy(L, T, V, rows), (H @ V)[rows], atol=1e-13)


def test_structural_nnz_small_case():
    """Structural pattern = pairs linked by popcount-limited moves with equal M.

    Brute force: (i, j) is structurally linked iff the A parts and B parts
    differ by at most two particles in total, checked pair by pair.
    """
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    P = oh.structural_pattern(B, inter)
    cnt = 0
    st = B.states
    for (A1, B1) in st:
        for (A2, B2) in st:
            dA = (A1 ^ A2).bit_count() // 2
            dB = (B1 ^ B2).bit_count() // 2
            if dA + dB <= 2:
                cnt += 1
    assert P.nnz == cnt
