"""Planted mistakes in the oracle: each must fail one of its pins.

A pin that a plausible mistake cannot fail pins nothing, so every mistake
below is planted in the oracle (on the CPU, through monkeypatch, only for
the test that plants it) and the test checks that a pin catches it:

* a dropped fermion sign, swapped annihilators in the like-particle
  two-body term (c_c c_d instead of c_d c_c, Sec. II), a creation onto an
  occupied mode not blocked, a dropped coefficient sign: the element-wise
  Jordan-Wigner comparison, and where it applies the closed form for two
  like particles;
* determinants sorted by bit value only (not by 2M first): the M-block
  structure of the product basis (App. A Eq. (part)): states of the wrong
  total 2M appear;
* Lanczos without reorthogonalisation (Alg. 1 as printed reorthogonalises):
  the comparison with dense eigh on the 640-dim space;
* a gradient that drops the Hermitian-conjugate term of off-diagonal
  parameters: the Euler identity sum_theta theta dE/dtheta = E.

A reversed sign convention (occupied modes after x instead of before)
passes every pin, as it should: for operator strings that conserve each
species' particle number the two conventions give the same matrix.
"""
import numpy as np

import synth
from oracle import basis as ob
from oracle import gradient as og
from oracle import hamiltonian as oh
from oracle import jw
from oracle import lanczos as ol

SMALL_SHELLS = ((1, 0.3), (3, -0.7))  # 6 m-states per species
_apply = oh.apply_string


def _small_inter(seed):
    sp = synth.make_space(SMALL_SHELLS)
    inter = synth.draw_interaction(sp, sp, seed)
    rng = np.random.default_rng(seed + 1)
    for h1 in (inter.h1A, inter.h1B):
        for a in range(sp.n):
            for c in range(a + 1, sp.n):
                if sp.twom[a] == sp.twom[c]:
                    h1[a, c] = h1[c, a] = rng.standard_normal()
    return sp, inter


def jw_error():
    """Largest |H - H_JW| over three tiny two-species spaces."""
    sp, inter = _small_inter(9)
    HJW = jw.hamiltonian(inter)
    err = 0.0
    for kA, kB, twoM in ((2, 2, 0), (3, 2, -1), (1, 2, 1)):
        B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
        H = oh.assemble(B, inter).toarray()
        err = max(err, np.abs(H - jw.restrict(HJW, B.states, sp.n, sp.n)).max())
    return err


def pair_block_error():
    """Two like particles: H = the pair block of V^BB plus energies."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 13)
    B = ob.ProductBasis(sp.twom, 0, sp.twom, 2, 0)
    H = oh.assemble(B, inter).toarray()
    pairs = [tuple(i for i in range(sp.n) if SB >> i & 1) for _, SB in B.states]
    want = np.array([[inter.VBB[a, b, c, d] for (c, d) in pairs] for (a, b) in pairs])
    want += np.diag([sp.eps[a] + sp.eps[b] for (a, b) in pairs])
    return np.abs(H - want).max()


def m_block_errors():
    """Basis states whose total 2M is wrong, and duplicated states."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    B = ob.ProductBasis(sp.twom, 2, sp.twom, 2, 0)
    m = lambda S: sum(sp.twom[i] for i in range(sp.n) if S >> i & 1)
    wrong_m = sum(1 for SA, SB in B.states if m(SA) + m(SB) != 0)
    return wrong_m + (len(B.states) - len(set(B.states)))


def test_pins_hold_on_the_unchanged_oracle():
    assert jw_error() < 1e-12
    assert pair_block_error() < 1e-14
    assert m_block_errors() == 0


def test_dropped_fermion_sign_fails(monkeypatch):
    def no_sign(SA, SB, ops):
        s, A2, B2 = _apply(SA, SB, ops)
        return (1 if s else 0), A2, B2
    monkeypatch.setattr(oh, "apply_string", no_sign)
    assert jw_error() > 1e-3


def test_swapped_like_particle_annihilators_fail(monkeypatch):
    def swapped(SA, SB, ops):
        if len(ops) == 4 and len({o[0] for o in ops}) == 1:
            ops = (ops[0], ops[1], ops[3], ops[2])
        return _apply(SA, SB, ops)
    monkeypatch.setattr(oh, "apply_string", swapped)
    assert jw_error() > 1e-3
    assert pair_block_error() > 1e-3


def test_unblocked_creation_fails(monkeypatch):
    def unblocked(SA, SB, ops):
        sign = 1
        for spc, dag, x in reversed(ops):
            bit = 1 << x
            S = SA if spc == 0 else SB
            before = (S & (bit - 1)).bit_count() + (SA.bit_count() if spc == 1 else 0)
            if dag:
                S |= bit  # the Pauli test on creation is missing
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
    monkeypatch.setattr(oh, "apply_string", unblocked)
    try:
        err = jw_error()
    except KeyError:  # a term lost a particle: its target is not a basis state
        return
    assert err > 1e-3


def test_dropped_coefficient_sign_fails(monkeypatch):
    base = oh.TermTables

    class AbsTables(base):
        def __init__(self, inter, tol=0.0):
            super().__init__(inter, tol)
            for fam in (self.twoAA, self.twoBB, self.pn):
                for key, L in fam.items():
                    fam[key] = [(a, b, abs(v)) for a, b, v in L]
    monkeypatch.setattr(oh, "TermTables", AbsTables)
    assert jw_error() > 1e-3
    assert pair_block_error() > 1e-3


def test_reversed_sign_convention_passes(monkeypatch):
    def after(SA, SB, ops):
        sign = 1
        for spc, dag, x in reversed(ops):
            bit = 1 << x
            S = SA if spc == 0 else SB
            n_after = (S >> (x + 1)).bit_count() + (SB.bit_count() if spc == 0 else 0)
            if dag:
                if S & bit:
                    return 0, 0, 0
                S |= bit
            else:
                if not S & bit:
                    return 0, 0, 0
                S ^= bit
            if n_after & 1:
                sign = -sign
            if spc == 0:
                SA = S
            else:
                SB = S
        return sign, SA, SB
    monkeypatch.setattr(oh, "apply_string", after)
    assert jw_error() < 1e-12
    assert pair_block_error() < 1e-14


def test_determinants_sorted_by_value_only_fail(monkeypatch):
    orig = ob.species_determinants

    def by_value(twom, k):
        return sorted(orig(twom, k), key=lambda t: t[1])
    monkeypatch.setattr(ob, "species_determinants", by_value)
    assert m_block_errors() > 0


def _lanczos_no_reorth(matvec, D, nev, tol, normH, v1, max_iter=None):
    """Alg. 1 with the reorthogonalisation left out (the planted mistake)."""
    import scipy.linalg as sla
    max_iter = min(max_iter or D, D)
    Vs = np.zeros((D, max_iter + 1))
    Vs[:, 0] = v1 / np.linalg.norm(v1)
    alpha, beta = np.zeros(max_iter), np.zeros(max_iter)
    for k in range(max_iter):
        w = matvec(Vs[:, k])
        alpha[k] = Vs[:, k] @ w
        w = w - alpha[k] * Vs[:, k] - (beta[k - 1] * Vs[:, k - 1] if k else 0.0)
        beta[k] = np.linalg.norm(w)
        m = k + 1
        if m >= nev:
            theta, U = sla.eigh_tridiagonal(alpha[:m], beta[:m - 1])
            res = beta[k] * np.abs(U[m - 1, :nev])
            if np.all(res <= tol * normH) or m == D:
                return theta[:nev], Vs[:, :m] @ U[:, :nev], res, m
        Vs[:, k + 1] = w / beta[k]
    raise RuntimeError("not converged")


def test_lanczos_without_reorthogonalisation_fails(monkeypatch):
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    ev = np.linalg.eigvalsh(H.toarray())
    normH = max(abs(ev[0]), abs(ev[-1]))
    v1 = synth.random_block(B.dim, 1, 99)[:, 0]
    th, X, _, _ = ol.lanczos(lambda x: H @ x, B.dim, w.nev, w.tol, normH, v1)
    assert np.abs(th - ev[:w.nev]).max() <= 1e-9 * normH
    monkeypatch.setattr(ol, "lanczos", _lanczos_no_reorth)
    th, X, _, _ = ol.lanczos(lambda x: H @ x, B.dim, w.nev, w.tol, normH, v1)
    ok_values = np.abs(th - ev[:w.nev]).max() <= 1e-9 * normH
    ok_vectors = np.abs(X.T @ X - np.eye(w.nev)).max() < 1e-10
    assert not (ok_values and ok_vectors)


def test_gradient_without_conjugate_terms_fails(monkeypatch):
    def no_conjugate(basis, inter, vecs):
        bins = og.term_expectations(basis, inter.spaceA.twom, inter.spaceB.twom, vecs)
        g = np.zeros(len(inter.param_index))
        for p, (name, ix) in enumerate(inter.param_index):
            g[p] = bins.get((name,) + tuple(ix), 0.0)
        return g
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    ev, U = np.linalg.eigh(oh.assemble(B, inter).toarray())
    euler = lambda: abs(og.hf_gradient(B, inter, U[:, :1]) @ inter.theta - ev[0])
    assert euler() < 1e-10 * abs(ev[0])
    monkeypatch.setattr(og, "hf_gradient", no_conjugate)
    assert euler() > 1e-3 * abs(ev[0])
