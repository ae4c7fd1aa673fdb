"""Pins of the oracle's eigensolver (Algorithm 1 with full reorthogonalisation)
and of its Hellmann-Feynman gradient.

* Lanczos Ritz values against numpy's dense eigh (a library routine) and
  against a diagonal matrix with a known spectrum.
* Gradient: the Euler identity for a Hamiltonian linear and homogeneous in
  its parameters (sum_theta theta dE/dtheta = E) and central finite
  differences of the dense eigenvalues.
"""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import gradient as og
from oracle import hamiltonian as oh
from oracle import lanczos as ol


@pytest.fixture(scope="module")
def small():
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    return w, B, inter, H


def test_lanczos_matches_dense_eigh(small):
    w, B, inter, H = small
    ev, U = ol.dense_eigh(H)
    normH = max(abs(ev[0]), abs(ev[-1]))
    v1 = synth.random_block(B.dim, 1, 99)[:, 0]
    th, X, res, it = ol.lanczos(lambda x: H @ x, B.dim, w.nev, w.tol, normH, v1)
    assert np.abs(th - ev[: w.nev]).max() <= 1e-9 * normH
    R = H @ X - X * th
    assert np.linalg.norm(R, axis=0).max() <= 1e-8 * normH
    assert np.abs(X.T @ X - np.eye(w.nev)).max() < 1e-10


def test_lanczos_known_spectrum():
    D = 300
    lam = np.linspace(-3.0, 5.0, D) ** 3
    v1 = synth.random_block(D, 1, 3)[:, 0]
    th, X, res, it = ol.lanczos(lambda x: lam * x, D, 5, 1e-12, np.abs(lam).max(), v1)
    assert np.allclose(th, np.sort(lam)[:5], atol=1e-9 * np.abs(lam).max())


def test_hf_gradient_euler_identity(small):
    w, B, inter, H = small
    ev, U = ol.dense_eigh(H)
    for k in (0, 3, 7):
        g = og.hf_gradient(B, inter, U[:, k:k + 1])
        assert abs(g @ inter.theta - ev[k]) < 1e-10 * max(1.0, abs(ev[k]))


def test_hf_gradient_finite_differences():
    sp = synth.make_space(((1, 0.0), (3, 1.0)))
    inter = synth.draw_interaction(sp, sp, 21)
    B = ob.ProductBasis(sp.twom, 2, sp.twom, 1, 1)
    ev, U = ol.dense_eigh(oh.assemble(B, inter))
    cl = og.clusters(ev, 1e-6)
    target = cl[0]
    g = og.hf_gradient(B, inter, U[:, target])
    h = 1e-4
    for p in range(len(inter.theta)):
        tp = inter.theta.copy(); tp[p] += h
        tm = inter.theta.copy(); tm[p] -= h
        ep = ol.dense_eigh(oh.assemble(B, synth.interaction_from_theta(sp, sp, tp, inter.param_index)))[0]
        em = ol.dense_eigh(oh.assemble(B, synth.interaction_from_theta(sp, sp, tm, inter.param_index)))[0]
        fd = (ep[target].sum() - em[target].sum()) / (2 * h)
        assert abs(fd - g[p]) <= 1e-5 * max(1.0, abs(g[p])), (p, inter.param_index[p], fd, g[p])


def test_interaction_theta_roundtrip():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 4)
    back = synth.interaction_from_theta(sp, sp, inter.theta, inter.param_index)
    for a, b in ((inter.h1A, back.h1A), (inter.VAA, back.VAA), (inter.VBB, back.VBB), (inter.VAB, back.VAB)):
        assert np.array_equal(a, b)
