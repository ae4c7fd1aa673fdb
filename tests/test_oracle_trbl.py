"""Pins of the oracle's thick-restart block Lanczos (Sec. III C/D, Alg. 3/4,
Eq. (trb-tmat)).

* Eigenvalues against numpy's dense eigh on the 640-dim space, with thick
  restarts (basis 40 for 10 pairs).
* Block size 1 without restarts is Alg. 1: the same Ritz values and step
  count as the oracle's simple Lanczos from the same start vector.
* The algebra at every step: the stored vectors are orthonormal, and
  H V[:, :n-p] = V T[:, :n-p] (the block-tridiagonal relation of
  Eq. (tmat-blan), and after a restart the arrow form of Eq. (trb-tmat)
  with the kept Ritz values on the diagonal).
* A doubly degenerate lowest eigenvalue is found twice with block size 2.
"""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh
from oracle import lanczos as ol
from oracle import trbl as ot


@pytest.fixture(scope="module")
def small():
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    ev = np.linalg.eigvalsh(H.toarray())
    return w, H, ev, max(abs(ev[0]), abs(ev[-1]))


def test_trbl_matches_dense_eigh(small):
    w, H, ev, normH = small
    V1 = synth.random_block(H.shape[0], 4, 3)
    th, X, res, st = ot.trbl(ot.block_matvec(H), H.shape[0], 10, 4, 40, 17, 1e-10, normH, V1)
    assert st["restarts"] >= 1
    assert np.abs(th - ev[:10]).max() <= 1e-9 * normH
    assert np.linalg.norm(H @ X - X * th, axis=0).max() <= 1e-8 * normH
    assert np.abs(X.T @ X - np.eye(10)).max() <= 1e-12


def test_block_size_one_is_simple_lanczos(small):
    w, H, ev, normH = small
    v1 = synth.random_block(H.shape[0], 1, 99)
    th, X, res, st = ot.trbl(ot.block_matvec(H), H.shape[0], 5, 1, 400, 5, 1e-9, normH, v1)
    th1, X1, res1, it1 = ol.lanczos(lambda x: H @ x, H.shape[0], 5, 1e-9, normH, v1[:, 0])
    assert st["restarts"] == 0
    assert abs(st["steps"] - it1) <= 1
    assert np.abs(th - th1).max() <= 1e-10 * normH


def test_lanczos_relation_and_orthogonality_at_every_step(small):
    w, H, ev, normH = small
    seen = {"restarted": 0, "steps": 0}

    def check(s):
        V, T = s["V"], s["T"]
        n = V.shape[1]
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13
        if s["restarted"] or n > 4:
            m = n - 4
            assert np.abs(H @ V[:, :m] - V @ T[:, :m]).max() <= 1e-12 * normH
        if s["restarted"]:
            ls = n - 4
            assert np.array_equal(np.diag(T[:ls, :ls]), s["theta"][:ls])
            assert np.count_nonzero(T[:ls, :ls] - np.diag(np.diag(T[:ls, :ls]))) == 0
            seen["restarted"] += 1
        seen["steps"] += 1

    V1 = synth.random_block(H.shape[0], 4, 3)
    ot.trbl(ot.block_matvec(H), H.shape[0], 10, 4, 40, 17, 1e-10, normH, V1, snapshot=check)
    assert seen["restarted"] >= 1 and seen["steps"] > 10


def test_degenerate_pair_found_with_block_size_two():
    D = 400
    lam = np.concatenate(([-1.0, -1.0], np.linspace(0.0, 3.0, D - 2)))
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
    H = (Q * lam) @ Q.T
    V1 = synth.random_block(D, 2, 4)
    th, X, res, st = ot.trbl(ot.block_matvec(H), D, 3, 2, 40, 8, 1e-11, 3.0, V1)
    assert np.abs(th[:2] + 1.0).max() <= 1e-10 and abs(th[2]) <= 1e-10


def test_relation_catches_a_wrong_restart_coupling(small):
    """The relation test is sharp: in a restarted snapshot, dropping the
    coupling r of Eq. (trb-tmat), or flipping its sign, breaks
    H V[:, :l_s] = V T[:, :l_s] by far more than rounding."""
    w, H, ev, normH = small
    snaps = []
    V1 = synth.random_block(H.shape[0], 4, 3)
    ot.trbl(ot.block_matvec(H), H.shape[0], 10, 4, 40, 17, 1e-10, normH, V1,
            snapshot=lambda s: snaps.append(s) if s["restarted"] else None)
    s = snaps[0]
    V, T = s["V"], s["T"]
    ls = V.shape[1] - 4
    assert np.abs(H @ V[:, :ls] - V @ T[:, :ls]).max() <= 1e-12 * normH
    for bad in (0.0, -1.0):
        Tb = T.copy()
        Tb[ls:, :ls] *= bad
        assert np.abs(H @ V[:, :ls] - V @ Tb[:, :ls]).max() > 1e-3 * normH
