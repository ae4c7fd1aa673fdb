"""Hellmann-Feynman gradient on the GPU (trbl_grad) against the oracle.

H of Sec. II is linear in its parameters, so dE_k/dtheta = <x_k|dH/dtheta|x_k>.
Pins: element-wise agreement with the oracle's term-by-term expectation on
the same vectors (FP64, 1e-10); cluster sums equal the sum of single-vector
gradients; the Euler identity sum_theta theta dE/dtheta = E (H homogeneous of
degree one in its parameters); central finite differences of the GPU
eigenvalues with h = 1e-4 (relative 1e-5); the autograd wrapper's backward."""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import gradient as og
from oracle import hamiltonian as oh

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    w, sa, sb, inter = synth.workload("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    ev, U = np.linalg.eigh(H.toarray())
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    return w, sa, inter, B, ev, U, tb, th


def test_grad_matches_oracle_single_vectors(small):
    w, sa, inter, B, ev, U, tb, th = small
    for k in (0, 1, 5):
        x = U[:, k:k + 1]
        g_or = og.hf_gradient(B, inter, x)
        g_gpu = trbl.hf_gradient(th, torch.from_numpy(np.ascontiguousarray(x)).cuda())
        assert np.abs(g_gpu - g_or).max() <= 1e-10, np.abs(g_gpu - g_or).max()


def test_grad_cluster_sum_and_fp32(small):
    w, sa, inter, B, ev, U, tb, th = small
    X = torch.from_numpy(np.ascontiguousarray(U[:, :4])).cuda()
    g4 = trbl.hf_gradient(th, X)
    g1 = sum(trbl.hf_gradient(th, X[:, k:k + 1].contiguous()) for k in range(4))
    assert np.abs(g4 - g1).max() <= 1e-10
    g32 = trbl.hf_gradient(th, X.float())
    assert np.abs(g32 - g4).max() <= 1e-5 * max(1.0, np.abs(g4).max())


def test_grad_euler_identity_with_gpu_eigenvectors(small):
    w, sa, inter, B, ev, U, tb, th = small
    evals, resid, X, st = trbl.solve(th, w.nev, w.q, w.max_basis, w.tol)
    normH = max(abs(ev[0]), abs(ev[-1]))
    for cl in trbl.clusters_of(evals, 1e-8 * normH):
        g = trbl.hf_gradient(th, X, cl)
        assert abs(g @ inter.theta - evals[cl].sum()) <= 1e-9 * normH * len(cl)


def test_grad_central_differences_gpu_solver(small):
    w, sa, inter, B, ev, U, tb, th = small
    evals, resid, X, st = trbl.solve(th, 3, 4, w.max_basis, 1e-12)
    g = trbl.hf_gradient(th, X, [0])
    rng = np.random.default_rng(5)
    names = [n for n, _ in inter.param_index]
    picks = set(rng.choice(len(names), 10, replace=False).tolist())
    for kind in ("h1A", "h1B", "VAA", "VBB", "VAB"):
        idx = [i for i, n in enumerate(names) if n == kind]
        picks.add(idx[0])
        picks.add(idx[len(idx) // 2])
    hstep = 1e-4
    for p in sorted(picks):
        e = []
        for sgn in (1, -1):
            t = inter.theta.copy()
            t[p] += sgn * hstep
            hp = trbl.Hamiltonian(tb, *trbl.arrays_from_theta(sa.twom, sa.twom, t))
            e.append(trbl.solve(hp, 3, 4, w.max_basis, 1e-12, want_vectors=False)[0][0])
        fd = (e[0] - e[1]) / (2 * hstep)
        assert abs(fd - g[p]) <= 1e-5 * max(1.0, abs(g[p])), (p, inter.param_index[p], fd, g[p])


def test_grad_autograd_function(small):
    w, sa, inter, B, ev, U, tb, th = small
    theta = torch.from_numpy(inter.theta.copy()).requires_grad_(True)
    evals = trbl.LowestEigenvalues.apply(theta, tb, 4, 4, w.max_basis, 1e-12)
    loss = evals[0] + 0.5 * evals[2]
    loss.backward()
    assert np.allclose(evals.detach().numpy(), ev[:4], atol=1e-9 * abs(ev).max())
    ref = og.hf_gradient(B, inter, U[:, 0:1]) + 0.5 * og.hf_gradient(B, inter, U[:, 2:3])
    assert np.abs(theta.grad.numpy() - ref).max() <= 1e-8


def test_grad_on_gradient_batch_space():
    """The 12-m-state 4+4 space (D = 28,503) with parameter set seed 100: the
    GPU gradient of the lowest level against the oracle's gradient of the same
    vector, and the Euler identity for the 20 lowest levels."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 100)
    tb = trbl.Basis(sp, 4, sp, 4, 0)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    evals, resid, X, st = trbl.solve(th, 20, 8, 256, 1e-10)
    normH = st["normH"]
    for cl in trbl.clusters_of(evals, 1e-8 * normH):
        g = trbl.hf_gradient(th, X, cl)
        assert abs(g @ inter.theta - evals[cl].sum()) <= 1e-9 * normH * len(cl)
    B = ob.ProductBasis(sp.twom, 4, sp.twom, 4, 0)
    x0 = X[:, 0:1].cpu().numpy()
    g_or = og.hf_gradient(B, inter, x0)
    g_gpu = trbl.hf_gradient(th, X, [0])
    assert np.abs(g_gpu - g_or).max() <= 1e-10


def test_grad_clusters_in_one_pass():
    """trbl_grad_clusters: the gradients of all level clusters from one pass
    equal those of one trbl_grad call per cluster (FP64: to 1e-12 of the
    largest component; the atomic adds sum in a different order), each
    satisfies the Euler identity, and the oracle agrees for the lowest
    level.  Uneven clusters (1, 3 and 2 vectors) of the small space's exact
    eigenvectors check the lane segmentation."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 100)
    tb = trbl.Basis(sp, 4, sp, 4, 0)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    evals, resid, X, st = trbl.solve(th, 20, 8, 256, 1e-10)
    normH = st["normH"]
    cls = trbl.clusters_of(evals, 1e-8 * normH)
    many = trbl.hf_gradient_clusters(th, X, cls)
    for cl, g in zip(cls, many):
        g1 = trbl.hf_gradient(th, X, cl)
        assert np.abs(g - g1).max() <= 1e-12 * np.abs(g1).max()
        assert abs(g @ inter.theta - evals[cl].sum()) <= 1e-9 * normH * len(cl)
    odd = [[0], [1, 2, 3], [4, 5]]
    for cl, g in zip(odd, trbl.hf_gradient_clusters(th, X, odd)):
        g1 = trbl.hf_gradient(th, X, cl)
        assert np.abs(g - g1).max() <= 1e-12 * np.abs(g1).max()
    g32 = trbl.hf_gradient_clusters(th, X.float(), odd)
    for cl, g in zip(odd, g32):
        g1 = trbl.hf_gradient(th, X, cl)
        assert np.abs(g - g1).max() <= 1e-5 * np.abs(g1).max()


def test_grad_clusters_rejects_bad_boundaries(small):
    w, sa, inter, B, ev, U, tb, th = small
    X = torch.from_numpy(np.ascontiguousarray(U[:, :4])).cuda()
    n = trbl.trbl_param_count(tb.handle)
    out = np.zeros((2, n))
    import ctypes
    for first in ([0, 2, 2], [1, 2, 4], [0, 3, 5]):
        fa = (ctypes.c_int * 3)(*first)
        rc = trbl.lib().trbl_grad_clusters(th.handle, X.data_ptr(), 4, 4, trbl.TRBL_F64, fa, 2,
                                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, 0)
        assert rc == trbl.TRBL_ERR_ARG
