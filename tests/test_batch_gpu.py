"""Batched thick-restart block Lanczos (trbl_solve_batch): many parameter
sets on one basis, one persistent product launch per step and the rest of
each step replayed from CUDA graphs.

Parity: every set's eigenvalues against dense eigh (D = 640, FP64 1e-9 ||H||,
mixed 1e-6 ||H||) and, on the 12-m-state 4+4 space (D = 28,503), against the
single-Hamiltonian solver, which the solver tests pin to the oracle; the
Hellmann-Feynman Euler identity for every set; the apply autotuner keeps the
product's results."""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu


def _sets(kA, kB, seeds):
    sp = synth.make_space(synth.SPACE12_SHELLS)
    tb = trbl.Basis(sp, kA, sp, kB, 0)
    inters = [synth.draw_interaction(sp, sp, sd) for sd in seeds]
    hs = [trbl.Hamiltonian.from_interaction(tb, it) for it in inters]
    return sp, tb, inters, hs


@pytest.mark.parametrize("reorth", [trbl.TRBL_REORTH_SELECTIVE, trbl.TRBL_REORTH_TWICE])
@pytest.mark.parametrize("precision,tol,bar", [(trbl.TRBL_PREC_F64, 1e-10, 1e-9), (trbl.TRBL_PREC_MIXED, 1e-6, 1e-6)])
def test_batch_small_against_dense(precision, tol, bar, reorth):
    """Both reorthogonalisation schedules of the batched step (the selective
    one takes its DGKS decision per set on the device)."""
    seeds = list(range(200, 208))
    sp, tb, inters, hs = _sets(2, 2, seeds)
    B = ob.ProductBasis(sp.twom, 2, sp.twom, 2, 0)
    ev, rs, X, status, st = trbl.solve_batch(hs, 10, 4, 40, tol, precision=precision, want_vectors=True,
                                             reorth=reorth)
    assert st["rc"] == trbl.TRBL_OK, st["message"]
    assert status == [0] * len(seeds)
    for k, it in enumerate(inters):
        ref = np.linalg.eigvalsh(oh.assemble(B, it).toarray())
        normH = max(abs(ref[0]), abs(ref[-1]))
        assert np.abs(ev[k] - ref[:10]).max() <= bar * normH, (k, np.abs(ev[k] - ref[:10]).max())
    assert st["iterations"] > 0


def test_batch_gradient_space_matches_single_solves():
    seeds = list(range(100, 108))
    sp, tb, inters, hs = _sets(4, 4, seeds)
    ev, rs, X, status, st = trbl.solve_batch(hs, 20, 8, 256, 1e-10, want_vectors=True)
    assert st["rc"] == trbl.TRBL_OK, st["message"]
    for k in (0, 3, 7):
        e1 = trbl.solve(hs[k], 20, 8, 256, 1e-10, want_vectors=False)[0]
        assert np.abs(ev[k] - e1).max() <= 1e-9 * st["normH"]
    for k, (h, it) in enumerate(zip(hs, inters)):
        for cl in trbl.clusters_of(ev[k], 1e-8 * st["normH"]):
            g = trbl.hf_gradient(h, X[k], cl)
            assert abs(g @ it.theta - ev[k][cl].sum()) <= 1e-9 * st["normH"] * len(cl)


def test_apply_autotune_keeps_results():
    sp, tb, inters, hs = _sets(4, 4, [100])
    h = hs[0]
    V = torch.from_numpy(synth.random_block(tb.dim, 8, 4)).float().cuda()
    W0 = h.apply(V).clone()
    ms, best = trbl.apply_autotune(h, 8, trbl.TRBL_F32)
    # every shape applies to 32-byte FP32 rows except the split products (q = 16, 32, 64)
    assert best in (16, 32, 64, 128) and all(m > 0 for m in ms[:13]) and not any(np.isfinite(ms[13:]))
    W1 = h.apply(V)
    torch.cuda.synchronize()
    assert torch.allclose(W0, W1, rtol=1e-6, atol=1e-6 * W0.abs().max().item())


@pytest.mark.parametrize("precision,tol,bar", [(trbl.TRBL_PREC_F64, 1e-10, 1e-9), (trbl.TRBL_PREC_MIXED, 1e-6, 1e-6)])
def test_batch_sectors_of_uneven_dimension(precision, tol, bar):
    """Sectors of other particle numbers and 2M (each on its own basis, with
    its own tables, work list and dimension) in one batched solve: every
    sector's eigenvalues against dense eigh of the oracle's H, and its Ritz
    vectors against that H (residual)."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 301)
    sectors = [(2, 2, 0), (2, 2, 2), (3, 2, 1), (2, 3, -1), (1, 3, 0)]
    bases = [trbl.Basis(sp, kA, sp, kB, tm) for kA, kB, tm in sectors]
    hs = [trbl.Hamiltonian.from_interaction(b, inter) for b in bases]
    dims = [b.dim for b in bases]
    assert len(set(dims)) > 2
    nev, q, mb = 8, 4, 40
    ev, rs, X, status, st = trbl.solve_batch(hs, nev, q, mb, tol, precision=precision, want_vectors=True)
    assert st["rc"] == trbl.TRBL_OK, st["message"]
    assert status == [0] * len(sectors)
    assert isinstance(X, list) and [x.shape[0] for x in X] == dims
    for k, (kA, kB, tm) in enumerate(sectors):
        B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, tm)
        H = oh.assemble(B, inter)
        ref = np.linalg.eigvalsh(H.toarray())
        normH = max(abs(ref[0]), abs(ref[-1]))
        assert np.abs(ev[k] - ref[:nev]).max() <= bar * normH, (k, np.abs(ev[k] - ref[:nev]).max())
        x = X[k].double().cpu().numpy()
        r = np.linalg.norm(H @ x - x * ev[k], axis=0)
        assert r.max() <= (1e-8 if precision == trbl.TRBL_PREC_F64 else 1e-4) * normH, (k, r.max() / normH)
