"""Checkpoint and resume of the stepwise solver (trbl_solver_save / _load).

The state between block steps of Alg. 4 -- the basis (after a thick
restart, Eq. (trb-tmat), the kept Ritz vectors and the new block), the
current block, T and the counters -- saved after 10 steps (past a restart)
and loaded into a second solver continues the iteration: 10 more steps
there give the same Ritz values, residuals and counters as 10 more steps of
the uninterrupted solver.  Every kernel sums in a fixed order and the
Rayleigh-Ritz cadence is fixed (check_every = 1), so the two runs agree
bit for bit.  Loading checks sizes and format; a converged solver is
finished, not saved."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    w, sa, sb, inter = synth.workload("s12_4p4n")
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    return tb, trbl.Hamiltonian.from_interaction(tb, inter)


def _solver(th, precision, q=8):
    return trbl.Solver(th, 8, q, 64, 1e-12, precision=precision, check_every=1, seed=5)


@pytest.mark.parametrize("precision", [trbl.TRBL_PREC_F64, trbl.TRBL_PREC_MIXED])
def test_resume_continues_the_iteration(medium, precision):
    tb, th = medium
    a = _solver(th, precision)
    for _ in range(10):
        a.step()
    assert a.stats()["restarts"] >= 1
    state = a.save()
    assert state.nbytes == trbl.trbl_solver_state_bytes(a.handle)
    b = _solver(th, precision)
    b.load(state)
    for sv in (a, b):
        for _ in range(10):
            sv.step()
    ea, ra, Xa, sa = a.finish(raise_on_noconv=False)
    eb, rb, Xb, sb = b.finish(raise_on_noconv=False)
    for k in ("iterations", "restarts", "converged"):
        assert sa[k] == sb[k], k
    assert sa["iterations"] == 20
    assert np.array_equal(ea, eb) and np.array_equal(ra, rb)
    assert torch.equal(Xa, Xb)


def test_load_rejects_foreign_or_damaged_states(medium):
    tb, th = medium
    a = _solver(th, trbl.TRBL_PREC_F64)
    a.step()
    state = a.save()
    for other in (_solver(th, trbl.TRBL_PREC_F64, q=4), _solver(th, trbl.TRBL_PREC_MIXED)):
        with pytest.raises(trbl.TrblError) as e:
            other.load(state)
        assert e.value.code == trbl.TRBL_ERR_ARG
    b = _solver(th, trbl.TRBL_PREC_F64)
    for bad in (state[:-8], state[:64], np.zeros_like(state)):
        with pytest.raises(trbl.TrblError) as e:
            b.load(bad)
        assert e.value.code == trbl.TRBL_ERR_ARG
    with pytest.raises(trbl.TrblError) as e:
        trbl.trbl_solver_save(a.handle, state.ctypes.data, state.nbytes - 1)
    assert e.value.code == trbl.TRBL_ERR_ARG


def test_converged_solver_is_not_saved():
    w, sa, sb, inter = synth.workload("s12_2p2n")
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    sv = trbl.Solver(th, 4, 4, 40, 1e-6, check_every=1)
    for _ in range(200):
        if sv.step() == 4:
            break
    with pytest.raises(trbl.TrblError) as e:
        sv.save()
    assert e.value.code == trbl.TRBL_ERR_ARG


@pytest.mark.parametrize("precision", [trbl.TRBL_PREC_F64, trbl.TRBL_PREC_MIXED])
def test_state_saved_at_max_iter_finishes_like_the_original(medium, precision):
    """A step that stops at max_iter runs Rayleigh-Ritz on the whole T and
    appends nothing; a state saved there and finished in another solver
    gives the Ritz pairs the original solver's finish gives (all nb rows of
    T, not nb - q)."""
    tb, th = medium
    mk = lambda: trbl.Solver(th, 8, 8, 64, 1e-14, precision=precision, check_every=0, seed=5, max_iter=7)
    a = mk()
    for _ in range(7):
        a.step()
    state = a.save()
    b = mk()
    b.load(state)
    ea, ra, Xa, sa = a.finish(raise_on_noconv=False)
    eb, rb, Xb, sb = b.finish(raise_on_noconv=False)
    assert sa["iterations"] == sb["iterations"] == 7
    assert np.array_equal(ea, eb) and np.array_equal(ra, rb)
    assert torch.equal(Xa, Xb)
