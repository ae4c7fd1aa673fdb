"""Host-buffer solver steps (trbl_solver_step_host) with page-locked buffers
from trbl_host_alloc (page-locked, with the host memory node nearest the GPU
reported).  A block that goes out to such a buffer and comes back in each step
leaves the iteration (Alg. 4) bit for bit as the device-only steps run it."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu


def test_host_round_trip_steps_match_device_steps():
    w, sa, sb, inter = synth.workload("s12_4p4n")
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)

    def mk():
        return trbl.Solver(th, 8, 8, 64, 1e-12, precision=trbl.TRBL_PREC_MIXED, check_every=1, seed=9)

    a, b = mk(), mk()
    _, nbytes = b.block()
    bufs = [trbl.HostBuffer(nbytes, 0), trbl.HostBuffer(nbytes, 0)]
    assert bufs[0].numa_node >= -1 and bufs[0].array.nbytes == nbytes
    b.step_host(None, bufs[0])
    a.step()
    for k in range(9):  # past the first thick restart (basis 64, block 8)
        b.step_host(bufs[k % 2], bufs[(k + 1) % 2])
        a.step()
        assert np.isfinite(bufs[(k + 1) % 2].array).all()
    assert a.stats()["restarts"] >= 1
    ea, ra, Xa, _ = a.finish(raise_on_noconv=False)
    eb, rb, Xb, _ = b.finish(raise_on_noconv=False)
    assert np.array_equal(ea, eb) and np.array_equal(ra, rb)
    assert torch.equal(Xa, Xb)
    for buf in bufs:
        buf.free()


def test_host_alloc_and_free():
    hb = trbl.HostBuffer(1 << 20, 0)
    hb.array[:] = 3.0
    assert float(hb.array.sum()) == 3.0 * (1 << 18)
    hb.free()
    hb.free()  # a second free does nothing
    with pytest.raises(trbl.TrblError) as e:
        trbl._lib._check(trbl.lib().trbl_host_free(12345))
    assert e.value.code == trbl.TRBL_ERR_ARG


def test_copy_out_after_convergence_and_timing():
    """Once the solver has converged a host step runs no block step: the
    current block is copied out as it is (twice the same bytes), and the
    copy times accumulate in the statistics."""
    w, sa, sb, inter = synth.workload("s12_2p2n")
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    sv = trbl.Solver(th, 4, 4, 40, 1e-8, precision=trbl.TRBL_PREC_F64, check_every=1, seed=3)
    ptr, nbytes = sv.block()
    bufs = [trbl.HostBuffer(nbytes, 0, dtype=np.float64) for _ in range(2)]
    for _ in range(200):
        if sv.step() >= 4:
            break
    assert sv.step() >= 4  # converged: further steps do nothing
    st0 = sv.stats()
    sv.step_host(None, bufs[0])
    sv.step_host(None, bufs[1])
    st1 = sv.stats()
    assert st1["iterations"] == st0["iterations"]
    assert st1["ms_copy_out"] > st0["ms_copy_out"]
    assert np.array_equal(bufs[0].array, bufs[1].array)
    assert np.isfinite(bufs[0].array).all() and np.abs(bufs[0].array).max() > 0
    for b in bufs:
        b.free()
