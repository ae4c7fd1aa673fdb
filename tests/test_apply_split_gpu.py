"""Parity of the split block product (TRBL_APPLY_SPLIT, TRBL_APPLY_SPLIT_X4):
like-particle terms (App. B.1) by the grouped kernel, then the factorised
proton-neutron term (App. B.2, Eq. (pntwobodybit)) by the source-stationary
kernel, which adds each gathered source row into all outgoing neutron jumps
of its row at once.

Every element of W is compared with the oracle's explicit CSR H times the
same V (spaces of 640 and 28,503 determinants, several slabs per transfer
class, slabs of uneven size, more outgoing jumps per source row than one
register batch holds), and sampled rows at full size with the oracle's
one-row product.  Bar as for the other kernels: |W - H V|_ij <= 1e-5
(|H| |V|)_ij in FP32.  The cross term's sums are formed with shared-memory
atomic adds (order not fixed), so results are compared with the oracle, and
between kernels to the same bound, never bit for bit.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu

RTOL = 1e-5
# (kernel, blocks per SM): every variant of the cross-term kernel
VARIANTS = [(trbl.TRBL_APPLY_SPLIT, 2), (trbl.TRBL_APPLY_SPLIT, 1), (trbl.TRBL_APPLY_SPLIT_X4, 2),
            (trbl.TRBL_APPLY_SPLIT_TMA, 1)]


def _setup(name):
    w, sa, sb, inter = synth.workload(name)
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    return w, B, H, tb, th


@pytest.fixture(scope="module")
def small():
    return _setup("s12_2p2n")


@pytest.fixture(scope="module")
def medium():
    return _setup("s12_4p4n")


def _check(W, H, V):
    Vd = V.astype(np.float64)
    ref = H @ Vd
    bound = abs(H) @ np.abs(Vd)
    err = np.abs(W.astype(np.float64) - ref)
    assert np.all(err <= RTOL * bound + 1e-300), float((err / (bound + 1e-300)).max())


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("q", [16, 32, 64])
def test_split_small_all_elements(small, variant, q):
    w, B, H, tb, th = small
    trbl.apply_set_shape(th, variant[0], 16, variant[1])
    V = torch.from_numpy(synth.random_block(B.dim, q, 40 + q)).float()
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.numpy())
    assert trbl.apply_get_shape(th) == (variant[0], 16, variant[1])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("q,rows", [(16, 16), (32, 16), (32, 64)])
def test_split_medium_all_elements(medium, variant, q, rows):
    w, B, H, tb, th = medium
    trbl.apply_set_shape(th, variant[0], rows, variant[1])
    V = torch.from_numpy(synth.random_block(B.dim, q, 50 + q)).float()
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.numpy())


def test_split_strided_rows_leave_other_columns(medium):
    """Leading dimensions above q (multiples of 4 floats): the columns
    outside the block are neither read as rows nor written."""
    w, B, H, tb, th = medium
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_SPLIT, 16, 2)
    q, ldv, ldw = 32, 40, 44
    big = torch.from_numpy(synth.random_block(B.dim, ldv, 61)).float().cuda()
    V = big[:, 4:4 + q]
    Wbig = torch.full((B.dim, ldw), 3.0, dtype=torch.float32, device="cuda")
    W = Wbig[:, 8:8 + q]
    th.apply(V, W)
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.cpu().numpy())
    assert torch.all(Wbig[:, :8] == 3.0) and torch.all(Wbig[:, 8 + q:] == 3.0)


@pytest.mark.parametrize("kA,kB,twoM", [(0, 2, 0), (2, 0, 0), (1, 1, 2), (3, 1, -2), (2, 3, 3), (6, 2, 0)])
def test_split_edge_particle_numbers(kA, kB, twoM):
    """An empty species (no cross term at all), one particle per species,
    odd 2M, and six protons with two neutrons (slabs of very uneven size)."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 35)
    B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    H = oh.assemble(B, inter)
    tb = trbl.Basis(sp, kA, sp, kB, twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_SPLIT, 16, 2)
    V = torch.from_numpy(synth.random_block(B.dim, 16, 4)).float()
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.numpy())


def test_split_falls_back_for_other_blocks(medium):
    """q = 8 and FP64 blocks are not split products: they run on the grouped
    kernel, with its results."""
    w, B, H, tb, th = medium
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_SPLIT, 16, 2)
    for q, dt in ((8, torch.float32), (16, torch.float64)):
        V = torch.from_numpy(synth.random_block(B.dim, q, 70 + q)).to(dt)
        W = th.apply(V.cuda())
        torch.cuda.synchronize()
        _check(W.cpu().double().numpy(), H, V.double().numpy())
    with pytest.raises(trbl.TrblError):
        trbl.apply_set_shape(th, trbl.TRBL_APPLY_SPLIT, 16, 8)
    with pytest.raises(trbl.TrblError):
        trbl.apply_set_shape(th, trbl.TRBL_APPLY_SPLIT_X4, 16, 1)


def test_split_row_restricted_products(medium):
    """The shards of a 3-way plan, each computed alone with the split product,
    give the full product's rows (to the FP32 bound) and leave every other
    row of W untouched."""
    w, B, H, tb, th = medium
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_SPLIT, 16, 2)
    bounds, work = trbl.shard_plan(tb, 3)
    V = torch.from_numpy(synth.random_block(B.dim, 32, 78)).float()
    Vc = V.cuda()
    for r in range(3):
        th.set_rows(bounds[r], bounds[r + 1])
        W = torch.full((B.dim, 32), 7.0, dtype=torch.float32, device="cuda")
        th.apply(Vc, W)
        torch.cuda.synchronize()
        Wh = W.cpu().numpy()
        lo, hi = bounds[r], bounds[r + 1]
        Hr = H[lo:hi]
        Vd = V.double().numpy()
        err = np.abs(Wh[lo:hi].astype(np.float64) - Hr @ Vd)
        assert np.all(err <= RTOL * (abs(Hr) @ np.abs(Vd)) + 1e-300)
        assert np.all(Wh[:lo] == 7.0) and np.all(Wh[hi:] == 7.0)
    th.set_rows(0, B.dim)


def _sample_rows(L, n_rand, seed):
    rows = {0, L.dim - 1}
    for (_, _, off, na, nb, _, _) in L.blocks:
        rows.add(off)
        rows.add(off + na * nb - 1)
    rng = np.random.default_rng(seed)
    rows.update(rng.integers(0, L.dim, n_rand).tolist())
    return sorted(rows)


@pytest.mark.parametrize("name,q,variant", [("s20_4p4n", 16, (trbl.TRBL_APPLY_SPLIT, 2)),
                                            ("s20_5p5n", 32, (trbl.TRBL_APPLY_SPLIT, 2)),
                                            ("s20_5p5n", 32, (trbl.TRBL_APPLY_SPLIT_X4, 2)),
                                            ("s20_4p4n", 32, (trbl.TRBL_APPLY_SPLIT_TMA, 1)),
                                            ("s20_5p5n", 32, (trbl.TRBL_APPLY_SPLIT_TMA, 1))])
def test_split_full_size_sampled_rows(name, q, variant):
    """Sampled rows of the 2M- and 18.6M-dim products (slabs of up to 1,651
    rows, 20 proton jumps per transfer class) against the oracle's one-row
    product, in the launch shapes the bench tunes over."""
    w, sa, sb, inter = synth.workload(name)
    L = oh.LazyIndex(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    T = oh.TermTables(inter)
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    trbl.apply_set_shape(th, variant[0], 16, variant[1])
    g = torch.Generator(device="cuda")
    g.manual_seed(w.seed + 7)
    V = torch.rand((tb.dim, q), generator=g, device="cuda", dtype=torch.float32) * 2 - 1
    W = th.apply(V)
    torch.cuda.synchronize()
    rows = _sample_rows(L, 24, w.seed + 7)
    Wr = W[torch.tensor(rows, device="cuda")].double().cpu().numpy()
    for k, r in enumerate(rows):
        SA, SB = L.state(r)
        terms = oh.column_terms(SA, SB, T)
        idx = torch.tensor([L.index(A2, B2) for _, A2, B2 in terms], device="cuda")
        Vs = V[idx].double().cpu().numpy()
        coef = np.array([v for v, _, _ in terms])
        ref = coef @ Vs
        bound = np.abs(coef) @ np.abs(Vs)
        assert np.all(np.abs(Wr[k] - ref) <= RTOL * bound), (r, np.abs(Wr[k] - ref).max())
    # every row against the grouped kernel's product: both sit within
    # 1e-5 |H| |V| of H V, and |H| |V| stays within a few times max |H V| for
    # these uniform random blocks, so 1e-4 max |W| bounds their difference
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_GROUPED, 16, 8)
    W2 = th.apply(V)
    torch.cuda.synchronize()
    assert (W - W2).abs().max().item() <= 1e-4 * W2.abs().max().item()


def test_split_mixed_solve_matches_oracle_eigenvalues():
    """The mixed-precision solver (Alg. 4) running on the split product
    reaches the oracle's stored eigenvalues of the 28,503-dim space within
    1e-6 ||H|| (block size 16, so the split product is the one that runs)."""
    w, sa, sb, inter = synth.workload("s12_4p4n")
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "eigs_s12_4p4n.json")))
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_SPLIT, 16, 2)
    nev = 40
    evals, resid, X, st = trbl.solve(th, nev, 16, 256, 1e-6, precision=trbl.TRBL_PREC_MIXED, want_vectors=False)
    err = np.abs(evals - np.array(gold["evals"][:nev])).max()
    assert err <= 1e-6 * gold["normH"], err
