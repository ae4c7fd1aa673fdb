"""Parity of the CUDA block product W = H V (App. B) with the oracle.

Small spaces: every element of W against the oracle's explicit CSR H times
the same V.  Full 20-m-state spaces: sampled rows (block edges, first/last
row, random rows) against the oracle's one-row-at-a-time product.

Tolerance (elementwise, derived from recursive-summation error bounds):
|W - H V|_ij <= rtol * (|H| |V|)_ij with rtol = 1e-12 in FP64 and 1e-5 in
FP32 (coefficients rounded to FP32 once; V is rounded to FP32 before the
oracle sees it, so input rounding is not counted).
"""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu

RTOL = {torch.float64: 1e-12, torch.float32: 1e-5}


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


def _check(W, H, V, dtype):
    Vd = V.astype(np.float64)
    ref = H @ Vd
    bound = abs(H) @ np.abs(Vd)
    err = np.abs(W.astype(np.float64) - ref)
    assert np.all(err <= RTOL[dtype] * bound + 1e-300), float((err / (bound + 1e-300)).max())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("q", [1, 3, 4, 8, 16, 32, 64])
def test_apply_small_all_elements(small, dtype, q):
    w, B, H, tb, th = small
    V = torch.from_numpy(synth.random_block(B.dim, q, 10 + q)).to(dtype)
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.numpy(), dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("q", [8, 16])
def test_apply_medium_all_elements(medium, dtype, q):
    w, B, H, tb, th = medium
    V = torch.from_numpy(synth.random_block(B.dim, q, 20 + q)).to(dtype)
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.numpy(), dtype)


def test_apply_strided_leading_dimension(small):
    w, B, H, tb, th = small
    q, ld = 4, 11
    big = torch.from_numpy(synth.random_block(B.dim, ld, 3)).cuda()
    V = big[:, 2:2 + q]
    Wbig = torch.full((B.dim, 9), 7.0, dtype=torch.float64, device="cuda")
    W = Wbig[:, 1:1 + q]
    th.apply(V, W)
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.cpu().numpy(), torch.float64)
    assert torch.all(Wbig[:, 0] == 7.0) and torch.all(Wbig[:, 1 + q:] == 7.0)


def test_apply_columns_independent(medium):
    """Column j of H [V] equals H applied to column j alone (q = 1)."""
    w, B, H, tb, th = medium
    V = torch.from_numpy(synth.random_block(B.dim, 32, 5)).cuda()
    W = th.apply(V)
    for j in (0, 13, 31):
        Wj = th.apply(V[:, j:j + 1].contiguous())
        assert torch.allclose(W[:, j:j + 1], Wj, rtol=0, atol=1e-12 * W.abs().max().item())


@pytest.mark.parametrize("kA,kB,twoM", [(0, 2, 0), (1, 1, 2), (3, 1, -2), (2, 3, 3)])
def test_apply_edge_particle_numbers(kA, kB, twoM):
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 31)
    B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    H = oh.assemble(B, inter)
    tb = trbl.Basis(sp, kA, sp, kB, twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    V = torch.from_numpy(synth.random_block(B.dim, 5, 1))
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.numpy(), torch.float64)


def test_apply_rejects_bad_arguments(small):
    w, B, H, tb, th = small
    V = torch.zeros((B.dim, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(trbl.TrblError):
        trbl.trbl_apply_block(th.handle, V.data_ptr(), 4, V.data_ptr(), 4, 4, trbl.TRBL_F64, 0)
    with pytest.raises(trbl.TrblError):
        trbl.trbl_apply_block(th.handle, V.data_ptr(), 2, V.data_ptr(), 4, 4, trbl.TRBL_F64, 0)
    host = np.zeros((B.dim, 4))
    W = torch.zeros_like(V)
    with pytest.raises(trbl.TrblError):
        trbl.trbl_apply_block(th.handle, host.ctypes.data, 4, W.data_ptr(), 4, 4, trbl.TRBL_F64, 0)


def _sample_rows(L, n_rand, seed):
    rows = {0, L.dim - 1}
    for (_, _, off, na, nb, _, _) in L.blocks:
        rows.add(off)
        rows.add(off + na * nb - 1)
    rng = np.random.default_rng(seed)
    rows.update(rng.integers(0, L.dim, n_rand).tolist())
    return sorted(rows)


@pytest.mark.parametrize("name,q,dtype,kernel", [("s20_4p4n", 16, torch.float64, trbl.TRBL_APPLY_GROUPED),
                                                 ("s20_4p4n", 16, torch.float32, trbl.TRBL_APPLY_FAST),
                                                 ("s20_4p4n", 32, torch.float32, trbl.TRBL_APPLY_GROUPED),
                                                 ("s20_5p5n", 32, torch.float32, trbl.TRBL_APPLY_FAST)])
def test_apply_full_size_sampled_rows(name, q, dtype, kernel):
    """Sampled rows at full size, in the launch shape the bench times for
    the 18.6M-dim workload (fast kernel, 16 rows per work item)."""
    w, sa, sb, inter = synth.workload(name)
    L = oh.LazyIndex(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    T = oh.TermTables(inter)
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    assert tb.dim == L.dim
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    trbl.apply_set_shape(th, kernel, 16, 8)
    g = torch.Generator(device="cuda")
    g.manual_seed(w.seed)
    V = torch.rand((tb.dim, q), generator=g, device="cuda", dtype=dtype) * 2 - 1
    W = th.apply(V)
    torch.cuda.synchronize()
    rows = _sample_rows(L, 24, w.seed)
    Wr = W[torch.tensor(rows, device="cuda")].double().cpu().numpy()
    for k, r in enumerate(rows):
        SA, SB = L.state(r)
        terms = oh.column_terms(SA, SB, T)
        idx = torch.tensor([L.index(A2, B2) for _, A2, B2 in terms], device="cuda")
        Vs = V[idx].double().cpu().numpy()
        coef = np.array([v for v, _, _ in terms])
        ref = coef @ Vs
        bound = np.abs(coef) @ np.abs(Vs)
        assert np.all(np.abs(Wr[k] - ref) <= RTOL[dtype] * bound), (r, np.abs(Wr[k] - ref).max())
    # symmetry of H at full size: <x, H y> = <H x, y>
    x = V[:, :1].double().contiguous()
    y = V[:, 1:2].double().contiguous()
    Hx, Hy = th.apply(x), th.apply(y)
    a, b = torch.dot(x[:, 0], Hy[:, 0]).item(), torch.dot(Hx[:, 0], y[:, 0]).item()
    assert abs(a - b) <= 1e-10 * (abs(a) + abs(b))


@pytest.mark.parametrize("kA,kB,twoM,q,dtype", [(0, 2, 0, 4, torch.float32), (2, 0, 0, 2, torch.float64),
                                                (1, 1, 2, 8, torch.float32), (3, 2, 1, 16, torch.float64)])
def test_apply_edge_cases_grouped_path(kA, kB, twoM, q, dtype):
    """Row sizes that are multiples of 16 bytes take the grouped kernel (FP32
    rows of 32, 64 or 128 bytes the fast kernel)."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 33)
    B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    H = oh.assemble(B, inter)
    tb = trbl.Basis(sp, kA, sp, kB, twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    V = torch.from_numpy(synth.random_block(B.dim, q, 2)).to(dtype)
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().numpy(), H, V.numpy(), dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_grouped_and_row_kernels_agree(medium, dtype):
    """Aligned rows (grouped kernel) against a leading dimension that is not a
    multiple of 16 bytes (row kernel): same products to rounding."""
    w, B, H, tb, th = medium
    q = 16
    Vb = torch.from_numpy(synth.random_block(B.dim, q + 1, 8)).to(dtype).cuda()
    Va = Vb[:, :q].contiguous()
    Wa = th.apply(Va)
    Wr = torch.empty((B.dim, q + 1), dtype=dtype, device="cuda")
    trbl.trbl_apply_block(th.handle, Vb.data_ptr(), q + 1, Wr.data_ptr(), q + 1, q,
                          trbl.TRBL_F64 if dtype == torch.float64 else trbl.TRBL_F32,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    bound = torch.from_numpy(abs(H) @ np.abs(Va.double().cpu().numpy())).cuda()
    diff = (Wa.double() - Wr[:, :q].double()).abs()
    assert torch.all(diff <= 2 * RTOL[dtype] * bound)


def test_launch_shape_does_not_change_results(medium):
    """trbl_apply_set_rows only regroups rows into thread blocks: every row's
    summation order is the same, so W is bit-identical for any shape."""
    w, B, H, tb, th = medium
    V = torch.from_numpy(synth.random_block(B.dim, 32, 5)).float().cuda()
    outs = []
    for rows in (1, 7, 16, 128, 4096):
        trbl.apply_set_rows(th, rows)
        outs.append(th.apply(V).cpu())
    trbl.apply_set_rows(th, 128)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    _check(outs[0].double().numpy(), H, V.cpu().double().numpy(), torch.float32)
    with pytest.raises(trbl.TrblError):
        trbl.apply_set_rows(th, 0)


SHAPES = [(trbl.TRBL_APPLY_GROUPED, 16, 8), (trbl.TRBL_APPLY_FAST, 16, 8), (trbl.TRBL_APPLY_FAST, 64, 6),
          (trbl.TRBL_APPLY_FAST, 1, 8), (trbl.TRBL_APPLY_FAST, 4096, 6)]
X2 = (trbl.TRBL_APPLY_GROUPED_X2, 32, 8)


@pytest.mark.parametrize("q", [8, 16, 32])
def test_fast_kernel_every_element_matches_oracle(small, medium, q):
    """The FP32 fast kernel (packed tables, 32-bit offsets, paired FMAs) and
    the grouped kernel, each at several launch shapes, against the oracle's
    CSR H V on every element; with plain sums both kernels sum each row in
    the same order, so their results are also bit-identical.  The same with
    compensated sums (fast kernel only), each shape against the oracle."""
    for w, B, H, tb, th in (small, medium):
        V = torch.from_numpy(synth.random_block(B.dim, q, 40 + q)).float()
        Vc = V.cuda()
        outs = []
        for kern, rows, bps in SHAPES:
            trbl.apply_set_shape(th, kern, rows, bps)
            assert trbl.apply_get_shape(th) == (kern, rows, bps)
            W = th.apply(Vc)
            torch.cuda.synchronize()
            _check(W.cpu().double().numpy(), H, V.double().numpy(), torch.float32)
            outs.append(W.cpu())
        trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 8)
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        # two chunks per lane: same products, summed in another lane layout
        trbl.apply_set_shape(th, *X2)
        W = th.apply(Vc)
        torch.cuda.synchronize()
        _check(W.cpu().double().numpy(), H, V.double().numpy(), torch.float32)
        trbl.apply_set_compensated(th, True)
        for kern, rows, bps in SHAPES[1:]:
            trbl.apply_set_shape(th, kern, rows, bps)
            W = th.apply(Vc)
            torch.cuda.synchronize()
            _check(W.cpu().double().numpy(), H, V.double().numpy(), torch.float32)
        trbl.apply_set_compensated(th, False)
        trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 8)


@pytest.mark.parametrize("kA,kB,twoM,q", [(0, 2, 0, 8), (2, 0, 0, 16), (1, 1, 2, 32), (3, 2, 1, 8), (4, 1, -3, 16)])
def test_fast_kernel_edge_particle_numbers(kA, kB, twoM, q):
    """Empty species, one particle, odd 2M: the fast kernel against the oracle."""
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 34)
    B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    H = oh.assemble(B, inter)
    tb = trbl.Basis(sp, kA, sp, kB, twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 8)
    V = torch.from_numpy(synth.random_block(B.dim, q, 3)).float()
    W = th.apply(V.cuda())
    torch.cuda.synchronize()
    _check(W.cpu().double().numpy(), H, V.double().numpy(), torch.float32)


def test_fast_kernel_strided_rows_and_fallback(medium):
    """A leading dimension above q (still 16-byte rows) takes the fast kernel;
    q = 4 (16-byte rows) falls back to the grouped kernel; both against the
    oracle."""
    w, B, H, tb, th = medium
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 8)
    big = torch.from_numpy(synth.random_block(B.dim, 24, 6)).float().cuda()
    V = big[:, 4:20]
    Wbig = torch.full((B.dim, 20), 3.0, dtype=torch.float32, device="cuda")
    W = Wbig[:, 4:20]
    th.apply(V, W)
    torch.cuda.synchronize()
    _check(W.cpu().double().numpy(), H, V.cpu().double().numpy(), torch.float32)
    assert torch.all(Wbig[:, :4] == 3.0)
    V4 = torch.from_numpy(synth.random_block(B.dim, 4, 7)).float()
    W4 = th.apply(V4.cuda())
    torch.cuda.synchronize()
    _check(W4.cpu().double().numpy(), H, V4.double().numpy(), torch.float32)


def test_autotune_candidates_and_choice(medium):
    """The autotuner times every shape that applies (NaN for the others),
    keeps the fastest, and leaves W unchanged."""
    w, B, H, tb, th = medium
    V = torch.from_numpy(synth.random_block(B.dim, 32, 9)).float().cuda()
    ref = th.apply(V).cpu()
    ms, rows = trbl.apply_autotune(th, 32, trbl.TRBL_F32)
    assert len(ms) == trbl.TRBL_TUNE_CANDIDATES and all(np.isfinite(ms))
    kern, r, bps = trbl.apply_get_shape(th)
    assert r == rows
    W = th.apply(V).cpu()
    if kern in (trbl.TRBL_APPLY_SPLIT, trbl.TRBL_APPLY_SPLIT_X4, trbl.TRBL_APPLY_SPLIT_TMA):
        # the split product's cross-term sums are not in a fixed order
        _check(W.double().numpy(), H, V.cpu().double().numpy(), torch.float32)
    else:
        assert kern in (trbl.TRBL_APPLY_GROUPED, trbl.TRBL_APPLY_FAST, trbl.TRBL_APPLY_GROUPED_X2)
        assert torch.equal(W, ref)
    ms64, _ = trbl.apply_autotune(th, 16, trbl.TRBL_F64)
    assert all(np.isfinite(ms64[:4])) and not any(np.isfinite(ms64[4:10])) and all(np.isfinite(ms64[10:13]))
    assert len(ms64) == 15 and not any(np.isfinite(ms64[13:]))  # split products are FP32 only
    with pytest.raises(trbl.TrblError):
        trbl.apply_set_shape(th, 7, 16, 8)
    with pytest.raises(trbl.TrblError):
        trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 5)
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 8)


def test_compensated_sums_match_oracle_and_cut_rounding(medium):
    """Compensated row sums (TwoSum of short partial sums) against the
    oracle's FP64 H V: within the FP32 bound, and with a smaller maximum
    error than the plain FP32 sums on the same inputs."""
    w, B, H, tb, th = medium
    V = torch.from_numpy(synth.random_block(B.dim, 32, 12)).float()
    Vd = V.double().numpy()
    ref = H @ Vd
    bound = abs(H) @ np.abs(Vd)
    errs = {}
    for comp in (False, True):
        trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 8)
        trbl.apply_set_compensated(th, comp)
        W = th.apply(V.cuda()).cpu().double().numpy()
        _check(W, H, Vd, torch.float32)
        errs[comp] = float((np.abs(W - ref) / (bound + 1e-300)).max())
        # the launch shape does not change the compensated result either
        trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 64, 6)
        assert np.array_equal(th.apply(V.cuda()).cpu().double().numpy(), W)
    trbl.apply_set_compensated(th, False)
    trbl.apply_set_shape(th, trbl.TRBL_APPLY_FAST, 16, 8)
    print("max |W - HV| / (|H||V|): plain %.2e compensated %.2e" % (errs[False], errs[True]))
    assert errs[True] < errs[False]


@pytest.mark.parametrize("dtype,q", [(torch.float32, 32), (torch.float64, 16)])
def test_row_restricted_products_tile_the_full_product(medium, dtype, q):
    """The shards of a 3-way plan (trbl_shard_plan), each computed alone with
    trbl_hamiltonian_set_rows, reproduce the full product's rows bit for bit
    and leave every other row of W untouched."""
    w, B, H, tb, th = medium
    bounds, work = trbl.shard_plan(tb, 3)
    V = torch.from_numpy(synth.random_block(B.dim, q, 77)).to(dtype).cuda()
    full = th.apply(V)
    for r in range(3):
        th.set_rows(bounds[r], bounds[r + 1])
        W = torch.full_like(full, 7.0)
        th.apply(V, W)
        torch.cuda.synchronize()
        assert torch.equal(W[bounds[r]:bounds[r + 1]], full[bounds[r]:bounds[r + 1]])
        assert torch.all(W[:bounds[r]] == 7.0) and torch.all(W[bounds[r + 1]:] == 7.0)
    th.set_rows(0, tb.dim)
    assert torch.equal(th.apply(V), full)
    with pytest.raises(trbl.TrblError):
        th.set_rows(1, tb.dim)
    th.set_rows(bounds[1], bounds[2])
    with pytest.raises(trbl.TrblError):
        trbl.solve(th, 4, 4, 40, 1e-8)
    th.set_rows(0, tb.dim)
