"""Row sharding of the block product (the distributed matrix-vector product
of App. C recast for GPUs that each hold the tables), checked on the CPU
with two gloo ranks.

Each rank owns the rows of W, and of the vector blocks, in its slab-aligned
range from trbl_shard_plan.  Before the product it receives V's rows in the
ranges trbl_shard_sources lists (an all-gather of every rank's slice, of
which it keeps only those ranges), forms its rows of W = H V from them, and
for the projection C = B^T W contributes its rows' partial sum to an
all-reduce.  The oracle's explicit H (test infrastructure) plays the GPU
product's part: the check is on the partition and the exchange plan.  The
gathered W must equal the single-process H V bit for bit (each row is
summed the same way), and C must equal B^T W to rounding."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(name):
    sys.path.insert(0, ROOT)
    import paper_1902_02064_gb300 as trbl
    import synth
    from oracle import basis as ob
    from oracle import hamiltonian as oh
    w, sa, sb, inter = synth.workload(name)
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter).tocsr()
    return trbl, synth, tb, H


def _rank(rank, world, port, name, out):
    import torch.distributed as dist
    trbl, synth, tb, H = _setup(name)
    D = tb.dim
    q, m = 8, 24
    V = synth.random_block(D, q, 71)      # every rank can generate it; a rank only uses its own slice
    Bm = synth.random_block(D, m, 72)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        bounds, work = trbl.shard_plan(tb, world)
        r0, r1 = bounds[rank], bounds[rank + 1]
        # exchange: all-gather the ranks' slices of V (padded to the largest)
        n_max = max(bounds[i + 1] - bounds[i] for i in range(world))
        mine = torch.zeros((n_max, q), dtype=torch.float64)
        mine[:r1 - r0] = torch.from_numpy(V[r0:r1])
        parts = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        # keep only the rows the plan lists; everything else stays zero, so a
        # missing range would show in W
        Vloc = np.zeros((D, q))
        src = trbl.shard_sources(tb, r0, r1)
        for b, e in src:
            for i in range(world):
                lo, hi = max(b, bounds[i]), min(e, bounds[i + 1])
                if lo < hi:
                    Vloc[lo:hi] = parts[i][lo - bounds[i]:hi - bounds[i]].numpy()
        Wloc = H[r0:r1] @ Vloc
        # gather W rows for the check
        wpad = torch.zeros((n_max, q), dtype=torch.float64)
        wpad[:r1 - r0] = torch.from_numpy(Wloc)
        wparts = [torch.zeros_like(wpad) for _ in range(world)]
        dist.all_gather(wparts, wpad)
        Wfull = np.concatenate([wparts[i][:bounds[i + 1] - bounds[i]].numpy() for i in range(world)])
        # projection: per-rank partial sums, all-reduced
        C = torch.from_numpy(Bm[r0:r1].T @ Wfull[r0:r1])
        dist.all_reduce(C)
        out.put((rank, bounds, work, src, Wfull, C.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["s12_2p2n"])
def test_two_rank_sharded_product_and_projection(name):
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, name, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    trbl, synth, tb, H = _setup(name)
    D = tb.dim
    V = synth.random_block(D, 8, 71)
    Bm = synth.random_block(D, 24, 72)
    ref = H @ V
    bounds, work = res[0][1], res[0][2]
    assert bounds[0] == 0 and bounds[-1] == D and bounds[0] < bounds[1] < bounds[2]
    assert max(work) <= 1.15 * (sum(work) / len(work))  # balanced by generated elements
    for rank, b, wk, src, Wfull, C in res:
        assert b == bounds
        assert np.array_equal(Wfull, ref)
        Cref = Bm.T @ ref
        assert np.all(np.abs(C - Cref) <= 1e-12 * (np.abs(Bm).T @ np.abs(ref)) + 1e-300)


def test_source_ranges_cover_every_nonzero_and_reject_bad_rows():
    """For a 3-way plan of the 28,503-dim space, every column with a nonzero
    in a shard's rows of H lies in the shard's source ranges; the ranges
    are sorted and disjoint; rows that are not slab boundaries are rejected."""
    trbl, synth, tb, H = _setup("s12_4p4n")
    bounds, work = trbl.shard_plan(tb, 3)
    for r in range(3):
        src = trbl.shard_sources(tb, bounds[r], bounds[r + 1])
        mask = np.zeros(tb.dim, dtype=bool)
        for b, e in src:
            assert 0 <= b < e <= tb.dim
            mask[b:e] = True
        assert all(src[i][1] < src[i + 1][0] for i in range(len(src) - 1))
        cols = np.unique(H[bounds[r]:bounds[r + 1]].indices)
        assert mask[cols].all()
    with pytest.raises(trbl.TrblError):
        trbl.shard_sources(tb, 1, tb.dim)
    one, _ = trbl.shard_plan(tb, 1)
    assert one == [0, tb.dim]
