"""Host-side pieces of the benchmark.

* The reference arm (the FP64 oracle's one-row-at-a-time product on the
  host cores) prints one JSON line in the shape of the GPU arm's: same
  metric, unit, direction and workload, with the oracle described as the
  CPU baseline and no host-device traffic.
* The work counts behind the metric and the roofline: the structural nnz
  (GNZ) from the library's exported basis equals the oracle's structural
  pattern, and the slab-row count R of the factorised slab model (App. B.2:
  one neutron slab per proton source -> target pair) equals a count built
  from the oracle's own one-body jump lists and explicit two-particle moves.
"""
import itertools
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["value"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0 and e2e["value"] == d["value"]


def _exported(name):
    import synth
    import paper_1902_02064_gb300 as trbl
    w, sa, sb, inter = synth.workload(name)
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    return w, sa, inter, tb.export()


def test_structural_nnz_equals_the_oracle_pattern():
    from oracle import basis as ob
    from oracle import hamiltonian as oh
    w, sa, inter, (bitsA, mA, bitsB, mB, blocks) = _exported("s12_2p2n")
    B = ob.ProductBasis(sa.twom, w.nA, sa.twom, w.nB, w.twoM)
    assert bench.structural_nnz(bitsA, mA, bitsB, mB, blocks) == oh.structural_pattern(B, inter).nnz


@pytest.mark.parametrize("name", ["s12_2p2n", "s12_4p4n"])
def test_slab_rows_equal_a_count_from_the_oracle_moves(name):
    from oracle import basis as ob
    from oracle import hamiltonian as oh
    w, sa, inter, (bitsA, mA, bitsB, mB, blocks) = _exported(name)
    twom = sa.twom
    dets = ob.species_determinants(twom, w.nA)
    detsB = ob.species_determinants(twom, w.nB)
    nB = {}
    for m, _ in detsB:
        nB[m] = nB.get(m, 0) + 1
    NB = [nB.get(w.twoM - m, 0) for m, _ in dets]
    src = {t: set() for t in range(len(dets))}
    for t, s_, a, c, sign in oh.one_body_jumps(twom, w.nA):  # one particle moved, any 2M, and t itself
        src[t].add(s_)
    where = {b: i for i, (_, b) in enumerate(dets)}
    n = len(twom)
    for i, (m, S) in enumerate(dets):  # two particles moved inside the M block
        occ = [x for x in range(n) if S >> x & 1]
        empty = [x for x in range(n) if not S >> x & 1]
        for p, q in itertools.combinations(occ, 2):
            for a, b in itertools.combinations(empty, 2):
                if twom[p] + twom[q] == twom[a] + twom[b]:
                    src[where[S ^ (1 << p) ^ (1 << q) ^ (1 << a) ^ (1 << b)]].add(i)
    R = sum(sum(NB[s_] for s_ in src[t]) for t in range(len(dets)) if NB[t] > 0)
    assert bench.slab_rows(bitsA, mA, mB, w.twoM) == R


def test_traffic_lookup_is_tied_to_kernel_source_and_shape(tmp_path):
    """The roofline's DRAM traffic is taken from a committed ncu summary only
    when the summary names the kernel the bench ran, with its launch shape,
    and the kernel's source file still hashes to the value stored with the
    counters; otherwise it is reported as unknown (None).  The split
    product's figure needs both of its source files unchanged."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1902_02064_gb300", "csrc")
    sha = lambda f: hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest()
    name = bench.product_kernel_name((0, 16, 8), 32)
    assert name == "apply_grouped_kernel<float, 8, 1>"
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps({"kernel": name, "rows_per_item": 16, "source_sha256": sha("apply_grouped.cu"),
                             "dram_bytes_per_launch_full_size": 1.5e11}))
    assert bench.ncu_traffic(name, 16, str(p)) == (1.5e11, name)
    assert bench.ncu_traffic(name, 64, str(p))[0] is None  # another launch shape
    assert bench.ncu_traffic(bench.product_kernel_name((1, 16, 8), 32), 16, str(p))[0] is None  # another kernel
    p.write_text(json.dumps({"kernel": name, "rows_per_item": 16, "source_sha256": "0" * 64,
                             "dram_bytes_per_launch_full_size": 1.5e11}))
    assert bench.ncu_traffic(name, 16, str(p))[0] is None  # source changed since the counters
    split = bench.product_kernel_name((3, 64, 2), 32)
    assert split == "apply_grouped_kernel<float, 8, 1> + apply_pn_kernel<8, 2, 384, 2>"
    p.write_text(json.dumps({"kernel": split, "rows_per_item": 64,
                             "source_sha256": {"apply_grouped.cu": sha("apply_grouped.cu"),
                                               "apply_pn.cu": sha("apply_pn.cu")},
                             "dram_bytes_per_launch_full_size": 1.0e11}))
    assert bench.ncu_traffic(split, 64, str(p)) == (1.0e11, split)
    p.write_text(json.dumps({"kernel": split, "rows_per_item": 64, "source_sha256": sha("apply_grouped.cu"),
                             "dram_bytes_per_launch_full_size": 1.0e11}))
    assert bench.ncu_traffic(split, 64, str(p))[0] is None
