"""C-ABI checks that need no GPU: the library loads and exports every entry
point of include/trbl.h, and its host-side basis builder reproduces the
oracle's enumeration, product blocks and one-body jump lists bit-exactly
(App. A Table I / Eq. (part); App. B.2 one-body jumps)."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh

trbl = pytest.importorskip("paper_1902_02064_gb300")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "trbl.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(trbl_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = trbl.lib()
    names = declared_symbols()
    assert "trbl_apply_block" in names and "trbl_solve" in names
    for n in names:
        assert hasattr(L, n), n


def test_python_constants_match_the_header():
    txt = open(HEADER).read()
    m = re.search(r"#define TRBL_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", txt)
    assert m, "TRBL_NOALLOC_SCRATCH_BYTES not found in the header"
    assert trbl.TRBL_NOALLOC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))


@pytest.mark.parametrize("shells,kA,kB,twoM", [
    (synth.SPACE12_SHELLS, 2, 2, 0), (synth.SPACE12_SHELLS, 4, 4, 0), (synth.SPACE12_SHELLS, 3, 2, 1),
    (synth.SPACE12_SHELLS, 0, 2, 0), (synth.SPACE12_SHELLS, 1, 1, 4), (synth.TABLE1_SHELLS, 3, 0, 1),
])
def test_basis_bit_exact(shells, kA, kB, twoM):
    sp = synth.make_space(shells)
    B = trbl.Basis(sp, kA, sp, kB, twoM)
    bitsA, mA, bitsB, mB, blocks = B.export()
    oB = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    assert B.dim == oB.dim
    assert [int(x) for x in bitsA] == [b for _, b in oB.detsA]
    assert [int(x) for x in mA] == [m for m, _ in oB.detsA]
    assert [int(x) for x in bitsB] == [b for _, b in oB.detsB]
    assert [tuple(int(v) for v in r) for r in blocks] == [tuple(r) for r in oB.blocks]


def test_basis_blocks_pf_spaces():
    sp = synth.make_space(synth.SPACE20_SHELLS)
    for k in (4, 5):
        B = trbl.Basis(sp, k, sp, k, 0)
        L = oh.LazyIndex(sp.twom, k, sp.twom, k, 0)
        assert B.dim == L.dim
        blocks = B.export()[4]
        assert [tuple(int(v) for v in r) for r in blocks] == [tuple(r) for r in L.blocks]
    assert trbl.Basis(sp, 4, sp, 4, 0).dim == 1963461
    assert trbl.Basis(sp, 5, sp, 5, 0).dim == 18600516


@pytest.mark.parametrize("shells,k", [(synth.SPACE12_SHELLS, 2), (synth.SPACE12_SHELLS, 4),
                                      (synth.TABLE1_SHELLS, 3), (synth.SPACE12_SHELLS, 1)])
def test_jump_lists_bit_exact(shells, k):
    sp = synth.make_space(shells)
    # species A carries k particles; species B one particle (any 2M with a basis)
    twoM = ob.species_determinants(sp.twom, k)[0][0] + sp.twom[0]
    B = trbl.Basis(sp, k, sp, 1, twoM)
    tgt, src, a, c, sign = B.export_jumps(0)
    got = set(zip(tgt.tolist(), src.tolist(), a.tolist(), c.tolist(), sign.tolist()))
    want = oh.one_body_jumps(sp.twom, k)
    assert len(got) == len(tgt)
    assert got == want
    ndet = len(ob.species_determinants(sp.twom, k))
    assert len(tgt) == ndet * (k * (sp.n - k) + k)
    # ordered by target, then 2m transfer, then source
    dm = np.array(sp.twom)[a] - np.array(sp.twom)[c]
    key = list(zip(tgt.tolist(), dm.tolist(), src.tolist(), a.tolist()))
    assert key == sorted(key)


def test_errors_are_reported():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    with pytest.raises(trbl.TrblError) as e:
        trbl.Basis(sp, 13, sp, 1, 0)
    assert e.value.code == trbl.TRBL_ERR_ARG
    assert "n_particles" in str(e.value)
    with pytest.raises(trbl.TrblError):
        trbl.Basis(sp, 2, sp, 2, 41)  # no determinants reach 2M = 41


def test_non_finite_coefficients_are_rejected_before_any_upload():
    sp = synth.make_space(synth.SPACE12_SHELLS)
    inter = synth.draw_interaction(sp, sp, 3)
    tb = trbl.Basis(sp, 2, sp, 2, 0)
    for name, val in (("h1A", np.nan), ("VBB", np.inf), ("VAB", -np.inf)):
        arrs = {k: getattr(inter, k).copy() for k in ("h1A", "h1B", "VAA", "VBB", "VAB")}
        arrs[name].flat[7] = val
        with pytest.raises(trbl.TrblError) as e:
            trbl.Hamiltonian(tb, arrs["h1A"], arrs["h1B"], arrs["VAA"], arrs["VBB"], arrs["VAB"])
        assert e.value.code == trbl.TRBL_ERR_ARG
        assert name + "[7] is not finite" in str(e.value)


def test_parameter_order_matches_generator():
    for shells in (synth.SPACE12_SHELLS, synth.SPACE20_SHELLS, synth.TABLE1_SHELLS):
        sp = synth.make_space(shells)
        inter = synth.draw_interaction(sp, sp, 9)
        b = trbl.Basis(sp, 1, sp, 1, sp.twom[0] + sp.twom[-1])
        assert trbl.trbl_param_count(b.handle) == len(inter.theta)
        arrs = trbl.arrays_from_theta(sp.twom, sp.twom, inter.theta)
        for a, r in zip(arrs, (inter.h1A, inter.h1B, inter.VAA, inter.VBB, inter.VAB)):
            assert np.array_equal(a, r)
