"""Single-species systems (one species empty, as for the tin isotopes of
Sec. IV, where only neutrons are active): the product basis degenerates to
one species' determinants, there are no cross-species elements, and H is the
like-particle part plus one-body energies.  The CUDA product is checked
element by element against the oracle's explicit CSR H, and the solver's
eigenvalues against dense eigh.

Tolerances as in the other product and solver tests: |W - H V|_ij <=
rtol (|H| |V|)_ij with rtol 1e-12 (FP64) and 1e-5 (FP32); eigenvalues
within 1e-9 ||H|| (FP64) and 1e-6 ||H|| (mixed)."""
import functools

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import hamiltonian as oh

torch = pytest.importorskip("torch")
trbl = pytest.importorskip("paper_1902_02064_gb300")

pytestmark = pytest.mark.gpu
RTOL = {torch.float64: 1e-12, torch.float32: 1e-5}

CASES = [  # shells, particles of A, particles of B, 2M, seed
    (synth.SPACE12_SHELLS, 4, 0, 0, 41),
    (synth.SPACE12_SHELLS, 0, 3, 1, 42),
    (synth.SPACE20_SHELLS, 5, 0, 1, 43),
    (synth.SPACE20_SHELLS, 0, 6, 0, 44),
]


@functools.lru_cache(maxsize=None)
def _setup(shells, kA, kB, twoM, seed):
    sp = synth.make_space(shells)
    inter = synth.draw_interaction(sp, sp, seed)
    B = ob.ProductBasis(sp.twom, kA, sp.twom, kB, twoM)
    H = oh.assemble(B, inter)
    tb = trbl.Basis(sp, kA, sp, kB, twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    assert tb.dim == B.dim
    return B, H, tb, th


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype,q", [(torch.float64, 4), (torch.float32, 8), (torch.float32, 32)])
def test_single_species_product_all_elements(case, dtype, q):
    B, H, tb, th = _setup(*case)
    V = torch.from_numpy(synth.random_block(B.dim, q, 7)).to(dtype)
    W = th.apply(V.cuda()).cpu().double().numpy()
    Vd = V.double().numpy()
    ref = H @ Vd
    bound = abs(H) @ np.abs(Vd)
    err = np.abs(W - ref)
    assert np.all(err <= RTOL[dtype] * bound + 1e-300), float((err / (bound + 1e-300)).max())


@pytest.mark.parametrize("case", [CASES[0], CASES[3]])
@pytest.mark.parametrize("precision,tol,bar", [(1, 1e-10, 1e-9), (2, 1e-6, 1e-6)])
def test_single_species_lowest_eigenvalues(case, precision, tol, bar):
    B, H, tb, th = _setup(*case)
    ev = np.linalg.eigvalsh(H.toarray())
    normH = max(abs(ev[0]), abs(ev[-1]))
    nev, q = 10, 4
    mb = min(48, B.dim)
    evals, resid, X, st = trbl.solve(th, nev, q, mb, tol, precision=precision)
    assert np.abs(evals - ev[:nev]).max() <= bar * normH
