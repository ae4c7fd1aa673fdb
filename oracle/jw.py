"""Jordan-Wigner matrix construction of the Hamiltonian (oracle pin only).

Test infrastructure only (see the package docstring).

An independent route to the same matrix on tiny spaces: each fermion
annihilator is the textbook Kronecker product
    c_j = Z (x) ... (x) Z (x) a (x) 1 (x) ... (x) 1,
with a = |0><1| on mode j and Z = diag(1, -1) on every earlier mode, modes of
species A first and then species B.  The Hamiltonian of Sec. II / App. B is
then a sum of sparse matrix products, and its restriction to the M-scheme
basis must equal the bit-string assembly element by element: a basis state
(A creators ascending)(B creators ascending)|0> is the plain occupation
vector with sign +1 in this representation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def annihilators(n_modes: int):
    a = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    I = sp.identity(2, format="csr")
    ops = []
    for j in range(n_modes):
        M = sp.identity(1, format="csr")
        for k in range(n_modes):
            f = Z if k < j else (a if k == j else I)
            M = sp.kron(M, f, format="csr")
        ops.append(M)
    return ops


def occupation_index(bits_by_mode, n_modes: int) -> int:
    """Row of the Kronecker basis for an occupation list (mode 0 most significant)."""
    idx = 0
    for j in range(n_modes):
        idx = (idx << 1) | bits_by_mode[j]
    return idx


def hamiltonian(inter) -> sp.csr_matrix:
    nA, nB = inter.h1A.shape[0], inter.h1B.shape[0]
    n = nA + nB
    c = annihilators(n)
    cd = [x.T.tocsr() for x in c]
    H = sp.csr_matrix((2 ** n, 2 ** n))
    for a in range(nA):
        for cc in range(nA):
            if inter.h1A[a, cc] != 0:
                H = H + inter.h1A[a, cc] * (cd[a] @ c[cc])
    for b in range(nB):
        for d in range(nB):
            if inter.h1B[b, d] != 0:
                H = H + inter.h1B[b, d] * (cd[nA + b] @ c[nA + d])
    for V, off, m in ((inter.VAA, 0, nA), (inter.VBB, nA, nB)):
        for a in range(m):
            for b in range(a + 1, m):
                for cc in range(m):
                    for d in range(cc + 1, m):
                        v = V[a, b, cc, d]
                        if v != 0:
                            H = H + v * (cd[off + a] @ cd[off + b] @ c[off + d] @ c[off + cc])
    for a in range(nA):
        for b in range(nB):
            for cc in range(nA):
                for d in range(nB):
                    v = inter.VAB[a, b, cc, d]
                    if v != 0:
                        H = H + v * (cd[a] @ cd[nA + b] @ c[nA + d] @ c[cc])
    return H.tocsr()


def restrict(HJW: sp.csr_matrix, states, nA: int, nB: int) -> np.ndarray:
    """Dense restriction of the JW matrix to the listed (bitsA, bitsB) states."""
    n = nA + nB
    idx = []
    for SA, SB in states:
        occ = [SA >> j & 1 for j in range(nA)] + [SB >> j & 1 for j in range(nB)]
        idx.append(occupation_index(occ, n))
    idx = np.array(idx)
    return HJW[idx][:, idx].toarray()
