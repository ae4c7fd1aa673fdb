"""Thick-restart block Lanczos method in FP64 (oracle).

Test infrastructure only (see the package docstring).

The steps of Sec. III C/D in the paper's notation, with numpy doing each
dense step:

* a block V_1 of p orthonormal columns starts the iteration; k_x = 0;
* block step k: W := H V_k and alpha_k := V_k^T W (Alg. 3 / Alg. 4), which
  fills the diagonal block of T at rows k_x + p(k-1) .. k_x + pk; W is then
  orthogonalised against every stored Lanczos vector (classical
  Gram-Schmidt applied twice), and V_{k+1} beta_k := QR(W) (numpy's
  Householder QR) fills the off-diagonal blocks beta_k and beta_k^T;
* the Ritz pairs of T^(k) are tested after the QR: the residual estimate of
  pair i is ||beta_k U[last p rows, i]||, and the iteration stops when the
  nev lowest all reach tol ||H|| (the paper tests a change of the Ritz
  values; the residual form is the reading used throughout);
* when one more block would exceed l_m vectors, the thick restart of
  Eq. (trb-tmat) keeps the l_s lowest Ritz vectors v_k := sum_j v_j U_jk,
  takes V_1 := V_{k_m+1} as the next block, sets the leading l_s x l_s part
  of T to diag(e_1 .. e_ls) and the coupling r := beta_{k_m} U[last p
  rows, 1:l_s] beside it, and continues with k_x := l_s.

Nothing here is blocked, fused or reordered beyond those steps.
"""
from __future__ import annotations

from typing import Callable, Dict, Optional

import numpy as np


def trbl(matvec: Callable[[np.ndarray], np.ndarray], D: int, nev: int, p: int, l_m: int, l_s: int,
         tol: float, normH: float, V1: np.ndarray, max_steps: int = 10000,
         snapshot: Optional[Callable[[Dict], None]] = None):
    """Lowest nev eigenpairs of the symmetric operator behind matvec.

    matvec maps a D x p block to H times it.  Returns (theta[:nev],
    X (D x nev), residual estimates[:nev], stats dict with 'steps' and
    'restarts').  snapshot, when given, receives after every block step a
    dict with the stored vectors 'V' (D x n), 'T' (n x n), the new block
    'Vnext', 'beta' and 'restarted' (whether this step restarted), for
    tests of the algebra.
    """
    if not (nev <= l_s and l_s + 2 * p <= l_m):
        raise ValueError("need nev <= l_s and l_s + 2p <= l_m")
    V = np.zeros((D, l_m))
    T = np.zeros((l_m, l_m))
    Q, _ = np.linalg.qr(np.asarray(V1, dtype=np.float64))
    V[:, :p] = Q
    n = p          # stored Lanczos vectors, the current block included
    steps = restarts = 0
    while steps < max_steps:
        k0 = n - p  # first column of the current block V_k
        Vk = V[:, k0:n]
        W = matvec(Vk)
        alpha = Vk.T @ W
        T[k0:n, k0:n] = alpha
        for _ in range(2):  # full reorthogonalisation, twice
            W = W - V[:, :n] @ (V[:, :n].T @ W)
        Vnext, beta = np.linalg.qr(W)
        steps += 1
        theta, U = np.linalg.eigh(T[:n, :n])
        res = np.linalg.norm(beta @ U[k0:n, :], axis=0)
        m = min(nev, n)
        done = n >= nev and np.all(res[:m] <= tol * normH)
        restarted = False
        if not done:
            if n + p > l_m:
                # thick restart, Eq. (trb-tmat)
                kept = V[:, :n] @ U[:, :l_s]
                r = beta @ U[k0:n, :l_s]
                V[:, :l_s] = kept
                V[:, l_s:] = 0.0
                T[:, :] = 0.0
                T[:l_s, :l_s] = np.diag(theta[:l_s])
                T[l_s:l_s + p, :l_s] = r
                T[:l_s, l_s:l_s + p] = r.T
                V[:, l_s:l_s + p] = Vnext
                n = l_s + p
                restarts += 1
                restarted = True
            else:
                T[n:n + p, k0:n] = beta
                T[k0:n, n:n + p] = beta.T
                V[:, n:n + p] = Vnext
                n += p
        if snapshot is not None:
            snapshot({"V": V[:, :n].copy(), "T": T[:n, :n].copy(), "Vnext": Vnext, "beta": beta,
                      "restarted": restarted, "theta": theta, "U": U})
        if done:
            X = V[:, :n] @ U[:, :nev]
            return theta[:nev], X, res[:nev], {"steps": steps, "restarts": restarts}
    raise RuntimeError("thick-restart block Lanczos did not converge in %d steps" % max_steps)


def block_matvec(H) -> Callable[[np.ndarray], np.ndarray]:
    """Block product by an explicit (sparse or dense) matrix."""
    return lambda X: np.asarray(H @ X)
