"""Eigenpairs of the explicit Hamiltonian (oracle).

Test infrastructure only (see the package docstring).

* ``dense_eigh``: numpy's symmetric eigensolver on the dense matrix (small D).
* ``lanczos``: Algorithm 1 of Sec. III A (the simple Lanczos method) in FP64,
  with the reorthogonalisation against every stored Lanczos vector run twice
  (classical Gram-Schmidt applied twice).  Ritz values come from the
  tridiagonal T^(k) of Eq. (tmat); the residual of Ritz pair i is
  beta_k |U[k, i]|, the standard Lanczos residual bound.  The paper stops on
  a change of Ritz values below a threshold; here the residual criterion
  beta_k |U[k, i]| <= tol * ||H|| is used for the first nev pairs.
"""
from __future__ import annotations

from typing import Callable, Tuple

import numpy as np
import scipy.linalg as sla


def dense_eigh(H) -> Tuple[np.ndarray, np.ndarray]:
    A = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    return np.linalg.eigh(A)


def lanczos(matvec: Callable[[np.ndarray], np.ndarray], D: int, nev: int,
            tol: float, normH: float, v1: np.ndarray, max_iter: int = None,
            ) -> Tuple[np.ndarray, np.ndarray, np.ndarray, int]:
    """Algorithm 1 with full reorthogonalisation (applied twice).

    Returns (ritz values[:nev], ritz vectors D x nev, residual bounds[:nev],
    iterations).  Raises RuntimeError when max_iter passes unconverged.
    """
    if max_iter is None:
        max_iter = D
    max_iter = min(max_iter, D)
    Vs = np.zeros((D, max_iter + 1))
    v = v1 / np.linalg.norm(v1)
    Vs[:, 0] = v
    alpha = np.zeros(max_iter)
    beta = np.zeros(max_iter)
    for k in range(max_iter):
        w = matvec(Vs[:, k])
        alpha[k] = Vs[:, k] @ w
        w = w - alpha[k] * Vs[:, k]
        if k > 0:
            w = w - beta[k - 1] * Vs[:, k - 1]
        for _ in range(2):  # full reorthogonalisation, twice
            w = w - Vs[:, :k + 1] @ (Vs[:, :k + 1].T @ w)
        beta[k] = np.linalg.norm(w)
        m = k + 1
        if m >= nev:
            theta, U = sla.eigh_tridiagonal(alpha[:m], beta[:m - 1])
            res = beta[k] * np.abs(U[m - 1, :nev])
            if np.all(res <= tol * normH) or m == D:
                X = Vs[:, :m] @ U[:, :nev]
                return theta[:nev], X, res, m
        if beta[k] == 0.0:
            raise RuntimeError("Lanczos breakdown before convergence")
        Vs[:, k + 1] = w / beta[k]
    raise RuntimeError("Lanczos did not converge in %d iterations" % max_iter)


def extreme_eigenvalues(matvec, D: int, seed_vec: np.ndarray, tol=1e-12, normH_guess=1.0,
                        max_iter: int = 600) -> Tuple[float, float]:
    """Lowest and highest eigenvalue by Algorithm 1 on H and on -H."""
    lo = lanczos(matvec, D, 1, tol, normH_guess, seed_vec, max_iter)[0][0]
    hi = -lanczos(lambda x: -matvec(x), D, 1, tol, normH_guess, seed_vec, max_iter)[0][0]
    return float(lo), float(hi)
