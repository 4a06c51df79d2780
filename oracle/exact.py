"""The exact result of the OMM by its plain definition (test infrastructure only).

Sec. 2.1 (Eqs. 7-8): at the minimum of the OMM functional S_W = I and the
functional equals the band energy E_0 = 2 sum_{i<=n} eps_i (factor 2 for spin)
of the n lowest generalised eigenpairs of H x = eps S x (Eq. 1). The density
matrix is D = 2 sum_{i<=n} x_i x_i^T with x_i^T S x_i = 1, and the energy
density matrix EDM = 2 sum_{i<=n} eps_i x_i x_i^T.

The eigenpairs come from scipy.linalg.eigh (a library primitive), or from the
project's own Jacobi solver (`method="jacobi"`, tiny inputs only).
"""
from __future__ import annotations

import numpy as np


def eigenpairs(H: np.ndarray, S: np.ndarray, method: str = "lapack"):
    if method == "jacobi":
        from .jacobi import generalized_eigh
        return generalized_eigh(H, S)
    import scipy.linalg
    w, X = scipy.linalg.eigh(H, S)
    return w, X


def exact_minimum(H: np.ndarray, S: np.ndarray, n: int, method: str = "lapack", want_matrices=True):
    """E*, D*, EDM*, eigenvalues and the occupied eigenvectors X (m x n, S-orthonormal)."""
    w, X = eigenpairs(H, S, method)
    occ = X[:, :n]
    out = {"E": 2.0 * float(np.sum(w[:n])), "eps": w, "homo": float(w[n - 1]),
           "lumo": float(w[n]) if n < len(w) else float("nan")}
    if want_matrices:
        out["X"] = occ
        out["D"] = 2.0 * occ @ occ.T
        out["EDM"] = 2.0 * (occ * w[:n][None, :]) @ occ.T
    return out


def homo_lumo(H: np.ndarray, S: np.ndarray, n: int):
    """(eps_n, eps_{n+1}) only (for the eigenspectrum shift eta of Sec. 2.2)."""
    import scipy.linalg
    w = scipy.linalg.eigh(H, S, eigvals_only=True, subset_by_index=[n - 1, n])
    return float(w[0]), float(w[1])
