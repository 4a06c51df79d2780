"""Brute-force generalised eigensolver for tiny inputs (test infrastructure only).

Solves H x = eps S x (the problem statement of Sec. 2.1, Eq. 1) without any
library eigensolver: a Cholesky factor S = L L^T (plain loops), the reduced
matrix A = L^-1 H L^-T (plain forward substitution) and the cyclic Jacobi
method (Jacobi 1846; e.g. Golub & Van Loan, Matrix Computations, Sec. 8.5) on
A. Pure-Python loops: meant for m up to a few dozen.
"""
from __future__ import annotations

import math

import numpy as np


def cholesky_lower(S: np.ndarray) -> np.ndarray:
    """Lower-triangular L with S = L L^T (row-by-row Cholesky-Banachiewicz)."""
    m = S.shape[0]
    L = np.zeros_like(S, dtype=float)
    for i in range(m):
        for j in range(i + 1):
            acc = S[i, j]
            for k in range(j):
                acc -= L[i, k] * L[j, k]
            if i == j:
                if acc <= 0.0:
                    raise np.linalg.LinAlgError("matrix is not positive definite")
                L[i, i] = math.sqrt(acc)
            else:
                L[i, j] = acc / L[j, j]
    return L


def forward_solve(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L X = B for lower-triangular L (column by column)."""
    m = L.shape[0]
    X = np.array(B, dtype=float, copy=True)
    for i in range(m):
        for k in range(i):
            X[i] -= L[i, k] * X[k]
        X[i] /= L[i, i]
    return X


def backward_solve_transpose(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L^T X = B for lower-triangular L."""
    m = L.shape[0]
    X = np.array(B, dtype=float, copy=True)
    for i in range(m - 1, -1, -1):
        for k in range(i + 1, m):
            X[i] -= L[k, i] * X[k]
        X[i] /= L[i, i]
    return X


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Eigenvalues (ascending) and orthonormal eigenvectors of a symmetric A by cyclic Jacobi."""
    A = np.array(A, dtype=float, copy=True)
    m = A.shape[0]
    V = np.eye(m)
    for _ in range(max_sweeps):
        off = math.sqrt(sum(A[p, q] ** 2 for p in range(m) for q in range(m) if p != q))
        scale = math.sqrt(sum(A[p, p] ** 2 for p in range(m))) + 1e-300
        if off <= tol * scale:
            break
        for p in range(m - 1):
            for q in range(p + 1, m):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                # rotation angle that zeroes A[p, q]
                theta = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                for k in range(m):
                    akp = A[k, p]
                    akq = A[k, q]
                    A[k, p] = c * akp - s * akq
                    A[k, q] = s * akp + c * akq
                for k in range(m):
                    apk = A[p, k]
                    aqk = A[q, k]
                    A[p, k] = c * apk - s * aqk
                    A[q, k] = s * apk + c * aqk
                for k in range(m):
                    vkp = V[k, p]
                    vkq = V[k, q]
                    V[k, p] = c * vkp - s * vkq
                    V[k, q] = s * vkp + c * vkq
    w = np.array([A[i, i] for i in range(m)])
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def generalized_eigh(H: np.ndarray, S: np.ndarray):
    """All eigenpairs of H x = eps S x with x^T S x = 1 (S symmetric positive definite)."""
    L = cholesky_lower(S)
    Y = forward_solve(L, H)                 # L^-1 H
    A = forward_solve(L, Y.T)               # L^-1 H L^-T (H symmetric)
    A = 0.5 * (A + A.T)
    w, Z = jacobi_eigh(A)
    X = backward_solve_transpose(L, Z)      # x = L^-T z
    return w, X
