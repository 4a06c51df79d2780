"""Plain complex128 OMM for Hermitian matrices (k points), from the paper (test infrastructure only).

The paper writes the method for complex matrices throughout (Sec. 2.1-2.3:
C^H, D^H, (S_W')^H); its k-point tests (Sec. 3.3) solve one Hermitian problem
per point of a Monkhorst-Pack grid. This module takes the same steps as
`oracle.omm` in that notation, in complex arithmetic:

  shift            H~ = H - eta S                              Sec. 2.2, Eq. 9
  preconditioner   P = (S + T/tau)^-1                           Sec. 2.4, Eq. 17
  subspace         H_W = C^H H~ C, S_W = C^H S C                Sec. 2.1, Eqs. 5-6
  functional       E~ = 4 Tr H_W - 2 Tr(S_W H_W)  (real)        Sec. 2.1, Eq. 8
  gradient         G = 8 HC - 4 SC H_W - 4 HC S_W               Sec. 2.3, Eq. 12
  direction        Polak-Ribiere with Re<A, B> = Re Tr(A^H B)   Sec. 2.3
  quartic          alpha_0..alpha_4 from the traces of Eq. 13 with (S_W')^H, real parts
  update           H_W += x (H_W' + H_W'^H) + x^2 H_W''         Sec. 2.3, Eq. 16
  outputs          E = E~ + 2 n eta, D = 2 C (2I - S_W) C^H, EDM
  Cholesky flavour S = L L^H, H_r = L^-1 H L^-H, S -> I        Sec. 2.4 (last paragraph)

Conventions: C is m x n (column i = Wannier function i); inputs given in the
library's n x m row-major layout are transposed (not conjugated) on entry, so
row j of that layout is column j of C. The gradient G is that of E~ as a real
function of (Re C, Im C): dE~ = Re Tr(G^H dC). The functional, the traces of
Hermitian products and the line minimum are real; the Polak-Ribiere and
descent tests use the real part of the Frobenius product.
"""
from __future__ import annotations

import math

import numpy as np

from .omm import STATUS_NO_CONVERGENCE, STATUS_OK, STATUS_UNBOUNDED, line_minimum, quartic_value


def _h(A: np.ndarray) -> np.ndarray:
    return A.conj().T


def _rtr(A: np.ndarray) -> float:
    return float(np.real(np.trace(A)))


def _rdot(A: np.ndarray, B: np.ndarray) -> float:
    """Re <A, B> = Re Tr(A^H B) (np.vdot conjugates its first argument)."""
    return float(np.real(np.vdot(A, B)))


def preconditioner(S: np.ndarray, T, tau: float) -> np.ndarray:
    """P = (S + T/tau)^-1 (Sec. 2.4, Eq. 17) by a complex Cholesky factorisation."""
    A = S + (T / tau if (T is not None and np.isfinite(tau)) else 0.0)
    L = np.linalg.cholesky(A)
    Linv = np.linalg.inv(L)
    return _h(Linv) @ Linv


def functional(HW: np.ndarray, SW: np.ndarray) -> float:
    """E~ = 4 Tr H_W - 2 Tr(S_W H_W) (Sec. 2.1, Eq. 8), real for Hermitian H_W, S_W."""
    return 4.0 * _rtr(HW) - 2.0 * _rtr(SW @ HW)


def gradient(HC, SC, HW, SW) -> np.ndarray:
    """G = 8 HC - 4 SC H_W - 4 HC S_W (Sec. 2.3, Eq. 12)."""
    return 8.0 * HC - 4.0 * SC @ HW - 4.0 * HC @ SW


def quartic_coefficients(E, HW, SW, HW1, SW1, HW2, SW2) -> np.ndarray:
    """alpha_0..alpha_4 of E~(C + x Delta) (Eq. 13 with Hermitian conjugates), all real.

    HW1 = Delta^H H C, HW2 = Delta^H H Delta (Eqs. 14-15), likewise SW1, SW2.
    """
    a1 = 8.0 * _rtr(HW1) - 4.0 * _rtr(SW1 @ HW) - 4.0 * _rtr(SW @ HW1)
    a2 = (4.0 * _rtr(HW2) - 2.0 * _rtr(SW2 @ HW) - 2.0 * _rtr(SW @ HW2)
          - 4.0 * _rtr(SW1 @ HW1) - 4.0 * _rtr(_h(SW1) @ HW1))
    a3 = -4.0 * _rtr(SW2 @ HW1) - 4.0 * _rtr(SW1 @ HW2)
    a4 = -2.0 * _rtr(SW2 @ HW2)
    return np.array([E, a1, a2, a3, a4], dtype=float)


def solve(H, S, T, eta, tau, C0_nm, tol_grad=1e-9, max_iter=2000, precondition=True,
          callback=None, want_matrices=True):
    """Minimise the OMM functional over complex C by preconditioned CG with exact line searches.

    tol_grad applies to max over the entries of max(|Re G|, |Im G|). Returns C (m x n), E, E~,
    H_W, S_W, gmax, the iteration count, status and, when asked, D and EDM (m x m, Hermitian).
    """
    H = np.asarray(H, dtype=complex)
    S = np.asarray(S, dtype=complex)
    Ht = H - eta * S
    P = preconditioner(S, None if T is None else np.asarray(T, dtype=complex), tau) if precondition else None
    C = np.array(np.asarray(C0_nm).T, dtype=complex, copy=True)
    n = C.shape[1]

    def state(C):
        HC = Ht @ C
        SC = S @ C
        return HC, SC, _h(C) @ HC, _h(C) @ SC

    def gmax_of(G):
        return float(max(np.abs(G.real).max(), np.abs(G.imag).max()))

    HC, SC, HW, SW = state(C)
    E = functional(HW, SW)
    G = gradient(HC, SC, HW, SW)
    Delta = PG_old = gpg_old = None
    status = STATUS_NO_CONVERGENCE
    it = 0
    for it in range(max_iter + 1):
        if gmax_of(G) < tol_grad:
            status = STATUS_OK
            break
        if it == max_iter:
            break
        PG = P @ G if P is not None else G.copy()
        gpg = _rdot(G, PG)
        beta = 0.0 if Delta is None else max(0.0, _rdot(G, PG - PG_old) / gpg_old)
        Dn = -PG + beta * Delta if beta > 0.0 else -PG
        if _rdot(G, Dn) >= 0.0:
            Dn = -PG
        HD = Ht @ Dn
        SD = S @ Dn
        HW1, SW1 = _h(Dn) @ HC, _h(Dn) @ SC
        HW2, SW2 = _h(Dn) @ HD, _h(Dn) @ SD
        a = quartic_coefficients(E, HW, SW, HW1, SW1, HW2, SW2)
        x, st = line_minimum(a)
        if st != STATUS_OK:
            status = st
            break
        C = C + x * Dn
        HC = HC + x * HD
        SC = SC + x * SD
        HW = HW + x * (HW1 + _h(HW1)) + x * x * HW2
        SW = SW + x * (SW1 + _h(SW1)) + x * x * SW2
        E_new = quartic_value(a, x)
        PG_old, gpg_old, Delta = PG, gpg, Dn
        G = gradient(HC, SC, HW, SW)
        if callback is not None:
            callback(it, E_new, x, beta)
        E = E_new
    # certificate: every output recomputed from the final C
    HC, SC, HW, SW = state(C)
    Et = functional(HW, SW)
    G = gradient(HC, SC, HW, SW)
    out = {"C": C, "E": Et + 2.0 * n * eta, "Etilde": Et, "HW": HW, "SW": SW, "gmax": gmax_of(G),
           "iters": it, "status": status}
    if want_matrices:
        D = 2.0 * C @ (2.0 * np.eye(n) - SW) @ _h(C)
        out["D"] = D
        out["EDM"] = 2.0 * C @ HW @ _h(C) + eta * D
    return out


def exact_minimum(H, S, n):
    """E* = 2 sum of the n lowest eigenvalues of H x = eps S x (Hermitian), D*, EDM* (LAPACK)."""
    import scipy.linalg
    w, X = scipy.linalg.eigh(np.asarray(H, dtype=complex), np.asarray(S, dtype=complex))
    occ = X[:, :n]
    return {"E": 2.0 * float(np.sum(w[:n])), "eps": w, "X": occ, "D": 2.0 * occ @ _h(occ),
            "EDM": 2.0 * (occ * w[:n][None, :]) @ _h(occ), "homo": float(w[n - 1]),
            "lumo": float(w[n]) if n < len(w) else math.nan}


def embed(A: np.ndarray) -> np.ndarray:
    """The real form [[Re A, -Im A], [Im A, Re A]] of a complex matrix (a ring homomorphism)."""
    A = np.asarray(A, dtype=complex)
    return np.block([[A.real, -A.imag], [A.imag, A.real]])


def solve_cholesky(H, S, eta, C0_nm, tol_grad=1e-9, max_iter=2000, callback=None, want_matrices=True):
    """The Cholesky flavour for Hermitian matrices (Sec. 2.4, last paragraph, with C^H): S = L L^H,
    H_r = L^-1 H L^-H, C_r = L^H C, the OMM with S = I and no preconditioner, then C = L^-H C_r.
    H_W, S_W and E are the same in both bases; tol_grad applies to the reduced gradient."""
    H = np.asarray(H, dtype=complex)
    S = np.asarray(S, dtype=complex)
    m = H.shape[0]
    L = np.linalg.cholesky(S)
    Linv = np.linalg.inv(L)
    Hr = Linv @ H @ _h(Linv)
    Hr = 0.5 * (Hr + _h(Hr))
    C = np.asarray(C0_nm, dtype=complex).T
    Cr0 = _h(L) @ C
    r = solve(Hr, np.eye(m, dtype=complex), None, eta, math.inf, Cr0.T, tol_grad=tol_grad, max_iter=max_iter,
              precondition=False, callback=callback, want_matrices=False)
    Cback = _h(Linv) @ r["C"]
    out = dict(r)
    out["C"] = Cback
    if want_matrices:
        n = Cback.shape[1]
        D = 2.0 * Cback @ (2.0 * np.eye(n) - r["SW"]) @ _h(Cback)
        out["D"] = D
        out["EDM"] = 2.0 * Cback @ r["HW"] @ _h(Cback) + eta * D
    return out
