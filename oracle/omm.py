"""Plain float64 OMM, step by step from the paper (test infrastructure only).

Convention: C is m x n (paper, Sec. 2.1): column i holds Wannier function i
over the m basis functions. Inputs given as n x m row-major arrays (the
library's layout) are transposed on entry.

Steps and their sources (Corsetti, arXiv:1312.1549):
  shift            H~ = H - eta S                          Sec. 2.2, Eq. 9
  preconditioner   P = (S + T/tau)^-1                       Sec. 2.4, Eq. 17
  functional       E~ = 4 Tr H_W - 2 Tr(S_W H_W)            Sec. 2.1, Eq. 8 (Eqs. 5-6)
  gradient         G = 8 HC - 4 SC H_W - 4 HC S_W           Sec. 2.3, Eq. 12
  direction        Polak-Ribiere conjugate direction        Sec. 2.3
  quartic          alpha_0 .. alpha_4 from traces           Sec. 2.3, Eqs. 13-15
  line minimum     x = argmin of the quartic                Sec. 2.3
  update           C, H_W, S_W (and HC, SC)                 Sec. 2.3, Eq. 16 and its footnote
  stopping         |G|_inf < tol, and optionally Eq. 18     Sec. 2.5.2
  outputs          E = E~ + 2 n eta, D, EDM                 Sec. 2.1-2.2
  Cholesky flavour S = L L^T, H_r = L^-1 H L^-T, S -> I,    Sec. 2.4 (last paragraph)
                   C_r = L^T C, no preconditioner, and back

Readings where the paper is silent or ambiguous (each one also listed in the
design notes of the repository):
  * Eq. 10 writes E~ -> E~ + n eta; with the spin factor 2 of Eq. 7 the shift
    lowers 2 sum eps_i by 2 n eta, so E = E~_shifted + 2 n eta.
  * Polak-Ribiere with the preconditioner: beta = <G_k, P(G_k - G_{k-1})> /
    <G_{k-1}, P G_{k-1}> (Frobenius products), clipped at 0 (PR+); the
    direction restarts at -P G when beta = 0 or when it is not a descent
    direction (<G, Delta> >= 0).
  * Eq. 18 is read with an absolute value.
  * Line minimum: the first local minimum along the descent direction (the
    smallest x > 0 with p' = 0 and p'' > 0); none -> the functional is
    unbounded along the line (Sec. 2.2 footnote). Taking the lowest of two
    minima instead can jump into the region where the shifted functional has
    no lower bound (observed without preconditioning on the Si64 workload).
"""
from __future__ import annotations

import math

import numpy as np

STATUS_OK = 0
STATUS_UNBOUNDED = 3
STATUS_NO_CONVERGENCE = 4


def shift(H: np.ndarray, S: np.ndarray, eta: float) -> np.ndarray:
    """H~ = H - eta S (Sec. 2.2, Eq. 9)."""
    return H - eta * S


def preconditioner(S: np.ndarray, T: np.ndarray, tau: float) -> np.ndarray:
    """P = (S + T/tau)^-1 (Sec. 2.4, Eq. 17), by a Cholesky factorisation.

    tau = inf gives P = S^-1 (the pure tensorial correction).
    """
    A = S + (T / tau if np.isfinite(tau) else 0.0)
    L = np.linalg.cholesky(A)
    Linv = np.linalg.inv(L)
    return Linv.T @ Linv


def subspace_operators(C: np.ndarray, Ht: np.ndarray, S: np.ndarray):
    """HC, SC and H_W = C^T H C, S_W = C^T S C (Sec. 2.1, Eqs. 5-6)."""
    HC = Ht @ C
    SC = S @ C
    return HC, SC, C.T @ HC, C.T @ SC


def functional_from_subspace(HW: np.ndarray, SW: np.ndarray) -> float:
    """E~ = 2 Tr[(2I - S_W) H_W] = 4 Tr H_W - 2 Tr(S_W H_W) (Sec. 2.1, Eq. 8)."""
    return 4.0 * np.trace(HW) - 2.0 * np.trace(SW @ HW)


def functional(C: np.ndarray, Ht: np.ndarray, S: np.ndarray) -> float:
    _, _, HW, SW = subspace_operators(C, Ht, S)
    return functional_from_subspace(HW, SW)


def gradient(HC: np.ndarray, SC: np.ndarray, HW: np.ndarray, SW: np.ndarray) -> np.ndarray:
    """G = 8 HC - 4 SC H_W - 4 HC S_W (Sec. 2.3, Eq. 12): the exact dE~/dC."""
    return 8.0 * HC - 4.0 * SC @ HW - 4.0 * HC @ SW


def quartic_coefficients(E: float, HW, SW, HW1, SW1, HW2, SW2) -> np.ndarray:
    """alpha_0 .. alpha_4 of E~(C + x Delta) (Sec. 2.3, Eq. 13).

    HW1 = Delta^T H C, HW2 = Delta^T H Delta (Eqs. 14-15), likewise SW1, SW2.
    """
    tr = np.trace
    a0 = E
    a1 = 8.0 * tr(HW1) - 4.0 * tr(SW1 @ HW) - 4.0 * tr(SW @ HW1)
    a2 = (4.0 * tr(HW2) - 2.0 * tr(SW2 @ HW) - 2.0 * tr(SW @ HW2)
          - 4.0 * tr(SW1 @ HW1) - 4.0 * tr(SW1.T @ HW1))
    a3 = -4.0 * tr(SW2 @ HW1) - 4.0 * tr(SW1 @ HW2)
    a4 = -2.0 * tr(SW2 @ HW2)
    return np.array([a0, a1, a2, a3, a4], dtype=float)


def quartic_value(a: np.ndarray, x: float) -> float:
    return float(a[0] + x * (a[1] + x * (a[2] + x * (a[3] + x * a[4]))))


def line_minimum(a: np.ndarray):
    """(x, status): the line minimum of the quartic with coefficients a (Sec. 2.3).

    The search direction is a descent direction (a1 = <G, Delta> < 0), so the
    step is the first local minimum met when moving along it: the smallest
    x > 0 with p'(x) = 0 and p''(x) > 0. Stationary points are the real roots
    of a1 + 2 a2 x + 3 a3 x^2 + 4 a4 x^3, found as companion-matrix eigenvalues
    (numpy.roots) and polished by two Newton steps. No such root means the
    functional decreases without bound along the line (Sec. 2.2, footnote).
    """
    d = np.array([4.0 * a[4], 3.0 * a[3], 2.0 * a[2], a[1]])
    roots = np.roots(d) if np.any(d[:3] != 0.0) else np.array([])
    cands = []
    for r in roots:
        if abs(r.imag) > 1e-8 * (1.0 + abs(r.real)):
            continue
        x = float(r.real)
        for _ in range(2):
            f1 = a[1] + x * (2 * a[2] + x * (3 * a[3] + x * 4 * a[4]))
            f2 = 2 * a[2] + x * (6 * a[3] + x * 12 * a[4])
            if f2 != 0.0:
                x -= f1 / f2
        if x > 0.0 and 2 * a[2] + x * (6 * a[3] + x * 12 * a[4]) > 0.0:
            cands.append(x)
    if a[1] >= 0.0 or not cands:
        return 0.0, STATUS_UNBOUNDED
    return min(cands), STATUS_OK


def density_matrix(C: np.ndarray, SW: np.ndarray) -> np.ndarray:
    """D = 2 C (2I - S_W) C^T = dE/dH at the minimum (equals 2 sum x_i x_i^T there)."""
    n = SW.shape[0]
    return 2.0 * C @ (2.0 * np.eye(n) - SW) @ C.T


def energy_density_matrix(C: np.ndarray, HW_shifted: np.ndarray, D: np.ndarray, eta: float):
    """EDM = 2 C H~_W C^T + eta D; dE/dS = -EDM at the minimum."""
    return 2.0 * C @ HW_shifted @ C.T + eta * D


def solve(H, S, T, eta, tau, C0_nm, tol_grad=1e-9, max_iter=2000, precondition=True,
          e_tol=0.0, C_is_mn=False, callback=None, want_matrices=True):
    """Minimise the OMM functional by preconditioned CG with exact line searches.

    Returns a dict with the converged C (m x n), the band energy E (unshifted),
    E~ (shifted functional), H_W, S_W, |G|_inf, the iteration count and, when
    asked, D and EDM.
    """
    m = H.shape[0]
    Ht = shift(H, S, eta)
    P = preconditioner(S, T, tau) if precondition else None
    C = np.array(C0_nm if C_is_mn else np.asarray(C0_nm).T, dtype=float, copy=True)
    n = C.shape[1]
    HC, SC, HW, SW = subspace_operators(C, Ht, S)
    E = functional_from_subspace(HW, SW)
    G = gradient(HC, SC, HW, SW)
    Delta = None
    G_old = None
    PG_old = None
    gpg_old = None
    status = STATUS_NO_CONVERGENCE
    it = 0
    history = []
    for it in range(max_iter + 1):
        gmax = float(np.max(np.abs(G)))
        history.append((E, gmax))
        if gmax < tol_grad:
            status = STATUS_OK
            break
        if it == max_iter:
            break
        PG = P @ G if P is not None else G.copy()
        gpg = float(np.vdot(G, PG))
        if Delta is None:
            beta = 0.0
        else:
            beta = max(0.0, float(np.vdot(G, PG - PG_old)) / gpg_old)
        Dn = -PG + beta * Delta if beta > 0.0 else -PG
        if float(np.vdot(G, Dn)) >= 0.0:
            Dn = -PG
        HD = Ht @ Dn
        SD = S @ Dn
        HW1 = Dn.T @ HC
        SW1 = Dn.T @ SC
        HW2 = Dn.T @ HD
        SW2 = Dn.T @ SD
        a = quartic_coefficients(E, HW, SW, HW1, SW1, HW2, SW2)
        x, st = line_minimum(a)
        if st != STATUS_OK:
            status = st
            break
        C = C + x * Dn
        HC = HC + x * HD
        SC = SC + x * SD
        HW = HW + x * (HW1 + HW1.T) + x * x * HW2
        SW = SW + x * (SW1 + SW1.T) + x * x * SW2
        E_new = quartic_value(a, x)
        G_old, PG_old, gpg_old, Delta = G, PG, gpg, Dn
        G = gradient(HC, SC, HW, SW)
        if callback is not None:
            callback(it, E_new, x, beta)
        if e_tol > 0.0 and abs(2.0 * (E_new - E) / (E_new + E)) <= e_tol:
            E = E_new
            status = STATUS_OK
            break
        E = E_new
    # certification: every output recomputed from the final C
    HC, SC, HW, SW = subspace_operators(C, Ht, S)
    Et = functional_from_subspace(HW, SW)
    G = gradient(HC, SC, HW, SW)
    out = {"C": C, "E": Et + 2.0 * n * eta, "Etilde": Et, "HW": HW, "SW": SW,
           "gmax": float(np.max(np.abs(G))), "iters": it, "status": status, "history": history}
    if want_matrices:
        D = density_matrix(C, SW)
        out["D"] = D
        out["EDM"] = energy_density_matrix(C, HW, D, eta)
    return out


def solve_cholesky(H, S, eta, C0_nm, tol_grad=1e-9, max_iter=2000, e_tol=0.0, C_is_mn=False,
                   callback=None, want_matrices=True):
    """The Cholesky flavour of the OMM (Sec. 2.4, last paragraph).

    The generalised problem is reduced to standard form with the Cholesky factor
    S = L L^T: H_r = L^-1 H L^-T and C_r = L^T C, so that S_W = C_r^T C_r. The OMM then
    minimises with S = I and without a preconditioner, and the result goes back to the
    original basis, C = L^-T C_r (the density matrix with it: D = L^-T D_r L^-1). H_W,
    S_W, the energies and the line-search steps are the same in both bases; the
    gradient and its stopping test (tol_grad) are those of the reduced problem.
    """
    m = H.shape[0]
    L = np.linalg.cholesky(S)
    Linv = np.linalg.inv(L)
    Hr = Linv @ H @ Linv.T
    Hr = 0.5 * (Hr + Hr.T)
    C = np.array(C0_nm if C_is_mn else np.asarray(C0_nm).T, dtype=float, copy=True)
    Cr0 = L.T @ C
    r = solve(Hr, np.eye(m), None, eta, math.inf, Cr0, tol_grad=tol_grad, max_iter=max_iter,
              precondition=False, e_tol=e_tol, C_is_mn=True, callback=callback, want_matrices=False)
    Cback = Linv.T @ r["C"]
    out = dict(r)
    out["C"] = Cback
    out["C_reduced"] = r["C"]
    if want_matrices:
        D = density_matrix(Cback, r["SW"])
        HW_shifted = Cback.T @ shift(H, S, eta) @ Cback
        out["D"] = D
        out["EDM"] = energy_density_matrix(Cback, HW_shifted, D, eta)
    return out
