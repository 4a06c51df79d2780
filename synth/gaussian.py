"""Analytic overlap and kinetic integrals between real Cartesian Gaussian orbitals.

Input generation only: nothing here is part of the orbital minimization method.
The orbitals are primitive Gaussians (x-A_x)^i (y-A_y)^j (z-A_z)^k exp(-a|r-A|^2)
combined into real s, p and d functions (the five d functions are xy, yz, zx,
x^2-y^2 and 3z^2-r^2), each normalised to unit self-overlap.

One-dimensional overlaps follow the Obara-Saika recurrences (Obara & Saika,
J. Chem. Phys. 84, 3963 (1986)); the kinetic integral uses the action of
d^2/dx^2 on a Cartesian Gaussian,
    d^2/dx^2 G_j = j(j-1) G_{j-2} - 2b(2j+1) G_j + 4 b^2 G_{j+2},
so that T_ij = -1/2 <G_i| d^2/dx^2 |G_j> and, in 3D,
    T = T_x S_y S_z + S_x T_y S_z + S_x S_y T_z.
All arrays are vectorised over a batch of centre displacements.
"""
from __future__ import annotations

import numpy as np

# real orbital -> list of (cartesian exponent triple, coefficient)
ORBITALS = {
    "s": [[((0, 0, 0), 1.0)]],
    "p": [[((1, 0, 0), 1.0)], [((0, 1, 0), 1.0)], [((0, 0, 1), 1.0)]],
    "d": [
        [((1, 1, 0), 1.0)],
        [((0, 1, 1), 1.0)],
        [((1, 0, 1), 1.0)],
        [((2, 0, 0), 1.0), ((0, 2, 0), -1.0)],
        [((0, 0, 2), 2.0), ((2, 0, 0), -1.0), ((0, 2, 0), -1.0)],
    ],
}

NFUNC = {"s": 1, "p": 3, "d": 5}


def overlap_1d(a: float, b: float, X: np.ndarray, imax: int, jmax: int) -> np.ndarray:
    """1D overlaps S[i, j, ...] = int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) dx.

    X = A - B (any shape). Returns an array of shape (imax+1, jmax+1) + X.shape.
    """
    p = a + b
    mu = a * b / p
    xpa = -b / p * X
    xpb = a / p * X
    S = np.zeros((imax + 1, jmax + 1) + np.shape(X))
    S[0, 0] = np.sqrt(np.pi / p) * np.exp(-mu * X * X)
    inv2p = 0.5 / p
    for j in range(jmax):
        S[0, j + 1] = xpb * S[0, j] + (j * S[0, j - 1] * inv2p if j > 0 else 0.0)
    for i in range(imax):
        for j in range(jmax + 1):
            t = xpa * S[i, j]
            if i > 0:
                t = t + i * inv2p * S[i - 1, j]
            if j > 0:
                t = t + j * inv2p * S[i, j - 1]
            S[i + 1, j] = t
    return S


def kinetic_1d(b: float, S: np.ndarray, imax: int, jmax: int) -> np.ndarray:
    """1D kinetic integrals T[i, j] from a table S with at least jmax+2 columns."""
    T = np.zeros((imax + 1, jmax + 1) + S.shape[2:])
    for i in range(imax + 1):
        for j in range(jmax + 1):
            t = -2.0 * b * (2 * j + 1) * S[i, j] + 4.0 * b * b * S[i, j + 2]
            if j >= 2:
                t = t + j * (j - 1) * S[i, j - 2]
            T[i, j] = -0.5 * t
    return T


def _cart_blocks(la: str, a: float, lb: str, b: float, R: np.ndarray):
    """Un-normalised S and T blocks (na, nb, P) for shells on A=0 and B=R (R: (P, 3))."""
    X = -R  # A - B
    tabs_S = []
    tabs_T = []
    for ax in range(3):
        S1 = overlap_1d(a, b, X[:, ax], 2, 4)
        tabs_S.append(S1)
        tabs_T.append(kinetic_1d(b, S1, 2, 2))
    fa = ORBITALS[la]
    fb = ORBITALS[lb]
    P = R.shape[0]
    Sblk = np.zeros((len(fa), len(fb), P))
    Tblk = np.zeros((len(fa), len(fb), P))
    for ia, comb_a in enumerate(fa):
        for ib, comb_b in enumerate(fb):
            s_acc = np.zeros(P)
            t_acc = np.zeros(P)
            for (ea, ca) in comb_a:
                for (eb, cb) in comb_b:
                    sx = tabs_S[0][ea[0], eb[0]]
                    sy = tabs_S[1][ea[1], eb[1]]
                    sz = tabs_S[2][ea[2], eb[2]]
                    tx = tabs_T[0][ea[0], eb[0]]
                    ty = tabs_T[1][ea[1], eb[1]]
                    tz = tabs_T[2][ea[2], eb[2]]
                    s_acc += ca * cb * sx * sy * sz
                    t_acc += ca * cb * (tx * sy * sz + sx * ty * sz + sx * sy * tz)
            Sblk[ia, ib] = s_acc
            Tblk[ia, ib] = t_acc
    return Sblk, Tblk


def shell_norms(l: str, a: float) -> np.ndarray:
    """Normalisation constants 1/sqrt(<f|f>) of the real functions of one shell."""
    S, _ = _cart_blocks(l, a, l, a, np.zeros((1, 3)))
    return 1.0 / np.sqrt(np.array([S[i, i, 0] for i in range(S.shape[0])]))


def pair_blocks(la: str, a: float, lb: str, b: float, R: np.ndarray):
    """Normalised overlap and kinetic blocks, shapes (na, nb, P), for B - A = R."""
    Sblk, Tblk = _cart_blocks(la, a, lb, b, R)
    na = shell_norms(la, a)
    nb = shell_norms(lb, b)
    scale = na[:, None, None] * nb[None, :, None]
    return Sblk * scale, Tblk * scale
