"""Synthetic finite-range atomic-orbital Hamiltonians: S, T and H on a periodic cell.

Input generation only (no orbital-minimization arithmetic). The model:

* S = S_gauss * f(r) and T = T_gauss * f(r), with S_gauss and T_gauss the
  analytic overlap and kinetic integrals of normalised real Gaussians and
  f(r) = (1 - (r/r_c)^2)^2 for r < r_c, 0 beyond (r = centre distance).
* H = T + V, with V a separable operator sum_kl |phi_k> (U + M)_kl <phi_l|
  over the first-zeta s and p functions phi_k (the projectors). U is
  diagonal, U_k = eps_l - T_kk, so that a first-zeta function alone has the
  tabulated on-site level eps_l; M holds two-centre Slater-Koster couplings
  between projectors on different centres (Slater & Koster, Phys. Rev. 94,
  1498 (1954)) scaled by (d0/r)^2 f(r) / f(d0) (Harrison's 1/d^2 law with the
  same cutoff; the tabulated couplings are the values at r = d0). Second-zeta
  and polarisation functions feel V only through their overlaps with the
  projectors.
* A seeded Gaussian jitter (sigma = 0.01 Ha by default) is added to the
  diagonal of H.

Periodic boundary conditions are handled by summing each pair block over the
lattice translations that bring the centres within r_c (Gamma point).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .gaussian import NFUNC, pair_blocks


@dataclass(frozen=True)
class Shell:
    name: str          # e.g. "s1"
    l: str             # "s" | "p" | "d"
    alpha: float       # Gaussian exponent (bohr^-2)
    sk: bool           # takes part in the Slater-Koster two-centre terms


@dataclass
class Species:
    symbol: str
    shells: list
    eps: dict          # on-site level per channel l for the first-zeta function (Ha)

    @property
    def norb(self) -> int:
        return sum(NFUNC[s.l] for s in self.shells)

    def onsite_U(self) -> dict:
        """U_l = eps_l - T_ii of the first-zeta function of channel l."""
        U = {}
        for s in self.shells:
            if s.l not in U:
                U[s.l] = self.eps[s.l] - (2 * "spd".index(s.l) + 3) * s.alpha / 2.0
        return U


@dataclass
class SKPair:
    d0: float
    ss: float = 0.0
    sp: float = 0.0      # <s on first | V | p on second>, sigma
    ps: float = 0.0      # <s on second | V | p on first>, sigma
    pp_sigma: float = 0.0
    pp_pi: float = 0.0


@dataclass
class Model:
    species: dict
    sk: dict                               # (sym_a, sym_b) -> SKPair (both orders present)
    rc: float = 9.0
    params: dict = field(default_factory=dict)


def cutoff(r: np.ndarray, rc: float) -> np.ndarray:
    x = np.clip(r / rc, 0.0, 1.0)
    return np.where(r < rc, (1.0 - x * x) ** 2, 0.0)


def _sk_block(sa: Species, sb: Species, pair: SKPair, R: np.ndarray, rc: float) -> np.ndarray:
    """Two-centre SK block (norb_a, norb_b, P) between first-zeta s/p functions."""
    P = R.shape[0]
    out = np.zeros((sa.norb, sb.norb, P))
    r = np.linalg.norm(R, axis=1)
    safe = np.where(r > 0, r, 1.0)
    dc = R / safe[:, None]                       # direction cosines from A to B
    # the tabulated couplings are the cut-off couplings at r = d0
    scale = (pair.d0 / safe) ** 2 / cutoff(np.array(pair.d0), rc)
    oa = 0
    for sha in sa.shells:
        ob = 0
        for shb in sb.shells:
            if sha.sk and shb.sk:
                if sha.l == "s" and shb.l == "s":
                    out[oa, ob] = pair.ss * scale
                elif sha.l == "s" and shb.l == "p":
                    for k in range(3):
                        out[oa, ob + k] = dc[:, k] * pair.sp * scale
                elif sha.l == "p" and shb.l == "s":
                    for k in range(3):
                        out[oa + k, ob] = -dc[:, k] * pair.ps * scale
                elif sha.l == "p" and shb.l == "p":
                    for i in range(3):
                        for j in range(3):
                            v = dc[:, i] * dc[:, j] * (pair.pp_sigma - pair.pp_pi)
                            if i == j:
                                v = v + pair.pp_pi
                            out[oa + i, ob + j] = v * scale
            ob += NFUNC[shb.l]
        oa += NFUNC[sha.l]
    return out


def build_matrices(model: Model, symbols: list, pos: np.ndarray, cell: np.ndarray,
                   jitter: np.ndarray | None = None):
    """Dense S, T, H (float64, m x m) for atoms `symbols` at `pos` in the orthorhombic `cell`.

    The potential is a separable operator over the first-zeta (projector)
    functions K: V = S[:, K] (U + M) S[K, :], with U the on-site levels and M
    the two-centre Slater-Koster couplings between projector functions on
    different centres. Being a true operator, its generalised spectrum is
    bounded by |U + M| * lambda_max(S) however ill-conditioned S is. V is then
    cut off elementwise by f(r) of the minimum-image centre distance.

    Returns (S, T, H, offsets) with offsets[a] the first basis index of atom a.
    """
    import scipy.sparse as sp

    nat = len(symbols)
    norbs = np.array([model.species[s].norb for s in symbols])
    offsets = np.concatenate([[0], np.cumsum(norbs)[:-1]])
    m = int(norbs.sum())
    atom_of = np.repeat(np.arange(nat), norbs)
    # projector functions: first-zeta SK shells
    is_proj = np.zeros(m, dtype=bool)
    U = np.zeros(m)
    for a, sym in enumerate(symbols):
        spc = model.species[sym]
        Ul = spc.onsite_U()
        o = offsets[a]
        for sh in spc.shells:
            k = NFUNC[sh.l]
            if sh.sk:
                is_proj[o:o + k] = True
                U[o:o + k] = Ul[sh.l]
            o += k
    S = np.zeros((m, m))
    T = np.zeros((m, m))
    m_rows, m_cols, m_vals = [], [], []
    rc = model.rc
    cell = np.asarray(cell, dtype=float)
    shifts = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)],
                      dtype=float) * cell[None, :]
    sym_arr = np.array(symbols)
    for a0 in range(0, nat, 256):
        a1 = min(nat, a0 + 256)
        d = pos[None, :, :] - pos[a0:a1, None, :]              # (A, nat, 3) from a to b
        d -= cell * np.round(d / cell)
        for sh in shifts:
            dd = d + sh
            r = np.linalg.norm(dd, axis=2)
            ia, ib = np.nonzero(r < rc)
            if ia.size == 0:
                continue
            ia_g = ia + a0
            Rv = dd[ia, ib]
            rv = r[ia, ib]
            f = cutoff(rv, rc)
            for sa_sym in model.species:
                for sb_sym in model.species:
                    sel = (sym_arr[ia_g] == sa_sym) & (sym_arr[ib] == sb_sym)
                    if not np.any(sel):
                        continue
                    A = ia_g[sel]
                    B = ib[sel]
                    R = Rv[sel]
                    fr = f[sel]
                    onsite = rv[sel] == 0.0
                    sa = model.species[sa_sym]
                    sb = model.species[sb_sym]
                    Sblk = np.zeros((sa.norb, sb.norb, R.shape[0]))
                    Tblk = np.zeros_like(Sblk)
                    oa = 0
                    for sha in sa.shells:
                        ob = 0
                        for shb in sb.shells:
                            s_, t_ = pair_blocks(sha.l, sha.alpha, shb.l, shb.alpha, R)
                            Sblk[oa:oa + NFUNC[sha.l], ob:ob + NFUNC[shb.l]] = s_
                            Tblk[oa:oa + NFUNC[sha.l], ob:ob + NFUNC[shb.l]] = t_
                            ob += NFUNC[shb.l]
                        oa += NFUNC[sha.l]
                    Sblk *= fr[None, None, :]
                    Tblk *= fr[None, None, :]
                    na, nb = sa.norb, sb.norb
                    rows = (offsets[A][None, None, :] + np.arange(na)[:, None, None])
                    cols = (offsets[B][None, None, :] + np.arange(nb)[None, :, None])
                    rows = np.broadcast_to(rows, Sblk.shape).ravel()
                    cols = np.broadcast_to(cols, Sblk.shape).ravel()
                    np.add.at(S, (rows, cols), Sblk.ravel())
                    np.add.at(T, (rows, cols), Tblk.ravel())
                    pair = model.sk.get((sa_sym, sb_sym))
                    if pair is not None and not np.all(onsite):
                        V = _sk_block(sa, sb, pair, R, rc) * fr[None, None, :]
                        V[:, :, onsite] = 0.0
                        keep = V.ravel() != 0.0
                        m_rows.append(rows[keep])
                        m_cols.append(cols[keep])
                        m_vals.append(V.ravel()[keep])
    S = 0.5 * (S + S.T)
    T = 0.5 * (T + T.T)
    # separable potential over the projector functions
    K = np.nonzero(is_proj)[0]
    kpos = -np.ones(m, dtype=np.int64)
    kpos[K] = np.arange(K.size)
    if m_rows:
        mr = np.concatenate(m_rows)
        mc = np.concatenate(m_cols)
        mv = np.concatenate(m_vals)
    else:
        mr = mc = np.zeros(0, dtype=np.int64)
        mv = np.zeros(0)
    Mk = sp.coo_matrix((mv, (kpos[mr], kpos[mc])), shape=(K.size, K.size)).tocsr()
    Mk = 0.5 * (Mk + Mk.T) + sp.diags(U[K])
    SK = sp.csr_matrix(S[:, K])
    V = (SK @ Mk @ SK.T).tocoo()
    dv = pos[atom_of[V.col]] - pos[atom_of[V.row]]
    dv -= cell * np.round(dv / cell)
    fv = cutoff(np.linalg.norm(dv, axis=1), rc)
    H = T.copy()
    np.add.at(H, (V.row, V.col), V.data * fv)
    H = 0.5 * (H + H.T)
    if jitter is not None:
        H[np.diag_indices(m)] += jitter
    return S, T, H, offsets
