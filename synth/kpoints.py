"""Complex Hermitian k-point problems of crystalline Si (input generation only).

The paper's k-point tests (Sec. 3.3) solve bulk Si in its 8-atom cell (DZP: m = 104,
n = 16) at every point of a Monkhorst-Pack grid. Here the Bloch matrices come from the
Gamma-point matrices of a supercell of g1 x g2 x g3 conventional cells built by the same
finite-range model as the other workloads, folded back:

    H(k)_{mu nu} = sum_c H_sc[mu in cell 0, nu in cell c] exp(i k . R_c),
    k = 2 pi (j1/g1, j2/g2, j3/g3) / a,

which is exact for the k of this Gamma-centred grid: the supercell's Gamma-point spectrum
is the union of the spectra of H(k) x = eps S(k) x. The diagonal jitter is periodic (the
same for every cell) so that the supercell keeps the lattice's translation symmetry. One
eta for all k: above the highest occupied level of the grid and inside the gap.

For any other k (a Monkhorst-Pack grid such as the paper's 9 x 9 x 9) the real-space
blocks h(R) are read from a 4 x 4 x 4 supercell (edge 41 bohr): every matrix element of
the model has range r_c = 9 bohr and its separable potential sums paths of at most 3 r_c,
so no element of that supercell mixes two periodic images, and each atom pair's element
belongs to the translation of its minimum image. Then H(k) = sum_R h(R) exp(i k . R).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .configs import ETA_ABOVE_HOMO, JITTER_SIGMA, TAU_10RY, _streams
from .model import build_matrices
from .systems import A_SI, si_model, si_supercell


@dataclass
class KProblem:
    name: str
    m: int
    n: int
    k: np.ndarray                 # (nk, 3) wave vectors (bohr^-1)
    H: list                       # nk complex m x m
    S: list
    T: list
    eta: float
    tau: float
    C0: list                      # nk complex n x m (library layout)
    seed: int
    meta: dict = field(default_factory=dict)
    supercell: tuple | None = None   # (H_sc, S_sc) when kept


def silicon_kpoints(grid=(2, 2, 2), basis="DZP", seed=0, keep_supercell=False) -> KProblem:
    """Bulk Si, 8-atom conventional cell, on a g1 x g2 x g3 Gamma-centred k grid."""
    streams = _streams(seed)
    model = si_model(basis)
    norb = model.species["Si"].norb
    m = 8 * norb
    ncell = int(np.prod(grid))
    jitter_cell = streams[1].normal(0.0, JITTER_SIGMA, size=m)
    symbols, pos, cell = si_supercell(*grid)
    S_sc, T_sc, H_sc, _ = build_matrices(model, symbols, pos, cell, np.tile(jitter_cell, ncell))
    cells = np.array([(i, j, k) for i in range(grid[0]) for j in range(grid[1]) for k in range(grid[2])], float)
    R = cells * A_SI                                                   # (ncell, 3)
    ks = np.array([(i / grid[0], j / grid[1], k / grid[2]) for i in range(grid[0])
                   for j in range(grid[1]) for k in range(grid[2])]) * (2.0 * np.pi / A_SI)

    def fold(M, kv):
        ph = np.exp(1j * (R @ kv))                                     # (ncell,)
        blocks = M[:m, :].reshape(m, ncell, m)                         # [mu, c, nu]
        A = np.einsum("acb,c->ab", blocks, ph)
        return 0.5 * (A + A.conj().T)

    Hk = [fold(H_sc, kv) for kv in ks]
    Sk = [fold(S_sc, kv) for kv in ks]
    Tk = [fold(T_sc, kv) for kv in ks]
    n = 16
    import scipy.linalg
    homo = max(float(scipy.linalg.eigh(h, s, eigvals_only=True, subset_by_index=[n - 1, n - 1])[0])
               for h, s in zip(Hk, Sk))
    lumo = min(float(scipy.linalg.eigh(h, s, eigvals_only=True, subset_by_index=[n, n])[0])
               for h, s in zip(Hk, Sk))
    eta = homo + min(ETA_ABOVE_HOMO, 0.5 * (lumo - homo))
    C0 = [(streams[2].normal(0.0, 0.1, size=(n, m)) + 1j * streams[2].normal(0.0, 0.1, size=(n, m)))
          / np.sqrt(2 * m) for _ in ks]
    meta = {"system": "Si", "basis": basis, "grid": list(grid), "homo": homo, "lumo": lumo,
            "gap": lumo - homo, "atoms_per_cell": 8}
    return KProblem(name=f"si8_{basis}_k{grid[0]}x{grid[1]}x{grid[2]}", m=m, n=n, k=ks, H=Hk, S=Sk, T=Tk,
                    eta=float(eta), tau=TAU_10RY, C0=C0, seed=seed, meta=meta,
                    supercell=(H_sc, S_sc) if keep_supercell else None)


def _bloch_blocks(basis, seed, sc=(4, 4, 4)):
    """Real-space blocks of the 8-atom cell read from an sc supercell.

    Returns (m, norb, H_rows, S_rows, T_rows, R): rows of cell 0 against the whole supercell
    (m x m_sc each) and R[a, b'] the lattice translation of atom b' relative to the cell-0 copy
    of its sublattice site, taken at the minimum image from atom a (shape 8 x natoms x 3).
    """
    streams = _streams(seed)
    model = si_model(basis)
    norb = model.species["Si"].norb
    m = 8 * norb
    ncell = int(np.prod(sc))
    jitter_cell = streams[1].normal(0.0, JITTER_SIGMA, size=m)
    symbols, pos, cell = si_supercell(*sc)
    S_sc, T_sc, H_sc, _ = build_matrices(model, symbols, pos, cell, np.tile(jitter_cell, ncell))
    nat = len(symbols)
    d = pos[None, :, :] - pos[:8, None, :]                      # (8, nat, 3) from atom a to b'
    d -= cell * np.round(d / cell)
    site = pos[np.arange(nat) % 8]                              # cell-0 copy of b'
    R = pos[:8, None, :] + d - site[None, :, :]
    return m, norb, H_sc[:m], S_sc[:m], T_sc[:m], R, streams


def monkhorst_pack(q, time_reversal=True):
    """Monkhorst-Pack grid q1 x q2 x q3 of the cubic cell: (k vectors, weights summing to 1).

    With time_reversal, k and -k (H(-k) = conj H(k) for real h(R)) are merged: one of each
    pair is kept with twice the weight.
    """
    axes = [(2.0 * np.arange(1, qi + 1) - qi - 1) / (2.0 * qi) for qi in q]
    frac = np.array([(x, y, z) for x in axes[0] for y in axes[1] for z in axes[2]])
    w = np.full(len(frac), 1.0 / len(frac))
    if time_reversal:
        key = {tuple(np.round(f, 12)): i for i, f in enumerate(frac)}
        keep, wk = [], []
        for i, f in enumerate(frac):
            j = key.get(tuple(np.round(-f, 12)))
            if j is None or j > i:
                keep.append(i)
                wk.append(w[i] * (2.0 if j is not None and j != i else 1.0))
            elif j == i:
                keep.append(i)
                wk.append(w[i])
        frac, w = frac[keep], np.array(wk)
    return frac * (2.0 * np.pi / A_SI), w


def bloch_matrices(ks, basis="DZP", seed=0, sc=(4, 4, 4)):
    """H(k), S(k), T(k) = sum_R h(R) exp(i k . R) of the 8-atom cell at the wave vectors ks,
    with h(R) read from an sc supercell. Returns (Hk, Sk, Tk, streams)."""
    m, norb, Hr, Sr, Tr, R, streams = _bloch_blocks(basis, seed, sc)
    nat = R.shape[1]

    def bloch(rows, kv):
        ph = np.exp(1j * (R @ kv))                                  # (8, nat)
        full = rows.reshape(8, norb, nat, norb) * ph[:, None, :, None]   # [a, mu, b', nu]
        out = full.reshape(8, norb, nat // 8, 8, norb).sum(axis=2).reshape(m, m)
        return 0.5 * (out + out.conj().T)

    return ([bloch(Hr, kv) for kv in ks], [bloch(Sr, kv) for kv in ks], [bloch(Tr, kv) for kv in ks],
            streams)


def silicon_mp_grid(q=(9, 9, 9), basis="DZP", seed=0, time_reversal=True) -> KProblem:
    """Bulk Si (8-atom cell) on a q1 x q2 x q3 Monkhorst-Pack grid, the paper's k-point test
    shape (Sec. 3.3: 9 x 9 x 9); k and -k merged with time_reversal (weights in meta)."""
    ks, wk = monkhorst_pack(q, time_reversal)
    Hk, Sk, Tk, streams = bloch_matrices(ks, basis, seed)
    m, n = Hk[0].shape[0], 16
    import scipy.linalg
    ev = [scipy.linalg.eigh(h, s, eigvals_only=True, subset_by_index=[n - 1, n]) for h, s in zip(Hk, Sk)]
    homo = max(float(e[0]) for e in ev)
    lumo = min(float(e[1]) for e in ev)
    eta = homo + min(ETA_ABOVE_HOMO, 0.5 * (lumo - homo))
    C0 = [(streams[2].normal(0.0, 0.1, size=(n, m)) + 1j * streams[2].normal(0.0, 0.1, size=(n, m)))
          / np.sqrt(2 * m) for _ in ks]
    meta = {"system": "Si", "basis": basis, "mp_grid": list(q), "time_reversal": time_reversal,
            "weights": wk.tolist(), "homo": homo, "lumo": lumo, "gap": lumo - homo, "atoms_per_cell": 8}
    return KProblem(name=f"si8_{basis}_mp{q[0]}x{q[1]}x{q[2]}", m=m, n=n, k=ks, H=Hk, S=Sk, T=Tk,
                    eta=float(eta), tau=TAU_10RY, C0=C0, seed=seed, meta=meta)


def hexagonal_mp(q1, q2, time_reversal=True):
    """Monkhorst-Pack grid q1 x q2 of the hexagonal cell (reciprocal vectors of a1 = a(1, 0),
    a2 = a(1/2, sqrt 3/2)): (k vectors, weights summing to 1)."""
    from .systems import A_GRAPHENE
    a = A_GRAPHENE
    b1 = 2.0 * np.pi / a * np.array([1.0, -1.0 / np.sqrt(3.0), 0.0])
    b2 = 2.0 * np.pi / a * np.array([0.0, 2.0 / np.sqrt(3.0), 0.0])
    u1 = (2.0 * np.arange(1, q1 + 1) - q1 - 1) / (2.0 * q1)
    u2 = (2.0 * np.arange(1, q2 + 1) - q2 - 1) / (2.0 * q2)
    frac = np.array([(x, y) for x in u1 for y in u2])
    w = np.full(len(frac), 1.0 / len(frac))
    if time_reversal:
        key = {tuple(np.round(f, 12)): i for i, f in enumerate(frac)}
        keep, wk = [], []
        for i, f in enumerate(frac):
            j = key.get(tuple(np.round(-f, 12)))
            if j is None or j > i or j == i:
                keep.append(i)
                wk.append(w[i] * (2.0 if (j is not None and j != i) else 1.0))
        frac, w = frac[keep], np.array(wk)
    return frac[:, :1] * b1[None, :] + frac[:, 1:] * b2[None, :], w


def graphene_mp_grid(q=(19, 19), basis="DZP", seed=0, time_reversal=True, sc=(9, 6)) -> KProblem:
    """One graphene layer on a q1 x q2 Monkhorst-Pack grid (the paper's second k-point test,
    Sec. 3.3: 19 x 19 x 1, DZP m = 26, n = 4). h(R) is read from an sc rectangular supercell
    (9 x 6: 42 x 48 bohr in the layer, 41 bohr of vacuum: no element mixes periodic images). This
    model does not reproduce graphene's Dirac points: its fourth and fifth bands keep a gap of at
    least 0.10 Ha over the grid, so one eta above every occupied level fits (when a grid has no
    common gap, eta is nan and meta holds an eta per k point, inside each one's gap)."""
    from .systems import carbon_model, graphene_supercell
    streams = _streams(seed)
    model = carbon_model(basis)
    norb = model.species["C"].norb
    m = 2 * norb
    symbols, pos, cell, sub = graphene_supercell(*sc)
    ncell = len(pos) // 2
    jitter_cell = streams[1].normal(0.0, JITTER_SIGMA, size=m)
    jitter = np.concatenate([jitter_cell[s * norb:(s + 1) * norb] for s in sub])
    S_sc, T_sc, H_sc, _ = build_matrices(model, symbols, pos, cell, jitter)
    nat = len(symbols)
    d = pos[None, :, :] - pos[:2, None, :]
    d -= cell * np.round(d / cell)
    R = pos[:2, None, :] + d - pos[sub][None, :, :]                  # (2, nat, 3) lattice translations
    ks, wk = hexagonal_mp(q[0], q[1], time_reversal)

    def bloch(M, kv):
        ph = np.exp(1j * (R @ kv))
        full = M[:m].reshape(2, norb, nat, norb) * ph[:, None, :, None]
        out = np.zeros((2, norb, 2, norb), dtype=complex)
        for b in range(2):
            out[:, :, b, :] = full[:, :, sub == b, :].sum(axis=2)
        out = out.reshape(m, m)
        return 0.5 * (out + out.conj().T)

    Hk = [bloch(H_sc, kv) for kv in ks]
    Sk = [bloch(S_sc, kv) for kv in ks]
    Tk = [bloch(T_sc, kv) for kv in ks]
    n = 4
    import scipy.linalg
    ev = [scipy.linalg.eigh(h, s, eigvals_only=True, subset_by_index=[n - 1, n]) for h, s in zip(Hk, Sk)]
    etas = [float(e[0] + min(ETA_ABOVE_HOMO, 0.5 * (e[1] - e[0]))) for e in ev]
    homo, lumo = max(float(e[0]) for e in ev), min(float(e[1]) for e in ev)
    eta = homo + min(ETA_ABOVE_HOMO, 0.5 * (lumo - homo)) if lumo > homo else float("nan")
    C0 = [(streams[2].normal(0.0, 0.1, size=(n, m)) + 1j * streams[2].normal(0.0, 0.1, size=(n, m)))
          / np.sqrt(2 * m) for _ in ks]
    gaps = [float(e[1] - e[0]) for e in ev]
    meta = {"system": "graphene", "basis": basis, "mp_grid": [q[0], q[1], 1], "time_reversal": time_reversal,
            "weights": wk.tolist(), "etas": etas, "gaps": gaps, "min_gap": min(gaps), "homo": homo, "lumo": lumo,
            "cells_in_supercell": ncell}
    return KProblem(name=f"graphene_{basis}_mp{q[0]}x{q[1]}x1", m=m, n=n, k=ks, H=Hk, S=Sk, T=Tk,
                    eta=float(eta), tau=TAU_10RY, C0=C0, seed=seed, meta=meta)
