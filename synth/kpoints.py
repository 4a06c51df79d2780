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
