"""Geometries and parameter sets for the synthetic Si and liquid-water workloads.

Input generation only. Units: bohr and hartree.

Si: diamond structure, conventional cubic cell a = 10.26 bohr (8 atoms).
  Slater-Koster couplings follow Harrison's universal sp parameters
  (W. A. Harrison, "Electronic Structure and the Properties of Solids", 1980):
  V_ll'm = eta_ll'm * hbar^2/(m d^2) with eta_sss = -1.40, eta_sps = 1.84,
  eta_pps = 3.24, eta_ppp = -0.81; hbar^2/m = 1 in atomic units, d0 = sqrt(3) a / 4.
  On-site levels eps_s = -13.55 eV and eps_p = -6.52 eV (Harrison's term values).
  With this model's kinetic and overlap terms the 64-atom cell has a gap of
  0.13 Ha (single-zeta) and 0.11 Ha (DZP-like) at half filling of the s/p bands.
Water: rigid molecules, O-H 1.81 bohr, H-O-H 104.5 degrees, 1 g/cm^3. The
  on-site levels and couplings are chosen for this project so that the four
  lowest molecular levels per molecule sit well below the rest (64-molecule
  boxes, seeds 0-4: generalised HOMO-LUMO gaps 0.11-0.21 Ha).
"""
from __future__ import annotations

import numpy as np

from .model import Model, Shell, SKPair, Species

HARTREE_EV = 27.211386245988
A_SI = 10.26
D0_SI = np.sqrt(3.0) * A_SI / 4.0

DIAMOND_BASIS = np.array([
    [0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


# Basis sets by orbitals per atom (n = 2 per Si atom, so the occupied fraction is 2 / norb):
#   SZ 4 (50%), DZ 8 (25%), TZ 12 (16.7%), DZP 13 (15.4%), DZP+p 16 (12.5%).
# Higher zetas are tighter Gaussians; only the first zeta enters the two-centre terms.
SI_SHELLS = {
    "s1": Shell("s1", "s", 0.35, True), "p1": Shell("p1", "p", 0.30, True),
    "s2": Shell("s2", "s", 0.875, False), "p2": Shell("p2", "p", 0.75, False),
    "s3": Shell("s3", "s", 2.2, False), "p3": Shell("p3", "p", 1.9, False),
    "d": Shell("d", "d", 0.35, False),
}
SI_BASES = {
    "SZ": ["s1", "p1"],
    "DZ": ["s1", "p1", "s2", "p2"],
    "TZ": ["s1", "p1", "s2", "p2", "s3", "p3"],
    "DZP": ["s1", "p1", "s2", "p2", "d"],
    "DZP+p": ["s1", "p1", "s2", "p2", "d", "p3"],
}


def si_species(basis: str) -> Species:
    eps = {"s": -13.55 / HARTREE_EV, "p": -6.52 / HARTREE_EV, "d": 0.15}
    if basis not in SI_BASES:
        raise ValueError(basis)
    return Species("Si", [SI_SHELLS[k] for k in SI_BASES[basis]], eps)


def si_model(basis: str) -> Model:
    inv = 1.0 / D0_SI ** 2
    pair = SKPair(d0=D0_SI, ss=-1.40 * inv, sp=1.84 * inv, ps=1.84 * inv,
                  pp_sigma=3.24 * inv, pp_pi=-0.81 * inv)
    return Model(species={"Si": si_species(basis)}, sk={("Si", "Si"): pair}, rc=9.0,
                 params={"system": "Si", "basis": basis, "a": A_SI, "d0": D0_SI})


def si_supercell(k1: int, k2: int, k3: int):
    """Diamond supercell of k1 x k2 x k3 conventional cells."""
    cells = np.array([(i, j, k) for i in range(k1) for j in range(k2) for k in range(k3)], float)
    frac = (cells[:, None, :] + DIAMOND_BASIS[None, :, :]).reshape(-1, 3)
    pos = frac * A_SI
    cell = np.array([k1, k2, k3], float) * A_SI
    return ["Si"] * len(pos), pos, cell


# ---------------------------------------------------------------- water
R_OH = 1.81
ANGLE_HOH = np.deg2rad(104.5)
WATER_MOLAR_G = 18.015
AVOGADRO = 6.02214076e23
BOHR_CM = 0.529177210903e-8


# Water basis sets by orbitals per molecule (n = 4 per molecule):
#   DZ+d 17 (O s,p,s,p,d; H s,s: 23.5%), DZP 23 (H adds p: 17.4%),
#   TZP 29 (O and H add a third, tighter s and O a third p: 13.8%).
O_SHELLS = {
    "s1": Shell("s1", "s", 0.80, True), "p1": Shell("p1", "p", 0.60, True),
    "s2": Shell("s2", "s", 2.0, False), "p2": Shell("p2", "p", 1.5, False),
    "s3": Shell("s3", "s", 5.0, False), "p3": Shell("p3", "p", 3.8, False),
    "d": Shell("d", "d", 0.8, False),
}
H_SHELLS = {
    "s1": Shell("s1", "s", 0.60, True), "s2": Shell("s2", "s", 1.5, False),
    "s3": Shell("s3", "s", 3.8, False), "p": Shell("p", "p", 0.75, False),
}
WATER_BASES = {
    "DZ+d": (["s1", "p1", "s2", "p2", "d"], ["s1", "s2"]),
    "DZP": (["s1", "p1", "s2", "p2", "d"], ["s1", "s2", "p"]),
    "TZP": (["s1", "p1", "s2", "p2", "s3", "p3", "d"], ["s1", "s2", "s3", "p"]),
}


def water_species(basis: str = "DZP"):
    if basis not in WATER_BASES:
        raise ValueError(basis)
    o_keys, h_keys = WATER_BASES[basis]
    o = Species("O", [O_SHELLS[k] for k in o_keys], {"s": -1.20, "p": -0.45, "d": 0.40})
    h = Species("H", [H_SHELLS[k] for k in h_keys], {"s": -0.20, "p": 0.40})
    return o, h


def water_model(basis: str = "DZP") -> Model:
    o, h = water_species(basis)
    oh = SKPair(d0=R_OH, ss=-0.60, sp=0.0, ps=0.80)          # s_O-s_H, s_H-p_O
    ho = SKPair(d0=R_OH, ss=-0.60, sp=0.80, ps=0.0)
    oo = SKPair(d0=5.4, ss=-0.02, sp=0.03, ps=0.03, pp_sigma=0.05, pp_pi=-0.012)
    d_hh = 2.0 * R_OH * np.sin(ANGLE_HOH / 2.0)
    hh = SKPair(d0=d_hh, ss=-0.03)
    return Model(species={"O": o, "H": h},
                 sk={("O", "H"): oh, ("H", "O"): ho, ("O", "O"): oo, ("H", "H"): hh},
                 rc=9.0, params={"system": "water", "basis": basis})


def water_box_length(nmol: int, density_g_cm3: float = 1.0) -> float:
    vol_cm3 = nmol * WATER_MOLAR_G / (AVOGADRO * density_g_cm3)
    return vol_cm3 ** (1.0 / 3.0) / BOHR_CM


def _random_rotation(u: np.ndarray) -> np.ndarray:
    """Uniform random rotation from three uniforms (Shoemake's quaternion method)."""
    u1, u2, u3 = u
    q = np.array([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)])
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_box(nmol: int, rng: np.random.Generator, dmin: float = 4.7, max_tries: int = 200000):
    """Random water box: O centres uniform with minimum O-O distance dmin, random orientations."""
    L = water_box_length(nmol)
    cell = np.array([L, L, L])
    centres = np.zeros((0, 3))
    tries = 0
    while centres.shape[0] < nmol:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("water_box: could not place molecules")
        c = rng.uniform(0.0, L, size=3)
        if centres.shape[0]:
            d = centres - c
            d -= cell * np.round(d / cell)
            if np.min(np.einsum("ij,ij->i", d, d)) < dmin * dmin:
                continue
        centres = np.vstack([centres, c])
    h1 = R_OH * np.array([np.sin(ANGLE_HOH / 2), 0.0, np.cos(ANGLE_HOH / 2)])
    h2 = R_OH * np.array([-np.sin(ANGLE_HOH / 2), 0.0, np.cos(ANGLE_HOH / 2)])
    symbols = []
    pos = []
    for c in centres:
        Rm = _random_rotation(rng.uniform(size=3))
        symbols += ["O", "H", "H"]
        pos += [c, c + Rm @ h1, c + Rm @ h2]
    pos = np.array(pos)
    pos -= cell * np.floor(pos / cell)
    return symbols, pos, cell


# ---------------------------------------------------------------- graphene
# One layer, a = 2.46 Angstrom; the 2-atom hexagonal cell of the paper's second k-point test
# (DZP: m = 26, n = 4). Carbon shells are the Si ones scaled to the shorter bond (exponents times
# (d_Si / d_C)^2 ~ 2.7); Harrison's universal couplings at d0 = a / sqrt(3) and his carbon term
# values eps_s = -17.52 eV, eps_p = -8.97 eV.
A_GRAPHENE = 2.46 / 0.529177210903
D0_C = A_GRAPHENE / np.sqrt(3.0)
C_SHELLS = {
    "s1": Shell("s1", "s", 0.96, True), "p1": Shell("p1", "p", 0.82, True),
    "s2": Shell("s2", "s", 2.4, False), "p2": Shell("p2", "p", 2.05, False),
    "d": Shell("d", "d", 0.96, False),
}
C_BASES = {"SZ": ["s1", "p1"], "DZP": ["s1", "p1", "s2", "p2", "d"]}


def carbon_model(basis: str = "DZP") -> Model:
    if basis not in C_BASES:
        raise ValueError(basis)
    eps = {"s": -17.52 / HARTREE_EV, "p": -8.97 / HARTREE_EV, "d": 0.15}
    c = Species("C", [C_SHELLS[k] for k in C_BASES[basis]], eps)
    inv = 1.0 / D0_C ** 2
    pair = SKPair(d0=D0_C, ss=-1.40 * inv, sp=1.84 * inv, ps=1.84 * inv,
                  pp_sigma=3.24 * inv, pp_pi=-0.81 * inv)
    return Model(species={"C": c}, sk={("C", "C"): pair}, rc=9.0,
                 params={"system": "graphene", "basis": basis, "a": A_GRAPHENE, "d0": D0_C})


def graphene_supercell(n1: int, n2: int, vacuum: float = 41.0):
    """n1 x n2 rectangular cells (a x sqrt(3) a, 4 atoms each) of one graphene layer in an
    orthorhombic box of height `vacuum`. Atoms 0 and 1 are the A and B sites of the hexagonal cell
    at the origin; sublattice[i] says which of the two atom i is a lattice translate of."""
    a = A_GRAPHENE
    rect = np.array([[0.0, 0.0], [a / 2, a / (2 * np.sqrt(3.0))], [a / 2, np.sqrt(3.0) * a / 2],
                     [0.0, 2 * a / np.sqrt(3.0)]])
    sub = np.array([0, 1, 0, 1])
    pos, sl = [], []
    for i in range(n1):
        for j in range(n2):
            for r, s in zip(rect, sub):
                pos.append([r[0] + i * a, r[1] + j * np.sqrt(3.0) * a, 0.0])
                sl.append(s)
    cell = np.array([n1 * a, n2 * np.sqrt(3.0) * a, vacuum])
    return ["C"] * len(pos), np.array(pos), cell, np.array(sl)
