"""The five seeded synthetic workloads (and small variants for tests).

Input generation only. Every random number comes from numpy's PCG64 through a
SeedSequence: child stream 0 drives the geometry (water), child 1 the on-site
jitter of H, child 2 the starting coefficients C0.

Layout: H, S, T are m x m float64 (symmetric). C0 is n x m row-major: row j is
Wannier function j over the m basis functions (the same bytes as an m x n
column-major matrix).

eta is the eigenspectrum shift: 0.1 Ha above the highest occupied generalised
eigenvalue. It needs one eigensolve of the generated matrices; the value is
read from `eta_table.json` (written by `synth/make_eta_table.py`) when the
entry exists, else computed here with scipy.linalg.eigh on the host.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

from .model import build_matrices
from .systems import si_model, si_supercell, water_box, water_model

TAU_10RY = 5.0           # tau = 10 Ry expressed in hartree
ETA_ABOVE_HOMO = 0.1     # Ha
GAP_MIN = 0.05           # Ha
JITTER_SIGMA = 0.01      # Ha

_TABLE_PATH = os.path.join(os.path.dirname(__file__), "eta_table.json")


@dataclass
class Problem:
    name: str
    m: int
    n: int
    H: np.ndarray
    S: np.ndarray
    T: np.ndarray
    eta: float
    tau: float
    C0: np.ndarray
    seed: int
    meta: dict = field(default_factory=dict)


def _streams(seed: int):
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]


def _load_table() -> dict:
    if os.path.exists(_TABLE_PATH):
        with open(_TABLE_PATH) as fh:
            return json.load(fh)
    return {}


def spectrum_edges(H: np.ndarray, S: np.ndarray, n: int):
    """(HOMO, LUMO) = (eps_n, eps_{n+1}) of H x = eps S x (host eigensolve)."""
    import scipy.linalg
    w = scipy.linalg.eigh(H, S, eigvals_only=True, subset_by_index=[n - 1, n])
    return float(w[0]), float(w[1])


def _finish(name, key, H, S, T, n, seed, streams, meta, need_eta=True, eta=None):
    m = H.shape[0]
    table = _load_table()
    ent = table.get(f"{key}@{seed}")
    if eta is None and need_eta:
        if ent is not None and ent.get("m") == m:
            homo, lumo = ent["homo"], ent["lumo"]
        else:
            homo, lumo = spectrum_edges(H, S, n)
        meta.update(homo=homo, lumo=lumo, gap=lumo - homo)
        eta = homo + ETA_ABOVE_HOMO
    C0 = streams[2].normal(0.0, 0.1, size=(n, m)) / np.sqrt(m)
    meta["table_key"] = f"{key}@{seed}"
    return Problem(name=name, m=m, n=n, H=H, S=S, T=T, eta=float(eta) if eta is not None else 0.0,
                   tau=TAU_10RY, C0=C0, seed=seed, meta=meta)


def silicon(k=(2, 2, 2), basis="SZ", seed=0, name=None, need_eta=True, eta=None) -> Problem:
    """Si diamond supercell of k conventional cells; n = 2 per atom."""
    streams = _streams(seed)
    model = si_model(basis)
    symbols, pos, cell = si_supercell(*k)
    m = model.species["Si"].norb * len(symbols)
    jitter = streams[1].normal(0.0, JITTER_SIGMA, size=m)
    S, T, H, _ = build_matrices(model, symbols, pos, cell, jitter)
    n = 2 * len(symbols)
    key = f"si_{basis}_{k[0]}x{k[1]}x{k[2]}"
    meta = {"system": "Si", "basis": basis, "atoms": len(symbols), "cell": cell.tolist()}
    return _finish(name or key, key, H, S, T, n, seed, streams, meta, need_eta, eta)


def water(nmol=256, seed=0, name=None, need_eta=True, eta=None, basis="DZP") -> Problem:
    """Liquid-water box of nmol molecules at 1 g/cm^3; n = 4 per molecule."""
    streams = _streams(seed)
    model = water_model(basis)
    symbols, pos, cell = water_box(nmol, streams[0])
    m = sum(model.species[s].norb for s in symbols)
    jitter = streams[1].normal(0.0, JITTER_SIGMA, size=m)
    S, T, H, _ = build_matrices(model, symbols, pos, cell, jitter)
    n = 4 * nmol
    key = f"water_{nmol}" if basis == "DZP" else f"water_{basis}_{nmol}"
    meta = {"system": "water", "basis": basis, "molecules": nmol, "cell": cell.tolist()}
    return _finish(name or key, key, H, S, T, n, seed, streams, meta, need_eta, eta)


def _gap_guarded(builder, seed, **kw):
    """Apply the gap guard: resample with seed+1 while the HOMO-LUMO gap < GAP_MIN."""
    for s in range(seed, seed + 20):
        p = builder(seed=s, **kw)
        if p.meta.get("gap", 1.0) >= GAP_MIN:
            return p
    raise RuntimeError("gap guard: no seed gave a gap >= %g Ha" % GAP_MIN)


# ------------------------------------------------------------------ named configs
def si64_sz(seed=0) -> Problem:
    """Si64 sp single-zeta: m = 256, n = 128."""
    return _gap_guarded(silicon, seed, k=(2, 2, 2), basis="SZ", name="si64_sz")


def si512_dzp(seed=0) -> Problem:
    """Si512 DZP-like (13 orbitals per atom): m = 6656, n = 1024."""
    return _gap_guarded(silicon, seed, k=(4, 4, 4), basis="DZP", name="si512_dzp")


def water256_dzp(seed=0) -> Problem:
    """Water256 DZP-like (23 orbitals per molecule): m = 5888, n = 1024."""
    return _gap_guarded(water, seed, nmol=256, name="water256_dzp")


SI_CELL_SHAPES = {4: (1, 2, 2), 5: (1, 1, 5), 6: (1, 2, 3), 8: (2, 2, 2), 9: (1, 3, 3), 10: (1, 2, 5),
                  12: (2, 2, 3), 16: (2, 2, 4), 18: (2, 3, 3), 20: (2, 2, 5), 24: (2, 3, 4),
                  27: (3, 3, 3), 30: (2, 3, 5), 32: (2, 4, 4), 36: (3, 3, 4), 40: (2, 4, 5),
                  45: (3, 3, 5), 48: (3, 4, 4), 50: (2, 5, 5), 60: (3, 4, 5), 64: (4, 4, 4)}

# occupied fraction n/m of each basis (n = 2 per Si atom, 4 per water molecule)
SI_BASIS_FRACTION = {"DZ": 2 / 8, "TZ": 2 / 12, "DZP": 2 / 13, "DZP+p": 2 / 16}
WATER_BASIS_FRACTION = {"DZ+d": 4 / 17, "DZP": 4 / 23, "TZP": 4 / 29}


def batch_recipe(i: int):
    """(builder, kwargs) of instance i of the uneven batch.

    m ~ U[512, 4096] and a target occupied fraction ~ U[0.12, 0.25]; the basis is the one
    whose fraction is nearest the target, the cell the one whose m is nearest. Si for even
    i, water for odd i.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([4, i])))
    target = rng.uniform(512, 4096)
    frac = rng.uniform(0.12, 0.25)
    if i % 2 == 0:
        basis = min(SI_BASIS_FRACTION, key=lambda b: abs(SI_BASIS_FRACTION[b] - frac))
        per_cell = 8 * 2 / SI_BASIS_FRACTION[basis]   # orbitals per 8-atom cubic cell
        ncell = min(SI_CELL_SHAPES, key=lambda c: abs(per_cell * c - target))
        return silicon, dict(k=SI_CELL_SHAPES[ncell], basis=basis,
                             name=f"batch{i:02d}_si{8 * ncell}_{basis}")
    basis = min(WATER_BASIS_FRACTION, key=lambda b: abs(WATER_BASIS_FRACTION[b] - frac))
    nmol = int(np.clip(round(target * WATER_BASIS_FRACTION[basis] / 4.0), 18, 241))
    return water, dict(nmol=nmol, basis=basis, name=f"batch{i:02d}_water{nmol}_{basis}")


def batch_instance(i: int) -> Problem:
    """Instance i of the uneven batch (see batch_recipe), gap-guarded."""
    builder, kw = batch_recipe(i)
    return _gap_guarded(builder, i, **kw)


def batch_instances(indices, workers=None) -> list:
    """batch_instance(i) for every i in indices, built by a pool of worker processes.

    The workers are started with the "spawn" method (never forked from a process that may
    already hold a GPU context) and with one BLAS thread each; the result is the list of
    problems in the order of `indices`, the same bits as building them one by one.
    """
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    indices = list(indices)
    workers = workers or min(len(indices), max(1, (os.cpu_count() or 2) // 2), 16)
    if workers <= 1 or len(indices) <= 1:
        return [batch_instance(i) for i in indices]
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        # a worker that dies raises BrokenProcessPool here instead of leaving the map waiting
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
            return list(pool.map(batch_instance, indices))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def si4096_sz(seed=0) -> Problem:
    """Si4096 single-zeta: m = 16384, n = 8192 (the warm-start sequence's H_0)."""
    return _gap_guarded(silicon, seed, k=(8, 8, 8), basis="SZ", name="si4096_sz")


def warm_start_delta(p: Problem, k: int, sigma: float = JITTER_SIGMA) -> np.ndarray:
    """Symmetric on-site perturbation delta (diagonal, seeded) for H_k = H_0 + k * delta."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([5, p.seed])))
    return rng.normal(0.0, sigma, size=p.m)


NAMED = {"si64_sz": si64_sz, "si512_dzp": si512_dzp, "water256_dzp": water256_dzp}
