"""Write the exact band energies of the workloads (test infrastructure only).

At the minimum of the OMM functional the energy is E* = 2 sum_{i<=n} eps_i, the n lowest
generalised eigenvalues of H x = eps S x (Sec. 2.1, Eqs. 1 and 7-8). For the 64-instance batch
(m up to 4096) and the Si4096 warm-start sequence (m = 16384, H_k = H_0 + k diag(delta)) those
eigensolves take minutes on the host, so they are done once here, by the oracle's definition
(`oracle.exact`), and stored next to this script (with the single-problem workloads, whose
solves are quicker, so that the bench need not repeat them):

    named_exact.json             E*, HOMO, LUMO of the single-problem workloads (Si64, Si512,
                                 water256)
    batch64_exact.json           E*, HOMO, LUMO of each batch instance
    si4096_sequence_exact.json   E*, HOMO, LUMO of H_k, k = 0 .. K-1

Inputs come from `synth` (seeded, bit-identical on every machine up to the last bits of the
host's libm); nothing here touches the GPU library. Run from the repository root:

    python -m tests.golden.make_exact_energies [--named] [--batch] [--sequence K]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import exact  # noqa: E402
from synth import configs  # noqa: E402

CITATION = ("Sec. 2.1, Eqs. 1 and 7-8: the minimum of the OMM functional is the band energy "
            "E* = 2 sum_{i<=n} eps_i of the n lowest generalised eigenvalues of H x = eps S x; "
            "values from oracle.exact (LAPACK eigenvalues of the seeded synth inputs)")


def _energy(H, S, n):
    import scipy.linalg
    w = scipy.linalg.eigh(H, S, eigvals_only=True, subset_by_index=[0, n])
    return 2.0 * float(np.sum(w[:n])), float(w[n - 1]), float(w[n])


def _write(path, doc):
    with open(path, "w") as fh:
        json.dump(doc, fh, indent=1, sort_keys=True)


def named(path=os.path.join(HERE, "named_exact.json")):
    doc = {"citation": CITATION, "workloads": {}}
    for name, builder in configs.NAMED.items():
        t0 = time.time()
        p = builder()
        ex = exact.exact_minimum(p.H, p.S, p.n, want_matrices=False)
        doc["workloads"][name] = {"m": p.m, "n": p.n, "seed": p.seed, "eta": p.eta, "E": ex["E"],
                                  "homo": ex["homo"], "lumo": ex["lumo"]}
        _write(path, doc)
        print(f"{name} m={p.m} n={p.n} E*={ex['E']:.12f} ({time.time() - t0:.1f} s)", flush=True)


def batch(path=os.path.join(HERE, "batch64_exact.json")):
    doc = {"citation": CITATION, "instances": []}
    for i in range(64):
        t0 = time.time()
        p = configs.batch_instance(i)
        ex = exact.exact_minimum(p.H, p.S, p.n, want_matrices=False)
        doc["instances"].append({"i": i, "name": p.name, "m": p.m, "n": p.n, "seed": p.seed, "eta": p.eta,
                                 "E": ex["E"], "homo": ex["homo"], "lumo": ex["lumo"]})
        _write(path, doc)
        print(f"{i:2d} {p.name} m={p.m} n={p.n} E*={ex['E']:.12f} ({time.time() - t0:.1f} s)", flush=True)


def sequence(K, path=os.path.join(HERE, "si4096_sequence_exact.json")):
    doc = {"citation": CITATION + "; H_k = H_0 + k diag(delta), delta = synth.configs.warm_start_delta(p, 1)",
           "steps": []}
    if os.path.exists(path):
        with open(path) as fh:
            doc["steps"] = json.load(fh)["steps"]
    p = configs.si4096_sz()
    delta = configs.warm_start_delta(p, 1)
    done = {s["k"] for s in doc["steps"]}
    H = p.H.copy()
    for k in range(K):
        if k in done:
            continue
        t0 = time.time()
        np.copyto(H, p.H)
        H[np.diag_indices(p.m)] += k * delta
        E, homo, lumo = _energy(H, p.S, p.n)
        doc["steps"].append({"k": k, "m": p.m, "n": p.n, "E": E, "homo": homo, "lumo": lumo})
        doc["steps"].sort(key=lambda s: s["k"])
        _write(path, doc)
        print(f"k={k} E*={E:.12f} gap={lumo - homo:.4f} ({time.time() - t0:.1f} s)", flush=True)


if __name__ == "__main__":
    if "--named" in sys.argv:
        named()
    if "--batch" in sys.argv:
        batch()
    if "--sequence" in sys.argv:
        sequence(int(sys.argv[sys.argv.index("--sequence") + 1]))
