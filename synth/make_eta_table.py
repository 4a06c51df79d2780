"""Write synth/eta_table.json: the HOMO/LUMO of each named workload.

The eigenspectrum shift of every workload is eta = HOMO + 0.1 Ha, which needs
one generalised eigensolve of the generated matrices. This script does those
solves once (scipy.linalg.eigh, host) so that building a workload later does
not repeat them. Run from the repository root:

    python -m synth.make_eta_table [--batch]
"""
from __future__ import annotations

import json
import sys

from . import configs


def main(argv):
    table = configs._load_table()

    def record(p):
        homo, lumo = configs.spectrum_edges(p.H, p.S, p.n)
        table[p.meta["table_key"]] = {"m": p.m, "n": p.n, "homo": homo, "lumo": lumo,
                                      "gap": lumo - homo}
        with open(configs._TABLE_PATH, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        print(p.meta["table_key"], p.m, p.n, "gap %.4f" % (lumo - homo), flush=True)
        return lumo - homo

    def guarded(builder, seed, **kw):
        for s in range(seed, seed + 20):
            p = builder(seed=s, need_eta=False, **kw)
            if record(p) >= configs.GAP_MIN:
                return

    guarded(configs.silicon, 0, k=(2, 2, 2), basis="SZ")
    guarded(configs.silicon, 0, k=(4, 4, 4), basis="DZP")
    guarded(configs.water, 0, nmol=256)
    if "--batch" in argv:
        import numpy as np
        for i in range(64):
            rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([4, i])))
            target = rng.uniform(512, 4096)
            if i % 2 == 0:
                ncell = min(configs.SI_CELL_SHAPES, key=lambda c: abs(104 * c - target))
                guarded(configs.silicon, i, k=configs.SI_CELL_SHAPES[ncell], basis="DZP")
            else:
                nmol = int(np.clip(round(target / 23.0), 23, 178))
                guarded(configs.water, i, nmol=nmol)


if __name__ == "__main__":
    main(sys.argv[1:])
