"""Write synth/eta_table.json: the HOMO/LUMO of each named workload.

The eigenspectrum shift of every workload is eta = HOMO + 0.1 Ha, which needs
one generalised eigensolve of the generated matrices. This script does those
solves once (scipy.linalg.eigh, host) so that building a workload later does
not repeat them. Run from the repository root:

    python -m synth.make_eta_table [--batch] [--sequence] [--fresh]

--fresh starts from an empty table instead of updating the stored one.
"""
from __future__ import annotations

import json
import sys

from . import configs


def main(argv):
    table = {} if "--fresh" in argv else configs._load_table()

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
    if "--sequence" in argv:
        guarded(configs.silicon, 0, k=(8, 8, 8), basis="SZ")   # m = 16384: a long solve
    if "--batch" in argv:
        for i in range(64):
            builder, kw = configs.batch_recipe(i)
            kw.pop("name")
            guarded(builder, i, **kw)

if __name__ == "__main__":
    main(sys.argv[1:])
