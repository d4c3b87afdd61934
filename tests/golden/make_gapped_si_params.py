"""Find the first seeded sp3d5s* Si parameter draw whose bulk bands have a gap.

The paper models P delta layers in Si (Section III-B) with a published sp3d5s* Si parameter
set that is not available here; the workloads use seeded synthetic parameters instead.  A
draw is accepted when the two-atom bulk band structure (oracle) on the folded 16^3 k-grid has
a gap of at least 0.5 eV between bands 4 and 5.  This script calls only the oracle and the
seeded draws, and writes gapped_si_params.json next to itself.

    python tests/golden/make_gapped_si_params.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import bulk  # noqa: E402


def band_edges(p, n):
    ks = bulk.folded_wavevectors(n, n, n, synth.SI_A_NM)
    ev = np.array([np.linalg.eigvalsh(bulk.bulk_hk(p, k, synth.SI_A_NM)) for k in ks])
    return float(ev[:, 3].max()), float(ev[:, 4].min()), float(ev.min()), float(ev.max())


def main():
    for seed in range(10000):
        p = synth.draw_tb_params(seed, synth.SP3D5S, 1)
        vb, cb, lo, hi = band_edges(p, 4)
        if cb - vb < 0.5:
            continue
        vb, cb, lo, hi = band_edges(p, 16)
        if cb - vb >= 0.5:
            out = {"seed": seed, "E_v": vb, "E_c": cb, "gap": cb - vb, "band_min": lo, "band_max": hi,
                   "kgrid": "4*16^3 folded wave vectors"}
            path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gapped_si_params.json")
            with open(path, "w") as f:
                json.dump(out, f, indent=1)
            print(out)
            return


if __name__ == "__main__":
    main()
