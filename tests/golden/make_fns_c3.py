"""Write the oracle's FNS++ and plain-FNS truncation of the full-size FNS++
workload (O=16, V=1000 -> 300 kept, L=2000, seed 2, static): the |occupation|
spectrum of all 1000 natural spinors, the semicanonical energies of the kept
300 and the MP2 energies of Eq. 51 in both spaces.

Calls only oracle/ (the block form of the truncation, which needs only the
virtual-occupied factor block) and the seeded generator; nothing here comes
from the CUDA path.  Usage: python tests/golden/make_fns_c3.py -> tests/golden/fns_c3.json
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import fns  # noqa: E402


def main():
    cfg = synth.CONFIGS["c3"]
    O, V, L, seed, keep = cfg["O"], cfg["V"], cfg["L"], cfg["seed"], cfg["keep"]
    t0 = time.time()
    sv = synth.make_system_vo(O, V, L, seed)
    print(f"generated in {time.time() - t0:.0f} s", flush=True)
    out = dict(O=O, V=V, L=L, seed=seed, keep=keep, omega=0.0, results={})
    for density in ("fnspp", "mp2"):
        r = fns.truncation_from_vo(sv["eps"], sv["Bvo"], sv["mu"], O, True, keep, density=density)
        out["results"][density] = dict(occ=r["occ"].tolist(), eps_virt=r["eps_virt"].tolist(),
                                       e_mp2_full=[float(np.real(r["e_mp2_full"])), float(np.imag(r["e_mp2_full"]))],
                                       e_mp2_trunc=[float(np.real(r["e_mp2_trunc"])),
                                                    float(np.imag(r["e_mp2_trunc"]))],
                                       gap_at_cut=float(r["gap"]))
        print(density, f"done at {time.time() - t0:.0f} s, gap at the cut {r['gap']:.3e}", flush=True)
    out["seconds"] = time.time() - t0
    out["source"] = "oracle.fns.truncation_from_vo (numpy complex128, CPU)"
    path = os.path.join(ROOT, "tests", "golden", "fns_c3.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


if __name__ == "__main__":
    main()
