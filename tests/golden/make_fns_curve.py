"""Write the oracle's truncation-error curves of plain FNS (ground-state MP2
density, Eq. 40) and FNS++ (perturbation-sensitive density, Eq. 45): the
polarisability tensor after keeping k natural spinors, for a range of k, next
to the untruncated one, with the MP2-level alpha of each basis (the
Delta alpha_MP2 ingredient, Eq. 53-54) -- a synthetic counterpart of the
paper's comparison of the two truncations and of the corrected curves
(Sec. III).

Calls only oracle/ (and the seeded generator); nothing here comes from the
CUDA path.  Usage: python tests/golden/make_fns_curve.py [o4v30|o4v24_weak]
-> tests/golden/fns_curve_<name>.json
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402
from oracle import ccsd, fns  # noqa: E402

# b_scale multiplies the generator's B (0.4: weakly correlated variant)
PRESETS = {
    "o4v30": dict(system=dict(O=4, V=30, L=40, seed=1, b_scale=1.0), omegas=[0.0, 0.05],
                  counts=[6, 9, 12, 15, 18, 21, 24, 27]),
    "o4v24_weak": dict(system=dict(O=4, V=24, L=40, seed=1, b_scale=0.4), omegas=[0.0, 0.05],
                       counts=[6, 10, 14, 18]),
}
TOL = 1e-11


def make(sd):
    s = synth.make_system(sd["O"], sd["V"], sd["L"], sd["seed"])
    s["B"] = sd["b_scale"] * s["B"]
    return s


def _pairs(a):
    return dict(re=np.real(a).tolist(), im=np.imag(a).tolist())


def main(name):
    p = PRESETS[name]
    t0 = time.time()
    sd, oms, counts = p["system"], p["omegas"], p["counts"]
    s = make(sd)
    comps = [0, 1, 2]
    full = ccsd.polarizability(s, comps, oms, tol=TOL)
    out = dict(system=sd, omegas=oms, comps=comps, counts=counts, tol_X_Y=TOL,
               full=_pairs(full), mp2_alpha_full=_pairs(fns.mp2_polarizability(s, comps, oms)), curves={})
    for density in ("fnspp", "mp2"):
        rows = []
        for k in counts:
            new, occ, _ = fns.truncate(s, True, k, density=density)
            a = ccsd.polarizability(new, comps, oms, tol=TOL)
            e_tr = fns.mp2_energy(new["eps"], new["B"], sd["O"])
            rows.append(dict(k=k, alpha=_pairs(a), occ_kept_min=float(occ[k - 1]),
                             e_mp2_trunc=[float(np.real(e_tr)), float(np.imag(e_tr))],
                             mp2_alpha=_pairs(fns.mp2_polarizability(new, comps, oms))))
            print(density, k, f"{time.time() - t0:.0f} s", flush=True)
        out["curves"][density] = rows
    e_full = fns.mp2_energy(s["eps"], s["B"], sd["O"])
    out["e_mp2_full"] = [float(np.real(e_full)), float(np.imag(e_full))]
    out["seconds"] = time.time() - t0
    out["threads"] = torch.get_num_threads()
    out["source"] = "oracle.fns.truncate, oracle.fns.mp2_polarizability, oracle.ccsd.polarizability (complex128, CPU)"
    path = os.path.join(ROOT, "tests", "golden", f"fns_curve_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "o4v30")
