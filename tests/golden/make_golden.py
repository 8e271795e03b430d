"""Write oracle-computed expected values for the full-size parity tests.

Calls only oracle/ (and the seeded generator); nothing here comes from the
CUDA path.  Usage: python tests/golden/make_golden.py c2  -> tests/golden/c2_alpha.json
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
from oracle import ccsd  # noqa: E402


def main(name):
    cfg = synth.CONFIGS[name]
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    t0 = time.time()
    model = ccsd.build(s)
    t, E, itT = ccsd.solve_ccsd(model, tol=1e-11)
    lam, itL = ccsd.solve_lambda(model, t, tol=1e-11)
    print(f"ground done in {time.time() - t0:.0f} s: E = {complex(E)}", flush=True)
    comps, oms = list(cfg["comps"]), list(cfg["omegas"])
    alpha = ccsd.polarizability(s, comps, oms, tol=1e-10, ground=(t, E, lam))
    out = dict(config=name, O=cfg["O"], V=cfg["V"], L=cfg["L"], seed=cfg["seed"], comps=comps, omegas=oms,
               E_corr=[complex(E).real, complex(E).imag],
               alpha_re=np.real(alpha).tolist(), alpha_im=np.imag(alpha).tolist(),
               tolerances=dict(T=1e-11, Lambda=1e-11, X_Y=1e-10),
               seconds=time.time() - t0, threads=torch.get_num_threads(),
               source="oracle.ccsd.polarizability (complex128, CPU)")
    path = os.path.join(ROOT, "tests", "golden", f"{name}_alpha.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, f"({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "c2")
