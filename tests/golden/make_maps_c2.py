"""Write sampled outputs of the two maps the benchmark times -- sigma = A X
(Eq. 30) and the transpose product A^T X -- at the benchmark workload's size
(O=10, V=120, L=240): linearised at the MP2 amplitudes (one Jacobi step from
T = 0), applied to the benchmark's first right-hand side
(synth.random_amplitudes(..., seed=2000)).  Stores all 200 sampled singles and 600
sampled unique doubles (i<j, a<b) of each map, by unique index, with the
maps' largest magnitudes.

Calls only oracle/ (and the seeded generator); nothing here comes from the
CUDA path.  Usage: python tests/golden/make_maps_c2.py -> tests/golden/maps_c2.json
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


def main():
    cfg = synth.CONFIGS["c2"]
    O, V, L, seed = cfg["O"], cfg["V"], cfg["L"], cfg["seed"]
    t0 = time.time()
    s = synth.make_system(O, V, L, seed)
    model = ccsd.build(s)
    t, _ = ccsd.mp2(model)
    amp = synth.random_amplitudes(O, V, 1, seed=2000)
    X = model.lay.join(torch.as_tensor(amp["t1"][0]), torch.as_tensor(amp["t2u"][0]))
    sig = model.jvp(t, X).resolve_conj().numpy()
    vjp = model.vjp(t, X).resolve_conj().numpy()
    n1, n = O * V, sig.shape[0]
    rng = np.random.default_rng(77)
    idx = np.concatenate([np.sort(rng.choice(n1, 200, replace=False)),
                          np.sort(n1 + rng.choice(n - n1, 600, replace=False))])
    out = dict(O=O, V=V, L=L, seed=seed, x_seed=2000, linearisation="MP2 (one Jacobi step from T = 0)",
               index=idx.tolist(),
               sigma_re=sig[idx].real.tolist(), sigma_im=sig[idx].imag.tolist(),
               vjp_re=vjp[idx].real.tolist(), vjp_im=vjp[idx].imag.tolist(),
               sigma_max=float(np.abs(sig).max()), vjp_max=float(np.abs(vjp).max()),
               seconds=time.time() - t0, source="oracle.ccsd CCModel.jvp / .vjp (complex128, CPU)")
    path = os.path.join(ROOT, "tests", "golden", "maps_c2.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, f"({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
