"""Write sampled outputs of the two residual maps -- sigma = A X (Eq. 30) and
the transpose product A^T lambda -- at the dynamic-spectrum workload's size
(O=28, V=600, L=1200, seed 3), where no full oracle residual fits in memory.

Linearisation point: the MP2 amplitudes (t1 = 0, t2 of Eq. 39).  X is the
seeded right-hand side synth.random_amplitudes(..., seed=2000).  The rows are
every singles (i, a) and unique doubles (i<j, a<b) with i, j in a seeded set So
of 6 occupied and a, b in a seeded set Sv of 8 virtual spinors (48 + 420 rows),
computed by oracle.sampled (the residual restricted to those rows, integral
slices formed from B).  lambda is a seeded complex vector on the same rows and
zero elsewhere; A^T lambda is then exact in every coordinate, and the file keeps
its values on the rows plus 300 random singles and 600 random unique doubles.

Calls only oracle/ (and the seeded generator); nothing here comes from the
CUDA path.  Usage: python tests/golden/make_maps_c4.py -> tests/golden/maps_c4.json
(about 10 minutes and 40 GB of host memory).
"""
import gc
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402
from oracle import ccsd, fns, sampled  # noqa: E402


def main():
    cfg = synth.CONFIGS["c4"]
    O, V, L, seed = cfg["O"], cfg["V"], cfg["L"], cfg["seed"]
    t0 = time.time()
    s = synth.make_system(O, V, L, seed, with_mu=False)
    eps, B = s["eps"], s["B"]
    rng = np.random.default_rng(4004)
    so = np.sort(rng.choice(O, 6, replace=False))
    sv = np.sort(rng.choice(V, 8, replace=False))
    H = sampled.RowIntegrals(np.diag(eps).astype(np.complex128), O, B, so, sv)
    t2 = fns.mp2_doubles(eps, B, O)
    del s, B
    gc.collect()
    print(f"integrals and MP2 amplitudes: {time.time() - t0:.0f} s", flush=True)
    rm = sampled.RowModel(H)
    lay = rm.lay
    t = lay.vec(torch.zeros(O, V, dtype=ccsd.CT), torch.as_tensor(t2))
    del t2
    gc.collect()
    amp = synth.random_amplitudes(O, V, 1, seed=2000)
    x = lay.join(torch.as_tensor(amp["t1"][0]), torch.as_tensor(amp["t2u"][0]))
    del amp
    sig = rm.jvp(t, x).numpy()
    print(f"sigma rows: {time.time() - t0:.0f} s", flush=True)
    n_rows = sig.shape[0]
    lam = rng.standard_normal(n_rows) + 1j * rng.standard_normal(n_rows)
    g = rm.vjp(t, torch.as_tensor(lam)).resolve_conj().numpy()
    print(f"A^T lambda: {time.time() - t0:.0f} s", flush=True)
    sing, dbl = rm.rows()
    n1, pv = O * V, V * (V - 1) // 2
    pair = lambda p, q, n: p * (2 * n - p - 1) // 2 + (q - p - 1)
    row_idx = [i * V + a for i, a in sing] + [n1 + pair(i, j, O) * pv + pair(a, b, V) for i, j, a, b in dbl]
    extra = np.concatenate([np.sort(rng.choice(n1, 300, replace=False)),
                            np.sort(n1 + rng.choice(g.shape[0] - n1, 600, replace=False))])
    vidx = np.concatenate([np.asarray(row_idx), extra])
    out = dict(O=O, V=V, L=L, seed=seed, x_seed=2000, linearisation="MP2 (t1 = 0, t2 of Eq. 39)",
               so=so.tolist(), sv=sv.tolist(), rows=row_idx,
               sigma_re=sig.real.tolist(), sigma_im=sig.imag.tolist(),
               lam_re=lam.real.tolist(), lam_im=lam.imag.tolist(),
               vjp_index=vidx.tolist(), vjp_re=g[vidx].real.tolist(), vjp_im=g[vidx].imag.tolist(),
               sigma_max=float(np.abs(sig).max()), vjp_max=float(np.abs(g).max()),
               seconds=time.time() - t0,
               source="oracle.sampled RowModel.jvp / .vjp (complex128, CPU), rows So x Sv")
    path = os.path.join(ROOT, "tests", "golden", "maps_c4.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, f"({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
