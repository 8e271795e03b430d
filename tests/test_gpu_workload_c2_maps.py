"""The two maps the benchmark times -- sigma = A X (Eq. 30) and A^T X -- at
the benchmark workload's size (O=10, V=120, L=240) through the C ABI, in every
precision, against the oracle's sampled outputs in tests/golden/maps_c2.json
(written by tests/golden/make_maps_c2.py, which calls only the oracle): 200
singles and 600 unique doubles of each map, linearised at the MP2 amplitudes
and applied to the benchmark's first right-hand side."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from oracle import fns

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "maps_c2.json")


@pytest.fixture(scope="module")
def L():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    assert torch.cuda.is_available()
    return lrcc


@pytest.fixture(scope="module")
def setup(L):
    g = json.load(open(GOLDEN))
    O, V = g["O"], g["V"]
    s = synth.make_system(O, V, g["L"], g["seed"])
    # linearisation point: MP2 doubles, no singles (canonical reference)
    t2 = fns.mp2_doubles(s["eps"], s["B"], O)
    t = L.pack_amplitudes(np.zeros((1, O, V)), t2[None])[0]
    # the benchmark's first right-hand side, expanded to full antisymmetric doubles
    a = synth.random_amplitudes(O, V, 1, seed=g["x_seed"])
    iu, ju = np.triu_indices(O, 1)
    au, bu = np.triu_indices(V, 1)
    x2 = np.zeros((O, O, V, V), dtype=np.complex128)
    u = a["t2u"][0]
    I, J, A, B = iu[:, None], ju[:, None], au[None, :], bu[None, :]
    x2[I, J, A, B] = u
    x2[J, I, A, B] = -u
    x2[I, J, B, A] = -u
    x2[J, I, B, A] = u
    x = L.pack_amplitudes(a["t1"], x2[None])
    # unique index -> (singles flat index) or (i, j, a, b) of the full doubles
    idx = np.array(g["index"])
    n1, pv = O * V, len(au)
    dbl = idx[idx >= n1] - n1
    coords = (iu[dbl // pv], ju[dbl // pv], au[dbl % pv], bu[dbl % pv])
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V)
    return g, t, x, idx < n1, idx[idx < n1], coords, ctx


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 1e-10), (2, 1e-4), (1, 3e-3)])
def test_c2_maps_against_oracle(L, setup, prec, tol):
    g, t, x, is1, i1, coords, ctx = setup
    O, V = g["O"], g["V"]
    for kind, key in ((L.LRCC_RES_SIGMA, "sigma"), (L.LRCC_RES_VJP, "vjp")):
        out = L.lrcc_residual(ctx, kind, t, x, prec=prec)
        o1, o2 = L.unpack_amplitudes(out, O, V)
        got = np.concatenate([o1[0].reshape(-1)[i1], o2[0][coords]])
        ref = np.array(g[key + "_re"]) + 1j * np.array(g[key + "_im"])
        ref = np.concatenate([ref[is1], ref[~is1]])
        err = np.abs(got - ref).max() / g[key + "_max"]
        assert err < tol, (key, prec, err)
