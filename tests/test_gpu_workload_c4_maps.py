"""The residual maps at the dynamic-spectrum workload's full size (O=28, V=600,
L=1200) through the C ABI: sigma = A X (Eq. 30) on the seeded right-hand side
and A^T lambda for a lambda supported on sampled rows, linearised at the MP2
amplitudes, against tests/golden/maps_c4.json (written by
tests/golden/make_maps_c4.py, which calls only the oracle's row-restricted
residual).  The O V^3 integral blocks never exist on the device at this size;
the terms that read them run through the factor B and the slab-assembled Q map.

Precisions: FP64-class products on the tensor cores (emulated FP64, 1e-10 of the
map's largest element), bf16x3 (1e-4) and TF32 (3e-3), the tolerances of the
benchmark-size maps test.  Plain FP64 SIMT products are checked at the
benchmark size only: at this size one map takes about a quarter of an hour at
the GB300's FP64 rate."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from oracle import fns

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "maps_c4.json")


@pytest.fixture(scope="module")
def L():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    assert torch.cuda.is_available()
    return lrcc


def _expand(O, V, t2u):
    iu, ju = np.triu_indices(O, 1)
    au, bu = np.triu_indices(V, 1)
    x2 = np.zeros((O, O, V, V), dtype=np.complex128)
    I, J, A, B = iu[:, None], ju[:, None], au[None, :], bu[None, :]
    x2[I, J, A, B] = t2u
    x2[J, I, A, B] = -t2u
    x2[I, J, B, A] = -t2u
    x2[J, I, B, A] = t2u
    return x2


@pytest.fixture(scope="module")
def setup(L):
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/maps_c4.json not written")
    g = json.load(open(GOLDEN))
    O, V = g["O"], g["V"]
    s = synth.make_system(O, V, g["L"], g["seed"])
    t2 = fns.mp2_doubles(s["eps"], s["B"], O)
    t = L.pack_amplitudes(np.zeros((1, O, V)), t2[None])[0]
    del t2
    a = synth.random_amplitudes(O, V, 1, seed=g["x_seed"])
    x = L.pack_amplitudes(a["t1"], _expand(O, V, a["t2u"][0])[None])
    del a
    # lambda: the golden row values, zero elsewhere (unique -> full antisymmetric)
    n1, po, pv = O * V, O * (O - 1) // 2, V * (V - 1) // 2
    rows = np.array(g["rows"])
    lam = np.array(g["lam_re"]) + 1j * np.array(g["lam_im"])
    l1 = np.zeros(n1, dtype=np.complex128)
    l2u = np.zeros(po * pv, dtype=np.complex128)
    l1[rows[rows < n1]] = lam[rows < n1]
    l2u[rows[rows >= n1] - n1] = lam[rows >= n1]
    lamf = L.pack_amplitudes(l1.reshape(1, O, V), _expand(O, V, l2u.reshape(po, pv))[None])
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V)
    del s
    return g, t, x, lamf, ctx, L.lrcc_memory_stats(ctx)


def _unique(flat, idx, O, V):
    """values of a flat [n_amp] full-layout vector at unique indices"""
    n1, pv = O * V, V * (V - 1) // 2
    iu, ju = np.triu_indices(O, 1)
    au, bu = np.triu_indices(V, 1)
    out = np.empty(len(idx), dtype=np.complex128)
    s1 = idx < n1
    out[s1] = flat[idx[s1]]
    d = idx[~s1] - n1
    i, j, a, b = iu[d // pv], ju[d // pv], au[d % pv], bu[d % pv]
    out[~s1] = flat[n1 + ((i * O + j) * V + a) * V + b]
    return out


@pytest.mark.parametrize("prec,tol", [(3, 1e-10), (2, 1e-4), (1, 3e-3)])
def test_c4_maps_against_oracle(L, setup, prec, tol):
    g, t, x, lamf, ctx, _ = setup
    O, V = g["O"], g["V"]
    sig = L.lrcc_residual(ctx, L.LRCC_RES_SIGMA, t, x, prec=prec)[0]
    got = _unique(sig, np.array(g["rows"]), O, V)
    ref = np.array(g["sigma_re"]) + 1j * np.array(g["sigma_im"])
    err = np.abs(got - ref).max() / g["sigma_max"]
    assert err < tol, ("sigma", prec, err)
    del sig
    vj = L.lrcc_residual(ctx, L.LRCC_RES_VJP, t, lamf, prec=prec)[0]
    got = _unique(vj, np.array(g["vjp_index"]), O, V)
    ref = np.array(g["vjp_re"]) + 1j * np.array(g["vjp_im"])
    err = np.abs(got - ref).max() / g["vjp_max"]
    assert err < tol, ("vjp", prec, err)


def test_c4_no_buffer_of_ov3_size(L, setup):
    """After lrcc_setup, and after the maps above in all three precisions, no
    device buffer of the context was as large as a quarter of one complex
    O V^3 block (16 O V^3 bytes = 97 GB here): the three-virtual integrals are
    never stored, not even in their unique half (e<f)."""
    g, t, x, lamf, ctx, at_setup = setup
    O, V = g["O"], g["V"]
    block = 16 * O * V ** 3
    live, peak, largest = L.lrcc_memory_stats(ctx)
    print(f"setup: peak {at_setup[1] / 1e9:.1f} GB; maps: peak {peak / 1e9:.1f} GB, largest buffer {largest / 1e9:.1f} GB")
    assert at_setup[2] < block / 4, at_setup
    assert largest < block / 4, (live, peak, largest)
