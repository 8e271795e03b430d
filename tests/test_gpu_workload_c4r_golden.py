"""Full solves with the dynamic-spectrum system's occupied count and factor rank
(O=28, L=1200, seed 3) on a virtual space small enough for the full oracle
(V=60): ground state, Lambda, X, F X, Y and the 3x3 polarisability tensor at
both ends of that workload's frequency grid (omega = 0 and 0.15) through the C
ABI, against tests/golden/c4r_alpha.json (written by tests/golden/make_golden.py
c4r, which calls only the oracle).  FP64 and FP64-class (emulated) paths at
1e-9, the bf16x3 mixed path at 1e-6."""
import json
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c4r_alpha.json")


@pytest.fixture(scope="module")
def L():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    assert torch.cuda.is_available()
    return lrcc


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/c4r_alpha.json not written")
    g = json.load(open(GOLDEN))
    s = synth.make_system(g["O"], g["V"], g["L"], g["seed"])
    ref = np.array(g["alpha_re"]) + 1j * np.array(g["alpha_im"])
    return g, s, ref


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (3, 1e-9), (2, 1e-6)])
def test_c4r_energy_and_alpha_against_oracle(L, golden, prec, tol):
    g, s, ref = golden
    o = L.lrcc_default_options()
    o.prec = prec
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], s["O"], s["V"], o)
    e, _, _ = L.lrcc_ccsd_ground(ctx)
    e_ref = complex(*g["E_corr"])
    assert abs(e - e_ref) < 1e-9 * abs(e_ref)
    a, err = L.lrcc_solve(ctx, g["omegas"], g["comps"])
    assert a.shape == ref.shape
    assert np.abs(a - ref).max() < tol * np.abs(ref).max()
    assert err.max() < 1e-8
