"""FNS++ and plain-FNS truncation of the full-size FNS++ workload (O=16,
V=1000 -> 300 kept, L=2000, seed 2, static) on the GPU against the oracle's
values in tests/golden/fns_c3.json (written by tests/golden/make_fns_c3.py,
which calls only the oracle): all 1000 |occupations| and the MP2 energies of
Eq. 51 in the full and the truncated space."""
import json
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fns_c3.json")


@pytest.fixture(scope="module")
def L():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    assert torch.cuda.is_available()
    return lrcc


@pytest.fixture(scope="module")
def c3():
    g = json.load(open(GOLDEN))
    s = synth.make_system(g["O"], g["V"], g["L"], g["seed"])
    return g, s


@pytest.mark.parametrize("density,kind", [("fnspp", 0), ("mp2", 1)])
def test_full_size_truncation_against_oracle(L, c3, density, kind):
    g, s = c3
    r = g["results"][density]
    o = L.lrcc_default_options()
    o.fns_density = kind
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], s["O"], s["V"], o)
    vk, occ = L.lrcc_fns_truncate(ctx, True, g["keep"], omega=g["omega"])
    assert vk == g["keep"]
    occ_ref = np.array(r["occ"])
    assert np.abs(occ - occ_ref).max() < 1e-11 * occ_ref[0]
    ef, et, _ = L.lrcc_mp2_correction(ctx)
    ef_ref, et_ref = complex(*r["e_mp2_full"]), complex(*r["e_mp2_trunc"])
    assert abs(ef - ef_ref) < 1e-12 * abs(ef_ref)
    assert abs(et - et_ref) < 1e-10 * abs(ef_ref)
