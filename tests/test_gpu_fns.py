"""FNS++ and plain FNS truncation on the GPU (lrcc_fns_truncate) against the oracle."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from oracle import ccsd, fns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    assert torch.cuda.is_available()
    return lrcc


def _ctx(L, s, **kw):
    o = L.lrcc_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return L.lrcc_setup(s["eps"], s["B"], s["mu"], s["O"], s["V"], o)


def test_fnspp_truncated_alpha_and_occupations(L):
    s = synth.make_system(4, 31, 40, seed=2)
    keep, oms = 13, [0.0, 0.05]
    new, occ_ref, _ = fns.truncate(s, True, keep)
    a_ref = ccsd.polarizability(new, (0, 1, 2), oms, tol=1e-11)
    ctx = _ctx(L, s, x_tol=1e-10)
    with pytest.raises(L.LrccError):
        L.lrcc_mp2_correction(ctx)
    vk, occ = L.lrcc_fns_truncate(ctx, True, keep)
    assert vk == keep
    # MP2 correction of Eq. 51 against the oracle's MP2 energies in both bases
    ef, et, de = L.lrcc_mp2_correction(ctx)
    ef_ref = fns.mp2_energy(s["eps"], s["B"], 4)
    et_ref = fns.mp2_energy(new["eps"], new["B"], 4)
    assert abs(ef - ef_ref) < 1e-12 * abs(ef_ref)
    assert abs(et - et_ref) < 1e-12 * abs(ef_ref)
    assert abs(de - (ef_ref - et_ref)) < 1e-12 * abs(ef_ref)
    assert np.abs(occ - occ_ref).max() < 1e-12 * occ_ref.max()
    L.lrcc_ccsd_ground(ctx)
    a, _ = L.lrcc_solve(ctx, oms, [0, 1, 2])
    assert np.abs(a - a_ref).max() < 1e-9 * np.abs(a_ref).max()


def test_plain_fns_truncated_alpha_and_occupations(L):
    """Plain FNS (ground-state MP2 density, Eq. 40): occupations, MP2 energies
    and the truncated alpha against the oracle."""
    s = synth.make_system(4, 31, 40, seed=2)
    keep, oms = 13, [0.0, 0.05]
    new, occ_ref, _ = fns.truncate(s, True, keep, density="mp2")
    a_ref = ccsd.polarizability(new, (0, 1, 2), oms, tol=1e-11)
    ctx = _ctx(L, s, x_tol=1e-10, fns_density=1)
    vk, occ = L.lrcc_fns_truncate(ctx, True, keep)
    assert vk == keep
    assert np.abs(occ - occ_ref).max() < 1e-12 * occ_ref.max()
    ef, et, de = L.lrcc_mp2_correction(ctx)
    et_ref = fns.mp2_energy(new["eps"], new["B"], 4)
    assert abs(et - et_ref) < 1e-12 * abs(ef)
    L.lrcc_ccsd_ground(ctx)
    a, _ = L.lrcc_solve(ctx, oms, [0, 1, 2])
    assert np.abs(a - a_ref).max() < 1e-9 * np.abs(a_ref).max()


def test_fnspp_threshold_mode_and_frequency(L):
    s = synth.make_system(3, 24, 30, seed=5)
    thr, w = 2e-3, 0.03
    new, occ_ref, _ = fns.truncate(s, False, thr, omega=w)
    ctx = _ctx(L, s)
    vk, occ = L.lrcc_fns_truncate(ctx, False, thr, omega=w)
    assert vk == new["V"] == int(np.sum(occ_ref >= thr))
    assert np.abs(occ - occ_ref).max() < 1e-12 * occ_ref.max()


def test_fnspp_untruncated_reproduces_full_alpha(L):
    s = synth.make_system(3, 14, 20, seed=9)
    oms = [0.0, 0.06]
    c_full = _ctx(L, s, x_tol=1e-10)
    L.lrcc_ccsd_ground(c_full)
    a_full, _ = L.lrcc_solve(c_full, oms, [0, 1, 2])
    c_tr = _ctx(L, s, x_tol=1e-10)
    vk, _ = L.lrcc_fns_truncate(c_tr, True, 14)
    assert vk == 14
    L.lrcc_ccsd_ground(c_tr)
    a_tr, _ = L.lrcc_solve(c_tr, oms, [0, 1, 2])
    assert np.abs(a_tr - a_full).max() < 1e-10 * np.abs(a_full).max()


def test_fnspp_config3_recipe_reduced_size(L):
    """The FNS++ workload's recipe (O=16, seed 2, static, 3 components) at a
    virtual space the oracle handles: V=100 -> 30, mixed-precision solve."""
    s = synth.make_system(16, 100, 400, seed=2)
    keep = 30
    new, occ_ref, _ = fns.truncate(s, True, keep)
    a_ref = ccsd.polarizability(new, (0, 1, 2), [0.0], tol=1e-10)
    ctx = _ctx(L, s, prec=2)
    vk, occ = L.lrcc_fns_truncate(ctx, True, keep)
    assert vk == keep
    assert np.abs(occ - occ_ref).max() < 1e-11 * occ_ref.max()
    L.lrcc_ccsd_ground(ctx)
    a, _ = L.lrcc_solve(ctx, [0.0], [0, 1, 2])
    assert np.abs(a - a_ref).max() < 1e-6 * np.abs(a_ref).max()


def test_fnspp_large_virtual_space_v800(L):
    """V = 800 (V^2 beyond one wave of the element-wise kernels' capped grids):
    occupations and the truncated alpha against the oracle."""
    s = synth.make_system(3, 800, 6, seed=8)
    s["B"] = 0.05 * s["B"]   # weakly correlated: with L = 6 the recipe's integrals are large for 800 virtuals
    keep = 16
    new, occ_ref, _ = fns.truncate(s, True, keep)
    a_ref = ccsd.polarizability(new, (0, 2), [0.0], tol=1e-11)
    ctx = _ctx(L, s, x_tol=1e-10)
    vk, occ = L.lrcc_fns_truncate(ctx, True, keep)
    assert vk == keep
    assert np.abs(occ - occ_ref).max() < 1e-11 * occ_ref.max()
    L.lrcc_ccsd_ground(ctx)
    a, _ = L.lrcc_solve(ctx, [0.0], [0, 2])
    assert np.abs(a - a_ref).max() < 1e-9 * np.abs(a_ref).max()


def _golden_alpha(d):
    return np.array(d["re"]) + 1j * np.array(d["im"])


@pytest.mark.parametrize("name", ["o4v30", "o4v24_weak"])
def test_truncation_curves_against_oracle(L, name):
    """Every point of the oracle's plain-FNS and FNS++ truncation curves
    (alpha after keeping k natural spinors, and the MP2-level alpha of each
    truncated basis) and the untruncated values, through the GPU path."""
    path = os.path.join(os.path.dirname(__file__), "golden", f"fns_curve_{name}.json")
    g = json.load(open(path))
    sd = g["system"]
    s = synth.make_system(sd["O"], sd["V"], sd["L"], sd["seed"])
    s["B"] = sd["b_scale"] * s["B"]
    oms, comps = g["omegas"], g["comps"]
    full = _golden_alpha(g["full"])
    c = _ctx(L, s, x_tol=1e-10)
    m2 = L.lrcc_mp2_alpha(c, oms, comps)
    m2_ref = _golden_alpha(g["mp2_alpha_full"])
    assert np.abs(m2 - m2_ref).max() < 1e-12 * np.abs(m2_ref).max()
    L.lrcc_ccsd_ground(c)
    a, _ = L.lrcc_solve(c, oms, comps)
    assert np.abs(a - full).max() < 1e-9 * np.abs(full).max()
    for density, kind in (("fnspp", 0), ("mp2", 1)):
        for row in g["curves"][density]:
            ref = _golden_alpha(row["alpha"])
            ctx = _ctx(L, s, x_tol=1e-10, fns_density=kind)
            vk, occ = L.lrcc_fns_truncate(ctx, True, row["k"])
            assert vk == row["k"]
            assert abs(occ[vk - 1] - row["occ_kept_min"]) < 1e-12 * occ[0]
            m2 = L.lrcc_mp2_alpha(ctx, oms, comps)
            m2_ref = _golden_alpha(row["mp2_alpha"])
            assert np.abs(m2 - m2_ref).max() < 1e-10 * np.abs(m2_ref).max(), (density, row["k"])
            L.lrcc_ccsd_ground(ctx)
            a, _ = L.lrcc_solve(ctx, oms, comps)
            assert np.abs(a - ref).max() < 1e-9 * np.abs(ref).max(), (density, row["k"])


@pytest.mark.parametrize("density,kind", [("fnspp", 0), ("mp2", 1)])
def test_mp2_alpha_and_correction_against_oracle(L, density, kind):
    """lrcc_mp2_alpha (the Delta alpha_MP2 ingredient, Eq. 53-54) in the full
    canonical space and after truncation, against the oracle; a frequency
    above the lowest excitation energy is rejected."""
    s = synth.make_system(4, 31, 40, seed=2)
    comps, oms, keep = [0, 1, 2], [0.0, 0.05], 13
    ref_full = fns.mp2_polarizability(s, comps, oms)
    new, _, _ = fns.truncate(s, True, keep, density=density)
    ref_tr = fns.mp2_polarizability(new, comps, oms)
    ctx = _ctx(L, s, fns_density=kind)
    full = L.lrcc_mp2_alpha(ctx, oms, comps)
    assert np.abs(full - ref_full).max() < 1e-12 * np.abs(ref_full).max()
    L.lrcc_fns_truncate(ctx, True, keep)
    tr = L.lrcc_mp2_alpha(ctx, oms, comps)
    assert np.abs(tr - ref_tr).max() < 1e-10 * np.abs(ref_tr).max()
    # the correction itself (Eq. 54)
    assert np.abs((full - tr) - (ref_full - ref_tr)).max() < 1e-10 * np.abs(ref_full).max()
    with pytest.raises(L.LrccError) as e:
        L.lrcc_mp2_alpha(ctx, [50.0], comps)
    assert e.value.status == L.LRCC_EINVAL
