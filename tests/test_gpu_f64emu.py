"""FP64-class products on the tensor cores (LRCC_FP64_EMULATED: 7 integer
slices of 6 bits per operand, exact FP32 chains, FP64 sums) through the C ABI:

* residual maps (sigma = A X, A^T Y) and the ladder against the FP64 SIMT path,
  on shapes large enough to take the tensor-core route (several tiles, ragged
  edges, split K);
* alpha from the emulated path against the oracle at the FP64 tolerance;
* the mixed modes with their FP64-accurate maps emulated (the default) and in
  FP64 SIMT, both within 1e-6 of the oracle.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import ccsd

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


def _antisym_x(R, O, V, seed, scale=0.05):
    g = np.random.default_rng(seed)
    x = g.standard_normal((R, O, O, V, V)) + 1j * g.standard_normal((R, O, O, V, V))
    x = x - x.transpose(0, 2, 1, 3, 4)
    x = scale * (x - x.transpose(0, 1, 2, 4, 3))
    t1 = scale * (g.standard_normal((R, O, V)) + 1j * g.standard_normal((R, O, V)))
    return t1, x


# Tolerance: each slice product is exact; what is dropped per product is below
# about 8 x 2^-42 (~2e-12) of max|A_row| max|B_col|, and the terms of a K-sum
# add such errors with random signs, so the relative error of a map stays
# near 1e-11 at these sizes (measured 1.3e-11); 1e-10 bounds it.
EMU_TOL = 1e-10


def test_maps_match_fp64(L):
    """sigma and A^T at the ground state: emulated vs FP64 SIMT."""
    O, V, Lx, R = 8, 60, 96, 4
    s = synth.make_system(O, V, Lx, seed=12)
    ctx = _ctx(L, s)
    L.lrcc_ccsd_ground(ctx)
    t1, t2 = _antisym_x(R, O, V, 3)
    x = torch.as_tensor(L.pack_amplitudes(t1, t2)).cuda()
    for kind in (L.LRCC_RES_SIGMA, L.LRCC_RES_VJP):
        ref = L.lrcc_residual_dev(ctx, kind, None, x, prec=L.LRCC_FP64)
        got = L.lrcc_residual_dev(ctx, kind, None, x, prec=L.LRCC_FP64_EMULATED)
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert err < EMU_TOL, (kind, err)


@pytest.mark.parametrize("slab_rows", [0, 9])
def test_ladder_matches_fp64(L, slab_rows):
    """Packed ladder, cached <ab||ef> and slab assembly, both directions."""
    O, V, Lx = 3, 41, 50
    s = synth.make_system(O, V, Lx, seed=13)
    ctx = _ctx(L, s, slab_rows=slab_rows)
    pv = V * (V - 1) // 2
    g = np.random.default_rng(4)
    for ncol in (1, 37, 300):
        xt = torch.as_tensor(g.standard_normal((ncol, pv)) + 1j * g.standard_normal((ncol, pv))).cuda()
        for tr in (False, True):
            ref = L.lrcc_ladder_packed_dev(ctx, xt, transpose=tr, prec=L.LRCC_FP64)
            got = L.lrcc_ladder_packed_dev(ctx, xt, transpose=tr, prec=L.LRCC_FP64_EMULATED)
            err = (got - ref).abs().max().item() / ref.abs().max().item()
            assert err < EMU_TOL, (ncol, tr, err)


def test_emulated_alpha_against_oracle(L):
    s = synth.make_system(5, 19, 30, seed=21)
    oms = [0.0, 0.04, 0.08]
    ref = ccsd.polarizability(s, (0, 1, 2), oms, tol=1e-11)
    ce = _ctx(L, s, x_tol=1e-9, prec=L.LRCC_FP64_EMULATED)
    L.lrcc_ccsd_ground(ce)
    ae, err = L.lrcc_solve(ce, oms, [0, 1, 2])
    assert np.abs(ae - ref).max() < 1e-9 * np.abs(ref).max()
    assert err.max() < 1e-9


@pytest.mark.parametrize("fp64_products", [0, 1])
def test_mixed_with_and_without_emulated_outer_maps(L, fp64_products):
    s = synth.make_system(5, 19, 30, seed=21)
    oms = [0.0, 0.05]
    ref = ccsd.polarizability(s, (0, 1, 2), oms, tol=1e-11)
    cm = _ctx(L, s, x_tol=1e-9, prec=L.LRCC_MIXED_BF16X3, fp64_products=fp64_products)
    L.lrcc_ccsd_ground(cm)
    am, err = L.lrcc_solve(cm, oms, [0, 1, 2])
    assert np.abs(am - ref).max() < 1e-6 * np.abs(ref).max()
    assert err.max() < 1e-9
