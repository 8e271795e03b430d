"""Tensor-core contractions run as sub-GEMMs when their embedded operands
exceed the memory budget (options.embed_budget_mb), and lrcc_linearize fixes
the amplitudes at which the Jacobian maps of Eq. 30 are applied.

* With a 1 MiB budget every tensor-core contraction of sigma = A X and A^T Y is
  cut into halves along N, M and K (two-level index groups included) down to
  single tiles; the maps stay within the tolerance of their precision of the
  unsplit maps (emulated FP64 against FP64 SIMT at 1e-10; bf16x3 split against
  bf16x3 unsplit at 1e-5) on a system whose contractions span several tiles.
* lrcc_linearize(t) followed by maps with t = NULL equals the maps with t given.
"""
import numpy as np
import pytest
import torch

import synth

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


def _antisym(R, O, V, seed, scale):
    g = np.random.default_rng(seed)
    x = g.standard_normal((R, O, O, V, V)) + 1j * g.standard_normal((R, O, O, V, V))
    x = x - x.transpose(0, 2, 1, 3, 4)
    x = scale * (x - x.transpose(0, 1, 2, 4, 3))
    t1 = scale * (g.standard_normal((R, O, V)) + 1j * g.standard_normal((R, O, V)))
    return t1, x


@pytest.fixture(scope="module")
def system(L):
    O, V, Lx, R = 8, 60, 96, 3
    s = synth.make_system(O, V, Lx, seed=12)
    t = L.pack_amplitudes(*_antisym(1, O, V, 5, 0.05))[0]
    x = L.pack_amplitudes(*_antisym(R, O, V, 6, 0.3))
    return s, t, x


def test_split_maps_emulated_vs_fp64(L, system):
    s, t, x = system
    ref_ctx = _ctx(L, s)
    split_ctx = _ctx(L, s, embed_budget_mb=1)
    for kind in (L.LRCC_RES_SIGMA, L.LRCC_RES_VJP):
        ref = L.lrcc_residual(ref_ctx, kind, t, x, prec=L.LRCC_FP64)
        got = L.lrcc_residual(split_ctx, kind, t, x, prec=L.LRCC_FP64_EMULATED)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-10, (kind, err)


def test_split_maps_bf16x3_vs_unsplit(L, system):
    s, t, x = system
    a = _ctx(L, s, prec=L.LRCC_MIXED_BF16X3)
    b = _ctx(L, s, prec=L.LRCC_MIXED_BF16X3, embed_budget_mb=1)
    for kind in (L.LRCC_RES_SIGMA, L.LRCC_RES_VJP):
        ref = L.lrcc_residual(a, kind, t, x, prec=L.LRCC_MIXED_BF16X3)
        got = L.lrcc_residual(b, kind, t, x, prec=L.LRCC_MIXED_BF16X3)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-5, (kind, err)


def test_linearize_equals_explicit_point(L, system):
    s, t, x = system
    ctx = _ctx(L, s)
    with pytest.raises(L.LrccError) as e:
        L.lrcc_residual(ctx, L.LRCC_RES_SIGMA, None, x)
    assert e.value.status == L.LRCC_ESTATE
    L.lrcc_linearize(ctx, t)
    for kind in (L.LRCC_RES_SIGMA, L.LRCC_RES_VJP):
        ref = L.lrcc_residual(ctx, kind, t, x)
        got = L.lrcc_residual(ctx, kind, None, x)
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max(), kind
    # the ground state is not implied: lrcc_solve still refuses
    with pytest.raises(L.LrccError) as e:
        L.lrcc_solve(ctx, [0.0], [0])
    assert e.value.status == L.LRCC_ESTATE
