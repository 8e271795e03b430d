"""The particle-particle ladder on packed amplitudes (lrcc_ladder_packed_dev)
and on full amplitudes (lrcc_ladder_dev), through the C ABI:

* FP64, with <ab||ef> cached and assembled per call in ragged slabs, against
  the oracle's <ab||ef> block (both directions; the transpose map is checked
  against <ef||ab> itself, not against a conjugate);
* the tensor-core precisions against the FP64 map, at widths that select every
  accumulator tile (32..256 columns) and shapes that split K.
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


def _wpacked(s):
    """<ab||ef> over the pairs a<b (rows) and e<f (columns), from the oracle."""
    model = ccsd.build(s)
    vvvv = model.H.vvvv.numpy()
    au, bu = np.triu_indices(s["V"], 1)
    return vvvv[au, bu][:, au, bu]


def _xt(ncol, pv, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ncol, pv)) + 1j * rng.standard_normal((ncol, pv))


SYS = dict(O=3, V=19, L=30, seed=5)
# 2*ncol real accumulator columns: 2 -> 32-wide tile, 48 -> 64, 120 -> 128, 400 -> 256
WIDTHS = (1, 24, 60, 200)


@pytest.fixture(scope="module")
def sys19():
    s = synth.make_system(**SYS)
    return s, _wpacked(s)


@pytest.mark.parametrize("slab_rows", [0, 5])
def test_packed_fp64_against_oracle(L, sys19, slab_rows):
    s, W = sys19
    pv = W.shape[0]
    ctx = _ctx(L, s, slab_rows=slab_rows)
    for ncol in WIDTHS:
        xt = _xt(ncol, pv, 100 + ncol)
        xd = torch.as_tensor(xt).cuda()
        for tr in (False, True):
            got = L.lrcc_ladder_packed_dev(ctx, xd, transpose=tr).cpu().numpy()
            ref = xt @ (W if not tr else W.T).T
            assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max(), (ncol, tr)


@pytest.mark.parametrize("prec,tol", [(1, 3e-3), (2, 1e-4)])
@pytest.mark.parametrize("slab_rows,herm", [(0, 0), (7, -1), (7, 1)])
def test_packed_tensor_core_vs_fp64(L, sys19, prec, tol, slab_rows, herm):
    """Cached <ab||ef>, and per-call assembly by whole rows (herm -1) or by the
    Hermitian half of each row group with the conjugate-transpose products
    (herm 1; groups of 21 rows, so the k-block boundary below each group's
    first column and the zeroed columns up to it are exercised)."""
    s, W = sys19
    pv = W.shape[0]
    ctx = _ctx(L, s, slab_rows=slab_rows, ladder_hermitian=herm)
    for ncol in WIDTHS:
        xd = torch.as_tensor(_xt(ncol, pv, 200 + ncol)).cuda()
        for tr in (False, True):
            z64 = L.lrcc_ladder_packed_dev(ctx, xd, transpose=tr)
            z = L.lrcc_ladder_packed_dev(ctx, xd, transpose=tr, prec=prec)
            assert (z - z64).abs().max().item() < tol * z64.abs().max().item(), (ncol, tr)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_full_layout_slab_path(L, prec):
    """lrcc_ladder_dev with <ab||ef> assembled per call in 6-row slabs, on a
    shape whose embedded K needs split-K and ragged tiles."""
    O, V, Lx, R = 4, 37, 50, 2
    s = synth.make_system(O, V, Lx, seed=8)
    vvvv = ccsd.build(s).H.vvvv.numpy()
    g = np.random.default_rng(3)
    x = g.standard_normal((R, O, O, V, V)) + 1j * g.standard_normal((R, O, O, V, V))
    x = x - x.transpose(0, 2, 1, 3, 4)
    x = x - x.transpose(0, 1, 2, 4, 3)
    ctx = _ctx(L, s, slab_rows=6)
    xd = torch.as_tensor(x).cuda()
    for tr in (False, True):
        ref = 0.5 * np.einsum('abef,rijef->rijab' if not tr else 'efab,rijef->rijab', vvvv, x)
        got = L.lrcc_ladder_dev(ctx, xd, transpose=tr, prec=prec).cpu().numpy()
        tol = {0: 1e-13, 1: 3e-3, 2: 1e-4}[prec]
        assert np.abs(got - ref).max() < tol * np.abs(ref).max(), tr


def test_packed_matches_full_layout(L, sys19):
    """The packed entry and the full-amplitude entry give the same map."""
    s, W = sys19
    O, V = s["O"], s["V"]
    ctx = _ctx(L, s)
    g = np.random.default_rng(9)
    x = g.standard_normal((2, O, O, V, V)) + 1j * g.standard_normal((2, O, O, V, V))
    x = x - x.transpose(0, 2, 1, 3, 4)
    x = x - x.transpose(0, 1, 2, 4, 3)
    iu, ju = np.triu_indices(O, 1)
    au, bu = np.triu_indices(V, 1)
    xt = x[:, iu, ju][:, :, au, bu].reshape(-1, len(au))
    for prec in (0, 2):
        zf = L.lrcc_ladder_dev(ctx, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
        zp = L.lrcc_ladder_packed_dev(ctx, torch.as_tensor(xt).cuda(), prec=prec).cpu().numpy()
        assert np.abs(zf[:, iu, ju][:, :, au, bu].reshape(zp.shape) - zp).max() < 1e-12 * np.abs(zp).max()


@pytest.mark.parametrize("prec,tol", [(1, 3e-3), (2, 1e-4)])
@pytest.mark.parametrize("slab_rows,herm", [(0, 0), (13, -1), (13, 1), (600, 1)])
def test_packed_long_rows_in_panels(L, prec, tol, slab_rows, herm):
    """V = 60: the embedded rows (6 P_V bf16 = 10 620 elements, 2 P_V TF32) are
    longer than one 16 KB panel, so <ab||ef> and X' are stored in K panels; with
    the Hermitian half (herm 1) the K ranges start inside panels, and a group of
    all 1770 rows (slab_rows 600) gives a conjugate-transpose operand whose rows
    (K = 1770: 21 KB in bf16x3) are stored in panels too."""
    s = synth.make_system(3, 60, 40, seed=14)
    ctx = _ctx(L, s, slab_rows=slab_rows, ladder_hermitian=herm)
    pv = 60 * 59 // 2
    for ncol in (5, 48):
        xd = torch.as_tensor(_xt(ncol, pv, 300 + ncol)).cuda()
        for tr in (False, True):
            z64 = L.lrcc_ladder_packed_dev(ctx, xd, transpose=tr)
            z = L.lrcc_ladder_packed_dev(ctx, xd, transpose=tr, prec=prec)
            assert (z - z64).abs().max().item() < tol * z64.abs().max().item(), (ncol, tr)


@pytest.mark.parametrize("prec,tol", [(1, 3e-3), (2, 1e-4)])
@pytest.mark.parametrize("slab_rows,herm", [(7, -1), (7, 1)])
def test_long_factor_rank_in_panels(L, prec, tol, slab_rows, herm):
    """L = 2100: the embedded factor rows of the <ab|ef> assembly products
    (6 L bf16 = 25 KB, 2 L TF32 = 16.8 KB) are longer than one 16 KB panel, so
    the cached B^L_bf operand is stored in K panels, and every slab after the
    first reads it from a row offset inside each panel (slabs of 7 rows)."""
    s = synth.make_system(2, 40, 2100, seed=16)
    ctx = _ctx(L, s, slab_rows=slab_rows, ladder_hermitian=herm)
    pv = 40 * 39 // 2
    for ncol in (3, 40):
        xd = torch.as_tensor(_xt(ncol, pv, 400 + ncol)).cuda()
        for tr in (False, True):
            z64 = L.lrcc_ladder_packed_dev(ctx, xd, transpose=tr)
            z = L.lrcc_ladder_packed_dev(ctx, xd, transpose=tr, prec=prec)
            assert (z - z64).abs().max().item() < tol * z64.abs().max().item(), (ncol, tr)
