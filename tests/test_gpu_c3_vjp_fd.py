"""The hand-written transpose product of the residual (the vector-Jacobian
product behind the Lambda equations, Eq. 20, and the left response, Eq. 32)
checked by finite differences on the FNS++ workload after truncation (O=16,
V=1000 -> 300 kept, L=2000, seed 2), linearised at its converged ground state,
with lambda = the converged Lambda, through the C ABI:

* central differences with step h = 1e-6 and FP64 products,
  <lambda, [R(T + h d) - R(T - h d)] / (2h)> against <d, J^T lambda>, on 4
  random unit directions d, within 1e-7 of the largest of those values;
* the 5-point stencil, which is exact for the residual (a polynomial of degree
  4 in T), [R(T-2hd) - 8R(T-hd) + 8R(T+hd) - R(T+2hd)] / (12h), with FP64-class
  (emulated) products, on 64 random unit directions, within 1e-7 as well.

Dot products run over unique amplitudes (sum over singles + 1/4 sum over the
full antisymmetric doubles); directions have unit norm in that product."""
import numpy as np
import pytest
import torch

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def L():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    assert torch.cuda.is_available()
    return lrcc


def _udot(a, b, n1):
    return np.sum(a[..., :n1] * b[..., :n1], axis=-1) + 0.25 * np.sum(a[..., n1:] * b[..., n1:], axis=-1)


def _directions(L, O, V, n, seed):
    a = synth.random_amplitudes(O, V, n, seed=seed, scale=1.0)
    iu, ju = np.triu_indices(O, 1)
    au, bu = np.triu_indices(V, 1)
    out = []
    for r in range(n):
        x2 = np.zeros((O, O, V, V), dtype=np.complex128)
        u = a["t2u"][r]
        I, J, A, B = iu[:, None], ju[:, None], au[None, :], bu[None, :]
        x2[I, J, A, B] = u
        x2[J, I, A, B] = -u
        x2[I, J, B, A] = -u
        x2[J, I, B, A] = u
        d = L.pack_amplitudes(a["t1"][r][None], x2[None])[0]
        out.append(d / np.sqrt(abs(_udot(d, d, O * V))))
    return np.array(out)


@pytest.fixture(scope="module")
def c3_ground(L):
    cfg = synth.CONFIGS["c3"]
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    o = L.lrcc_default_options()
    o.prec = L.LRCC_MIXED_BF16X3
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], cfg["O"], cfg["V"], o)
    del s
    vk, _ = L.lrcc_fns_truncate(ctx, True, cfg["keep"])
    assert vk == cfg["keep"]
    L.lrcc_ccsd_ground(ctx)
    T = L.lrcc_get_amplitudes(ctx, 0)
    lam = L.lrcc_get_amplitudes(ctx, 1)
    return ctx, cfg["O"], vk, T, lam


def _fd_check(L, ctx, O, V, T, lam, dirs, h, stencil, prec):
    n1 = O * V
    g = L.lrcc_residual(ctx, L.LRCC_RES_VJP, T, lam[None], prec=L.LRCC_FP64)[0]   # J^T lambda
    ref = _udot(dirs, g[None], n1)
    coef = {2: [(1, 1.0), (-1, -1.0)], 4: [(-2, 1.0), (-1, -8.0), (1, 8.0), (2, -1.0)]}[stencil]
    den = 2.0 * h if stencil == 2 else 12.0 * h
    fd = np.zeros(len(dirs), dtype=np.complex128)
    for k0 in range(0, len(dirs), 8):
        blk = dirs[k0:k0 + 8]
        pts = np.concatenate([T[None] + m * h * blk for m, _ in coef])
        Rs = L.lrcc_residual(ctx, L.LRCC_RES_T, None, pts, prec=prec)
        proj = _udot(Rs, lam[None], n1).reshape(len(coef), len(blk))
        fd[k0:k0 + len(blk)] = sum(c * proj[q] for q, (_, c) in enumerate(coef)) / den
    return np.abs(fd - ref).max() / np.abs(ref).max()


def test_vjp_central_differences_h1e6_fp64(L, c3_ground):
    ctx, O, V, T, lam = c3_ground
    dirs = _directions(L, O, V, 4, seed=601)
    err = _fd_check(L, ctx, O, V, T, lam, dirs, 1e-6, 2, L.LRCC_FP64)
    assert err < 1e-7, err


def test_vjp_exact_stencil_64_directions(L, c3_ground):
    ctx, O, V, T, lam = c3_ground
    dirs = _directions(L, O, V, 64, seed=602)
    tn = np.sqrt(abs(_udot(T, T, O * V)))
    err = _fd_check(L, ctx, O, V, T, lam, dirs, 0.1 * tn, 4, L.LRCC_FP64_EMULATED)
    assert err < 1e-7, err
