"""The ladder at the largest virtual space (O=20, V=1200, L=1800, 12 right-hand
sides: ncol = 12 x 190 = 2280 packed columns, P_V = 719400), in the launch
configuration the ladder benchmark times (<ab||ef> assembled per call in
slabs).  The oracle cannot form the whole map at this size, so it computes
sampled outputs one by one: for a sampled row (a,b) it builds <ab||ef> for all
e<f from B (Eq. 39 notation: <ab|ef> = sum_L B^L_ae B^L_bf), and dots it with
sampled columns of the same packed input."""
import numpy as np
import pytest
import torch

import synth
from oracle import ccsd

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c5():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    cfg = synth.CONFIGS["c5"]
    O, V, Lx = cfg["O"], cfg["V"], cfg["L"]
    s = synth.make_system(O, V, Lx, cfg["seed"])
    ctx = lrcc.lrcc_setup(s["eps"], s["B"], s["mu"], O, V)
    R = len(cfg["comps"]) * len(cfg["omegas"])
    ncol, pv = R * (O * (O - 1) // 2), V * (V - 1) // 2
    xt = synth.random_packed(ncol, pv, seed=55)
    return lrcc, s, ctx, xt


def _sample_rows(V):
    """(a,b) rows: first, last, and rows at slab-chunk edges and in between."""
    return [(0, 1), (0, V - 1), (0, 640), (1, 641), (597, 598), (V - 2, V - 1)]


# Tolerances: the <ab|ef> products accumulate in FP32 over K = L = 1800 (one
# chain of 169 bf16x3 k-blocks, 676 MMA steps, each rounding at most 2^-24
# relative: <= 4.1e-5; TF32 113 k-blocks), the contraction in FP32 chains of
# 128 k-blocks summed in FP64 (<= 3.1e-5), plus the split representation
# (bf16x3: 2^-17 per operand, 3 cross products; TF32: 2^-11 per operand).
@pytest.mark.parametrize("prec,tol", [(2, 1e-4), (1, 5e-3)])
def test_ladder_c5_sampled(c5, prec, tol):
    L, s, ctx, xt = c5
    O, V = s["O"], s["V"]
    xd = torch.as_tensor(xt).cuda()
    zt = L.lrcc_ladder_packed_dev(ctx, xd, prec=prec)
    del xd
    cols = [0, 1, 777, xt.shape[0] - 1]
    B = torch.as_tensor(s["B"])
    vv = slice(O, O + V)
    eu, fu = np.triu_indices(V, 1)
    worst = 0.0
    for (a, b) in _sample_rows(V):
        w = ccsd.antisym_block(B, slice(O + a, O + a + 1), slice(O + b, O + b + 1), vv, vv)[0, 0].numpy()[eu, fu]
        ab = a * (2 * V - a - 1) // 2 + (b - a - 1)
        ref = xt[cols] @ w
        got = zt[cols, ab].cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        assert err < tol, ((a, b), err)
    print(f"prec {prec}: max sampled relative error {worst:.2e}")
