"""Failure detection without a GPU fault: the tensor-core GEMM's producer is
told (host-side switch) to skip its TMA copies, so the consumers' bounded
mbarrier waits run out.  The kernel raises the context's error word and
returns; the host reports LRCC_ETIMEOUT and the context stays usable."""
import os

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2503_23144_gb300 import build, lrcc
    build.build()
    return lrcc


def test_expired_wait_reports_timeout_and_context_survives(L):
    O, V = 4, 12
    s = synth.make_system(O, V, 10, seed=3)
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V)
    x = torch.randn(1, O, O, V, V, dtype=torch.complex128, device="cuda")
    x = x - x.transpose(1, 2)
    x = x - x.transpose(3, 4)
    ref = L.lrcc_ladder_dev(ctx, x, prec=L.LRCC_MIXED_BF16X3)
    os.environ["LRCC_INJECT_TMA_SKIP"] = "1"
    try:
        with pytest.raises(L.LrccError) as e:
            L.lrcc_ladder_dev(ctx, x, prec=L.LRCC_MIXED_BF16X3)
        assert e.value.status == L.LRCC_ETIMEOUT
    finally:
        del os.environ["LRCC_INJECT_TMA_SKIP"]
    again = L.lrcc_ladder_dev(ctx, x, prec=L.LRCC_MIXED_BF16X3)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
