"""The ladder entry point that allocates nothing (lrcc_ladder_noalloc), called
through the C ABI and compared with the context-based lrcc_ladder_dev.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test.  It must also pass alone in a fresh
process: the first call on the device sets up the scratch address."""
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


def _antisym(R, O, V, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(R, O, O, V, V, dtype=torch.complex128, device="cuda", generator=g)
    x = x - x.transpose(1, 2)
    return x - x.transpose(3, 4)


def test_noalloc_matches_context_ladder_twice(L):
    O, V, Lx, R = 5, 19, 30, 3
    s = synth.make_system(O, V, Lx, seed=21)
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V)
    bvv = torch.as_tensor(np.ascontiguousarray(s["B"][:, O:, O:])).cuda()
    # two calls in a row on the shared scratch, different inputs and both directions
    for call, (seed, transpose) in enumerate([(1, False), (2, True)]):
        x = _antisym(R, O, V, seed)
        ref = L.lrcc_ladder_dev(ctx, x, transpose=transpose)
        got = L.lrcc_ladder_noalloc(bvv, x, transpose=transpose)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item()
        assert err < 1e-13 * ref.abs().max().item(), (call, err)


def _slab_count(O, V, R):
    """Slabs of a over which the entry point cuts <ab|ef>, by the rule stated
    in include/lrcc.h: after the packed X and Z (2 P_V R P_O complex), the
    32 MiB scratch holds G and W rows of as many a values as fit."""
    cap = (32 << 20) // 16
    po, pv = O * (O - 1) // 2, V * (V - 1) // 2
    per_a = V * (V - 1) * V + (V - 1) * pv
    na = min(V - 1, (cap - 2 * pv * R * po) // per_a)
    return -(-(V - 1) // na)


def test_noalloc_several_slabs_and_no_allocation(L):
    """A size that needs several slabs of the scratch array (a0 > 0 offsets into
    B_vv, W and Z), both directions, against the context ladder; and a second
    call with the output given changes neither the device's free memory nor
    PyTorch's allocated bytes."""
    O, V, Lx, R = 4, 60, 40, 2
    assert _slab_count(O, V, R) >= 5
    s = synth.make_system(O, V, Lx, seed=23)
    ctx = L.lrcc_setup(s["eps"], s["B"], s["mu"], O, V)
    bvv = torch.as_tensor(np.ascontiguousarray(s["B"][:, O:, O:])).cuda()
    for seed, transpose in [(3, False), (4, True)]:
        x = _antisym(R, O, V, seed)
        ref = L.lrcc_ladder_dev(ctx, x, transpose=transpose)
        got = L.lrcc_ladder_noalloc(bvv, x, transpose=transpose)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item()
        assert err < 1e-13 * ref.abs().max().item(), (transpose, err)
    out = torch.empty_like(x)
    L.lrcc_ladder_noalloc(bvv, x, out=out)      # warm-up: the first call may load the module
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    L.lrcc_ladder_noalloc(bvv, x, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_oversized_problem(L):
    """Sizes whose packed amplitudes alone (2 x 19900 x 8 x 435 complex) exceed
    the fixed scratch are refused before any kernel runs or pointer is read."""
    import ctypes
    small = torch.zeros(16, dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(small.data_ptr())
    lib = L.library()
    st = lib.lrcc_ladder_noalloc(p, 4, 30, 200, 8, p, p, 0, ctypes.c_void_p(0))
    assert st == L.LRCC_EINVAL
    assert "MiB of scratch" in lib.lrcc_last_error(None).decode()
