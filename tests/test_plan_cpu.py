"""Host-only layout rules of the ladder (no GPU): the K panels of the
embedded tensor-core operands and the assembly chunks of the uncached
<ab||ef>, through the library's own planning code (lrcc_embed_layout,
lrcc_plan_slabs)."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2503_23144_gb300 import build, lrcc
    if not os.path.exists(lrcc._LIB_PATH):
        build.build()
    return lrcc


def _pv(V):
    return V * (V - 1) // 2


# K values of the workloads' embedded operands: P_V of V = 19 .. 1200, the
# auxiliary dimensions L, O*V of the ring, and sizes around the 16 KB panel
# boundary of both element types
KS = sorted({_pv(v) for v in (19, 60, 120, 300, 600, 1000, 1200)} | {48, 240, 1200, 1800, 2000}
            | {10 * 120, 20 * 1200} | {1365, 1366, 1367, 2047, 2048, 2049, 4095, 4096, 4097}
            | {int(k) for k in np.random.default_rng(0).integers(1, 3_000_000, 200)})


@pytest.mark.parametrize("prec,es,slots", [(2, 2, 6), (1, 4, 2)])
def test_embed_layout_rules(lib, prec, es, slots):
    pmax, kel, q = 16384 // es, 128 // es, 16 // es
    for K in KS:
        kd = slots * K
        for batch in (1, 3):
            n, w = lib.lrcc_embed_layout(prec, K, 100, batch)
            assert n >= 1 and n * w >= kd, (K, batch)
            if n == 1:
                assert w % q == 0 and w - kd < q, (K, batch)        # row padded to 16 bytes only
                assert batch > 1 or kd <= pmax or w <= pmax, K
            else:
                assert batch == 1
                assert w % kel == 0 and w <= pmax, K              # whole 128-byte k-blocks, <= 16 KB
                assert n == -(-kd // pmax), K                     # fewest panels
                assert (n - 1) * w < kd, K                        # the last panel holds data
            if batch > 1:
                assert n == 1
    with pytest.raises(lib.LrccError):
        lib.lrcc_embed_layout(0, 100, 10, 1)                      # FP64 has no embedded layout
    with pytest.raises(lib.LrccError):
        lib.lrcc_embed_layout(2, 0, 10, 1)


def _pairs(V):
    return {(a, b): k for k, (a, b) in enumerate((a, b) for a in range(V) for b in range(a + 1, V))}


@pytest.mark.parametrize("V", [2, 3, 7, 19, 60, 121])
def test_slab_plan_covers_every_pair_once(lib, V):
    idx = _pairs(V)
    for budget in (1, V * V, 7 * V * V, V ** 3, 10 * V ** 4):
        for row_cap in (0, 1, 5, 13):
            for cap_rows in (1, 128, 1000, 10 ** 9):
                plan = lib.lrcc_plan_slabs(V, budget, row_cap, cap_rows)
                row = 0
                for a0, a1, b0, b1, prow0, nrows, g in plan:
                    assert prow0 == row and nrows >= 1
                    rows = [idx[(a, b)] for a in range(a0, a1) for b in range(max(b0, a + 1), b1)]
                    assert rows == list(range(prow0, prow0 + nrows))
                    if a1 - a0 > 1:                               # several a per chunk: all their b
                        assert row_cap == 0 and b0 == a0 + 1 and b1 == V
                        assert (a1 - a0) * V * V * (V - a0 - 1) <= budget
                    if row_cap > 0:
                        assert a1 - a0 == 1 and b1 - b0 <= row_cap
                    elif a1 - a0 == 1 and (b0 > a0 + 1 or b1 < V):  # one a cut along b
                        assert (b1 - b0) * V * V <= max(budget, V * V)
                    row += nrows
                assert row == _pv(V)
                # groups: consecutive, within cap_rows unless one chunk exceeds it
                groups = plan[:, 6]
                assert groups[0] == 0 and np.all(np.diff(groups) >= 0) and np.all(np.diff(groups) <= 1)
                for gid in np.unique(groups):
                    sel = plan[groups == gid]
                    assert sel[:, 5].sum() <= cap_rows or len(sel) == 1
                    if gid + 1 <= groups.max():                 # greedy: the next chunk did not fit
                        nxt = plan[groups == gid + 1][0, 5]
                        assert sel[:, 5].sum() + nxt > cap_rows
    assert len(lib.lrcc_plan_slabs(120, 1 << 40, 0, 10 ** 9)) == 1    # everything in one chunk
    with pytest.raises(lib.LrccError):
        lib.lrcc_plan_slabs(1, 100, 0, 1)
