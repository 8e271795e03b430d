"""Pins of the row-restricted oracle (oracle/sampled.py), which writes the
full-size golden samples at O=28, V=600: on systems where the full oracle runs,
its residual rows, the rows of A X (Eq. 30) and the transpose product A^T lambda
for a lambda supported on those rows equal the full oracle's (which is pinned by
brute-force projection in tests/test_oracle_pins.py), for a non-canonical Fock
matrix, non-zero singles and several row sets."""
import numpy as np
import pytest
import torch

import synth
from oracle import ccsd, sampled


def _system(O, V, L, seed):
    s = synth.make_system(O, V, L, seed)
    N = O + V
    rng = np.random.default_rng(seed + 100)
    f = np.diag(s["eps"]).astype(complex) + 0.05 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    return s, f


def _pick(lay, vec, sing, dbl):
    t1, t2 = lay.full(vec)
    return torch.cat([torch.stack([t1[i, a] for i, a in sing]), torch.stack([t2[i, j, a, b] for i, j, a, b in dbl])])


def _embed(lay, O, V, lam, sing, dbl):
    t1 = torch.zeros(O, V, dtype=torch.complex128)
    t2 = torch.zeros(O, O, V, V, dtype=torch.complex128)
    for k, (i, a) in enumerate(sing):
        t1[i, a] = lam[k]
    for k, (i, j, a, b) in enumerate(dbl):
        t2[i, j, a, b] = lam[len(sing) + k]
    return lay.vec(t1, t2)


@pytest.mark.parametrize("O,V,so,sv", [(5, 9, [0, 2, 3], [1, 4, 5, 8]), (4, 7, [0, 1, 2, 3], [0, 1, 2, 3, 4, 5, 6]),
                                       (6, 8, [1, 5], [2, 7])])
def test_rows_equal_full_oracle(O, V, so, sv):
    s, f = _system(O, V, 11, O * 10 + V)
    model = ccsd.CCModel(ccsd.Hamiltonian(f, O, s["B"]))
    lay = model.lay
    a = synth.random_amplitudes(O, V, 2, seed=5, scale=0.2)
    x = lay.join(torch.as_tensor(a["t1"][0]), torch.as_tensor(a["t2u"][0]))
    dx = lay.join(torch.as_tensor(a["t1"][1]), torch.as_tensor(a["t2u"][1]))
    rm = sampled.RowModel(sampled.RowIntegrals(f, O, s["B"], so, sv))
    sing, dbl = rm.rows()
    ref = _pick(lay, model.R(x), sing, dbl)
    assert float((rm.R(x) - ref).abs().max()) < 1e-13 * float(ref.abs().max())
    ref = _pick(lay, model.jvp(x, dx), sing, dbl)
    assert float((rm.jvp(x, dx) - ref).abs().max()) < 1e-13 * float(ref.abs().max())
    rng = np.random.default_rng(7)
    n = len(sing) + len(dbl)
    lam = torch.as_tensor(rng.standard_normal(n) + 1j * rng.standard_normal(n))
    ref = model.vjp(x, _embed(lay, O, V, lam, sing, dbl))
    got = rm.vjp(x, lam)
    assert float((got - ref).abs().max()) < 1e-13 * float(ref.abs().max())


def test_rows_detect_planted_mistake(monkeypatch):
    """A dropped term in the row residual (the T1-weighted <am||ef> piece of
    W_abef) makes the comparison with the full oracle fail."""
    O, V = 5, 9
    s, f = _system(O, V, 11, 59)
    model = ccsd.CCModel(ccsd.Hamiltonian(f, O, s["B"]))
    lay = model.lay
    a = synth.random_amplitudes(O, V, 1, seed=5, scale=0.2)
    x = lay.join(torch.as_tensor(a["t1"][0]), torch.as_tensor(a["t2u"][0]))
    H = sampled.RowIntegrals(f, O, s["B"], [0, 2, 3], [1, 4, 5, 8])
    H.vovv_v = torch.zeros_like(H.vovv_v)
    rm = sampled.RowModel(H)
    sing, dbl = rm.rows()
    ref = _pick(lay, model.R(x), sing, dbl)
    assert float((rm.R(x) - ref).abs().max()) > 1e-6 * float(ref.abs().max())
