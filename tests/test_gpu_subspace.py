"""Shared-subspace solver (options.solver = 1) through the C ABI: every
right-hand side of a batch (all frequencies and components) is solved in one
subspace.  alpha (Eq. 35 and Eq. 36 forms) and the ground state against the
oracle at the FP64 tolerance, with FP64 and emulated-FP64 products, with the
automatic subspace and with one small enough to force restarts."""
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


SYS = dict(O=5, V=19, L=30, seed=21)
OMS = [0.0, 0.04, 0.08]


@pytest.fixture(scope="module")
def reference():
    s = synth.make_system(**SYS)
    model = ccsd.build(s)
    t, E, _ = ccsd.solve_ccsd(model, tol=1e-12)
    lam, _ = ccsd.solve_lambda(model, t, tol=1e-12)
    a = ccsd.polarizability(s, (0, 1, 2), OMS, tol=1e-11, ground=(t, E, lam))
    return s, complex(E), a


@pytest.mark.parametrize("prec,subspace_max", [(0, 0), (3, 0), (0, 24)])
def test_subspace_alpha_and_ground_state(L, reference, prec, subspace_max):
    s, E_ref, a_ref = reference
    c = _ctx(L, s, x_tol=1e-9, prec=prec, solver=1, subspace_max=subspace_max)
    E, _, _ = L.lrcc_ccsd_ground(c)
    assert abs(E - E_ref) < 1e-10 * abs(E_ref)
    a, err = L.lrcc_solve(c, OMS, [0, 1, 2])
    assert np.abs(a - a_ref).max() < 1e-9 * np.abs(a_ref).max()
    assert err.max() < 1e-9


def test_subspace_matches_diis_and_pm_omega(L, reference):
    s, _, a_ref = reference
    c_d = _ctx(L, s, x_tol=1e-10, pm_omega=1)
    L.lrcc_ccsd_ground(c_d)
    a_d, _ = L.lrcc_solve(c_d, OMS[1:], [0, 2])
    c_s = _ctx(L, s, x_tol=1e-10, pm_omega=1, solver=1)
    L.lrcc_ccsd_ground(c_s)
    a_s, _ = L.lrcc_solve(c_s, OMS[1:], [0, 2])
    assert np.abs(a_s - a_d).max() < 1e-9 * np.abs(a_d).max()


def test_subspace_too_small_is_rejected(L, reference):
    """subspace_max = 5 holds Lambda's single right-hand side but not a batch of 9."""
    s, _, _ = reference
    c = _ctx(L, s, solver=1, subspace_max=5)
    L.lrcc_ccsd_ground(c)
    with pytest.raises(L.LrccError) as e:
        L.lrcc_solve(c, OMS, [0, 1, 2])
    assert e.value.status == L.LRCC_EINVAL
