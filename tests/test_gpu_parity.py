"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Sizes are chosen so that the oracle finishes in seconds while the GPU
contractions span several 64x64 tiles and ragged tails (odd O and V)."""
import numpy as np
import pytest
import torch

import synth
from oracle import ccsd, fci

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


def _rand(lay, R, seed, scale):
    a = synth.random_amplitudes(lay.O, lay.V, R, seed=seed, scale=scale)
    xs = [lay.join(torch.as_tensor(a["t1"][r]), torch.as_tensor(a["t2u"][r])) for r in range(R)]
    return xs


def _flat(lay, xs):
    t1 = np.stack([lay.split(x)[0].numpy() for x in xs])
    t2 = np.stack([lay.expand(lay.split(x)[1]).numpy() for x in xs])
    return t1, t2


def _unique(L, lay, flat):
    t1, t2 = L.unpack_amplitudes(flat, lay.O, lay.V)
    return [lay.join(torch.as_tensor(t1[r]), lay.pack(torch.as_tensor(t2[r]))) for r in range(flat.shape[0])]


SYS = dict(O=5, V=19, L=30, seed=21)


@pytest.fixture(scope="module")
def small(L):
    s = synth.make_system(**SYS)
    model = ccsd.build(s)
    return s, model, _ctx(L, s)


def test_residual_and_energy_parity(L, small):
    s, model, ctx = small
    lay = model.lay
    xs = _rand(lay, 2, 3, 0.1)
    t1, t2 = _flat(lay, xs)
    out = L.lrcc_residual(ctx, L.LRCC_RES_T, None, L.pack_amplitudes(t1, t2))
    E = L.lrcc_residual(ctx, L.LRCC_RES_ENERGY, None, L.pack_amplitudes(t1, t2))
    got = _unique(L, lay, out)
    for r, x in enumerate(xs):
        ref = model.R(x)
        assert float((got[r] - ref).abs().max()) < 1e-12 * float(ref.abs().max())
        e = complex(model.E(x))
        assert abs(E[r] - e) < 1e-13 * abs(e)
    # the doubles block of the output is antisymmetric
    _, r2 = L.unpack_amplitudes(out, lay.O, lay.V)
    assert np.abs(r2 + r2.transpose(0, 2, 1, 3, 4)).max() < 1e-14 * np.abs(r2).max()


def test_sigma_and_transpose_parity(L, small):
    s, model, ctx = small
    lay = model.lay
    t = _rand(lay, 1, 7, 0.1)[0]
    xs = _rand(lay, 3, 8, 0.3)
    tf = L.pack_amplitudes(*_flat(lay, [t]))[0]
    xf = L.pack_amplitudes(*_flat(lay, xs))
    sig = _unique(L, lay, L.lrcc_residual(ctx, L.LRCC_RES_SIGMA, tf, xf))
    vjp = _unique(L, lay, L.lrcc_residual(ctx, L.LRCC_RES_VJP, tf, xf))
    for r, x in enumerate(xs):
        ref = model.jvp(t, x)
        assert float((sig[r] - ref).abs().max()) < 1e-12 * float(ref.abs().max())
        ref = model.vjp(t, x)
        assert float((vjp[r] - ref).abs().max()) < 1e-12 * float(ref.abs().max())


def test_xi_parity(L, small):
    s, model, ctx = small
    lay = model.lay
    t = _rand(lay, 1, 9, 0.1)[0]
    tf = L.pack_amplitudes(*_flat(lay, [t]))[0]
    for comp in range(3):
        got = _unique(L, lay, L.lrcc_residual(ctx, L.LRCC_RES_XI, tf, tf[None], comp=comp))[0]
        ref = ccsd.dipole_model(s, comp).R(t)
        assert float((got - ref).abs().max()) < 1e-13 * float(ref.abs().max())


def test_ladder_parity(L, small):
    s, model, ctx = small
    O, V = s["O"], s["V"]
    lay = model.lay
    xs = _rand(lay, 3, 11, 1.0)
    _, x2 = _flat(lay, xs)
    vvvv = model.H.vvvv.numpy()
    ref = 0.5 * np.einsum('abef,rijef->rijab', vvvv, x2)
    refT = 0.5 * np.einsum('efab,rijef->rijab', vvvv, x2)
    xd = torch.as_tensor(x2).cuda()
    z = L.lrcc_ladder_dev(ctx, xd).cpu().numpy()
    zt = L.lrcc_ladder_dev(ctx, xd, transpose=True).cpu().numpy()
    assert np.abs(z - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(zt - refT).max() < 1e-13 * np.abs(refT).max()


def test_autograd_wrapper(L):
    s = synth.make_system(2, 3, 4, seed=5)
    ctx = _ctx(L, s)
    n = ctx.n_amp
    g = torch.Generator().manual_seed(0)
    t = (0.1 * torch.randn(n, dtype=torch.complex128, generator=g)).cuda().requires_grad_(True)
    F = L.ResidualFn()
    assert torch.autograd.gradcheck(lambda x: F.apply(ctx, x), (t,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_ground_state_and_alpha_c1(L):
    cfg = synth.CONFIGS["c1"]
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    oms = [0.0, 0.05]
    ref, P = ccsd.polarizability(s, (0, 1, 2), oms, tol=1e-11, return_parts=True)
    ctx = _ctx(L, s, r_tol=1e-11, x_tol=1e-10)
    E, itT, itL = L.lrcc_ccsd_ground(ctx)
    assert abs(E - complex(P["E"])) < 1e-11 * abs(E)
    alpha, err = L.lrcc_solve(ctx, oms, [0, 1, 2])
    assert np.abs(alpha - ref).max() < 1e-9 * np.abs(ref).max()
    assert err.max() < 1e-10


def test_two_electron_alpha_equals_sos(L):
    cfg = synth.CONFIGS["c1b"]
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    oms = list(cfg["omegas"])
    ctx = _ctx(L, s, r_tol=1e-12, x_tol=1e-11)
    E, _, _ = L.lrcc_ccsd_ground(ctx)
    Ef, _, _, _, eref = fci.fci_states(ccsd.fock_of(s), s["B"], s["O"])
    assert abs(E - (Ef[0] - eref)) < 1e-10
    alpha, _ = L.lrcc_solve(ctx, oms, [0, 1, 2])
    sos, _, _ = fci.sos_polarizability(ccsd.fock_of(s), s["B"], s["mu"], s["O"], (0, 1, 2), oms)
    assert np.abs(alpha - sos).max() < 1e-9 * np.abs(sos).max()


def test_separable_four_electrons_alpha_equals_sos(L):
    """Two non-interacting 2-electron fragments (4 electrons in all): E_CCSD
    and alpha at omega != 0 are exact, for Eq. 35 and Eq. 36."""
    fa, fb = synth.make_system(2, 4, 6, seed=31), synth.make_system(2, 4, 5, seed=32)
    s = synth.two_fragment_system(fa, fb)
    oms = [0.0, 0.03, 0.07]
    f = ccsd.fock_of(s)
    Ef, _, _, _, eref = fci.fci_states(f, s["B"], s["O"])
    sos, _, _ = fci.sos_polarizability(f, s["B"], s["mu"], s["O"], (0, 1, 2), oms)
    for pm in (0, 1):
        ctx = _ctx(L, s, r_tol=1e-12, x_tol=1e-11, pm_omega=pm)
        E, _, _ = L.lrcc_ccsd_ground(ctx)
        assert abs(E - (Ef[0] - eref)) < 1e-10
        alpha, _ = L.lrcc_solve(ctx, oms, [0, 1, 2])
        assert np.abs(alpha - sos).max() < 1e-9 * np.abs(sos).max(), pm


def test_rhs_chunking_invariance_and_state(L):
    s = synth.make_system(3, 9, 12, seed=4)
    ctx = _ctx(L, s)
    with pytest.raises(L.LrccError) as e:
        L.lrcc_solve(ctx, [0.0], [0])
    assert e.value.status == L.LRCC_ESTATE
    L.lrcc_ccsd_ground(ctx)
    a12, _ = L.lrcc_solve(ctx, [0.0, 0.03], [0, 1, 2])
    ctx2 = _ctx(L, s, rhs_chunk=4)
    L.lrcc_ccsd_ground(ctx2)
    a4, _ = L.lrcc_solve(ctx2, [0.0, 0.03], [0, 1, 2])
    assert np.abs(a12 - a4).max() < 1e-9 * np.abs(a12).max()


@pytest.mark.parametrize("prec,tol", [(1, 3e-3), (2, 1e-4)])
def test_ladder_tensor_core_vs_fp64(L, prec, tol):
    """Split-precision tcgen05 ladder (TF32, bf16x3) against the FP64 ladder on
    shapes with several M tiles, K pipelines longer than the stage ring, and
    ragged edges."""
    for (O, V, Lx, R, seed) in [(5, 19, 30, 3, 1), (6, 40, 64, 4, 2)]:
        s = synth.make_system(O, V, Lx, seed)
        ctx = _ctx(L, s)
        g = torch.Generator(device="cuda").manual_seed(seed)
        x = torch.randn(R, O, O, V, V, dtype=torch.complex128, device="cuda", generator=g)
        x = x - x.transpose(1, 2)
        x = x - x.transpose(3, 4)
        for tr in (False, True):
            z64 = L.lrcc_ladder_dev(ctx, x, transpose=tr)
            z = L.lrcc_ladder_dev(ctx, x, transpose=tr, prec=prec)
            assert (z - z64).abs().max().item() < tol * z64.abs().max().item()


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_alpha_within_1e6(L, prec):
    """Iterative refinement with tensor-core inner products: every alpha within
    1e-6 relative of the FP64 path (and of the oracle)."""
    s = synth.make_system(5, 19, 30, seed=21)
    oms = [0.0, 0.04, 0.08]
    ref = ccsd.polarizability(s, (0, 1, 2), oms, tol=1e-11)
    c64 = _ctx(L, s, x_tol=1e-9)
    L.lrcc_ccsd_ground(c64)
    a64, _ = L.lrcc_solve(c64, oms, [0, 1, 2])
    cm = _ctx(L, s, x_tol=1e-9, prec=prec, rhs_chunk=9)
    L.lrcc_ccsd_ground(cm)
    am, err = L.lrcc_solve(cm, oms, [0, 1, 2])
    n64, nmix = L.lrcc_solve_counts(cm)
    assert nmix > 0
    scale = np.abs(a64).max()
    assert np.abs(am - a64).max() < 1e-6 * scale
    assert np.abs(am - ref).max() < 1e-6 * scale
    assert np.abs(a64 - ref).max() < 1e-9 * scale


def test_amplitude_readback(L, small):
    s, model, ctx = small
    with pytest.raises(L.LrccError) as e:
        L.lrcc_get_amplitudes(ctx, 0)
    assert e.value.status == L.LRCC_ESTATE
    E, _, _ = L.lrcc_ccsd_ground(ctx)
    t = L.lrcc_get_amplitudes(ctx, 0)
    lam = L.lrcc_get_amplitudes(ctx, 1)
    lay = model.lay
    tu = _unique(L, lay, t[None])[0]
    assert float(model.R(tu).abs().max()) < 1e-9
    assert abs(complex(model.E(tu)) - E) < 1e-12 * abs(E)
    lu = _unique(L, lay, lam[None])[0]
    gE = model.lagrangian_grad(tu, torch.zeros_like(tu))
    assert float((model.vjp(tu, lu) + gE).abs().max()) < 1e-9


def test_pm_omega_form_parity_and_two_electron_sos(L):
    """Eq. 36 option (X(+w), X(-w), no Y) against the oracle, and exact for
    two electrons."""
    s = synth.make_system(4, 15, 20, seed=31)
    oms = [0.0, 0.045]
    ref = ccsd.polarizability_pm(s, (0, 1, 2), oms, tol=1e-11)
    ctx = _ctx(L, s, x_tol=1e-10, pm_omega=1)
    L.lrcc_ccsd_ground(ctx)
    a, _ = L.lrcc_solve(ctx, oms, [0, 1, 2])
    assert np.abs(a - ref).max() < 1e-9 * np.abs(ref).max()
    cfg = synth.CONFIGS["c1b"]
    s2 = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    c2 = _ctx(L, s2, r_tol=1e-12, x_tol=1e-11, pm_omega=1, prec=2)
    L.lrcc_ccsd_ground(c2)
    a2, _ = L.lrcc_solve(c2, list(cfg["omegas"]), [0, 1, 2])
    sos, _, _ = fci.sos_polarizability(ccsd.fock_of(s2), s2["B"], s2["mu"], s2["O"], (0, 1, 2), list(cfg["omegas"]))
    assert np.abs(a2 - sos).max() < 1e-9 * np.abs(sos).max()


def test_residual_hook_at_converged_ground_state(L, small):
    """t = NULL linearises at the converged T (cached primal): same maps as
    passing that T explicitly."""
    s, model, ctx = small
    lay = model.lay
    L.lrcc_ccsd_ground(ctx)
    t = L.lrcc_get_amplitudes(ctx, 0)
    xs = _rand(lay, 2, 5, 0.3)
    xf = L.pack_amplitudes(*_flat(lay, xs))
    for kind in (L.LRCC_RES_SIGMA, L.LRCC_RES_VJP):
        a = L.lrcc_residual(ctx, kind, None, xf)
        b = L.lrcc_residual(ctx, kind, t, xf)
        assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()
