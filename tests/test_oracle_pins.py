"""Pins of the CPU oracle against what the theory fixes (no GPU needed).

Each check compares the oracle with something other than itself:
brute-force second quantisation, FCI and sum-over-states, closed forms,
polynomial exactness of finite differences, invariances.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import ccsd, fci, fns


def _herm(rng, n, s):
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return s * (g + g.conj().T)


def _random_x(lay, seed, scale):
    a = synth.random_amplitudes(lay.O, lay.V, 1, seed=seed, scale=scale)
    return lay.join(torch.as_tensor(a["t1"][0]), torch.as_tensor(a["t2u"][0]))


# --- P5: residual and energy against the determinant-space projection -------

@pytest.mark.parametrize("O,V,L,seed", [(2, 4, 6, 1), (3, 5, 12, 7), (4, 5, 9, 3)])
def test_residual_matches_bruteforce_projection(O, V, L, seed):
    """R_mu = <mu|e^-T H e^T|0> (Eq. 9-10) for random T and a non-canonical
    Hermitian Fock matrix, against the explicit determinant-space series."""
    s = synth.make_system(O, V, L, seed=seed)
    rng = np.random.default_rng(seed + 100)
    f = ccsd.fock_of(s) + _herm(rng, O + V, 0.05)
    model = ccsd.CCModel(ccsd.Hamiltonian(f, O, s["B"]))
    x = _random_x(model.lay, seed + 5, 0.2)
    t1, t2 = model.lay.full(x)
    R1, R2 = ccsd.residual_full(t1, t2, model.H)
    E = complex(ccsd.energy_full(t1, t2, model.H))
    Eb, R1b, R2b, _ = fci.cc_projections(f, s["B"], O, t1.numpy(), t2.numpy())
    scale = max(np.abs(R1b).max(), np.abs(R2b).max())
    assert np.abs(R1.numpy() - R1b).max() < 1e-13 * scale
    assert np.abs(R2.numpy() - R2b).max() < 1e-13 * scale
    assert abs(E - Eb) < 1e-13 * max(1.0, abs(Eb))


def test_one_body_residual_is_xi():
    """xi = <nu|e^-T A e^T|0> (Eq. 31): the residual with f -> A and no
    two-body part equals the brute-force projection of the one-body operator."""
    O, V = 3, 4
    s = synth.make_system(O, V, 5, seed=2)
    A = s["mu"][1]
    m = ccsd.dipole_model(s, 1)
    x = _random_x(m.lay, 8, 0.3)
    t1, t2 = m.lay.full(x)
    R1, R2 = ccsd.residual_full(t1, t2, m.H)
    zeroB = np.zeros_like(s["B"])
    _, R1b, R2b, _ = fci.cc_projections(A, zeroB, O, t1.numpy(), t2.numpy())
    assert np.abs(R1.numpy() - R1b).max() < 1e-13
    assert np.abs(R2.numpy() - R2b).max() < 1e-13


@pytest.mark.parametrize("mutation", ["real_driver", "transpose_ovvv", "flip_vvvo", "drop_pab"])
def test_bruteforce_detects_planted_mistakes(mutation, monkeypatch):
    """A plausible mistake planted in the oracle (the real-spinor driver
    <ij||ab>, a transposed operand, a sign, a dropped antisymmetriser) makes
    the brute-force pin fail, so the pin is sensitive to such errors."""
    O, V = 3, 4
    s = synth.make_system(O, V, 6, seed=4)
    rng = np.random.default_rng(9)
    f = ccsd.fock_of(s) + _herm(rng, O + V, 0.05)
    H = ccsd.Hamiltonian(f, O, s["B"])
    if mutation == "real_driver":
        H.vvoo = H.oovv.permute(2, 3, 0, 1)
    elif mutation == "transpose_ovvv":
        H.ovvv = H.ovvv.transpose(2, 3).contiguous()
    elif mutation == "flip_vvvo":
        H.vvvo = -H.vvvo
    elif mutation == "drop_pab":
        monkeypatch.setattr(ccsd, "_Pab", lambda x: x)
    model = ccsd.CCModel(H)
    x = _random_x(model.lay, 3, 0.2)
    t1, t2 = model.lay.full(x)
    R1, R2 = ccsd.residual_full(t1, t2, model.H)
    _, R1b, R2b, _ = fci.cc_projections(f, s["B"], O, t1.numpy(), t2.numpy())
    err = max(np.abs(R1.numpy() - R1b).max(), np.abs(R2.numpy() - R2b).max())
    assert err > 1e-6


# --- P1: two electrons, CCSD is exact ---------------------------------------

def test_two_electron_ccsd_equals_fci_and_sos():
    cfg = synth.CONFIGS["c1b"]
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    model = ccsd.build(s)
    t, E, _ = ccsd.solve_ccsd(model)
    lam, _ = ccsd.solve_lambda(model, t)
    Efci, _, _, _, eref = fci.fci_states(ccsd.fock_of(s), s["B"], s["O"])
    assert abs(complex(E) - (Efci[0] - eref)) < 1e-10
    oms = list(cfg["omegas"])
    a_lr = ccsd.polarizability(s, (0, 1, 2), oms, ground=(t, E, lam))
    a_sos, _, wmin = fci.sos_polarizability(ccsd.fock_of(s), s["B"], s["mu"], s["O"], (0, 1, 2), oms)
    assert max(oms) < wmin
    assert np.abs(a_lr - a_sos).max() < 1e-9 * np.abs(a_sos).max()


def test_pm_omega_form_equals_sos_for_two_electrons():
    """Eq. 36 (X(+w), X(-w), no Y) is exact for 2 electrons as well, and agrees
    with the Eq. 35 form there."""
    cfg = synth.CONFIGS["c1b"]
    s = synth.make_system(cfg["O"], cfg["V"], cfg["L"], cfg["seed"])
    oms = [0.0, 0.05]
    a36 = ccsd.polarizability_pm(s, (0, 1, 2), oms)
    sos, _, _ = fci.sos_polarizability(ccsd.fock_of(s), s["B"], s["mu"], s["O"], (0, 1, 2), oms)
    assert np.abs(a36 - sos).max() < 1e-9 * np.abs(sos).max()


def test_separable_four_electrons_exact_at_every_frequency():
    """Two non-interacting 2-electron fragments: CCSD is exact for each and
    size-extensive, so for the 4-electron whole E_CCSD = E_FCI and the LR-CCSD
    alpha (Eq. 35 and Eq. 36 forms) equals the exact sum over states of the
    whole at every frequency -- an exact answer for more than two electrons at
    omega != 0."""
    fa, fb = synth.make_system(2, 4, 6, seed=31), synth.make_system(2, 4, 5, seed=32)
    s = synth.two_fragment_system(fa, fb)
    f = ccsd.fock_of(s)
    model = ccsd.build(s)
    t, E, _ = ccsd.solve_ccsd(model)
    lam, _ = ccsd.solve_lambda(model, t)
    Efci, _, _, _, eref = fci.fci_states(f, s["B"], s["O"])
    assert abs(complex(E) - (Efci[0] - eref)) < 1e-10
    oms = [0.0, 0.03, 0.07]
    comps = (0, 1, 2)
    sos, _, wmin = fci.sos_polarizability(f, s["B"], s["mu"], s["O"], comps, oms)
    assert max(oms) < wmin
    # the construction: the whole's exact alpha is the sum of the fragments'
    sa, _, _ = fci.sos_polarizability(ccsd.fock_of(fa), fa["B"], fa["mu"], 2, comps, oms)
    sb, _, _ = fci.sos_polarizability(ccsd.fock_of(fb), fb["B"], fb["mu"], 2, comps, oms)
    assert np.abs(sos - (sa + sb)).max() < 1e-11 * np.abs(sos).max()
    a35 = ccsd.polarizability(s, comps, oms, ground=(t, E, lam))
    a36 = ccsd.polarizability_pm(s, comps, oms, ground=(t, E, lam))
    assert np.abs(a35 - sos).max() < 1e-9 * np.abs(sos).max()
    assert np.abs(a36 - sos).max() < 1e-9 * np.abs(sos).max()


def test_pm_omega_form_close_to_eq35_for_more_electrons():
    """For more than two electrons the two forms are different approximations;
    at omega = 0 both equal d^2E/dF^2 (the same number), at omega != 0 they
    differ only slightly."""
    s = synth.make_system(3, 7, 10, seed=14)
    a35 = ccsd.polarizability(s, (0, 2), [0.0, 0.05])
    a36 = ccsd.polarizability_pm(s, (0, 2), [0.0, 0.05])
    scale = np.abs(a35).max()
    assert np.abs(a36[0] - a35[0]).max() < 1e-9 * scale
    assert np.abs(a36[1] - a35[1]).max() < 1e-2 * scale


def test_noninteracting_response_closed_form():
    """Without two-electron terms T = 0 and alpha is the independent-particle
    sum over (i, a): A_ia B_ai/(d - w) + B_ia A_ai/(d + w), d = e_a - e_i.
    Checks both the determinant-space SOS and the LR-CC expression of Eq. 35."""
    O, V = 2, 5
    s = synth.make_system(O, V, 4, seed=6)
    s0 = dict(s)
    s0["B"] = np.zeros_like(s["B"])
    oms = [0.0, 0.1]
    comps = (0, 2)
    eps, mu = s["eps"], s["mu"]
    d = eps[O:][None, :] - eps[:O][:, None]
    ref = np.zeros((2, 2, 2), dtype=np.complex128)
    for wi, w in enumerate(oms):
        for a, A in enumerate(comps):
            for b, Bc in enumerate(comps):
                Aia, Aai = mu[A][:O, O:], mu[A][O:, :O].T
                Bia, Bai = mu[Bc][:O, O:], mu[Bc][O:, :O].T
                ref[wi, a, b] = np.sum(Aia * Bai / (d - w) + Bia * Aai / (d + w))
    sos, E0, _ = fci.sos_polarizability(ccsd.fock_of(s), s0["B"], mu, O, comps, oms)
    assert abs(E0 - eps[:O].sum()) < 1e-12
    assert np.abs(sos - ref).max() < 1e-12 * np.abs(ref).max()
    lr = ccsd.polarizability(s0, comps, oms)
    assert np.abs(lr - ref).max() < 1e-10 * np.abs(ref).max()


# --- P2: MP2 is the first Jacobi step ---------------------------------------

def test_first_iteration_is_mp2():
    O, V, L = 4, 9, 20
    s = synth.make_system(O, V, L, seed=3)
    model = ccsd.build(s)
    x1, E1 = ccsd.mp2(model)
    B, eps = s["B"], s["eps"]
    # closed form with the integrals built element by element
    e = 0.0
    for i in range(O):
        for j in range(O):
            for a in range(O, O + V):
                for b in range(O, O + V):
                    v = np.sum(B[:, a, i] * B[:, b, j]) - np.sum(B[:, a, j] * B[:, b, i])
                    e -= abs(v) ** 2 / (eps[a] + eps[b] - eps[i] - eps[j])
    e *= 0.25
    assert abs(complex(E1).imag) < 1e-15
    assert e < 0
    assert abs(complex(E1).real - e) < 1e-13 * abs(e)
    t1, _ = model.lay.split(x1)
    assert float(t1.abs().max()) == 0.0           # canonical reference: f_ai = 0
    assert abs(fns.mp2_energy(eps, B, O) - e) < 1e-13 * abs(e)


# --- derivatives: exact polynomial stencils, bilinear identity ---------------

def test_torch_complex_conventions():
    c = torch.tensor(0.3 - 0.7j, dtype=torch.complex128)
    z = torch.tensor([1.0 + 2.0j], dtype=torch.complex128)
    v = torch.tensor([0.5 + 0.25j], dtype=torch.complex128)
    f = lambda y: c * y * y
    _, j = torch.func.jvp(f, (z,), (v,))
    assert torch.allclose(j, 2 * c * z * v)
    _, g = torch.func.vjp(f, z)
    assert torch.allclose(g(v.conj())[0].conj(), 2 * c * z * v)


def _stencil(fun, x, d, h):
    return (-fun(x + 2 * h * d) + 8 * fun(x + h * d) - 8 * fun(x - h * d) + fun(x - 2 * h * d)) / (12 * h)


def test_jacobian_products_are_exact_derivatives():
    """R is a polynomial of degree <= 4 in t, so the 5-point stencil is exact
    for any step; A X (Eq. 30) must match it.  The bilinear identity
    u.(A^T l) = l.(A u) pins the transpose (left) product, and F X (Eq. 34)
    is the exact stencil of the Lagrangian gradient (degree <= 3)."""
    s = synth.make_system(3, 6, 10, seed=5)
    model = ccsd.build(s)
    t, _, _ = ccsd.solve_ccsd(model)
    u = _random_x(model.lay, 1, 0.3)
    lam = _random_x(model.lay, 2, 0.3)
    Au = model.jvp(t, u)
    for h in (0.5, 1.0):
        st = _stencil(model.R, t, u, h)
        assert float((Au - st).abs().max()) < 1e-13 * float(Au.abs().max())
    ATl = model.vjp(t, lam)
    lhs, rhs = complex(torch.sum(u * ATl)), complex(torch.sum(lam * Au))
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)
    FX = model.FX(t, lam, u)
    st = _stencil(lambda y: model.lagrangian_grad(y, lam), t, u, 0.5)
    assert float((FX - st).abs().max()) < 1e-12 * float(FX.abs().max())


# --- P3: finite field --------------------------------------------------------

def test_static_alpha_equals_finite_field():
    """g_AA(0) = d^2 E_CCSD/dF^2 with f -> f + F mu_A (orbital-unrelaxed),
    complex values, 5-point second difference with Richardson extrapolation."""
    s = synth.make_system(3, 8, 16, seed=11)
    _, P = ccsd.polarizability(s, (2,), [0.0], tol=1e-12, return_parts=True)
    X, Y = P["parts"][0.0]["X"][2], P["parts"][0.0]["Y"][2]
    g = complex(torch.sum(Y * P["xi"][2]) + torch.sum(P["eta"][2] * X))

    def d2(h):
        E = [complex(ccsd.field_energy(s, 2, k * h)) for k in (-2, -1, 0, 1, 2)]
        return (-E[0] + 16 * E[1] - 30 * E[2] + 16 * E[3] - E[4]) / (12 * h * h)

    rich = (16 * d2(1e-3) - d2(2e-3)) / 15
    assert abs(rich - g) < 1e-8 * abs(g)


# --- P4: integral symmetries --------------------------------------------------

def test_integral_symmetries():
    s = synth.make_system(3, 5, 7, seed=8)
    B, mu = s["B"], s["mu"]
    assert np.array_equal(B, B.conj().transpose(0, 2, 1))
    assert np.array_equal(mu, mu.conj().transpose(0, 2, 1))
    g = fci.full_antisym(B)
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() < 1e-15
    assert np.abs(g + g.transpose(0, 1, 3, 2)).max() < 1e-15
    assert np.abs(g - g.transpose(2, 3, 0, 1).conj()).max() < 1e-15
    # no real 8-fold symmetry for complex spinors
    assert np.abs(g - g.transpose(2, 1, 0, 3)).max() > 1e-3


# --- P6: FNS++ ----------------------------------------------------------------

def test_fnspp_untruncated_and_rotation_invariance():
    O, V = 3, 7
    s = synth.make_system(O, V, 16, seed=12)
    oms = [0.0, 0.05]
    a_full = ccsd.polarizability(s, (0, 1, 2), oms)
    new, occ, info = fns.truncate(s, True, V)
    a_tr = ccsd.polarizability(new, (0, 1, 2), oms)
    assert np.abs(a_full - a_tr).max() < 1e-10 * np.abs(a_full).max()
    # random (non-semicanonical) unitary virtual rotation: general-f path
    U = synth.random_unitary(V, 3)
    Uf = np.eye(O + V, dtype=np.complex128)
    Uf[O:, O:] = U
    s3 = dict(s)
    s3["B"] = np.einsum('pr,lpq,qs->lrs', Uf.conj(), s["B"], Uf)
    s3["mu"] = np.einsum('pr,cpq,qs->crs', Uf.conj(), s["mu"], Uf)
    f3 = Uf.conj().T @ ccsd.fock_of(s) @ Uf
    m3 = ccsd.CCModel(ccsd.Hamiltonian(f3, O, s3["B"]))
    t3, E3, _ = ccsd.solve_ccsd(m3)
    _, E0, _ = ccsd.solve_ccsd(ccsd.build(s))
    assert abs(complex(E3) - complex(E0)) < 1e-11


def test_fnspp_density_properties():
    O, V = 3, 9
    s = synth.make_system(O, V, 12, seed=13)
    M = fns.fnspp_density(s["eps"], s["B"], s["mu"], O)
    assert np.abs(M - M.conj().T).max() < 1e-15 * np.abs(M).max() * 10
    n, Vn = np.linalg.eigh(M)
    assert n.min() > -1e-14 * n.max()                     # PSD under the conj reading
    assert np.abs(M @ Vn - Vn * n).max() < 1e-12 * np.abs(n).max()
    # Abar equals xi^A at T1 = 0, T2 = MP2 (reading of Eq. 47-48)
    model = ccsd.build(s)
    x1, _ = ccsd.mp2(model)
    t2 = fns.mp2_doubles(s["eps"], s["B"], O)
    _, t2x = model.lay.full(x1)
    assert np.abs(t2 - t2x.numpy()).max() < 1e-14
    Hii, Haa = fns.hbar_diagonals(s["eps"], s["B"], O, t2)
    zero = np.zeros(V)
    A1, A2 = fns.first_order_amplitudes(s["eps"], s["B"], s["mu"][0], O, t2,
                                        np.zeros(O), zero + 1.0, 0.0)
    xi = ccsd.dipole_model(s, 0).R(x1)
    xi1, xi2 = model.lay.full(xi)
    d2 = 2.0  # Haa + Hbb - Hii - Hjj with Haa = 1, Hii = 0
    assert np.abs(A1 * 1.0 - xi1.numpy()).max() < 1e-14
    assert np.abs(A2 * d2 - xi2.numpy()).max() < 1e-14
    # trace of the kept subspace + discarded = trace(M)
    new, occ, info = fns.truncate(s, True, 4)
    assert abs(np.sum(occ) - np.trace(M).real) < 1e-14 * abs(np.trace(M))
    assert new["V"] == 4 and new["B"].shape == (12, O + 4, O + 4)
    Bn = new["B"]
    assert np.abs(Bn - Bn.conj().transpose(0, 2, 1)).max() < 1e-15


# --- FNS (Eq. 37-41) and FNS++ (Eq. 45) densities from the wave function ----

def _vv_density_bruteforce(psi, O, V, dets, index):
    """D_ab = <psi| a_b^+ a_a |psi>: the virtual block of the one-particle
    density whose eigenvectors are natural-spinor coefficients (columns)."""
    N = O + V
    D = np.zeros((V, V), dtype=np.complex128)
    for a in range(V):
        for b in range(V):
            h = np.zeros((N, N))
            h[O + b, O + a] = 1.0
            G = fci.one_body_matrix(h, dets, index)
            D[a, b] = psi.conj() @ (G @ psi)
    return D


@pytest.mark.parametrize("O,V,seed", [(2, 5, 3), (3, 4, 6)])
def test_fns_densities_equal_wavefunction_densities(O, V, seed):
    """Plain FNS: |Psi1> = 1/4 sum t_ij^ab |Phi_ij^ab> with MP2 doubles
    (Eq. 38-39); FNS++: |Psi1^A> = (T1^(1) + T2^(1))|Phi_0> with the Eq. 46
    amplitudes.  Their virtual densities, evaluated in the determinant space,
    equal the contracted forms of Eq. 40 and Eq. 45 (conjugate on the second
    amplitude)."""
    s = synth.make_system(O, V, 6, seed=seed)
    N = O + V
    dets, index = fci.determinants(N, O)
    ref = index[(1 << O) - 1]
    phi0 = np.zeros(len(dets), dtype=np.complex128)
    phi0[ref] = 1.0
    t2 = fns.mp2_doubles(s["eps"], s["B"], O)
    assert np.abs(t2).max() > 1e-3                        # a non-trivial check
    T = fci.cluster_matrix(np.zeros((O, V)), t2, O, dets, index)
    D = _vv_density_bruteforce(T @ phi0, O, V, dets, index)
    M = fns.mp2_density(s["eps"], s["B"], O)
    assert np.abs(M - D).max() < 1e-14 * np.abs(D).max() * 10
    assert np.abs(M - M.T).max() > 1e-6 * np.abs(M).max()  # complex: M differs from its transpose
    # FNS++ (Eq. 45): singles and doubles of each component, averaged
    Hii, Haa = fns.hbar_diagonals(s["eps"], s["B"], O, t2)
    Dpp = np.zeros((V, V), dtype=np.complex128)
    for c in range(3):
        t1p, t2p = fns.first_order_amplitudes(s["eps"], s["B"], s["mu"][c], O, t2, Hii, Haa, 0.03)
        Tp = fci.cluster_matrix(t1p, t2p, O, dets, index)
        Dpp += _vv_density_bruteforce(Tp @ phi0, O, V, dets, index) / 3.0
    Mpp = fns.fnspp_density(s["eps"], s["B"], s["mu"], O, 0.03)
    assert np.abs(Mpp - Dpp).max() < 1e-14 * np.abs(Dpp).max() * 10


def test_plain_fns_exact_when_doubles_span_a_subspace():
    """If only the virtuals in S couple to the occupied space (B^L_ai = 0 for
    a outside S), the MP2 doubles vanish outside S, the plain-FNS density has
    exactly |S| non-zero occupations, and keeping them reproduces the
    full-space MP2 energy (Eq. 51-52: Delta E_MP2 = 0)."""
    O, V, L = 3, 9, 10
    s = synth.make_system(O, V, L, seed=17)
    S = [0, 2, 3, 7]
    out = [a for a in range(V) if a not in S]
    B = s["B"].copy()
    for a in out:
        B[:, O + a, :O] = 0.0
        B[:, :O, O + a] = 0.0
    s = dict(s, B=B)
    new, occ, info = fns.truncate(s, True, len(S), density="mp2")
    assert occ[len(S) - 1] > 1e-8 and occ[len(S):].max() < 1e-15 * occ[0]
    e_full = fns.mp2_energy(s["eps"], B, O)
    e_tr = fns.mp2_energy(new["eps"], new["B"], O)
    assert abs(e_full) > 1e-4
    assert abs(e_full - e_tr) < 1e-13 * abs(e_full)
    assert np.allclose(np.sort(new["eps"][O:]), np.sort(s["eps"][O:][S]), rtol=0, atol=1e-13)
    # the FNS++ density also sees mu_vv, which mixes in virtuals outside S
    _, occ_pp, _ = fns.truncate(s, True, len(S))
    assert occ_pp[len(S):].max() > 1e-10


def test_plain_fns_untruncated_reproduces_full_alpha():
    O, V = 3, 6
    s = synth.make_system(O, V, 12, seed=4)
    oms = [0.0, 0.04]
    a_full = ccsd.polarizability(s, (0, 1, 2), oms)
    new, occ, _ = fns.truncate(s, True, V, density="mp2")
    a_tr = ccsd.polarizability(new, (0, 1, 2), oms)
    assert np.abs(a_full - a_tr).max() < 1e-10 * np.abs(a_full).max()


# --- MP2-level polarisability (Delta alpha_MP2 ingredient, Eq. 53-54) -------

def test_mp2_polarizability_is_determinant_sum_over_states():
    """The contracted form equals the sum over excited determinants k of
    conj(<k|Abar>) <k|Bbar> / (Dbar_k - w) + <k|Abar> conj(<k|Bbar>) / (Dbar_k + w),
    with |Abar> = (Abar_1 + Abar_2)|Phi_0> built in the determinant space and
    Dbar_k = sum of Hbar over the particles minus the holes of k."""
    O, V = 3, 4
    s = synth.make_system(O, V, 7, seed=19)
    comps, oms = (0, 2), [0.0, 0.07]
    got = fns.mp2_polarizability(s, comps, oms)
    N = O + V
    dets, index = fci.determinants(N, O)
    ref_det = (1 << O) - 1
    phi0 = np.zeros(len(dets), dtype=np.complex128)
    phi0[index[ref_det]] = 1.0
    t2 = fns.mp2_doubles(s["eps"], s["B"], O)
    Hii, Haa = fns.hbar_diagonals(s["eps"], s["B"], O, t2)
    H = np.concatenate([Hii, Haa])
    dk = np.array([sum(H[p] for p in range(N) if (d >> p) & 1 and p >= O)
                   - sum(H[p] for p in range(O) if not (d >> p) & 1) for d in dets])
    vec = {}
    for c in comps:
        a1, a2 = fns.perturbed_moments(s["eps"], s["B"], s["mu"][c], O, t2)
        vec[c] = fci.cluster_matrix(a1, a2, O, dets, index) @ phi0
    exc = np.arange(len(dets)) != index[ref_det]
    ref = np.zeros_like(got)
    for wi, w in enumerate(oms):
        for a, A in enumerate(comps):
            for b, Bc in enumerate(comps):
                x, y = vec[A][exc], vec[Bc][exc]
                ref[wi, a, b] = np.sum(x.conj() * y / (dk[exc] - w) + x * y.conj() / (dk[exc] + w))
    assert np.abs(ref).max() > 1e-2
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(got - got.conj().transpose(0, 2, 1)).max() < 1e-14 * np.abs(got).max()


def test_mp2_polarizability_noninteracting_limit_and_untruncated_basis():
    """Without two-electron terms it is the exact independent-particle alpha
    (determinant-space SOS); with every natural spinor kept the FNS rotation
    leaves it unchanged (Delta alpha_MP2 = 0)."""
    O, V = 2, 5
    s = synth.make_system(O, V, 4, seed=6)
    s0 = dict(s, B=np.zeros_like(s["B"]))
    comps, oms = (0, 1, 2), [0.0, 0.1]
    sos, _, _ = fci.sos_polarizability(ccsd.fock_of(s), s0["B"], s["mu"], O, comps, oms)
    got = fns.mp2_polarizability(s0, comps, oms)
    assert np.abs(got - sos).max() < 1e-12 * np.abs(sos).max()
    s2 = synth.make_system(3, 6, 9, seed=2)
    full = fns.mp2_polarizability(s2, comps, oms)
    for density in ("fnspp", "mp2"):
        new, _, _ = fns.truncate(s2, True, 6, density=density)
        assert np.abs(fns.mp2_polarizability(new, comps, oms) - full).max() < 1e-12 * np.abs(full).max()
        new, _, _ = fns.truncate(s2, True, 3, density=density)
        assert np.abs(fns.mp2_polarizability(new, comps, oms) - full).max() > 1e-6 * np.abs(full).max()


def _mutated_fns(old, new):
    """oracle.fns with one source edit (a planted mistake), as a fresh module namespace."""
    import inspect
    src = inspect.getsource(fns)
    assert src.count(old) == 1, old
    ns = {"__name__": "fns_planted"}
    exec(compile(src.replace(old, new), "fns_planted", "exec"), ns)
    return ns


@pytest.mark.parametrize("old,new", [
    ("np.einsum('ijac,ijbc->ab', t2, t2.conj())", "np.einsum('ijac,ijbc->ab', t2.conj(), t2)"),    # conj side
    ("return 0.5 * np.einsum('ijac,ijbc->ab'", "return 1.0 * np.einsum('ijac,ijbc->ab'"),            # lost 1/2
    ("np.einsum('ijac,ijbc->ab', t2, t2.conj())", "np.einsum('ijca,ijbc->ab', t2, t2.conj())"),    # index
    ("+ np.einsum('ia,ib->ab', t1p, t1p.conj())", "+ np.einsum('ia,ib->ab', t1p.conj(), t1p)"),    # FNS++ singles
])
def test_density_pin_detects_planted_mistakes(old, new, monkeypatch):
    ns = _mutated_fns(old, new)
    monkeypatch.setattr(fns, "mp2_density", ns["mp2_density"])
    monkeypatch.setattr(fns, "fnspp_density", ns["fnspp_density"])
    with pytest.raises(AssertionError):
        test_fns_densities_equal_wavefunction_densities(2, 5, 3)


@pytest.mark.parametrize("old,new", [
    ("out[wi, a, b] = s1 + 0.25 * s2", "out[wi, a, b] = s1 + 0.5 * s2"),                 # doubles weight
    ("np.sum(a1.conj() * b1 / (D1 - w)", "np.sum(a1 * b1.conj() / (D1 - w)"),            # conjugate side
    ("a2 * b2.conj() / (D2 + w))", "a2 * b2.conj() / (D2 - w))"),                         # sign of omega
    ("D1 = Haa[None, :] - Hii[:, None]", "D1 = Haa[None, :] + 0 * Hii[:, None]"),         # dropped Hbar_ii
])
def test_mp2_alpha_pin_detects_planted_mistakes(old, new, monkeypatch):
    ns = _mutated_fns(old, new)
    monkeypatch.setattr(fns, "mp2_polarizability", ns["mp2_polarizability"])
    with pytest.raises(AssertionError):
        test_mp2_polarizability_is_determinant_sum_over_states()


def test_hbar_diagonals_are_one_hole_and_one_particle_energies():
    """Eq. 49-50 from the wave function: with T = T2(MP2) and
    Hbar = e^-T H e^T built in the determinant spaces of N-1 and N+1
    electrons, Hbar_ii = -(<Phi_i|Hbar|Phi_i> - <Phi_0|Hbar|Phi_0>) for
    Phi_i = a_i Phi_0 and Hbar_aa = <Phi^a|Hbar|Phi^a> - <Phi_0|Hbar|Phi_0> for
    Phi^a = a_a^+ Phi_0 (real parts)."""
    O, V = 3, 4
    N = O + V
    s = synth.make_system(O, V, 6, seed=23)
    t2 = fns.mp2_doubles(s["eps"], s["B"], O)
    Hii, Haa = fns.hbar_diagonals(s["eps"], s["B"], O, t2)
    gA = fci.full_antisym(s["B"])
    h = fci.core_hamiltonian(ccsd.fock_of(s), gA, O)

    def hbar_diag(nel, det):
        dets, index = fci.determinants(N, nel)
        H = fci.hamiltonian_matrix(h, gA, dets, index)
        T = fci.cluster_matrix(np.zeros((O, V)), t2, O, dets, index)
        v = np.zeros(len(dets), dtype=np.complex128)
        v[index[det]] = 1.0
        ev, term = v.copy(), v.copy()
        for k in range(1, 4):                  # e^T v (T is nilpotent)
            term = T @ term / k
            ev = ev + term
        return (v.conj() @ H @ ev).real        # <v| e^-T = <v| (T only excites)

    ref = (1 << O) - 1
    e0 = hbar_diag(O, ref)
    hi = np.array([-(hbar_diag(O - 1, ref ^ (1 << i)) - e0) for i in range(O)])
    ha = np.array([hbar_diag(O + 1, ref | (1 << (O + a))) - e0 for a in range(V)])
    assert np.abs(Hii - s["eps"][:O]).max() > 1e-3     # the correlation shift is not negligible
    assert np.abs(hi - Hii).max() < 1e-12 * np.abs(Hii).max()
    assert np.abs(ha - Haa).max() < 1e-12 * np.abs(Haa).max()


@pytest.mark.parametrize("density", ["fnspp", "mp2"])
def test_truncation_from_vo_block_equals_full_factor(density):
    """The memory-light variant (only B^L_ai, drawn by synth.make_system_vo)
    gives the same occupations, semicanonical energies and MP2 energies as the
    full-factor truncation."""
    O, V, L, keep = 3, 9, 7, 4
    s = synth.make_system(O, V, L, seed=27)
    sv = synth.make_system_vo(O, V, L, seed=27)
    new, occ, _ = fns.truncate(s, True, keep, omega=0.02, density=density)
    r = fns.truncation_from_vo(sv["eps"], sv["Bvo"], sv["mu"], O, True, keep, omega=0.02, density=density)
    assert np.abs(r["occ"] - occ).max() < 1e-13 * occ[0]
    assert np.abs(r["eps_virt"] - new["eps"][O:]).max() < 1e-13
    e_full = fns.mp2_energy(s["eps"], s["B"], O)
    e_tr = fns.mp2_energy(new["eps"], new["B"], O)
    assert abs(r["e_mp2_full"] - e_full) < 1e-13 * abs(e_full)
    assert abs(r["e_mp2_trunc"] - e_tr) < 1e-13 * abs(e_full)
    assert 0.0 < r["gap"] <= 1.0
