"""Oracle: spin-orbital CCSD, left-CCSD and LR-CCSD in complex128 (test infrastructure).

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may use this module.  Everything is plain PyTorch CPU arithmetic in complex128.

Paper anchors (arXiv:2503.23144, Sec. II.A):

* amplitudes t_i^a, t_ij^ab (Eq. 3-5; T1 carries no 1/2, T2 carries 1/4),
* CCSD energy and residual  E = <0|Hbar|0>,  R_mu = <mu|Hbar|0>  (Eq. 9-10),
* Jacobian A_{mu nu} = <mu|[Hbar, tau_nu]|0> = dR_mu/dt_nu  (Eq. 30),
* xi_nu = <nu|Vbar|0>  (Eq. 31),  eta_nu = <(1+Lambda)|[Vbar, tau_nu]|0>  (Eq. 33),
* F_{nu gamma} = <(1+Lambda)|[[Hbar, tau_nu], tau_gamma]|0>  (Eq. 34),
* (A - omega) X = -xi  (Eq. 29),   Y (A + omega) = -(eta + F X)  (Eq. 32),
* <<A;B>> = 1/2 P(A,B) [Y^B . xi^A + eta^A . X^B],  alpha = -<<mu;mu>>  (Eq. 35).

The paper does not print the CCSD equations themselves.  The residual below is
the spin-orbital CCSD of Stanton, Gauss, Watts and Bartlett (J. Chem. Phys. 94,
4334 (1991)) written for a general, non-canonical Fock matrix, with the two
driver terms in their general complex form (<ab||ij> and f_ai, which equal
<ij||ab> and f_ia only for real spinors).  Every integral appears with its
creation (bra) indices first: <pq||rs> = <pq|rs> - <pq|sr>,
<pq|rs> = sum_L B^L_pr B^L_qs.  No conjugation appears anywhere in R or E; the
brute-force determinant-space residual in ``oracle.fci`` pins this.

Derivatives: R and E are polynomials in the amplitudes, so A X, A^T lambda and
F X are exact directional derivatives, taken here with ``torch.func`` on the
written-out residual.  PyTorch returns conj(J)^T v for reverse mode; the
holomorphic transpose J^T v that the Lambda and Y equations need is
conj(vjp(conj(v))).  Pinned by the 5-point polynomial stencil (exact for
degree <= 4) and the bilinear identity.

Amplitude vectors are flat: [t1 (O*V), t2 unique (P_O*P_V)] with the pairs
i<j, a<b in row-major order of the strict upper triangle.  Dot products over
amplitude vectors are unconjugated sums over these unique entries.
"""
from __future__ import annotations

import numpy as np
import torch

CT = torch.complex128
torch.set_default_dtype(torch.float64)


def as_c(x) -> torch.Tensor:
    return torch.as_tensor(np.asarray(x), dtype=CT)


# ----------------------------------------------------------------------------
# integrals
# ----------------------------------------------------------------------------

def coulomb_block(B: torch.Tensor, P, Q, R, S) -> torch.Tensor:
    """<pq|rs> = sum_L B^L_pr B^L_qs for p in P, q in Q, r in R, s in S."""
    return torch.einsum('lpr,lqs->pqrs', B[:, P, R], B[:, Q, S])


def antisym_block(B: torch.Tensor, P, Q, R, S) -> torch.Tensor:
    """<pq||rs> = <pq|rs> - <pq|sr>  (Eq. 39 notation)."""
    return coulomb_block(B, P, Q, R, S) - coulomb_block(B, P, Q, S, R).permute(0, 1, 3, 2)


class Hamiltonian:
    """Normal-ordered spinor Hamiltonian: general Fock matrix f [N, N] plus,
    if ``B`` is given, the antisymmetrised two-electron integral blocks.

    ``B=None`` gives a pure one-body operator (used with f -> dipole matrix to
    form xi and eta, Eq. 31 and 33)."""

    def __init__(self, f, O: int, B=None):
        f = as_c(f)
        N = f.shape[0]
        self.O, self.V, self.N = O, N - O, N
        o, v = slice(0, O), slice(O, N)
        self.foo, self.fov, self.fvo, self.fvv = f[o, o], f[o, v], f[v, o], f[v, v]
        self.two_body = B is not None
        if self.two_body:
            B = as_c(B)
            self.oooo = antisym_block(B, o, o, o, o)   # <mn||ij>
            self.ooov = antisym_block(B, o, o, o, v)   # <mn||ie>
            self.oovo = antisym_block(B, o, o, v, o)   # <mn||ej>
            self.ovoo = antisym_block(B, o, v, o, o)   # <mb||ij>
            self.oovv = antisym_block(B, o, o, v, v)   # <mn||ef>
            self.vvoo = antisym_block(B, v, v, o, o)   # <ab||ij>
            self.ovov = antisym_block(B, o, v, o, v)   # <na||if>
            self.ovvo = antisym_block(B, o, v, v, o)   # <mb||ej>
            self.ovvv = antisym_block(B, o, v, v, v)   # <ma||fe>
            self.vovv = antisym_block(B, v, o, v, v)   # <am||ef>
            self.vvvo = antisym_block(B, v, v, v, o)   # <ab||ej>
            self.vvvv = antisym_block(B, v, v, v, v)   # <ab||ef>
        fd = torch.diagonal(f).real
        self.eo, self.ev = fd[:O], fd[O:]


def fock_of(system) -> np.ndarray:
    """Canonical reference: f = diag(eps)."""
    return np.diag(np.asarray(system["eps"], dtype=np.float64)).astype(np.complex128)


# ----------------------------------------------------------------------------
# amplitude packing (unique i<j, a<b)
# ----------------------------------------------------------------------------

class Layout:
    def __init__(self, O: int, V: int):
        self.O, self.V = O, V
        self.io, self.jo = torch.triu_indices(O, O, offset=1)
        self.av, self.bv = torch.triu_indices(V, V, offset=1)
        self.po, self.pv = self.io.numel(), self.av.numel()
        self.n1, self.n2 = O * V, self.po * self.pv
        self.n = self.n1 + self.n2
        self._I = self.io[:, None].expand(self.po, self.pv)
        self._J = self.jo[:, None].expand(self.po, self.pv)
        self._A = self.av[None, :].expand(self.po, self.pv)
        self._B = self.bv[None, :].expand(self.po, self.pv)

    def split(self, x):
        return x[:self.n1].reshape(self.O, self.V), x[self.n1:].reshape(self.po, self.pv)

    def join(self, t1, t2u):
        return torch.cat([t1.reshape(-1), t2u.reshape(-1)])

    def expand(self, t2u):
        """unique doubles -> full antisymmetric [O, O, V, V]"""
        O, V = self.O, self.V
        z = torch.zeros((O, O, V, V), dtype=t2u.dtype)
        I, J, A, B = self._I, self._J, self._A, self._B
        z = z.index_put((I, J, A, B), t2u)
        z = z.index_put((J, I, A, B), -t2u)
        z = z.index_put((I, J, B, A), -t2u)
        z = z.index_put((J, I, B, A), t2u)
        return z

    def pack(self, t2):
        return t2[self._I, self._J, self._A, self._B]

    def full(self, x):
        t1, t2u = self.split(x)
        return t1, self.expand(t2u)

    def vec(self, t1, t2):
        return self.join(t1, self.pack(t2))

    def denominators(self, H: Hamiltonian) -> torch.Tensor:
        """Diagonal of the zeroth-order Jacobian: f_aa - f_ii and
        f_aa + f_bb - f_ii - f_jj (real)."""
        eo, ev = H.eo, H.ev
        d1 = ev[None, :] - eo[:, None]
        d2 = (ev[self.av] + ev[self.bv])[None, :] - (eo[self.io] + eo[self.jo])[:, None]
        return torch.cat([d1.reshape(-1), d2.reshape(-1)]).to(CT)


# ----------------------------------------------------------------------------
# CCSD residual and energy (Eq. 9-10; Stanton-Gauss intermediates)
# ----------------------------------------------------------------------------

def _Pij(x):  # antisymmetriser P(ij) on the first two indices of [i,j,a,b]
    return x - x.transpose(0, 1)


def _Pab(x):  # P(ab) on the last two indices
    return x - x.transpose(2, 3)


def residual_full(t1, t2, H: Hamiltonian):
    """R_i^a = <Phi_i^a|Hbar|0>, R_ij^ab = <Phi_ij^ab|Hbar|0> for general f."""
    ein = torch.einsum
    w = H.two_body
    tau_t = t2 + 0.5 * (ein('ia,jb->ijab', t1, t1) - ein('ib,ja->ijab', t1, t1))
    tau = t2 + ein('ia,jb->ijab', t1, t1) - ein('ib,ja->ijab', t1, t1)

    # one-body intermediates (Fock diagonal kept; R = 0 at the solution)
    Fae = H.fvv - 0.5 * ein('me,ma->ae', H.fov, t1)
    Fmi = H.foo + 0.5 * ein('ie,me->mi', t1, H.fov)
    Fme = H.fov.clone()
    if w:
        Fae = Fae + ein('mf,mafe->ae', t1, H.ovvv) - 0.5 * ein('mnaf,mnef->ae', tau_t, H.oovv)
        Fmi = Fmi + ein('ne,mnie->mi', t1, H.ooov) + 0.5 * ein('inef,mnef->mi', tau_t, H.oovv)
        Fme = Fme + ein('nf,mnef->me', t1, H.oovv)

    # singles
    R1 = H.fvo.T.clone()
    R1 = R1 + ein('ie,ae->ia', t1, Fae) - ein('ma,mi->ia', t1, Fmi) + ein('imae,me->ia', t2, Fme)
    if w:
        R1 = R1 - ein('nf,naif->ia', t1, H.ovov)
        R1 = R1 - 0.5 * ein('imef,maef->ia', t2, H.ovvv)
        R1 = R1 - 0.5 * ein('mnae,nmei->ia', t2, H.oovo)

    # doubles
    Fbe_t = Fae - 0.5 * ein('mb,me->be', t1, Fme)
    Fmj_t = Fmi + 0.5 * ein('je,me->mj', t1, Fme)
    R2 = _Pab(ein('ijae,be->ijab', t2, Fbe_t)) - _Pij(ein('imab,mj->ijab', t2, Fmj_t))
    if w:
        R2 = R2 + H.vvoo.permute(2, 3, 0, 1)
        X = ein('je,mnie->mnij', t1, H.ooov)
        Wmnij = H.oooo + X - X.transpose(2, 3) + 0.25 * ein('ijef,mnef->mnij', tau, H.oovv)
        Y = ein('mb,amef->abef', t1, H.vovv)
        Wabef = H.vvvv - Y + Y.transpose(0, 1) + 0.25 * ein('mnab,mnef->abef', tau, H.oovv)
        Wmbej = (H.ovvo + ein('jf,mbef->mbej', t1, H.ovvv) - ein('nb,mnej->mbej', t1, H.oovo)
                 - ein('jnfb,mnef->mbej', 0.5 * t2 + ein('jf,nb->jnfb', t1, t1), H.oovv))
        R2 = R2 + 0.5 * ein('mnab,mnij->ijab', tau, Wmnij)
        R2 = R2 + 0.5 * ein('ijef,abef->ijab', tau, Wabef)
        ring = ein('imae,mbej->ijab', t2, Wmbej) - ein('ie,ma,mbej->ijab', t1, t1, H.ovvo)
        R2 = R2 + _Pij(_Pab(ring))
        R2 = R2 + _Pij(ein('ie,abej->ijab', t1, H.vvvo))
        R2 = R2 - _Pab(ein('ma,mbij->ijab', t1, H.ovoo))
    return R1, R2


def energy_full(t1, t2, H: Hamiltonian):
    """Correlation energy <0|Hbar|0> - E_ref for general f (complex)."""
    e = torch.einsum('ia,ia->', H.fov, t1)
    if H.two_body:
        e = e + 0.25 * torch.einsum('ijab,ijab->', H.oovv, t2)
        e = e + 0.5 * torch.einsum('ijab,ia,jb->', H.oovv, t1, t1)
    return e


class CCModel:
    """Residual, energy and their exact derivatives on unique-amplitude vectors."""

    def __init__(self, H: Hamiltonian):
        self.H = H
        self.lay = Layout(H.O, H.V)
        self.D = self.lay.denominators(H)

    def R(self, x):
        t1, t2 = self.lay.full(x)
        R1, R2 = residual_full(t1, t2, self.H)
        return self.lay.vec(R1, R2)

    def E(self, x):
        t1, t2 = self.lay.full(x)
        return energy_full(t1, t2, self.H)

    def jvp(self, x, dx):
        """A dx = (dR/dt) dx  (Eq. 30)."""
        return torch.func.jvp(self.R, (x,), (dx,))[1]

    def vjp(self, x, lam):
        """A^T lam (holomorphic transpose, no conjugation of the Jacobian)."""
        _, f = torch.func.vjp(self.R, x)
        return f(lam.conj())[0].conj()

    def lagrangian_grad(self, x, lam):
        """d/dt [E(t) + lam . R(t)]: the left-hand side of the Lambda
        equations and, for a one-body H, eta (Eq. 33)."""
        def L(y):
            return self.E(y) + torch.sum(lam * self.R(y))
        _, f = torch.func.vjp(L, x)
        return f(torch.ones((), dtype=CT))[0].conj()

    def FX(self, x, lam, dx):
        """F dx = d/de [dL/dt](t + e dx)  (Eq. 34)."""
        return torch.func.jvp(lambda y: self.lagrangian_grad(y, lam), (x,), (dx,))[1]


# ----------------------------------------------------------------------------
# solvers: Jacobi preconditioning + Pulay DIIS (the paper does not state its
# solver; this is the reading used throughout the project)
# ----------------------------------------------------------------------------

def diis_solve(resid, x0, denom, tol, maxit=300, nvec=8):
    """Iterate x <- x - r(x)/denom with Pulay extrapolation until
    max|r| < tol.  Returns (x, iterations, max|r|)."""
    xs, es = [], []
    x = x0
    rn = float('inf')
    for it in range(maxit):
        r = resid(x)
        rn = float(r.abs().max())
        if not np.isfinite(rn):
            raise FloatingPointError("residual is not finite")
        if rn < tol:
            return x, it, rn
        xn = x - r / denom
        xs.append(xn)
        es.append(xn - x)
        if len(xs) > nvec:
            xs.pop(0)
            es.pop(0)
        k = len(xs)
        if k >= 2:
            Bm = torch.zeros((k + 1, k + 1), dtype=CT)
            for i in range(k):
                for j in range(k):
                    Bm[i, j] = torch.vdot(es[i], es[j])
            Bm[k, :k] = -1
            Bm[:k, k] = -1
            rhs = torch.zeros(k + 1, dtype=CT)
            rhs[k] = -1
            c = torch.linalg.solve(Bm, rhs)[:k]
            xn = sum(c[i] * xs[i] for i in range(k))
        x = xn
    raise RuntimeError(f"no convergence after {maxit} iterations (max|r|={rn:.3e})")


def mp2(model: CCModel):
    """One Jacobi step from T=0: t1 = f_ai/(f_ii-f_aa), t2 = <ab||ij>/(e_i+e_j-e_a-e_b)
    (Eq. 39) and the energy of that step."""
    x0 = torch.zeros(model.lay.n, dtype=CT)
    x1 = x0 - model.R(x0) / model.D
    return x1, model.E(x1)


def solve_ccsd(model: CCModel, tol=1e-12, maxit=300):
    x0, _ = mp2(model)
    x, it, rn = diis_solve(model.R, x0, model.D, tol, maxit)
    return x, model.E(x), it


def solve_lambda(model: CCModel, t, tol=1e-12, maxit=300):
    """lambda . A + dE/dt = 0  (left CCSD, stationarity of the Lagrangian)."""
    gE = model.lagrangian_grad(t, torch.zeros_like(t))
    lam0 = -gE / model.D
    lam, it, rn = diis_solve(lambda l: model.vjp(t, l) + gE, lam0, model.D, tol, maxit)
    return lam, it


def solve_x(model: CCModel, t, xi, omega, tol=1e-11, maxit=300):
    """(A - omega) X = -xi  (Eq. 29, the infinitesimal dropped)."""
    den = model.D - omega
    x, it, rn = diis_solve(lambda X: model.jvp(t, X) - omega * X + xi, -xi / den, den, tol, maxit)
    return x, it


def solve_y(model: CCModel, t, rhs, omega, tol=1e-11, maxit=300):
    """Y (A + omega) = -rhs, rhs = eta + F X  (Eq. 32)."""
    den = model.D + omega
    y, it, rn = diis_solve(lambda Y: model.vjp(t, Y) + omega * Y + rhs, -rhs / den, den, tol, maxit)
    return y, it


# ----------------------------------------------------------------------------
# linear response driver (Eq. 29-35)
# ----------------------------------------------------------------------------

def build(system, f=None):
    O = system["O"]
    if f is None:
        f = fock_of(system)
    return CCModel(Hamiltonian(f, O, system["B"]))


def dipole_model(system, comp):
    return CCModel(Hamiltonian(system["mu"][comp], system["O"], None))


def polarizability(system, comps, omegas, tol=1e-11, ground=None, return_parts=False):
    """alpha_AB(omega) = -<<A;B>>_omega with
    <<A;B>> = 1/2 [g_AB + conj(g_BA)],  g_AB = Y^B(omega) . xi^A + eta^A . X^B(omega)
    (Eq. 35; P(A,B) swaps A and B and conjugates).  Only +omega is solved.

    Returns a complex array [n_w, n_c, n_c]; Re is the polarizability."""
    model = build(system)
    if ground is None:
        t, E, _ = solve_ccsd(model)
        lam, _ = solve_lambda(model, t)
    else:
        t, E, lam = ground
    comps = list(comps)
    xi, eta = {}, {}
    for A in comps:
        mA = dipole_model(system, A)
        xi[A] = mA.R(t)
        eta[A] = mA.lagrangian_grad(t, lam)
    nc, nw = len(comps), len(omegas)
    alpha = np.zeros((nw, nc, nc), dtype=np.complex128)
    parts = {}
    for w_i, w in enumerate(omegas):
        X, Y = {}, {}
        for B in comps:
            X[B], _ = solve_x(model, t, xi[B], w, tol)
            Y[B], _ = solve_y(model, t, eta[B] + model.FX(t, lam, X[B]), w, tol)
        g = np.zeros((nc, nc), dtype=np.complex128)
        for a, A in enumerate(comps):
            for b, B in enumerate(comps):
                g[a, b] = complex(torch.sum(Y[B] * xi[A]) + torch.sum(eta[A] * X[B]))
        alpha[w_i] = -0.5 * (g + g.conj().T)
        parts[w] = dict(X=X, Y=Y)
    if return_parts:
        return alpha, dict(t=t, E=E, lam=lam, xi=xi, eta=eta, parts=parts)
    return alpha


def polarizability_pm(system, comps, omegas, tol=1e-11, ground=None):
    """alpha_AB(omega) = -<<A;B>>_omega from Eq. 36: the +-omega form, which
    solves X(+omega) and X(-omega) instead of Y.  With P(A(-w), B(w)) applied,
    G_AB(w) = eta^A.X^B(w) + eta^B.X^A(-w) + X^A(-w).F.X^B(w), and
    C^{+-w} gives <<A;B>>_w = 1/2 [G_AB(w) + conj G_AB(-w)].  F is symmetric, so
    X^A(w).F.X^B(-w) = (F X^A(w)).X^B(-w).  Returns [n_w, n_c, n_c]."""
    model = build(system)
    if ground is None:
        t, E, _ = solve_ccsd(model)
        lam, _ = solve_lambda(model, t)
    else:
        t, E, lam = ground
    comps = list(comps)
    xi, eta = {}, {}
    for A in comps:
        mA = dipole_model(system, A)
        xi[A] = mA.R(t)
        eta[A] = mA.lagrangian_grad(t, lam)
    nc = len(comps)
    out = np.zeros((len(omegas), nc, nc), dtype=np.complex128)
    dot = lambda u, v: complex(torch.sum(u * v))
    for wi, w in enumerate(omegas):
        Xp = {B: solve_x(model, t, xi[B], w, tol)[0] for B in comps}
        Xm = {B: solve_x(model, t, xi[B], -w, tol)[0] for B in comps}
        FXp = {B: model.FX(t, lam, Xp[B]) for B in comps}
        Gp = np.zeros((nc, nc), dtype=np.complex128)
        Gm = np.zeros((nc, nc), dtype=np.complex128)
        for a, A in enumerate(comps):
            for b, B in enumerate(comps):
                Gp[a, b] = dot(eta[A], Xp[B]) + dot(eta[B], Xm[A]) + dot(Xm[A], FXp[B])
                Gm[a, b] = dot(eta[A], Xm[B]) + dot(eta[B], Xp[A]) + dot(FXp[A], Xm[B])
        out[wi] = -0.5 * (Gp + Gm.conj())
    return out


def field_energy(system, comp, F, tol=1e-13):
    """CCSD correlation energy with f -> f + F mu_A (orbital-unrelaxed field)."""
    f = fock_of(system) + F * np.asarray(system["mu"][comp])
    model = build(system, f)
    _, E, _ = solve_ccsd(model, tol=tol)
    return E
