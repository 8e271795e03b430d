"""Oracle: FNS++ perturbation-sensitive natural-spinor truncation (test infrastructure).

Only tests and the CPU-baseline leg of ``bench.py`` may use this module.
Plain numpy, complex128, following Sec. II.B-C of the paper:

1. MP2 doubles t_ij^ab = <ab||ij>/(e_i + e_j - e_a - e_b)             (Eq. 39)
2. Hbar_ii = f_ii + 1/2 sum_nef t_in^ef <in||ef>,
   Hbar_aa = f_aa - 1/2 sum_mnf t_mn^fa <mn||fa>                        (Eq. 49-50)
3. per dipole direction A: Abar_ij^ab = P(ab) sum_e t_ij^ae A_be
   - P(ij) sum_m t_im^ab A_mj, Abar_i^a = A_ai + sum_me A_me t_im^ae    (Eq. 48)
4. t^(1) = Abar / (Dbar - omega), Dbar from Hbar                       (Eq. 46-47)
5. D^A_ab = 1/2 sum_ijc t_ij^ac conj(t_ij^bc) + sum_i t_i^a conj(t_i^b),
   averaged over x, y, z                                               (Eq. 45)
6. eigenvectors of the averaged density = natural spinors (Eq. 41); keep by
   |n| descending (stable in the eigen-solver's order), by count or by
   threshold (the density is not positive definite, so |n| is used)
7. Ftilde = Vt^H F_vv Vt, diagonalise (Eq. 42-43); U = Vt Z (Eq. 44 read as
   a column-vector transformation)
8. rotate B^L and mu into the new virtual basis; new virtual energies are the
   semicanonical eigenvalues.

Plain FNS (Eq. 40) replaces step 2-5 by the ground-state MP2 virtual density
D_ab = 1/2 sum_ijc t_ij^ac conj(t_ij^bc) and keeps steps 6-8.

Readings where the paper is ambiguous (the project's readings): Eq. 40/45 are
taken with the complex conjugate on the second amplitude (Hermitian density);
the three directions are averaged at the level of densities; the denominator
sign follows Eq. 29 (Dbar - omega), with ``plus_omega=True`` giving Eq. 46 as
printed.
"""
from __future__ import annotations

import numpy as np


def _anti(B, P, Q, R, S):
    d = np.einsum('lpr,lqs->pqrs', B[:, P, R], B[:, Q, S], optimize=True)
    x = np.einsum('lps,lqr->pqrs', B[:, P, S], B[:, Q, R], optimize=True)
    return d - x


def mp2_doubles(eps, B, O):
    N = eps.shape[0]
    o, v = slice(0, O), slice(O, N)
    vvoo = _anti(B, v, v, o, o)                      # <ab||ij>
    eo, ev = eps[:O], eps[O:]
    D = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return vvoo.transpose(2, 3, 0, 1) / D           # t[i,j,a,b]


def mp2_energy(eps, B, O):
    N = eps.shape[0]
    o, v = slice(0, O), slice(O, N)
    t2 = mp2_doubles(eps, B, O)
    oovv = _anti(B, o, o, v, v)
    return 0.25 * np.einsum('ijab,ijab->', oovv, t2)


def hbar_diagonals(eps, B, O, t2):
    N = eps.shape[0]
    o, v = slice(0, O), slice(O, N)
    oovv = _anti(B, o, o, v, v)                      # <mn||ef>
    Hii = eps[:O] + 0.5 * np.einsum('inef,inef->i', t2, oovv).real
    Haa = eps[O:] - 0.5 * np.einsum('mnfa,mnfa->a', t2, oovv).real
    return Hii, Haa


def perturbed_moments(eps, B, mu_c, O, t2):
    """Abar for one perturbation A = mu_c (Eq. 48 for the doubles; singles
    A_ai + sum_me A_me t_im^ae).  Returns ([O, V], [O, O, V, V])."""
    A = np.asarray(mu_c)
    Aoo, Aov, Avo, Avv = A[:O, :O], A[:O, O:], A[O:, :O], A[O:, O:]
    X = np.einsum('ijae,be->ijab', t2, Avv, optimize=True)
    Yy = np.einsum('imab,mj->ijab', t2, Aoo, optimize=True)
    A2 = (X - X.transpose(0, 1, 3, 2)) - (Yy - Yy.transpose(1, 0, 2, 3))
    A1 = Avo.T + np.einsum('me,imae->ia', Aov, t2, optimize=True)
    return A1, A2


def hbar_denominators(Hii, Haa):
    """Dbar of Eq. 47: Hbar_aa - Hbar_ii (singles), Hbar_aa + Hbar_bb -
    Hbar_ii - Hbar_jj (doubles)."""
    D2 = (Haa[None, None, :, None] + Haa[None, None, None, :]
          - Hii[:, None, None, None] - Hii[None, :, None, None])
    D1 = Haa[None, :] - Hii[:, None]
    return D1, D2


def first_order_amplitudes(eps, B, mu_c, O, t2, Hii, Haa, omega=0.0, plus_omega=False):
    """Abar over (Dbar -/+ omega) for one perturbation A = mu_c (Eq. 46-48)."""
    A1, A2 = perturbed_moments(eps, B, mu_c, O, t2)
    s = 1.0 if plus_omega else -1.0
    D1, D2 = hbar_denominators(Hii, Haa)
    return A1 / (D1 + s * omega), A2 / (D2 + s * omega)


def fnspp_density(eps, B, mu, O, omega=0.0, plus_omega=False):
    """Averaged perturbation-sensitive virtual density M [V, V] (Eq. 45)."""
    t2 = mp2_doubles(eps, B, O)
    Hii, Haa = hbar_diagonals(eps, B, O, t2)
    V = eps.shape[0] - O
    M = np.zeros((V, V), dtype=np.complex128)
    for c in range(3):
        t1p, t2p = first_order_amplitudes(eps, B, mu[c], O, t2, Hii, Haa, omega, plus_omega)
        M += 0.5 * np.einsum('ijac,ijbc->ab', t2p, t2p.conj()) + np.einsum('ia,ib->ab', t1p, t1p.conj())
    return M / 3.0


def mp2_density(eps, B, O):
    """Ground-state MP2 virtual density [V, V] of plain FNS (Eq. 40)."""
    t2 = mp2_doubles(eps, B, O)
    return 0.5 * np.einsum('ijac,ijbc->ab', t2, t2.conj())


def mp2_polarizability(system, comps, omegas):
    """MP2-level polarisability (the ingredient of the Delta alpha_MP2
    correction, Eq. 53-54), in the system's own virtual basis.

    Reading: the sum-over-states response function (Eq. 18, alpha =
    -<<A;B>>) over the singly and doubly excited determinants mu, with the
    MP2-dressed transition moments Abar_mu of Eq. 48 and the diagonal
    excitation energies Dbar_mu of Eq. 47 (Hbar of Eq. 49-50):

        alpha_AB(w) = sum_mu conj(Abar_mu) Bbar_mu / (Dbar_mu - w)
                             + Abar_mu conj(Bbar_mu) / (Dbar_mu + w)

    i.e. sum_mu conj(Abar_mu) t^(1)_mu(B; w) + Abar_mu conj(t^(1)_mu(B; -w))
    with the Eq. 46 amplitudes t^(1) = Bbar / (Dbar - w); the doubles run over
    unique (i<j, a<b), a quarter of the full-array sum.
    Returns [n_w, n_c, n_c] complex."""
    eps = np.asarray(system["eps"], dtype=np.float64)
    B = np.asarray(system["B"])
    mu = np.asarray(system["mu"])
    O = system["O"]
    t2 = mp2_doubles(eps, B, O)
    Hii, Haa = hbar_diagonals(eps, B, O, t2)
    D1, D2 = hbar_denominators(Hii, Haa)
    mom = {c: perturbed_moments(eps, B, mu[c], O, t2) for c in comps}
    out = np.zeros((len(omegas), len(comps), len(comps)), dtype=np.complex128)
    for wi, w in enumerate(omegas):
        for a, A in enumerate(comps):
            for b, Bc in enumerate(comps):
                (a1, a2), (b1, b2) = mom[A], mom[Bc]
                s1 = np.sum(a1.conj() * b1 / (D1 - w) + a1 * b1.conj() / (D1 + w))
                s2 = np.sum(a2.conj() * b2 / (D2 - w) + a2 * b2.conj() / (D2 + w))
                out[wi, a, b] = s1 + 0.25 * s2
    return out


# --- the same steps from the virtual-occupied factor block alone ------------
# MP2 (Eq. 39, 51), the Hbar diagonals (Eq. 49-50) and the densities need only
# <ab||ij> and <ij||ab>, i.e. B^L_ai and B^L_ia = conj(B^L_ai) (B^L Hermitian):
# these variants take Bvo [L, V, O] so that systems whose full factor does not
# fit in host memory can be checked.

def vvoo_from_vo(Bvo):
    """<ab||ij> = sum_L B_ai B_bj - B_aj B_bi  -> [a, b, i, j]."""
    d = np.einsum('lai,lbj->abij', Bvo, Bvo, optimize=True)
    return d - d.transpose(0, 1, 3, 2)


def oovv_from_vo(Bvo):
    """<ij||ab> = sum_L B_ia B_jb - B_ib B_ja with B_ia = conj(B_ai)  -> [i, j, a, b]."""
    Bov = Bvo.conj().transpose(0, 2, 1)
    d = np.einsum('lia,ljb->ijab', Bov, Bov, optimize=True)
    return d - d.transpose(0, 1, 3, 2)


def mp2_doubles_vo(eps, Bvo, O):
    eo, ev = eps[:O], eps[O:]
    D = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return vvoo_from_vo(Bvo).transpose(2, 3, 0, 1) / D


def mp2_energy_vo(eps, Bvo, O):
    return 0.25 * np.einsum('ijab,ijab->', oovv_from_vo(Bvo), mp2_doubles_vo(eps, Bvo, O))


def hbar_diagonals_vo(eps, Bvo, O, t2):
    oovv = oovv_from_vo(Bvo)
    Hii = eps[:O] + 0.5 * np.einsum('inef,inef->i', t2, oovv).real
    Haa = eps[O:] - 0.5 * np.einsum('mnfa,mnfa->a', t2, oovv).real
    return Hii, Haa


def truncation_from_vo(eps, Bvo, mu, O, by_count, value, omega=0.0, plus_omega=False, density="fnspp"):
    """Steps 1-7 of ``truncate`` and the MP2 energies of Eq. 51 from the
    virtual-occupied factor block: returns dict(occ = |n| sorted descending,
    eps_virt = semicanonical energies of the kept space, e_mp2_full,
    e_mp2_trunc, gap = (|n_k| - |n_k+1|) / |n_k| at the cut)."""
    eps = np.asarray(eps, dtype=np.float64)
    N = eps.shape[0]
    t2 = mp2_doubles_vo(eps, Bvo, O)
    if density == "fnspp":
        Hii, Haa = hbar_diagonals_vo(eps, Bvo, O, t2)
        M = np.zeros((N - O, N - O), dtype=np.complex128)
        for c in range(3):
            t1p, t2p = first_order_amplitudes(eps, None, mu[c], O, t2, Hii, Haa, omega, plus_omega)
            M += 0.5 * np.einsum('ijac,ijbc->ab', t2p, t2p.conj(), optimize=True)
            M += np.einsum('ia,ib->ab', t1p, t1p.conj())
            del t1p, t2p
        M /= 3.0
    elif density == "mp2":
        M = 0.5 * np.einsum('ijac,ijbc->ab', t2, t2.conj(), optimize=True)
    else:
        raise ValueError("density must be 'fnspp' or 'mp2'")
    e_full = 0.25 * np.einsum('ijab,ijab->', oovv_from_vo(Bvo), t2)
    del t2
    n, Vn = np.linalg.eigh(M)
    keep = select(n, by_count, value)
    occ = np.abs(n[np.argsort(-np.abs(n), kind='stable')])
    k = keep.shape[0]
    gap = (occ[k - 1] - occ[k]) / occ[k - 1] if k < occ.shape[0] else 1.0
    Vt = Vn[:, keep]
    et, Z = np.linalg.eigh(Vt.conj().T @ np.diag(eps[O:]) @ Vt)
    U = Vt @ Z
    Bvo_new = np.einsum('ar,lai->lri', U.conj(), Bvo, optimize=True)   # (Uf^H B Uf)[v', o]
    eps_new = np.concatenate([eps[:O], et])
    return dict(occ=occ, eps_virt=et, e_mp2_full=e_full, e_mp2_trunc=mp2_energy_vo(eps_new, Bvo_new, O), gap=gap)


def select(n: np.ndarray, by_count: bool, value: float) -> np.ndarray:
    """Indices of kept natural spinors: sort by |n| descending, ties in the
    eigen-solver's order; keep the first ``value`` (count) or all with
    |n| >= value (threshold)."""
    order = np.argsort(-np.abs(n), kind='stable')
    if by_count:
        k = int(value)
        if k < 1 or k > n.shape[0]:
            raise ValueError("count out of range")
        return order[:k]
    keep = order[np.abs(n[order]) >= value]
    if keep.size == 0:
        raise ValueError("threshold removes every virtual")
    return keep


def truncate(system, by_count=True, value=None, omega=0.0, plus_omega=False, density="fnspp"):
    """FNS++ (``density="fnspp"``, Eq. 45) or plain FNS (``density="mp2"``,
    Eq. 40) truncation.  Returns (new_system, occupations sorted by |n| desc,
    details)."""
    eps = np.asarray(system["eps"], dtype=np.float64)
    B = np.asarray(system["B"])
    mu = np.asarray(system["mu"])
    O = system["O"]
    if density == "fnspp":
        M = fnspp_density(eps, B, mu, O, omega, plus_omega)
    elif density == "mp2":
        M = mp2_density(eps, B, O)
    else:
        raise ValueError("density must be 'fnspp' or 'mp2'")
    n, Vn = np.linalg.eigh(M)
    keep = select(n, by_count, value)
    Vt = Vn[:, keep]
    Ft = Vt.conj().T @ np.diag(eps[O:]) @ Vt
    et, Z = np.linalg.eigh(Ft)
    U = Vt @ Z
    N, Vk = eps.shape[0], U.shape[1]
    Uf = np.zeros((N, O + Vk), dtype=np.complex128)
    Uf[:O, :O] = np.eye(O)
    Uf[O:, O:] = U
    Bn = np.einsum('pr,lpq,qs->lrs', Uf.conj(), B, Uf, optimize=True)
    mun = np.einsum('pr,cpq,qs->crs', Uf.conj(), mu, Uf, optimize=True)
    new = dict(system)
    new.update(V=Vk, N=O + Vk, eps=np.concatenate([eps[:O], et]), B=Bn, mu=mun)
    occ = np.abs(n[np.argsort(-np.abs(n), kind='stable')])
    return new, occ, dict(M=M, n=n, U=U)
