"""Oracle: determinant-space second quantisation (test infrastructure).

Only tests may use this module.  It works on explicit Slater determinants
(bit strings) and never uses the coupled-cluster equations of ``oracle.ccsd``;
it exists to pin them.

* ``hamiltonian_matrix``: H = sum_pq h_pq p^+ q + 1/4 sum_pqrs <pq||rs> p^+ q^+ s r
  in the n-electron determinant basis.
* ``cc_projections``: <Phi_0|e^-T H e^T|Phi_0> and the projections onto
  |Phi_i^a> = a_a^+ a_i |Phi_0>, |Phi_ij^ab> = a_a^+ a_b^+ a_j a_i |Phi_0>
  (Eq. 9-10), by the terminating series of e^{+-T}, for arbitrary amplitudes.
* ``sos_polarizability``: exact response function of Eq. 18 from the FCI
  states, alpha = -<<A;B>>.

The one-body part h is chosen so that the reference Fock matrix is the given f:
h_pq = f_pq - sum_i <pi||qi>, E_ref = sum_i f_ii - 1/2 sum_ij <ij||ij>.
"""
from __future__ import annotations

import itertools

import numpy as np


def _sign_and_apply(det: int, p: int, create: bool):
    """Apply a^+_p (create) or a_p to the determinant bit string ``det``.
    Returns (sign, new_det) or None when the result vanishes.  The sign is
    (-1)^(number of occupied spinors with index < p)."""
    occ = (det >> p) & 1
    if create == bool(occ):
        return None
    sign = -1 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1
    return sign, det ^ (1 << p)


def apply_string(det: int, ops):
    """Apply an operator string, given left-to-right as written, e.g.
    [('c', a), ('c', b), ('a', j), ('a', i)] for a_a^+ a_b^+ a_j a_i.  The
    rightmost operator acts first."""
    sign = 1
    for kind, p in reversed(ops):
        r = _sign_and_apply(det, p, kind == 'c')
        if r is None:
            return None
        s, det = r
        sign *= s
    return sign, det


def determinants(N: int, nel: int):
    dets = []
    for occ in itertools.combinations(range(N), nel):
        d = 0
        for p in occ:
            d |= 1 << p
        dets.append(d)
    return dets, {d: k for k, d in enumerate(dets)}


def full_antisym(B: np.ndarray) -> np.ndarray:
    """<pq||rs> over all spinors from <pq|rs> = sum_L B^L_pr B^L_qs."""
    g = np.einsum('lpr,lqs->pqrs', B, B)
    return g - g.transpose(0, 1, 3, 2)


def core_hamiltonian(f: np.ndarray, gA: np.ndarray, O: int) -> np.ndarray:
    return f - np.einsum('piqi->pq', gA[:, :O, :, :O])


def one_body_matrix(h: np.ndarray, dets, index) -> np.ndarray:
    """Matrix of sum_pq h_pq p^+ q in the determinant basis."""
    n = len(dets)
    N = h.shape[0]
    M = np.zeros((n, n), dtype=np.complex128)
    for k, d in enumerate(dets):
        occ = [p for p in range(N) if (d >> p) & 1]
        for q in occ:
            for p in range(N):
                r = apply_string(d, [('c', p), ('a', q)])
                if r is None:
                    continue
                s, d2 = r
                M[index[d2], k] += s * h[p, q]
    return M


def hamiltonian_matrix(h: np.ndarray, gA: np.ndarray, dets, index) -> np.ndarray:
    """H = sum h_pq p^+q + sum_{p<q, r<s} <pq||rs> p^+ q^+ s r."""
    N = h.shape[0]
    H = one_body_matrix(h, dets, index)
    for k, d in enumerate(dets):
        occ = [p for p in range(N) if (d >> p) & 1]
        for r, s in itertools.combinations(occ, 2):
            for p, q in itertools.combinations(range(N), 2):
                val = gA[p, q, r, s]
                if val == 0:
                    continue
                res = apply_string(d, [('c', p), ('c', q), ('a', s), ('a', r)])
                if res is None:
                    continue
                sg, d2 = res
                H[index[d2], k] += sg * val
    return H


def cluster_matrix(t1: np.ndarray, t2: np.ndarray, O: int, dets, index) -> np.ndarray:
    """T = sum_ia t_i^a a_a^+ a_i + sum_{i<j,a<b} t_ij^ab a_a^+ a_b^+ a_j a_i
    (Eq. 3-4 with T1 unscaled; the 1/4 of T2 absorbed by the ordered sums)."""
    V = t1.shape[1]
    n = len(dets)
    T = np.zeros((n, n), dtype=np.complex128)
    for k, d in enumerate(dets):
        for i in range(O):
            for a in range(V):
                if t1[i, a] == 0:
                    continue
                r = apply_string(d, [('c', O + a), ('a', i)])
                if r is not None:
                    T[index[r[1]], k] += r[0] * t1[i, a]
        for i, j in itertools.combinations(range(O), 2):
            for a, b in itertools.combinations(range(V), 2):
                if t2[i, j, a, b] == 0:
                    continue
                r = apply_string(d, [('c', O + a), ('c', O + b), ('a', j), ('a', i)])
                if r is not None:
                    T[index[r[1]], k] += r[0] * t2[i, j, a, b]
    return T


def _exp_apply(T: np.ndarray, v: np.ndarray, sign: float, kmax: int) -> np.ndarray:
    out = v.copy()
    term = v.copy()
    for k in range(1, kmax + 1):
        term = sign * (T @ term) / k
        out = out + term
    return out


def cc_projections(f, B, O, t1, t2):
    """Brute-force <Phi_0|Hbar|Phi_0> - E_ref and the projected residuals
    R_i^a = <Phi_i^a|Hbar|Phi_0>, R_ij^ab = <Phi_ij^ab|Hbar|Phi_0>
    (full antisymmetric [O,O,V,V]) with Hbar = e^-T H e^T."""
    f = np.asarray(f, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    N = f.shape[0]
    V = N - O
    gA = full_antisym(B)
    h = core_hamiltonian(f, gA, O)
    dets, index = determinants(N, O)
    H = hamiltonian_matrix(h, gA, dets, index)
    T = cluster_matrix(t1, t2, O, dets, index)
    ref = (1 << O) - 1
    phi0 = np.zeros(len(dets), dtype=np.complex128)
    phi0[index[ref]] = 1.0
    w = _exp_apply(T, H @ _exp_apply(T, phi0, +1.0, O), -1.0, O)
    e_ref = (H @ phi0)[index[ref]]
    E = w[index[ref]] - e_ref
    R1 = np.zeros((O, V), dtype=np.complex128)
    for i in range(O):
        for a in range(V):
            s, d = apply_string(ref, [('c', O + a), ('a', i)])
            R1[i, a] = s * w[index[d]]
    R2 = np.zeros((O, O, V, V), dtype=np.complex128)
    for i, j in itertools.combinations(range(O), 2):
        for a, b in itertools.combinations(range(V), 2):
            s, d = apply_string(ref, [('c', O + a), ('c', O + b), ('a', j), ('a', i)])
            val = s * w[index[d]]
            R2[i, j, a, b] = val
            R2[j, i, a, b] = -val
            R2[i, j, b, a] = -val
            R2[j, i, b, a] = val
    return E, R1, R2, e_ref


def fci_states(f, B, O):
    """All eigenpairs of the n-electron Hamiltonian (n = O) and E_ref."""
    f = np.asarray(f, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    N = f.shape[0]
    gA = full_antisym(B) if B is not None else np.zeros((N,) * 4, dtype=np.complex128)
    h = core_hamiltonian(f, gA, O)
    dets, index = determinants(N, O)
    H = hamiltonian_matrix(h, gA, dets, index)
    if not np.allclose(H, H.conj().T, atol=1e-12):
        raise ValueError("determinant-space Hamiltonian is not Hermitian")
    E, C = np.linalg.eigh(H)
    ref = (1 << O) - 1
    e_ref = H[index[ref], index[ref]].real
    return E, C, dets, index, e_ref


def sos_polarizability(f, B, mu, O, comps, omegas):
    """alpha_AB(omega) = sum_k [A_0k B_k0/(w_k - omega) + B_0k A_k0/(w_k + omega)]
    from Eq. 18 with alpha = -<<A;B>>.  Returns ([n_w, n_c, n_c], E0, w_min)."""
    E, C, dets, index, _ = fci_states(f, B, O)
    ops = {c: one_body_matrix(np.asarray(mu[c]), dets, index) for c in comps}
    psi0 = C[:, 0]
    wk = E[1:] - E[0]
    amp = {c: psi0.conj() @ ops[c] @ C[:, 1:] for c in comps}      # <0|A|k>
    ampk = {c: C[:, 1:].conj().T @ ops[c] @ psi0 for c in comps}  # <k|A|0>
    out = np.zeros((len(omegas), len(comps), len(comps)), dtype=np.complex128)
    for wi, w in enumerate(omegas):
        for a, A in enumerate(comps):
            for b, Bc in enumerate(comps):
                out[wi, a, b] = np.sum(amp[A] * ampk[Bc] / (wk - w) + amp[Bc] * ampk[A] / (wk + w))
    return out, E[0], wk.min()
