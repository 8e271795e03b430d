"""Oracle: the CCSD residual on a subset of its rows, for systems too large for
the full oracle (test infrastructure; only tests and the golden-file scripts use
it).

Same equations, same notation and same term order as ``ccsd.residual_full``
(Stanton-Gauss spin-orbital CCSD for a general Fock matrix, the residual of
Eq. 9-10 of arXiv:2503.23144), evaluated only for the singles rows (i, a) and
the doubles rows (i, j, a, b) whose occupied indices lie in a chosen set So and
whose virtual indices lie in a chosen set Sv.  Every intermediate is restricted
to the indices those rows read, and every integral block is formed from the
factor, <pq||rs> = sum_L B^L_pr B^L_qs - B^L_ps B^L_qr (``ccsd.antisym_block``),
only over those index ranges.  The largest pieces at O=28, V=600 are the full
<mn||ef> block (4.5 GB) and the slices <ma||fe>, <am||ef> with a in Sv; the
sums over <mn||ef> are written as matrix products on fixed layouts of that
block so that no extra copy of it is made (the sums themselves are unchanged).

The rows of A X (Eq. 30) are the forward derivative of the restricted residual
along X.  For a left vector lambda that is zero outside the sampled rows, the
whole transpose product A^T lambda is the reverse derivative of
lambda . R_rows, because no other row of R contributes to it; the holomorphic
transpose is conj(vjp(conj(lambda))) as in ``ccsd``.  Pinned in the tests
against ``ccsd.residual_full`` and ``CCModel.jvp`` / ``.vjp`` at sizes where the
full oracle runs.
"""
from __future__ import annotations

import numpy as np
import torch

from .ccsd import CT, Layout, as_c

ein = torch.einsum


def block(B, P, Q, R, S):
    """<pq||rs> = sum_L B^L_pr B^L_qs - B^L_ps B^L_qr for index lists P, Q, R, S
    (the definition of ``ccsd.antisym_block``, over arbitrary index sets)."""
    g = lambda X, Y: B[:, X][:, :, Y]
    return ein('lpr,lqs->pqrs', g(P, R), g(Q, S)) - ein('lps,lqr->pqrs', g(P, S), g(Q, R))


def _Pij(x):
    return x - x.transpose(0, 1)


def _Pab(x):
    return x - x.transpose(2, 3)


class RowIntegrals:
    """Fock blocks and the integral slices that the rows So x Sv read.

    ``so`` and ``sv`` are sorted occupied and virtual indices (virtuals counted
    from 0 within the virtual block)."""

    def __init__(self, f, O: int, B, so, sv):
        f = as_c(f)
        B = as_c(B)
        N = f.shape[0]
        V = N - O
        self.O, self.V = O, V
        self.so = torch.as_tensor(np.asarray(so), dtype=torch.long)
        self.sv = torch.as_tensor(np.asarray(sv), dtype=torch.long)
        o, v = torch.arange(0, O), torch.arange(O, N)
        po, pv = self.so, O + self.sv          # global orbital indices of the samples
        self.foo, self.fov, self.fvo, self.fvv = f[:O, :O], f[:O, O:], f[O:, :O], f[O:, O:]
        self.oooo = block(B, o, o, o, o)         # <mn||ij>
        self.ooov = block(B, o, o, o, v)         # <mn||ie>
        self.oovo = block(B, o, o, v, o)         # <mn||ej>
        self.oovv = block(B, o, o, v, v)         # <mn||ef>
        # the same block laid out [m][e][n][f], so that the sums over (n, f)
        # below are plain matrix products of views (no hidden copies of this
        # 4.5 GB block are made or kept by the reverse sweep)
        self.oovv_menf = self.oovv.permute(0, 2, 1, 3).contiguous()
        self.ovov_vo = block(B, o, pv, po, v)    # <na||if>, a in Sv, i in So
        self.ovvo_vo = block(B, o, pv, v, po)    # <mb||ej>, b in Sv, j in So
        self.ovvv_v = block(B, o, pv, v, v)      # <ma||fe>, a in Sv
        self.vovv_v = block(B, pv, o, v, v)      # <am||ef>, a in Sv
        self.vvvv_vv = block(B, pv, pv, v, v)    # <ab||ef>, a, b in Sv
        self.vvoo_vvoo = block(B, pv, pv, po, po)  # <ab||ij>
        self.vvvo_vvo = block(B, pv, pv, v, po)    # <ab||ej>
        self.ovoo_voo = block(B, o, pv, po, po)    # <mb||ij>


def residual_rows(t1, t2, H: RowIntegrals):
    """R_i^a (i in So, a in Sv) and R_ij^ab (i, j in So; a, b in Sv) of
    ``ccsd.residual_full``, term for term."""
    o, v = H.so, H.sv
    t1o, t1v = t1[o], t1[:, v]                       # t_i^e (i in So), t_m^a (a in Sv)
    t2o = t2[o]                                      # t_im^ef, i in So
    tau_t = t2 + 0.5 * (ein('ia,jb->ijab', t1, t1) - ein('ib,ja->ijab', t1, t1))
    tau_oo = t2o[:, o] + ein('ia,jb->ijab', t1o, t1o) - ein('ib,ja->ijab', t1o, t1o)
    tau_vv = t2[:, :, v][:, :, :, v] + ein('ia,jb->ijab', t1v, t1v) - ein('ib,ja->ijab', t1v, t1v)

    O, V, no, nv = H.O, H.V, len(o), len(v)
    W_mn_ef = H.oovv.reshape(O * O, V * V)          # <mn||ef> as [(m,n)][(e,f)]
    W_me_nf = H.oovv_menf.reshape(O * V, O * V)     # <mn||ef> as [(m,e)][(n,f)]

    # one-body intermediates: F_ae for a in Sv, F_mi and F_me in full
    Fae = H.fvv[v] - 0.5 * ein('me,ma->ae', H.fov, t1v)
    Fmi = H.foo + 0.5 * ein('ie,me->mi', t1, H.fov)
    Fme = H.fov.clone()
    # sum_mnf tau~_mn^af <mn||ef>: for each m, [e][(n,f)] x [(n,f)][a], summed over m
    tt_v = tau_t[:, :, v].permute(0, 1, 3, 2).reshape(O, O * V, nv)            # [m][(n,f)][a]
    Fae = Fae + ein('mf,mafe->ae', t1, H.ovvv_v) - 0.5 * torch.bmm(H.oovv_menf.reshape(O, V, O * V), tt_v).sum(0).T
    # sum_nef tau~_in^ef <mn||ef>: [i][(n,e,f)] x [(n,e,f)][m]
    Fmi = Fmi + ein('ne,mnie->mi', t1, H.ooov) + 0.5 * (tau_t.reshape(O, O * V * V)
                                                       @ H.oovv.reshape(O, O * V * V).T).T
    Fme = Fme + (W_me_nf @ t1.reshape(O * V)).reshape(O, V)                   # sum_nf t_n^f <mn||ef>

    # singles rows
    R1 = H.fvo[v][:, o].T.clone()
    R1 = R1 + ein('ie,ae->ia', t1o, Fae) - ein('ma,mi->ia', t1v, Fmi[:, o]) + ein('imae,me->ia', t2o[:, :, v], Fme)
    R1 = R1 - ein('nf,naif->ia', t1, H.ovov_vo)
    R1 = R1 - 0.5 * ein('imef,maef->ia', t2o, H.ovvv_v)
    R1 = R1 - 0.5 * ein('mnae,nmei->ia', t2[:, :, v], H.oovo[:, :, :, o])

    # doubles rows
    Fbe_t = Fae - 0.5 * ein('mb,me->be', t1v, Fme)
    Fmj_t = Fmi[:, o] + 0.5 * ein('je,me->mj', t1o, Fme)
    t2oov = t2o[:, o][:, :, v]                       # t_ij^ae: i, j in So, a in Sv
    t2ovv = t2o[:, :, v][:, :, :, v]                 # t_im^ab: i in So, a, b in Sv
    R2 = _Pab(ein('ijae,be->ijab', t2oov, Fbe_t)) - _Pij(ein('imab,mj->ijab', t2ovv, Fmj_t))
    R2 = R2 + H.vvoo_vvoo.permute(2, 3, 0, 1)
    X = ein('je,mnie->mnij', t1o, H.ooov[:, :, o])
    # sum_ef tau_ij^ef <mn||ef>: [(i,j)][(e,f)] x [(e,f)][(m,n)]
    P_ijmn = (tau_oo.reshape(no * no, V * V) @ W_mn_ef.T).reshape(no, no, O, O)
    Wmnij = H.oooo[:, :, o][:, :, :, o] + X - X.transpose(2, 3) + 0.25 * P_ijmn.permute(2, 3, 0, 1)
    Y = ein('mb,amef->abef', t1v, H.vovv_v)
    # sum_mn tau_mn^ab <mn||ef>: [(a,b)][(m,n)] x [(m,n)][(e,f)]
    T_abef = (tau_vv.reshape(O * O, nv * nv).T @ W_mn_ef).reshape(nv, nv, V, V)
    Wabef = H.vvvv_vv - Y + Y.transpose(0, 1) + 0.25 * T_abef
    # sum_nf Z_jn^fb <mn||ef>, Z = t2/2 + t1 t1: [(m,e)][(n,f)] x [(n,f)][(j,b)]
    Zt = 0.5 * t2o[:, :, :, v] + ein('jf,nb->jnfb', t1o, t1v)                 # [j][n][f][b]
    ZW = (W_me_nf @ Zt.permute(1, 2, 0, 3).reshape(O * V, no * nv)).reshape(O, V, no, nv)   # [m][e][j][b]
    Wmbej = (H.ovvo_vo + ein('jf,mbef->mbej', t1o, H.ovvv_v) - ein('nb,mnej->mbej', t1v, H.oovo[:, :, :, o])
             - ZW.permute(0, 3, 1, 2))
    R2 = R2 + 0.5 * ein('mnab,mnij->ijab', tau_vv, Wmnij)
    R2 = R2 + 0.5 * ein('ijef,abef->ijab', tau_oo, Wabef)
    ring = ein('imae,mbej->ijab', t2o[:, :, v], Wmbej) - ein('ie,ma,mbej->ijab', t1o, t1v, H.ovvo_vo)
    R2 = R2 + _Pij(_Pab(ring))
    R2 = R2 + _Pij(ein('ie,abej->ijab', t1o, H.vvvo_vvo))
    R2 = R2 - _Pab(ein('ma,mbij->ijab', t1v, H.ovoo_voo))
    return R1, R2


class RowModel:
    """The residual rows So x Sv as a function of the unique-amplitude vector
    (``ccsd.Layout`` order) and its exact derivatives.  The derivatives are
    taken with respect to t1 and the full antisymmetric t2 (the expansion of
    the unique doubles is linear and is applied outside the differentiation):
    a unique coordinate x_ijab (i<j, a<b) enters t2 at [i,j,a,b] and [j,i,b,a]
    with +1 and at [j,i,a,b] and [i,j,b,a] with -1."""

    def __init__(self, H: RowIntegrals):
        self.H = H
        self.lay = Layout(H.O, H.V)
        no, nv = len(H.so), len(H.sv)
        self.io, self.jo = torch.triu_indices(no, no, offset=1)
        self.av, self.bv = torch.triu_indices(nv, nv, offset=1)

    def rows(self):
        """Global unique-output coordinates of the rows, in output order:
        singles (i, a) then doubles (i, j, a, b) with i < j, a < b."""
        so, sv = self.H.so, self.H.sv
        s = [(int(i), int(a)) for i in so for a in sv]
        d = [(int(so[i]), int(so[j]), int(sv[a]), int(sv[b]))
             for i, j in zip(self.io.tolist(), self.jo.tolist()) for a, b in zip(self.av.tolist(), self.bv.tolist())]
        return s, d

    def _rows_of(self, t1, t2):
        R1, R2 = residual_rows(t1, t2, self.H)
        I, J = self.io[:, None], self.jo[:, None]
        A, B = self.av[None, :], self.bv[None, :]
        return torch.cat([R1.reshape(-1), R2[I, J, A, B].reshape(-1)])

    def R(self, x):
        with torch.no_grad():
            t1, t2 = self.lay.full(x)
            return self._rows_of(t1, t2)

    def jvp(self, x, dx):
        """Rows of A dx (Eq. 30)."""
        with torch.no_grad():
            t1, t2 = self.lay.full(x)
            d1, d2 = self.lay.full(dx)
        return torch.func.jvp(self._rows_of, (t1, t2), (d1, d2))[1]

    def vjp(self, x, lam_rows):
        """A^T lambda (all unique coordinates) for lambda supported on the rows."""
        with torch.no_grad():
            t1, t2 = self.lay.full(x)
        _, f = torch.func.vjp(self._rows_of, t1, t2)
        g1, g2 = f(lam_rows.conj())
        del f
        lay = self.lay
        I, J, A, B = lay._I, lay._J, lay._A, lay._B
        g2u = g2[I, J, A, B] - g2[J, I, A, B] - g2[I, J, B, A] + g2[J, I, B, A]
        return lay.join(g1, g2u).conj()
