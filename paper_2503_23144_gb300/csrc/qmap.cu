// The Q map of the CCSD doubles residual, Q_amij = sum_ef <am||ef> X_ij^ef,
// contracted from the three-index factor instead of a stored O V^3 block.
//
// In the spin-orbital CCSD residual (Stanton-Gauss intermediates, used for the
// ground state of Eq. 9-10 and, differentiated, for the Jacobian of Eq. 30) the
// T1-weighted part of W_abef contributes -1/2 P(ab) sum_m t_m^b Q_amij with
// tau in place of X.  With <pq|rs> = sum_L B^L_pr B^L_qs,
//   <am||ef> = sum_L (B^L_ae B^L_mf - B^L_af B^L_me),
// so for a slab of a the products GT[(m,f)][(a,e)] = sum_L Bov^L_mf Bvv^L_ae come
// from one GEMM over L and W[(a,m)][e<f] = GT[(m,f)][(a,e)] - GT[(m,e)][(a,f)].
// Each slab is contracted with the packed X (pairs i<j, e<f) before the next is
// built: the O V^3 block never exists in memory (97 GB at O=28, V=600).
#include "lrcc_internal.h"

#include <algorithm>

namespace {

int grid_of(Dev& D, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)D.sm_count * 16));
}

// W[(a*O + m)][pair(e,f)] = GT[m][f][a][e] - GT[m][e][a][f] for e < f, with
// GT [O][V][na][V] (a relative to the slab).  One 32x32 (f, e) tile per block
// and (a, m) row per blockIdx.z; both GT reads go through shared memory so that
// they are coalesced, and consecutive threads write consecutive f (consecutive
// pair indices).
constexpr int QT = 32;
__global__ void k_antisym_q(const cplx* __restrict__ GT, cplx* __restrict__ W, int64_t na, int64_t O, int64_t V) {
    __shared__ cplx ta[QT][QT + 1];  // ta[fr][ec] = GT[m][fb+fr][a][eb+ec]
    __shared__ cplx tb[QT][QT + 1];  // tb[er][fc] = GT[m][eb+er][a][fb+fc]
    const int64_t row = blockIdx.z;  // a * O + m
    const int64_t a = row / O, m = row - a * O;
    const int64_t fb = (int64_t)blockIdx.x * QT, eb = (int64_t)blockIdx.y * QT;
    if (fb + QT - 1 <= eb) return;  // no e < f in this tile
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
    const int64_t rs = na * V;                     // GT stride of f (and of e in the second read)
    const cplx* g = GT + m * V * rs + a * V;
    for (int r = ty; r < QT; r += 8) {
        const int64_t f = fb + r, e = eb + tx;
        ta[r][tx] = (f < V && e < V) ? g[f * rs + e] : make_double2(0.0, 0.0);
        const int64_t e2 = eb + r, f2 = fb + tx;
        tb[r][tx] = (e2 < V && f2 < V) ? g[e2 * rs + f2] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int64_t PV = V * (V - 1) / 2;
    cplx* w = W + row * PV;
    for (int r = ty; r < QT; r += 8) {
        const int64_t e = eb + r, f = fb + tx;
        if (e >= V || f >= V || e >= f) continue;
        const cplx u = ta[tx][r], v = tb[r][tx];
        w[e * (2 * V - e - 1) / 2 + (f - e - 1)] = make_double2(u.x - v.x, u.y - v.y);
    }
}

// Q[r][a][m][i][j] = alpha * sign * Zq[a*O + m][r*PO + pair(min(i,j), max(i,j))] + beta * Q
// (sign -1 for i > j, 0 for i == j)
__global__ void k_unpack_q(const cplx* __restrict__ Zq, cplx* __restrict__ Q, int64_t R, int64_t V, int64_t O,
                           cplx alpha, cplx beta, int beta0) {
    const int64_t PO = O * (O - 1) / 2;
    const int64_t total = R * V * O * O * O;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = idx;
        const int64_t j = t % O;
        t /= O;
        const int64_t i = t % O;
        t /= O;
        const int64_t am = t % (V * O), r = t / (V * O);
        cplx v = make_double2(0.0, 0.0);
        if (i != j) {
            const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
            const double sg = i < j ? 1.0 : -1.0;
            const cplx z = Zq[am * (R * PO) + r * PO + lo * (2 * O - lo - 1) / 2 + (hi - lo - 1)];
            v = make_double2(sg * (alpha.x * z.x - alpha.y * z.y), sg * (alpha.x * z.y + alpha.y * z.x));
        }
        if (!beta0) {
            const cplx o = Q[idx];
            v.x += beta.x * o.x - beta.y * o.y;
            v.y += beta.x * o.y + beta.y * o.x;
        }
        Q[idx] = v;
    }
}

// Qt[a*O + m][r*PO + ij] = Qb[r][a][m][i][j] for i < j
__global__ void k_pack_q(const cplx* __restrict__ Qb, cplx* __restrict__ Qt, int64_t R, int64_t V, int64_t O) {
    const int64_t PO = O * (O - 1) / 2;
    const int64_t total = R * V * O * O * O;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = idx;
        const int64_t j = t % O;
        t /= O;
        const int64_t i = t % O;
        t /= O;
        if (i >= j) continue;
        const int64_t am = t % (V * O), r = t / (V * O);
        Qt[am * (R * PO) + r * PO + i * (2 * O - i - 1) / 2 + (j - i - 1)] = Qb[idx];
    }
}

// a values per slab: GT and W of one slab within a modest share of memory
int64_t slab_a(Dev& D, int64_t O, int64_t V) {
    const double per_a = 16.0 * double(O) * double(V) * double(V) + 16.0 * double(O) * double(V * (V - 1) / 2);
    const double bytes = std::max(double(1 << 26), std::min(0.12 * free_bytes(D), 6.0 * double(1 << 30)));
    const int64_t cap = std::min<int64_t>(V, 65535 / std::max<int64_t>(O, 1));  // rows per grid z
    return std::max<int64_t>(1, std::min<int64_t>(cap, (int64_t)(bytes / per_a)));
}

// rows (a, m), a in [a0, a0 + na), of <am||ef> (e < f) into W [na*O][PV]
void assemble_q(Dev& D, LadderCtx& LC, int64_t a0, int64_t na, int prec, Tensor& GT, Tensor& W) {
    const int64_t O = LC.Bov.d[1], V = LC.Bov.d[2];
    Tensor g = GT.slice(0, 0, O * V * na * V).reshape({O, V, na, V});
    ein(D, "Lmf,Lae->mfae", mkc(1.0), LC.Bov, false, LC.Bvv.slice(1, a0, na), false, mkc(0.0), g, prec);
    dim3 grid((unsigned)((V + QT - 1) / QT), (unsigned)((V + QT - 1) / QT), (unsigned)(na * O));
    k_antisym_q<<<grid, dim3(QT, 8), 0, D.st>>>(g.p, W.p, na, O, V);
    LAUNCH_CHECK(D);
}

// The whole W [V*O][P_V] once, when it fits in a sixth of the free memory,
// built with FP64 products for the FP64 path and FP64-class (integer-slice)
// products otherwise; a matrix built with FP64 products serves every precision.
bool ensure_qcache(Dev& D, LadderCtx& LC, int prec) {
    const int builder = prec == LRCC_FP64 ? LRCC_FP64 : LRCC_FP64_EMULATED;
    if (LC.wq64.p && (LC.wq64_prec == LRCC_FP64 || LC.wq64_prec == builder)) return true;
    if (LC.wq64_disabled) return false;
    const int64_t O = LC.Bov.d[1], V = LC.Bov.d[2], PV = V * (V - 1) / 2;
    if (16.0 * double(V * O) * double(PV) > free_bytes(D) / 6.0) {
        LC.wq64_disabled = true;
        return false;
    }
    LC.wq64 = Tensor();
    Tensor W = empty(D, {V * O, PV});
    const int64_t na = slab_a(D, O, V);
    Tensor GT = empty(D, {O * V * na * V});
    for (int64_t a0 = 0; a0 < V; a0 += na) {
        const int64_t n = std::min(na, V - a0);
        Tensor Ws = W.slice(0, a0 * O, n * O);
        assemble_q(D, LC, a0, n, builder, GT, Ws);
    }
    LC.wq64 = W;
    LC.wq64_prec = builder;
    return true;
}

}  // namespace

void qmap(Dev& D, LadderCtx& LC, const Tensor& X, cplx alpha, cplx beta, Tensor& Q, int prec) {
    REQUIRE(X.nd == 5 && Q.nd == 5 && X.contiguous() && Q.contiguous(), "qmap needs contiguous operands");
    const int64_t R = X.d[0], O = X.d[1], V = X.d[3];
    REQUIRE(LC.Bov.p && LC.Bov.d[1] == O && LC.Bov.d[2] == V && LC.Bvv.d[1] == V, "qmap: factor blocks");
    REQUIRE(Q.d[0] == R && Q.d[1] == V && Q.d[2] == O && Q.d[3] == O && Q.d[4] == O, "qmap: output shape");
    const int64_t PO = O * (O - 1) / 2, PV = V * (V - 1) / 2;
    const bool beta0 = beta.x == 0.0 && beta.y == 0.0;
    if (PO == 0 || PV == 0) {
        if (beta0) fill(D, Q, mkc(0.0));
        else axpby(D, mkc(0.0), Q, false, beta, Q);
        return;
    }
    Tensor Xt = empty(D, {R * PO, PV});
    ladder_pack_xt(D, X.p, Xt.p, R, O, V);
    Tensor Zq = empty(D, {V * O, R * PO});
    if (ensure_qcache(D, LC, prec)) {
        ein(D, "xk,nk->xn", mkc(2.0), LC.wq64, false, Xt, false, mkc(0.0), Zq, prec);
        k_unpack_q<<<grid_of(D, R * V * O * O * O), 256, 0, D.st>>>(Zq.p, Q.p, R, V, O, alpha, beta, beta0);
        LAUNCH_CHECK(D);
        return;
    }
    const int64_t na = slab_a(D, O, V);
    Tensor GT = empty(D, {O * V * na * V});
    Tensor W = empty(D, {na * O, PV});
    for (int64_t a0 = 0; a0 < V; a0 += na) {
        const int64_t n = std::min(na, V - a0);
        Tensor Ws = W.slice(0, 0, n * O);
        assemble_q(D, LC, a0, n, prec, GT, Ws);
        Tensor Zs = Zq.slice(0, a0 * O, n * O);
        // sum over all (e, f) = 2 sum over e < f of <am||ef> (X_ef - X_fe)/2
        ein(D, "xk,nk->xn", mkc(2.0), Ws, false, Xt, false, mkc(0.0), Zs, prec);
    }
    k_unpack_q<<<grid_of(D, R * V * O * O * O), 256, 0, D.st>>>(Zq.p, Q.p, R, V, O, alpha, beta, beta0);
    LAUNCH_CHECK(D);
}

void qmap_t(Dev& D, LadderCtx& LC, const Tensor& Qb, cplx alpha, cplx beta, Tensor& Xb, int prec) {
    REQUIRE(Qb.nd == 5 && Xb.nd == 5 && Qb.contiguous() && Xb.contiguous(), "qmap_t needs contiguous operands");
    const int64_t R = Xb.d[0], O = Xb.d[1], V = Xb.d[3];
    REQUIRE(LC.Bov.p && LC.Bov.d[1] == O && LC.Bov.d[2] == V && LC.Bvv.d[1] == V, "qmap_t: factor blocks");
    REQUIRE(Qb.d[0] == R && Qb.d[1] == V && Qb.d[2] == O && Qb.d[3] == O && Qb.d[4] == O, "qmap_t: input shape");
    const int64_t PO = O * (O - 1) / 2, PV = V * (V - 1) / 2;
    if (PO == 0 || PV == 0) {
        if (beta.x == 0.0 && beta.y == 0.0) fill(D, Xb, mkc(0.0));
        else axpby(D, mkc(0.0), Xb, false, beta, Xb);
        return;
    }
    Tensor Qt = empty(D, {V * O, R * PO});
    k_pack_q<<<grid_of(D, R * V * O * O * O), 256, 0, D.st>>>(Qb.p, Qt.p, R, V, O);
    LAUNCH_CHECK(D);
    Tensor Zt = empty(D, {R * PO, PV});
    if (ensure_qcache(D, LC, prec)) {
        ein(D, "xn,xk->nk", mkc(1.0), Qt, false, LC.wq64, false, mkc(0.0), Zt, prec);
        ladder_unpack_zt(D, Zt.p, Xb.p, R, O, V, alpha, beta);
        return;
    }
    const int64_t na = slab_a(D, O, V);
    Tensor GT = empty(D, {O * V * na * V});
    Tensor W = empty(D, {na * O, PV});
    for (int64_t a0 = 0; a0 < V; a0 += na) {
        const int64_t n = std::min(na, V - a0);
        Tensor Ws = W.slice(0, 0, n * O);
        assemble_q(D, LC, a0, n, prec, GT, Ws);
        // Xbar_ijef (i<j, e<f) = sum_am Qbar_amij <am||ef>
        ein(D, "xn,xk->nk", mkc(1.0), Qt.slice(0, a0 * O, n * O), false, Ws, false, mkc(a0 == 0 ? 0.0 : 1.0), Zt,
            prec);
    }
    ladder_unpack_zt(D, Zt.p, Xb.p, R, O, V, alpha, beta);
}
