// FNS++: perturbation-sensitive frozen natural spinors (Sec. II.B-C of the
// paper), entirely on the device.
//
//  1. MP2 doubles t_ij^ab = <ab||ij> / (e_i + e_j - e_a - e_b)           (Eq. 39)
//  2. Hbar_ii = f_ii + 1/2 sum_nef t_in^ef <in||ef>,
//     Hbar_aa = f_aa - 1/2 sum_mnf t_mn^fa <mn||fa>   (real parts)       (Eq. 49-50)
//  3. per dipole component A: Abar = xi^A at T1 = 0, T2 = MP2 (the one-body
//     residual; its doubles block is Eq. 48, its singles block
//     A_ai + sum_me A_me t_im^ae), t^(1) = Abar / (Dbar - omega)       (Eq. 46-48)
//  4. M_ab = 1/3 sum_A [1/2 sum_ijc t_ij^ac conj t_ij^bc + sum_i t_i^a conj t_i^b]   (Eq. 45)
//  5. natural spinors = eigenvectors of M (Eq. 41); keep by |n| descending
//  6. Ftilde = Vt^H F_vv Vt, its eigenvectors Z (Eq. 42-43), U = Vt Z (Eq. 44)
//  7. rotate B^L and mu with diag(1_O, U); virtual energies = eig(Ftilde).
//
// Plain FNS (options.fns_density = 1) takes the ground-state MP2 virtual
// density M_ab = 1/2 sum_ijc t_ij^ac conj t_ij^bc (Eq. 40) in place of 3-4.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "ctx.h"

namespace {

int grid_n(Dev& D, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)D.sm_count * 16));
}

// out[p] = base[p] + scale * Re(in[p])
__global__ void k_real_axpy(int64_t n, const double* base, double scale, const cplx* in, double* out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        out[p] = base[p] + scale * in[p].x;
}

// dst[p][j] = src[p][idx[j]]
__global__ void k_gather_cols(int64_t n, int64_t m, const cplx* src, const int* idx, cplx* dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * m; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = e / m, j = e % m;
        dst[e] = src[p * n + idx[j]];
    }
}

// diag(v) as a complex matrix
__global__ void k_diag(int64_t n, const double* v, cplx* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = e / n, q = e % n;
        out[e] = make_double2(p == q ? v[p] : 0.0, 0.0);
    }
}

struct DevDoubles {
    std::shared_ptr<DevBuf> hold;
    double* p = nullptr;
};

DevDoubles dev_doubles(Dev& D, const std::vector<double>& v) {
    DevDoubles d;
    size_t n = sizeof(double) * std::max<size_t>(1, v.size());
    d.p = (double*)D.pool.get(n);
    d.hold.reset(new DevBuf{&D.pool, d.p, n});
    CK(cudaMemcpyAsync(d.p, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, D.st));
    return d;
}

#define CS(x)                                                                                        \
    do {                                                                                             \
        cusolverStatus_t s_ = (x);                                                                   \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                           \
            throw LrccError(LRCC_ECUDA, std::string(#x) + " failed: " + std::to_string((int)s_));  \
    } while (0)

// Hermitian eigen-decomposition of A [n][n] (row-major).  Returns eigenvalues
// ascending and the eigenvectors as the COLUMNS of a new row-major [n][n].
// The row-major Hermitian matrix read column-major is conj(A); the solver's
// eigenvectors of conj(A) are the conjugates of those of A.
Tensor eigh(Dev& D, const Tensor& A, std::vector<double>& w) {
    int64_t n = A.d[0];
    REQUIRE(A.nd == 2 && A.d[1] == n && n < INT32_MAX, "eigh: square matrix expected");
    Tensor W = empty(D, {n, n});
    axpby(D, mkc(1.0), A, false, mkc(0.0), W);
    cusolverDnHandle_t h = nullptr;
    CS(cusolverDnCreate(&h));
    std::shared_ptr<void> guard(nullptr, [h](void*) { cusolverDnDestroy(h); });
    CS(cusolverDnSetStream(h, D.st));
    double* wd = (double*)D.pool.get(sizeof(double) * n);
    std::shared_ptr<DevBuf> hw(new DevBuf{&D.pool, wd, sizeof(double) * (size_t)n});
    int lwork = 0;
    CS(cusolverDnZheevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)n,
                                   (cuDoubleComplex*)W.p, (int)n, wd, &lwork));
    size_t wb = sizeof(cuDoubleComplex) * std::max(lwork, 1);
    void* work = D.pool.get(wb);
    std::shared_ptr<DevBuf> hwork(new DevBuf{&D.pool, work, wb});
    int* info = (int*)D.pool.get(sizeof(int));
    std::shared_ptr<DevBuf> hinfo(new DevBuf{&D.pool, info, sizeof(int)});
    CS(cusolverDnZheevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)n, (cuDoubleComplex*)W.p, (int)n,
                        wd, (cuDoubleComplex*)work, lwork, info));
    int hinfo_v = 0;
    w.resize(n);
    CK(cudaMemcpyAsync(w.data(), wd, sizeof(double) * n, cudaMemcpyDeviceToHost, D.st));
    CK(cudaMemcpyAsync(&hinfo_v, info, sizeof(int), cudaMemcpyDeviceToHost, D.st));
    CK(cudaStreamSynchronize(D.st));
    if (hinfo_v != 0) throw LrccError(LRCC_ECUDA, "zheevd info = " + std::to_string(hinfo_v));
    // W (column-major) column k = eigenvector k of conj(A): row k of W viewed row-major.
    Tensor Vn = empty(D, {n, n});
    axpby(D, mkc(1.0), W.permute({1, 0}), true, mkc(0.0), Vn);
    return Vn;
}

Tensor block(Dev& D, const Tensor& M, int64_t r0, int64_t nr, int64_t c0, int64_t nc) {
    Tensor out = empty(D, {nr, nc});
    axpby(D, mkc(1.0), M.slice(0, r0, nr).slice(1, c0, nc), false, mkc(0.0), out);
    return out;
}

}  // namespace

// one-body residual program of component k in the context's current basis
static void one_body_program(lrcc_ctx* c, int k, CCProg& cp) {
    Dev& D = c->D;
    int O = c->O, V = c->V;
    Ham h;
    h.w = false;
    Tensor M = c->mu.index(k);
    h.foo = block(D, M, 0, O, 0, O);
    h.fov = block(D, M, 0, O, O, V);
    h.fvo = block(D, M, O, V, 0, O);
    h.fvv = block(D, M, O, V, O, V);
    build_ccsd(cp, h, nullptr);
}

// MP2 doubles t_ij^ab = -<ab||ij> / (e_a + e_b - e_i - e_j) (Eq. 39) as one
// amplitude set with t1 = 0; eo/ev: device orbital energies
static Amp mp2_doubles_dev(Dev& D, const Tensor& B, int64_t O, int64_t V, const double* eo, const double* ev) {
    Amp t = amp_zeros(D, 1, O, V);
    Tensor vvoo = anti_block(D, B, O, V, O, V, 0, O, 0, O);
    Amp r = amp_zeros(D, 1, O, V);
    Tensor r2 = r.t2.index(0);
    perm_axpby(D, "abij->ijab", mkc(1.0), vvoo, mkc(0.0), r2);
    std::vector<double> zero(1, 0.0);
    DevDoubles z0 = dev_doubles(D, zero);
    precond(D, nullptr, r, t, eo, ev, z0.p);
    return t;
}

// Hbar diagonals of Eq. 49-50 (real parts) into the device arrays Hii [O] and
// Haa [V], and the MP2 energy 1/4 sum <ij||ab> t_ij^ab (Eq. 51) into *e_mp2
// (host; the copy is complete when this returns)
static void hbar_diagonals_dev(Dev& D, const Tensor& B, int64_t O, int64_t V, const Amp& t, const double* eo,
                               const double* ev, double* Hii, double* Haa, cplx* e_mp2) {
    Tensor oovv = anti_block(D, B, 0, O, 0, O, O, V, O, V);
    Tensor t2 = t.t2.index(0);
    Tensor ef = ein_new(D, "ijab,ijab->", mkc(0.25), oovv, false, t2, false);
    CK(cudaMemcpyAsync(e_mp2, ef.p, sizeof(cplx), cudaMemcpyDeviceToHost, D.st));
    Tensor si = ein_new(D, "inef,inef->i", mkc(1.0), t2, false, oovv, false);
    Tensor sa = ein_new(D, "mnfa,mnfa->a", mkc(1.0), t2, false, oovv, false);
    k_real_axpy<<<grid_n(D, O), 256, 0, D.st>>>(O, eo, 0.5, si.p, Hii);
    LAUNCH_CHECK(D);
    k_real_axpy<<<grid_n(D, V), 256, 0, D.st>>>(V, ev, -0.5, sa.p, Haa);
    LAUNCH_CHECK(D);
    CK(cudaStreamSynchronize(D.st));
}

void fns_truncate_impl(lrcc_ctx* c, int by_count, double value, double omega, int* v_kept, double* occ_out) {
    Dev& D = c->D;
    const int64_t O = c->O, V = c->V, L = c->L, N = O + V;
    REQUIRE(std::isfinite(value) && std::isfinite(omega), "fns: value and omega must be finite");
    if (by_count) REQUIRE(value >= 1.0 && std::llround(value) <= V, "fns: count out of range");
    else REQUIRE(value >= 0.0, "fns: threshold must be >= 0");
    const Tensor& B = c->B;
    std::vector<double> eo(c->eps.begin(), c->eps.begin() + O), ev(c->eps.begin() + O, c->eps.end());
    DevDoubles deo = dev_doubles(D, eo), dev = dev_doubles(D, ev);

    // 1. MP2 doubles
    Amp t = mp2_doubles_dev(D, B, O, V, deo.p, dev.p);
    // 2. Hbar diagonals (and the full-space MP2 energy, Eq. 51)
    DevDoubles Hii = dev_doubles(D, eo), Haa = dev_doubles(D, ev);
    cplx e_full = mkc(0.0);
    hbar_diagonals_dev(D, B, O, V, t, deo.p, dev.p, Hii.p, Haa.p, &e_full);
    // 3-4. first-order amplitudes per component and the averaged density
    // (plain FNS: the MP2 density of the doubles of step 1)
    Tensor M = zeros(D, {V, V});
    if (c->opt.fns_density == 1) {
        Tensor t2 = t.t2.index(0);
        ein(D, "ijac,ijbc->ab", mkc(0.5), t2, false, t2, true, mkc(1.0), M);
    } else {
        std::vector<double> sh(1, omega * (c->opt.plus_omega ? 1.0 : -1.0));
        DevDoubles dsh = dev_doubles(D, sh);
        for (int k = 0; k < c->ncomp; ++k) {
            CCProg cp;
            one_body_program(c, k, cp);
            cp.P.eval(D, {t.t1.index(0), t.t2.index(0)}, LRCC_FP64);
            Amp abar{cp.P.val[cp.R1].reshape({1, O, V}), cp.P.val[cp.R2].reshape({1, O, O, V, V})};
            Amp tp = amp_empty(D, 1, O, V);
            precond(D, nullptr, abar, tp, Hii.p, Haa.p, dsh.p);  // -Abar/(Dbar -/+ omega); sign drops out of M
            Tensor t1p = tp.t1.index(0), t2p = tp.t2.index(0);
            double w = 1.0 / c->ncomp;
            ein(D, "ijac,ijbc->ab", mkc(0.5 * w), t2p, false, t2p, true, mkc(1.0), M);
            ein(D, "ia,ib->ab", mkc(w), t1p, false, t1p, true, mkc(1.0), M);
        }
    }
    // 5. natural spinors
    std::vector<double> n;
    Tensor Vn = eigh(D, M, n);
    std::vector<int> order(V);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(n[a]) > std::fabs(n[b]); });
    std::vector<int> keep;
    if (by_count) {
        keep.assign(order.begin(), order.begin() + std::llround(value));
    } else {
        for (int a : order)
            if (std::fabs(n[a]) >= value) keep.push_back(a);
        REQUIRE(!keep.empty(), "fns: threshold removes every virtual spinor");
    }
    if (occ_out)
        for (int64_t a = 0; a < V; ++a) occ_out[a] = std::fabs(n[order[a]]);
    const int64_t Vk = (int64_t)keep.size();
    Tensor Vt = empty(D, {V, Vk});
    {
        int* idx = (int*)D.pool.get(sizeof(int) * Vk);
        std::shared_ptr<DevBuf> hi(new DevBuf{&D.pool, idx, sizeof(int) * (size_t)Vk});
        CK(cudaMemcpyAsync(idx, keep.data(), sizeof(int) * Vk, cudaMemcpyHostToDevice, D.st));
        k_gather_cols<<<grid_n(D, V * Vk), 256, 0, D.st>>>(V, Vk, Vn.p, idx, Vt.p);
        LAUNCH_CHECK(D);
        CK(cudaStreamSynchronize(D.st));
    }
    // 6. semicanonical virtuals
    Tensor Fvv = empty(D, {V, V});
    k_diag<<<grid_n(D, V * V), 256, 0, D.st>>>(V, dev.p, Fvv.p);
    LAUNCH_CHECK(D);
    Tensor FV = ein_new(D, "pq,qb->pb", mkc(1.0), Fvv, false, Vt, false);
    Tensor Ft = ein_new(D, "pa,pb->ab", mkc(1.0), Vt, true, FV, false);
    std::vector<double> et;
    Tensor Z = eigh(D, Ft, et);
    Tensor U = ein_new(D, "pa,ab->pb", mkc(1.0), Vt, false, Z, false);   // [V][Vk]
    // 7. rotate B and mu with diag(1_O, U):  X' = Uf^H X Uf
    const int64_t Nk = O + Vk;
    auto rotate = [&](const Tensor& X) {
        int64_t nl = X.d[0];
        Tensor Y = empty(D, {nl, Nk, Nk});
        Tensor yoo = Y.slice(1, 0, O).slice(2, 0, O), yov = Y.slice(1, 0, O).slice(2, O, Vk);
        Tensor yvo = Y.slice(1, O, Vk).slice(2, 0, O), yvv = Y.slice(1, O, Vk).slice(2, O, Vk);
        axpby(D, mkc(1.0), X.slice(1, 0, O).slice(2, 0, O), false, mkc(0.0), yoo);
        ein(D, "Lia,ab->Lib", mkc(1.0), X.slice(1, 0, O).slice(2, O, V), false, U, false, mkc(0.0), yov);
        ein(D, "Lai,ab->Lbi", mkc(1.0), X.slice(1, O, V).slice(2, 0, O), false, U, true, mkc(0.0), yvo);
        // U^H X_vv U in chunks over L to bound the intermediate
        int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nl, (int64_t(2) << 30) / (16 * V * Vk)));
        for (int64_t l0 = 0; l0 < nl; l0 += chunk) {
            int64_t nc = std::min(chunk, nl - l0);
            Tensor tmp = ein_new(D, "Lac,cd->Lad", mkc(1.0), X.slice(0, l0, nc).slice(1, O, V).slice(2, O, V), false,
                                 U, false);
            Tensor dst = yvv.slice(0, l0, nc);
            ein(D, "Lad,ab->Lbd", mkc(1.0), tmp, false, U, true, mkc(0.0), dst);
        }
        return Y;
    };
    Tensor Bn = rotate(B);
    Tensor mun = rotate(c->mu);
    // MP2 energy in the truncated semicanonical basis (Eq. 51)
    cplx e_trunc = mkc(0.0);
    {
        std::vector<double> etv(et.begin(), et.end());
        DevDoubles det = dev_doubles(D, etv);
        Tensor vvoo = anti_block(D, Bn, O, Vk, O, Vk, 0, O, 0, O);
        Tensor oovv = anti_block(D, Bn, 0, O, 0, O, O, Vk, O, Vk);
        Amp r = amp_zeros(D, 1, O, Vk), tt = amp_zeros(D, 1, O, Vk);
        Tensor r2 = r.t2.index(0);
        perm_axpby(D, "abij->ijab", mkc(1.0), vvoo, mkc(0.0), r2);
        std::vector<double> zero(1, 0.0);
        DevDoubles z0 = dev_doubles(D, zero);
        precond(D, nullptr, r, tt, deo.p, det.p, z0.p);
        Tensor tt2 = tt.t2.index(0);
        Tensor e = ein_new(D, "ijab,ijab->", mkc(0.25), oovv, false, tt2, false);
        CK(cudaMemcpyAsync(&e_trunc, e.p, sizeof(cplx), cudaMemcpyDeviceToHost, D.st));
    }
    CK(cudaStreamSynchronize(D.st));
    c->e_mp2_full = e_full;
    c->e_mp2_trunc = e_trunc;
    c->truncated = true;
    // 8. replace the virtual space
    c->B = Bn;
    c->mu = mun;
    c->V = (int)Vk;
    std::vector<double> eps(c->eps.begin(), c->eps.begin() + O);
    eps.insert(eps.end(), et.begin(), et.end());
    c->eps = eps;
    c->ham_built = false;
    c->ground = false;
    c->linearized = false;
    c->cc.reset();
    c->ccfx.reset();
    c->ccmu.clear();
    c->H = Ham();
    c->Hmu.clear();
    c->lad = LadderCtx();
    c->T = Amp();
    c->Lam = Amp();
    D.pool.trim();
    if (v_kept) *v_kept = (int)Vk;
    (void)L;
    (void)N;
}

// MP2-level polarisability in the context's current virtual basis (the
// ingredient of Delta alpha_MP2, Eq. 53-54): the sum over the singly and doubly
// excited determinants mu of the response function of Eq. 18 with the Eq. 48
// transition moments Abar_mu (one-body residual at T1 = 0, T2 = MP2) and the
// Eq. 47 excitation energies Dbar_mu:
//   alpha_AB(w) = P_AB(w) + conj P_AB(-w),
//   P_AB(w) = sum_mu conj(Abar_mu) Bbar_mu / (Dbar_mu - w)      (unique mu)
static void mp2_alpha_impl(lrcc_ctx* c, const double* omegas, int n_w, const int* comps, int n_c, double* alpha) {
    Dev& D = c->D;
    const int64_t O = c->O, V = c->V;
    REQUIRE(omegas && comps && alpha && n_w >= 1 && n_c >= 1, "mp2_alpha: null array or empty list");
    for (int k = 0; k < n_c; ++k) REQUIRE(comps[k] >= 0 && comps[k] < c->ncomp, "mp2_alpha: component out of range");
    for (int w = 0; w < n_w; ++w) REQUIRE(std::isfinite(omegas[w]), "mp2_alpha: frequency not finite");
    std::vector<double> eo(c->eps.begin(), c->eps.begin() + O), ev(c->eps.begin() + O, c->eps.end());
    DevDoubles deo = dev_doubles(D, eo), dev = dev_doubles(D, ev);
    Amp t = mp2_doubles_dev(D, c->B, O, V, deo.p, dev.p);
    DevDoubles Hii = dev_doubles(D, eo), Haa = dev_doubles(D, ev);
    cplx e_mp2 = mkc(0.0);
    hbar_diagonals_dev(D, c->B, O, V, t, deo.p, dev.p, Hii.p, Haa.p, &e_mp2);
    // every |w| must stay below the lowest Dbar (singles: min Haa - max Hii;
    // doubles: the two lowest Haa minus the two highest Hii)
    {
        std::vector<double> hi(O), ha(V);
        CK(cudaMemcpyAsync(hi.data(), Hii.p, sizeof(double) * O, cudaMemcpyDeviceToHost, D.st));
        CK(cudaMemcpyAsync(ha.data(), Haa.p, sizeof(double) * V, cudaMemcpyDeviceToHost, D.st));
        CK(cudaStreamSynchronize(D.st));
        std::sort(hi.begin(), hi.end());
        std::sort(ha.begin(), ha.end());
        double d1 = ha[0] - hi[O - 1], d2 = ha[0] + ha[1] - hi[O - 1] - hi[O - 2];
        double lo = std::min(d1, d2);
        for (int w = 0; w < n_w; ++w)
            REQUIRE(std::fabs(omegas[w]) < lo, "mp2_alpha: |omega| must lie below the lowest Hbar excitation energy");
    }
    std::vector<Amp> mom(n_c);
    for (int k = 0; k < n_c; ++k) {
        CCProg cp;
        one_body_program(c, comps[k], cp);
        cp.P.eval(D, {t.t1.index(0), t.t2.index(0)}, LRCC_FP64);
        Amp abar{cp.P.val[cp.R1].reshape({1, O, V}), cp.P.val[cp.R2].reshape({1, O, O, V, V})};
        mom[k] = amp_copy(D, abar);
    }
    // P[w][sign][A][B], sign 0: +w, 1: -w
    std::vector<cplx> P((size_t)n_w * 2 * n_c * n_c);
    Amp tp = amp_empty(D, 1, O, V);
    for (int w = 0; w < n_w; ++w)
        for (int sg = 0; sg < 2; ++sg) {
            std::vector<double> shv(1, sg ? omegas[w] : -omegas[w]);
            DevDoubles sh = dev_doubles(D, shv);
            for (int b = 0; b < n_c; ++b) {
                precond(D, nullptr, mom[b], tp, Hii.p, Haa.p, sh.p);   // tp = -Bbar / (Dbar -/+ w)
                for (int a = 0; a < n_c; ++a) {
                    Tensor d = amp_dot(D, mom[a], true, tp);
                    cplx v = mkc(0.0);
                    CK(cudaMemcpyAsync(&v, d.p, sizeof(cplx), cudaMemcpyDeviceToHost, D.st));
                    CK(cudaStreamSynchronize(D.st));
                    P[(((size_t)w * 2 + sg) * n_c + a) * n_c + b] = make_double2(-v.x, -v.y);
                }
            }
        }
    for (int w = 0; w < n_w; ++w)
        for (int a = 0; a < n_c; ++a)
            for (int b = 0; b < n_c; ++b) {
                const cplx p = P[(((size_t)w * 2 + 0) * n_c + a) * n_c + b];
                const cplx m = P[(((size_t)w * 2 + 1) * n_c + a) * n_c + b];
                double* out = alpha + 2 * (((size_t)w * n_c + a) * n_c + b);
                out[0] = p.x + m.x;
                out[1] = p.y - m.y;
            }
}

extern "C" lrcc_status lrcc_mp2_alpha(lrcc_ctx* c, const double* omegas, int n_w, const int* comps, int n_c,
                                      double* alpha) {
    if (!c) return LRCC_EINVAL;
    try {
        mp2_alpha_impl(c, omegas, n_w, comps, n_c, alpha);
        return LRCC_OK;
    } catch (const LrccError& e) {
        c->err = e.what();
        return e.st;
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

extern "C" lrcc_status lrcc_fns_truncate(lrcc_ctx* c, int by_count, double value, double omega, int* v_kept,
                                         double* occ_out) {
    if (!c) return LRCC_EINVAL;
    try {
        fns_truncate_impl(c, by_count, value, omega, v_kept, occ_out);
        return LRCC_OK;
    } catch (const LrccError& e) {
        c->err = e.what();
        return e.st;
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

extern "C" lrcc_status lrcc_mp2_correction(const lrcc_ctx* c, double e_full[2], double e_trunc[2], double delta[2]) {
    if (!c) return LRCC_EINVAL;
    if (!c->truncated) return LRCC_ESTATE;
    if (e_full) { e_full[0] = c->e_mp2_full.x; e_full[1] = c->e_mp2_full.y; }
    if (e_trunc) { e_trunc[0] = c->e_mp2_trunc.x; e_trunc[1] = c->e_mp2_trunc.y; }
    if (delta) {
        delta[0] = c->e_mp2_full.x - c->e_mp2_trunc.x;
        delta[1] = c->e_mp2_full.y - c->e_mp2_trunc.y;
    }
    return LRCC_OK;
}
