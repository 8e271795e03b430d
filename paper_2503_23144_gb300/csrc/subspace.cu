// Shared-subspace solver for the shifted response systems (an option of the
// library; the paper does not state its solver).
//
// All R right-hand sides (M + s_r) z_r = -b_r of one batch -- every frequency
// and every component -- share one subspace V with orthonormal columns in the
// unique-amplitude Hermitian product <u, w> = sum_ia conj(u) w +
// 1/4 sum_ijab conj(u) w.  Each product M v is taken once and serves every
// shift and right-hand side:
//
//   G = V^H M V,   (G + s_r I) y_r = -V^H b_r   (Galerkin),   z_r = V y_r,
//   r_r = (M V) y_r + s_r z_r + b_r             (no further product),
//
// and the residuals of the unconverged right-hand sides, through the diagonal
// preconditioner (D + s_r)^-1, are orthonormalised against V (classical
// Gram-Schmidt, twice) and appended.  When V is full it restarts: the current
// solutions become a fixed base z0, and the next subspace solves for the
// correction, (M + s_r) d_r = -(residual of z0_r).  Frequencies of one
// component thus share their products instead of each iterating on its own.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <limits>

#include "solver.h"

namespace {

using zc = std::complex<double>;
static_assert(sizeof(zc) == sizeof(cplx), "complex layout");

std::vector<zc> to_host(Dev& D, const Tensor& t) {
    std::vector<zc> h((size_t)t.numel());
    CK(cudaMemcpyAsync(h.data(), t.p, sizeof(cplx) * h.size(), cudaMemcpyDeviceToHost, D.st));
    CK(cudaStreamSynchronize(D.st));
    return h;
}

Tensor to_dev(Dev& D, const std::vector<zc>& h, int64_t rows, int64_t cols) {
    Tensor t = empty(D, {rows, cols});
    CK(cudaMemcpyAsync(t.p, h.data(), sizeof(cplx) * h.size(), cudaMemcpyHostToDevice, D.st));
    CK(cudaStreamSynchronize(D.st));
    return t;
}

// G[p][q] = <U_p, W_q>; prec: LRCC_FP64 or LRCC_FP64_EMULATED products
std::vector<zc> hgram(Dev& D, const Amp& U, const Amp& W, int prec) {
    const int64_t P = U.t1.d[0], Q = W.t1.d[0];
    Tensor G = empty(D, {P, Q});
    ein(D, "Pia,Qia->PQ", mkc(1.0), U.t1, true, W.t1, false, mkc(0.0), G, prec);
    ein(D, "Pijab,Qijab->PQ", mkc(0.25), U.t2, true, W.t2, false, mkc(1.0), G, prec);
    return to_host(D, G);
}

// out_q = beta out_q + sum_p C[p][q] V_p,  C [P][Q] on the host
void lincomb(Dev& D, const Amp& Vb, const std::vector<zc>& C, int64_t P, int64_t Q, cplx beta, Amp& out, int prec) {
    Tensor Cd = to_dev(D, C, P, Q);
    ein(D, "Pia,PQ->Qia", mkc(1.0), Vb.t1, false, Cd, false, beta, out.t1, prec);
    ein(D, "Pijab,PQ->Qijab", mkc(1.0), Vb.t2, false, Cd, false, beta, out.t2, prec);
}

// b <- A^-1 b for A [n][n] (row-major, taken by value): Gaussian elimination
// with partial pivoting; false if A is singular
bool lu_solve(std::vector<zc> A, std::vector<zc>& b, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double best = std::abs(A[k * n + k]);
        for (int64_t i = k + 1; i < n; ++i)
            if (std::abs(A[i * n + k]) > best) {
                best = std::abs(A[i * n + k]);
                p = i;
            }
        if (!(best > 0.0) || !std::isfinite(best)) return false;
        if (p != k) {
            for (int64_t j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
            std::swap(b[k], b[p]);
        }
        for (int64_t i = k + 1; i < n; ++i) {
            const zc f = A[i * n + k] / A[k * n + k];
            if (f == zc(0.0)) continue;
            for (int64_t j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        zc s = b[i];
        for (int64_t j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
    return true;
}

// Coefficients T [k][m] such that Q = C T has orthonormal columns, by modified
// Gram-Schmidt (two sweeps per column) in the metric G = C^H C; column j is
// dropped when its remaining norm is below drop * ref[j].
std::vector<zc> orth_coeffs(const std::vector<zc>& G, int64_t k, const std::vector<double>& ref, double drop,
                            int64_t& m) {
    std::vector<std::vector<zc>> kept;
    auto gdot = [&](const std::vector<zc>& u, const std::vector<zc>& w) {  // u^H G w
        zc s = 0.0;
        for (int64_t a = 0; a < k; ++a) {
            zc gw = 0.0;
            for (int64_t c = 0; c < k; ++c) gw += G[a * k + c] * w[c];
            s += std::conj(u[a]) * gw;
        }
        return s;
    };
    for (int64_t j = 0; j < k; ++j) {
        std::vector<zc> t(k, zc(0.0));
        t[j] = 1.0;
        for (int sweep = 0; sweep < 2; ++sweep)
            for (const auto& q : kept) {
                const zc h = gdot(q, t);
                for (int64_t a = 0; a < k; ++a) t[a] -= h * q[a];
            }
        const double nn = std::sqrt(std::max(gdot(t, t).real(), 0.0));
        if (!(nn > drop * ref[j]) || !std::isfinite(nn)) continue;
        for (auto& x : t) x /= nn;
        kept.push_back(t);
    }
    m = (int64_t)kept.size();
    std::vector<zc> T((size_t)(k * std::max<int64_t>(m, 1)), zc(0.0));
    for (int64_t q = 0; q < m; ++q)
        for (int64_t a = 0; a < k; ++a) T[a * m + q] = kept[q][a];
    return T;
}

// Orthonormalise the candidates C against V[0, n) and among themselves, in
// two rounds: projection against V (two classical Gram-Schmidt passes in the
// first round, one in the second), then Gram-matrix Gram-Schmidt within the
// block.  A candidate whose part outside the span of V and of the candidates
// before it is below 1e-3 of its norm is dropped: it would add almost nothing,
// and its rescaling would magnify the rounding of the projections.  The kept
// vectors are written to V[n, n + m).  Returns m.
int64_t extend_basis(Dev& D, int O, int V, Amp& Vs, int64_t n, const Amp& C0, int prec) {
    Amp C = amp_copy(D, C0);
    int64_t k = C0.t1.d[0];
    std::vector<double> ref(k);
    {
        const std::vector<zc> g0 = hgram(D, C, C, prec);
        for (int64_t j = 0; j < k; ++j) ref[j] = std::sqrt(std::max(g0[j * k + j].real(), 0.0));
    }
    for (int round = 0; round < 2 && k > 0; ++round) {
        if (n > 0) {
            const Amp Vo = amp_rows(Vs, 0, n);
            for (int pass = 0; pass < (round == 0 ? 2 : 1); ++pass) {
                std::vector<zc> H = hgram(D, Vo, C, prec);  // [n][k]
                for (auto& h : H) h = -h;
                lincomb(D, Vo, H, n, k, mkc(1.0), C, prec);
            }
        }
        const std::vector<zc> G = hgram(D, C, C, prec);
        int64_t m = 0;
        const std::vector<zc> T = orth_coeffs(G, k, ref, 1e-3, m);
        if (m == 0) return 0;
        Amp Q = amp_empty(D, m, O, V);
        lincomb(D, C, T, k, m, mkc(0.0), Q, prec);
        C = Q;
        k = m;
        ref.assign(k, 1.0);
    }
    if (k > 0) {
        Amp dst = amp_rows(Vs, n, k);
        amp_axpby(D, mkc(1.0), C, mkc(0.0), dst);
    }
    return k;
}

// rows idx of x, as a new batch
Amp gather_rows(Dev& D, int O, int V, const Amp& x, const std::vector<int64_t>& idx) {
    Amp out = amp_empty(D, (int64_t)idx.size(), O, V);
    for (size_t q = 0; q < idx.size(); ++q) {
        Amp src = amp_rows(x, idx[q], 1), dst = amp_rows(out, (int64_t)q, 1);
        amp_axpby(D, mkc(1.0), src, mkc(0.0), dst);
    }
    return out;
}

}  // namespace

int64_t subspace_capacity(Dev& D, int O, int V, int64_t R, int requested) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    const double vb = 16.0 * ((double)O * V + (double)O * O * V * V);
    const double avail = 0.3 * (double)(fr + D.pool.cached);
    const int64_t by_mem = (int64_t)(avail / (2.0 * vb));
    const int64_t want = requested > 0 ? requested : std::min<int64_t>(400, std::max<int64_t>(48, 8 * R));
    if (want < 2 * R)
        throw LrccError(LRCC_EINVAL, "subspace_max must hold at least 2 x " + std::to_string(R) + " vectors");
    if (by_mem < 2 * R)
        throw LrccError(LRCC_ENOMEM, "shared-subspace solver: no room for 2 x " + std::to_string(R) + " vectors");
    return std::min(want, by_mem);
}

void subspace_solve(Dev& D, int O, int V, const double* eo, const double* ev, Amp& z, const Amp& b,
                    const double* shift_dev, const std::vector<double>& shift,
                    const std::function<Amp(const Amp&)>& apply, int prec, double tol, int max_iter,
                    int requested_max, std::vector<double>& final_res, int& n_products) {
    const int64_t R = b.t1.d[0];
    const int64_t nmax = subspace_capacity(D, O, V, R, requested_max);
    static const bool verbose = getenv("LRCC_VERBOSE") != nullptr;
    std::vector<double> rn;
    max_abs_amp(D, b, rn);  // the residual of z = 0
    if (*std::max_element(rn.begin(), rn.end()) < tol) {
        fill(D, z.t1, mkc(0.0));
        fill(D, z.t2, mkc(0.0));
        final_res = rn;
        return;
    }
    Amp Vs = amp_empty(D, nmax, O, V), AVs = amp_empty(D, nmax, O, V);
    int64_t n = 0;
    std::vector<zc> G;   // [n][n]  <v_p, M v_q>
    std::vector<zc> Vb;  // [n][R]  <v_p, be_r>
    // z = zb + V y solves (M + s) z = -b when (M + s)(V y) = -be with
    // be = b + (M + s) zb; zb = 0, be = b until the first restart
    Amp zb = amp_zeros(D, R, O, V), be = amp_copy(D, b);
    Amp cand = amp_empty(D, R, O, V);
    precond(D, nullptr, be, cand, eo, ev, shift_dev);  // -b / (D + s)
    Amp res = amp_empty(D, R, O, V), pre = amp_empty(D, R, O, V), S = amp_empty(D, R, O, V),
        dz = amp_empty(D, R, O, V);
    for (int it = 0; it < max_iter; ++it) {
        // restart when the candidates do not fit: the current solutions become
        // the base and their residuals the new right-hand sides
        if (n + cand.t1.d[0] > nmax) {
            amp_axpby(D, mkc(1.0), z, mkc(0.0), zb);
            amp_axpby(D, mkc(1.0), res, mkc(0.0), be);
            n = 0;
            G.clear();
            Vb.clear();
            if (verbose) fprintf(stderr, "  subspace restart at iteration %d\n", it);
        }
        const int64_t m = extend_basis(D, O, V, Vs, n, cand, prec);
        if (m == 0) throw LrccError(LRCC_ENOCONV, "shared-subspace solver stagnated (no new direction)");
        const Amp Vn = amp_rows(Vs, n, m);
        {
            Amp prod = apply(Vn);
            ++n_products;
            Amp dst = amp_rows(AVs, n, m);
            amp_axpby(D, mkc(1.0), prod, mkc(0.0), dst);
        }
        const int64_t n1 = n + m;
        // projected matrix and right-hand sides, extended by the new rows and columns
        {
            const std::vector<zc> cols = hgram(D, amp_rows(Vs, 0, n1), amp_rows(AVs, n, m), prec);  // [n1][m]
            std::vector<zc> rows;                                                                   // [m][n]
            if (n > 0) rows = hgram(D, Vn, amp_rows(AVs, 0, n), prec);
            std::vector<zc> G1((size_t)(n1 * n1));
            for (int64_t p = 0; p < n; ++p)
                for (int64_t q = 0; q < n; ++q) G1[p * n1 + q] = G[p * n + q];
            for (int64_t p = 0; p < n1; ++p)
                for (int64_t q = 0; q < m; ++q) G1[p * n1 + n + q] = cols[p * m + q];
            for (int64_t p = 0; p < m; ++p)
                for (int64_t q = 0; q < n; ++q) G1[(n + p) * n1 + q] = rows[p * n + q];
            G.swap(G1);
            const std::vector<zc> vb = hgram(D, Vn, be, prec);  // [m][R]
            Vb.insert(Vb.end(), vb.begin(), vb.end());
        }
        n = n1;
        // Galerkin solution of every right-hand side in the subspace
        std::vector<zc> Y((size_t)(n * R));
        for (int64_t r = 0; r < R; ++r) {
            std::vector<zc> A(G);
            for (int64_t p = 0; p < n; ++p) A[p * n + p] += shift[r];
            std::vector<zc> y(n);
            for (int64_t p = 0; p < n; ++p) y[p] = -Vb[p * R + r];
            if (!lu_solve(A, y, n)) throw LrccError(LRCC_ENOCONV, "shared-subspace solver: singular projected matrix");
            for (int64_t p = 0; p < n; ++p) Y[p * R + r] = y[p];
        }
        lincomb(D, amp_rows(Vs, 0, n), Y, n, R, mkc(0.0), dz, prec);
        lincomb(D, amp_rows(AVs, 0, n), Y, n, R, mkc(0.0), S, prec);
        combine(D, S, dz, shift_dev, &be, res);  // (M + s) dz + be = (M + s) z + b
        amp_axpby(D, mkc(1.0), zb, mkc(0.0), z);
        amp_axpby(D, mkc(1.0), dz, mkc(1.0), z);
        max_abs_amp(D, res, rn);
        const double worst = *std::max_element(rn.begin(), rn.end());
        if (verbose)
            fprintf(stderr, "  subspace iter %3d  n=%lld  max|r| = %.3e\n", it, (long long)n, worst);
        if (!std::isfinite(worst) || worst > 1e250) throw LrccError(LRCC_ENOCONV, "residual is not finite");
        if (worst < tol) {
            final_res = rn;
            return;
        }
        precond(D, nullptr, res, pre, eo, ev, shift_dev);
        std::vector<int64_t> open;
        for (int64_t r = 0; r < R; ++r)
            if (rn[r] >= tol) open.push_back(r);
        cand = gather_rows(D, O, V, pre, open);
    }
    final_res = rn;
    throw LrccError(LRCC_ENOCONV, "shared-subspace solver: no convergence after " + std::to_string(max_iter) +
                                      " iterations");
}
