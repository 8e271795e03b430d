// Context, set-up, ground state, linear response and the extern "C" entry
// points declared in include/lrcc.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <cstdio>
#include <cstdlib>
#include <limits>
#include <string>

#include "ctx.h"

static std::string g_setup_err = "";

void set_global_error(const std::string& msg) { g_setup_err = msg; }

namespace {

bool is_mixed(int prec) { return prec == LRCC_MIXED_TF32 || prec == LRCC_MIXED_BF16X3; }

// precision of the maps that must be FP64-accurate (outer residuals, F X,
// ground-state polish): FP64 products in the plain FP64 mode, tensor-core
// integer slices in the emulated mode and (by default) in the mixed modes
int p64(const lrcc_ctx* c) {
    if (c->opt.prec == LRCC_FP64) return LRCC_FP64;
    if (c->opt.prec == LRCC_FP64_EMULATED || c->opt.fp64_products) return LRCC_FP64_EMULATED;
    return LRCC_FP64;
}

struct Timer {
    cudaEvent_t a, b;
    Dev& D;
    explicit Timer(Dev& d) : D(d) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, D.st);
    }
    double stop() {
        cudaEventRecord(b, D.st);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

Tensor dev_copy_c(Dev& D, const double* host, std::vector<int64_t> shape) {
    Tensor t = empty(D, shape);
    CK(cudaMemcpyAsync(t.p, host, t.numel() * sizeof(cplx), cudaMemcpyHostToDevice, D.st));
    return t;
}

// the virtual-virtual block of B, the only integrals the ladder reads
void ensure_bvv(lrcc_ctx* c) {
    if (c->lad.Bvv.p) return;
    Dev& D = c->D;
    const int O = c->O, V = c->V;
    c->lad.Bvv = empty(D, {(int64_t)c->L, (int64_t)V, (int64_t)V});
    axpby(D, mkc(1.0), c->B.slice(1, O, V).slice(2, O, V), false, mkc(0.0), c->lad.Bvv);
    c->lad.slab_rows = c->opt.slab_rows;
    c->lad.hermitian = c->opt.ladder_hermitian;
}

void build_ham_impl(lrcc_ctx* c) {
    Dev& D = c->D;
    int O = c->O, V = c->V;
    int64_t N = O + V;
    Ham& H = c->H;
    // Fock = diag(eps) (canonical reference)
    std::vector<double> f(2 * N * N, 0.0);
    for (int64_t p = 0; p < N; ++p) f[2 * (p * N + p)] = c->eps[p];
    Tensor F = dev_copy_c(D, f.data(), {N, N});
    auto blk = [&](const Tensor& M, int64_t r0, int64_t nr, int64_t c0, int64_t nc) {
        Tensor out = empty(D, {nr, nc});
        axpby(D, mkc(1.0), M.slice(0, r0, nr).slice(1, c0, nc), false, mkc(0.0), out);
        return out;
    };
    H.w = true;
    H.foo = blk(F, 0, O, 0, O);
    H.fov = blk(F, 0, O, O, V);
    H.fvo = blk(F, O, V, 0, O);
    H.fvv = blk(F, O, V, O, V);
    const Tensor& B = c->B;
    H.oooo = anti_block(D, B, 0, O, 0, O, 0, O, 0, O);
    H.ooov = anti_block(D, B, 0, O, 0, O, 0, O, O, V);
    H.oovo = anti_block(D, B, 0, O, 0, O, O, V, 0, O);
    H.ovoo = anti_block(D, B, 0, O, O, V, 0, O, 0, O);
    H.oovv = anti_block(D, B, 0, O, 0, O, O, V, O, V);
    H.vvoo = anti_block(D, B, O, V, O, V, 0, O, 0, O);
    H.ovov = anti_block(D, B, 0, O, O, V, 0, O, O, V);
    H.ovvo = anti_block(D, B, 0, O, O, V, O, V, 0, O);
    // factor blocks for the terms with three virtual indices (no O V^3 block)
    ensure_bvv(c);
    H.Bvv = c->lad.Bvv;
    H.Bov = empty(D, {(int64_t)c->L, (int64_t)O, (int64_t)V});
    axpby(D, mkc(1.0), B.slice(1, 0, O).slice(2, O, V), false, mkc(0.0), H.Bov);
    H.Bvo = empty(D, {(int64_t)c->L, (int64_t)V, (int64_t)O});
    axpby(D, mkc(1.0), B.slice(1, O, V).slice(2, 0, O), false, mkc(0.0), H.Bvo);
    c->lad.Bov = H.Bov;
    c->Hmu.clear();
    for (int k = 0; k < c->ncomp; ++k) {
        Ham h;
        h.w = false;
        Tensor M = c->mu.index(k);
        h.foo = blk(M, 0, O, 0, O);
        h.fov = blk(M, 0, O, O, V);
        h.fvo = blk(M, O, V, 0, O);
        h.fvv = blk(M, O, V, O, V);
        c->Hmu.push_back(h);
    }
    c->cc.reset(new CCProg());
    build_ccsd(*c->cc, c->H, &c->lad);
    c->ccfx.reset(new CCProg());
    build_ccsd(*c->ccfx, c->H, &c->lad);
    c->ccmu.clear();
    for (int k = 0; k < c->ncomp; ++k) {
        c->ccmu.emplace_back(new CCProg());
        build_ccsd(*c->ccmu.back(), c->Hmu[k], nullptr);
    }
    std::vector<double> eo(c->eps.begin(), c->eps.begin() + O), ev(c->eps.begin() + O, c->eps.end());
    if (c->eo) cudaFree(c->eo);
    if (c->ev) cudaFree(c->ev);
    CK(cudaMalloc(&c->eo, sizeof(double) * O));
    CK(cudaMalloc(&c->ev, sizeof(double) * V));
    CK(cudaMemcpy(c->eo, eo.data(), sizeof(double) * O, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->ev, ev.data(), sizeof(double) * V, cudaMemcpyHostToDevice));
    c->ground = false;
    c->ham_built = true;
}

// amplitudes of one RHS as program inputs (leading R dropped)
std::vector<Tensor> inputs_of(const Amp& a, int64_t r) { return {a.t1.index(r), a.t2.index(r)}; }

Amp add_batch(const Tensor& t1, const Tensor& t2) {
    Amp a;
    std::vector<int64_t> s1 = t1.shape(), s2 = t2.shape();
    s1.insert(s1.begin(), 1);
    s2.insert(s2.begin(), 1);
    a.t1 = t1.reshape(s1);
    a.t2 = t2.reshape(s2);
    return a;
}

// R(T) for one amplitude set (primal evaluation of the program)
Amp residual_T(Dev& D, CCProg& cp, const Amp& T, int64_t r, int prec, cplx* energy_out = nullptr) {
    cp.P.eval(D, inputs_of(T, r), prec);
    Amp out = add_batch(cp.P.val[cp.R1], cp.P.val[cp.R2]);
    if (energy_out) {
        CK(cudaMemcpyAsync(energy_out, cp.P.val[cp.E].p, sizeof(cplx), cudaMemcpyDeviceToHost, D.st));
        CK(cudaStreamSynchronize(D.st));
    }
    return out;
}

// sigma = A X  (program must hold the primal at T)
Amp sigma(Dev& D, CCProg& cp, const Amp& X, int prec) {
    std::vector<Tensor> r = cp.P.jvp(D, {X.t1, X.t2}, {cp.R1, cp.R2}, prec);
    return Amp{r[0], r[1]};
}

// unique-amplitude transpose product A^T y (+ e_scale * dE/dT), program at T
Amp vjp_unique(Dev& D, CCProg& cp, const Amp& Y, double e_scale, int prec) {
    int64_t R = Y.t1.d[0];
    Tensor c2 = empty(D, Y.t2.shape());
    axpby(D, mkc(0.25), Y.t2, false, mkc(0.0), c2);
    Tensor ce;
    if (e_scale != 0.0) {
        ce = empty(D, {R});
        fill(D, ce, mkc(e_scale));
    }
    std::vector<Tensor> g = cp.P.vjp(D, {Y.t1, c2, ce}, {cp.R1, cp.R2, cp.E}, prec);
    return Amp{g[0], antisym4(D, g[1])};
}

Amp grad_energy(Dev& D, CCProg& cp, int64_t O, int64_t V, int prec) {
    Tensor ce = empty(D, {1});
    fill(D, ce, mkc(1.0));
    std::vector<Tensor> g = cp.P.vjp(D, {Tensor(), Tensor(), ce}, {cp.R1, cp.R2, cp.E}, prec);
    (void)O;
    (void)V;
    return Amp{g[0], antisym4(D, g[1])};
}

double* dev_doubles(Dev& D, const std::vector<double>& v, std::shared_ptr<DevBuf>& hold) {
    size_t n = sizeof(double) * std::max<size_t>(1, v.size());
    double* p = (double*)D.pool.get(n);
    hold.reset(new DevBuf{&D.pool, p, n});
    CK(cudaMemcpyAsync(p, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, D.st));
    CK(cudaStreamSynchronize(D.st));
    return p;
}

// generic preconditioned DIIS loop on R right-hand sides:
//   r = resid(x);  x <- extrapolate(x - r/(D + shift))
// kernels with bounded waits raise a device error word instead of hanging
void check_device_error(Dev& D);

template <class F>
int solve_loop(lrcc_ctx* c, Amp& x, F&& resid, const std::vector<double>& shift, double tol, int max_iter,
               std::vector<double>* final_res = nullptr, bool throw_on_max = true) {
    Dev& D = c->D;
    int64_t R = x.t1.d[0];
    std::shared_ptr<DevBuf> hold;
    double* sh = dev_doubles(D, shift, hold);
    Diis diis(D, (int)R, c->opt.diis_size);
    std::vector<double> rn;
    // non-throwing mode (tensor-core phases): stop at the products' noise floor
    // -- no improvement in 8 iterations or growth past 10x the best residual --
    // and return the best iterate seen
    double best = std::numeric_limits<double>::infinity();
    int since_best = 0;
    Amp best_x;
    for (int it = 0; it < max_iter; ++it) {
        Amp r = resid(x);
        max_abs_amp(D, r, rn);
        double m = *std::max_element(rn.begin(), rn.end());
        static const bool verbose = getenv("LRCC_VERBOSE") != nullptr;
        if (verbose)
            fprintf(stderr, "  iter %3d  R=%lld  max|r| = %.3e%s\n", it, (long long)R, m, throw_on_max ? "" : "  (tc)");
        if (!std::isfinite(m) || m > 1e250) {
            check_device_error(D);
            if (!throw_on_max && best_x.t1.p) {
                x = best_x;
                return it;
            }
            throw LrccError(LRCC_ENOCONV, "residual is not finite");
        }
        if (m < tol) {
            if (final_res) *final_res = rn;
            return it;
        }
        if (!throw_on_max) {
            if (m < best) {
                best = m;
                since_best = 0;
                best_x = amp_copy(D, x);
            } else if (++since_best >= 8 || m > 10.0 * best) {
                x = best_x;
                if (final_res) *final_res = rn;
                return it;
            }
        }
        Amp xn = amp_empty(D, R, c->O, c->V);
        precond(D, &x, r, xn, c->eo, c->ev, sh);
        Amp e = amp_empty(D, R, c->O, c->V);
        amp_axpby(D, mkc(1.0), xn, mkc(0.0), e);
        amp_axpby(D, mkc(-1.0), x, mkc(1.0), e);
        x = diis.push_extrapolate(D, xn, e);
    }
    if (final_res) *final_res = rn;
    if (!throw_on_max) {
        if (best_x.t1.p) x = best_x;
        return max_iter;
    }
    throw LrccError(LRCC_ENOCONV, "no convergence after " + std::to_string(max_iter) + " iterations (max|r| = " +
                                      std::to_string(rn.empty() ? -1.0 : *std::max_element(rn.begin(), rn.end())) + ")");
}

template <class Apply>
void response_solve(lrcc_ctx* c, Amp& z, const Amp& b, const std::vector<double>& shift, const double* shift_dev,
                    Apply&& apply, std::vector<double>& final_res, int& n64, int& nmix);

void do_ground(lrcc_ctx* c, cplx& E, int& itT, int& itL) {
    Dev& D = c->D;
    int O = c->O, V = c->V;
    std::vector<double> zero(1, 0.0);
    std::shared_ptr<DevBuf> hold;
    double* sh = dev_doubles(D, zero, hold);
    {
        Timer tm(D);
        // MP2 start: one Jacobi step from T = 0
        Amp T0 = amp_zeros(D, 1, O, V);
        Amp r0 = residual_T(D, *c->cc, T0, 0, p64(c));
        Amp T = amp_empty(D, 1, O, V);
        precond(D, nullptr, r0, T, c->eo, c->ev, sh);
        itT = 0;
        if (is_mixed(c->opt.prec)) {
            // tensor-core residual until it stalls near its own precision, then FP64
            const int p = c->opt.prec;
            auto resm = [&](const Amp& x) { return amp_copy(D, residual_T(D, *c->cc, x, 0, p)); };
            itT += solve_loop(c, T, resm, zero, std::max(1e-6, c->opt.r_tol), c->opt.max_iter, nullptr, false);
        }
        auto res = [&](const Amp& x) { return amp_copy(D, residual_T(D, *c->cc, x, 0, p64(c))); };
        itT += solve_loop(c, T, res, zero, c->opt.r_tol, c->opt.max_iter);
        c->T = amp_copy(D, T);
        residual_T(D, *c->cc, c->T, 0, p64(c), &E);  // primal cached at converged T
        c->linearized = true;
        c->phase_ms[0] = tm.stop();
    }
    {
        // Lambda: A^T lambda = -dE/dT  (same refinement scheme as the left response)
        Timer tm(D);
        Amp gE = grad_energy(D, *c->cc, O, V, p64(c));
        Amp Lm = amp_empty(D, 1, O, V);
        std::vector<double> res;
        int n64 = 0, nmix = 0;
        auto apply = [&](const Amp& y, int p) { return vjp_unique(D, *c->cc, y, 0.0, p); };
        double xt = c->opt.x_tol;
        c->opt.x_tol = c->opt.r_tol;
        try {
            response_solve(c, Lm, gE, zero, sh, apply, res, n64, nmix);
        } catch (...) {
            c->opt.x_tol = xt;
            throw;
        }
        c->opt.x_tol = xt;
        itL = n64 + nmix;
        c->Lam = amp_copy(D, Lm);
        c->phase_ms[1] = tm.stop();
    }
    c->ground = true;
}

// F X for each RHS of X (Eq. 34): the directional derivative along X of the
// Lagrangian gradient g(T) = A(T)^T lambda + dE/dT, taken exactly by
// differentiating the reverse sweep (forward-over-reverse) at the converged T.
Amp fx_product(lrcc_ctx* c, const Amp& X) {
    Dev& D = c->D;
    int64_t R = X.t1.d[0];
    int O = c->O, V = c->V;
    CCProg& cp = *c->cc;  // holds the primal at the converged T
    Tensor l2 = empty(D, c->Lam.t2.shape());
    axpby(D, mkc(0.25), c->Lam.t2, false, mkc(0.0), l2);
    Tensor ce = empty(D, {1});
    fill(D, ce, mkc(1.0));
    std::vector<Tensor> d = cp.P.jvp_of_vjp(D, {X.t1, X.t2}, {c->Lam.t1, l2, ce}, {cp.R1, cp.R2, cp.E}, p64(c));
    (void)O;
    (void)V;
    (void)R;
    return Amp{d[0], antisym4(D, d[1])};
}

// Linear response solve (M - shift_r) z = -b  for R right-hand sides where
// M z is `apply(z, prec)` (sigma or the transpose product):
//  FP64: preconditioned DIIS on the FP64 residual.
//  mixed: iterative refinement; outer residual r = M z + shift z + b in FP64,
//  inner correction d from (M + shift) d = -r by DIIS on tensor-core products
//  until the inner residual drops by inner_tol, then z += d.
template <class Apply>
void response_solve(lrcc_ctx* c, Amp& z, const Amp& b, const std::vector<double>& shift, const double* shift_dev,
                    Apply&& apply, std::vector<double>& final_res, int& n64, int& nmix) {
    Dev& D = c->D;
    int64_t R = b.t1.d[0];
    int O = c->O, V = c->V;
    if (c->opt.solver == 1) {
        // one subspace for every right-hand side of the batch (FP64-class products only)
        std::function<Amp(const Amp&)> ap = [&](const Amp& v) { return apply(v, p64(c)); };
        subspace_solve(D, O, V, c->eo, c->ev, z, b, shift_dev, shift, ap, p64(c), c->opt.x_tol, c->opt.max_iter,
                       c->opt.subspace_max, final_res, n64);
        return;
    }
    precond(D, nullptr, b, z, c->eo, c->ev, shift_dev);
    auto res64 = [&](const Amp& x) {
        Amp s = apply(x, p64(c));
        n64++;
        Amp r = amp_empty(D, R, O, V);
        combine(D, s, x, shift_dev, &b, r);
        return r;
    };
    if (!is_mixed(c->opt.prec)) {
        solve_loop(c, z, res64, shift, c->opt.x_tol, c->opt.max_iter, &final_res);
        return;
    }
    const int prec = c->opt.prec;
    std::vector<double> rn;
    // phase 1: the whole solve on tensor-core products, down to their accuracy floor
    {
        std::vector<double> bn;
        max_abs_amp(D, b, bn);
        double bmax = *std::max_element(bn.begin(), bn.end());
        auto resd = [&](const Amp& x) {
            Amp s = apply(x, prec);
            nmix++;
            Amp q = amp_empty(D, R, O, V);
            combine(D, s, x, shift_dev, &b, q);
            return q;
        };
        solve_loop(c, z, resd, shift, std::max(c->opt.inner_tol * bmax, 0.5 * c->opt.x_tol),
                   std::min(c->opt.max_iter, 60), nullptr, false);
    }
    // phase 2: FP64 residual, tensor-core correction (iterative refinement)
    for (int outer = 0; outer < 30; ++outer) {
        Amp r = res64(z);
        max_abs_amp(D, r, rn);
        double m = *std::max_element(rn.begin(), rn.end());
        if (!std::isfinite(m) || m > 1e250) throw LrccError(LRCC_ENOCONV, "residual is not finite");
        if (m < c->opt.x_tol) {
            final_res = rn;
            return;
        }
        Amp d = amp_empty(D, R, O, V);
        precond(D, nullptr, r, d, c->eo, c->ev, shift_dev);
        auto resm = [&](const Amp& x) {
            Amp s = apply(x, prec);
            nmix++;
            Amp q = amp_empty(D, R, O, V);
            combine(D, s, x, shift_dev, &r, q);
            return q;
        };
        // aim the correction at the final tolerance, within the products' accuracy
        double tol = std::max(0.3 * c->opt.x_tol, c->opt.inner_tol * m);
        solve_loop(c, d, resm, shift, tol, std::min(c->opt.max_iter, 60), nullptr, false);
        amp_axpby(D, mkc(1.0), d, mkc(1.0), z);
    }
    final_res = rn;
    throw LrccError(LRCC_ENOCONV, "iterative refinement did not converge");
}

// Eq. 36: per frequency, X(+w) and X(-w) for all components in one batch,
// F X(+w), and the Gram matrices of the unique-amplitude dots.
void solve_pm_omega(lrcc_ctx* c, const double* omegas, int n_w, const int* comps, int n_c,
                    const std::vector<Amp>& xi, const std::vector<Amp>& eta, double* alpha, double* err_est) {
    Dev& D = c->D;
    int O = c->O, V = c->V;
    Amp etaS = amp_empty(D, n_c, O, V);
    for (int a = 0; a < n_c; ++a) {
        Tensor e1 = etaS.t1.index(a), e2 = etaS.t2.index(a);
        axpby(D, mkc(1.0), eta[comps[a]].t1.index(0), false, mkc(0.0), e1);
        axpby(D, mkc(1.0), eta[comps[a]].t2.index(0), false, mkc(0.0), e2);
    }
    for (int w = 0; w < n_w; ++w) {
        const int64_t R = 2 * n_c;
        Amp xiR = amp_empty(D, R, O, V);
        std::vector<double> sh(R);
        for (int64_t r = 0; r < R; ++r) {
            int a = (int)(r % n_c);
            Tensor a1 = xiR.t1.index(r), a2 = xiR.t2.index(r);
            axpby(D, mkc(1.0), xi[comps[a]].t1.index(0), false, mkc(0.0), a1);
            axpby(D, mkc(1.0), xi[comps[a]].t2.index(0), false, mkc(0.0), a2);
            sh[r] = r < n_c ? -omegas[w] : omegas[w];   // (A - w') X = -xi, w' = +w then -w
        }
        std::shared_ptr<DevBuf> hs;
        double* shd = dev_doubles(D, sh, hs);
        Amp X = amp_empty(D, R, O, V);
        std::vector<double> resX;
        {
            Timer tm(D);
            auto apply = [&](const Amp& x, int p) { return sigma(D, *c->cc, x, p); };
            response_solve(c, X, xiR, sh, shd, apply, resX, c->n_sigma64, c->n_sigma_mixed);
            c->phase_ms[3] += tm.stop();
        }
        Amp Xp = amp_rows(X, 0, n_c), Xm = amp_rows(X, n_c, n_c);
        Amp FXp;
        {
            Timer tm(D);
            Amp Xpc = amp_copy(D, Xp);
            FXp = fx_product(c, Xpc);
            c->phase_ms[4] += tm.stop();
        }
        Timer tm(D);
        Tensor g[6] = {amp_gram(D, etaS, Xp), amp_gram(D, Xm, etaS), amp_gram(D, Xm, FXp),
                       amp_gram(D, etaS, Xm), amp_gram(D, Xp, etaS), amp_gram(D, FXp, Xm)};
        std::vector<cplx> h(6 * n_c * n_c);
        for (int q = 0; q < 6; ++q)
            CK(cudaMemcpyAsync(h.data() + q * n_c * n_c, g[q].p, sizeof(cplx) * n_c * n_c, cudaMemcpyDeviceToHost, D.st));
        CK(cudaStreamSynchronize(D.st));
        c->phase_ms[6] += tm.stop();
        for (int a = 0; a < n_c; ++a)
            for (int b = 0; b < n_c; ++b) {
                auto at = [&](int q) { return h[q * n_c * n_c + a * n_c + b]; };
                cplx gp = mkc(at(0).x + at(1).x + at(2).x, at(0).y + at(1).y + at(2).y);   // G_AB(+w)
                cplx gm = mkc(at(3).x + at(4).x + at(5).x, at(3).y + at(4).y + at(5).y);   // G_AB(-w)
                size_t o = ((size_t)w * n_c + a) * n_c + b;
                alpha[2 * o] = -0.5 * (gp.x + gm.x);
                alpha[2 * o + 1] = -0.5 * (gp.y - gm.y);
            }
        if (err_est)
            for (int a = 0; a < n_c; ++a) err_est[(size_t)w * n_c + a] = std::max(resX[a], resX[n_c + a]);
    }
}

void do_solve(lrcc_ctx* c, const double* omegas, int n_w, const int* comps, int n_c, double* alpha,
              double* err_est) {
    Dev& D = c->D;
    int O = c->O, V = c->V;
    for (int q = 0; q < 7; ++q) if (q >= 2) c->phase_ms[q] = 0;
    c->n_sigma64 = 0;
    c->n_sigma_mixed = 0;
    // xi^A, eta^A per component (Eq. 31, 33)
    std::vector<Amp> xi(c->ncomp), eta(c->ncomp);
    std::vector<char> need(c->ncomp, 0);
    for (int k = 0; k < n_c; ++k) need[comps[k]] = 1;
    {
        Timer tm(D);
        for (int k = 0; k < c->ncomp; ++k) {
            if (!need[k]) continue;
            xi[k] = amp_copy(D, residual_T(D, *c->ccmu[k], c->T, 0, LRCC_FP64));
            eta[k] = vjp_unique(D, *c->ccmu[k], c->Lam, 1.0, LRCC_FP64);
        }
        c->phase_ms[2] += tm.stop();
    }
    if (c->opt.pm_omega) {
        solve_pm_omega(c, omegas, n_w, comps, n_c, xi, eta, alpha, err_est);
        return;
    }
    // right-hand sides (omega, component), rhs_chunk at a time
    struct Rhs { int w, comp_idx; };
    std::vector<Rhs> all;
    for (int w = 0; w < n_w; ++w)
        for (int k = 0; k < n_c; ++k) all.push_back({w, k});
    std::vector<cplx> g((size_t)n_w * n_c * n_c, mkc(0.0));
    std::vector<double> errs((size_t)n_w * n_c, 0.0);
    int chunk = std::max(1, c->opt.rhs_chunk);
    for (size_t c0 = 0; c0 < all.size(); c0 += chunk) {
        size_t c1 = std::min(all.size(), c0 + chunk);
        int64_t R = (int64_t)(c1 - c0);
        Amp xiR = amp_empty(D, R, O, V), rhsY = amp_empty(D, R, O, V);
        std::vector<double> mw(R), pw(R);
        for (int64_t r = 0; r < R; ++r) {
            const Rhs& q = all[c0 + r];
            int comp = comps[q.comp_idx];
            Tensor a1 = xiR.t1.index(r), a2 = xiR.t2.index(r);
            axpby(D, mkc(1.0), xi[comp].t1.index(0), false, mkc(0.0), a1);
            axpby(D, mkc(1.0), xi[comp].t2.index(0), false, mkc(0.0), a2);
            mw[r] = -omegas[q.w];
            pw[r] = omegas[q.w];
        }
        std::shared_ptr<DevBuf> h1, h2;
        double* mwd = dev_doubles(D, mw, h1);
        double* pwd = dev_doubles(D, pw, h2);
        // X: (A - w) X = -xi
        Amp X = amp_empty(D, R, O, V);
        std::vector<double> resX, resY;
        {
            Timer tm(D);
            auto apply = [&](const Amp& x, int p) { return sigma(D, *c->cc, x, p); };
            response_solve(c, X, xiR, mw, mwd, apply, resX, c->n_sigma64, c->n_sigma_mixed);
            c->phase_ms[3] += tm.stop();
        }
        // eta + F X
        {
            Timer tm(D);
            Amp FX = fx_product(c, X);
            for (int64_t r = 0; r < R; ++r) {
                int comp = comps[all[c0 + r].comp_idx];
                Tensor y1 = rhsY.t1.index(r), y2 = rhsY.t2.index(r);
                axpby(D, mkc(1.0), eta[comp].t1.index(0), false, mkc(0.0), y1);
                axpby(D, mkc(1.0), eta[comp].t2.index(0), false, mkc(0.0), y2);
            }
            amp_axpby(D, mkc(1.0), FX, mkc(1.0), rhsY);
            c->phase_ms[4] += tm.stop();
        }
        // Y: Y (A + w) = -(eta + F X)
        Amp Y = amp_empty(D, R, O, V);
        {
            Timer tm(D);
            auto apply = [&](const Amp& y, int p) { return vjp_unique(D, *c->cc, y, 0.0, p); };
            response_solve(c, Y, rhsY, pw, pwd, apply, resY, c->n_sigma64, c->n_sigma_mixed);
            c->phase_ms[5] += tm.stop();
        }
        // g_AB = Y^B . xi^A + eta^A . X^B
        {
            Timer tm(D);
            for (int a = 0; a < n_c; ++a) {
                int compA = comps[a];
                Tensor d1 = amp_dot_fixed(D, Y, xi[compA]);
                Tensor d2 = amp_dot_fixed(D, X, eta[compA]);
                std::vector<cplx> h1v(R), h2v(R);
                CK(cudaMemcpyAsync(h1v.data(), d1.p, sizeof(cplx) * R, cudaMemcpyDeviceToHost, D.st));
                CK(cudaMemcpyAsync(h2v.data(), d2.p, sizeof(cplx) * R, cudaMemcpyDeviceToHost, D.st));
                CK(cudaStreamSynchronize(D.st));
                for (int64_t r = 0; r < R; ++r) {
                    const Rhs& q = all[c0 + r];
                    g[((size_t)q.w * n_c + a) * n_c + q.comp_idx] = mkc(h1v[r].x + h2v[r].x, h1v[r].y + h2v[r].y);
                }
            }
            for (int64_t r = 0; r < R; ++r) {
                const Rhs& q = all[c0 + r];
                errs[(size_t)q.w * n_c + q.comp_idx] = std::max(resX[r], resY[r]);
            }
            c->phase_ms[6] += tm.stop();
        }
    }
    // alpha_AB = -1/2 (g_AB + conj g_BA)   (Eq. 35, P(A,B) = swap + conjugate)
    for (int w = 0; w < n_w; ++w)
        for (int a = 0; a < n_c; ++a)
            for (int b = 0; b < n_c; ++b) {
                cplx gab = g[((size_t)w * n_c + a) * n_c + b], gba = g[((size_t)w * n_c + b) * n_c + a];
                size_t o = ((size_t)w * n_c + a) * n_c + b;
                alpha[2 * o] = -0.5 * (gab.x + gba.x);
                alpha[2 * o + 1] = -0.5 * (gab.y - gba.y);
            }
    if (err_est) std::memcpy(err_est, errs.data(), sizeof(double) * errs.size());
}

// kernels with bounded waits raise a device error word instead of hanging
void check_device_error(Dev& D) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, D.err_flag, sizeof(int), cudaMemcpyDeviceToHost, D.st));
    CK(cudaStreamSynchronize(D.st));
    if (h != 0) {
        CK(cudaMemsetAsync(D.err_flag, 0, sizeof(int), D.st));
        CK(cudaStreamSynchronize(D.st));
        throw LrccError(LRCC_ETIMEOUT, "a device-side wait expired (tensor-core pipeline did not complete)");
    }
}

lrcc_status fail(lrcc_ctx* c, const LrccError& e) {
    if (c) c->err = e.what();
    else g_setup_err = e.what();
    return e.st;
}

}  // namespace

void ensure_ham(lrcc_ctx* c) {
    if (!c->ham_built) build_ham_impl(c);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void lrcc_default_options(lrcc_options* o) {
    if (!o) return;
    o->r_tol = 1e-10;
    o->x_tol = 1e-9;
    o->max_iter = 200;
    o->diis_size = 8;
    o->rhs_chunk = 12;
    o->prec = LRCC_FP64;
    o->inner_tol = 1e-5;
    o->plus_omega = 0;
    o->slab_rows = 0;
    o->pm_omega = 0;
    o->fp64_products = 1;
    o->fns_density = 0;
    o->solver = 0;
    o->subspace_max = 0;
    o->ladder_hermitian = 0;
    o->embed_budget_mb = 0;
}

const char* lrcc_last_error(const lrcc_ctx* c) { return c ? c->err.c_str() : g_setup_err.c_str(); }

lrcc_status lrcc_setup(const double* eps, const double* B, int L, const double* mu, int ncomp, int O, int V,
                       const lrcc_options* opt, lrcc_ctx** out) {
    if (!out) {
        g_setup_err = "out is NULL";
        return LRCC_EINVAL;
    }
    *out = nullptr;
    lrcc_ctx* c = nullptr;
    try {
        REQUIRE(eps && B && mu, "null input array");
        REQUIRE(O >= 2 && V >= 2 && L >= 1 && ncomp >= 1 && ncomp <= 3, "sizes out of range (O>=2, V>=2, L>=1, 1<=ncomp<=3)");
        int64_t N = (int64_t)O + V;
        for (int64_t p = 0; p < N; ++p) REQUIRE(std::isfinite(eps[p]), "eps not finite");
        double homo = *std::max_element(eps, eps + O), lumo = *std::min_element(eps + O, eps + N);
        REQUIRE(homo < lumo, "every occupied energy must be below every virtual energy");
        // Hermiticity of B^L and mu (relative to the largest element)
        auto herm = [&](const double* M, int64_t nmat, const char* what) {
            double mx = 0.0, dev = 0.0;
            for (int64_t l = 0; l < nmat; ++l) {
                const double* m = M + 2 * l * N * N;
                for (int64_t p = 0; p < N; ++p)
                    for (int64_t q = 0; q < N; ++q) {
                        double re = m[2 * (p * N + q)], im = m[2 * (p * N + q) + 1];
                        double re2 = m[2 * (q * N + p)], im2 = m[2 * (q * N + p) + 1];
                        REQUIRE(std::isfinite(re) && std::isfinite(im), std::string(what) + " not finite");
                        mx = std::max(mx, std::hypot(re, im));
                        dev = std::max(dev, std::hypot(re - re2, im + im2));
                    }
            }
            REQUIRE(dev <= 1e-12 * std::max(mx, 1e-300), std::string(what) + " is not Hermitian");
        };
        herm(B, L, "B");
        herm(mu, ncomp, "mu");
        c = new lrcc_ctx();
        if (opt) c->opt = *opt;
        else lrcc_default_options(&c->opt);
        REQUIRE(c->opt.prec >= LRCC_FP64 && c->opt.prec <= LRCC_FP64_EMULATED, "bad precision mode");
        REQUIRE(c->opt.max_iter >= 1 && c->opt.diis_size >= 2 && c->opt.rhs_chunk >= 1, "bad solver options");
        REQUIRE(c->opt.fns_density == 0 || c->opt.fns_density == 1, "fns_density must be 0 (FNS++) or 1 (MP2)");
        REQUIRE(c->opt.solver == 0 || c->opt.solver == 1, "solver must be 0 (DIIS) or 1 (shared subspace)");
        REQUIRE(c->opt.solver == 0 || !is_mixed(c->opt.prec),
                "the shared-subspace solver needs FP64-class products (LRCC_FP64 or LRCC_FP64_EMULATED)");
        REQUIRE(c->opt.subspace_max >= 0, "subspace_max must be >= 0");
        REQUIRE(c->opt.embed_budget_mb >= 0, "embed_budget_mb must be >= 0");
        REQUIRE(c->opt.ladder_hermitian >= -1 && c->opt.ladder_hermitian <= 1, "ladder_hermitian must be -1, 0 or 1");
        c->D.embed_budget = double(c->opt.embed_budget_mb) * double(1 << 20);
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&c->D.sm_count, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaStreamCreateWithFlags(&c->D.st, cudaStreamNonBlocking));
        CK(cudaMalloc(&c->D.err_flag, sizeof(int)));
        CK(cudaMemset(c->D.err_flag, 0, sizeof(int)));
        c->O = O;
        c->V = V;
        c->L = L;
        c->ncomp = ncomp;
        c->eps.assign(eps, eps + N);
        c->B = dev_copy_c(c->D, B, {L, N, N});
        c->mu = dev_copy_c(c->D, mu, {ncomp, N, N});
        CK(cudaStreamSynchronize(c->D.st));
        *out = c;
        return LRCC_OK;
    } catch (const LrccError& e) {
        g_setup_err = e.what();
        delete c;
        return e.st;
    } catch (const std::exception& e) {
        g_setup_err = e.what();
        delete c;
        return LRCC_ECUDA;
    }
}

void lrcc_destroy(lrcc_ctx* c) {
    if (!c) return;
    cudaStream_t st = c->D.st;
    if (st) cudaStreamSynchronize(st);
    delete c;
    if (st) cudaStreamDestroy(st);
}

lrcc_status lrcc_ccsd_ground(lrcc_ctx* c, double e_corr[2], int* iters_T, int* iters_L) {
    if (!c) return LRCC_EINVAL;
    try {
        cplx E = mkc(0.0);
        int itT = 0, itL = 0;
        ensure_ham(c);
        do_ground(c, E, itT, itL);
        check_device_error(c->D);
        if (e_corr) {
            e_corr[0] = E.x;
            e_corr[1] = E.y;
        }
        if (iters_T) *iters_T = itT;
        if (iters_L) *iters_L = itL;
        return LRCC_OK;
    } catch (const LrccError& e) {
        return fail(c, e);
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

lrcc_status lrcc_solve(lrcc_ctx* c, const double* omegas, int n_w, const int* comps, int n_c, double* alpha,
                       double* err_est) {
    if (!c) return LRCC_EINVAL;
    try {
        if (!c->ground) throw LrccError(LRCC_ESTATE, "lrcc_solve before lrcc_ccsd_ground");
        REQUIRE(omegas && comps && alpha && n_w >= 1 && n_c >= 1, "bad solve arguments");
        for (int k = 0; k < n_c; ++k) REQUIRE(comps[k] >= 0 && comps[k] < c->ncomp, "component out of range");
        for (int w = 0; w < n_w; ++w) REQUIRE(std::isfinite(omegas[w]), "omega not finite");
        do_solve(c, omegas, n_w, comps, n_c, alpha, err_est);
        check_device_error(c->D);
        return LRCC_OK;
    } catch (const LrccError& e) {
        return fail(c, e);
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

static lrcc_status residual_impl(lrcc_ctx* c, int kind, const double* t, const double* in, int R, int comp,
                                 int prec, double* out, bool device) {
    Dev& D = c->D;
    int64_t O = c->O, V = c->V;
    int64_t n1 = O * V, n2 = O * O * V * V, nt = n1 + n2;
    REQUIRE(R >= 1 && in && out, "bad residual arguments");
    REQUIRE(kind >= LRCC_RES_T && kind <= LRCC_RES_VJP_FULL, "bad residual kind");
    REQUIRE(prec >= LRCC_FP64 && prec <= LRCC_FP64_EMULATED, "bad precision");
    ensure_ham(c);
    // stage inputs as [R][nt] on the device
    Tensor inb;
    if (device) inb = wrap((cplx*)in, {R, nt});
    else inb = dev_copy_c(D, in, {R, nt});
    auto to_amp = [&](const Tensor& flat, int64_t RR) {
        Amp a = amp_empty(D, RR, O, V);
        Tensor v1 = flat.slice(1, 0, n1), v2 = flat.slice(1, n1, n2);
        // views [RR][O][V] and [RR][O][O][V][V] of the flat rows
        Tensor s1 = v1;
        s1.nd = 3; s1.d[0] = RR; s1.d[1] = O; s1.d[2] = V; s1.s[0] = nt; s1.s[1] = V; s1.s[2] = 1;
        Tensor s2 = v2;
        s2.nd = 5; s2.d[0] = RR; s2.d[1] = O; s2.d[2] = O; s2.d[3] = V; s2.d[4] = V;
        s2.s[0] = nt; s2.s[1] = O * V * V; s2.s[2] = V * V; s2.s[3] = V; s2.s[4] = 1;
        axpby(D, mkc(1.0), s1, false, mkc(0.0), a.t1);
        // P: antisymmetric projection 1/4 (x - P_ij x - P_ab x + P_ij P_ab x)
        perm_axpby(D, "Zijab->Zijab", mkc(0.25), s2, mkc(0.0), a.t2);
        perm_axpby(D, "Zijab->Zjiab", mkc(-0.25), s2, mkc(1.0), a.t2);
        perm_axpby(D, "Zijab->Zijba", mkc(-0.25), s2, mkc(1.0), a.t2);
        perm_axpby(D, "Zijab->Zjiba", mkc(0.25), s2, mkc(1.0), a.t2);
        return a;
    };
    Amp X = to_amp(inb, R);
    Amp res;
    std::vector<cplx> energies;
    if ((kind == LRCC_RES_SIGMA || kind == LRCC_RES_VJP || kind == LRCC_RES_VJP_FULL) && !t) {
        // linearised at the converged ground state: the primal values cached in
        // the solver's program are reused (exactly the maps lrcc_solve applies)
        if (!c->ground && !c->linearized)
            throw LrccError(LRCC_ESTATE, "t == NULL needs lrcc_ccsd_ground or lrcc_linearize first");
        if (kind == LRCC_RES_SIGMA) {
            res = sigma(D, *c->cc, X, prec);
        } else if (kind == LRCC_RES_VJP) {
            res = vjp_unique(D, *c->cc, X, 0.0, prec);
        } else {
            Amp Xs = amp_copy(D, X);
            axpby(D, mkc(4.0), X.t2, false, mkc(0.0), Xs.t2);
            res = vjp_unique(D, *c->cc, Xs, 0.0, prec);
            Tensor q = empty(D, res.t2.shape());
            axpby(D, mkc(0.25), res.t2, false, mkc(0.0), q);
            res.t2 = q;
        }
    } else if (kind == LRCC_RES_SIGMA || kind == LRCC_RES_VJP || kind == LRCC_RES_VJP_FULL || kind == LRCC_RES_XI) {
        REQUIRE(t, "t is required for XI");
        Tensor tb = device ? wrap((cplx*)t, {1, nt}) : dev_copy_c(D, t, {1, nt});
        Amp T = to_amp(tb, 1);
        if (kind == LRCC_RES_XI) {
            REQUIRE(comp >= 0 && comp < c->ncomp, "component out of range");
            res = amp_copy(D, residual_T(D, *c->ccmu[comp], T, 0, LRCC_FP64));
            // same xi for every RHS row of `in` is not meaningful; XI uses t only
            Amp rep = amp_empty(D, R, O, V);
            for (int64_t r = 0; r < R; ++r) {
                Tensor a1 = rep.t1.index(r), a2 = rep.t2.index(r);
                axpby(D, mkc(1.0), res.t1.index(0), false, mkc(0.0), a1);
                axpby(D, mkc(1.0), res.t2.index(0), false, mkc(0.0), a2);
            }
            res = rep;
        } else {
            c->ccfx->P.eval(D, inputs_of(T, 0), prec);
            if (kind == LRCC_RES_SIGMA) {
                res = sigma(D, *c->ccfx, X, prec);
            } else if (kind == LRCC_RES_VJP) {
                res = vjp_unique(D, *c->ccfx, X, 0.0, prec);
            } else {
                // adjoint with cotangent `in` on every full entry, then P
                Amp Xs = amp_copy(D, X);
                axpby(D, mkc(4.0), X.t2, false, mkc(0.0), Xs.t2);
                res = vjp_unique(D, *c->ccfx, Xs, 0.0, prec);
                Tensor q = empty(D, res.t2.shape());
                axpby(D, mkc(0.25), res.t2, false, mkc(0.0), q);
                res.t2 = q;
            }
        }
    } else {
        res = amp_empty(D, R, O, V);
        energies.resize(R);
        for (int64_t r = 0; r < R; ++r) {
            cplx e;
            Amp rr = residual_T(D, *c->ccfx, X, r, prec, &e);
            energies[r] = e;
            Tensor a1 = res.t1.index(r), a2 = res.t2.index(r);
            axpby(D, mkc(1.0), rr.t1.index(0), false, mkc(0.0), a1);
            axpby(D, mkc(1.0), rr.t2.index(0), false, mkc(0.0), a2);
        }
    }
    if (kind == LRCC_RES_ENERGY) {
        if (device) {
            CK(cudaMemcpyAsync(out, energies.data(), sizeof(cplx) * R, cudaMemcpyHostToDevice, D.st));
            CK(cudaStreamSynchronize(D.st));
        } else {
            std::memcpy(out, energies.data(), sizeof(cplx) * R);
        }
        return LRCC_OK;
    }
    Tensor ob = device ? wrap((cplx*)out, {R, nt}) : empty(D, {R, nt});
    {
        Tensor v1 = ob.slice(1, 0, n1), v2 = ob.slice(1, n1, n2);
        Tensor s1 = v1;
        s1.nd = 3; s1.d[0] = R; s1.d[1] = O; s1.d[2] = V; s1.s[0] = nt; s1.s[1] = V; s1.s[2] = 1;
        Tensor s2 = v2;
        s2.nd = 5; s2.d[0] = R; s2.d[1] = O; s2.d[2] = O; s2.d[3] = V; s2.d[4] = V;
        s2.s[0] = nt; s2.s[1] = O * V * V; s2.s[2] = V * V; s2.s[3] = V; s2.s[4] = 1;
        axpby(D, mkc(1.0), res.t1, false, mkc(0.0), s1);
        axpby(D, mkc(1.0), res.t2, false, mkc(0.0), s2);
    }
    if (!device) {
        CK(cudaMemcpyAsync(out, ob.p, sizeof(cplx) * R * nt, cudaMemcpyDeviceToHost, D.st));
    }
    CK(cudaStreamSynchronize(D.st));
    return LRCC_OK;
}

lrcc_status lrcc_residual(lrcc_ctx* c, int kind, const double* t, const double* in, int R, int comp, int prec,
                          double* out) {
    if (!c) return LRCC_EINVAL;
    try {
        lrcc_status s = residual_impl(c, kind, t, in, R, comp, prec, out, false);
        check_device_error(c->D);
        return s;
    } catch (const LrccError& e) {
        return fail(c, e);
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

lrcc_status lrcc_linearize(lrcc_ctx* c, const double* t, int prec) {
    if (!c) return LRCC_EINVAL;
    try {
        REQUIRE(t, "t is NULL");
        REQUIRE(prec >= LRCC_FP64 && prec <= LRCC_FP64_EMULATED, "bad precision");
        ensure_ham(c);
        Dev& D = c->D;
        const int64_t O = c->O, V = c->V, n1 = O * V, n2 = O * O * V * V;
        c->ground = false;
        c->linearized = false;
        Tensor tb = dev_copy_c(D, t, {n1 + n2});
        Amp T = amp_empty(D, 1, O, V);
        axpby(D, mkc(1.0), tb.slice(0, 0, n1).reshape({1, O, V}), false, mkc(0.0), T.t1);
        Tensor s2 = tb.slice(0, n1, n2).reshape({1, O, O, V, V});
        // antisymmetric projection of the doubles block
        perm_axpby(D, "Zijab->Zijab", mkc(0.25), s2, mkc(0.0), T.t2);
        perm_axpby(D, "Zijab->Zjiab", mkc(-0.25), s2, mkc(1.0), T.t2);
        perm_axpby(D, "Zijab->Zijba", mkc(-0.25), s2, mkc(1.0), T.t2);
        perm_axpby(D, "Zijab->Zjiba", mkc(0.25), s2, mkc(1.0), T.t2);
        tb = Tensor();
        c->T = T;
        residual_T(D, *c->cc, c->T, 0, prec);
        CK(cudaStreamSynchronize(D.st));
        check_device_error(D);
        c->linearized = true;
        return LRCC_OK;
    } catch (const LrccError& e) {
        return fail(c, e);
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

lrcc_status lrcc_residual_dev(lrcc_ctx* c, int kind, const double* t, const double* in, int R, int comp, int prec,
                              double* out, void* stream) {
    if (!c) return LRCC_EINVAL;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        // order after the caller's stream, run on ours, order the caller after us
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, st));
        CK(cudaStreamWaitEvent(c->D.st, ev, 0));
        lrcc_status s = residual_impl(c, kind, t, in, R, comp, prec, out, true);
        check_device_error(c->D);
        CK(cudaEventRecord(ev, c->D.st));
        CK(cudaStreamWaitEvent(st, ev, 0));
        CK(cudaEventDestroy(ev));
        return s;
    } catch (const LrccError& e) {
        return fail(c, e);
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

lrcc_status lrcc_ladder_dev(lrcc_ctx* c, const double* x, double* z, int R, int transpose, int prec, void* stream) {
    if (!c) return LRCC_EINVAL;
    try {
        REQUIRE(x && z && R >= 1, "bad ladder arguments");
        REQUIRE(prec >= LRCC_FP64 && prec <= LRCC_FP64_EMULATED, "bad precision");
        ensure_ham(c);
        cudaStream_t st = (cudaStream_t)stream;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, st));
        CK(cudaStreamWaitEvent(c->D.st, ev, 0));
        Tensor X = wrap((cplx*)x, {R, c->O, c->O, c->V, c->V});
        Tensor Z = wrap((cplx*)z, {R, c->O, c->O, c->V, c->V});
        ladder(c->D, c->lad, X, mkc(1.0), mkc(0.0), Z, transpose != 0, prec);
        check_device_error(c->D);
        CK(cudaEventRecord(ev, c->D.st));
        CK(cudaStreamWaitEvent(st, ev, 0));
        CK(cudaEventDestroy(ev));
        return LRCC_OK;
    } catch (const LrccError& e) {
        return fail(c, e);
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

lrcc_status lrcc_ladder_packed_dev(lrcc_ctx* c, const double* xt, double* zt, int64_t ncol, int transpose, int prec,
                                   void* stream) {
    if (!c) return LRCC_EINVAL;
    try {
        REQUIRE(xt && zt && ncol >= 1, "bad ladder arguments");
        REQUIRE(prec >= LRCC_FP64 && prec <= LRCC_FP64_EMULATED, "bad precision");
        ensure_bvv(c);
        cudaStream_t st = (cudaStream_t)stream;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, st));
        CK(cudaStreamWaitEvent(c->D.st, ev, 0));
        ladder_packed(c->D, c->lad, (const cplx*)xt, (cplx*)zt, ncol, transpose != 0, prec);
        check_device_error(c->D);
        CK(cudaEventRecord(ev, c->D.st));
        CK(cudaStreamWaitEvent(st, ev, 0));
        CK(cudaEventDestroy(ev));
        return LRCC_OK;
    } catch (const LrccError& e) {
        return fail(c, e);
    } catch (const std::exception& e) {
        c->err = e.what();
        return LRCC_ECUDA;
    }
}

lrcc_status lrcc_get_amplitudes(lrcc_ctx* c, int which, double* out) {
    if (!c || !out || (which != 0 && which != 1)) return LRCC_EINVAL;
    try {
        if (!c->ground) throw LrccError(LRCC_ESTATE, "no ground state yet");
        const Amp& a = which == 0 ? c->T : c->Lam;
        int64_t n1 = a.t1.numel(), n2 = a.t2.numel();
        CK(cudaMemcpyAsync(out, a.t1.p, sizeof(cplx) * n1, cudaMemcpyDeviceToHost, c->D.st));
        CK(cudaMemcpyAsync(out + 2 * n1, a.t2.p, sizeof(cplx) * n2, cudaMemcpyDeviceToHost, c->D.st));
        CK(cudaStreamSynchronize(c->D.st));
        return LRCC_OK;
    } catch (const LrccError& e) {
        return fail(c, e);
    }
}

lrcc_status lrcc_solve_counts(const lrcc_ctx* c, int* n_fp64, int* n_mixed) {
    if (!c) return LRCC_EINVAL;
    if (n_fp64) *n_fp64 = c->n_sigma64;
    if (n_mixed) *n_mixed = c->n_sigma_mixed;
    return LRCC_OK;
}

lrcc_status lrcc_phase_times(const lrcc_ctx* c, double* ms7) {
    if (!c || !ms7) return LRCC_EINVAL;
    for (int k = 0; k < 7; ++k) ms7[k] = c->phase_ms[k];
    return LRCC_OK;
}

int64_t lrcc_kernel_launches(const lrcc_ctx* c) { return c ? c->D.launches : 0; }

lrcc_status lrcc_memory_stats(const lrcc_ctx* c, int64_t* live, int64_t* peak, int64_t* largest) {
    if (!c || !live || !peak || !largest) return LRCC_EINVAL;
    *live = (int64_t)c->D.pool.live;
    *peak = (int64_t)c->D.pool.peak;
    *largest = (int64_t)c->D.pool.largest;
    return LRCC_OK;
}

static void clear_recs(Dev& D) {
    for (auto& r : D.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    D.recs.clear();
}

lrcc_status lrcc_profile(lrcc_ctx* c, int enable) {
    if (!c) return LRCC_EINVAL;
    cudaStreamSynchronize(c->D.st);
    if (enable) clear_recs(c->D);
    c->D.timing = enable != 0;
    return LRCC_OK;
}

lrcc_status lrcc_profile_dump(lrcc_ctx* c, const char* path) {
    if (!c || !path) return LRCC_EINVAL;
    if (cudaStreamSynchronize(c->D.st) != cudaSuccess) return LRCC_ECUDA;
    FILE* f = fopen(path, "w");
    if (!f) {
        c->err = std::string("cannot open ") + path;
        return LRCC_EINVAL;
    }
    fprintf(f, "kernel,M,N,K,batch,ms,flops\n");
    for (auto& r : c->D.recs) {
        float e = 0;
        cudaEventElapsedTime(&e, r.a, r.b);
        fprintf(f, "%s,%lld,%lld,%lld,%lld,%.6f,%.6e\n", r.name, (long long)r.m, (long long)r.n, (long long)r.k,
                (long long)r.batch, e, r.flops);
    }
    fclose(f);
    return LRCC_OK;
}

lrcc_status lrcc_kernel_stats(lrcc_ctx* c, int idx, const char** name, int64_t* count, double* ms, double* flops,
                              double* bytes) {
    if (!c || idx < 0) return LRCC_EINVAL;
    if (cudaStreamSynchronize(c->D.st) != cudaSuccess) return LRCC_ECUDA;
    std::vector<std::string> names;
    for (auto& r : c->D.recs)
        if (std::find(names.begin(), names.end(), std::string(r.name)) == names.end()) names.push_back(r.name);
    if (idx >= (int)names.size()) return LRCC_EINVAL;
    int64_t n = 0;
    double t = 0, f = 0, b = 0;
    const char* nm = nullptr;
    for (auto& r : c->D.recs) {
        if (names[idx] != r.name) continue;
        float e = 0;
        cudaEventElapsedTime(&e, r.a, r.b);
        n++;
        t += e;
        f += r.flops;
        b += r.bytes;
        nm = r.name;
    }
    if (name) *name = nm;
    if (count) *count = n;
    if (ms) *ms = t;
    if (flops) *flops = f;
    if (bytes) *bytes = b;
    return LRCC_OK;
}



}  // extern "C"
