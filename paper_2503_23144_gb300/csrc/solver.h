// Amplitude vectors and solver building blocks.
#pragma once
#include <functional>

#include "prog.h"

// amplitudes of R right-hand sides: singles [R][O][V], full antisymmetric
// doubles [R][O][O][V][V]
struct Amp {
    Tensor t1, t2;
};

Amp amp_empty(Dev& D, int64_t R, int64_t O, int64_t V);
Amp amp_zeros(Dev& D, int64_t R, int64_t O, int64_t V);
Amp amp_copy(Dev& D, const Amp& x);
void amp_axpby(Dev& D, cplx a, const Amp& x, cplx b, Amp& y);
// out = x - r/(D + shift[r]) (x == nullptr: x = 0); D from orbital energies
void precond(Dev& D, const Amp* x, const Amp& r, Amp& out, const double* eo, const double* ev,
             const double* shift_dev);
// out = s + coef[r] x + b
void combine(Dev& D, const Amp& s, const Amp& x, const double* coef_dev, const Amp* b, Amp& out);
// per-RHS unique-amplitude dot: sum_ia op(a)b + 1/4 sum_ijab op(a)b -> [R]
Tensor amp_dot(Dev& D, const Amp& a, bool conj_a, const Amp& b);
Tensor amp_dot_fixed(Dev& D, const Amp& a, const Amp& b1);
// Gram matrix of unconjugated unique-amplitude dots between the rows of U and W
Tensor amp_gram(Dev& D, const Amp& U, const Amp& W);
// rows [r0, r0+n) of a batched amplitude set (a view)
Amp amp_rows(const Amp& a, int64_t r0, int64_t n);
// 4-fold antisymmetriser over the (i,j) and (a,b) pairs
Tensor antisym4(Dev& D, const Tensor& x);
void max_abs_amp(Dev& D, const Amp& r, std::vector<double>& out);

// Shared-subspace solve of (M + shift_r) z_r = -b_r for all R right-hand sides
// at once (one orthonormal subspace, Galerkin projections, the products M v
// shared by every shift); apply(v) = M v on a batch of vectors; prec
// (LRCC_FP64 or LRCC_FP64_EMULATED) for the projections.  Counts the batched
// products in n_products.
void subspace_solve(Dev& D, int O, int V, const double* eo, const double* ev, Amp& z, const Amp& b,
                    const double* shift_dev, const std::vector<double>& shift,
                    const std::function<Amp(const Amp&)>& apply, int prec, double tol, int max_iter,
                    int requested_max, std::vector<double>& final_res, int& n_products);
// vectors the shared subspace holds for R right-hand sides: requested (> 0) or
// automatic (8 R within 48..400), at most what fits in 30 % of device memory
int64_t subspace_capacity(Dev& D, int O, int V, int64_t R, int requested);

// Pulay DIIS over R independent right-hand sides; Gram matrices, the small
// linear solves and the extrapolation all run on the device.
struct Diis {
    int R, nmax, count = 0;
    std::vector<Amp> xs, es;
    Tensor gram, coef;
    int* slots_dev = nullptr;
    Diis(Dev& D, int R, int nmax);
    ~Diis();
    Diis(const Diis&) = delete;
    Diis& operator=(const Diis&) = delete;
    Amp push_extrapolate(Dev& D, const Amp& x, const Amp& e);
};
