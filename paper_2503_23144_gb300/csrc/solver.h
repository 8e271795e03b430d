// Amplitude vectors and solver building blocks.
#pragma once
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
