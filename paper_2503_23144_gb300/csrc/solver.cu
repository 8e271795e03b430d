// Amplitude-vector kernels, device-side Pulay DIIS and the iterative solves
// of the ground state (T, Lambda) and of the response equations (X, Y).
#include "solver.h"

#include <algorithm>
#include <cmath>

namespace {

int grid_n(Dev& D, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)D.sm_count * 16));
}

// out = x - r / (D + shift[r]);  D1 = ev[a]-eo[i], D2 = ev[a]+ev[b]-eo[i]-eo[j]
__global__ void k_precond(const cplx* __restrict__ x1, const cplx* __restrict__ r1, cplx* __restrict__ o1,
                          const cplx* __restrict__ x2, const cplx* __restrict__ r2, cplx* __restrict__ o2,
                          int64_t R, int64_t O, int64_t V, FastDiv fO, FastDiv fV, FastDiv fn1, FastDiv fn2,
                          const double* __restrict__ eo, const double* __restrict__ ev,
                          const double* __restrict__ shift, int x_zero) {
    int64_t n1 = O * V, n2 = O * O * V * V;
    int64_t total = R * (n1 + n2);
    const bool fast = total < FAST_INDEX_LIMIT;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        bool singles = idx < R * n1;
        int64_t k = singles ? idx : idx - R * n1;
        int64_t r, i, j = 0, a, b = 0;
        if (fast) {
            uint32_t u = (uint32_t)k, q;
            if (singles) {
                q = fn1.div(u);
                r = q;
                u -= q * fn1.d;
                q = fV.div(u);
                a = u - q * fV.d;
                i = q;
            } else {
                q = fn2.div(u);
                r = q;
                u -= q * fn2.d;
                q = fV.div(u);
                b = u - q * fV.d;
                u = q;
                q = fV.div(u);
                a = u - q * fV.d;
                u = q;
                q = fO.div(u);
                j = u - q * fO.d;
                i = q;
            }
        } else {
            int64_t n = singles ? n1 : n2;
            r = k / n;
            int64_t e = k % n;
            if (singles) {
                a = e % V;
                i = e / V;
            } else {
                b = e % V;
                int64_t t = e / V;
                a = t % V;
                t /= V;
                j = t % O;
                i = t / O;
            }
        }
        double d = singles ? ev[a] - eo[i] : ev[a] + ev[b] - eo[i] - eo[j];
        const double inv = 1.0 / (d + shift[r]);
        const cplx* x = singles ? x1 : x2;
        const cplx* rr = singles ? r1 : r2;
        cplx* o = singles ? o1 : o2;
        cplx v = rr[k];
        cplx xv = x_zero ? make_double2(0.0, 0.0) : x[k];
        o[k] = make_double2(xv.x - v.x * inv, xv.y - v.y * inv);
    }
}

// out[r][e] = s[r][e] + coef[r] * x[r][e] + b[r][e]     (b may be null)
__global__ void k_combine(int64_t R, int64_t n, FastDiv fn, const cplx* __restrict__ s, const cplx* __restrict__ x,
                          const double* __restrict__ coef, const cplx* __restrict__ b, cplx* __restrict__ out) {
    int64_t total = R * n;
    const bool fast = total < FAST_INDEX_LIMIT;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = fast ? (int64_t)fn.div((uint32_t)idx) : idx / n;
        cplx v = s[idx], xv = x[idx];
        double c = coef[r];
        v.x += c * xv.x;
        v.y += c * xv.y;
        if (b) {
            v.x += b[idx].x;
            v.y += b[idx].y;
        }
        out[idx] = v;
    }
}

// G[r][i][s] = d[r], G[r][s][i] = conj d[r]
__global__ void k_gram_set(cplx* G, int R, int nmax, int i, int s, const cplx* d) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    cplx v = d[r];
    G[(int64_t(r) * nmax + i) * nmax + s] = v;
    G[(int64_t(r) * nmax + s) * nmax + i] = make_double2(v.x, -v.y);
}

__device__ inline cplx cm(cplx a, cplx b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline cplx cdv(cplx a, cplx b) {
    double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// Pulay system per right-hand side:  [G 1; 1^T 0] [c; l] = [0; 1] (scaled),
// slots[k] lists the stored vectors oldest first.  One thread per RHS.
__global__ void k_diis_solve(const cplx* G, int R, int nmax, const int* slots, int k, cplx* coef) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    constexpr int MX = 17;
    cplx A[MX][MX + 1];
    int n = k + 1;
    double sc = 0.0;
    for (int i = 0; i < k; ++i) {
        cplx g = G[(int64_t(r) * nmax + slots[i]) * nmax + slots[i]];
        sc = fmax(sc, g.x);
    }
    if (!(sc > 0.0)) sc = 1.0;
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) {
            cplx g = G[(int64_t(r) * nmax + slots[i]) * nmax + slots[j]];
            A[i][j] = make_double2(g.x / sc, g.y / sc);
        }
        A[i][k] = make_double2(-1.0, 0.0);
        A[k][i] = make_double2(-1.0, 0.0);
        A[i][n] = make_double2(0.0, 0.0);
    }
    A[k][k] = make_double2(0.0, 0.0);
    A[k][n] = make_double2(-1.0, 0.0);
    bool ok = true;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = 0.0;
        for (int i = c; i < n; ++i) {
            double m = A[i][c].x * A[i][c].x + A[i][c].y * A[i][c].y;
            if (m > best) { best = m; piv = i; }
        }
        if (!(best > 1e-300)) { ok = false; break; }
        if (piv != c)
            for (int j = 0; j <= n; ++j) { cplx t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
        for (int i = c + 1; i < n; ++i) {
            cplx f = cdv(A[i][c], A[c][c]);
            for (int j = c; j <= n; ++j) {
                cplx p = cm(f, A[c][j]);
                A[i][j].x -= p.x;
                A[i][j].y -= p.y;
            }
        }
    }
    cplx x[MX];
    if (ok) {
        for (int i = n - 1; i >= 0; --i) {
            cplx s = A[i][n];
            for (int j = i + 1; j < n; ++j) {
                cplx p = cm(A[i][j], x[j]);
                s.x -= p.x;
                s.y -= p.y;
            }
            x[i] = cdv(s, A[i][i]);
            if (!isfinite(x[i].x) || !isfinite(x[i].y)) ok = false;
        }
    }
    for (int i = 0; i < k; ++i) {
        cplx v = ok ? x[i] : make_double2(i == k - 1 ? 1.0 : 0.0, 0.0);
        coef[int64_t(r) * nmax + slots[i]] = v;
    }
}

struct Ptrs {
    const cplx* p[16];
};

// out[r][e] = sum_i coef[r][slot_i] * v_i[r][e]
__global__ void k_lincomb(int64_t R, int64_t n, FastDiv fn, Ptrs v, int k, const int* slots_unused,
                          const cplx* coef, int nmax, const int* slots, cplx* __restrict__ out) {
    (void)slots_unused;
    int64_t total = R * n;
    const bool fast = total < FAST_INDEX_LIMIT;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = fast ? (int64_t)fn.div((uint32_t)idx) : idx / n;
        double sx = 0, sy = 0;
        for (int i = 0; i < k; ++i) {
            cplx c = coef[r * nmax + slots[i]];
            cplx x = v.p[i][idx];
            sx += c.x * x.x - c.y * x.y;
            sy += c.x * x.y + c.y * x.x;
        }
        out[idx] = make_double2(sx, sy);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
Amp amp_empty(Dev& D, int64_t R, int64_t O, int64_t V) {
    return Amp{empty(D, {R, O, V}), empty(D, {R, O, O, V, V})};
}
Amp amp_zeros(Dev& D, int64_t R, int64_t O, int64_t V) {
    return Amp{zeros(D, {R, O, V}), zeros(D, {R, O, O, V, V})};
}

void precond(Dev& D, const Amp* x, const Amp& r, Amp& out, const double* eo, const double* ev,
             const double* shift_dev) {
    int64_t R = r.t1.d[0], O = r.t1.d[1], V = r.t1.d[2];
    int64_t total = R * (O * V + O * O * V * V);
    k_precond<<<grid_n(D, total), 256, 0, D.st>>>(x ? x->t1.p : nullptr, r.t1.p, out.t1.p, x ? x->t2.p : nullptr,
                                                     r.t2.p, out.t2.p, R, O, V, FastDiv(O), FastDiv(V),
                                                     FastDiv(O * V), FastDiv(O * O * V * V), eo, ev, shift_dev,
                                                     x ? 0 : 1);
    LAUNCH_CHECK(D);
}

void combine(Dev& D, const Amp& s, const Amp& x, const double* coef_dev, const Amp* b, Amp& out) {
    int64_t R = s.t1.d[0];
    int64_t n1 = s.t1.numel() / R, n2 = s.t2.numel() / R;
    k_combine<<<grid_n(D, R * n1), 256, 0, D.st>>>(R, n1, FastDiv(n1), s.t1.p, x.t1.p, coef_dev, b ? b->t1.p : nullptr, out.t1.p);
    LAUNCH_CHECK(D);
    k_combine<<<grid_n(D, R * n2), 256, 0, D.st>>>(R, n2, FastDiv(n2), s.t2.p, x.t2.p, coef_dev, b ? b->t2.p : nullptr, out.t2.p);
    LAUNCH_CHECK(D);
}

// per-RHS sum over unique amplitudes of op(a) b  (conj a if ca)
Tensor amp_dot(Dev& D, const Amp& a, bool ca, const Amp& b) {
    int64_t R = a.t1.d[0];
    Tensor out = empty(D, {R});
    ein(D, "Zia,Zia->Z", mkc(1.0), a.t1, ca, b.t1, false, mkc(0.0), out);
    ein(D, "Zijab,Zijab->Z", mkc(0.25), a.t2, ca, b.t2, false, mkc(1.0), out);
    return out;
}

// dots of each RHS of a [R] with one fixed (unbatched) vector b [1]
Tensor amp_dot_fixed(Dev& D, const Amp& a, const Amp& b1) {
    int64_t R = a.t1.d[0];
    Tensor out = empty(D, {R});
    ein(D, "Zia,ia->Z", mkc(1.0), a.t1, false, b1.t1.index(0), false, mkc(0.0), out);
    ein(D, "Zijab,ijab->Z", mkc(0.25), a.t2, false, b1.t2.index(0), false, mkc(1.0), out);
    return out;
}

// G[p][q] = sum over unique amplitudes of U_p W_q (unconjugated), U [P], W [Q]
Tensor amp_gram(Dev& D, const Amp& U, const Amp& W) {
    Tensor G = empty(D, {U.t1.d[0], W.t1.d[0]});
    ein(D, "Pia,Qia->PQ", mkc(1.0), U.t1, false, W.t1, false, mkc(0.0), G);
    ein(D, "Pijab,Qijab->PQ", mkc(0.25), U.t2, false, W.t2, false, mkc(1.0), G);
    return G;
}

Amp amp_rows(const Amp& a, int64_t r0, int64_t n) { return Amp{a.t1.slice(0, r0, n), a.t2.slice(0, r0, n)}; }

void amp_axpby(Dev& D, cplx a, const Amp& x, cplx b, Amp& y) {
    axpby(D, a, x.t1, false, b, y.t1);
    axpby(D, a, x.t2, false, b, y.t2);
}

Amp amp_copy(Dev& D, const Amp& x) {
    Amp y = amp_empty(D, x.t1.d[0], x.t1.d[1], x.t1.d[2]);
    amp_axpby(D, mkc(1.0), x, mkc(0.0), y);
    return y;
}

// y = x - P_ij x - P_ab x + P_ij P_ab x on [R][O][O][V][V]
Tensor antisym4(Dev& D, const Tensor& x) {
    Tensor y = empty(D, x.shape());
    asym_axpby(D, 3, mkc(1.0), x, mkc(0.0), y);
    return y;
}

void max_abs_amp(Dev& D, const Amp& r, std::vector<double>& out) {
    int64_t R = r.t1.d[0];
    double* dv = (double*)D.pool.get(sizeof(double) * 2 * R);
    std::shared_ptr<DevBuf> hold(new DevBuf{&D.pool, dv, sizeof(double) * 2 * R});
    max_abs_rows(D, r.t1, dv);
    max_abs_rows(D, r.t2, dv + R);
    std::vector<double> h(2 * R);
    CK(cudaMemcpyAsync(h.data(), dv, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, D.st));
    CK(cudaStreamSynchronize(D.st));
    out.resize(R);
    for (int64_t r = 0; r < R; ++r) out[r] = std::max(h[r], h[R + r]);
}

// ---------------------------------------------------------------------------
Diis::Diis(Dev& D, int R_, int nmax_) : R(R_), nmax(std::min(std::max(nmax_, 2), 16)) {
    gram = zeros(D, {R, nmax, nmax});
    coef = empty(D, {R, nmax});
    xs.resize(nmax);
    es.resize(nmax);
    CK(cudaMalloc(&slots_dev, sizeof(int) * 16));
}
Diis::~Diis() {
    if (slots_dev) cudaFree(slots_dev);
}

// The history is kept in packed form: singles as they are and the doubles by
// their unique pairs (i<j, a<b), [R][P_O P_V] -- a quarter of the full
// antisymmetric array, exact for antisymmetric amplitudes -- so that a long
// history of many right-hand sides fits next to the residual sweeps.
namespace {
Amp pack_amp(Dev& D, const Amp& x) {
    const int64_t R = x.t1.d[0], O = x.t1.d[1], V = x.t1.d[2];
    REQUIRE(x.t2.contiguous(), "DIIS: doubles must be contiguous");
    Amp p;
    p.t1 = empty(D, x.t1.shape());
    axpby(D, mkc(1.0), x.t1, false, mkc(0.0), p.t1);
    p.t2 = empty(D, {R, O * (O - 1) / 2 * (V * (V - 1) / 2)});
    ladder_pack_xt(D, x.t2.p, p.t2.p, R, O, V);
    return p;
}
// per-RHS dot over unique amplitudes of packed vectors (conjugated first)
Tensor packed_dot(Dev& D, const Amp& a, const Amp& b) {
    Tensor out = empty(D, {a.t1.d[0]});
    ein(D, "Zia,Zia->Z", mkc(1.0), a.t1, true, b.t1, false, mkc(0.0), out);
    ein(D, "Zk,Zk->Z", mkc(1.0), a.t2, true, b.t2, false, mkc(1.0), out);
    return out;
}
}  // namespace

Amp Diis::push_extrapolate(Dev& D, const Amp& x, const Amp& e) {
    int s = count % nmax;
    xs[s] = pack_amp(D, x);
    es[s] = pack_amp(D, e);
    count++;
    int k = std::min(count, nmax);
    // stored slots oldest first
    std::vector<int> sl;
    for (int q = count - k; q < count; ++q) sl.push_back(q % nmax);
    for (int i : sl) {
        Tensor d = packed_dot(D, es[i], es[s]);
        k_gram_set<<<(R + 127) / 128, 128, 0, D.st>>>(gram.p, R, nmax, i, s, d.p);
        LAUNCH_CHECK(D);
    }
    if (k < 2) return x;
    CK(cudaMemcpyAsync(slots_dev, sl.data(), sizeof(int) * k, cudaMemcpyHostToDevice, D.st));
    k_diis_solve<<<(R + 63) / 64, 64, 0, D.st>>>(gram.p, R, nmax, slots_dev, k, coef.p);
    LAUNCH_CHECK(D);
    const int64_t O = x.t1.d[1], V = x.t1.d[2];
    Amp out = amp_empty(D, R, O, V);
    Tensor t2p = empty(D, xs[s].t2.shape());
    Ptrs p1, p2;
    for (int i = 0; i < k; ++i) {
        p1.p[i] = xs[sl[i]].t1.p;
        p2.p[i] = xs[sl[i]].t2.p;
    }
    int64_t n1 = x.t1.numel() / R, n2 = t2p.numel() / R;
    k_lincomb<<<grid_n(D, R * n1), 256, 0, D.st>>>(R, n1, FastDiv(n1), p1, k, nullptr, coef.p, nmax, slots_dev, out.t1.p);
    LAUNCH_CHECK(D);
    k_lincomb<<<grid_n(D, R * n2), 256, 0, D.st>>>(R, n2, FastDiv(n2), p2, k, nullptr, coef.p, nmax, slots_dev, t2p.p);
    LAUNCH_CHECK(D);
    ladder_unpack_zt(D, t2p.p, out.t2.p, R, O, V, mkc(1.0), mkc(0.0));
    // the host copy of the slot list must outlive the async copy
    CK(cudaStreamSynchronize(D.st));
    return out;
}
