// Device memory pool, tensor helpers and the elementwise / reduction kernels.
#include "lrcc_internal.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>

// ---------------------------------------------------------------------------
// pool
// ---------------------------------------------------------------------------
static size_t round_size(size_t n) {
    if (n == 0) return 256;
    if (n <= (1u << 20)) return (n + 255) & ~size_t(255);
    return (n + (size_t(2) << 20) - 1) & ~((size_t(2) << 20) - 1);
}

void* Pool::get(size_t n) {
    n = round_size(n);
    largest = std::max(largest, n);
    auto it = cache.find(n);
    if (it != cache.end()) {
        void* p = it->second;
        cache.erase(it);
        cached -= n;
        live += n;
        peak = std::max(peak, live);
        return p;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        trim();
        e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw LrccError(LRCC_ENOMEM, "device allocation of " + std::to_string(n) + " bytes failed");
        }
    }
    live += n;
    peak = std::max(peak, live);
    return p;
}

void Pool::put(void* p, size_t n) {
    if (!p) return;
    n = round_size(n);
    live -= n;
    cached += n;
    cache.emplace(n, p);
}

void Pool::trim() {
    cudaDeviceSynchronize();
    for (auto& kv : cache) cudaFree(kv.second);
    cache.clear();
    cached = 0;
}

Pool::~Pool() {
    for (auto& kv : cache) cudaFree(kv.second);
}

// ---------------------------------------------------------------------------
// tensors
// ---------------------------------------------------------------------------
static void set_contig(Tensor& t, const std::vector<int64_t>& shape) {
    if ((int)shape.size() > MAXD) throw LrccError(LRCC_EINVAL, "tensor rank > 8");
    t.nd = (int)shape.size();
    int64_t st = 1;
    for (int i = t.nd - 1; i >= 0; --i) {
        t.d[i] = shape[i];
        t.s[i] = st;
        st *= shape[i];
    }
}

Tensor empty(Dev& D, std::vector<int64_t> shape) {
    Tensor t;
    set_contig(t, shape);
    size_t bytes = size_t(std::max<int64_t>(t.numel(), 1)) * sizeof(cplx);
    void* p = D.pool.get(bytes);
    t.buf = std::shared_ptr<DevBuf>(new DevBuf{&D.pool, p, bytes});
    t.p = (cplx*)p;
    return t;
}

Tensor zeros(Dev& D, std::vector<int64_t> shape) {
    Tensor t = empty(D, shape);
    if (t.numel() > 0) CK(cudaMemsetAsync(t.p, 0, t.numel() * sizeof(cplx), D.st));
    return t;
}

Tensor wrap(cplx* p, std::vector<int64_t> shape) {
    Tensor t;
    set_contig(t, shape);
    t.p = p;
    return t;
}

Tensor Tensor::reshape(std::vector<int64_t> shape) const {
    if (!contiguous()) throw LrccError(LRCC_EINVAL, "reshape of a non-contiguous tensor");
    Tensor t;
    t.buf = buf;
    set_contig(t, shape);
    if (t.numel() != numel()) throw LrccError(LRCC_EINVAL, "reshape changes the element count");
    t.p = p;
    return t;
}

Tensor Tensor::permute(const std::vector<int>& perm) const {
    Tensor t = *this;
    for (int k = 0; k < nd; ++k) {
        t.d[k] = d[perm[k]];
        t.s[k] = s[perm[k]];
    }
    return t;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
struct ShapeStrides {
    int nd;
    int fast;  // index space below 2^31: decode with fd[]
    int64_t d[MAXD];
    int64_t sx[MAXD];
    int64_t sy[MAXD];
    FastDiv fd[MAXD];
};

// offsets of linear index idx (innermost dimension last) in the x and y views
__device__ __forceinline__ void offsets2(const ShapeStrides& ss, int64_t idx, int64_t& ox, int64_t& oy) {
    ox = 0;
    oy = 0;
    if (ss.fast) {
        uint32_t r = (uint32_t)idx;
        for (int k = ss.nd - 1; k >= 0; --k) {
            const uint32_t q = ss.fd[k].div(r);
            const int64_t c = (int64_t)(r - q * ss.fd[k].d);
            r = q;
            ox += c * ss.sx[k];
            oy += c * ss.sy[k];
        }
        return;
    }
    int64_t r = idx;
    for (int k = ss.nd - 1; k >= 0; --k) {
        const int64_t c = r % ss.d[k];
        r /= ss.d[k];
        ox += c * ss.sx[k];
        oy += c * ss.sy[k];
    }
}

static void set_fast(ShapeStrides& ss, int64_t n) {
    ss.fast = n < FAST_INDEX_LIMIT;
    for (int k = 0; k < ss.nd; ++k) ss.fd[k] = FastDiv(ss.fast ? ss.d[k] : 1);
}

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }

// a * v with the kind of the coefficient decided once per launch (0: +1,
// 1: -1, 2: real, 3: complex): GB300 issues two FP64 FMAs per SM per clock,
// so these memory-bound kernels spend FP64 work only where a coefficient needs it
__device__ __forceinline__ cplx cscale(cplx a, int k, cplx v) {
    if (k == 0) return v;
    if (k == 1) return make_double2(-v.x, -v.y);
    if (k == 2) return make_double2(a.x * v.x, a.x * v.y);
    return cmul(a, v);
}

static int ckind(cplx a) {
    if (a.y == 0.0) {
        if (a.x == 1.0) return 0;
        if (a.x == -1.0) return 1;
        return 2;
    }
    return 3;
}

template <bool BETA0>
__global__ void k_axpby(ShapeStrides ss, int64_t n, cplx alpha, int ka, const cplx* __restrict__ x, int conjx,
                        cplx beta, int kb, cplx* __restrict__ y) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t ox, oy;
        offsets2(ss, idx, ox, oy);
        cplx v = x[ox];
        if (conjx) v.y = -v.y;
        v = cscale(alpha, ka, v);
        if (!BETA0) {
            cplx w = cscale(beta, kb, y[oy]);
            v.x += w.x;
            v.y += w.y;
        }
        y[oy] = v;
    }
}

__global__ void k_fill(ShapeStrides ss, int64_t n, cplx v, cplx* __restrict__ y) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t ox, oy;
        offsets2(ss, idx, ox, oy);
        y[oy] = v;
    }
}

// contiguous fast path
template <bool BETA0>
__global__ void k_axpby_contig(int64_t n, cplx alpha, int ka, const cplx* __restrict__ x, int conjx, cplx beta,
                               int kb, cplx* __restrict__ y) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        cplx v = x[idx];
        if (conjx) v.y = -v.y;
        v = cscale(alpha, ka, v);
        if (!BETA0) {
            cplx w = cscale(beta, kb, y[idx]);
            v.x += w.x;
            v.y += w.y;
        }
        y[idx] = v;
    }
}

static int grid_for(Dev& D, int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)D.sm_count * 16;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

// Drop size-1 dimensions and merge dimensions that are jointly contiguous in
// both x and y (fewer div/mod per element).
static ShapeStrides simplify(const Tensor& x, const Tensor& y) {
    ShapeStrides ss;
    ss.nd = 0;
    for (int k = 0; k < y.nd; ++k) {
        if (y.d[k] == 1) continue;
        if (ss.nd > 0) {
            int j = ss.nd - 1;
            if (ss.sx[j] == x.s[k] * y.d[k] && ss.sy[j] == y.s[k] * y.d[k]) {
                ss.d[j] *= y.d[k];
                ss.sx[j] = x.s[k];
                ss.sy[j] = y.s[k];
                continue;
            }
        }
        ss.d[ss.nd] = y.d[k];
        ss.sx[ss.nd] = x.s[k];
        ss.sy[ss.nd] = y.s[k];
        ss.nd++;
    }
    if (ss.nd == 0) {
        ss.nd = 1;
        ss.d[0] = 1;
        ss.sx[0] = 0;
        ss.sy[0] = 0;
    }
    set_fast(ss, y.numel());
    return ss;
}

// Tiled transpose-axpby for permutations whose innermost dimensions differ:
// a 32x32 tile over (dim kx with x-stride 1, dim ky with y-stride 1) is read
// coalesced along kx into shared memory and written coalesced along ky.
// The remaining dimensions are enumerated by blockIdx.y (batch).
struct TStr {
    int nb;                 // batch dims
    int64_t bd[MAXD];
    int64_t bsx[MAXD], bsy[MAXD];
    int64_t nx, ny;         // extents of the x-inner and y-inner dims
    int64_t sxy, syx;       // x stride of the y-inner dim, y stride of the x-inner dim
    int64_t nbatch;
};

template <bool BETA0>
__global__ void k_transpose(TStr t, cplx alpha, int ka, const cplx* __restrict__ x, int conjx, cplx beta, int kb,
                            cplx* __restrict__ y) {
    __shared__ cplx tile[32][33];
    const int64_t tiles_x = (t.nx + 31) / 32;
    for (int64_t bb = blockIdx.y; bb < t.nbatch; bb += gridDim.y) {
        int64_t r = bb, ox = 0, oy = 0;
        for (int k = t.nb - 1; k >= 0; --k) {
            int64_t c = r % t.bd[k];
            r /= t.bd[k];
            ox += c * t.bsx[k];
            oy += c * t.bsy[k];
        }
        const int64_t tx0 = (blockIdx.x % tiles_x) * 32, ty0 = (blockIdx.x / tiles_x) * 32;
        // read: threadIdx.x runs along the x-inner dim
        for (int j = threadIdx.y; j < 32; j += blockDim.y) {
            int64_t ix = tx0 + threadIdx.x, iy = ty0 + j;
            if (ix < t.nx && iy < t.ny) {
                cplx v = x[ox + ix + iy * t.sxy];
                if (conjx) v.y = -v.y;
                tile[j][threadIdx.x] = v;
            }
        }
        __syncthreads();
        // write: threadIdx.x runs along the y-inner dim
        for (int j = threadIdx.y; j < 32; j += blockDim.y) {
            int64_t iy = ty0 + threadIdx.x, ix = tx0 + j;
            if (ix < t.nx && iy < t.ny) {
                cplx v = tile[threadIdx.x][j];
                cplx o = cscale(alpha, ka, v);
                cplx* yp = y + oy + iy + ix * t.syx;
                if (!BETA0) {
                    const cplx w = cscale(beta, kb, *yp);
                    o.x += w.x;
                    o.y += w.y;
                }
                *yp = o;
            }
        }
        __syncthreads();
    }
}

static bool try_transpose(Dev& D, cplx alpha, const ShapeStrides& ss, const cplx* x, bool conjx, cplx beta, cplx* y) {
    static const bool verbose = getenv("LRCC_VERBOSE") != nullptr;
    if (verbose) {
        fprintf(stderr, "transpose-axpby:");
        for (int k = 0; k < ss.nd; ++k) fprintf(stderr, " %lld(x%lld,y%lld)", (long long)ss.d[k], (long long)ss.sx[k], (long long)ss.sy[k]);
        fprintf(stderr, "\n");
    }
    int kx = -1, ky = -1;
    for (int k = 0; k < ss.nd; ++k) {
        if (ss.sx[k] == 1) kx = k;
        if (ss.sy[k] == 1) ky = k;
    }
    if (kx < 0 || ky < 0 || kx == ky || ss.d[kx] < 8 || ss.d[ky] < 8) return false;
    TStr t;
    t.nb = 0;
    t.nbatch = 1;
    for (int k = 0; k < ss.nd; ++k) {
        if (k == kx || k == ky) continue;
        t.bd[t.nb] = ss.d[k];
        t.bsx[t.nb] = ss.sx[k];
        t.bsy[t.nb] = ss.sy[k];
        t.nbatch *= ss.d[k];
        t.nb++;
    }
    t.nx = ss.d[kx];
    t.ny = ss.d[ky];
    t.sxy = ss.sx[ky];
    t.syx = ss.sy[kx];
    int64_t tiles = ((t.nx + 31) / 32) * ((t.ny + 31) / 32);
    if (tiles > INT32_MAX) return false;
    dim3 block(32, 8);
    dim3 grid((unsigned)tiles, (unsigned)std::min<int64_t>(t.nbatch, 65535));
    bool beta0 = beta.x == 0.0 && beta.y == 0.0;
    const int ka = ckind(alpha), kb = ckind(beta);
    if (beta0) k_transpose<true><<<grid, block, 0, D.st>>>(t, alpha, ka, x, conjx, beta, kb, y);
    else k_transpose<false><<<grid, block, 0, D.st>>>(t, alpha, ka, x, conjx, beta, kb, y);
    LAUNCH_CHECK(D);
    return true;
}

void axpby(Dev& D, cplx alpha, const Tensor& x, bool conjx, cplx beta, Tensor& y) {
    if (x.nd != y.nd) throw LrccError(LRCC_EINVAL, "axpby rank mismatch");
    for (int k = 0; k < y.nd; ++k)
        if (x.d[k] != y.d[k]) throw LrccError(LRCC_EINVAL, "axpby shape mismatch");
    int64_t n = y.numel();
    if (n == 0) return;
    bool beta0 = (beta.x == 0.0 && beta.y == 0.0);
    int th = 256, g = grid_for(D, n, th);
    ShapeStrides ss = simplify(x, y);
    if (ss.nd == 1 && ss.sx[0] == 1 && ss.sy[0] == 1) {
        if (beta0) k_axpby_contig<true><<<g, th, 0, D.st>>>(n, alpha, ckind(alpha), x.p, conjx, beta, 0, y.p);
        else k_axpby_contig<false><<<g, th, 0, D.st>>>(n, alpha, ckind(alpha), x.p, conjx, beta, ckind(beta), y.p);
    } else if (try_transpose(D, alpha, ss, x.p, conjx, beta, y.p)) {
        return;
    } else {
        if (beta0) k_axpby<true><<<g, th, 0, D.st>>>(ss, n, alpha, ckind(alpha), x.p, conjx, beta, 0, y.p);
        else k_axpby<false><<<g, th, 0, D.st>>>(ss, n, alpha, ckind(alpha), x.p, conjx, beta, ckind(beta), y.p);
    }
    LAUNCH_CHECK(D);
}

void fill(Dev& D, Tensor& y, cplx v) {
    int64_t n = y.numel();
    if (n == 0) return;
    ShapeStrides ss = simplify(y, y);
    int th = 256, g = grid_for(D, n, th);
    k_fill<<<g, th, 0, D.st>>>(ss, n, v, y.p);
    LAUNCH_CHECK(D);
}

// max |y| per row block; out[row] (double) via atomicMax on the bit pattern
// (non-negative doubles order like their int64 images)
__global__ void k_maxabs(ShapeStrides ss, int64_t n, int64_t per_row, const cplx* __restrict__ y,
                         unsigned long long* out) {
    __shared__ double red[32];
    int64_t row = blockIdx.y;
    double m = 0.0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < per_row;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t ox, oy;
        offsets2(ss, row * per_row + idx, ox, oy);
        cplx v = y[oy];
        double a = sqrt(v.x * v.x + v.y * v.y);
        if (!(a <= 1e300)) a = 1e308;  // NaN / Inf -> huge
        m = fmax(m, a);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffff, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffff, m, o));
        if (threadIdx.x == 0) atomicMax(out + row, (unsigned long long)__double_as_longlong(m));
    }
}

void max_abs_rows(Dev& D, const Tensor& y, double* out_dev) {
    int64_t rows = y.nd > 0 ? y.d[0] : 1;
    int64_t n = y.numel();
    int64_t per_row = rows ? n / rows : 0;
    CK(cudaMemsetAsync(out_dev, 0, sizeof(double) * rows, D.st));
    if (n == 0) return;
    ShapeStrides ss = simplify(y, y);
    int th = 256;
    int gx = (int)std::max<int64_t>(1, std::min<int64_t>((per_row + th - 1) / th, std::max<int64_t>(1, D.sm_count * 8 / rows)));
    dim3 grid(gx, (unsigned)rows);
    k_maxabs<<<grid, th, 0, D.st>>>(ss, n, per_row, y.p, (unsigned long long*)out_dev);
    LAUNCH_CHECK(D);
}

double max_abs(Dev& D, const Tensor& y) {
    Tensor flat = y;
    // view as one row
    Tensor one;
    one = y;
    double* dv = (double*)D.pool.get(sizeof(double));
    std::shared_ptr<DevBuf> hold(new DevBuf{&D.pool, dv, sizeof(double)});
    // prepend a unit dimension
    Tensor v = y;
    if (v.nd >= MAXD) throw LrccError(LRCC_EINVAL, "rank too large for max_abs");
    for (int k = v.nd; k > 0; --k) {
        v.d[k] = v.d[k - 1];
        v.s[k] = v.s[k - 1];
    }
    v.d[0] = 1;
    v.s[0] = 0;
    v.nd++;
    max_abs_rows(D, v, dv);
    double h = 0;
    CK(cudaMemcpyAsync(&h, dv, sizeof(double), cudaMemcpyDeviceToHost, D.st));
    CK(cudaStreamSynchronize(D.st));
    return h;
}

// ---------------------------------------------------------------------------
// broadcast product: C = alpha * op(A) * op(B) + beta * C elementwise over C's
// index space (an einsum without contracted labels), offsets from strides
// ---------------------------------------------------------------------------
struct Str3 {
    int nd;
    int fast;
    int64_t d[MAXD];
    int64_t sa[MAXD], sb[MAXD], sc[MAXD];
    FastDiv fd[MAXD];
};

// LOWP (mixed-precision products): the product and alpha in FP32 arithmetic
// (relative error 2^-23, far below the tensor-core products it joins), only
// the accumulation into C in FP64
__device__ __forceinline__ float2 f2of(cplx v, int cj) {
    const float i = f64_to_f32_rz(v.y);
    return make_float2(f64_to_f32_rz(v.x), cj ? -i : i);
}
__device__ __forceinline__ float2 fscale(float2 a, int k, float2 v) {
    if (k == 0) return v;
    if (k == 1) return make_float2(-v.x, -v.y);
    return make_float2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
}

template <bool BETA0, bool LOWP>
__global__ void k_outer(Str3 s, int64_t n, cplx alpha, int ka, const cplx* __restrict__ a, int ca,
                        const cplx* __restrict__ b, int cb, cplx beta, int kb, cplx* __restrict__ c) {
    const float2 af = make_float2((float)alpha.x, (float)alpha.y);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t oa = 0, ob = 0, oc = 0;
        if (s.fast) {
            uint32_t r = (uint32_t)idx;
            for (int k = s.nd - 1; k >= 0; --k) {
                const uint32_t qq = s.fd[k].div(r);
                const int64_t q = (int64_t)(r - qq * s.fd[k].d);
                r = qq;
                oa += q * s.sa[k];
                ob += q * s.sb[k];
                oc += q * s.sc[k];
            }
        } else {
            int64_t r = idx;
            for (int k = s.nd - 1; k >= 0; --k) {
                int64_t q = r % s.d[k];
                r /= s.d[k];
                oa += q * s.sa[k];
                ob += q * s.sb[k];
                oc += q * s.sc[k];
            }
        }
        cplx p;
        if (LOWP) {
            const float2 u = f2of(a[oa], ca), v = f2of(b[ob], cb);
            const float2 q = fscale(af, ka, make_float2(u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x));
            p = make_double2(f32_to_f64(q.x), f32_to_f64(q.y));
        } else {
            cplx u = a[oa], v = b[ob];
            if (ca) u.y = -u.y;
            if (cb) v.y = -v.y;
            p = cscale(alpha, ka, cmul(u, v));
        }
        if (!BETA0) {
            cplx w = cscale(beta, kb, c[oc]);
            p.x += w.x;
            p.y += w.y;
        }
        c[oc] = p;
    }
}

// A, B given as views over C's dimensions (stride 0 where a label is absent)
void outer_axpby(Dev& D, cplx alpha, const Tensor& A, bool ca, const Tensor& B, bool cb, cplx beta, Tensor& C,
                 bool lowp) {
    Str3 s;
    s.nd = 0;
    for (int k = 0; k < C.nd; ++k) {
        if (C.d[k] == 1) continue;
        if (s.nd > 0) {
            int j = s.nd - 1;
            if (s.sa[j] == A.s[k] * C.d[k] && s.sb[j] == B.s[k] * C.d[k] && s.sc[j] == C.s[k] * C.d[k]) {
                s.d[j] *= C.d[k];
                s.sa[j] = A.s[k];
                s.sb[j] = B.s[k];
                s.sc[j] = C.s[k];
                continue;
            }
        }
        s.d[s.nd] = C.d[k];
        s.sa[s.nd] = A.s[k];
        s.sb[s.nd] = B.s[k];
        s.sc[s.nd] = C.s[k];
        s.nd++;
    }
    if (s.nd == 0) {
        s.nd = 1;
        s.d[0] = 1;
        s.sa[0] = s.sb[0] = s.sc[0] = 0;
    }
    int64_t n = C.numel();
    if (n == 0) return;
    s.fast = n < FAST_INDEX_LIMIT;
    for (int k = 0; k < s.nd; ++k) s.fd[k] = FastDiv(s.fast ? s.d[k] : 1);
    bool beta0 = beta.x == 0.0 && beta.y == 0.0;
    int th = 256, g = grid_for(D, n, th);
    const int ka = ckind(alpha), kb = ckind(beta);
    if (lowp) {
        if (beta0) k_outer<true, true><<<g, th, 0, D.st>>>(s, n, alpha, ka, A.p, ca, B.p, cb, beta, kb, C.p);
        else k_outer<false, true><<<g, th, 0, D.st>>>(s, n, alpha, ka, A.p, ca, B.p, cb, beta, kb, C.p);
    } else {
        if (beta0) k_outer<true, false><<<g, th, 0, D.st>>>(s, n, alpha, ka, A.p, ca, B.p, cb, beta, kb, C.p);
        else k_outer<false, false><<<g, th, 0, D.st>>>(s, n, alpha, ka, A.p, ca, B.p, cb, beta, kb, C.p);
    }
    LAUNCH_CHECK(D);
}

// ---------------------------------------------------------------------------
// antisymmetrisers on contiguous [nb][O][O][V][V]:
//   mode 1: x_ijab - x_jiab,  mode 2: x_ijab - x_ijba,  mode 3: both (4 terms)
// y = alpha * P x + beta * y.  Each P is its own transpose.
// ---------------------------------------------------------------------------
constexpr int AT = 16;  // antisymmetriser tile edge

// Tiled antisymmetriser: one block handles the (i<j) pair of planes
// x[r][i][j], x[r][j][i] and one (a-tile <= b-tile) pair of 16x16 tiles, so
// every input is read once, coalesced, and the four outputs
//   out(ij,ab) = x(ij,ab) - x(ji,ab) - x(ij,ba) + x(ji,ba)   (mode 3)
//   out(ji,ab) = -out(ij,ab), out(ij,ba) = -out(ij,ab), out(ji,ba) = out(ij,ab)
// are written from the same registers (modes 1 and 2 keep only their terms).
// Diagonal planes (i = j) and diagonal elements (a = b) come out as the mode
// defines them (zero where the antisymmetriser vanishes).
template <bool BETA0>
__global__ void __launch_bounds__(256) k_asym_t(int mode, int64_t R, int64_t O, int64_t V, cplx alpha, int ka,
                                                const cplx* __restrict__ x, cplx beta, int kb,
                                                cplx* __restrict__ y) {
    // [ij,ab] [ji,ab] [ij,ba] [ji,ba] tiles, as [row a][col b] / [row b][col a]
    __shared__ cplx tsm[4 * AT * (AT + 1)];
    const int64_t VV = V * V, OVV = O * VV;
    const int64_t T = (V + AT - 1) / AT, tpairs = T * (T + 1) / 2, opairs = O * (O + 1) / 2;
    const int64_t tasks = R * opairs * tpairs;
    const int tx = threadIdx.x % AT, ty = threadIdx.x / AT;
    for (int64_t task = blockIdx.x; task < tasks; task += gridDim.x) {
        int64_t rem = task % tpairs, ta = 0;
        const int64_t u = task / tpairs;
        while (rem >= T - ta) {
            rem -= T - ta;
            ++ta;
        }
        const int64_t tb = ta + rem;
        int64_t orem = u % opairs, i = 0;
        const int64_t r = u / opairs;
        while (orem >= O - i) {
            orem -= O - i;
            ++i;
        }
        const int64_t j = i + orem;  // i <= j
        const int64_t a0 = ta * AT, b0 = tb * AT;
        const cplx* xij = x + r * O * OVV + i * OVV + j * VV;
        const cplx* xji = x + r * O * OVV + j * OVV + i * VV;
        // load [ij][a][b] and [ji][a][b] tiles (rows a, cols b) and the
        // transposed-position tiles [ij][b][a], [ji][b][a] (rows b, cols a)
        for (int q = ty; q < AT; q += 256 / AT) {
            const int64_t a = a0 + q, b = b0 + tx;
            const bool in1 = a < V && b < V;
            tsm[(0 * AT + q) * (AT + 1) + tx] = in1 ? xij[a * V + b] : make_double2(0.0, 0.0);
            tsm[(1 * AT + q) * (AT + 1) + tx] = in1 ? xji[a * V + b] : make_double2(0.0, 0.0);
            const int64_t bb = b0 + q, aa = a0 + tx;
            const bool in2 = bb < V && aa < V;
            tsm[(2 * AT + q) * (AT + 1) + tx] = in2 ? xij[bb * V + aa] : make_double2(0.0, 0.0);
            tsm[(3 * AT + q) * (AT + 1) + tx] = in2 ? xji[bb * V + aa] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        cplx* yij = y + r * O * OVV + i * OVV + j * VV;
        cplx* yji = y + r * O * OVV + j * OVV + i * VV;
        // outputs at (a, b) for the (ij) and (ji) planes, rows a, cols b
        for (int q = ty; q < AT; q += 256 / AT) {
            const int64_t a = a0 + q, b = b0 + tx;
            if (a < V && b < V && (ta != tb || a <= b)) {
                const cplx p0 = tsm[(0 * AT + q) * (AT + 1) + tx], p1 = tsm[(1 * AT + q) * (AT + 1) + tx];
                const cplx p2 = tsm[(2 * AT + tx) * (AT + 1) + q], p3 = tsm[(3 * AT + tx) * (AT + 1) + q];
                cplx v = p0;
                if (mode & 1) { v.x -= p1.x; v.y -= p1.y; }
                if (mode & 2) { v.x -= p2.x; v.y -= p2.y; }
                if (mode == 3) { v.x += p3.x; v.y += p3.y; }
                v = cscale(alpha, ka, v);
                // (ij,ab) and, for i < j, (ji,ab) = -(ij,ab) in modes 1, 3; mode 2 has its own value there
                cplx w = v;
                if (!BETA0) w = cadd(w, cscale(beta, kb, yij[a * V + b]));
                yij[a * V + b] = w;
                if (i != j) {
                    cplx vj;
                    if (mode == 2) {
                        vj = make_double2(p1.x - p3.x, p1.y - p3.y);
                        vj = cscale(alpha, ka, vj);
                    } else {
                        vj = make_double2(-v.x, -v.y);
                    }
                    if (!BETA0) vj = cadd(vj, cscale(beta, kb, yji[a * V + b]));
                    yji[a * V + b] = vj;
                }
            }
        }
        // outputs at (b, a) (the transposed positions, a < b strictly), rows b, cols a
        for (int q = ty; q < AT; q += 256 / AT) {
            const int64_t bb = b0 + q, aa = a0 + tx;
            if (bb < V && aa < V && (ta != tb || aa < bb)) {
                // values at (ij,ba) built from the same four inputs
                const cplx p0 = tsm[(2 * AT + q) * (AT + 1) + tx], p1 = tsm[(3 * AT + q) * (AT + 1) + tx];
                const cplx p2 = tsm[(0 * AT + tx) * (AT + 1) + q], p3 = tsm[(1 * AT + tx) * (AT + 1) + q];
                cplx v = p0;
                if (mode & 1) { v.x -= p1.x; v.y -= p1.y; }
                if (mode & 2) { v.x -= p2.x; v.y -= p2.y; }
                if (mode == 3) { v.x += p3.x; v.y += p3.y; }
                v = cscale(alpha, ka, v);
                cplx w = v;
                if (!BETA0) w = cadd(w, cscale(beta, kb, yij[bb * V + aa]));
                yij[bb * V + aa] = w;
                if (i != j) {
                    cplx vj;
                    if (mode == 2) {
                        vj = make_double2(p1.x - p3.x, p1.y - p3.y);
                        vj = cscale(alpha, ka, vj);
                    } else {
                        vj = make_double2(-v.x, -v.y);
                    }
                    if (!BETA0) vj = cadd(vj, cscale(beta, kb, yji[bb * V + aa]));
                    yji[bb * V + aa] = vj;
                }
            }
        }
        __syncthreads();
    }
}

void asym_axpby(Dev& D, int mode, cplx alpha, const Tensor& x, cplx beta, Tensor& y) {
    REQUIRE(mode >= 1 && mode <= 3, "asym: bad mode");
    REQUIRE(x.contiguous() && y.contiguous() && x.numel() == y.numel() && x.nd >= 4 && y.nd >= 4,
            "asym: contiguous [..][O][O][V][V] tensors expected");
    int64_t O = x.d[x.nd - 4], V = x.d[x.nd - 1];
    REQUIRE(x.d[x.nd - 3] == O && x.d[x.nd - 2] == V, "asym: [..][O][O][V][V] expected");
    int64_t n = y.numel();
    if (n == 0) return;
    REQUIRE(x.p != y.p, "asym: in-place use is not supported");
    const int64_t R = n / (O * O * V * V);
    bool beta0 = beta.x == 0.0 && beta.y == 0.0;
    const int ka = ckind(alpha), kb = ckind(beta);
    const int64_t T = (V + AT - 1) / AT, tasks = R * (O * (O + 1) / 2) * (T * (T + 1) / 2);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(tasks, (int64_t)D.sm_count * 16));
    if (beta0) k_asym_t<true><<<g, 256, 0, D.st>>>(mode, R, O, V, alpha, ka, x.p, beta, kb, y.p);
    else k_asym_t<false><<<g, 256, 0, D.st>>>(mode, R, O, V, alpha, ka, x.p, beta, kb, y.p);
    LAUNCH_CHECK(D);
}
