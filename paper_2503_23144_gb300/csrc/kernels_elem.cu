// Device memory pool, tensor helpers and the elementwise / reduction kernels.
#include "lrcc_internal.h"

#include <algorithm>

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
    int64_t d[MAXD];
    int64_t sx[MAXD];
    int64_t sy[MAXD];
};

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool BETA0>
__global__ void k_axpby(ShapeStrides ss, int64_t n, cplx alpha, const cplx* __restrict__ x, int conjx,
                        cplx beta, cplx* __restrict__ y) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = idx, ox = 0, oy = 0;
        for (int k = ss.nd - 1; k >= 0; --k) {
            int64_t c = r % ss.d[k];
            r /= ss.d[k];
            ox += c * ss.sx[k];
            oy += c * ss.sy[k];
        }
        cplx v = x[ox];
        if (conjx) v.y = -v.y;
        v = cmul(alpha, v);
        if (!BETA0) {
            cplx w = cmul(beta, y[oy]);
            v.x += w.x;
            v.y += w.y;
        }
        y[oy] = v;
    }
}

__global__ void k_fill(ShapeStrides ss, int64_t n, cplx v, cplx* __restrict__ y) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = idx, oy = 0;
        for (int k = ss.nd - 1; k >= 0; --k) {
            int64_t c = r % ss.d[k];
            r /= ss.d[k];
            oy += c * ss.sy[k];
        }
        y[oy] = v;
    }
}

// contiguous fast path
template <bool BETA0>
__global__ void k_axpby_contig(int64_t n, cplx alpha, const cplx* __restrict__ x, int conjx, cplx beta,
                               cplx* __restrict__ y) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        cplx v = x[idx];
        if (conjx) v.y = -v.y;
        v = cmul(alpha, v);
        if (!BETA0) {
            cplx w = cmul(beta, y[idx]);
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
    return ss;
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
        if (beta0) k_axpby_contig<true><<<g, th, 0, D.st>>>(n, alpha, x.p, conjx, beta, y.p);
        else k_axpby_contig<false><<<g, th, 0, D.st>>>(n, alpha, x.p, conjx, beta, y.p);
    } else {
        if (beta0) k_axpby<true><<<g, th, 0, D.st>>>(ss, n, alpha, x.p, conjx, beta, y.p);
        else k_axpby<false><<<g, th, 0, D.st>>>(ss, n, alpha, x.p, conjx, beta, y.p);
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
        int64_t r = row * per_row + idx, oy = 0;
        for (int k = ss.nd - 1; k >= 0; --k) {
            int64_t c = r % ss.d[k];
            r /= ss.d[k];
            oy += c * ss.sy[k];
        }
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
