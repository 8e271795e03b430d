// FP64 complex GEMM on the CUDA cores (the plain-FP64 path and the FP64
// outer residual of the mixed path).  Operands are arbitrary-stride views, so
// most contractions of the residual need no transposition copy.
//
// Tiling: 64x64 output tile per 256-thread CTA, 4x4 complex accumulators per
// thread, K step 8 complex, register-prefetched double-buffered shared tiles.
// Split-K over grid.z with FP64 atomics when the tile grid is too small for
// the 152 SMs.
#include "lrcc_internal.h"

#include <algorithm>

namespace {

constexpr int BM = 64, BN = 64, BK = 8, TH = 256;

__device__ __forceinline__ void cfma(cplx& c, cplx a, cplx b) {
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
}
__device__ __forceinline__ void cfma(float2& c, float2 a, float2 b) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
}

// compute-type traits: FP64 (the FP64 path) or FP32 (the inner products of
// the mixed path, for contractions too small or too thin for the tensor cores)
template <typename T> struct CT;
template <> struct CT<double> {
    typedef cplx C;
    __device__ static C cvt(cplx v) { return v; }
    __device__ static cplx back(C v) { return v; }
    __device__ static C zero() { return make_double2(0.0, 0.0); }
    __device__ static cplx scale(C v, cplx a) { return make_double2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x); }
};
template <> struct CT<float> {
    typedef float2 C;
    __device__ static C cvt(cplx v) { return make_float2((float)v.x, (float)v.y); }
    __device__ static cplx back(C v) { return make_double2(f32_to_f64(v.x), f32_to_f64(v.y)); }
    __device__ static C zero() { return make_float2(0.f, 0.f); }
    // alpha applied in FP32: the FP64 pipe (2 FMA per SM per clock on GB300)
    // is left to the adds into C
    __device__ static cplx scale(C v, cplx a) {
        const float ax = (float)a.x, ay = (float)a.y;
        return make_double2(f32_to_f64(ax * v.x - ay * v.y), f32_to_f64(ax * v.y + ay * v.x));
    }
};

struct GemmK {
    int64_t M, N, K;
    const cplx* A;
    int64_t sAb, sAm, sAk;
    int cA;
    const cplx* B;
    int64_t sBb, sBk, sBn;
    int cB;
    cplx* C;
    int64_t sCb, sCm, sCn;
    cplx alpha, beta;
    int64_t kper;  // K range per split
    int atomic;    // 1: accumulate alpha*acc with atomics (C pre-scaled by beta)
    int a_kfast, b_nfast;
    Lvl am, ak, bk, bn, cm, cn;  // index group offsets (two-level groups of an einsum in place)
};

template <typename T>
__global__ void __launch_bounds__(TH) k_gemm(GemmK g) {
    typedef typename CT<T>::C cT;
    __shared__ cT As[2][BK][BM];
    __shared__ cT Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t tiles_n = (g.N + BN - 1) / BN;
    const int64_t m0 = (blockIdx.x / tiles_n) * BM;
    const int64_t n0 = (blockIdx.x % tiles_n) * BN;
    const int64_t b = blockIdx.y;
    const int64_t kbeg = blockIdx.z * g.kper;
    const int64_t kend = min(g.K, kbeg + g.kper);
    const cplx* A = g.A + b * g.sAb;
    const cplx* B = g.B + b * g.sBb;

    cT acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = CT<T>::zero();

    cT ra[2], rb[2];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int e = tid + r * TH;  // 0..511
            int mm, kk;
            if (g.a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
            int64_t m = m0 + mm, k = k0 + kk;
            cplx v = make_double2(0.0, 0.0);
            if (m < g.M && k < kend) v = A[lvl_off(g.am, m) + lvl_off(g.ak, k)];
            if (g.cA) v.y = -v.y;
            ra[r] = CT<T>::cvt(v);
            int nn;
            if (g.b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
            int64_t n = n0 + nn;
            k = k0 + kk;
            cplx w = make_double2(0.0, 0.0);
            if (n < g.N && k < kend) w = B[lvl_off(g.bk, k) + lvl_off(g.bn, n)];
            if (g.cB) w.y = -w.y;
            rb[r] = CT<T>::cvt(w);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int e = tid + r * TH;
            int mm, kk, nn;
            if (g.a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
            As[buf][kk][mm] = ra[r];
            if (g.b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
            Bs[buf][kk][nn] = rb[r];
        }
    };

    int buf = 0;
    if (kbeg < kend) {
        load(kbeg);
        store(0);
    }
    __syncthreads();
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
        bool more = k0 + BK < kend;
        if (more) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            cT a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], bb[j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }

    cplx* C = g.C + b * g.sCb;
    // old C values first (all loads in flight together), then the stores
    const bool rd = !g.atomic && (g.beta.x != 0.0 || g.beta.y != 0.0);
    const bool beta1 = rd && g.beta.x == 1.0 && g.beta.y == 0.0;
    cplx old[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            old[i][j] = (rd && m < g.M && n < g.N) ? C[lvl_off(g.cm, m) + lvl_off(g.cn, n)] : make_double2(0.0, 0.0);
        }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            cplx r = CT<T>::scale(acc[i][j], g.alpha);
            cplx* c = C + lvl_off(g.cm, m) + lvl_off(g.cn, n);
            if (g.atomic) {
                atomicAdd(&c->x, r.x);
                atomicAdd(&c->y, r.y);
            } else {
                const cplx o = old[i][j];
                if (beta1) {
                    r.x += o.x;
                    r.y += o.y;
                } else if (rd) {
                    r.x += g.beta.x * o.x - g.beta.y * o.y;
                    r.y += g.beta.x * o.y + g.beta.y * o.x;
                }
                *c = r;
            }
        }
    }
}

// Skinny GEMM (N <= NMAX): one thread per output row m keeps all N complex
// accumulators in registers; B is staged K-chunk by K-chunk in shared memory.
// Used for the O-sized index contractions (N or M = O), where 64x64 tiles
// would waste most of the FMA work.
constexpr int SK_KC = 32, SK_TH = 128;

template <int NMAX, typename T>
__global__ void __launch_bounds__(SK_TH) k_gemm_skinny(GemmK g) {
    typedef typename CT<T>::C cT;
    __shared__ cT Bs[SK_KC][NMAX];
    const int64_t m = blockIdx.x * (int64_t)SK_TH + threadIdx.x;
    const int64_t b = blockIdx.y;
    const cplx* A = g.A + b * g.sAb;
    const cplx* B = g.B + b * g.sBb;
    const int N = (int)g.N;
    const int64_t kbeg = blockIdx.z * g.kper, kend = min(g.K, kbeg + g.kper);
    cT acc[NMAX];
#pragma unroll
    for (int n = 0; n < NMAX; ++n) acc[n] = CT<T>::zero();
    for (int64_t k0 = kbeg; k0 < kend; k0 += SK_KC) {
        int kc = (int)min((int64_t)SK_KC, kend - k0);
        for (int e = threadIdx.x; e < SK_KC * NMAX; e += SK_TH) {
            int kk = g.b_nfast ? e / NMAX : e % SK_KC;
            int nn = g.b_nfast ? e % NMAX : e / SK_KC;
            cplx w = make_double2(0.0, 0.0);
            if (kk < kc && nn < N) w = B[lvl_off(g.bk, k0 + kk) + lvl_off(g.bn, nn)];
            if (g.cB) w.y = -w.y;
            Bs[kk][nn] = CT<T>::cvt(w);
        }
        __syncthreads();
        if (m < g.M) {
            for (int kk = 0; kk < kc; ++kk) {
                cplx a0 = A[lvl_off(g.am, m) + lvl_off(g.ak, k0 + kk)];
                if (g.cA) a0.y = -a0.y;
                cT a = CT<T>::cvt(a0);
#pragma unroll
                for (int n = 0; n < NMAX; ++n) cfma(acc[n], a, Bs[kk][n]);
            }
        }
        __syncthreads();
    }
    if (m >= g.M) return;
    cplx* C = g.C + b * g.sCb;
    const bool rd = !g.atomic && (g.beta.x != 0.0 || g.beta.y != 0.0);
    const bool beta1 = rd && g.beta.x == 1.0 && g.beta.y == 0.0;
    cplx old[NMAX];
#pragma unroll
    for (int n = 0; n < NMAX; ++n)
        old[n] = (rd && n < N) ? C[lvl_off(g.cm, m) + lvl_off(g.cn, n)] : make_double2(0.0, 0.0);
#pragma unroll
    for (int n = 0; n < NMAX; ++n) {
        if (n >= N) break;
        cplx r = CT<T>::scale(acc[n], g.alpha);
        cplx* c = C + lvl_off(g.cm, m) + lvl_off(g.cn, n);
        if (g.atomic) {
            atomicAdd(&c->x, r.x);
            atomicAdd(&c->y, r.y);
            continue;
        }
        const cplx o = old[n];
        if (beta1) {
            r.x += o.x;
            r.y += o.y;
        } else if (rd) {
            r.x += g.beta.x * o.x - g.beta.y * o.y;
            r.y += g.beta.x * o.y + g.beta.y * o.x;
        }
        *c = r;
    }
}

// C[b] += alpha * sum_k A[b][k] B[b][k]   (M = N = 1), C pre-scaled by beta
__global__ void k_dot(int64_t K, const cplx* A, int64_t sAb, int64_t sAk, int cA, const cplx* B,
                      int64_t sBb, int64_t sBk, int cB, cplx* C, int64_t sCb, cplx alpha) {
    __shared__ double rx[32], ry[32];
    int64_t b = blockIdx.y;
    const cplx* a = A + b * sAb;
    const cplx* bb = B + b * sBb;
    double sx = 0, sy = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        cplx u = a[k * sAk], v = bb[k * sBk];
        if (cA) u.y = -u.y;
        if (cB) v.y = -v.y;
        sx = fma(u.x, v.x, sx);
        sx = fma(-u.y, v.y, sx);
        sy = fma(u.x, v.y, sy);
        sy = fma(u.y, v.x, sy);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffff, sx, o);
        sy += __shfl_xor_sync(0xffffffff, sy, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rx[threadIdx.x >> 5] = sx;
        ry[threadIdx.x >> 5] = sy;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        sx = threadIdx.x < nw ? rx[threadIdx.x] : 0.0;
        sy = threadIdx.x < nw ? ry[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffff, sx, o);
            sy += __shfl_xor_sync(0xffffffff, sy, o);
        }
        if (threadIdx.x == 0) {
            cplx* c = C + b * sCb;
            atomicAdd(&c->x, alpha.x * sx - alpha.y * sy);
            atomicAdd(&c->y, alpha.x * sy + alpha.y * sx);
        }
    }
}

// C[b][m][n] *= beta (strided; m and n may be two-level: g = g1 d2 + g2 at
// offset g1 s1 + g2 s), beta == 0 -> zero
__global__ void k_scale(int64_t M, int64_t N, int64_t batch, cplx* C, int64_t sCb, int64_t sCm, int64_t sCn,
                        int64_t dm2, int64_t sm1, int64_t dn2, int64_t sn1, cplx beta) {
    int64_t total = M * N * batch;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = i % N, r = i / N, m = r % M, b = r / M;
        const int64_t mo = dm2 ? (m / dm2) * sm1 + (m % dm2) * sCm : m * sCm;
        const int64_t no = dn2 ? (n / dn2) * sn1 + (n % dn2) * sCn : n * sCn;
        cplx* c = C + b * sCb + mo + no;
        if (beta.x == 0.0 && beta.y == 0.0) {
            *c = make_double2(0.0, 0.0);
        } else {
            cplx o = *c;
            *c = make_double2(beta.x * o.x - beta.y * o.y, beta.x * o.y + beta.y * o.x);
        }
    }
}

}  // namespace

void gemm_prescale(Dev& D, const GemmArgs& g);
static void prescale(Dev& D, const GemmArgs& g) { gemm_prescale(D, g); }

void gemm_prescale(Dev& D, const GemmArgs& g) {
    if (g.beta.x == 1.0 && g.beta.y == 0.0) return;
    int64_t total = g.M * g.N * g.batch;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, D.sm_count * 16));
    k_scale<<<grid, 256, 0, D.st>>>(g.M, g.N, g.batch, g.C, g.sCb, g.sCm, g.sCn, g.dCm2, g.sCm1, g.dCn2, g.sCn1,
                                    g.beta);
    LAUNCH_CHECK(D);
}

template <typename T>
static void gemm_simt(Dev& D, const GemmArgs& g);

void gemm_f64(Dev& D, const GemmArgs& g) { gemm_simt<double>(D, g); }
void gemm_f32c(Dev& D, const GemmArgs& g) { gemm_simt<float>(D, g); }

template <typename T>
static void gemm_simt(Dev& D, const GemmArgs& g) {
    REQUIRE(g.flat() || (std::max(g.M, g.N) < FAST_INDEX_LIMIT && g.K < FAST_INDEX_LIMIT),
            "SIMT GEMM: two-level index groups need groups below 2^31");
    const char* kname = sizeof(T) == 8 ? "gemm_f64" : "gemm_f32";
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
    if (g.K <= 0) {
        prescale(D, g);
        return;
    }
    if (g.batch > 65535) throw LrccError(LRCC_EINVAL, "gemm batch > 65535");
    if (g.M == 1 && g.N == 1 && g.flat()) {
        prescale(D, g);
        int th = 256;
        int64_t want = (g.K + th * 8 - 1) / (th * 8);
        int gx = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::max<int64_t>(1, 4 * D.sm_count / g.batch)));
        dim3 grid(gx, (unsigned)g.batch);
        k_dot<<<grid, th, 0, D.st>>>(g.K, g.A, g.sAb, g.sAk, g.cA, g.B, g.sBb, g.sBk, g.cB, g.C, g.sCb, g.alpha);
        LAUNCH_CHECK(D);
        return;
    }
    // skinny shapes: one of M, N at most 32 (swap roles so that N is the small one)
    if (std::min(g.M, g.N) <= 32) {
        GemmK k{};
        bool swap = g.M < g.N;
        k.M = swap ? g.N : g.M;
        k.N = swap ? g.M : g.N;
        k.K = g.K;
        if (!swap) {
            k.A = g.A; k.sAb = g.sAb; k.sAm = g.sAm; k.sAk = g.sAk; k.cA = g.cA;
            k.B = g.B; k.sBb = g.sBb; k.sBk = g.sBk; k.sBn = g.sBn; k.cB = g.cB;
            k.C = g.C; k.sCb = g.sCb; k.sCm = g.sCm; k.sCn = g.sCn;
            k.am = mk_lvl(g.sAm, g.dAm2, g.sAm1); k.ak = mk_lvl(g.sAk, g.dAk2, g.sAk1);
            k.bk = mk_lvl(g.sBk, g.dBk2, g.sBk1); k.bn = mk_lvl(g.sBn, g.dBn2, g.sBn1);
            k.cm = mk_lvl(g.sCm, g.dCm2, g.sCm1); k.cn = mk_lvl(g.sCn, g.dCn2, g.sCn1);
        } else {  // C^T = B^T A^T
            k.A = g.B; k.sAb = g.sBb; k.sAm = g.sBn; k.sAk = g.sBk; k.cA = g.cB;
            k.B = g.A; k.sBb = g.sAb; k.sBk = g.sAk; k.sBn = g.sAm; k.cB = g.cA;
            k.C = g.C; k.sCb = g.sCb; k.sCm = g.sCn; k.sCn = g.sCm;
            k.am = mk_lvl(g.sBn, g.dBn2, g.sBn1); k.ak = mk_lvl(g.sBk, g.dBk2, g.sBk1);
            k.bk = mk_lvl(g.sAk, g.dAk2, g.sAk1); k.bn = mk_lvl(g.sAm, g.dAm2, g.sAm1);
            k.cm = mk_lvl(g.sCn, g.dCn2, g.sCn1); k.cn = mk_lvl(g.sCm, g.dCm2, g.sCm1);
        }
        k.alpha = g.alpha;
        k.beta = g.beta;
        k.b_nfast = (k.sBn == 1) || (k.sBk != 1 && std::llabs(k.sBn) < std::llabs(k.sBk));
        // split K until there are about 4 CTAs per SM: FP64 on this part is
        // ~8 GFLOP/s per SM, so work left on a few SMs dominates everything
        int64_t blocks = ((k.M + SK_TH - 1) / SK_TH) * g.batch;
        int64_t sp = std::max<int64_t>(1, std::min<int64_t>((4 * (int64_t)D.sm_count + blocks - 1) / blocks,
                                                            (g.K + 7) / 8));
        sp = std::min<int64_t>(sp, 1024);
        k.kper = (g.K + sp - 1) / sp;
        k.kper = (k.kper + 7) / 8 * 8;
        sp = (g.K + k.kper - 1) / k.kper;
        k.atomic = sp > 1;
        if (k.atomic) prescale(D, g);
        dim3 grid((unsigned)((k.M + SK_TH - 1) / SK_TH), (unsigned)g.batch, (unsigned)sp);
        KTimer kt(D, kname, 8.0 * g.M * g.N * g.K * g.batch, 16.0 * (g.M * g.K + g.K * g.N + g.M * g.N) * g.batch,
                  g.M, g.N, g.K, g.batch);
        if (k.N <= 1) k_gemm_skinny<1, T><<<grid, SK_TH, 0, D.st>>>(k);
        else if (k.N <= 2) k_gemm_skinny<2, T><<<grid, SK_TH, 0, D.st>>>(k);
        else if (k.N <= 4) k_gemm_skinny<4, T><<<grid, SK_TH, 0, D.st>>>(k);
        else if (k.N <= 8) k_gemm_skinny<8, T><<<grid, SK_TH, 0, D.st>>>(k);
        else if (k.N <= 12) k_gemm_skinny<12, T><<<grid, SK_TH, 0, D.st>>>(k);
        else if (k.N <= 16) k_gemm_skinny<16, T><<<grid, SK_TH, 0, D.st>>>(k);
        else if (k.N <= 24) k_gemm_skinny<24, T><<<grid, SK_TH, 0, D.st>>>(k);
        else k_gemm_skinny<32, T><<<grid, SK_TH, 0, D.st>>>(k);
        LAUNCH_CHECK(D);
        return;
    }
    int64_t tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    if (tiles > INT32_MAX) throw LrccError(LRCC_EINVAL, "gemm too large");
    int64_t ctas = tiles * g.batch;
    int64_t splits = 1;
    int64_t target = 2 * (int64_t)D.sm_count;
    if (ctas < target && g.K >= 2 * BK) {
        splits = std::min<int64_t>((target + ctas - 1) / ctas, g.K / BK);
        splits = std::max<int64_t>(1, std::min<int64_t>(splits, 512));
    }
    GemmK k;
    k.M = g.M; k.N = g.N; k.K = g.K;
    k.A = g.A; k.sAb = g.sAb; k.sAm = g.sAm; k.sAk = g.sAk; k.cA = g.cA;
    k.B = g.B; k.sBb = g.sBb; k.sBk = g.sBk; k.sBn = g.sBn; k.cB = g.cB;
    k.C = g.C; k.sCb = g.sCb; k.sCm = g.sCm; k.sCn = g.sCn;
    k.am = mk_lvl(g.sAm, g.dAm2, g.sAm1); k.ak = mk_lvl(g.sAk, g.dAk2, g.sAk1);
    k.bk = mk_lvl(g.sBk, g.dBk2, g.sBk1); k.bn = mk_lvl(g.sBn, g.dBn2, g.sBn1);
    k.cm = mk_lvl(g.sCm, g.dCm2, g.sCm1); k.cn = mk_lvl(g.sCn, g.dCn2, g.sCn1);
    k.alpha = g.alpha; k.beta = g.beta;
    k.kper = (g.K + splits - 1) / splits;
    k.kper = (k.kper + BK - 1) / BK * BK;
    splits = (g.K + k.kper - 1) / k.kper;
    k.atomic = splits > 1;
    k.a_kfast = (g.sAk == 1) || (g.sAm != 1 && std::llabs(g.sAk) < std::llabs(g.sAm));
    k.b_nfast = (g.sBn == 1) || (g.sBk != 1 && std::llabs(g.sBn) < std::llabs(g.sBk));
    if (k.atomic) prescale(D, g);
    dim3 grid((unsigned)tiles, (unsigned)g.batch, (unsigned)splits);
    KTimer kt(D, kname, 8.0 * g.M * g.N * g.K * g.batch, 16.0 * (g.M * g.K + g.K * g.N + g.M * g.N) * g.batch,
              g.M, g.N, g.K, g.batch);
    k_gemm<T><<<grid, TH, 0, D.st>>>(k);
    LAUNCH_CHECK(D);
}
