// Internal interfaces of the LR-CCSD library: device tensors, the caching
// pool, the kernel launchers and the contraction engine.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/lrcc.h"

typedef double2 cplx;

static inline cplx mkc(double re, double im = 0.0) { return make_double2(re, im); }

struct LrccError : std::runtime_error {
    lrcc_status st;
    LrccError(lrcc_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define CK(x)                                                                              \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess)                                                             \
            throw LrccError(e_ == cudaErrorMemoryAllocation ? LRCC_ENOMEM : LRCC_ECUDA,    \
                            std::string(#x) + ": " + cudaGetErrorString(e_));              \
    } while (0)

#define REQUIRE(cond, msg)                                         \
    do {                                                           \
        if (!(cond)) throw LrccError(LRCC_EINVAL, std::string(msg)); \
    } while (0)

#define LAUNCH_CHECK(D)                                 \
    do {                                                \
        (D).launches++;                                 \
        cudaError_t e_ = cudaGetLastError();            \
        if (e_ != cudaSuccess)                          \
            throw LrccError(LRCC_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------
// caching device allocator (stream-ordered reuse on the context's one stream)
// ---------------------------------------------------------------------------
struct Pool {
    std::multimap<size_t, void*> cache;
    size_t live = 0, cached = 0, peak = 0, largest = 0;  // bytes; largest single request
    void* get(size_t n);
    void put(void* p, size_t n);
    void trim();
    ~Pool();
};

struct DevBuf {
    Pool* pool;
    void* p;
    size_t n;
    ~DevBuf() { pool->put(p, n); }
};

// per-launch CUDA-event records (enabled for measurement only)
struct KRec {
    const char* name;
    cudaEvent_t a, b;
    double flops, bytes;
    int64_t m = 0, n = 0, k = 0, batch = 0;  // GEMM shape (0 for other kernels)
};

struct Dev {
    cudaStream_t st = nullptr;
    Pool pool;
    int64_t launches = 0;
    int* err_flag = nullptr;  // device word set by kernels whose bounded waits expire
    int sm_count = 148;
    double embed_budget = 0;  // bytes for one GEMM's embedded operands (0: automatic)
    bool timing = false;
    std::vector<KRec> recs;
};

// RAII event pair around one launch on D.st when D.timing is set
struct KTimer {
    Dev& D;
    KRec r;
    bool on;
    KTimer(Dev& d, const char* name, double flops, double bytes, int64_t m = 0, int64_t n = 0, int64_t k = 0,
           int64_t batch = 0)
        : D(d), on(d.timing) {
        if (!on) return;
        r.name = name;
        r.flops = flops;
        r.bytes = bytes;
        r.m = m;
        r.n = n;
        r.k = k;
        r.batch = batch;
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
        cudaEventRecord(r.a, D.st);
    }
    ~KTimer() {
        if (!on) return;
        cudaEventRecord(r.b, D.st);
        D.recs.push_back(r);
    }
};

// ---------------------------------------------------------------------------
// n / d and n % d for 0 <= n < 2^31 with one multiply-high (the round-up
// method of Granlund and Montgomery, PLDI 1994): s = ceil(log2 d),
// m = floor(2^32 (2^s - d) / d) + 1, n / d = (mulhi(n, m) + n) >> s.
// Index decoding in the elementwise kernels uses it instead of 64-bit division.
// ---------------------------------------------------------------------------
struct FastDiv {
    uint32_t d = 1, m = 1, s = 0;
    FastDiv() = default;
    explicit FastDiv(int64_t div) {
        d = (uint32_t)(div < 1 ? 1 : div);
        s = 0;
        while ((uint64_t(1) << s) < d) ++s;
        m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << s) - d)) / d + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> s; }
};
// FP64 -> FP32 by truncating the significand, from the IEEE-754 bit fields with
// integer operations only (GB300 issues two FP64 instructions per SM per clock,
// which made FP64-side conversions the bottleneck of these memory-bound
// kernels).  Magnitudes below the FP32 normal range flush to zero; overflow
// gives infinity; NaN stays NaN.  The dropped bits are below 2^-23 relative,
// far under the 2^-17 of the bf16x3 split and the 2^-11 of TF32.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0x7FF)
        return __uint_as_float(sign | 0x7F800000u | ((b & 0xFFFFFFFFFFFFFull) ? 0x400000u : 0u));
    const int ef = ex - 1023 + 127;
    if (ef <= 0) return __uint_as_float(sign);
    if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((uint32_t)ef << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
}

// store the embedding of v = op(S)[b][r][k]: A rows (slots S*k..) or the B row
// pair (2r: real output, 2r+1: imaginary output)
// FP32 -> FP64 (exact) from the bit fields with integer operations, keeping
// conversions off the FP64 pipe; FP32 subnormals (below 1.2e-38) become zero
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if (ex == 0) return __longlong_as_double((long long)sign);
    if (ex == 0xFFu)
        return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | ((u & 0x7FFFFFu) ? (1ull << 51) : 0ull)));
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(ex - 127 + 1023) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// elementwise index spaces below 2^31 decode with FastDiv
constexpr int64_t FAST_INDEX_LIMIT = int64_t(1) << 31;

// Offset of index g of a GEMM index group: g * s (flat), or with two levels
// g = g1 d2 + g2 at g1 s1 + g2 s (an einsum group whose labels are not
// adjacent in memory; d2 < 2^31).
struct Lvl {
    int64_t s = 0, s1 = 0;
    FastDiv f2;
    int two = 0;
};
__device__ __forceinline__ int64_t lvl_off(const Lvl& L, int64_t g) {
    if (!L.two) return g * L.s;
    const uint32_t q = L.f2.div((uint32_t)g);
    return (int64_t)q * L.s1 + (int64_t)((uint32_t)g - q * L.f2.d) * L.s;
}
inline Lvl mk_lvl(int64_t s, int64_t d2 = 0, int64_t s1 = 0) {
    Lvl L;
    L.s = s;
    if (d2 > 0) {
        L.two = 1;
        L.s1 = s1;
        L.f2 = FastDiv(d2);
    }
    return L;
}

// ---------------------------------------------------------------------------
// strided complex tensor (row-major by default), up to 8 dimensions
// ---------------------------------------------------------------------------
constexpr int MAXD = 8;

struct Tensor {
    std::shared_ptr<DevBuf> buf;
    cplx* p = nullptr;
    int nd = 0;
    int64_t d[MAXD] = {0};
    int64_t s[MAXD] = {0};

    int64_t numel() const {
        int64_t n = 1;
        for (int i = 0; i < nd; ++i) n *= d[i];
        return n;
    }
    bool contiguous() const {
        int64_t st = 1;
        for (int i = nd - 1; i >= 0; --i) {
            if (d[i] != 1 && s[i] != st) return false;
            st *= d[i];
        }
        return true;
    }
    bool defined() const { return p != nullptr || numel() == 0; }
    Tensor slice(int dim, int64_t start, int64_t len) const {
        Tensor t = *this;
        t.p = p + start * s[dim];
        t.d[dim] = len;
        return t;
    }
    Tensor index(int64_t i) const {  // drop leading dim
        Tensor t;
        t.buf = buf;
        t.p = p + i * s[0];
        t.nd = nd - 1;
        for (int k = 1; k < nd; ++k) { t.d[k - 1] = d[k]; t.s[k - 1] = s[k]; }
        return t;
    }
    // reinterpret a contiguous tensor with a new shape
    Tensor reshape(std::vector<int64_t> shape) const;
    // permuted view: new dim k = old dim perm[k]
    Tensor permute(const std::vector<int>& perm) const;
    std::vector<int64_t> shape() const { return std::vector<int64_t>(d, d + nd); }
};

Tensor empty(Dev& D, std::vector<int64_t> shape);
Tensor zeros(Dev& D, std::vector<int64_t> shape);
// wrap external device memory (not owned)
Tensor wrap(cplx* p, std::vector<int64_t> shape);

// ---------------------------------------------------------------------------
// elementwise kernels (kernels_elem.cu)
// ---------------------------------------------------------------------------
// y = alpha * op(x) + beta * y over identical shapes; beta == 0 overwrites.
void axpby(Dev& D, cplx alpha, const Tensor& x, bool conjx, cplx beta, Tensor& y);
void fill(Dev& D, Tensor& y, cplx v);
// C = alpha op(A) op(B) + beta C elementwise; A and B are views over C's dims
// (stride 0 along dims they do not carry)
void outer_axpby(Dev& D, cplx alpha, const Tensor& A, bool ca, const Tensor& B, bool cb, cplx beta, Tensor& C,
                 bool lowp = false);
// y = alpha P x + beta y on contiguous [..][O][O][V][V]; P = P(ij) (mode 1),
// P(ab) (mode 2) or P(ij)P(ab) (mode 3)
void asym_axpby(Dev& D, int mode, cplx alpha, const Tensor& x, cplx beta, Tensor& y);
// max |y| over all elements (host result; synchronises the stream)
double max_abs(Dev& D, const Tensor& y);
// per-leading-index max |y| into dev out[R] (double), no sync
void max_abs_rows(Dev& D, const Tensor& y, double* out_dev);

// ---------------------------------------------------------------------------
// FP64 complex GEMM (gemm_f64.cu):  C[b][m][n] = alpha sum_k op(A)[b][m][k] op(B)[b][k][n] + beta C
// ---------------------------------------------------------------------------
struct GemmArgs {
    int64_t M, N, K, batch;
    const cplx* A;
    int64_t sAb, sAm, sAk;
    bool cA;
    const cplx* B;
    int64_t sBb, sBk, sBn;
    bool cB;
    cplx* C;
    int64_t sCb, sCm, sCn;
    cplx alpha, beta;
    // two-level index groups (tensor-core path only): index g of a group is
    // split as g = g1 d2 + g2 with offset g1 s1 + g2 s, s being the stride
    // above; d2 = 0 marks a flat group
    int64_t dAm2 = 0, sAm1 = 0, dAk2 = 0, sAk1 = 0;
    int64_t dBk2 = 0, sBk1 = 0, dBn2 = 0, sBn1 = 0;
    int64_t dCm2 = 0, sCm1 = 0, dCn2 = 0, sCn1 = 0;
    bool flat() const { return !(dAm2 | dAk2 | dBk2 | dBn2 | dCm2 | dCn2); }
};
void gemm_f64(Dev& D, const GemmArgs& g);
// same GEMM with FP32 arithmetic (FP64 in and out): inner products of the
// mixed path that are too thin or too short in K for the tensor cores
void gemm_f32c(Dev& D, const GemmArgs& g);
// C *= beta on the GEMM's output view (before split-K accumulation)
void gemm_prescale(Dev& D, const GemmArgs& g);

// tensor-core split-precision GEMM (gemm_tc.cu); prec = LRCC_MIXED_*
bool gemm_tc_available();
void gemm_tc(Dev& D, const GemmArgs& g, int prec);
// pieces: embedded-operand layout [batch][rows_e][pitch] (rows_e = rows for
// A, 2 rows for B; pitch = S K rounded up to 16 bytes; nothing outside S K
// columns is written or read), the split/convert kernels, and the GEMM on
// already embedded operands (complex K)
size_t tc_embed_bytes(int prec, int64_t rows, int64_t K, int64_t batch, int64_t& rows_e, int64_t& pitch, bool is_b);
// (rows_tot: embedded rows of the whole destination buffer, whose K panels are
// that many rows apart; out may point at a row inside it)
void tc_embed_a(Dev& D, int prec, const cplx* A, int64_t sAb, int64_t sAm, int64_t sAk, bool cA, int64_t batch,
                int64_t M, int64_t K, int64_t pitch, int64_t rows_tot, void* out);
void tc_embed_b(Dev& D, int prec, const cplx* B, int64_t sBb, int64_t sBk, int64_t sBn, bool cB, int64_t batch,
                int64_t K, int64_t N, int64_t pitch, int64_t rows_tot, void* out);
// zeros beyond the used K in the last panel of rows [0, nrows) at out (buffers
// filled by tc_embed_antisym_slab)
void tc_zero_tail(Dev& D, int prec, void* out, int64_t rows_tot, int64_t K, int64_t nrows);
// FP64-class complex GEMM on bf16 tensor cores (integer slices with per-row
// exponents, exact FP32 chains, FP64 sums): gemm_tc_f64 is the whole GEMM;
// the pieces embed operands as [batch][rows_e][7 kpad] bf16 and run the
// diagonals on them
void gemm_tc_f64(Dev& D, const GemmArgs& g);
size_t oz_embed_bytes(int64_t rows, int64_t K, int64_t batch, int64_t& rows_e, int64_t& kpad, bool is_b);
void oz_embed_a(Dev& D, const cplx* A, int64_t sAb, int64_t sAm, int64_t sAk, bool cA, int64_t batch, int64_t M,
                int64_t K, int64_t kpad, void* out);
void oz_embed_b(Dev& D, const cplx* B, int64_t sBb, int64_t sBk, int64_t sBn, bool cB, int64_t batch, int64_t K,
                int64_t N, int64_t kpad, void* out);
void oz_gemm_embedded(Dev& D, const void* pa, const void* pb, int64_t batch, int64_t M, int64_t N, int64_t K,
                      int64_t kpad, cplx* C, int64_t sCb, int64_t sCm, int64_t sCn, cplx alpha, cplx beta,
                      bool conj_acc);
void tc_gemm_embedded(Dev& D, int prec, const void* pa, const void* pb, int64_t batch, int64_t M, int64_t N,
                      int64_t K, int64_t pitch, int64_t rows_a, int64_t rows_b, cplx* C, int64_t sCb, int64_t sCm,
                      int64_t sCn, cplx alpha, cplx beta, bool conj_acc, double useful_flops);
// the same on the complex K range [k0, K_total) of operands embedded with K_total
// (batch 1; k0 a multiple of tc_k_align(prec)), optionally skipping tiles: with
// mask_v > 0 a tile runs only if one of its rows and one of its complex
// columns have (index mod mask_v) >= mask_emin
void tc_gemm_embedded_ex(Dev& D, int prec, const void* pa, const void* pb, int64_t M, int64_t N, int64_t K_total,
                         int64_t k0, int64_t pitch, int64_t rows_a, int64_t rows_b, cplx* C, int64_t sCm,
                         int64_t sCn, cplx alpha, cplx beta, bool conj_acc, double useful_flops, int mask_v,
                         int mask_emin, bool f32out = false);
int64_t tc_k_align(int prec);

// ---------------------------------------------------------------------------
// contraction engine (engine.cu)
// ---------------------------------------------------------------------------
// einsum "ab,bc->ac"-style, single-letter labels, every label in >= 2 operands
// prec: LRCC_FP64 or a mixed mode (large GEMMs go to the tensor cores)
void ein(Dev& D, const std::string& spec, cplx alpha, const Tensor& A, bool cA, const Tensor& B,
         bool cB, cplx beta, Tensor& C, int prec = LRCC_FP64);
// allocate C from the spec and operands, then C = alpha * A.B
Tensor ein_new(Dev& D, const std::string& spec, cplx alpha, const Tensor& A, bool cA, const Tensor& B,
               bool cB, int prec = LRCC_FP64);
// permuted axpby by labels: y(spec rhs) = alpha * x(spec lhs) + beta * y
void perm_axpby(Dev& D, const std::string& spec, cplx alpha, const Tensor& x, cplx beta, Tensor& y);

// particle-particle ladder Z = 1/2 sum_ef <ab||ef> X_ij^ef (X, Z: [R][O][O][V][V]),
// <ab|ef> = sum_L Bvv^L_ae Bvv^L_bf; transpose -> Bvv conjugated.
struct LadderCtx {
    Tensor Bvv;      // [L][V][V]
    Tensor Bov;      // [L][O][V] (B^L_me): the occupied-virtual factor of the Q map
    // assembled <am||ef> rows W [V*O][P_V] (FP64 or FP64-class products), cached
    // when they fit in a sixth of free memory; otherwise assembled per call
    Tensor wq64;
    int wq64_prec = -1;
    bool wq64_disabled = false;
    int slab_rows = 0;  // > 0: no <ab||ef> cache; assemble per call in slabs of this many rows
    int hermitian = 0;  // per-call assembly: 1 Hermitian half, -1 whole rows, 0 automatic
    // cached embedded <ab||ef> matrix W' [P_V][pitch] (rows a<b, K = pairs e<f)
    // for one mixed precision, built on first use when it fits in device memory
    std::shared_ptr<DevBuf> wcache;
    int wcache_prec = -1;
    int64_t w_pitch = 0;
    bool wcache_disabled = false;
    // embedded Bvv as the B operand (n = (b,f), k = L) of the slab assembly
    std::shared_ptr<DevBuf> bcache;
    int bcache_prec = -1;
    int64_t b_pitch = 0, b_rows = 0;
    // cached FP64 <ab||ef> matrix [P_V][P_V] for the FP64 ladder, when it fits,
    // built with FP64 (LRCC_FP64) or FP64-class (LRCC_FP64_EMULATED) products
    Tensor w64;
    int w64_prec = -1;
    bool w64_disabled = false;
    // that matrix sliced for the FP64-class products
    std::shared_ptr<DevBuf> ozcache;
    int64_t oz_kpad = 0;
    bool ozcache_disabled = false;
};
void ladder(Dev& D, LadderCtx& L, const Tensor& X, cplx alpha, cplx beta, Tensor& Z, bool transpose, int prec);
// packed form: Zt[n][ab] = sum_{e<f} <ab||ef> Xt[n][ef] (transpose: conj <ab||ef>),
// Xt, Zt [ncol][P_V] (pair order a<b row-major), Zt overwritten
void ladder_packed(Dev& D, LadderCtx& L, const cplx* Xt, cplx* Zt, int64_t ncol, bool transpose, int prec);
// embedded <ab||ef> rows of one slab from GT[(b,f)][(a,e)] (leading dimension ldt),
// rows (a,b) = pair(prow0 + row), written as A operand rows [nrows][pitch]
void tc_embed_antisym_slab(Dev& D, int prec, const cplx* GT, int64_t ldt, int64_t a0, int64_t gb0, int64_t prow0,
                           int64_t nrows, int64_t V, int64_t pitch, int64_t rows_tot, void* out, int64_t emin = 0,
                           int64_t cmin = 0, bool gt_f32 = false);
// dst[c - c0][r] = conj(src[r][c]): the conjugate transpose of columns
// [c0, c0 + nc) of rows [0, nr) of an embedded A operand (K_src complex columns,
// rows_src rows) into an embedded A operand with K = nr (rows_dst rows)
void tc_transpose_conj_a(Dev& D, int prec, const void* src, int64_t K_src, int64_t rows_src, int64_t nr, int64_t c0,
                         int64_t nc, void* dst, int64_t rows_dst);
// zeros in complex columns [c_lo, c_hi) of rows [0, nr) of an embedded A operand
void tc_zero_cols_a(Dev& D, int prec, void* out, int64_t K, int64_t rows_tot, int64_t nr, int64_t c_lo,
                    int64_t c_hi);

// Q map of the T1-weighted ladder piece: Q_amij = sum_ef <am||ef> X_ij^ef with
// <am||ef> = sum_L (Bvv^L_ae Bov^L_mf - Bvv^L_af Bov^L_me), assembled from the
// factor in slabs over a (never stored as an O V^3 block).  X [R][O][O][V][V]
// antisymmetric in (i,j); Q [R][V][O][O][O] = alpha * map + beta * Q.
// Transpose (qmap_t): Xbar_ijef = sum_am Qbar_amij <am||ef> for Qbar
// antisymmetric in (i,j); Xbar = alpha * map + beta * Xbar.
void qmap(Dev& D, LadderCtx& L, const Tensor& X, cplx alpha, cplx beta, Tensor& Q, int prec);
void qmap_t(Dev& D, LadderCtx& L, const Tensor& Qb, cplx alpha, cplx beta, Tensor& Xb, int prec);
// packed ladder layouts on caller-provided buffers:
// Xt[r*PO + ij][ef] = 1/2 (X_ijef - X_ijfe) (i<j, e<f), and
// Z[r][i][j][a][b] = alpha * sign * Zt[r*PO + ij][ab] + beta * Z (antisymmetric fill)
void ladder_pack_xt(Dev& D, const cplx* X, cplx* Xt, int64_t R, int64_t O, int64_t V);
void ladder_unpack_zt(Dev& D, const cplx* Zt, cplx* Z, int64_t R, int64_t O, int64_t V, cplx alpha, cplx beta);
// free device memory plus the pool's cached bytes
double free_bytes(Dev& D);

// pair index of (p<q) among n, row-major strict upper triangle
__host__ __device__ inline int64_t pair_index(int64_t p, int64_t q, int64_t n) {
    return p * (2 * n - p - 1) / 2 + (q - p - 1);
}

// ladder layout kernels on caller-provided buffers
void ladder_pack_x(Dev& D, const cplx* X, cplx* Xp, int64_t R, int64_t O, int64_t V);
void ladder_antisym_slab(Dev& D, const cplx* G, int64_t ldg, cplx* W, int64_t a0, int64_t nrows, int64_t V);
void ladder_unpack_z(Dev& D, const cplx* Zp, cplx* Z, int64_t R, int64_t O, int64_t V);

// message returned by lrcc_last_error(NULL)
void set_global_error(const std::string& msg);
