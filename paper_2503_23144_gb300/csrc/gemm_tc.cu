// Tensor-core complex GEMM on sm_103a: tcgen05.mma with TMEM accumulators,
// operands staged by TMA into 128B-swizzled shared memory.
//
// Complex arithmetic uses the real embedding
//   Re C = sum_k (Ar Br - Ai Bi),  Im C = sum_k (Ar Bi + Ai Br)
// written as ONE real GEMM over an extended K: every complex k becomes S real
// k' slots, and output column n becomes the accumulator column pair
// (2n, 2n+1) = (Re, Im), so the epilogue writes whole complex numbers.
//   kind::tf32  (S = 2):  A' = (Ar, Ai)                 B'_re = (Br, -Bi)   B'_im = (Bi, Br)
//   kind::f16 bf16x3 (S = 6): hi/lo bf16 splits, products hi.hi + hi.lo + lo.hi
//        A' = (Arh, Aih, Arh, Aih, Arl, Ail)
//        B'_re = (Brh, -Bih, Brl, -Bil, Brh, -Bih)   B'_im = (Bih, Brh, Bil, Brl, Bih, Brh)
// Accumulation is FP32 in TMEM; the epilogue scales by the complex alpha and
// adds beta * C in FP64.
//
// Persistent kernel, one CTA of 192 threads per SM: warp 0 issues TMA into a
// ring of shared-memory stages (128 bytes of K per row each), warp 1 issues
// tcgen05.mma into one of two TMEM accumulators of 128 x BN FP32 columns
// (BN = 32..256, picked per call from N), warps 2-5 drain the other
// accumulator (warp w owns TMEM lanes 32 (w % 4) .. +31), so epilogues overlap
// main loops.  Work units are (M tile, N tile, batch, K split); split units
// add into C with FP64 atomics.  Every mbarrier wait is bounded; on expiry the
// kernel raises the context's error word, drains its copies and MMAs, frees
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

#include "lrcc_internal.h"

namespace {

constexpr int BM = 128;
constexpr int ROWB = 128;                 // bytes of K per row per stage
constexpr int A_STAGE = BM * ROWB;        // 16 KB
constexpr int smem_bytes(int bn, int stages) { return stages * (A_STAGE + bn * ROWB) + 1024 + 256; }
constexpr uint32_t WAIT_LIMIT = 1u << 25;  // polls (with backoff) before giving up
// k-blocks (of 128 bytes of K per row, 4 MMAs each) summed in one FP32 TMEM
// accumulator; longer K ranges are added chunk by chunk into C in FP64, so
// the FP32 accumulation error does not grow with the full contraction length
constexpr int KCHUNK = 128;
constexpr uint32_t WAIT_LIMIT_INJECT = 1u << 14;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok;
}
// bounded wait; false (and the error word set) if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;             // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

// instruction descriptor: D f32, A/B format, both K-major, N, M
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_fmt, int M, int N) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// FP64 work in the epilogue is kept to the adds into C (GB300 issues two FP64
// FMAs per SM per clock): alpha scales the FP32 accumulator in FP32 unless
// the products are exact integer chains (exact_alpha), and beta = 0 / 1 skip
// their multiplies.
struct Epi {
    int64_t M, N;
    cplx* C;
    int64_t sCb;
    Lvl lm, ln;  // output row and column offsets
    cplx alpha, beta;
    int conj_acc;     // use conj(accumulator): conj(A.conj(B)) = conj(A).B
    int atomic;       // split-K: accumulate alpha*acc into C with FP64 atomics (C pre-scaled)
    int exact_alpha;  // apply alpha in FP64 (accumulators that are exact sums)
    int f32out;       // C holds complex FP32 pairs (float2): alpha acc (+ C) in FP32, no split K
};

// alpha * accumulator (FP32 pair) as FP64: in FP32 arithmetic unless alpha must
// be applied exactly (sums of exact integer chains)
__device__ __forceinline__ cplx out_value(const Epi& ep, bool alpha1, float afx, float afy, float fr, float fi) {
    if (alpha1) return make_double2(f32_to_f64(fr), f32_to_f64(fi));
    if (ep.exact_alpha) {
        const double re = f32_to_f64(fr), im = f32_to_f64(fi);
        return make_double2(ep.alpha.x * re - ep.alpha.y * im, ep.alpha.x * im + ep.alpha.y * re);
    }
    return make_double2(f32_to_f64(afx * fr - afy * fi), f32_to_f64(afx * fi + afy * fr));
}

// v += old (factor 1), or beta * old, or nothing
__device__ __forceinline__ void add_old(cplx& v, const cplx& old, bool add1, bool beta0, const cplx& beta) {
    if (add1) {
        v.x += old.x;
        v.y += old.y;
    } else if (!beta0) {
        v.x += beta.x * old.x - beta.y * old.y;
        v.y += beta.x * old.y + beta.y * old.x;
    }
}

// Work units of the persistent kernel: (M tile, N tile, batch, K split).
// Inside one split and batch the tiles run in groups of `group` M tiles with
// the M tile fastest, so CTAs resident together share the B tiles they read.
struct Sched {
    int tiles_m, tiles_n, batch, splits, kps, num_kb, group;
    int kchunk;  // k-blocks accumulated in FP32 before the epilogue adds them to C in FP64
    int kpb;     // k-blocks per K panel of the operands (0: rows stored whole)
    int kbase;   // k-block of the operands where this GEMM's K range starts
    // tile mask (mv > 0): rows m and complex columns n are grouped in blocks of
    // mv; a tile runs only if one of its rows and one of its columns have
    // (index mod mv) >= memin
    int mv, memin;
    long long mrows, mcols;
    long long units;
};

// does the index range [i0, i1] contain an index with (index mod v) >= e?
__device__ __forceinline__ bool range_live(long long i0, long long i1, int v, int e) {
    return (i0 / v != i1 / v) || (int)(i1 % v) >= e;
}

template <int BN>
__device__ __forceinline__ bool unit_live(const Sched& s, int tm, int tn) {
    if (s.mv <= 0) return true;
    const long long r0 = (long long)tm * BM, c0 = (long long)tn * (BN / 2);
    const long long r1 = min(s.mrows, r0 + BM) - 1, c1 = min(s.mcols, c0 + BN / 2) - 1;
    return range_live(r0, r1, s.mv, s.memin) && range_live(c0, c1, s.mv, s.memin);
}

__device__ __forceinline__ void unit_coords(const Sched& s, long long u, int& tm, int& tn, int& bz, int& kb0,
                                            int& kb1) {
    const long long tiles = (long long)s.tiles_m * s.tiles_n;
    const long long per_split = tiles * s.batch;
    const int sp = (int)(u / per_split);
    const long long r = u - (long long)sp * per_split;
    bz = (int)(r / tiles);
    const long long t = r - (long long)bz * tiles;
    const long long gsz = (long long)s.group * s.tiles_n;
    const int g = (int)(t / gsz);
    const int w = (int)(t - (long long)g * gsz);
    const int m0 = g * s.group;
    const int gh = min(s.group, s.tiles_m - m0);
    tm = m0 + w % gh;
    tn = w / gh;
    kb0 = sp * s.kps;
    kb1 = min(s.num_kb, kb0 + s.kps);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// bounded wait taken by a whole warp: every lane polls, and the warp goes on
// only if all lanes saw the phase complete (so the .sync.aligned TMEM loads
// that follow run converged)
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* err, uint32_t limit) {
    bool ok = mbar_wait(bar, parity, err, limit);
    return __all_sync(0xffffffffu, ok);
}

// Persistent tcgen05 GEMM.  192 threads: warp 0 lane 0 issues TMA, warp 1
// lane 0 issues MMAs, warps 2-5 drain accumulators (warp w reads TMEM lanes
// 32 (w % 4) .. +31).  Two TMEM accumulators of BN columns alternate, so the
// epilogue of one unit overlaps the main loop of the next.
template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(192, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, Sched sc, Epi ep,
              int* err, int skip_tma, uint32_t wait_limit) {
    constexpr int B_STAGE = BN * ROWB;
    constexpr uint32_t TMEM_COLS = 2 * BN;
    constexpr int KELEM = KIND == 0 ? 64 : 32;  // elements per 128-byte row
    constexpr uint32_t IDESC = instr_desc(KIND == 0 ? 1u : 2u, BM, BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_STAGE;
    uint64_t* full = (uint64_t*)(sB + STAGES * B_STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;  // [2] accumulator complete
    uint64_t* acce = accf + 2;        // [2] accumulator drained
    uint64_t* done = acce + 2;        // every MMA of this CTA complete
    uint32_t* tslot = (uint32_t*)(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], 4);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            int it = 0;  // stage uses armed so far
            bool ok = true;
            for (long long u = blockIdx.x; ok && u < sc.units; u += gridDim.x) {
                int tm, tn, bz, kb0, kb1;
                unit_coords(sc, u, tm, tn, bz, kb0, kb1);
                if (!unit_live<BN>(sc, tm, tn)) continue;
                for (int kb = kb0; kb < kb1; ++kb) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, err, wait_limit)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], A_STAGE + B_STAGE);
                    ++it;
                    if (skip_tma) continue;  // fault injection: the stage's bytes never arrive
                    const int kg = kb + sc.kbase;
                    const int kx = sc.kpb ? (kg % sc.kpb) * KELEM : kg * KELEM;
                    const int kz = sc.kpb ? kg / sc.kpb : bz;
                    tma_load_3d(sA + s * A_STAGE, &ta, &full[s], kx, tm * BM, kz);
                    tma_load_3d(sB + s * B_STAGE, &tb, &full[s], kx, tn * BN, kz);
                }
            }
            // copies still in flight land before the CTA exits: wait for the
            // last armed phase of every stage (already complete on the normal path)
            for (int s = 0; s < STAGES && s < it; ++s) {
                const int last = s + STAGES * ((it - 1 - s) / STAGES);
                mbar_wait(&full[s], (uint32_t)(last / STAGES) & 1u, err, wait_limit);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            int it = 0, ti = 0;
            bool ok = true;
            for (long long u = blockIdx.x; ok && u < sc.units; u += gridDim.x) {
                int tm, tn, bz, kb0, kb1;
                unit_coords(sc, u, tm, tn, bz, kb0, kb1);
                if (!unit_live<BN>(sc, tm, tn)) continue;
                // the unit's K range in chunks, each into the next accumulator
                for (int c0 = kb0; ok && c0 < kb1; c0 += sc.kchunk) {
                    const int c1 = min(kb1, c0 + sc.kchunk);
                    const int acc = ti & 1;
                    if (!mbar_wait(&acce[acc], ((uint32_t)(ti >> 1) & 1u) ^ 1u, err, wait_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * BN);
                    for (int kb = c0; kb < c1; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                        if (!mbar_wait(&full[s], ph, err, wait_limit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = smem_desc(su32(sA + s * A_STAGE));
                        const uint64_t bd = smem_desc(su32(sB + s * B_STAGE));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            // 32 bytes of K per MMA (16 bf16 or 8 tf32): +2 in the >>4 address field
                            mma<KIND>(d, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), IDESC,
                                      (kb > c0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit(&accf[acc]);
                    ++ti;
                }
            }
            mma_commit(done);
        }
    } else {
        // epilogue: FP32 accumulator pairs (Re, Im) -> alpha * acc (+ beta C) in FP64
        const int q = warp & 3;
        const bool beta0 = ep.beta.x == 0.0 && ep.beta.y == 0.0;
        const bool beta1 = ep.beta.x == 1.0 && ep.beta.y == 0.0;
        const bool alpha1 = ep.alpha.x == 1.0 && ep.alpha.y == 0.0;
        const float afx = (float)ep.alpha.x, afy = (float)ep.alpha.y;
        int ti = 0;
        bool ok = true;
        for (long long u = blockIdx.x; ok && u < sc.units; u += gridDim.x) {
            int tm, tn, bz, kb0, kb1;
            unit_coords(sc, u, tm, tn, bz, kb0, kb1);
            if (!unit_live<BN>(sc, tm, tn)) continue;
            for (int c0 = kb0; c0 < kb1; c0 += sc.kchunk) {
                // first chunk: C = alpha acc + beta C; later chunks: C += alpha acc
                const bool first = c0 == kb0;
                const bool rd = !ep.atomic && (!first || !beta0);
                const bool add1 = !first || beta1;  // old C enters with factor 1
                const int acc = ti & 1;
                if (!warp_wait(&accf[acc], (uint32_t)(ti >> 1) & 1u, err, wait_limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int64_t m = (int64_t)tm * BM + q * 32 + lane;
                const bool live = m < ep.M;
                cplx* Cb = ep.C + (int64_t)bz * ep.sCb + (live ? lvl_off(ep.lm, m) : 0);
                if (ep.f32out) {
                    // complex FP32 output (an intermediate read only by a split/convert kernel)
                    float2* Cf = (float2*)ep.C + (int64_t)bz * ep.sCb + (live ? lvl_off(ep.lm, m) : 0);
#pragma unroll 1
                    for (int c = 0; c < BN / 32; ++c) {
                        uint32_t r[32];
                        const int64_t n0 = (int64_t)tn * (BN / 2) + c * 16;
                        float2 oldf[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            oldf[j] = (rd && live && n0 + j < ep.N) ? Cf[lvl_off(ep.ln, n0 + j)] : make_float2(0.f, 0.f);
                        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c * 32), r);
                        if (live) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int64_t n = n0 + j;
                                if (n < ep.N) {
                                    const float fr = __uint_as_float(r[2 * j]);
                                    const float fi = ep.conj_acc ? -__uint_as_float(r[2 * j + 1]) : __uint_as_float(r[2 * j + 1]);
                                    float vr = alpha1 ? fr : afx * fr - afy * fi;
                                    float vi = alpha1 ? fi : afx * fi + afy * fr;
                                    if (rd) {
                                        vr += oldf[j].x;
                                        vi += oldf[j].y;
                                    }
                                    Cf[lvl_off(ep.ln, n)] = make_float2(vr, vi);
                                }
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acce[acc]);
                    ++ti;
                    continue;
                }
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t r[32];
                    const int64_t n0 = (int64_t)tn * (BN / 2) + c * 16;
                    // old C values are loaded before the TMEM read, all in flight together
                    cplx old[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        old[j] = (rd && live && n0 + j < ep.N) ? Cb[lvl_off(ep.ln, n0 + j)] : make_double2(0.0, 0.0);
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c * 32), r);
                    if (live) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int64_t n = n0 + j;
                            if (n < ep.N) {
                                const float fi = __uint_as_float(r[2 * j + 1]);
                                cplx v = out_value(ep, alpha1, afx, afy, __uint_as_float(r[2 * j]),
                                                   ep.conj_acc ? -fi : fi);
                                cplx* cp = Cb + lvl_off(ep.ln, n);
                                if (ep.atomic) {
                                    atomicAdd(&cp->x, v.x);
                                    atomicAdd(&cp->y, v.y);
                                    continue;
                                }
                                add_old(v, old[j], add1, beta0, ep.beta);
                                *cp = v;
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[acc]);
                ++ti;
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        // every MMA issued by this CTA has finished before its TMEM is released
        bool fin = warp_wait(done, 0, err, wait_limit);
        if (!fin) warp_wait(done, 0, err, wait_limit);
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// operand embedding (split / convert).  Embedded operands are [batch][rows][pitch]
// with only the first S*K columns written: the tensor maps cover S*K columns and
// the true row count, and TMA fills everything outside with zeros.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t bf2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Embedded-operand layout.  Rows of up to 16 KB are stored whole:
// [batch][rows][pw].  Longer rows are cut into np equal panels of at most
// 16 KB (pw a multiple of 128 bytes, batch 1): [panel][rows][pw], so that one TMA box
// (rows x 128 bytes of K) reads from a few pages instead of one page per row
// (rows of megabytes otherwise miss the TLB on every row).  `rows` is the row
// count of the whole buffer (the panel stride); pointers may be offset by whole
// rows inside panel 0.
struct EL {
    int64_t rows = 0, pw = 0;
    int np = 1;
    FastDiv fpw;
};
__device__ __forceinline__ int64_t el_off(const EL& L, int64_t b, int64_t row, int64_t col) {
    if (L.np == 1) return (b * L.rows + row) * L.pw + col;
    const uint32_t p = L.fpw.div((uint32_t)col);
    return ((int64_t)p * L.rows + row) * L.pw + (col - (int64_t)p * L.pw);
}

template <int KIND, bool IS_B>
__device__ __forceinline__ void embed_store(void* __restrict__ out, const EL& L, int64_t b, int64_t r, int64_t k,
                                            float vr, float vi) {
    if (KIND == 0) {
        const __nv_bfloat16 rh = __float2bfloat16(vr), ih = __float2bfloat16(vi);
        const __nv_bfloat16 rl = __float2bfloat16(vr - __bfloat162float(rh));
        const __nv_bfloat16 il = __float2bfloat16(vi - __bfloat162float(ih));
        __nv_bfloat16* o = (__nv_bfloat16*)out;
        if (!IS_B) {
            const uint32_t hh = bf2(rh, ih);
            *(uint32_t*)(o + el_off(L, b, r, 6 * k)) = hh;
            *(uint32_t*)(o + el_off(L, b, r, 6 * k + 2)) = hh;
            *(uint32_t*)(o + el_off(L, b, r, 6 * k + 4)) = bf2(rl, il);
        } else {
            const __nv_bfloat16 nih = __hneg(ih), nil = __hneg(il);
            const uint32_t re_h = bf2(rh, nih), im_h = bf2(ih, rh);
            *(uint32_t*)(o + el_off(L, b, 2 * r, 6 * k)) = re_h;
            *(uint32_t*)(o + el_off(L, b, 2 * r, 6 * k + 2)) = bf2(rl, nil);
            *(uint32_t*)(o + el_off(L, b, 2 * r, 6 * k + 4)) = re_h;
            *(uint32_t*)(o + el_off(L, b, 2 * r + 1, 6 * k)) = im_h;
            *(uint32_t*)(o + el_off(L, b, 2 * r + 1, 6 * k + 2)) = bf2(il, rl);
            *(uint32_t*)(o + el_off(L, b, 2 * r + 1, 6 * k + 4)) = im_h;
        }
    } else {
        const uint32_t br = to_tf32(vr), bi = to_tf32(vi);
        uint32_t* o = (uint32_t*)out;
        if (!IS_B) {
            *(uint2*)(o + el_off(L, b, r, 2 * k)) = make_uint2(br, bi);
        } else {
            *(uint2*)(o + el_off(L, b, 2 * r, 2 * k)) = make_uint2(br, bi ^ 0x80000000u);
            *(uint2*)(o + el_off(L, b, 2 * r + 1, 2 * k)) = make_uint2(bi, br);
        }
    }
}

// source S[b][r][k] with strides (sb, sr, sk); k fastest across threads
template <int KIND, bool IS_B>
__global__ void k_embed(const cplx* __restrict__ S, int64_t sb, Lvl lr, Lvl lk, int cj, int64_t batch,
                        int64_t Rn, int64_t K, FastDiv fR, FastDiv fK, EL L, void* __restrict__ out) {
    const int64_t total = batch * Rn * K;
    const bool fast = total < FAST_INDEX_LIMIT;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t k, r, b;
        if (fast) {
            const uint32_t t = fK.div((uint32_t)idx), bb = fR.div(t);
            k = (uint32_t)idx - t * fK.d;
            r = t - bb * fR.d;
            b = bb;
        } else {
            const int64_t t = idx / K;
            k = idx % K;
            r = t % Rn;
            b = t / Rn;
        }
        const cplx v = S[b * sb + lvl_off(lr, r) + lvl_off(lk, k)];
        const float vi = f64_to_f32_rz(v.y);
        embed_store<KIND, IS_B>(out, L, b, r, k, f64_to_f32_rz(v.x), cj ? -vi : vi);
    }
}

// the same for sources contiguous in r: 32x32 tiles read along r, written along k
template <int KIND, bool IS_B>
__global__ void __launch_bounds__(256) k_embed_t(const cplx* __restrict__ S, int64_t sb, Lvl lr, Lvl lk, int cj,
                                                 int64_t batch, int64_t Rn, int64_t K, EL L,
                                                 void* __restrict__ out) {
    __shared__ cplx tile[32][33];
    const int64_t tr_n = (Rn + 31) / 32, tk_n = (K + 31) / 32;
    const int64_t ntiles = batch * tr_n * tk_n;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t tk = t % tk_n, u = t / tk_n, tr = u % tr_n, b = u / tr_n;
        const int64_t r0 = tr * 32, k0 = tk * 32;
        for (int j = ty; j < 32; j += 8) {
            const int64_t r = r0 + tx, k = k0 + j;
            cplx v = make_double2(0.0, 0.0);
            if (r < Rn && k < K) v = S[b * sb + lvl_off(lr, r) + lvl_off(lk, k)];
            tile[j][tx] = v;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t r = r0 + j, k = k0 + tx;
            if (r < Rn && k < K) {
                const cplx v = tile[tx][j];
                const float vi = f64_to_f32_rz(v.y);
                embed_store<KIND, IS_B>(out, L, b, r, k, f64_to_f32_rz(v.x), cj ? -vi : vi);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP64-class products on bf16 tensor cores (the splitting scheme of Ozaki,
// Ogita, Oishi and Rump, Numer. Algorithms 59 (2012), with integer slices).
// Every row r of an operand gets an exponent e_r with |x| < 2^e_r for all its
// elements (real and imaginary parts); x 2^-e_r is written as OZ_S digits of
// OZ_BITS bits, d_s in (-2^OZ_BITS, 2^OZ_BITS), x = sum_s d_s 2^(e_r - OZ_BITS (s+1))
// + (remainder below 2^(e_r - OZ_BITS OZ_S)).  Each slice d_s 2^(...) is exact
// in bf16.  For one output element, all products of the slice pairs (s, t)
// with s + t = d are integer multiples of one power of two, each at most
// (2^OZ_BITS - 1)^2 < 2^12 of it, so an FP32 accumulation chain of up to
// 4096 products (64 k-blocks of 64 bf16) is exact; the chains are added into
// C in FP64.  Diagonals d = 0 .. OZ_S-1 are kept (products below
// 2^-(OZ_BITS OZ_S) of the leading term are dropped): relative error ~1e-12
// of max|A_row| max|B_col| per product.
// ---------------------------------------------------------------------------
constexpr int OZ_S = 7, OZ_BITS = 6, OZ_KCHUNK = 64;

// Row exponents from the IEEE bit fields (integer operations only): for
// non-negative doubles the bit patterns order like the values, so the row
// maximum of |Re|, |Im| is an integer maximum; e = biased exponent - 1022 gives
// max < 2^e (zero rows: e = 0; subnormal maxima: e = -1022).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ int exp_of_bits(unsigned long long m) {
    if (m == 0) return 0;
    const int ex = (int)(m >> 52);
    return ex == 0 ? -1022 : ex - 1022;
}

// one warp per row, lanes along k
__global__ void k_row_exp_w(const cplx* __restrict__ S, int64_t sb, int64_t sr, int64_t sk, int64_t batch,
                            int64_t Rn, int64_t K, int* __restrict__ e) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = batch * Rn;
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < rows;
         row += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t b = row / Rn, r = row % Rn;
        const cplx* p = S + b * sb + r * sr;
        unsigned long long m = 0;
        for (int64_t k = lane; k < K; k += 32) {
            const cplx v = p[k * sk];
            m = max(m, max(abs_bits(v.x), abs_bits(v.y)));
        }
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) e[row] = exp_of_bits(m);
    }
}

// one thread per row (for sources contiguous along r: consecutive threads read
// consecutive addresses)
__global__ void k_row_exp_t(const cplx* __restrict__ S, int64_t sb, int64_t sr, int64_t sk, int64_t batch,
                            int64_t Rn, int64_t K, int* __restrict__ e) {
    const int64_t rows = batch * Rn;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = row / Rn, r = row % Rn;
        const cplx* p = S + b * sb + r * sr;
        unsigned long long m = 0;
        for (int64_t k = 0; k < K; ++k) {
            const cplx v = p[k * sk];
            m = max(m, max(abs_bits(v.x), abs_bits(v.y)));
        }
        e[row] = exp_of_bits(m);
    }
}

// F = floor(|x| 2^(OZ_BITS OZ_S - e)) from the bit fields: x = M 2^(ex - 1075)
// with the 53-bit integer M; |x| < 2^e keeps F below 2^(OZ_BITS OZ_S).
// Its base-2^OZ_BITS digits, most significant first, are the slices' digits
// (truncation toward zero of |x|; the sign is carried separately).
__device__ __forceinline__ unsigned long long oz_fixed(double x, int e, uint32_t& sign) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    sign = (uint32_t)(b >> 63);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) return 0;  // zero; subnormals lie below every slice kept
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1075 - e + OZ_BITS * OZ_S;
    if (sh >= 0) return M << sh;
    return sh <= -64 ? 0ull : (M >> (-sh));
}

// bf16 bit pattern of sign * d * 2^p for a digit 0 <= d < 2^OZ_BITS (exact:
// d has at most 6 significant bits); below the bf16 normal range -> zero
__device__ __forceinline__ uint32_t bf16_digit(uint32_t d, int p, uint32_t sign) {
    if (d == 0) return 0u;
    const int len = 32 - __clz(d);
    const int be = p + len - 1 + 127;
    if (be <= 0) return 0u;
    if (be >= 255) return (sign << 15) | 0x7F80u;
    return (sign << 15) | ((uint32_t)be << 7) | ((d << (8 - len)) & 0x7Fu);
}

// slices of v = op(S)[b][r][k] with row exponent e.  A rows: slice s at
// columns s*kpad + 2k, 2k+1 = (Re, Im).  B row pairs (2r: real output, 2r+1:
// imaginary output) in reversed slice order: slice t at (OZ_S-1-t)*kpad,
// real row (Re, -Im), imaginary row (Im, Re).
template <bool IS_B>
__device__ __forceinline__ void oz_store(void* __restrict__ out, int64_t rows_e, int64_t kpad, int64_t b, int64_t r,
                                         int64_t k, cplx v, bool conj, int e) {
    const int64_t pitch = OZ_S * kpad;
    uint16_t* row = (uint16_t*)out + (b * rows_e + (IS_B ? 2 * r : r)) * pitch + 2 * k;
    uint32_t sr, si;
    const unsigned long long Fr = oz_fixed(v.x, e, sr), Fi = oz_fixed(v.y, e, si);
    if (conj) si ^= 1u;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
        const int sh = OZ_BITS * (OZ_S - 1 - s), p = e - OZ_BITS * (s + 1);
        const uint32_t dr = (uint32_t)(Fr >> sh) & ((1u << OZ_BITS) - 1u);
        const uint32_t di = (uint32_t)(Fi >> sh) & ((1u << OZ_BITS) - 1u);
        const uint32_t hr = bf16_digit(dr, p, sr), hi = bf16_digit(di, p, si);
        if (!IS_B) {
            *(uint32_t*)(row + s * kpad) = hr | (hi << 16);
        } else {
            const int64_t off = (OZ_S - 1 - s) * kpad;
            const uint32_t nhi = hi ? hi ^ 0x8000u : 0u;
            *(uint32_t*)(row + off) = hr | (nhi << 16);
            *(uint32_t*)(row + pitch + off) = hi | (hr << 16);
        }
    }
}

// k runs over the padded range [0, kpad/2); positions k >= K are written as zeros
template <bool IS_B>
__global__ void k_oz_embed(const cplx* __restrict__ S, int64_t sb, int64_t sr, int64_t sk, int cj, int64_t batch,
                           int64_t Rn, int64_t K, int64_t K2, FastDiv fR, FastDiv fK2, const int* __restrict__ e,
                           int64_t rows_e, int64_t kpad, void* __restrict__ out) {
    const int64_t total = batch * Rn * K2;
    const bool fast = total < FAST_INDEX_LIMIT;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t k, r, b;
        if (fast) {
            const uint32_t t = fK2.div((uint32_t)idx), bb = fR.div(t);
            k = (uint32_t)idx - t * fK2.d;
            r = t - bb * fR.d;
            b = bb;
        } else {
            const int64_t t = idx / K2;
            k = idx % K2;
            r = t % Rn;
            b = t / Rn;
        }
        cplx v = make_double2(0.0, 0.0);
        if (k < K) v = S[b * sb + r * sr + k * sk];
        oz_store<IS_B>(out, rows_e, kpad, b, r, k, v, cj != 0, e[b * Rn + r]);
    }
}

// the same for sources contiguous in r: 32x32 tiles read along r, written along k
template <bool IS_B>
__global__ void __launch_bounds__(256) k_oz_embed_t(const cplx* __restrict__ S, int64_t sb, int64_t sk, int cj,
                                                    int64_t batch, int64_t Rn, int64_t K, int64_t K2,
                                                    const int* __restrict__ e, int64_t rows_e, int64_t kpad,
                                                    void* __restrict__ out) {
    __shared__ cplx tile[32][33];
    const int64_t tr_n = (Rn + 31) / 32, tk_n = (K2 + 31) / 32;
    const int64_t ntiles = batch * tr_n * tk_n;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t tk = t % tk_n, u = t / tk_n, tr = u % tr_n, b = u / tr_n;
        const int64_t r0 = tr * 32, k0 = tk * 32;
        for (int j = ty; j < 32; j += 8) {
            const int64_t r = r0 + tx, k = k0 + j;
            cplx v = make_double2(0.0, 0.0);
            if (r < Rn && k < K) v = S[b * sb + r + k * sk];
            tile[j][tx] = v;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t r = r0 + j, k = k0 + tx;
            if (r < Rn && k < K2) oz_store<IS_B>(out, rows_e, kpad, b, r, k, tile[tx][j], cj != 0, e[b * Rn + r]);
        }
        __syncthreads();
    }
}

// (p, q) of pair index k among n (p < q, row-major strict upper triangle)
__device__ __forceinline__ void pair_of(int64_t k, int64_t n, int64_t& p, int64_t& q) {
    const double a = double(2 * n - 1);
    int64_t pp = (int64_t)floor((a - sqrt(fmax(a * a - 8.0 * double(k), 0.0))) * 0.5);
    if (pp < 0) pp = 0;
    while (pp > 0 && pp * (2 * n - pp - 1) / 2 > k) --pp;
    while (pp < n - 2 && (pp + 1) * (2 * n - pp - 2) / 2 <= k) ++pp;
    p = pp;
    q = k - pp * (2 * n - pp - 1) / 2 + pp + 1;
}

// Embedded <ab||ef> rows of one ladder slab, straight from the assembly GEMM:
//   W_ab,ef = GT[(b-gb0)V + f][(a-a0)V + e] - GT[(b-gb0)V + e][(a-a0)V + f],  e < f,
// GT[(b,f)][(a,e)] = sum_L Bvv^L_ae Bvv^L_bf = <ab|ef>.  One task = one row
// (a,b) and one 32x32 (e,f) tile pair with te <= tf; both GT blocks are read
// along their contiguous (a,e) index and transposed through shared memory.
// GT holds complex FP64 or complex FP32 (GTE = float2) values.  The FP64
// difference is truncated to FP32; the FP32 difference is taken in FP32
// (round to nearest): both within 2^-23 relative of the exact difference of
// the stored values, and no FP64 instruction touches FP32 input.  cmin > 0:
// only the columns (pairs e<f) >= cmin are written, and the 32x32 (e, f) tiles
// whose e are all below emin are skipped (their GT entries were not computed).
__device__ __forceinline__ float2 gt_diff(const cplx& u, const cplx& w) {
    return make_float2(f64_to_f32_rz(u.x - w.x), f64_to_f32_rz(u.y - w.y));
}
__device__ __forceinline__ float2 gt_diff(const float2& u, const float2& w) {
    return make_float2(u.x - w.x, u.y - w.y);
}
template <typename GTE>
__device__ __forceinline__ GTE gt_zero();
template <>
__device__ __forceinline__ cplx gt_zero<cplx>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ float2 gt_zero<float2>() { return make_float2(0.f, 0.f); }

template <int KIND, typename GTE>
__global__ void __launch_bounds__(256) k_embed_antisym(const GTE* __restrict__ GT, int64_t ldt, int64_t a0,
                                                       int64_t gb0, int64_t prow0, int64_t nrows, int64_t V, EL L,
                                                       void* __restrict__ out, int64_t emin, int64_t cmin) {
    __shared__ GTE t1[32][33];
    __shared__ GTE t2[32][33];
    const int64_t T = (V + 31) / 32, npair = T * (T + 1) / 2;
    const int64_t tasks = nrows * npair;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const GTE zero = gt_zero<GTE>();
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const int64_t row = t / npair;
        int64_t rem = t - row * npair, te = 0;
        while (rem >= T - te) {
            rem -= T - te;
            ++te;
        }
        const int64_t tf = te + rem;
        if (te * 32 + 31 < emin) continue;  // uniform across the block
        int64_t a, b;
        pair_of(prow0 + row, V, a, b);
        const int64_t ra = (a - a0) * V, cb = (b - gb0) * V;
        const int64_t e0 = te * 32, f0 = tf * 32;
        for (int j = ty; j < 32; j += 8) {
            const int64_t f = f0 + j, e = e0 + tx;
            t1[j][tx] = (f < V && e < V) ? GT[(cb + f) * ldt + ra + e] : zero;  // <ab|ef>, [f][e]
            const int64_t e2 = e0 + j, f2 = f0 + tx;
            t2[j][tx] = (e2 < V && f2 < V) ? GT[(cb + e2) * ldt + ra + f2] : zero;  // <ab|fe>, [e][f]
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t e = e0 + j, f = f0 + tx;
            if (e < f && f < V) {
                const int64_t ef = e * (2 * V - e - 1) / 2 + (f - e - 1);
                if (ef >= cmin) {
                    const float2 d = gt_diff(t1[tx][j], t2[j][tx]);
                    embed_store<KIND, false>(out, L, 0, row, ef, d.x, d.y);
                }
            }
        }
        __syncthreads();
    }
}

int grid_n(Dev& D, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)D.sm_count * 16));
}

// dst[c - c0][r] = conj(src[r][c]) for embedded A operands (rows r < nr of src
// with layout Ls, columns c in [c0, c0 + nc); dst rows with layout Ld), the
// embedded words moved as they are with the imaginary signs flipped (bf16x3:
// three words (re,im) per complex element, imaginary in the high half; TF32:
// (re, im)).  32 x 32 tiles through shared memory: reads along c, writes along r.
template <int KIND>
__global__ void __launch_bounds__(256) k_transpose_conj_a(const void* __restrict__ src, EL Ls, int64_t nr,
                                                          int64_t c0, int64_t nc, void* __restrict__ dst, EL Ld) {
    constexpr int W = KIND == 0 ? 3 : 2;  // 32-bit words per complex element
    __shared__ uint32_t tile[32][33][W];
    const int64_t tr_n = (nr + 31) / 32, tc_n = (nc + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const uint32_t* s32 = (const uint32_t*)src;
    uint32_t* d32 = (uint32_t*)dst;
    for (int64_t t = blockIdx.x; t < tr_n * tc_n; t += gridDim.x) {
        const int64_t r0 = (t / tc_n) * 32, cc0 = (t % tc_n) * 32;
        for (int j = ty; j < 32; j += 8) {
            const int64_t r = r0 + j, c = cc0 + tx;
            if (r < nr && c < nc) {
                if (KIND == 0) {
                    // element offsets are in bf16 units: word = offset / 2
                    for (int w = 0; w < 3; ++w)
                        tile[j][tx][w] = s32[el_off(Ls, 0, r, 6 * (c0 + c) + 2 * w) / 2] ^ 0x80000000u;
                } else {
                    const uint2 v = *(const uint2*)(s32 + el_off(Ls, 0, r, 2 * (c0 + c)));
                    tile[j][tx][0] = v.x;
                    tile[j][tx][1] = v.y ^ 0x80000000u;
                }
            }
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t c = cc0 + j, r = r0 + tx;
            if (r < nr && c < nc) {
                if (KIND == 0) {
                    for (int w = 0; w < 3; ++w) d32[el_off(Ld, 0, c, 6 * r + 2 * w) / 2] = tile[tx][j][w];
                } else {
                    *(uint2*)(d32 + el_off(Ld, 0, c, 2 * r)) = make_uint2(tile[tx][j][0], tile[tx][j][1]);
                }
            }
        }
        __syncthreads();
    }
}

// zeros in complex columns [c_lo, c_hi) of rows [0, nr) of an embedded A operand
template <int KIND>
__global__ void k_zero_cols_a(void* __restrict__ out, EL L, int64_t nr, int64_t c_lo, int64_t c_hi) {
    const int64_t w = c_hi - c_lo, total = nr * w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        embed_store<KIND, false>(out, L, 0, i / w, c_lo + i % w, 0.0f, 0.0f);
}

// cuTensorMapEncodeTiled from the driver, resolved through the runtime so the
// library itself does not link libcuda (it still loads on machines without a
// driver, where only host-side validation can run)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            throw LrccError(LRCC_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// dims: x = K extent (the true K, or a whole panel), y = rows of this operand
// view, z = batch or panel; strides: row pitch and batch/panel stride (the
// buffer's full row count times the pitch)
void encode(CUtensorMap* map, const void* base, int kind, uint64_t dx, uint64_t pitch, uint64_t rows,
            uint64_t rows_tot, uint64_t dz, uint32_t box_rows) {
    CUtensorMapDataType dt = kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint64_t es = kind == 0 ? 2 : 4;
    cuuint64_t dims[3] = {dx, rows, dz};
    cuuint64_t strides[2] = {pitch * es, pitch * rows_tot * es};
    cuuint32_t box[3] = {(cuuint32_t)(ROWB / es), box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw LrccError(LRCC_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

constexpr int stages_for(int bn) { return bn == 256 ? 4 : bn == 128 ? 6 : 8; }

template <int KIND, int BN>
void launch_tc(Dev& D, const CUtensorMap& ta, const CUtensorMap& tb, const Sched& sc, const Epi& ep, int grid,
               int skip, uint32_t limit) {
    constexpr int ST = stages_for(BN);
    constexpr int SMEM = smem_bytes(BN, ST);
    static_assert(SMEM <= 232448, "shared memory over the per-CTA limit");
    static bool attr = false;
    if (!attr) {
        CK(cudaFuncSetAttribute(k_tc_gemm<KIND, BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        attr = true;
    }
    k_tc_gemm<KIND, BN, ST><<<grid, 192, SMEM, D.st>>>(ta, tb, sc, ep, D.err_flag, skip, limit);
}

// accumulator tile width for n2 = 2N real output columns: the fewest padded
// columns, with a small penalty on narrow tiles (more A re-reads per output)
int bn_for(int64_t n2) {
    static const int cand[4] = {256, 128, 64, 32};
    static const double pen[4] = {1.0, 1.25, 1.6, 2.2};
    int best = 256;
    double bc = 1e300;
    for (int i = 0; i < 4; ++i) {
        double c = double((n2 + cand[i] - 1) / cand[i] * cand[i]) * pen[i];
        if (c < bc) {
            bc = c;
            best = cand[i];
        }
    }
    return best;
}

int64_t slots(int kind) { return kind == 0 ? 6 : 2; }

}  // namespace

bool gemm_tc_available() { return true; }

constexpr int64_t PANEL_BYTES = 16384;

// layout of an embedded operand with rows_tot rows and complex K
static EL make_el(int kind, int64_t K, int64_t rows_tot, int64_t batch) {
    const int64_t es = kind == 0 ? 2 : 4, q = 16 / es, kd = slots(kind) * K, full = (kd + q - 1) / q * q;
    const int64_t pmax = PANEL_BYTES / es, kel = ROWB / es;
    EL L;
    L.rows = rows_tot;
    if (batch == 1 && full > pmax) {
        L.np = (int)((kd + pmax - 1) / pmax);
        L.pw = ((kd + L.np - 1) / L.np + kel - 1) / kel * kel;  // equal panels, whole k-blocks
        L.fpw = FastDiv(L.pw);
    } else {
        L.pw = full;
    }
    return L;
}

extern "C" lrcc_status lrcc_embed_layout(int prec, int64_t K, int64_t rows, int64_t batch, int64_t* n_panels,
                                         int64_t* panel_width) {
    if ((prec != LRCC_MIXED_TF32 && prec != LRCC_MIXED_BF16X3) || K < 1 || rows < 1 || batch < 1 || !n_panels ||
        !panel_width)
        return LRCC_EINVAL;
    const EL L = make_el(prec == LRCC_MIXED_BF16X3 ? 0 : 1, K, rows, batch);
    *n_panels = L.np;
    *panel_width = L.pw;
    return LRCC_OK;
}

size_t tc_embed_bytes(int prec, int64_t rows, int64_t K, int64_t batch, int64_t& rows_e, int64_t& pitch, bool is_b) {
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const int64_t es = kind == 0 ? 2 : 4;
    rows_e = is_b ? 2 * rows : rows;
    const EL L = make_el(kind, K, rows_e, batch);
    pitch = L.pw;
    return (size_t)(batch * rows_e * L.np * L.pw * es);
}

// zeros in the last panel beyond the S K used columns, for rows [0, nrows) of
// the view at `out` (panelled layouts only: TMA reads whole panels)
static void zero_tail(Dev& D, int kind, void* out, const EL& L, int64_t K, int64_t nrows) {
    if (L.np == 1 || nrows <= 0) return;
    const int64_t es = kind == 0 ? 2 : 4, kd = slots(kind) * K, used = kd - (int64_t)(L.np - 1) * L.pw;
    if (used >= L.pw) return;
    char* p = (char*)out + (size_t)(((int64_t)(L.np - 1) * L.rows * L.pw + used) * es);
    CK(cudaMemset2DAsync(p, (size_t)(L.pw * es), 0, (size_t)((L.pw - used) * es), (size_t)nrows, D.st));
}

void tc_zero_tail(Dev& D, int prec, void* out, int64_t rows_tot, int64_t K, int64_t nrows) {
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    zero_tail(D, kind, out, make_el(kind, K, rows_tot, 1), K, nrows);
}

// embedding of op(S)[b][r][k] (rows r, K index k); tiled when consecutive rows
// are consecutive in memory and k is not
static void embed_impl(Dev& D, int prec, bool is_b, const cplx* S, int64_t sb, const Lvl& lr, const Lvl& lk, bool cj,
                       int64_t batch, int64_t Rn, int64_t K, int64_t pitch, int64_t rows_tot, void* out) {
    if (batch * Rn * K == 0) return;
    const bool tiled = lr.s == 1 && lk.s != 1;
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const EL L = make_el(kind, K, rows_tot, batch);
    REQUIRE(L.pw == pitch, "embed: pitch does not match the layout");
    zero_tail(D, kind, out, L, K, is_b ? 2 * Rn : Rn);
    const int64_t nt = batch * ((Rn + 31) / 32) * ((K + 31) / 32);
    const int gt = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)D.sm_count * 8));
    const int g = grid_n(D, batch * Rn * K);
    const int c = cj ? 1 : 0;
    const FastDiv fR(Rn), fK(K);
    if (prec == LRCC_MIXED_BF16X3) {
        if (is_b) {
            if (tiled) k_embed_t<0, true><<<gt, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, L, out);
            else k_embed<0, true><<<g, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, fR, fK, L, out);
        } else {
            if (tiled) k_embed_t<0, false><<<gt, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, L, out);
            else k_embed<0, false><<<g, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, fR, fK, L, out);
        }
    } else {
        if (is_b) {
            if (tiled) k_embed_t<1, true><<<gt, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, L, out);
            else k_embed<1, true><<<g, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, fR, fK, L, out);
        } else {
            if (tiled) k_embed_t<1, false><<<gt, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, L, out);
            else k_embed<1, false><<<g, 256, 0, D.st>>>(S, sb, lr, lk, c, batch, Rn, K, fR, fK, L, out);
        }
    }
    LAUNCH_CHECK(D);
}

void tc_embed_a(Dev& D, int prec, const cplx* A, int64_t sAb, int64_t sAm, int64_t sAk, bool cA, int64_t batch,
                int64_t M, int64_t K, int64_t pitch, int64_t rows_tot, void* out) {
    embed_impl(D, prec, false, A, sAb, mk_lvl(sAm), mk_lvl(sAk), cA, batch, M, K, pitch, rows_tot, out);
}

void tc_embed_b(Dev& D, int prec, const cplx* B, int64_t sBb, int64_t sBk, int64_t sBn, bool cB, int64_t batch,
                int64_t K, int64_t N, int64_t pitch, int64_t rows_tot, void* out) {
    embed_impl(D, prec, true, B, sBb, mk_lvl(sBn), mk_lvl(sBk), cB, batch, N, K, pitch, rows_tot, out);
}

// One persistent launch: C = alpha op(A' B'^T) + beta C on embedded operands
// A' [batch][M][pitch], B' [batch][2N][pitch] of which the first kd columns
// take part (kind 0: bf16, 1: tf32); FP32 accumulation chains of at most
// kchunk k-blocks, added to C in FP64.
// Options of one launch: the K range may start at k-block kbase of the
// operands (kd then counts the embedded columns from there), and a tile mask
// (mask_v > 0) skips the tiles whose rows and complex columns all have
// (index mod mask_v) < mask_emin.
struct TcExtra {
    int kbase = 0;
    int mask_v = 0, mask_emin = 0;
    bool f32out = false;  // C is complex FP32 (beta must be 0 or 1)
};

static void tc_launch(Dev& D, int kind, const void* pa, const void* pb, int64_t batch, int64_t M, int64_t N,
                      int64_t kd, int64_t pitch, int64_t rows_a, int64_t rows_b, int np, cplx* C, int64_t sCb,
                      const Lvl& lm, const Lvl& ln, cplx alpha, cplx beta, bool conj_acc, int kchunk,
                      bool exact_alpha, double useful_flops, const char* name, const TcExtra& ex = TcExtra()) {
    REQUIRE(D.err_flag != nullptr, "gemm_tc: no error word");
    if (M <= 0 || N <= 0 || batch <= 0) return;
    const int64_t es = kind == 0 ? 2 : 4, kelem = ROWB / es;
    const int64_t kext = (int64_t)ex.kbase * kelem + kd;  // embedded columns the operands hold up to the range end
    REQUIRE(ex.kbase >= 0 && (ex.kbase == 0 || batch == 1), "gemm_tc: K offset needs batch 1");
    REQUIRE(kd > 0 && (np > 1 || pitch >= kext) && (pitch * es) % 16 == 0 &&
                (np == 1 || (batch == 1 && pitch % kelem == 0 && kext <= (int64_t)np * pitch)),
            "gemm_tc: bad embedded K");
    REQUIRE(((uintptr_t)pa % 16) == 0 && ((uintptr_t)pb % 16) == 0, "gemm_tc: operands not 16-byte aligned");
    const int bn = bn_for(2 * N);
    CUtensorMap ta, tb;
    const uint64_t dx = np > 1 ? (uint64_t)pitch : (uint64_t)kext, dz = np > 1 ? (uint64_t)np : (uint64_t)batch;
    encode(&ta, pa, kind, dx, (uint64_t)pitch, (uint64_t)M, (uint64_t)rows_a, dz, BM);
    encode(&tb, pb, kind, dx, (uint64_t)pitch, (uint64_t)(2 * N), (uint64_t)rows_b, dz, (uint32_t)bn);
    const int64_t tiles_m = (M + BM - 1) / BM, tiles_n = (2 * N + bn - 1) / bn;
    const int64_t tiles = tiles_m * tiles_n * batch;
    REQUIRE(tiles_m < INT32_MAX && tiles_n < INT32_MAX && tiles < ((int64_t)1 << 40), "gemm_tc: too many tiles");
    const int num_kb = (int)((kd + kelem - 1) / kelem);
    // K splits: fewest estimated waves x (k-blocks per unit + per-unit overhead);
    // split units add their partial tiles to C with FP64 atomics
    const int64_t sm = D.sm_count;
    int splits = 1, kps = num_kb;
    double best = 1e300;
    for (int S = 1; S <= (ex.f32out ? 1 : 96); ++S) {
        if (S > 1 && num_kb / S < 8) break;
        const int k1 = (num_kb + S - 1) / S;
        const int se = (num_kb + k1 - 1) / k1;
        if (se != S) continue;
        const int64_t units = tiles * se;
        const double waves = double((units + sm - 1) / sm);
        const int chunks = (k1 + kchunk - 1) / kchunk;
        const double cost = waves * (k1 + 3.0 + (se > 1 ? 4.0 * bn / 256.0 * chunks : 0.0));
        if (cost < best * 0.97) {
            best = cost;
            splits = se;
            kps = k1;
        }
    }
    Sched sc;
    sc.tiles_m = (int)tiles_m;
    sc.tiles_n = (int)tiles_n;
    sc.batch = (int)batch;
    sc.splits = splits;
    sc.kps = kps;
    sc.num_kb = num_kb;
    sc.group = (int)std::min<int64_t>(tiles_m, 16);
    // complex-FP32 output adds its chunks in FP32 anyway: one chain over the whole K
    // (the same rounding as FP32 chunk sums) without a read-modify-write of C per chunk
    sc.kchunk = ex.f32out ? std::max(kchunk, num_kb) : kchunk;
    sc.kpb = np > 1 ? (int)(pitch / kelem) : 0;
    sc.kbase = ex.kbase;
    sc.mv = ex.mask_v;
    sc.memin = ex.mask_emin;
    sc.mrows = M;
    sc.mcols = N;
    sc.units = (long long)tiles * splits;
    REQUIRE(batch < INT32_MAX, "gemm_tc: batch too large");
    REQUIRE(!ex.f32out || ((beta.x == 0.0 || beta.x == 1.0) && beta.y == 0.0), "gemm_tc: FP32 output with beta 0 or 1");
    Epi ep{M, N, C, sCb, lm, ln, alpha, beta, conj_acc ? 1 : 0, splits > 1 ? 1 : 0, exact_alpha ? 1 : 0,
           ex.f32out ? 1 : 0};
    if (splits > 1) {
        GemmArgs pg{};
        pg.M = M; pg.N = N; pg.batch = batch; pg.C = C; pg.sCb = sCb; pg.sCm = lm.s; pg.sCn = ln.s; pg.beta = beta;
        pg.dCm2 = lm.two ? lm.f2.d : 0; pg.sCm1 = lm.s1; pg.dCn2 = ln.two ? ln.f2.d : 0; pg.sCn1 = ln.s1;
        gemm_prescale(D, pg);
    }
    // host-side fault injection for the failure-detection test: the producer
    // skips its TMA issues so the consumers' bounded waits expire (short limit)
    const char* inj = getenv("LRCC_INJECT_TMA_SKIP");
    const int skip = (inj && inj[0] == '1') ? 1 : 0;
    const uint32_t limit = skip ? WAIT_LIMIT_INJECT : WAIT_LIMIT;
    const int grid = (int)std::min<int64_t>(sc.units, sm);
    KTimer kt(D, name, useful_flops, (double)(batch * (M + 2 * N) * kd * es) + 16.0 * M * N * batch, M, N, kd,
              batch);
    switch (kind * 4 + (bn == 256 ? 0 : bn == 128 ? 1 : bn == 64 ? 2 : 3)) {
        case 0: launch_tc<0, 256>(D, ta, tb, sc, ep, grid, skip, limit); break;
        case 1: launch_tc<0, 128>(D, ta, tb, sc, ep, grid, skip, limit); break;
        case 2: launch_tc<0, 64>(D, ta, tb, sc, ep, grid, skip, limit); break;
        case 3: launch_tc<0, 32>(D, ta, tb, sc, ep, grid, skip, limit); break;
        case 4: launch_tc<1, 256>(D, ta, tb, sc, ep, grid, skip, limit); break;
        case 5: launch_tc<1, 128>(D, ta, tb, sc, ep, grid, skip, limit); break;
        case 6: launch_tc<1, 64>(D, ta, tb, sc, ep, grid, skip, limit); break;
        default: launch_tc<1, 32>(D, ta, tb, sc, ep, grid, skip, limit); break;
    }
    LAUNCH_CHECK(D);
}

// C = alpha * op(A' B'^T) + beta C on embedded operands A' [batch][M][pitch],
// B' [batch][2N][pitch], complex K (S*K embedded columns)
void tc_gemm_embedded(Dev& D, int prec, const void* pa, const void* pb, int64_t batch, int64_t M, int64_t N,
                      int64_t K, int64_t pitch, int64_t rows_a, int64_t rows_b, cplx* C, int64_t sCb, int64_t sCm,
                      int64_t sCn, cplx alpha, cplx beta, bool conj_acc, double useful_flops) {
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    REQUIRE(K > 0, "gemm_tc: bad embedded K");
    const EL L = make_el(kind, K, rows_a, batch);
    REQUIRE(L.pw == pitch, "gemm_tc: pitch does not match the layout");
    tc_launch(D, kind, pa, pb, batch, M, N, slots(kind) * K, pitch, rows_a, rows_b, L.np, C, sCb, mk_lvl(sCm),
              mk_lvl(sCn), alpha, beta, conj_acc, KCHUNK, false, useful_flops,
              kind == 0 ? "gemm_tc_bf16x3" : "gemm_tc_tf32");
}

void tc_gemm_embedded_ex(Dev& D, int prec, const void* pa, const void* pb, int64_t M, int64_t N, int64_t K_total,
                         int64_t k0, int64_t pitch, int64_t rows_a, int64_t rows_b, cplx* C, int64_t sCm,
                         int64_t sCn, cplx alpha, cplx beta, bool conj_acc, double useful_flops, int mask_v,
                         int mask_emin, bool f32out) {
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const int64_t es = kind == 0 ? 2 : 4, kelem = ROWB / es, S = slots(kind);
    REQUIRE(K_total > 0 && k0 >= 0 && k0 < K_total && (S * k0) % kelem == 0,
            "gemm_tc: K offset must start a k-block of the embedded operands");
    const EL L = make_el(kind, K_total, rows_a, 1);
    REQUIRE(L.pw == pitch, "gemm_tc: pitch does not match the layout");
    TcExtra ex;
    ex.kbase = (int)(S * k0 / kelem);
    ex.mask_v = mask_v;
    ex.mask_emin = mask_emin;
    ex.f32out = f32out;
    tc_launch(D, kind, pa, pb, 1, M, N, S * (K_total - k0), pitch, rows_a, rows_b, L.np, C, 0, mk_lvl(sCm),
              mk_lvl(sCn), alpha, beta, conj_acc, KCHUNK, false, useful_flops,
              kind == 0 ? "gemm_tc_bf16x3" : "gemm_tc_tf32", ex);
}

int64_t tc_k_align(int prec) {
    // complex K indices at which a k-block of the embedded operands starts:
    // multiples of lcm(slots, k-block) / slots
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const int64_t es = kind == 0 ? 2 : 4, kelem = ROWB / es, S = slots(kind);
    int64_t a = 1;
    while ((S * a) % kelem) ++a;
    return a;
}

// relative cost of running C[M][N] in this orientation: padded tensor-core
// work, with a penalty when the epilogue's lanes (consecutive m) do not write
// consecutive addresses
static double orient_cost(int64_t M, int64_t N, int64_t sCm) {
    const int bn = bn_for(2 * N);
    const double pm = double((M + BM - 1) / BM * BM), pn = double((2 * N + bn - 1) / bn * bn);
    return pm * pn * (sCm == 1 ? 1.0 : 1.15);
}

// ---------------------------------------------------------------------------
// Operand embeddings are transient copies (bf16x3: 12 bytes per complex A
// element, 24 per B element; integer slices: 28 and 56), so a contraction whose
// operands are amplitude-sized at large O, V (4.5 GB per right-hand side at
// O=28, V=600) would need tens of GB for them.  Such a GEMM runs as a sequence
// of sub-GEMMs over halves of N, M or K until the embedded operands of each fit
// in a bounded budget.  A half along a two-level index group (g = g1 d2 + g2)
// is cut at a multiple of d2 when the group has several outer blocks; within a
// single outer block the group is flat with stride s.  The second K half adds
// to C (beta = 1).
// ---------------------------------------------------------------------------
namespace {

// split [0, n) of one index group shared by two operands (x and y) at about
// n/2: returns the first part's size and both operands' offsets of the second
// part, and makes the groups of the second part consistent
bool halve_group(int64_t n, int64_t& d2x, int64_t s1x, int64_t sx, int64_t& d2y, int64_t s1y, int64_t sy,
                 int64_t& n1, int64_t& offx, int64_t& offy, bool& to_flat) {
    if (n < 2) return false;
    if (d2x > 0 && d2y > 0 && d2x != d2y) return false;  // groups cut at different labels
    const int64_t d2 = d2x > 0 ? d2x : d2y;
    to_flat = false;
    if (d2 > 0 && n / d2 >= 2) {
        const int64_t q = (n / d2) / 2;
        n1 = q * d2;
        offx = d2x > 0 ? q * s1x : n1 * sx;
        offy = d2y > 0 ? q * s1y : n1 * sy;
    } else {
        n1 = n / 2;
        offx = n1 * sx;
        offy = n1 * sy;
        to_flat = d2 > 0;  // one outer block: a flat group with stride s
    }
    return true;
}

// halves of g along dim 0 (M), 1 (N) or 2 (K)
bool halve_gemm(const GemmArgs& g, int dim, GemmArgs& g1, GemmArgs& g2) {
    g1 = g;
    g2 = g;
    int64_t n1 = 0, ox = 0, oy = 0;
    bool flat = false;
    if (dim == 0) {
        int64_t dx = g.dAm2, dy = g.dCm2;
        if (!halve_group(g.M, dx, g.sAm1, g.sAm, dy, g.sCm1, g.sCm, n1, ox, oy, flat)) return false;
        g1.M = n1;
        g2.M = g.M - n1;
        g2.A = g.A + ox;
        g2.C = g.C + oy;
        if (flat) g1.dAm2 = g2.dAm2 = g1.dCm2 = g2.dCm2 = 0;
    } else if (dim == 1) {
        int64_t dx = g.dBn2, dy = g.dCn2;
        if (!halve_group(g.N, dx, g.sBn1, g.sBn, dy, g.sCn1, g.sCn, n1, ox, oy, flat)) return false;
        g1.N = n1;
        g2.N = g.N - n1;
        g2.B = g.B + ox;
        g2.C = g.C + oy;
        if (flat) g1.dBn2 = g2.dBn2 = g1.dCn2 = g2.dCn2 = 0;
    } else {
        int64_t dx = g.dAk2, dy = g.dBk2;
        if (!halve_group(g.K, dx, g.sAk1, g.sAk, dy, g.sBk1, g.sBk, n1, ox, oy, flat)) return false;
        g1.K = n1;
        g2.K = g.K - n1;
        g2.A = g.A + ox;
        g2.B = g.B + oy;
        g2.beta = mkc(1.0);
        if (flat) g1.dAk2 = g2.dAk2 = g1.dBk2 = g2.dBk2 = 0;
    }
    return true;
}

// the dimension to halve: the largest of M, N, K (K halves both operands)
bool split_gemm(const GemmArgs& g, GemmArgs& g1, GemmArgs& g2) {
    int order[3];
    if (g.K >= std::max(g.M, g.N)) { order[0] = 2; order[1] = g.N >= g.M ? 1 : 0; order[2] = g.N >= g.M ? 0 : 1; }
    else if (g.N >= g.M) { order[0] = 1; order[1] = 2; order[2] = 0; }
    else { order[0] = 0; order[1] = 2; order[2] = 1; }
    for (int d : order)
        if (halve_gemm(g, d, g1, g2)) return true;
    return false;
}

// bytes the embedded operands of one GEMM may take
double embed_budget(Dev& D) {
    if (D.embed_budget > 0) return D.embed_budget;
    return std::min(6.0 * double(1ull << 30), 0.1 * free_bytes(D));
}

}  // namespace

void gemm_tc(Dev& D, const GemmArgs& g0, int prec) {
    if (g0.M <= 0 || g0.N <= 0 || g0.batch <= 0) return;
    if (g0.K > 0) {
        int64_t ra, pa_, rb, pb_;
        const double bytes = double(tc_embed_bytes(prec, g0.M, g0.K, g0.batch, ra, pa_, false)) +
                             double(tc_embed_bytes(prec, g0.N, g0.K, g0.batch, rb, pb_, true));
        GemmArgs g1, g2;
        if (bytes > embed_budget(D) && split_gemm(g0, g1, g2)) {
            gemm_tc(D, g1, prec);
            gemm_tc(D, g2, prec);
            return;
        }
    }
    REQUIRE(prec == LRCC_MIXED_TF32 || prec == LRCC_MIXED_BF16X3, "gemm_tc: bad precision");
    if (g0.K <= 0) {
        REQUIRE(g0.flat(), "gemm_tc: K = 0 with two-level groups");
        gemm_f64(D, g0);  // pure beta scaling
        return;
    }
    // C^T = B^T A^T: run the orientation with less padding / coalesced stores
    GemmArgs g = g0;
    if (orient_cost(g0.N, g0.M, g0.sCn) < orient_cost(g0.M, g0.N, g0.sCm)) {
        g.M = g0.N; g.N = g0.M;
        g.A = g0.B; g.sAb = g0.sBb; g.sAm = g0.sBn; g.sAk = g0.sBk; g.cA = g0.cB;
        g.B = g0.A; g.sBb = g0.sAb; g.sBk = g0.sAk; g.sBn = g0.sAm; g.cB = g0.cA;
        g.sCm = g0.sCn; g.sCn = g0.sCm;
        g.dAm2 = g0.dBn2; g.sAm1 = g0.sBn1; g.dAk2 = g0.dBk2; g.sAk1 = g0.sBk1;
        g.dBk2 = g0.dAk2; g.sBk1 = g0.sAk1; g.dBn2 = g0.dAm2; g.sBn1 = g0.sAm1;
        g.dCm2 = g0.dCn2; g.sCm1 = g0.sCn1; g.dCn2 = g0.dCm2; g.sCn1 = g0.sCm1;
    }
    REQUIRE(std::max(g.M, g.N) < FAST_INDEX_LIMIT && g.K < FAST_INDEX_LIMIT, "gemm_tc: index groups too large");
    int64_t rowsA, pitch, rowsB, pitch2;
    size_t bytesA = tc_embed_bytes(prec, g.M, g.K, g.batch, rowsA, pitch, false);
    size_t bytesB = tc_embed_bytes(prec, g.N, g.K, g.batch, rowsB, pitch2, true);
    void* pa = D.pool.get(bytesA);
    std::shared_ptr<DevBuf> ha(new DevBuf{&D.pool, pa, bytesA});
    void* pb = D.pool.get(bytesB);
    std::shared_ptr<DevBuf> hb(new DevBuf{&D.pool, pb, bytesB});
    embed_impl(D, prec, false, g.A, g.sAb, mk_lvl(g.sAm, g.dAm2, g.sAm1), mk_lvl(g.sAk, g.dAk2, g.sAk1), g.cA,
               g.batch, g.M, g.K, pitch, rowsA, pa);
    embed_impl(D, prec, true, g.B, g.sBb, mk_lvl(g.sBn, g.dBn2, g.sBn1), mk_lvl(g.sBk, g.dBk2, g.sBk1), g.cB,
               g.batch, g.N, g.K, pitch, rowsB, pb);
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const EL L = make_el(kind, g.K, rowsA, g.batch);
    tc_launch(D, kind, pa, pb, g.batch, g.M, g.N, slots(kind) * g.K, pitch, rowsA, rowsB, L.np, g.C, g.sCb,
              mk_lvl(g.sCm, g.dCm2, g.sCm1), mk_lvl(g.sCn, g.dCn2, g.sCn1), g.alpha, g.beta, false, KCHUNK, false,
              8.0 * g.M * g.N * g.K * g.batch, kind == 0 ? "gemm_tc_bf16x3" : "gemm_tc_tf32");
}

void tc_embed_antisym_slab(Dev& D, int prec, const cplx* GT, int64_t ldt, int64_t a0, int64_t gb0, int64_t prow0,
                           int64_t nrows, int64_t V, int64_t pitch, int64_t rows_tot, void* out, int64_t emin,
                           int64_t cmin, bool gt_f32) {
    const int64_t T = (V + 31) / 32, tasks = nrows * T * (T + 1) / 2;
    if (tasks <= 0) return;
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const EL L = make_el(kind, V * (V - 1) / 2, rows_tot, 1);
    REQUIRE(L.pw == pitch, "ladder: pitch does not match the layout");
    const int grid = (int)std::min<int64_t>(tasks, (int64_t)D.sm_count * 8);
    const float2* GF = (const float2*)GT;
    if (prec == LRCC_MIXED_BF16X3) {
        if (gt_f32) k_embed_antisym<0, float2><<<grid, 256, 0, D.st>>>(GF, ldt, a0, gb0, prow0, nrows, V, L, out, emin, cmin);
        else k_embed_antisym<0, cplx><<<grid, 256, 0, D.st>>>(GT, ldt, a0, gb0, prow0, nrows, V, L, out, emin, cmin);
    } else {
        if (gt_f32) k_embed_antisym<1, float2><<<grid, 256, 0, D.st>>>(GF, ldt, a0, gb0, prow0, nrows, V, L, out, emin, cmin);
        else k_embed_antisym<1, cplx><<<grid, 256, 0, D.st>>>(GT, ldt, a0, gb0, prow0, nrows, V, L, out, emin, cmin);
    }
    LAUNCH_CHECK(D);
}

void tc_transpose_conj_a(Dev& D, int prec, const void* src, int64_t K_src, int64_t rows_src, int64_t nr, int64_t c0,
                         int64_t nc, void* dst, int64_t rows_dst) {
    if (nr <= 0 || nc <= 0) return;
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const EL Ls = make_el(kind, K_src, rows_src, 1), Ld = make_el(kind, nr, rows_dst, 1);
    const int64_t tiles = ((nr + 31) / 32) * ((nc + 31) / 32);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)D.sm_count * 8));
    if (kind == 0) k_transpose_conj_a<0><<<grid, 256, 0, D.st>>>(src, Ls, nr, c0, nc, dst, Ld);
    else k_transpose_conj_a<1><<<grid, 256, 0, D.st>>>(src, Ls, nr, c0, nc, dst, Ld);
    LAUNCH_CHECK(D);
}

void tc_zero_cols_a(Dev& D, int prec, void* out, int64_t K, int64_t rows_tot, int64_t nr, int64_t c_lo,
                    int64_t c_hi) {
    if (nr <= 0 || c_hi <= c_lo) return;
    const int kind = prec == LRCC_MIXED_BF16X3 ? 0 : 1;
    const EL L = make_el(kind, K, rows_tot, 1);
    const int grid = grid_n(D, nr * (c_hi - c_lo));
    if (kind == 0) k_zero_cols_a<0><<<grid, 256, 0, D.st>>>(out, L, nr, c_lo, c_hi);
    else k_zero_cols_a<1><<<grid, 256, 0, D.st>>>(out, L, nr, c_lo, c_hi);
    LAUNCH_CHECK(D);
}

// ---------------------------------------------------------------------------
// FP64-class complex GEMM on the tensor cores (host side of the slicing
// scheme above)
// ---------------------------------------------------------------------------
size_t oz_embed_bytes(int64_t rows, int64_t K, int64_t batch, int64_t& rows_e, int64_t& kpad, bool is_b) {
    kpad = (2 * K + 7) / 8 * 8;
    rows_e = is_b ? 2 * rows : rows;
    return (size_t)(batch * rows_e * OZ_S * kpad * 2);
}

// exponents and slices of op(S)[b][r][k] (strides sb, sr, sk): e [batch*Rn]
static void oz_embed(Dev& D, bool is_b, const cplx* S, int64_t sb, int64_t sr, int64_t sk, bool cj, int64_t batch,
                     int64_t Rn, int64_t K, int64_t kpad, int* e, void* out) {
    if (batch * Rn == 0) return;
    const bool rows_contig = sr == 1 && sk != 1;
    const int64_t rows = batch * Rn;
    if (rows_contig) {
        k_row_exp_t<<<(int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, D.sm_count * 16)), 256, 0,
                      D.st>>>(S, sb, sr, sk, batch, Rn, K, e);
    } else {
        k_row_exp_w<<<(int)std::max<int64_t>(1, std::min<int64_t>((rows * 32 + 255) / 256, D.sm_count * 16)), 256,
                      0, D.st>>>(S, sb, sr, sk, batch, Rn, K, e);
    }
    LAUNCH_CHECK(D);
    const int64_t K2 = kpad / 2, rows_e = is_b ? 2 * Rn : Rn;
    if (rows_contig) {
        const int64_t nt = batch * ((Rn + 31) / 32) * ((K2 + 31) / 32);
        const int gt = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)D.sm_count * 8));
        if (is_b) k_oz_embed_t<true><<<gt, 256, 0, D.st>>>(S, sb, sk, cj, batch, Rn, K, K2, e, rows_e, kpad, out);
        else k_oz_embed_t<false><<<gt, 256, 0, D.st>>>(S, sb, sk, cj, batch, Rn, K, K2, e, rows_e, kpad, out);
    } else {
        const int g = grid_n(D, batch * Rn * K2);
        if (is_b)
            k_oz_embed<true><<<g, 256, 0, D.st>>>(S, sb, sr, sk, cj, batch, Rn, K, K2, FastDiv(Rn), FastDiv(K2), e,
                                                  rows_e, kpad, out);
        else
            k_oz_embed<false><<<g, 256, 0, D.st>>>(S, sb, sr, sk, cj, batch, Rn, K, K2, FastDiv(Rn), FastDiv(K2), e,
                                                   rows_e, kpad, out);
    }
    LAUNCH_CHECK(D);
}

void oz_embed_a(Dev& D, const cplx* A, int64_t sAb, int64_t sAm, int64_t sAk, bool cA, int64_t batch, int64_t M,
                int64_t K, int64_t kpad, void* out) {
    int* e = (int*)D.pool.get(sizeof(int) * batch * M);
    std::shared_ptr<DevBuf> he(new DevBuf{&D.pool, e, sizeof(int) * (size_t)(batch * M)});
    oz_embed(D, false, A, sAb, sAm, sAk, cA, batch, M, K, kpad, e, out);
}

void oz_embed_b(Dev& D, const cplx* B, int64_t sBb, int64_t sBk, int64_t sBn, bool cB, int64_t batch, int64_t K,
                int64_t N, int64_t kpad, void* out) {
    int* e = (int*)D.pool.get(sizeof(int) * batch * N);
    std::shared_ptr<DevBuf> he(new DevBuf{&D.pool, e, sizeof(int) * (size_t)(batch * N)});
    oz_embed(D, true, B, sBb, sBn, sBk, cB, batch, N, K, kpad, e, out);
}

// C = alpha op(A B) + beta C from sliced operands: one launch per diagonal
// d = s + t, over the concatenated K of the pairs (A_0..A_d) x (B_d..B_0)
void oz_gemm_embedded(Dev& D, const void* pa, const void* pb, int64_t batch, int64_t M, int64_t N, int64_t K,
                      int64_t kpad, cplx* C, int64_t sCb, int64_t sCm, int64_t sCn, cplx alpha, cplx beta,
                      bool conj_acc) {
    const double useful = 8.0 * M * N * K * batch, pairs = OZ_S * (OZ_S + 1) / 2.0;
    for (int d = 0; d < OZ_S; ++d) {
        const char* pbd = (const char*)pb + (size_t)((OZ_S - 1 - d) * kpad * 2);
        tc_launch(D, 0, pa, pbd, batch, M, N, (d + 1) * kpad, OZ_S * kpad, M, 2 * N, 1, C, sCb, mk_lvl(sCm),
                  mk_lvl(sCn), alpha,
                  d == 0 ? beta : mkc(1.0), conj_acc, OZ_KCHUNK, true, useful * (d + 1) / pairs, "gemm_tc_f64emu");
    }
}

void gemm_tc_f64(Dev& D, const GemmArgs& g0) {
    if (g0.M <= 0 || g0.N <= 0 || g0.batch <= 0) return;
    REQUIRE(g0.flat(), "gemm_tc_f64: two-level index groups are not supported");
    if (g0.K > 0) {
        int64_t ra, ka, rb, kb;
        const double bytes = double(oz_embed_bytes(g0.M, g0.K, g0.batch, ra, ka, false)) +
                             double(oz_embed_bytes(g0.N, g0.K, g0.batch, rb, kb, true));
        GemmArgs g1, g2;
        if (bytes > embed_budget(D) && split_gemm(g0, g1, g2)) {
            gemm_tc_f64(D, g1);
            gemm_tc_f64(D, g2);
            return;
        }
    }
    if (g0.K <= 0) {
        gemm_f64(D, g0);  // pure beta scaling
        return;
    }
    GemmArgs g = g0;
    if (orient_cost(g0.N, g0.M, g0.sCn) < orient_cost(g0.M, g0.N, g0.sCm)) {
        g.M = g0.N; g.N = g0.M;
        g.A = g0.B; g.sAb = g0.sBb; g.sAm = g0.sBn; g.sAk = g0.sBk; g.cA = g0.cB;
        g.B = g0.A; g.sBb = g0.sAb; g.sBk = g0.sAk; g.sBn = g0.sAm; g.cB = g0.cA;
        g.sCm = g0.sCn; g.sCn = g0.sCm;
    }
    int64_t rowsA, kpad, rowsB, kpad2;
    size_t bytesA = oz_embed_bytes(g.M, g.K, g.batch, rowsA, kpad, false);
    size_t bytesB = oz_embed_bytes(g.N, g.K, g.batch, rowsB, kpad2, true);
    void* pa = D.pool.get(bytesA);
    std::shared_ptr<DevBuf> ha(new DevBuf{&D.pool, pa, bytesA});
    void* pb = D.pool.get(bytesB);
    std::shared_ptr<DevBuf> hb(new DevBuf{&D.pool, pb, bytesB});
    oz_embed_a(D, g.A, g.sAb, g.sAm, g.sAk, g.cA, g.batch, g.M, g.K, kpad, pa);
    oz_embed_b(D, g.B, g.sBb, g.sBk, g.sBn, g.cB, g.batch, g.K, g.N, kpad, pb);
    oz_gemm_embedded(D, pa, pb, g.batch, g.M, g.N, g.K, kpad, g.C, g.sCb, g.sCm, g.sCn, g.alpha, g.beta, false);
}

