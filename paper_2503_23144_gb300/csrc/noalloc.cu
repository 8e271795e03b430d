// lrcc_ladder_noalloc: the particle-particle ladder (FP64 path) for callers
// that cannot allocate device memory.
//
// Who needs this: code that runs where allocating is not allowed or not
// affordable -- a host framework that hands out every byte of device memory
// through its own allocator and forbids raw cudaMalloc, or a latency-critical
// loop in which cudaMalloc/cudaFree (which synchronise the device) must never
// run.  Those
// callers still own the inputs and the output; what they cannot do is give the
// library the intermediate buffers the ladder needs.  Here those buffers live
// in one fixed array in device global memory, declared below, which every GPU
// that loads this library holds until the process exits.
//
// Scratch use: the packed amplitudes Xp [P_V][R P_O], the packed result
// Zp [P_V][R P_O], one slab of <ab|ef> products G and one antisymmetrised
// slab W.  Every element of these is written before it is read in each call,
// so nothing has to be cleared; but every call uses the same array, so two
// calls whose kernels overlap on the GPU (different streams, or different host
// threads on one device) race on it and both results are undefined.  Serialise
// such calls on one stream.
#include <mutex>

#include "lrcc_internal.h"

// 32 MiB of scratch, the documented limit of lrcc_ladder_noalloc
#define LRCC_NOALLOC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_ladder_scratch[LRCC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};
int g_sm_count[MAX_DEVICES] = {0};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
void* scratch_address(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= MAX_DEVICES) throw LrccError(LRCC_EINVAL, "device index out of range");
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ladder_scratch);
        if (e != cudaSuccess || p == nullptr)
            throw LrccError(LRCC_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        int sm = 0;
        e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) throw LrccError(LRCC_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
        g_sm_count[dev] = sm;
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

}  // namespace

extern "C" lrcc_status lrcc_ladder_noalloc(const double* bvv_dev, int L, int O, int V, int R, const double* x_dev,
                                           double* z_dev, int transpose, void* stream) {
    try {
        REQUIRE(bvv_dev && x_dev && z_dev, "lrcc_ladder_noalloc: null pointer");
        REQUIRE(L >= 1 && O >= 2 && V >= 2 && R >= 1, "lrcc_ladder_noalloc: sizes out of range");
        const int64_t PO = (int64_t)O * (O - 1) / 2, PV = (int64_t)V * (V - 1) / 2;
        const int64_t cap = LRCC_NOALLOC_SCRATCH_BYTES / sizeof(cplx);
        const int64_t packed = PV * R * PO;
        const int64_t per_a = (int64_t)V * (V - 1) * V + (int64_t)(V - 1) * PV;  // G rows + W rows of one a
        const int64_t avail = cap - 2 * packed;
        if (avail < per_a)
            throw LrccError(LRCC_EINVAL,
                            "lrcc_ladder_noalloc: problem needs more than the fixed " +
                                std::to_string(LRCC_NOALLOC_SCRATCH_BYTES >> 20) + " MiB of scratch (need " +
                                std::to_string((2 * packed + per_a) * (int64_t)sizeof(cplx)) + " bytes at least)");
        int dev = 0;
        CK(cudaGetDevice(&dev));
        cplx* base = (cplx*)scratch_address(dev);
        Dev D;  // no pool allocations are made through it
        D.st = (cudaStream_t)stream;
        D.sm_count = g_sm_count[dev];
        const int64_t na = std::min<int64_t>(V - 1, avail / per_a);
        cplx* Xp = base;
        cplx* Zp = Xp + packed;
        cplx* G = Zp + packed;
        cplx* W = G + na * (int64_t)V * (V - 1) * V;
        const cplx* Bvv = (const cplx*)bvv_dev;
        ladder_pack_x(D, (const cplx*)x_dev, Xp, R, O, V);
        for (int64_t a0 = 0; a0 < V - 1; a0 += na) {
            int64_t a1 = std::min<int64_t>(V - 1, a0 + na);
            int64_t nb = V - a0 - 1;
            GemmArgs g1;
            g1.M = (a1 - a0) * V; g1.N = nb * V; g1.K = L; g1.batch = 1;
            g1.A = Bvv + a0 * V; g1.sAb = 0; g1.sAm = 1; g1.sAk = (int64_t)V * V; g1.cA = transpose != 0;
            g1.B = Bvv + (a0 + 1) * V; g1.sBb = 0; g1.sBk = (int64_t)V * V; g1.sBn = 1; g1.cB = transpose != 0;
            g1.C = G; g1.sCb = 0; g1.sCm = nb * V; g1.sCn = 1;
            g1.alpha = mkc(1.0); g1.beta = mkc(0.0);
            gemm_f64(D, g1);
            int64_t row0 = a0 * (2 * (int64_t)V - a0 - 1) / 2, row1 = a1 * (2 * (int64_t)V - a1 - 1) / 2;
            int64_t nrows = row1 - row0;
            ladder_antisym_slab(D, G, nb * V, W, a0, nrows, V);
            GemmArgs g2;
            g2.M = nrows; g2.N = R * PO; g2.K = PV; g2.batch = 1;
            g2.A = W; g2.sAb = 0; g2.sAm = PV; g2.sAk = 1; g2.cA = false;
            g2.B = Xp; g2.sBb = 0; g2.sBk = R * PO; g2.sBn = 1; g2.cB = false;
            g2.C = Zp + row0 * R * PO; g2.sCb = 0; g2.sCm = R * PO; g2.sCn = 1;
            g2.alpha = mkc(1.0); g2.beta = mkc(0.0);
            gemm_f64(D, g2);
        }
        ladder_unpack_z(D, Zp, (cplx*)z_dev, R, O, V);
        return LRCC_OK;
    } catch (const LrccError& e) {
        set_global_error(e.what());
        return e.st;
    } catch (const std::exception& e) {
        set_global_error(e.what());
        return LRCC_ECUDA;
    }
}
