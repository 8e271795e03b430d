// Context of the C ABI (shared by lrcc.cu and fns.cu).
#pragma once
#include "solver.h"

struct lrcc_ctx {
    Dev D;
    lrcc_options opt;
    int O = 0, V = 0, L = 0, ncomp = 0;
    std::vector<double> eps;
    double* eo = nullptr;  // device
    double* ev = nullptr;
    Tensor B, mu;          // [L][N][N], [ncomp][N][N]
    Ham H;
    std::vector<Ham> Hmu;
    LadderCtx lad;
    std::unique_ptr<CCProg> cc;          // two-body program, primal cached at T
    std::vector<std::unique_ptr<CCProg>> ccmu;  // one-body programs (xi, eta)
    std::unique_ptr<CCProg> ccfx;        // scratch program for the F.X stencil
    bool ground = false;
    bool linearized = false;               // cc holds the primal values at a fixed T (ground state or lrcc_linearize)
    bool truncated = false;                // lrcc_fns_truncate ran
    cplx e_mp2_full = {0, 0}, e_mp2_trunc = {0, 0};  // Eq. 51 pieces
    bool ham_built = false;               // integral blocks and programs exist
    Amp T, Lam;                          // R = 1
    std::string err;
    double phase_ms[7] = {0};
    int n_sigma64 = 0, n_sigma_mixed = 0;  // residual-map applications in the last solve
    ~lrcc_ctx() {
        cc.reset();
        ccmu.clear();
        ccfx.reset();
        if (eo) cudaFree(eo);
        if (ev) cudaFree(ev);
        if (D.err_flag) cudaFree(D.err_flag);
        for (auto& r : D.recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
};


// build the integral blocks, the ladder factor and the residual programs for
// the context's current basis (idempotent until the basis changes)
void ensure_ham(lrcc_ctx* c);
