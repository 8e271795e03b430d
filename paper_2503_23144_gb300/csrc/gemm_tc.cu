// Tensor-core split-precision complex GEMM (tcgen05 / TMEM / TMA).
#include "lrcc_internal.h"

bool gemm_tc_available() { return false; }

void gemm_tc(Dev& D, const GemmArgs& g, int prec) {
    (void)prec;
    gemm_f64(D, g);
}
