// Optimisation of the sparse matrix B (Algorithm 4.3) -- see infft.h.
#include "internal.h"

using namespace infft;

extern "C" {

infft_status infft_optimize_B(infft_plan_t p, unsigned opts, double* max_col_residual, void* stream) {
    (void)opts; (void)max_col_residual; (void)stream;
    if (!p) { set_error("null plan"); return INFFT_EINVAL; }
    set_error("infft_optimize_B: not built yet");
    return INFFT_EUNSUPPORTED;
}

infft_status infft_get_bopt(infft_plan_t p, void* coeff, void* stream) {
    (void)coeff; (void)stream;
    if (!p) { set_error("null plan"); return INFFT_EINVAL; }
    set_error("no B_opt");
    return INFFT_ESTATE;
}

}  // extern "C"
