// Tensor-core (tcgen05) split-precision contraction path.
#include "acse_internal.h"

int tc_plan_create(acse_ctx* c) { (void)c; return ACSE_ERR_UNSUPPORTED; }
void tc_plan_destroy(acse_ctx* c) { (void)c; }
int tc_contract(acse_ctx* c, const double* const D[3], const double* const W[3], int prep_D) {
    (void)c; (void)D; (void)W; (void)prep_D;
    return ACSE_ERR_UNSUPPORTED;
}
