// TR-SVD on the projected tensor (Algorithm 1 step 9, second decomposer).
#include "rtr_internal.cuh"

int run_trsvd(rtr_plan* p, const void* P, double tol, double* const* Z, int* ranks, cudaStream_t s) {
    (void)p; (void)P; (void)tol; (void)Z; (void)ranks; (void)s;
    return rtr_set_error(RTR_EUNSUPPORTED, "TR-SVD kernels are not built yet");
}
