// tcgen05 (5th-generation tensor core) sketch and mode product, BF16 hi+lo split.
#include "rtr_internal.cuh"

size_t tc_ws_bytes(const rtr_plan* p) { (void)p; return 0; }

int launch_sketch_tc(rtr_plan* p, const float* X, double* const* Y, cudaStream_t s) {
    (void)p; (void)X; (void)Y; (void)s;
    return rtr_set_error(RTR_EUNSUPPORTED, "BF16 tensor-core sketch is not built yet");
}

int launch_ttm_tc(rtr_plan* p, const float* X, int64_t A, int64_t I, int64_t B, const double* Q, int K, float* out,
                  cudaStream_t s) {
    (void)p; (void)X; (void)A; (void)I; (void)B; (void)Q; (void)K; (void)out; (void)s;
    return rtr_set_error(RTR_EUNSUPPORTED, "BF16 tensor-core mode product is not built yet");
}
