// SIMT mode-n product for the projection chain of Algorithm 1 step 7:
//     out[a, k, b] = sum_i X[a, i, b] * Q[i, k]        (X x_n Q^T)
// in float32 or float64.  A tile is CT consecutive columns (a, b) of the
// (A, I, B) view (a run of b inside one a, or a run of a when B == 1, so that
// loads and stores go along the contiguous index).  Q (float64 in memory) is
// staged in shared memory in the compute type, I in chunks of IC rows.
#include <algorithm>
#include "rtr_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int TKO = 4;    // k per thread
constexpr int TC = 2;     // columns per thread

template <typename T>
__global__ void __launch_bounds__(NT) ttm_kernel(const T* __restrict__ X, int64_t A, int I, int64_t B,
                                                 const double* __restrict__ Q, int K, T* __restrict__ out,
                                                 int NKT, int CT, int IC, int64_t ntiles, int64_t nbt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int KP = NKT * TKO;
    const int xld = CT + 1;
    T* Qs = reinterpret_cast<T*>(smem_raw);     // [IC][KP]
    T* Xs = Qs + (size_t)IC * KP;              // [IC][xld]
    const int tid = threadIdx.x;
    const int NCT = CT / TC;
    const int tc = tid % NCT, tko = tid / NCT;
    const int nic = (I + IC - 1) / IC;

    auto load_q = [&](int i0) {
        const int ic = min(IC, I - i0);
        for (int e = tid; e < IC * KP; e += NT) {
            const int il = e / KP, k = e % KP;
            Qs[e] = (il < ic && k < K) ? (T)Q[(int64_t)(i0 + il) * K + k] : T(0);
        }
    };
    if (nic == 1) load_q(0);

    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int64_t a0, b0;
        int len;
        if (B == 1) { a0 = t * CT; b0 = 0; len = (int)min((int64_t)CT, A - a0); }
        else { a0 = t / nbt; b0 = (t % nbt) * CT; len = (int)min((int64_t)CT, B - b0); }
        T acc[TKO][TC];
#pragma unroll
        for (int o = 0; o < TKO; ++o)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[o][c] = T(0);
        for (int i0 = 0; i0 < I; i0 += IC) {
            const int ic = min(IC, I - i0);
            __syncthreads();
            if (nic > 1) load_q(i0);
            if (B == 1) {
                for (int e = tid; e < ic * CT; e += NT) {
                    const int il = e % ic, cc = e / ic;
                    Xs[il * xld + cc] = (cc < len) ? X[(a0 + cc) * (int64_t)I + i0 + il] : T(0);
                }
            } else {
                for (int e = tid; e < ic * CT; e += NT) {
                    const int cc = e % CT, il = e / CT;
                    Xs[il * xld + cc] = (cc < len) ? X[(a0 * I + i0 + il) * B + b0 + cc] : T(0);
                }
            }
            __syncthreads();
#pragma unroll 4
            for (int il = 0; il < ic; ++il) {
                T qv[TKO], xv[TC];
#pragma unroll
                for (int o = 0; o < TKO; ++o) qv[o] = Qs[il * KP + tko * TKO + o];
#pragma unroll
                for (int c = 0; c < TC; ++c) xv[c] = Xs[il * xld + tc * TC + c];
#pragma unroll
                for (int o = 0; o < TKO; ++o)
#pragma unroll
                    for (int c = 0; c < TC; ++c) acc[o][c] = fma(qv[o], xv[c], acc[o][c]);
            }
        }
#pragma unroll
        for (int o = 0; o < TKO; ++o) {
            const int k = tko * TKO + o;
            if (k >= K) continue;
#pragma unroll
            for (int c = 0; c < TC; ++c) {
                const int cc = tc * TC + c;
                if (cc >= len) continue;
                if (B == 1) out[(a0 + cc) * (int64_t)K + k] = acc[o][c];
                else out[(a0 * K + k) * B + b0 + cc] = acc[o][c];
            }
        }
    }
}

}  // namespace

int launch_ttm(rtr_plan* p, int is_f64, const void* X, int64_t A, int64_t I, int64_t B,
               const double* Q, int K, void* out, cudaStream_t s) {
    if (K < 1 || K > 64) return rtr_set_error(RTR_EINVAL, "mode product width %d out of range", K);
    int nkt = 1;
    while (nkt * TKO < K) nkt *= 2;
    const int CT = NT * TC / nkt;
    const size_t esz = is_f64 ? 8 : 4;
    const int IC = (int)std::min<int64_t>(I, is_f64 ? 128 : 256);
    const size_t smem = esz * ((size_t)IC * nkt * TKO + (size_t)IC * (CT + 1));
    int64_t ntiles, nbt = 1;
    if (B == 1) ntiles = rtr_ceil_div(A, CT);
    else { nbt = rtr_ceil_div(B, CT); ntiles = A * nbt; }
    int occ = 1;
    if (is_f64) {
        RTR_CUDA(cudaFuncSetAttribute(ttm_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RTR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ttm_kernel<double>, NT, smem));
    } else {
        RTR_CUDA(cudaFuncSetAttribute(ttm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RTR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ttm_kernel<float>, NT, smem));
    }
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)std::max(occ, 1) * p->num_sms));
    if (is_f64)
        ttm_kernel<double><<<(unsigned)grid, NT, smem, s>>>((const double*)X, A, (int)I, B, Q, K, (double*)out,
                                                            nkt, CT, IC, ntiles, nbt);
    else
        ttm_kernel<float><<<(unsigned)grid, NT, smem, s>>>((const float*)X, A, (int)I, B, Q, K, (float*)out,
                                                           nkt, CT, IC, ntiles, nbt);
    RTR_LAUNCH_CHECK("ttm_kernel");
    return RTR_OK;
}
