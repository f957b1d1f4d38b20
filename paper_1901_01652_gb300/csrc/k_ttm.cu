// SIMT mode-n product for the projection chain of Algorithm 1 step 7:
//     out[a, k, b] = sum_i X[a, i, b] * Q[i, k]        (X x_n Q^T)
// in float32 or float64.  A tile is CT consecutive columns (a, b) of the
// (A, I, B) view (a run of b inside one a, or a run of a when B == 1, so that
// loads and stores go along the contiguous index).  When 1 < B < CT a tile
// holds floor(CT / B) whole a-blocks instead (column cc -> a = cc / B,
// b = cc % B from a table in shared memory), so that short fibres (B = 25 in
// the middle of a chain) do not leave most of the tile empty.  Q (float64 in
// memory) is staged in shared memory in the compute type, I in chunks of IC rows.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include "rtr_internal.cuh"

namespace {

constexpr int NT = 256;

// TKO: output rows k per thread, TC: columns per thread (the tile variants
// the autotuner chooses between)
template <typename T, int TKO, int TC>
__global__ void __launch_bounds__(NT) ttm_kernel(const T* __restrict__ X, int64_t A, int I, int64_t B,
                                                 const double* __restrict__ Q, int K, T* __restrict__ out,
                                                 int NKT, int CT, int IC, int64_t ntiles, int64_t nbt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int KP = NKT * TKO;
    // X tile row pitch: odd for the scalar variants (conflict-free transposed
    // stores), a multiple of 4 for the 4-wide variants (16-byte vector loads)
    const int xld = (TC % 4 == 0) ? CT + 4 : CT + 1;
    T* Qs = reinterpret_cast<T*>(smem_raw);     // [IC][KP]
    T* Xs = Qs + (size_t)IC * KP;              // [IC][xld]
    int* cmap = reinterpret_cast<int*>(Xs + (size_t)IC * xld);   // [CT] (a << 16) | b, short fibres
    const int tid = threadIdx.x;
    const bool blocks = B > 1 && B < CT;        // tile = whole a-blocks
    const int nab = blocks ? CT / (int)B : 0;
    if (blocks)
        for (int cc = tid; cc < CT; cc += NT) cmap[cc] = ((cc / (int)B) << 16) | (cc % (int)B);
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
        else if (blocks) { a0 = t * nab; b0 = 0; len = (int)(min((int64_t)nab, A - a0) * B); }
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
            } else if (blocks) {
                for (int e = tid; e < ic * CT; e += NT) {
                    const int cc = e % CT, il = e / CT;
                    T v = T(0);
                    if (cc < len) {
                        const int m = cmap[cc];
                        v = X[((a0 + (m >> 16)) * I + i0 + il) * B + (m & 0xFFFF)];
                    }
                    Xs[il * xld + cc] = v;
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
                if constexpr (sizeof(T) == 4 && TKO % 4 == 0 && TC % 4 == 0) {
                    // 16-byte shared loads: KP and xld are multiples of 4 floats
#pragma unroll
                    for (int o = 0; o < TKO; o += 4)
                        *reinterpret_cast<float4*>(&qv[o]) = *reinterpret_cast<const float4*>(&Qs[il * KP + tko * TKO + o]);
#pragma unroll
                    for (int c = 0; c < TC; c += 4)
                        *reinterpret_cast<float4*>(&xv[c]) = *reinterpret_cast<const float4*>(&Xs[il * xld + tc * TC + c]);
                } else {
#pragma unroll
                    for (int o = 0; o < TKO; ++o) qv[o] = Qs[il * KP + tko * TKO + o];
#pragma unroll
                    for (int c = 0; c < TC; ++c) xv[c] = Xs[il * xld + tc * TC + c];
                }
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
                else if (blocks) {
                    const int m = cmap[cc];
                    out[((a0 + (m >> 16)) * K + k) * B + (m & 0xFFFF)] = acc[o][c];
                } else out[(a0 * K + k) * B + b0 + cc] = acc[o][c];
            }
        }
    }
}

template <typename T, int TKO, int TC>
int launch_variant(rtr_plan* p, const T* X, int64_t A, int64_t I, int64_t B, const double* Q, int K, T* out,
                   cudaStream_t s) {
    int nkt = 1;
    while (nkt * TKO < K) nkt *= 2;
    const int CT = NT * TC / nkt;
    if (CT < TC) return rtr_set_error(RTR_EINVAL, "mode product tile does not fit");
    // I chunk: at most 128 (float64) / 256 (float32) rows, and the staged Q
    // and X chunks within 100 KB so that two CTAs fit on an SM
    const int xld = (TC % 4 == 0) ? CT + 4 : CT + 1;
    const int64_t fit = (int64_t)(100 * 1024) / (int64_t)(sizeof(T) * (nkt * TKO + xld));
    const int IC = (int)std::max<int64_t>(1, std::min<int64_t>({I, sizeof(T) == 8 ? 128 : 256, fit}));
    const size_t smem = sizeof(T) * ((size_t)IC * nkt * TKO + (size_t)IC * xld) + sizeof(int) * (size_t)CT;
    int64_t ntiles, nbt = 1;
    if (B == 1) ntiles = rtr_ceil_div(A, CT);
    else if (B < CT) ntiles = rtr_ceil_div(A, CT / B);      // whole a-blocks per tile
    else { nbt = rtr_ceil_div(B, CT); ntiles = A * nbt; }
    auto kern = ttm_kernel<T, TKO, TC>;
    RTR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 1;
    RTR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)std::max(occ, 1) * p->num_sms));
    kern<<<(unsigned)grid, NT, smem, s>>>(X, A, (int)I, B, Q, K, out, nkt, CT, IC, ntiles, nbt);
    RTR_LAUNCH_CHECK("ttm_kernel");
    return RTR_OK;
}

template <typename T>
int run_variant(int v, rtr_plan* p, const T* X, int64_t A, int64_t I, int64_t B, const double* Q, int K, T* out,
                cudaStream_t s) {
    switch (v) {
        case 0: return launch_variant<T, 4, 2>(p, X, A, I, B, Q, K, out, s);
        case 1: return launch_variant<T, 2, 4>(p, X, A, I, B, Q, K, out, s);
        case 2: return launch_variant<T, 4, 4>(p, X, A, I, B, Q, K, out, s);
        case 3: return launch_variant<T, 8, 2>(p, X, A, I, B, Q, K, out, s);
        default: return launch_variant<T, 8, 4>(p, X, A, I, B, Q, K, out, s);
    }
}
constexpr int NVARIANTS = 5;

// Autotuner: the first product of a shape class (type, I, K, layout of B)
// outside stream capture times every tile variant on the call's own data
// (CUDA events, synchronous) and caches the fastest; later calls, and calls
// made while the stream is being captured, use the cache (variant 0 if the
// class has not been tuned yet).
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int, int>, int> g_tune;

template <typename T>
int tuned_ttm(rtr_plan* p, const T* X, int64_t A, int64_t I, int64_t B, const double* Q, int K, T* out,
              cudaStream_t s) {
    const auto key = std::make_tuple((int)sizeof(T), I, K, B == 1 ? 0 : (B < 64 ? 1 : 2));
    int v = -1;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) v = it->second;
    }
    if (v < 0) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        RTR_CUDA(cudaStreamIsCapturing(s, &cap));
        if (cap != cudaStreamCaptureStatusNone || (double)A * I * B < 1e6) {
            v = 0;   // not tuned: capturing, or too small for timing to matter
        } else {
            cudaEvent_t e0, e1;
            RTR_CUDA(cudaEventCreate(&e0));
            RTR_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            int bestv = 0;
            for (int c = 0; c < NVARIANTS; ++c) {
                int st = run_variant<T>(c, p, X, A, I, B, Q, K, out, s);      // warm-up
                if (st) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
                RTR_CUDA(cudaEventRecord(e0, s));
                st = run_variant<T>(c, p, X, A, I, B, Q, K, out, s);
                RTR_CUDA(cudaEventRecord(e1, s));
                RTR_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                RTR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; bestv = c; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            v = bestv;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune[key] = v;
        }
    }
    return run_variant<T>(v, p, X, A, I, B, Q, K, out, s);
}

}  // namespace

int launch_ttm(rtr_plan* p, int is_f64, const void* X, int64_t A, int64_t I, int64_t B,
               const double* Q, int K, void* out, cudaStream_t s) {
    if (K < 1 || K > 64) return rtr_set_error(RTR_EINVAL, "mode product width %d out of range", K);
    if (is_f64) return tuned_ttm<double>(p, (const double*)X, A, I, B, Q, K, (double*)out, s);
    return tuned_ttm<float>(p, (const float*)X, A, I, B, Q, K, (float*)out, s);
}

// the tile variant chosen for a shape class (-1 if not tuned), for tests
int ttm_tuned_variant(int elem_size, int64_t I, int K, int bclass) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(elem_size, I, K, bclass));
    return it == g_tune.end() ? -1 : it->second;
}
