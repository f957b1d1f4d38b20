// SIMT mode-n product for the projection chain of Algorithm 1 step 7:
//     out[a, k, b] = sum_i X[a, i, b] * Q[i, k]        (X x_n Q^T)
// in float32 or float64.  A tile is CT consecutive columns (a, b) of the
// (A, I, B) view (a run of b inside one a, or a run of a when B == 1, so that
// loads and stores go along the contiguous index).  When 1 < B < CT a tile
// holds floor(CT / B) whole a-blocks instead (column cc -> a = cc / B,
// b = cc % B from a table in shared memory), so that short fibres do not
// leave most of the tile empty.
// Q is converted once per launch to the compute type, its rows zero-padded
// to a 16-byte pitch (qconv_kernel), and is resident in shared memory when it fits;
// otherwise it is streamed in IC-row chunks next to X.  X chunks (IC rows x
// CT columns) are fetched with cp.async into two buffers, so the loads of the
// next chunk (of this tile, or of the CTA's next tile) are in flight while the
// current one is multiplied: without that overlap the product is bound by
// load latency, far below the HBM rate.  Columns and rows outside the tensor
// are zero-filled by the copy itself (source size 0).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include "rtr_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr size_t TTM_SMEM_BUDGET = 100 * 1024;   // two CTAs per SM
constexpr size_t TTM_QRES_MAX = 48 * 1024;       // resident Q up to this size

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// cp.async of one element (4 or 8 bytes); bytes = 0 writes zeros
template <int SZ>
__device__ __forceinline__ void cp_async_elem(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(SZ), "r"(bytes) : "memory");
}
// cp.async of 16 bytes (both addresses 16-byte aligned); bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Qc[i * ld + k] = Q[i * K + k] (k < K), 0 for K <= k < ld
template <typename T>
__global__ void qconv_kernel(const double* __restrict__ Q, int I, int K, int ld, T* __restrict__ Qc) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I * ld; e += gridDim.x * blockDim.x) {
        const int i = e / ld, k = e % ld;
        Qc[e] = k < K ? (T)Q[(int64_t)i * K + k] : T(0);
    }
}

template <typename T>
struct TtmArgs {
    const T* X;
    int64_t A, B;
    int I, K;
    const T* Qc;          // I x qld, compute type (columns >= K zero)
    T* out;
    int NKT, CT, IC, xld, qld;
    int qres;             // 1: all of Q resident (IC may still be < I)
    int vec;              // 1: b-run rows start 16-byte aligned and B is a multiple of 16 bytes
    int64_t ntiles, nbt;
};

// TKO: output rows k per thread, TC: columns per thread (the tile variants
// the autotuner chooses between)
template <typename T, int TKO, int TC>
__global__ void __launch_bounds__(NT) ttm_kernel(const TtmArgs<T> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int I = p.I, IC = p.IC, CT = p.CT, xld = p.xld, qld = p.qld;
    const int64_t A = p.A, B = p.B;
    const int nic = (I + IC - 1) / IC;
    // shared layout: Q (I x qld resident, or 2 x IC x qld chunks), 2 x X chunks, column map
    T* Qs = reinterpret_cast<T*>(smem_raw);
    const size_t qelems = p.qres ? (size_t)I * qld : 2 * (size_t)IC * qld;
    T* Xs = Qs + qelems;
    int* cmap = reinterpret_cast<int*>(Xs + 2 * (size_t)IC * xld);
    const int tid = threadIdx.x;
    const bool blocks = B > 1 && B < CT;
    const int nab = blocks ? CT / (int)B : 0;
    if (blocks)
        for (int cc = tid; cc < CT; cc += NT) cmap[cc] = ((cc / (int)B) << 16) | (cc % (int)B);
    const int NCT = CT / TC;
    const int tc = tid % NCT, tko = tid / NCT;
    const int64_t ntl = (blockIdx.x < p.ntiles) ? (p.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nst = ntl * nic;
    if (blocks) __syncthreads();

    struct Tile { int64_t a0, b0; int len; };
    auto tile_of = [&](int64_t j) {
        const int64_t t = blockIdx.x + j * gridDim.x;
        Tile tl;
        if (B == 1) { tl.a0 = t * CT; tl.b0 = 0; tl.len = (int)min((int64_t)CT, A - tl.a0); }
        else if (blocks) { tl.a0 = t * nab; tl.b0 = 0; tl.len = (int)(min((int64_t)nab, A - tl.a0) * B); }
        else { tl.a0 = t / p.nbt; tl.b0 = (t % p.nbt) * CT; tl.len = (int)min((int64_t)CT, B - tl.b0); }
        return tl;
    };
    // issue the copies of stage s (tile j = s / nic, chunk c = s % nic) into buffer buf
    auto issue = [&](int64_t s, int buf) {
        const int64_t j = s / nic;
        const int c = (int)(s - j * nic);
        const Tile tl = tile_of(j);
        const int i0 = c * IC, ic = min(IC, I - i0);
        const uint32_t xb = smem_addr(Xs + (size_t)buf * IC * xld);
        if (B == 1) {
            // contiguous along i: consecutive threads take consecutive rows
            for (int e = tid; e < IC * CT; e += NT) {
                const int il = e % IC, cc = e / IC;
                const bool ok = il < ic && cc < tl.len;
                const T* src = ok ? p.X + (tl.a0 + cc) * (int64_t)I + i0 + il : p.X;
                cp_async_elem<sizeof(T)>(xb + (uint32_t)(il * xld + cc) * sizeof(T), src, ok ? (int)sizeof(T) : 0);
            }
        } else if (blocks) {
            for (int e = tid; e < IC * CT; e += NT) {
                const int cc = e % CT, il = e / CT;
                const bool ok = il < ic && cc < tl.len;
                const T* src = p.X;
                if (ok) {
                    const int m = cmap[cc];
                    src = p.X + ((tl.a0 + (m >> 16)) * I + i0 + il) * B + (m & 0xFFFF);
                }
                cp_async_elem<sizeof(T)>(xb + (uint32_t)(il * xld + cc) * sizeof(T), src, ok ? (int)sizeof(T) : 0);
            }
        } else if (p.vec) {
            constexpr int VE = 16 / sizeof(T);
            const int nv = CT / VE;
            for (int e = tid; e < IC * nv; e += NT) {
                const int il = e / nv, cc = (e % nv) * VE;
                const bool ok = il < ic && cc < tl.len;
                const T* src = ok ? p.X + (tl.a0 * I + i0 + il) * B + tl.b0 + cc : p.X;
                cp_async16(xb + (uint32_t)(il * xld + cc) * sizeof(T), src, ok ? 16 : 0);
            }
        } else {
            for (int e = tid; e < IC * CT; e += NT) {
                const int cc = e % CT, il = e / CT;
                const bool ok = il < ic && cc < tl.len;
                const T* src = ok ? p.X + (tl.a0 * I + i0 + il) * B + tl.b0 + cc : p.X;
                cp_async_elem<sizeof(T)>(xb + (uint32_t)(il * xld + cc) * sizeof(T), src, ok ? (int)sizeof(T) : 0);
            }
        }
        if (!p.qres) {
            const uint32_t qb = smem_addr(Qs + (size_t)buf * IC * qld);
            constexpr int VE = 16 / sizeof(T);
            const int nv = qld / VE;
            for (int e = tid; e < IC * nv; e += NT) {
                const int il = e / nv, k = (e % nv) * VE;
                const bool ok = il < ic;
                cp_async16(qb + (uint32_t)(il * qld + k) * sizeof(T), ok ? p.Qc + (int64_t)(i0 + il) * qld + k : p.Qc,
                           ok ? 16 : 0);
            }
        }
        cp_async_commit();
    };

    if (nst > 0) {
        if (p.qres) {
            constexpr int VE = 16 / sizeof(T);
            const uint32_t qb = smem_addr(Qs);
            for (int e = tid; e < I * qld / VE; e += NT) cp_async16(qb + (uint32_t)e * 16u, p.Qc + (int64_t)e * VE, 16);
        }
        issue(0, 0);                 // Q (if resident) travels in the first group
    }
    T acc[TKO][TC];
#pragma unroll
    for (int o = 0; o < TKO; ++o)
#pragma unroll
        for (int c = 0; c < TC; ++c) acc[o][c] = T(0);
    for (int64_t s = 0; s < nst; ++s) {
        const int buf = (int)(s & 1);
        if (s + 1 < nst) issue(s + 1, buf ^ 1);
        else cp_async_commit();      // empty group keeps the wait count uniform
        cp_async_wait1();
        __syncthreads();
        const int64_t j = s / nic;
        const int c = (int)(s - j * nic);
        const int i0 = c * IC, ic = min(IC, I - i0);
        const T* Qb = p.qres ? Qs + (size_t)i0 * qld : Qs + (size_t)buf * IC * qld;
        const T* Xb = Xs + (size_t)buf * IC * xld;
#pragma unroll 4
        for (int il = 0; il < ic; ++il) {
            T qv[TKO], xv[TC];
            if constexpr (sizeof(T) == 4 && TKO % 4 == 0 && TC % 4 == 0) {
                // 16-byte shared loads: qld and xld are multiples of 4 floats
#pragma unroll
                for (int o = 0; o < TKO; o += 4)
                    *reinterpret_cast<float4*>(&qv[o]) = *reinterpret_cast<const float4*>(&Qb[il * qld + tko * TKO + o]);
#pragma unroll
                for (int cc = 0; cc < TC; cc += 4)
                    *reinterpret_cast<float4*>(&xv[cc]) = *reinterpret_cast<const float4*>(&Xb[il * xld + tc * TC + cc]);
            } else {
#pragma unroll
                for (int o = 0; o < TKO; ++o) qv[o] = Qb[il * qld + tko * TKO + o];
#pragma unroll
                for (int cc = 0; cc < TC; ++cc) xv[cc] = Xb[il * xld + tc * TC + cc];
            }
#pragma unroll
            for (int o = 0; o < TKO; ++o)
#pragma unroll
                for (int cc = 0; cc < TC; ++cc) acc[o][cc] = fma(qv[o], xv[cc], acc[o][cc]);
        }
        if (c == nic - 1) {
            const Tile tl = tile_of(j);
#pragma unroll
            for (int o = 0; o < TKO; ++o) {
                const int k = tko * TKO + o;
#pragma unroll
                for (int cc0 = 0; cc0 < TC; ++cc0) {
                    const int cc = tc * TC + cc0;
                    if (k < p.K && cc < tl.len) {
                        if (B == 1) p.out[(tl.a0 + cc) * (int64_t)p.K + k] = acc[o][cc0];
                        else if (blocks) {
                            const int m = cmap[cc];
                            p.out[((tl.a0 + (m >> 16)) * p.K + k) * B + (m & 0xFFFF)] = acc[o][cc0];
                        } else p.out[(tl.a0 * p.K + k) * B + tl.b0 + cc] = acc[o][cc0];
                    }
                    acc[o][cc0] = T(0);
                }
            }
        }
        __syncthreads();             // buffer buf is refilled by the next iteration's issue
    }
}

template <typename T, int TKO, int TC>
int launch_variant(rtr_plan* p, const T* X, int64_t A, int64_t I, int64_t B, const double* Q, int K, T* out,
                   cudaStream_t s) {
    int nkt = 1;
    while (nkt * TKO < K) nkt *= 2;
    const int CT = NT * TC / nkt;
    if (CT < TC) return rtr_set_error(RTR_EINVAL, "mode product tile does not fit");
    // Q rows padded to 16 bytes (cp.async granularity)
    constexpr int VE = 16 / sizeof(T);
    const int qld = (nkt * TKO + VE - 1) / VE * VE;
    if ((size_t)I * qld * sizeof(T) > p->ttm_q_bytes) return rtr_set_error(RTR_EINVAL, "mode product Q workspace too small");
    T* Qc = reinterpret_cast<T*>(p->ttm_q);
    qconv_kernel<T><<<(unsigned)std::min<int64_t>(rtr_ceil_div(I * qld, 256), 1024), 256, 0, s>>>(Q, (int)I, K, qld, Qc);
    RTR_LAUNCH_CHECK("qconv_kernel");
    TtmArgs<T> a{};
    a.X = X; a.A = A; a.B = B; a.I = (int)I; a.K = K; a.Qc = Qc; a.out = out; a.NKT = nkt; a.CT = CT; a.qld = qld;
    // X chunk row pitch: odd for the transposed (B == 1) scalar variants
    // (conflict-free stores), else a multiple of 16 bytes (16-byte copies and
    // vector loads)
    a.xld = (B == 1 && TC % 4 != 0) ? CT + 1 : CT + 4;
    const size_t qbytes = (size_t)I * qld * sizeof(T);
    a.qres = qbytes <= TTM_QRES_MAX ? 1 : 0;
    const size_t per_row = sizeof(T) * (2 * (size_t)a.xld + (a.qres ? 0 : 2 * (size_t)qld));
    const size_t avail = TTM_SMEM_BUDGET - (a.qres ? qbytes : 0) - sizeof(int) * (size_t)CT;
    int64_t ic = (int64_t)(avail / per_row);
    ic = std::min<int64_t>({ic, I, sizeof(T) == 8 ? 64 : 128});
    if (ic < I) ic = std::max<int64_t>(8, ic & ~(int64_t)7);
    a.IC = (int)ic;
    a.vec = (B > 1 && B >= CT && (B * (int64_t)sizeof(T)) % 16 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) ? 1 : 0;
    const size_t smem = sizeof(T) * ((a.qres ? (size_t)I * qld : 2 * (size_t)a.IC * qld) + 2 * (size_t)a.IC * a.xld) +
                        sizeof(int) * (size_t)CT;
    if (smem > 227 * 1024) return rtr_set_error(RTR_EINVAL, "mode product tile exceeds shared memory");
    if (B == 1) a.ntiles = rtr_ceil_div(A, CT);
    else if (B < CT) a.ntiles = rtr_ceil_div(A, CT / B);      // whole a-blocks per tile
    else { a.nbt = rtr_ceil_div(B, CT); a.ntiles = A * a.nbt; }
    auto kern = ttm_kernel<T, TKO, TC>;
    RTR_SMEM(kern, smem);
    int occ = 1;
    RTR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ntiles, (int64_t)std::max(occ, 1) * p->num_sms));
    kern<<<(unsigned)grid, NT, smem, s>>>(a);
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
