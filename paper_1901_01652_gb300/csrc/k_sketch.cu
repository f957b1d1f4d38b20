// SIMT split-K mode contraction: the Gaussian sketch of Algorithm 1 step 5
// (Y_n = X_(n) Omega_n, Omega_n generated on the fly) and the TR-ALS
// contraction P_<n> S of Eq. 2 (S read from memory), in float32 or float64.
//
// Work decomposition: the reduction index r = a*B + b of the (A, I, B) view
// is cut into chunks of RC consecutive r (one a, a run of b; or a run of a
// when B == 1, so that global loads are always along the contiguous index).
// A CTA owns up to rows_cta rows i (grid.y splits larger I) and walks its
// chunks grid-stride, keeping a TM x TK register tile of Y per thread.  Each
// CTA writes one float64 partial of its rows; a second kernel sums the
// partials in CTA order (deterministic).
#include <cstdio>
#include <algorithm>
#include "rtr_internal.cuh"

namespace {

constexpr int RC = 32;        // reduction chunk
constexpr int NT = 256;       // threads per CTA

template <typename T, int TM, int TK, bool GEN>
__global__ void __launch_bounds__(NT) contract_kernel(
    const T* __restrict__ X, int64_t A, int I, int64_t B, int C, int NTK, int rows_cta,
    int64_t nchunks, int64_t nbc, int64_t aoff, uint64_t seed, int mode, const T* __restrict__ table,
    const T* __restrict__ M, int64_t ldm, int makb, double* __restrict__ partial, double* __restrict__ normp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int KP = NTK * TK;
    const int NTI = NT / NTK;
    const int xld = rows_cta + 1;
    T* Xs = reinterpret_cast<T*>(smem_raw);          // [RC][xld]
    T* Ms = Xs + RC * xld;                           // [RC][KP]
    T* tab = Ms + RC * KP;                           // [4096] (GEN)
    const int tid = threadIdx.x;
    const int ti = tid % NTI, tk = tid / NTI;
    const int rbeg = blockIdx.y * rows_cta;

    if (GEN) {
        for (int j = tid; j < 4096; j += NT) tab[j] = table[j];
    }
    T acc[TM][TK];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int q = 0; q < TK; ++q) acc[m][q] = T(0);
    double nsum = 0.0;
    const int ncalls = (C + 19) / 20;

    // chunk ch = a * nbc + bi, advanced by gridDim.x without 64-bit divisions
    // (a 64-bit division is a long instruction sequence per chunk)
    int64_t ca = 0, cb = 0;
    const int64_t qa = gridDim.x / nbc, qb = gridDim.x % nbc;
    if (B != 1) { ca = blockIdx.x / nbc; cb = blockIdx.x % nbc; }
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        int64_t a0, b0;
        int len;
        if (B == 1) {
            a0 = ch * RC; b0 = 0;
            len = (int)min((int64_t)RC, A - a0);
        } else {
            a0 = ca; b0 = cb * RC;
            len = (int)min((int64_t)RC, B - b0);
            cb += qb; ca += qa;
            if (cb >= nbc) { cb -= nbc; ++ca; }
        }
        const int64_t rbase = (B == 1) ? a0 : a0 * B + b0;   // r of rr = 0 (stored operand)
        // generated operand: the row of Omega_n counts a from aoff (a slab of a
        // larger tensor along its slowest modes)
        const int64_t gbase = (B == 1) ? a0 + aoff : (a0 + aoff) * B + b0;
        __syncthreads();
        // ---- X tile -> Xs[rr][il]
        if (B == 1) {
#pragma unroll 4
            for (int e = tid; e < rows_cta * RC; e += NT) {
                const int il = e % rows_cta, rr = e / rows_cta, i = rbeg + il;
                T v = T(0);
                if (i < I && rr < len) v = X[(a0 + rr) * (int64_t)I + i];
                Xs[rr * xld + il] = v;
                if (normp) nsum += (double)v * (double)v;
            }
        } else {
#pragma unroll 4
            for (int e = tid; e < rows_cta * RC; e += NT) {
                const int rr = e % RC, il = e / RC, i = rbeg + il;
                T v = T(0);
                if (i < I && rr < len) v = X[(a0 * I + i) * B + b0 + rr];
                Xs[rr * xld + il] = v;
                if (normp) nsum += (double)v * (double)v;
            }
        }
        // ---- operand tile -> Ms[rr][k]
        if (GEN) {
            for (int w = tid; w < RC * ncalls; w += NT) {
                const int rr = w % RC, cb = w / RC;
                uint64_t wd[4] = {0, 0, 0, 0};
                if (rr < len) rtr::omega_words(seed, mode, (uint64_t)(gbase + rr), (uint64_t)cb, wd);
#pragma unroll
                for (int t = 0; t < 20; ++t) {
                    const int k = cb * 20 + t;
                    if (k < KP) Ms[rr * KP + k] = (rr < len && k < C) ? tab[rtr::omega_field(wd, t)] : T(0);
                }
            }
            for (int e = tid; e < RC * KP; e += NT) {
                const int k = e % KP;
                if (k >= ncalls * 20) Ms[e] = T(0);
            }
        } else if (makb && B > 1) {
            // (A, C, B) layout: consecutive threads take consecutive b
            for (int e = tid; e < RC * KP; e += NT) {
                const int rr = e % RC, k = e / RC;
                T v = T(0);
                if (rr < len && k < C) v = M[(a0 * C + k) * B + b0 + rr];
                Ms[rr * KP + k] = v;
            }
        } else {
            for (int e = tid; e < RC * KP; e += NT) {
                const int rr = e / KP, k = e % KP;
                T v = T(0);
                if (rr < len && k < C) v = M[(rbase + rr) * ldm + k];
                Ms[e] = v;
            }
        }
        __syncthreads();
        // ---- register-tiled FMA
#pragma unroll 4
        for (int rr = 0; rr < RC; ++rr) {
            T xv[TM], mv[TK];
#pragma unroll
            for (int m = 0; m < TM; ++m) xv[m] = Xs[rr * xld + ti + NTI * m];
#pragma unroll
            for (int q = 0; q < TK; ++q) mv[q] = Ms[rr * KP + tk * TK + q];
#pragma unroll
            for (int m = 0; m < TM; ++m)
#pragma unroll
                for (int q = 0; q < TK; ++q) acc[m][q] = fma(xv[m], mv[q], acc[m][q]);
        }
    }
#pragma unroll
    for (int m = 0; m < TM; ++m) {
        const int i = rbeg + ti + NTI * m;
#pragma unroll
        for (int q = 0; q < TK; ++q) {
            const int k = tk * TK + q;
            if (i < I && k < C) partial[((int64_t)blockIdx.x * I + i) * C + k] = (double)acc[m][q];
        }
    }
    if (normp) {
        __shared__ double red[NT / 32];
        nsum = rtr::warp_sum(nsum);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = nsum;
        __syncthreads();
        if (tid == 0) {
            double s = 0;
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            normp[blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
    }
}

// Y[e] = sum_p partial[p * count + e], p in order; norm total likewise (a
// non-finite total raises RTR_FLAG_NONFINITE in *flags when flags is given).
__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nparts, int64_t count,
                                       double* __restrict__ Y, const double* __restrict__ normp,
                                       int nnorm, double* __restrict__ norm_out, int* __restrict__ flags) {
    // one warp per output: lanes stride over the partials, then a fixed-order
    // butterfly; the result does not depend on timing
    const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e < count) {
        double s = 0.0;
        for (int p = lane; p < nparts; p += 32) s += partial[p * count + e];
        s = rtr::warp_sum(s);
        if (lane == 0) Y[e] = s;
    }
    if (norm_out && blockIdx.x == 0 && threadIdx.x < 32) {
        double s = 0.0;
        for (int p = lane; p < nnorm; p += 32) s += normp[p];
        s = rtr::warp_sum(s);
        if (lane == 0) {
            *norm_out = s;
            if (flags && !isfinite(s)) atomicOr(flags, RTR_FLAG_NONFINITE);
        }
    }
}

struct Shape { int TM, TK, NTK, rows, gy; };

Shape choose_shape(int64_t I, int C) {
    Shape best{0, 0, 0, 0, 0};
    double best_cost = 1e300;
    for (int TK : {4, 8}) {
        int ntk = 1;
        while (ntk * TK < C) ntk *= 2;
        if (ntk > 32) continue;
        const int nti = NT / ntk;
        for (int TM : {1, 2, 4, 8}) {
            if (TM * TK > 64) continue;
            const int rows = nti * TM;
            const int64_t gy = rtr_ceil_div(I, rows);
            // padded work + a charge per extra row pass (operand regeneration)
            const double cost = (double)gy * rows * ntk * TK + 0.02 * gy * I * C + (rows > 256 ? 1e30 : 0);
            if (cost < best_cost) { best_cost = cost; best = Shape{TM, TK, ntk, rows, (int)gy}; }
        }
    }
    return best;
}

template <typename T, int TM, int TK, bool GEN>
int launch_one(rtr_plan* p, const ContractArgs& a, const Shape& sh, cudaStream_t s) {
    const int KP = sh.NTK * sh.TK;
    size_t smem = sizeof(T) * ((size_t)RC * (sh.rows + 1) + (size_t)RC * KP + (GEN ? 4096 : 0));
    auto kern = contract_kernel<T, TM, TK, GEN>;
    RTR_SMEM(kern, smem);
    int occ = 0;
    RTR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
    occ = std::max(1, occ);
    int64_t nchunks, nbc = 1;
    if (a.B == 1) nchunks = rtr_ceil_div(a.A, RC);
    else { nbc = rtr_ceil_div(a.B, RC); nchunks = a.A * nbc; }
    int64_t gx = std::max<int64_t>(1, (int64_t)occ * p->num_sms / sh.gy);
    // a stored operand (the TR-ALS contraction) is small: give every CTA a few
    // chunks so that the partial reduction stays short
    if (!GEN) gx = std::min<int64_t>(gx, std::max<int64_t>(1, nchunks / 2));
    gx = std::min<int64_t>(gx, nchunks);
    gx = std::max<int64_t>(gx, 1);
    const int64_t need = gx * a.I * a.C;
    if ((size_t)need > p->partial_elems) {
        gx = std::max<int64_t>(1, (int64_t)(p->partial_elems / (a.I * a.C)));
        if (gx < 1 || (size_t)(gx * a.I * a.C) > p->partial_elems)
            return rtr_set_error(RTR_ENOMEM, "contraction partials exceed the plan workspace");
    }
    dim3 grid((unsigned)gx, (unsigned)sh.gy);
    const bool want_norm = a.norm_out != nullptr;
    if (want_norm && (size_t)(gx * sh.gy) > p->normx_part_elems)
        return rtr_set_error(RTR_ENOMEM, "norm partials exceed the plan workspace");
    kern<<<grid, NT, smem, s>>>((const T*)a.X, a.A, (int)a.I, a.B, a.C, sh.NTK, sh.rows, nchunks, nbc,
                                a.aoff, a.seed, a.mode, (const T*)a.table, (const T*)a.M, a.makb ? (int64_t)a.C : a.ldm,
                                a.makb, p->partial, want_norm ? p->normx_part : nullptr);
    RTR_LAUNCH_CHECK("contract_kernel");
    const int64_t count = a.I * a.C;
    reduce_partials_kernel<<<(unsigned)rtr_ceil_div(count * 32, 256), 256, 0, s>>>(
        p->partial, (int)gx, count, a.Y, p->normx_part, (int)(gx * sh.gy), want_norm ? a.norm_out : nullptr,
        p->flags);
    RTR_LAUNCH_CHECK("reduce_partials_kernel");
    return RTR_OK;
}

template <typename T, bool GEN>
int dispatch_shape(rtr_plan* p, const ContractArgs& a, const Shape& sh, cudaStream_t s) {
#define RTR_CASE(tm, tk) if (sh.TM == tm && sh.TK == tk) return launch_one<T, tm, tk, GEN>(p, a, sh, s);
    RTR_CASE(1, 4) RTR_CASE(2, 4) RTR_CASE(4, 4) RTR_CASE(8, 4)
    RTR_CASE(1, 8) RTR_CASE(2, 8) RTR_CASE(4, 8) RTR_CASE(8, 8)
#undef RTR_CASE
    return rtr_set_error(RTR_EINVAL, "no contraction shape for TM=%d TK=%d", sh.TM, sh.TK);
}

}  // namespace

int launch_contract(rtr_plan* p, int is_f64, const ContractArgs& a, cudaStream_t s) {
    if (a.C < 1 || a.C > 256) return rtr_set_error(RTR_EINVAL, "contraction width %d out of range", a.C);
    const Shape sh = choose_shape(a.I, a.C);
    if (sh.TM == 0) return rtr_set_error(RTR_EINVAL, "no contraction shape for C=%d", a.C);
    if (is_f64) return a.gen ? dispatch_shape<double, true>(p, a, sh, s) : dispatch_shape<double, false>(p, a, sh, s);
    return a.gen ? dispatch_shape<float, true>(p, a, sh, s) : dispatch_shape<float, false>(p, a, sh, s);
}

// Worst-case partial count of a contraction, for workspace sizing.
size_t contract_partial_elems(int num_sms, int64_t I, int C) {
    const Shape sh = choose_shape(I, C);
    // occupancy never exceeds 8 CTAs of 256 threads; grid.x = occ * SMs / grid.y
    const int64_t gx = std::max<int64_t>(1, (int64_t)8 * num_sms / std::max(1, sh.gy));
    return (size_t)(gx * I * C);
}
size_t contract_norm_elems(int num_sms, int64_t I, int C) {
    const Shape sh = choose_shape(I, C);
    return (size_t)((int64_t)8 * num_sms * std::max(1, sh.gy) + 8);
}

// ---- allocation-free single-mode sketch ---------------------------------------
// For callers that cannot call cudaMalloc (for example code running inside a
// host framework that owns all device memory, or a process that must not grow
// its device footprint after start-up).  The split-K partials and the
// Gaussian tables live in file-scope __device__ arrays instead of a plan's
// workspace.  Every GPU that loads this library holds these arrays (16 MiB of
// partials plus 48 KiB of tables) until the process exits.
#include <mutex>

namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 21;    // 2 Mi doubles = 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
static __device__ __align__(256) double g_noalloc_tab64[4096];
static __device__ __align__(256) float g_noalloc_tab32[4096];

struct NoAllocDevice {
    bool ready = false;
    double* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    double* tab64 = nullptr;
    float* tab32 = nullptr;
    int num_sms = 0;
    // CTAs per SM of contract_kernel<T, TM, TK, true> for each shared-memory
    // size it launches with, found on first use: [float64][TM index][TK
    // index][log2 NTK], 0 = not yet; attr[float64][TM index][TK index] = 1
    // once the kernel's shared-memory limit is raised to its largest size
    int occ[2][4][2][6] = {};
    int attr[2][4][2] = {};
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

// Once per device, with that device current: resolve the device addresses of
// the file-scope arrays (host code cannot use their names as pointers) and
// fill the tables with synchronous copies.
int noalloc_setup(NoAllocDevice** out) {
    int dev = 0;
    RTR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return rtr_set_error(RTR_EINVAL, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        RTR_CUDA(cudaGetSymbolAddress((void**)&d.scratch, g_noalloc_scratch));
        RTR_CUDA(cudaGetSymbolAddress((void**)&d.tab64, g_noalloc_tab64));
        RTR_CUDA(cudaGetSymbolAddress((void**)&d.tab32, g_noalloc_tab32));
        RTR_CUDA(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
        static double t64[4096];
        static float t32[4096];
        rtr_host_tables(t64, t32);
        RTR_CUDA(cudaMemcpy(d.tab64, t64, sizeof(t64), cudaMemcpyHostToDevice));
        RTR_CUDA(cudaMemcpy(d.tab32, t32, sizeof(t32), cudaMemcpyHostToDevice));
        d.ready = true;
    }
    *out = &d;
    return RTR_OK;
}

// The kernel's shared memory depends on (T, TM, TK, NTK) only; its limit
// (set once to the largest size any NTK needs) and its occupancy per size are
// set up once per device and reused, so that the split-K width, and with it
// the float64 summation order, is the same on every call of a shape.
template <typename T, int TM, int TK>
int noalloc_occupancy(NoAllocDevice& d, int ntk, size_t smem, int* out) {
    constexpr int ti = TM == 1 ? 0 : TM == 2 ? 1 : TM == 4 ? 2 : 3;
    constexpr int tk = TK == 4 ? 0 : 1;
    int lg = 0;
    while ((1 << lg) < ntk) ++lg;
    if (lg > 5) return rtr_set_error(RTR_EINVAL, "contraction shape with %d column groups", ntk);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    auto kern = contract_kernel<T, TM, TK, true>;
    const int f64 = sizeof(T) == 8;
    if (!d.attr[f64][ti][tk]) {
        const size_t smem_max = sizeof(T) * ((size_t)RC * (256 + 1) + (size_t)RC * 32 * TK + 4096);
        RTR_SMEM(kern, smem_max);
        d.attr[f64][ti][tk] = 1;
    }
    int& o = d.occ[f64][ti][tk][lg];
    if (o == 0) {
        int occ = 0;
        RTR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
        o = std::max(1, occ);
    }
    *out = o;
    return RTR_OK;
}

template <typename T, int TM, int TK>
int launch_noalloc(NoAllocDevice& d, const ContractArgs& a, const Shape& sh, cudaStream_t s) {
    const int KP = sh.NTK * sh.TK;
    const size_t smem = sizeof(T) * ((size_t)RC * (sh.rows + 1) + (size_t)RC * KP + 4096);
    auto kern = contract_kernel<T, TM, TK, true>;
    int occ = 0;
    const int st = noalloc_occupancy<T, TM, TK>(d, sh.NTK, smem, &occ);
    if (st) return st;
    int64_t nchunks, nbc = 1;
    if (a.B == 1) nchunks = rtr_ceil_div(a.A, RC);
    else { nbc = rtr_ceil_div(a.B, RC); nchunks = a.A * nbc; }
    int64_t gx = std::max<int64_t>(1, (int64_t)occ * d.num_sms / sh.gy);
    gx = std::min<int64_t>(gx, nchunks);
    gx = std::min<int64_t>(gx, (int64_t)(kNoAllocScratchDoubles / (a.I * a.C)));   // >= 1, checked by caller
    dim3 grid((unsigned)gx, (unsigned)sh.gy);
    kern<<<grid, NT, smem, s>>>((const T*)a.X, a.A, (int)a.I, a.B, a.C, sh.NTK, sh.rows, nchunks, nbc, (int64_t)0,
                                a.seed, a.mode, (const T*)a.table, nullptr, 0, 0, d.scratch, nullptr);
    RTR_LAUNCH_CHECK("contract_kernel (no-alloc)");
    const int64_t count = a.I * a.C;
    reduce_partials_kernel<<<(unsigned)rtr_ceil_div(count * 32, 256), 256, 0, s>>>(d.scratch, (int)gx, count, a.Y,
                                                                                nullptr, 0, nullptr, nullptr);
    RTR_LAUNCH_CHECK("reduce_partials_kernel (no-alloc)");
    return RTR_OK;
}

template <typename T>
int dispatch_noalloc(NoAllocDevice& d, const ContractArgs& a, const Shape& sh, cudaStream_t s) {
#define RTR_CASE(tm, tk) if (sh.TM == tm && sh.TK == tk) return launch_noalloc<T, tm, tk>(d, a, sh, s);
    RTR_CASE(1, 4) RTR_CASE(2, 4) RTR_CASE(4, 4) RTR_CASE(8, 4)
    RTR_CASE(1, 8) RTR_CASE(2, 8) RTR_CASE(4, 8) RTR_CASE(8, 8)
#undef RTR_CASE
    return rtr_set_error(RTR_EINVAL, "no contraction shape for TM=%d TK=%d", sh.TM, sh.TK);
}

}  // namespace

extern "C" int rtr_sketch_mode_noalloc(int prec, const void* X, int64_t A, int64_t I, int64_t B, int K,
                                       uint64_t seed, int mode, double* Y, void* stream) {
    if (!X || !Y) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (prec != RTR_FP64 && prec != RTR_FP32)
        return rtr_set_error(RTR_EINVAL, "rtr_sketch_mode_noalloc supports RTR_FP64 and RTR_FP32 only");
    if (A < 1 || I < 1 || B < 1 || I > (1 << 30)) return rtr_set_error(RTR_EINVAL, "bad view (A, I, B)");
    if (K < 1 || K > RTR_MAX_KSKETCH) return rtr_set_error(RTR_EINVAL, "K = %d outside [1, 64]", K);
    if ((size_t)(I * K) > kNoAllocScratchDoubles)
        return rtr_set_error(RTR_EINVAL, "I*K = %lld exceeds the static scratch of %zu doubles",
                             (long long)(I * K), kNoAllocScratchDoubles);
    NoAllocDevice* d = nullptr;
    int st = noalloc_setup(&d);
    if (st) return st;
    const int f64 = prec == RTR_FP64;
    ContractArgs a{};
    a.X = X; a.A = A; a.I = I; a.B = B; a.C = K;
    a.gen = 1; a.seed = seed; a.mode = mode;
    a.table = f64 ? (const void*)d->tab64 : (const void*)d->tab32;
    a.Y = Y; a.norm_out = nullptr;
    const Shape sh = choose_shape(I, K);
    cudaStream_t s = (cudaStream_t)stream;
    return f64 ? dispatch_noalloc<double>(*d, a, sh, s) : dispatch_noalloc<float>(*d, a, sh, s);
}
