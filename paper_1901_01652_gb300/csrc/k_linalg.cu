// Orthonormal bases Q_n of Algorithm 1 step 6 (economy QR, diag(R) > 0) in
// float64, and a sum-of-squares reduction.
//
// QR method: CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014):
// Q1 = Y R1^-1 with R1 = chol(Y^T Y), then Q = Q1 R2^-1 with R2 = chol(Q1^T Q1).
// The Gram partials are spread over many CTAs because float64 throughput per
// SM is low on this part.  If a Cholesky pivot is not positive (Y numerically
// rank deficient), that mode falls back to classical Gram-Schmidt with one
// re-orthogonalisation ("twice is enough", Giraud et al. 2005) in one CTA;
// columns that vanish are completed with unit vectors.  Both give the unique
// Q with positive diag(R) when Y has full column rank.
#include <algorithm>
#include "rtr_internal.cuh"
#include "dense.cuh"

namespace {

constexpr int RCH = 16;   // rows per Gram partial

struct OrthJob {
    const double* Y[RTR_MAXN];
    double* Q[RTR_MAXN];
    int I[RTR_MAXN];
    int K[RTR_MAXN];
    int nmodes;
};

// part[mode][chunk][K*K] = sum over the chunk's rows of y y^T (upper triangle).
__global__ void gram_partial_kernel(OrthJob job, int src_is_q, double* __restrict__ part, int maxchunks,
                                    int kk_stride) {
    const int md = blockIdx.y;
    if (md >= job.nmodes) return;
    const int I = job.I[md], K = job.K[md];
    const double* Y = src_is_q ? job.Q[md] : job.Y[md];
    const int nch = (I + RCH - 1) / RCH;
    __shared__ double ys[RCH][64];
    for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int r0 = ch * RCH, nr = min(RCH, I - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < RCH * K; e += blockDim.x) {
            const int r = e / K, k = e % K;
            ys[r][k] = (r < nr) ? Y[(int64_t)(r0 + r) * K + k] : 0.0;
        }
        __syncthreads();
        double* out = part + ((int64_t)md * maxchunks + ch) * kk_stride;
        for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
            const int i = e / K, j = e % K;
            if (j < i) continue;
            double s = 0.0;
            for (int r = 0; r < RCH; ++r) s += ys[r][i] * ys[r][j];
            out[e] = s;
        }
    }
}

// gsum[mode][i * 64 + j] = sum over chunks of part (the full symmetric Gram),
// one thread per (i <= j) entry, spread over many CTAs: float64 adds are slow
// on this part, so the chunk sum runs as four interleaved chains (fixed
// order: chunk c goes to chain c mod 4, the chains are added pairwise).
__global__ void gram_sum_kernel(OrthJob job, const double* __restrict__ part, int maxchunks, int kk_stride,
                                double* __restrict__ gsum) {
    const int md = blockIdx.y;
    if (md >= job.nmodes) return;
    const int I = job.I[md], K = job.K[md];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * K) return;
    const int i = e / K, j = e % K;
    if (j < i) return;
    const int nch = (I + RCH - 1) / RCH;
    const double* src = part + (int64_t)md * maxchunks * kk_stride + e;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int c = 0;
    for (; c + 4 <= nch; c += 4) {
        a0 += src[(int64_t)c * kk_stride];
        a1 += src[(int64_t)(c + 1) * kk_stride];
        a2 += src[(int64_t)(c + 2) * kk_stride];
        a3 += src[(int64_t)(c + 3) * kk_stride];
    }
    if (c < nch) a0 += src[(int64_t)c * kk_stride];
    if (c + 1 < nch) a1 += src[(int64_t)(c + 1) * kk_stride];
    if (c + 2 < nch) a2 += src[(int64_t)(c + 2) * kk_stride];
    const double g = (a0 + a1) + (a2 + a3);
    gsum[(int64_t)md * 4096 + i * 64 + j] = g;
    gsum[(int64_t)md * 4096 + j * 64 + i] = g;
}

// One CTA per mode: G from gram_sum_kernel (in rfac), R = chol(G)^T written
// back to rfac (lower L, row-major, leading dimension 64).  On failure runs
// CGS2 on the source and writes Q directly, marking status[mode] = 1.
__global__ void chol_or_fallback_kernel(OrthJob job, int src_is_q, double* __restrict__ rfac,
                                        int* __restrict__ status, int* __restrict__ flags) {
    const int md = blockIdx.x;
    const int I = job.I[md], K = job.K[md];
    const double* Y = src_is_q ? job.Q[md] : job.Y[md];
    double* Q = job.Q[md];
    __shared__ double G[64 * 65];
    __shared__ double red[32];
    const int ld = 65;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, j = e % K;
        G[i * ld + j] = rfac[(int64_t)md * 4096 + i * 64 + j];
    }
    __syncthreads();
    int ok = 1;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x)
        if (!isfinite(G[(e / K) * ld + e % K])) ok = 0;
    ok = __syncthreads_and(ok);
    if (!ok) { if (threadIdx.x == 0) atomicOr(flags, RTR_FLAG_NONFINITE); }
    // pivots below 1e-14 of their diagonal mean kappa(Y) beyond ~1e7, where
    // CholeskyQR2 loses orthogonality: take the fallback instead
    if (ok) ok = rtr::block_cholesky(G, K, ld, 1e-14) ? 1 : 0;
    if (ok) {
        for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
            const int i = e / K, j = e % K;
            rfac[(int64_t)md * 64 * 64 + i * 64 + j] = (j <= i) ? G[i * ld + j] : 0.0;
        }
        if (threadIdx.x == 0) status[md] = 0;
        return;
    }
    // ---- fallback: classical Gram-Schmidt, twice, one column at a time.
    if (threadIdx.x == 0) { status[md] = 1; atomicOr(flags, RTR_FLAG_QR_FALLBACK); }
    __shared__ double coef[64];
    // Q may alias the source (pass 2): copy column by column through registers.
    for (int k = 0; k < K; ++k) {
        // v = y_k (into Q[:, k])
        double ynorm2 = 0.0;
        for (int i = threadIdx.x; i < I; i += blockDim.x) {
            const double v = Y[(int64_t)i * K + k];
            Q[(int64_t)i * K + k] = v;
            ynorm2 += v * v;
        }
        ynorm2 = rtr::block_sum(ynorm2, red);
        for (int pass = 0; pass < 2; ++pass) {
            for (int l = 0; l < k; ++l) {
                double s = 0.0;
                for (int i = threadIdx.x; i < I; i += blockDim.x) s += Q[(int64_t)i * K + l] * Q[(int64_t)i * K + k];
                s = rtr::block_sum(s, red);
                if (threadIdx.x == 0) coef[l] = s;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < I; i += blockDim.x) {
                double v = Q[(int64_t)i * K + k];
                for (int l = 0; l < k; ++l) v -= coef[l] * Q[(int64_t)i * K + l];
                Q[(int64_t)i * K + k] = v;
            }
            __syncthreads();
        }
        double nv = 0.0;
        for (int i = threadIdx.x; i < I; i += blockDim.x) nv += Q[(int64_t)i * K + k] * Q[(int64_t)i * K + k];
        nv = rtr::block_sum(nv, red);
        if (!(nv > 1e-28 * ynorm2) || nv == 0.0) {
            // completion: the unit vector e_m with the smallest component in span(Q[:, :k])
            for (int m = 0; m < I; ++m) {
                for (int l = 0; l < k; ++l) {
                    if (threadIdx.x == 0) coef[l] = Q[(int64_t)m * K + l];
                }
                __syncthreads();
                for (int i = threadIdx.x; i < I; i += blockDim.x) {
                    double v = (i == m) ? 1.0 : 0.0;
                    for (int l = 0; l < k; ++l) v -= coef[l] * Q[(int64_t)i * K + l];
                    Q[(int64_t)i * K + k] = v;
                }
                __syncthreads();
                double nn = 0.0;
                for (int i = threadIdx.x; i < I; i += blockDim.x) nn += Q[(int64_t)i * K + k] * Q[(int64_t)i * K + k];
                nn = rtr::block_sum(nn, red);
                if (nn > 0.5) { nv = nn; break; }
            }
        }
        const double inv = 1.0 / sqrt(nv);
        for (int i = threadIdx.x; i < I; i += blockDim.x) Q[(int64_t)i * K + k] *= inv;
        __syncthreads();
    }
}

// Q = Y L^-T, one warp per row (forward substitution with the upper factor
// L^T).  Row q solves q L^T = y: column-oriented, q_k = y_k / L[k][k] and then
// y_l -= q_k L[l][k] for l > k, with lane t holding y_t and y_{t+32}, so the
// float64 dependency chain per row is K steps long rather than K^2 / 2.
constexpr int TRSM_WARPS = 8;
__global__ void __launch_bounds__(TRSM_WARPS * 32) trsm_rows_kernel(OrthJob job, int src_is_q,
                                                                   const double* __restrict__ rfac,
                                                                   const int* __restrict__ status) {
    const int md = blockIdx.y;
    if (md >= job.nmodes || status[md]) return;
    const int I = job.I[md], K = job.K[md];
    const double* Y = src_is_q ? job.Q[md] : job.Y[md];
    double* Q = job.Q[md];
    __shared__ double Lt[64 * 64];      // Lt[k * 64 + l] = L[l][k]
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int l = e / K, k = e % K;
        Lt[k * 64 + l] = rfac[(int64_t)md * 4096 + l * 64 + k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * TRSM_WARPS + (threadIdx.x >> 5);
    for (int i = warp; i < I; i += gridDim.x * TRSM_WARPS) {
        const double* yr = Y + (int64_t)i * K;
        double y0 = lane < K ? yr[lane] : 0.0;
        double y1 = lane + 32 < K ? yr[lane + 32] : 0.0;
        for (int k = 0; k < K; ++k) {
            const double yk = __shfl_sync(0xffffffffu, k < 32 ? y0 : y1, k & 31);
            const double qk = yk / Lt[k * 64 + k];
            const double* col = Lt + k * 64;
            if (lane == k) y0 = qk;
            else if (lane > k) y0 -= qk * col[lane];
            if (lane + 32 == k) y1 = qk;
            else if (lane + 32 > k && lane + 32 < K) y1 -= qk * col[lane + 32];
        }
        double* qr = Q + (int64_t)i * K;
        if (lane < K) qr[lane] = y0;
        if (lane + 32 < K) qr[lane + 32] = y1;
    }
}

__global__ void identity_kernel(double* Q, int I) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I * I; e += gridDim.x * blockDim.x)
        Q[e] = (e / I == e % I) ? 1.0 : 0.0;
}

template <typename T>
__global__ void sumsq_kernel(const T* __restrict__ X, int64_t n, double* __restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)X[e];
        s += v * v;
    }
    s = rtr::block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// *out = sum of part[0 .. n) (one CTA; block_sum's fixed order); a
// non-finite sum raises RTR_FLAG_NONFINITE in *flags when flags is given
__global__ void sum_parts_kernel(const double* __restrict__ part, int n, double* __restrict__ out,
                                 int* __restrict__ flags) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = rtr::block_sum(s, red);
    if (threadIdx.x == 0) {
        *out = s;
        if (flags && !isfinite(s)) atomicOr(flags, RTR_FLAG_NONFINITE);
    }
}

}  // namespace

size_t orth_ws_elems(int num_sms, int64_t maxI) {
    const int64_t maxchunks = rtr_ceil_div(maxI, RCH);
    return (size_t)(RTR_MAXN * maxchunks * 64 * 64 + RTR_MAXN * 64 * 64 + RTR_MAXN);
}

int launch_orth(rtr_plan* p, const double* const* Y, double* const* Q, cudaStream_t s) {
    return launch_orth_mask(p, Y, Q, ~0u, s);
}

int launch_orth_mask(rtr_plan* p, const double* const* Y, double* const* Q, unsigned mask, cudaStream_t s) {
    OrthJob job{};
    int64_t maxI = 1;
    for (int n = 0; n < p->N; ++n) {
        if (!((mask >> n) & 1u)) continue;
        if (!p->proj[n]) {
            if (!Q[n]) return rtr_set_error(RTR_EINVAL, "Q[%d] is NULL", n);
            identity_kernel<<<64, 256, 0, s>>>(Q[n], (int)p->dims[n]);
            RTR_LAUNCH_CHECK("identity_kernel");
            continue;
        }
        if (!Y[n] || !Q[n]) return rtr_set_error(RTR_EINVAL, "Y[%d] or Q[%d] is NULL", n, n);
        const int md = job.nmodes++;
        job.Y[md] = Y[n]; job.Q[md] = Q[n]; job.I[md] = (int)p->dims[n]; job.K[md] = p->K[n];
        maxI = std::max<int64_t>(maxI, p->dims[n]);
    }
    if (job.nmodes == 0) return RTR_OK;
    const int maxchunks = (int)rtr_ceil_div(maxI, RCH);
    const int kk = 64 * 64;
    double* part = p->qr_ws;
    double* rfac = part + (size_t)RTR_MAXN * maxchunks * kk;
    int* status = reinterpret_cast<int*>(rfac + (size_t)RTR_MAXN * kk);
    (void)status;
    // status lives in its own small region of the workspace
    int* st = reinterpret_cast<int*>(p->scal + 16);
    for (int pass = 0; pass < 2; ++pass) {
        const int src_is_q = pass;   // pass 0 reads Y, pass 1 re-orthogonalises Q
        dim3 g1((unsigned)std::min(maxchunks, 4 * p->num_sms), (unsigned)job.nmodes);
        gram_partial_kernel<<<g1, 256, 0, s>>>(job, src_is_q, part, maxchunks, kk);
        RTR_LAUNCH_CHECK("gram_partial_kernel");
        dim3 g2(4096 / 256, (unsigned)job.nmodes);
        gram_sum_kernel<<<g2, 256, 0, s>>>(job, part, maxchunks, kk, rfac);
        RTR_LAUNCH_CHECK("gram_sum_kernel");
        chol_or_fallback_kernel<<<job.nmodes, 256, 0, s>>>(job, src_is_q, rfac, st, p->flags);
        RTR_LAUNCH_CHECK("chol_or_fallback_kernel");
        dim3 g3((unsigned)rtr_ceil_div(maxI, TRSM_WARPS), (unsigned)job.nmodes);
        trsm_rows_kernel<<<g3, TRSM_WARPS * 32, 0, s>>>(job, src_is_q, rfac, st);
        RTR_LAUNCH_CHECK("trsm_rows_kernel");
    }
    return RTR_OK;
}

namespace {
template <typename T>
__global__ void add_kernel(T* __restrict__ y, const T* __restrict__ x, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] += x[e];
}
}  // namespace

int launch_add(void* y, const void* x, int64_t n, int is_f64, cudaStream_t s) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(rtr_ceil_div(n, 256), 4096));
    if (is_f64) add_kernel<double><<<g, 256, 0, s>>>((double*)y, (const double*)x, n);
    else add_kernel<float><<<g, 256, 0, s>>>((float*)y, (const float*)x, n);
    RTR_LAUNCH_CHECK("add_kernel");
    return RTR_OK;
}

int launch_sumsq(const void* X, int is_f64, int64_t n, double* part, int nparts, double* out, int* flags,
                 cudaStream_t s) {
    if (is_f64) sumsq_kernel<double><<<nparts, 256, 0, s>>>((const double*)X, n, part);
    else sumsq_kernel<float><<<nparts, 256, 0, s>>>((const float*)X, n, part);
    RTR_LAUNCH_CHECK("sumsq_kernel");
    sum_parts_kernel<<<1, 1024, 0, s>>>(part, nparts, out, flags);
    RTR_LAUNCH_CHECK("sum_parts_kernel");
    return RTR_OK;
}
