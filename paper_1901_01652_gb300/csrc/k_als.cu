// TR-ALS on the projected tensor P (Algorithm 1 step 9), back-projection
// (step 11), the dense TR expansion Psi (Eq. 1) and the RSE identity.
//
// One core update (Eq. 2): with S_j = Z_{n+1}(i_{n+1}) ... Z_{n-1}(i_{n-1})
// (R_{n+1} x R_n), the least-squares core solves z_i G = w_i for every slice
// i of mode n, where
//   w_i[(beta, alpha)] = sum_j P_<n>[i, j] S_j[beta, alpha]      (contraction)
//   G = sum_j vec(S_j) vec(S_j)^T = E_{n+1} ... E_{n-1}           (transfer form)
//   E_m[(a,a'), (b,b')] = sum_i Z_m[a, i, b] Z_m[a', i, b']
// The subchain and the contraction run in the plan's compute type (float32
// for the FP32/BF16 plans, float64 for FP64); the transfer matrices, their
// product, the Cholesky factorisation and the solves are float64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include "rtr_internal.cuh"
#include "dense.cuh"

size_t contract_partial_elems(int num_sms, int64_t I, int C);

namespace {

// ---- subchain products --------------------------------------------------------
// Sout[(j'*Km + i), beta, gamma] = sum_c Sprev[j', beta, c] * Z[c, i, gamma]
// (Sprev == nullptr: Sout[i, beta, gamma] = Z[beta, i, gamma]).
// With final_tr, row j = b*A + a of the cyclic order is stored at a*B + b.
// With Zfirst set (and Sprev null), the previous level is the first core
// itself, read in its own layout Zfirst[beta, j', c] (Jp = its mode length).
// IDX: index type of the element decode (uint32_t when every index fits:
// a 64-bit division is a long instruction sequence per element).  TG: outputs
// per thread along gamma (consecutive), which share the loads of Sprev's row.
template <typename T, typename TZ, typename IDX, int TG>
__global__ void subchain_step_kernel(const T* __restrict__ Sprev, int64_t Jp_, int Rb, int Rc,
                                     const TZ* __restrict__ Z, int Km, int Rd, T* __restrict__ Sout,
                                     int final_tr, int64_t Aa_, int64_t Bb_, const TZ* __restrict__ Zfirst) {
    const IDX Jp = (IDX)Jp_, Aa = (IDX)Aa_, Bb = (IDX)Bb_;
    const int Rq = (Rd + TG - 1) / TG;
    const IDX total = Jp * (IDX)Km * (IDX)Rb * (IDX)Rq;
    for (IDX e = blockIdx.x * (IDX)blockDim.x + threadIdx.x; e < total; e += (IDX)gridDim.x * blockDim.x) {
        const int g0 = (int)(e % (IDX)Rq) * TG;
        const IDX q = e / (IDX)Rq;
        const int be = (int)(q % (IDX)Rb);
        const IDX j = q / (IDX)Rb;
        const int i = (int)(j % (IDX)Km);
        const IDX jp = j / (IDX)Km;
        T v[TG];
#pragma unroll
        for (int t = 0; t < TG; ++t) v[t] = T(0);
        const TZ* zc = Z + (IDX)i * (IDX)Rd + (IDX)g0;      // Z[c, i, g0 + t] = zc[c Km Rd + t]
        const IDX zs = (IDX)Km * (IDX)Rd;
        if (Zfirst != nullptr) {
            const TZ* zf = Zfirst + ((IDX)be * Jp + jp) * (IDX)Rc;
            for (int c = 0; c < Rc; ++c) {
                const T f = (T)zf[c];
#pragma unroll
                for (int t = 0; t < TG; ++t)
                    if (g0 + t < Rd) v[t] = fma(f, (T)zc[(IDX)c * zs + t], v[t]);
            }
        } else if (Sprev == nullptr) {
#pragma unroll
            for (int t = 0; t < TG; ++t)
                if (g0 + t < Rd) v[t] = (T)Z[((IDX)be * (IDX)Km + (IDX)i) * (IDX)Rd + (IDX)(g0 + t)];
        } else {
            const T* sp = Sprev + (jp * (IDX)Rb + (IDX)be) * (IDX)Rc;
            for (int c = 0; c < Rc; ++c) {
                const T f = sp[c];
#pragma unroll
                for (int t = 0; t < TG; ++t)
                    if (g0 + t < Rd) v[t] = fma(f, (T)zc[(IDX)c * zs + t], v[t]);
            }
        }
        IDX r = j;
        if (final_tr) { const IDX b = j / Aa, a = j % Aa; r = a * Bb + b; }
        T* out = Sout + (r * (IDX)Rb + (IDX)be) * (IDX)Rd + (IDX)g0;
#pragma unroll
        for (int t = 0; t < TG; ++t)
            if (g0 + t < Rd) out[t] = v[t];
    }
}

// E[(a,a'), (b,b')] = sum_i Z[a,i,b] Z[a',i,b']
__global__ void transfer_kernel(const double* __restrict__ Z, int Ra, int Km, int Rb, double* __restrict__ E) {
    const int total = Ra * Ra * Rb * Rb;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int col = e % (Rb * Rb), row = e / (Rb * Rb);
        const int a = row / Ra, a2 = row % Ra, b = col / Rb, b2 = col % Rb;
        double s = 0.0;
        for (int i = 0; i < Km; ++i) s += Z[((int64_t)a * Km + i) * Rb + b] * Z[((int64_t)a2 * Km + i) * Rb + b2];
        E[e] = s;
    }
}

// C (m x n) = A (m x k) B (k x n), float64.  8 x 8 output tiles per CTA (64
// threads) so that the float64 work of one product spreads over every SM;
// A rows and B columns of the tile are staged in shared memory (k <= 256).
__global__ void __launch_bounds__(64) matmul_f64_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                        double* __restrict__ C, int m, int k, int n) {
    __shared__ double As[8][257];
    __shared__ double Bs[256][9];
    const int i0 = blockIdx.y * 8, j0 = blockIdx.x * 8;
    for (int e = threadIdx.x; e < 8 * k; e += 64) {
        const int r = e / k, l = e % k;
        As[r][l] = (i0 + r < m) ? A[(int64_t)(i0 + r) * k + l] : 0.0;
    }
    for (int e = threadIdx.x; e < 8 * k; e += 64) {
        const int l = e / 8, c = e % 8;
        Bs[l][c] = (j0 + c < n) ? B[(int64_t)l * n + j0 + c] : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x / 8, c = threadIdx.x % 8;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s += As[r][l] * Bs[l][c];
    if (i0 + r < m && j0 + c < n) C[(int64_t)(i0 + r) * n + j0 + c] = s;
}

__global__ void trace_kernel(const double* __restrict__ M, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += M[i * n + i];
        *out = s;
    }
}

// Mprod = F_0 F_1 ... F_{cnt-1} (F_t: dim[t] x dim[t+1], float64), one CTA
// per output row: the row is carried through the chain in shared memory;
// each product splits the sum over l across 8 thread slices (independent
// load chains), reduced in shared memory in a fixed order.
struct GramChainArgs {
    const double* F[RTR_MAXN];
    int dim[RTR_MAXN + 1];
    int cnt;
    double* out;
    float* outf;              // optional float32 copy of out (converted here, on 100 SMs, not
                              // in the single-CTA kernels: float64 conversions are slow)
    float* outl;              // optional low part: out - (double)outf, as float32
    int reindex, Rb, Rn;      // reindex: write G[(b, a), (b', a')] = M[(b, b'), (a, a')]
};
constexpr int GC_THREADS = 1024;
constexpr int GC_COLS = GC_THREADS / 8;
__global__ void __launch_bounds__(GC_THREADS) gram_chain_kernel(const GramChainArgs g) {
    __shared__ double v0[256], v1[256];
    __shared__ double part[8][GC_COLS];
    const int r = blockIdx.x;
    const int tid = threadIdx.x, jl = tid % GC_COLS, q = tid / GC_COLS;
    int len = g.dim[1];
    for (int j = tid; j < len; j += blockDim.x) v0[j] = g.F[0][(int64_t)r * len + j];
    double* cur = v0;
    double* nxt = v1;
    for (int t = 1; t < g.cnt; ++t) {
        __syncthreads();
        const int cols = g.dim[t + 1];
        const double* Em = g.F[t];
        for (int j0 = 0; j0 < cols; j0 += GC_COLS) {
            const int j = j0 + jl;
            double s = 0.0;
            if (j < cols)
                for (int l = q; l < len; l += 8) s = fma(cur[l], Em[(int64_t)l * cols + j], s);
            part[q][jl] = s;
            __syncthreads();
            if (q == 0 && j < cols) {
                double t2 = part[0][jl];
#pragma unroll
                for (int u = 1; u < 8; ++u) t2 += part[u][jl];
                nxt[j] = t2;
            }
            __syncthreads();
        }
        double* tmp = cur; cur = nxt; nxt = tmp;
        len = cols;
    }
    __syncthreads();
    if (g.reindex) {
        const int C = g.Rb * g.Rn;
        const int be = r / g.Rb, be2 = r % g.Rb;
        for (int j = threadIdx.x; j < len; j += blockDim.x) {
            const int al = j / g.Rn, al2 = j % g.Rn;
            const int64_t o = (int64_t)(be * g.Rn + al) * C + be2 * g.Rn + al2;
            g.out[o] = cur[j];
            if (g.outf) {
                const float h = (float)cur[j];
                g.outf[o] = h;
                if (g.outl) g.outl[o] = (float)(cur[j] - (double)h);
            }
        }
    } else {
        for (int j = threadIdx.x; j < len; j += blockDim.x) g.out[(int64_t)r * len + j] = cur[j];
    }
}

__global__ void to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}

constexpr int SOLVE_MAXC = 160;       // R_n R_{n+1} <= 144

// Inverse of the Gram matrix of one core update, once per update (one CTA,
// run on the plan's side stream so that it overlaps the contraction).
// G (its float32 copy, C x C, (beta, alpha) order) is equilibrated, A = D G D with
// D = diag(G)^-1/2 in float32, and inverted in place by the sweep operator
// (Goodnight 1979): sweeping pivot k maps
//     a_kk -> -1/a_kk,  a_ik -> a_ik/a_kk,  a_kj -> a_kj/a_kk,
//     a_ij -> a_ij - a_ik a_kj / a_kk          (i, j != k),
// and sweeping every pivot of a positive definite A leaves -A^-1.  The pivots
// are the Schur-complement diagonals, i.e. the squared Cholesky pivots, so a
// pivot that is not positive means A is not numerically positive definite:
// the kernel then raises *need_slow and writes nothing (the float64 slow path
// takes over).  Writes Ginv = D A^-1 D (float32, C x C).
//
// 256 threads as a 16 x 16 grid; thread (ti, tj) keeps in registers the
// elements (ti + 16 m, tj + 16 m'), m, m' < T (T = ceil(C / 16) <= 9), so a
// pivot step costs T^2 register FMAs and 2T shared loads per thread; the
// pivot column travels through a double-buffered shared vector (one barrier
// per pivot).
template <int T>
__global__ void __launch_bounds__(256) gram_inverse_kernel(const float* __restrict__ G, int C,
                                                           float* __restrict__ Ginv, int* __restrict__ need_slow) {
    __shared__ float v[2][16 * T];
    __shared__ float sc[16 * T];
    const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
    // this kernel is the flag's only writer in an update, and runs after the
    // previous update's solve (stream order): clear it for this update
    if (tid == 0) *need_slow = 0;
    int ok = 1;
    for (int c = tid; c < 16 * T; c += blockDim.x) {
        float s = 0.f;
        if (c < C) {
            const float d = G[(int64_t)c * C + c];
            s = (d > 0.f && isfinite(d)) ? rsqrtf(d) : 0.f;
            if (!(s > 0.f)) ok = 0;
        }
        sc[c] = s;
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicExch(need_slow, 1);
        return;
    }
    float a[T][T];
#pragma unroll
    for (int m = 0; m < T; ++m) {
#pragma unroll
        for (int mm = 0; mm < T; ++mm) {
            const int r = ti + 16 * m, c = tj + 16 * mm;
            float x = 0.f;
            if (r < C && c < C) {
                // the upper triangle (min, max) for both (r, c) and (c, r): exactly symmetric
                const int lo = min(r, c), hi = max(r, c);
                x = (G[(int64_t)lo * C + hi] * sc[lo]) * sc[hi];
                if (!isfinite(x)) ok = 0;
            }
            a[m][mm] = x;
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicExch(need_slow, 1);
        return;
    }
    int buf = 0;
#pragma unroll
    for (int M = 0; M < T; ++M) {
        if (16 * M >= C) break;
        for (int kk = 0; kk < 16; ++kk) {
            const int k = 16 * M + kk;
            if (k >= C) break;
            // owners of column k publish it (padding rows hold 0)
            if (tj == kk) {
#pragma unroll
                for (int m = 0; m < T; ++m) v[buf][ti + 16 * m] = a[m][M];
            }
            __syncthreads();
            const float d = v[buf][k];
            if (!(d > 0.f) || !isfinite(d)) {          // same value in every thread: uniform exit
                if (tid == 0) atomicExch(need_slow, 1);
                return;
            }
            float inv;                                     // hardware reciprocal: the refinement absorbs its error
            asm("rcp.approx.f32 %0, %1;" : "=f"(inv) : "f"(d));
            float vi[T], vj[T];
#pragma unroll
            for (int m = 0; m < T; ++m) {
                vi[m] = v[buf][ti + 16 * m] * inv;
                vj[m] = v[buf][tj + 16 * m];
            }
#pragma unroll
            for (int m = 0; m < T; ++m) {
#pragma unroll
                for (int mm = 0; mm < T; ++mm) a[m][mm] = fmaf(-vi[m], vj[mm], a[m][mm]);
            }
            // column k and row k of the sweep (2 lanes per warp, resp. one warp)
            if (tj == kk) {
#pragma unroll
                for (int m = 0; m < T; ++m) a[m][M] = vi[m];
            }
            if (ti == kk) {
#pragma unroll
                for (int mm = 0; mm < T; ++mm) a[M][mm] = vj[mm] * inv;
                if (tj == kk) a[M][M] = -inv;
            }
            buf ^= 1;
        }
    }
#pragma unroll
    for (int m = 0; m < T; ++m) {
#pragma unroll
        for (int mm = 0; mm < T; ++mm) {
            const int r = ti + 16 * m, c = tj + 16 * mm;
            if (r < C && c < C) Ginv[(int64_t)r * C + c] = -a[m][mm] * sc[r] * sc[c];
        }
    }
}

// Slow path of a core update (one CTA, run by the solve kernel's first CTA
// when the Gram inverse raised *need_slow): float64
// Cholesky of G in shared memory and direct solves, or, if G is not SPD in
// float64 either, the eigen-pseudo-inverse with cutoff 1e-13 lambda_max
// (Jacobi eigendecomposition in global scratch).
__device__ void solve_slow_body(const double* __restrict__ Mprod, int Rn, int Rn1,
                                                             int In, const double* __restrict__ W,
                                                             double* __restrict__ Wz, double* __restrict__ Zn,
                                                             float* __restrict__ Znf, double* __restrict__ zw_out,
                                                             double* __restrict__ jac_ws, int* __restrict__ need_slow,
                                                             int* __restrict__ flags) {
    extern __shared__ __align__(16) double Gs[];
    const int C = Rn * Rn1;
    const int ld = C + 1;
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) Gs[(e / C) * ld + e % C] = Mprod[e];
    for (int e = threadIdx.x; e < In * C; e += blockDim.x) Wz[e] = W[e];
    __syncthreads();
    int ok = 1;
    for (int e = threadIdx.x; e < C * C; e += blockDim.x)
        if (!isfinite(Gs[(e / C) * ld + e % C])) ok = 0;
    ok = __syncthreads_and(ok);
    if (ok) ok = rtr::block_cholesky(Gs, C, ld) ? 1 : 0;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (ok) {
        for (int i = warp; i < In; i += nw) rtr::warp_chol_solve(Gs, C, ld, Wz + (int64_t)i * C);
        __syncthreads();
    } else {
        // pseudo-inverse with cutoff 1e-13 * lambda_max (Jacobi eigendecomposition)
        if (threadIdx.x == 0) atomicOr(flags, RTR_FLAG_GRAM_PINV);
        double* Aj = jac_ws;
        double* V = jac_ws + (int64_t)C * C;
        __shared__ int pairs[2 * 160];
        __shared__ double cs[2 * 160];
        for (int e = threadIdx.x; e < C * C; e += blockDim.x) Aj[e] = Mprod[e];
        __syncthreads();
        rtr::block_jacobi_eig<double>(Aj, V, C, C, pairs, cs, 40, 1e-30);
        double lmax = 0.0;
        for (int c = 0; c < C; ++c) lmax = fmax(lmax, Aj[c * C + c]);
        const double cut = 1e-13 * lmax;
        // z = w V diag(1/lambda) V^T  (row vectors), using Wz as scratch per row
        for (int i = 0; i < In; ++i) {
            __shared__ double t[160];
            for (int c = threadIdx.x; c < C; c += blockDim.x) {
                double s = 0.0;
                for (int l = 0; l < C; ++l) s += W[(int64_t)i * C + l] * V[l * C + c];
                const double lam = Aj[c * C + c];
                t[c] = (lam > cut) ? s / lam : 0.0;
            }
            __syncthreads();
            for (int c = threadIdx.x; c < C; c += blockDim.x) {
                double s = 0.0;
                for (int l = 0; l < C; ++l) s += t[l] * V[c * C + l];
                Wz[(int64_t)i * C + c] = s;
            }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < In * C; e += blockDim.x) {
        const int i = e / C, c = e % C;
        const int be = c / Rn, al = c % Rn;
        Zn[((int64_t)al * In + i) * Rn1 + be] = Wz[e];
        if (Znf) Znf[((int64_t)al * In + i) * Rn1 + be] = (float)Wz[e];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < In; i += blockDim.x) {
        double zw = 0.0;
        for (int c = 0; c < C; ++c) zw += Wz[(int64_t)i * C + c] * W[(int64_t)i * C + c];
        zw_out[i] = zw;
    }
    __syncthreads();
    (void)need_slow;
}

// Core update for slice i of mode n (one CTA per slice): z_i solves
// G z_i = w_i by iterative refinement (Wilkinson; Moler 1967) with the
// float32 inverse from gram_inverse_kernel:
//     z <- z + Ginv (w - G z),
// until ||dz|| <= sqrt(tol2) ||z||, the corrections stop shrinking (the
// rounding floor of the residual), or max_it steps.  z, w and the residual
// are kept as unevaluated float pairs (hi + lo, "double-float", Dekker 1971):
// the residual sum over l of G[c][l] z[l] uses G = Gh + Gl from the Gram
// kernel, error-free products (fma) and two-sum accumulation, about 2^-44
// relative to sum |G z|, all on the FP32 pipe (GB300's float64 rate is far
// lower).  Skips the slice if the inverse raised *need_slow (the slow path
// solves every slice then).  Ginv is staged in shared memory; each product is
// split over the 8 lanes of an aligned lane group (output c = group).
// Writes Z_n[alpha, i, beta] and zw[i] = z_i . w_i.
constexpr int SOLVE_THREADS = 1024;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__global__ void __launch_bounds__(SOLVE_THREADS) als_solve_inv_kernel(
    const float* __restrict__ Gh, const float* __restrict__ Gl, const float* __restrict__ Ginv, int Rn, int Rn1,
    int In, const double* __restrict__ W, double* __restrict__ Zn, float* __restrict__ Znf,
    double* __restrict__ zw_out, int* __restrict__ need_slow, float tol2, int max_it,
    const double* __restrict__ G, double* __restrict__ Wz, double* __restrict__ jac, int* __restrict__ flags) {
    extern __shared__ __align__(16) float gi[];          // C x C (the slow path: C x (C + 1) float64)
    __shared__ float wh[SOLVE_MAXC], wl[SOLVE_MAXC], zh[SOLVE_MAXC], zl[SOLVE_MAXC], rf[SOLVE_MAXC];
    __shared__ float redf[2][32];
    __shared__ double red[32];
    if (*(volatile const int*)need_slow) {
        // the inverse met a non-positive pivot: the first CTA solves every slice in float64
        if (blockIdx.x == 0) solve_slow_body(G, Rn, Rn1, In, W, Wz, Zn, Znf, zw_out, jac, need_slow, flags);
        return;
    }
    const int C = Rn * Rn1;
    const int i = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = tid & 7, grp = tid >> 3, ngrp = SOLVE_THREADS / 8;
    for (int e = tid; e < C * C; e += SOLVE_THREADS) gi[e] = Ginv[e];
    for (int c = tid; c < C; c += SOLVE_THREADS) {
        const double wd = W[(int64_t)i * C + c];
        const float h = (float)wd;
        wh[c] = h;
        wl[c] = (float)(wd - (double)h);
        zh[c] = 0.f;
        zl[c] = 0.f;
        rf[c] = h;
    }
    __syncthreads();
    float dz2_prev = 0.f;
    for (int it = 0; it < max_it; ++it) {
        // dz = Ginv r (float32; rows of the symmetric inverse read as columns), z += dz
        float d2 = 0.f, n2 = 0.f;
        for (int c0 = 0; c0 < C; c0 += ngrp) {          // every lane reaches the shuffles
            const int c = c0 + grp;
            float acc = 0.f;
            if (c < C)
                for (int l = q; l < C; l += 8) acc = fmaf(gi[l * C + c], rf[l], acc);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 4);
            if (q == 0 && c < C) {
                float sh, se;
                two_sum(zh[c], acc, sh, se);
                const float lo = zl[c] + se;
                const float nh = sh + lo;
                zh[c] = nh;
                zl[c] = lo - (nh - sh);
                d2 += acc * acc;
                n2 += nh * nh;
            }
        }
        // convergence sums (float32 is ample for a stopping test)
        d2 = rtr::warp_sum(d2);
        n2 = rtr::warp_sum(n2);
        if (lane == 0) { redf[0][warp] = d2; redf[1][warp] = n2; }
        __syncthreads();                                  // z complete, r no longer read
        float dz2 = 0.f, z2 = 0.f;
        for (int u = 0; u < SOLVE_THREADS / 32; ++u) { dz2 += redf[0][u]; z2 += redf[1][u]; }
        const bool conv = dz2 <= tol2 * z2 || (it >= 2 && dz2 > 0.25f * dz2_prev);
        dz2_prev = dz2;
        if (conv || it + 1 == max_it) break;              // uniform: every thread has the same sums
        // r = w - G z in double-float
        for (int c0 = 0; c0 < C; c0 += ngrp) {
            const int c = c0 + grp;
            float S = 0.f, E = 0.f;
            if (c < C) {
                const float* gh = Gh + (int64_t)c * C;
                const float* gl = Gl + (int64_t)c * C;
                for (int l = q; l < C; l += 8) {
                    const float a = gh[l], b = zh[l];
                    const float p = a * b;
                    const float pe = fmaf(a, b, -p);              // a b = p + pe exactly
                    float t;
                    two_sum(S, p, S, t);
                    E += t + pe;
                    E = fmaf(a, zl[l], E);
                    E = fmaf(gl[l], b, E);
                }
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const float S2 = __shfl_xor_sync(0xffffffffu, S, o);
                const float E2 = __shfl_xor_sync(0xffffffffu, E, o);
                float t;
                two_sum(S, S2, S, t);
                E += E2 + t;
            }
            if (q == 0 && c < C) {
                float rh, t;
                two_sum(wh[c], -S, rh, t);
                rf[c] = rh + ((wl[c] - E) + t);
            }
        }
        __syncthreads();
    }
    double zw = 0.0;
    for (int c = tid; c < C; c += SOLVE_THREADS) {
        const int be = c / Rn, al = c % Rn;
        const int64_t o = ((int64_t)al * In + i) * Rn1 + be;
        const double zd = (double)zh[c] + (double)zl[c];
        Zn[o] = zd;
        if (Znf) Znf[o] = zh[c] + zl[c];
        zw += zd * ((double)wh[c] + (double)wl[c]);
    }
    zw = rtr::block_sum(zw, red);
    if (tid == 0) zw_out[i] = zw;
}

// ||P - TR(Z)|| after the last update of a sweep: sqrt(||P||^2 - sum_i z_i . w_i)
// (at the least-squares solution ||TR(Z)||^2 = sum_i z_i . w_i).
__global__ void als_err_kernel(const double* __restrict__ zw, int In, const double* __restrict__ normP2,
                               double* __restrict__ err_out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < In; ++i) s += zw[i];
        *err_out = sqrt(fmax(*normP2 - s, 0.0));
    }
}


// Default start: entry e of core n is the fp64 table value at field e % 20 of
// Philox4x64-10(counter (e/20, 0, 0, 0), key (seed + 1, 256 + n)).
__global__ void init_core_kernel(double* __restrict__ Z, int64_t count, uint64_t seed, int n,
                                 const double* __restrict__ tab) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t c0 = (uint64_t)(e / 20), c1 = 0, c2 = 0, c3 = 0;
        rtr::philox4x64_10(c0, c1, c2, c3, seed + 1, 256 + (uint64_t)n);
        const uint64_t w[4] = {c0, c1, c2, c3};
        Z[e] = tab[rtr::omega_field(w, (int)(e % 20))];
    }
}

// scale every core by (||P|| / ||TR(Z)||)^(1/N)
__global__ void scale_cores_kernel(double* __restrict__ Z, int64_t count, const double* __restrict__ normP2,
                                   const double* __restrict__ normTR2, int N) {
    const double s = pow(sqrt(*normP2) / sqrt(fmax(*normTR2, 1e-300)), 1.0 / N);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        Z[e] *= s;
}

__global__ void backproject_kernel(const double* __restrict__ Z, const double* __restrict__ Q, double* __restrict__ G,
                                   int Ra, int K, int I, int Rb) {
    const int64_t total = (int64_t)Ra * I * Rb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e % Rb), i = (int)((e / Rb) % I), a = (int)(e / ((int64_t)Rb * I));
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += Z[((int64_t)a * K + k) * Rb + b] * Q[(int64_t)i * K + k];
        G[e] = s;
    }
}

// transpose each R1 x R2 block of rows: out[r, y, x] = in[r, x, y]
template <typename T>
__global__ void block_transpose_kernel(const T* __restrict__ in, int64_t rows, int R1, int R2, T* __restrict__ out) {
    const int64_t total = rows * R1 * R2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(e % R1);
        const int x = (int)((e / R1) % R2);
        const int64_t r = e / ((int64_t)R1 * R2);
        out[e] = in[(r * R1 + y) * R2 + x];
    }
}

// C[m][n] = sum_k A[m][k] * Bt[n][k], 64x64 tiles, 4x4 per thread.
template <typename T>
__global__ void __launch_bounds__(256) nt_gemm_kernel(const T* __restrict__ A, const T* __restrict__ Bt,
                                                      T* __restrict__ Cm, int64_t M, int64_t N, int Kd) {
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < Kd; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int r = e / 16, k = e % 16;
            As[k][r] = (m0 + r < M && k0 + k < Kd) ? A[(m0 + r) * Kd + k0 + k] : T(0);
            Bs[k][r] = (n0 + r < N && k0 + k < Kd) ? Bt[(n0 + r) * Kd + k0 + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t m = m0 + ty + 16 * a, n = n0 + tx + 16 * b;
            if (m < M && n < N) Cm[m * N + n] = acc[a][b];
        }
}

template <typename T>
__global__ void sqdiff_kernel(const T* __restrict__ P, const double* __restrict__ D, int64_t n, double* __restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)P[e] - D[e];
        s += d * d;
    }
    s = rtr::block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// one CTA: e2 = sum of the partials (block_sum's fixed order), then the RSE
__global__ void rse_final_kernel(const double* __restrict__ part, int nparts, const double* __restrict__ normX2,
                                 const double* __restrict__ normP2, double* __restrict__ out) {
    __shared__ double red[32];
    double e2 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) e2 += part[i];
    e2 = rtr::block_sum(e2, red);
    if (threadIdx.x == 0) {
        const double x2 = *normX2;
        *out = sqrt(fmax(x2 - *normP2 + e2, 0.0) / x2);
    }
}

__global__ void draw_omega_kernel(double* __restrict__ out, int64_t row0, int64_t nrows, int K, uint64_t seed,
                                  int mode, const double* __restrict__ tab64, const float* __restrict__ tab32,
                                  const uint16_t* __restrict__ tab16, int use64) {
    const int ncalls = (K + 19) / 20;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nrows * ncalls;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rr = w / ncalls;
        const int cb = (int)(w % ncalls);
        uint64_t wd[4];
        rtr::omega_words(seed, mode, (uint64_t)(row0 + rr), (uint64_t)cb, wd);
        for (int t = 0; t < 20; ++t) {
            const int k = cb * 20 + t;
            if (k < K) {
                const int j = rtr::omega_field(wd, t);
                out[rr * K + k] = use64 ? tab64[j]
                                  : tab16 ? (double)__uint_as_float((uint32_t)tab16[j] << 16)   // bfloat16 bits
                                          : (double)tab32[j];
            }
        }
    }
}

inline unsigned grid_for(int64_t n, int threads = 256, int64_t cap = 65535) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(rtr_ceil_div(n, threads), cap));
}

// ---- fused subchain and contraction (float32 plans) --------------------------
// W = P_<n> S_{!=n} (Eq. 2 and the update below it) without storing the
// subchain S: its slice for the other modes' indices j is the matrix product
// Z_{n+1}(j_{n+1}) ... Z_{n-1}(j_{n-1}) (R_{n+1} x R_n), and
//     W[i, be R_n + g] = sum_j P[.., i, ..](j) S(j)[be, g].
// The chain's cores before the last one are the "outer" modes, the last core
// (mode n-1) the "inner" one.  A CTA takes a contiguous range of outer
// multi-indices o in batches of up to gb; per batch it forms, in shared
// memory, M(o) = Z_{n+1}(j_{n+1}) ... Z_{n-2}(j_{n-2}), the slices
// S(o, l) = M(o) Z_{n-1}(l) for every inner index l, and the K_n x K_{n-1}
// blocks of P that meet them, then adds the block products to float32
// accumulators: a thread owns a 4 x 4 tile of W (4 rows i, 4 columns) and
// reads 4 + 4 values per 16 FMAs.  The products associate as in the stored
// subchain ((Z_{n+1} Z_{n+2}) Z_{n+3} ...).  Each CTA writes its partial W in
// float64; fused_reduce_kernel sums the partials in a fixed order.
constexpr int FC_THREADS = 256;
constexpr int FC_MAXB = 8;           // outer indices per batch

struct FusedContractArgs {
    const float* P;
    const float* Z[RTR_MAXN];   // chain order: Z[t] = core (n + 1 + t) mod N
    int R[RTR_MAXN + 1];        // R[t] x K[t] x R[t + 1] = shape of Z[t]; R[0] = R_{n+1}, R[L] = R_n
    int K[RTR_MAXN];
    int64_t st[RTR_MAXN];       // stride in P of chain core t's index
    int L;                      // chain length N - 1 (>= 2)
    int Kn;                     // K_n
    int64_t stn;                // stride in P of mode n
    int64_t nouter;             // product of K[0 .. L-2]
    int C, C4, Kn4, Rn4;        // R_{n+1} R_n, and C, K_n, R_n rounded up to multiples of 4
    int gb;                     // outer indices per batch (<= FC_MAXB)
    double* partial;            // gridDim.x x (K_n C)
};

// 4-byte asynchronous copy global -> shared (zero-filled when !valid), so
// that a thread's gathers are all in flight at once
__device__ __forceinline__ void fc_cp4(float* dst, const float* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void fc_cp_wait() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int NT>
__global__ void __launch_bounds__(FC_THREADS) fused_contract_kernel(const FusedContractArgs a) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ int64_t off_s[FC_MAXB];
    __shared__ int jo_s[FC_MAXB][RTR_MAXN];
    const int L = a.L, KL = a.K[L - 1], Rl = a.R[L - 1], Rn = a.R[L], R0 = a.R[0];
    const int C = a.C, C4 = a.C4, Kn = a.Kn, Kn4 = a.Kn4, Rn4 = a.Rn4, GB = a.gb;
    float* zl = fsm;                                   // inner core, Rl x KL x Rn4 (g >= Rn zero)
    float* mb = zl + Rl * KL * Rn4;                    // 2 x GB x 256: M of each outer index
    float* Pb = mb + 2 * GB * 256;                     // GB x KL x Kn4: P blocks, i fastest
    float* Sb = Pb + GB * KL * Kn4;                    // GB x KL x C4: slices of S
    float* zs = Sb + GB * KL * C4;                     // (L - 1) x GB x 256: the outer cores' slices
    const int tid = threadIdx.x;
    // every global read of the kernel is an asynchronous copy, issued before
    // the first use: the gathers of a batch wait for one L2 latency, not for
    // one per element a thread reads
    for (int e = tid; e < Rl * KL * Rn4; e += FC_THREADS) {
        const int g = e % Rn4, hl = e / Rn4;
        fc_cp4(zl + e, g < Rn ? a.Z[L - 1] + (int64_t)hl * Rn + g : a.Z[L - 1], g < Rn);
    }
    const int64_t per = a.nouter / gridDim.x, rem = a.nouter % gridDim.x;
    const int64_t o0 = blockIdx.x * per + min((int64_t)blockIdx.x, rem);
    const int64_t o1 = o0 + per + ((int64_t)blockIdx.x < rem ? 1 : 0);
    const int ti4 = Kn4 >> 2, tc4 = C4 >> 2, ntile = ti4 * tc4;
    float acc[NT][4][4];
#pragma unroll
    for (int q = 0; q < NT; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[q][u][0] = acc[q][u][1] = acc[q][u][2] = acc[q][u][3] = 0.f;

    for (int64_t ob = o0; ob < o1; ob += GB) {
        const int gb = (int)min((int64_t)GB, o1 - ob);
        __syncthreads();                               // the previous batch's readers are done
        if (tid < gb) {
            int64_t off = 0, rest = ob + tid;
            for (int t = L - 2; t >= 0; --t) {
                const int j = (int)(rest % a.K[t]);
                rest /= a.K[t];
                jo_s[tid][t] = j;
                off += (int64_t)j * a.st[t];
            }
            off_s[tid] = off;
        }
        __syncthreads();
        // P blocks (the inner index fastest in the reads), i fastest in shared memory
        for (int e = tid; e < gb * Kn4 * KL; e += FC_THREADS) {
            const int l = e % KL, r = e / KL, i = r % Kn4, b = r / Kn4;
            fc_cp4(Pb + (b * KL + l) * Kn4 + i,
                   i < Kn ? a.P + off_s[b] + (int64_t)l * a.st[L - 1] + (int64_t)i * a.stn : a.P, i < Kn);
        }
        // the outer cores' slices Z[t](j_t) (R[t] x R[t+1]) of every outer index
        for (int t = 0; t < L - 1; ++t) {
            const int Rt = a.R[t], Rt1 = a.R[t + 1];
            for (int e = tid; e < gb * Rt * Rt1; e += FC_THREADS) {
                const int b = e / (Rt * Rt1), hc = e - b * Rt * Rt1, h = hc / Rt1, c = hc - h * Rt1;
                fc_cp4(zs + (t * GB + b) * 256 + hc, a.Z[t] + ((int64_t)h * a.K[t] + jo_s[b][t]) * Rt1 + c, true);
            }
        }
        fc_cp_wait();
        __syncthreads();
        // M(o) = Z[0](j_0) ... Z[L-2](j_{L-2})   (R0 x Rl)
        int mw = 0;
        {
            const int R1 = a.R[1];
            for (int e = tid; e < gb * R0 * R1; e += FC_THREADS) {
                const int b = e / (R0 * R1), rc = e - b * R0 * R1;
                mb[b * 256 + rc] = zs[b * 256 + rc];
            }
            for (int t = 1; t < L - 1; ++t) {
                __syncthreads();
                const int Rt = a.R[t], Rt1 = a.R[t + 1];
                const float* cur = mb + mw * GB * 256;
                float* nxt = mb + (mw ^ 1) * GB * 256;
                for (int e = tid; e < gb * R0 * Rt1; e += FC_THREADS) {
                    const int b = e / (R0 * Rt1), rc = e - b * R0 * Rt1, r = rc / Rt1, c = rc - r * Rt1;
                    const float* zt = zs + (t * GB + b) * 256 + c;
                    float v = 0.f;
                    for (int h = 0; h < Rt; ++h) v = fmaf(cur[b * 256 + r * Rt + h], zt[h * Rt1], v);
                    nxt[b * 256 + rc] = v;
                }
                mw ^= 1;
            }
        }
        __syncthreads();
        // S(o, l)[be, g] = sum_h M(o)[be, h] Z_{n-1}[h, l, g]: a thread per (o, l, be)
        // keeps the R_n sums of its row in registers
        const float* M = mb + mw * GB * 256;
        for (int e = tid; e < gb * KL * R0; e += FC_THREADS) {
            const int be = e % R0, bl = e / R0, l = bl % KL, b = bl / KL;
            float v[16];
#pragma unroll
            for (int g = 0; g < 16; ++g) v[g] = 0.f;
            for (int h = 0; h < Rl; ++h) {
                const float mv = M[b * 256 + be * Rl + h];
                const float4* zr = reinterpret_cast<const float4*>(zl + (h * KL + l) * Rn4);
#pragma unroll
                for (int g4 = 0; g4 < 4; ++g4)
                    if (4 * g4 < Rn) {
                        const float4 z = zr[g4];
                        v[4 * g4] = fmaf(mv, z.x, v[4 * g4]); v[4 * g4 + 1] = fmaf(mv, z.y, v[4 * g4 + 1]);
                        v[4 * g4 + 2] = fmaf(mv, z.z, v[4 * g4 + 2]); v[4 * g4 + 3] = fmaf(mv, z.w, v[4 * g4 + 3]);
                    }
            }
            float* so = Sb + bl * C4 + be * Rn;
#pragma unroll
            for (int g = 0; g < 16; ++g)
                if (g < Rn) so[g] = v[g];
        }
        if (C4 > C)
            for (int e = tid; e < gb * KL * (C4 - C); e += FC_THREADS)
                Sb[(e / (C4 - C)) * C4 + C + e % (C4 - C)] = 0.f;
        __syncthreads();
        // acc[tile] += sum over (o, l) of Pb[o, l, i0 .. i0 + 3]^T Sb[o, l, c0 .. c0 + 3]
        const int nk = gb * KL;
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const int tl = tid + FC_THREADS * q;
            if (NT > 1 && tl >= ntile) break;
            if (tl < ntile) {
                const int i0 = 4 * (tl / tc4), c0 = 4 * (tl % tc4);
                const float* pa = Pb + i0;
                const float* sa = Sb + c0;
#pragma unroll 4
                for (int k = 0; k < nk; ++k) {
                    const float4 pv = *reinterpret_cast<const float4*>(pa + k * Kn4);
                    const float4 sv = *reinterpret_cast<const float4*>(sa + k * C4);
                    const float pp[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc[q][u][0] = fmaf(pp[u], sv.x, acc[q][u][0]);
                        acc[q][u][1] = fmaf(pp[u], sv.y, acc[q][u][1]);
                        acc[q][u][2] = fmaf(pp[u], sv.z, acc[q][u][2]);
                        acc[q][u][3] = fmaf(pp[u], sv.w, acc[q][u][3]);
                    }
                }
            }
        }
    }
    double* dst = a.partial + (int64_t)blockIdx.x * Kn * C;
#pragma unroll
    for (int q = 0; q < NT; ++q) {
        const int tl = tid + FC_THREADS * q;
        if (tl < ntile) {
            const int i0 = 4 * (tl / tc4), c0 = 4 * (tl % tc4);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (i0 + u < Kn && c0 + w < C) dst[(int64_t)(i0 + u) * C + c0 + w] = (double)acc[q][u][w];
        }
    }
}

// W[e] = sum of the partials: thread (g, x) of a CTA adds partials g, g + 8,
// ... of output e = 32 blockIdx.x + x (consecutive x: consecutive addresses),
// then the 8 group sums are added in order (the result does not depend on timing)
__global__ void __launch_bounds__(256) fused_reduce_kernel(const double* __restrict__ partial, int nparts, int count,
                                                           double* __restrict__ W) {
    __shared__ double red[8][33];
    const int x = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + x;
    double s = 0.0;
    if (e < count)
        for (int q = g; q < nparts; q += 8) s += partial[(int64_t)q * count + e];
    red[g][x] = s;
    __syncthreads();
    if (g == 0 && e < count) {
        double t = red[0][x];
#pragma unroll
        for (int u = 1; u < 8; ++u) t += red[u][x];
        W[e] = t;
    }
}

// shared memory of the fused contraction for batches of gb outer indices
size_t fused_contract_smem(int N, const int64_t* Kd, const int* R, int n, int gb) {
    const int m_last = (n + N - 1) % N;
    const size_t KL = (size_t)Kd[m_last], Rl = (size_t)R[m_last];
    const size_t Rn4 = (size_t)((R[n] + 3) & ~3), Kn4 = (size_t)((Kd[n] + 3) & ~3);
    const size_t C4 = (size_t)((R[(n + 1) % N] * R[n] + 3) & ~3);
    return sizeof(float) * (Rl * KL * Rn4 + 2 * (size_t)gb * 256 + (size_t)gb * KL * (Kn4 + C4) +
                            (size_t)(N - 2) * gb * 256);
}

constexpr size_t FC_SMEM_LIMIT = 200 * 1024;

// 0 if the fused form applies (every size within its shared memory and
// register tiling), else nonzero (the caller keeps the stored subchain then)
int fused_contract_ok(rtr_plan* p, int n) {
    const int N = p->N;
    int64_t Kd[RTR_MAXN];
    for (int m = 0; m < N; ++m) Kd[m] = p->K[m];
    if (N < 3) return 1;
    for (int m = 0; m < N; ++m) if (p->R[m] > 16) return 1;
    const int C4 = (p->R[(n + 1) % N] * p->R[n] + 3) & ~3;
    const int ntile = (int)(((Kd[n] + 3) & ~3) >> 2) * (C4 >> 2);
    if (ntile > 4 * FC_THREADS) return 1;
    if (fused_contract_smem(N, Kd, p->R, n, 1) > FC_SMEM_LIMIT) return 1;
    return 0;
}

int launch_fused_contract(rtr_plan* p, const float* P, const float* const* Zf, int n, double* W, cudaStream_t s) {
    const int N = p->N;
    int64_t Kd[RTR_MAXN];
    for (int m = 0; m < N; ++m) Kd[m] = p->K[m];
    FusedContractArgs a{};
    a.P = P;
    a.L = N - 1;
    int64_t stride[RTR_MAXN];
    stride[N - 1] = 1;
    for (int m = N - 2; m >= 0; --m) stride[m] = stride[m + 1] * Kd[m + 1];
    for (int t = 0; t < a.L; ++t) {
        const int m = (n + 1 + t) % N;
        a.Z[t] = Zf[m];
        a.R[t] = p->R[m];
        a.K[t] = (int)Kd[m];
        a.st[t] = stride[m];
    }
    a.R[a.L] = p->R[n];
    a.Kn = (int)Kd[n];
    a.stn = stride[n];
    a.nouter = 1;
    for (int t = 0; t + 1 < a.L; ++t) a.nouter *= a.K[t];
    a.C = p->R[(n + 1) % N] * p->R[n];
    a.C4 = (a.C + 3) & ~3;
    a.Kn4 = (a.Kn + 3) & ~3;
    a.Rn4 = (p->R[n] + 3) & ~3;
    const int count = a.Kn * a.C;
    int64_t gx = std::min<int64_t>(a.nouter, (int64_t)p->num_sms);
    gx = std::min<int64_t>(gx, (int64_t)(p->partial_elems / (size_t)count));
    if (gx < 1) return rtr_set_error(RTR_ENOMEM, "TR-ALS: contraction partials exceed the plan workspace");
    // one batch per CTA where shared memory allows
    int gb = (int)std::min<int64_t>(FC_MAXB, rtr_ceil_div(a.nouter, gx));
    while (gb > 1 && fused_contract_smem(N, Kd, p->R, n, gb) > FC_SMEM_LIMIT) --gb;
    a.gb = gb;
    a.partial = p->partial;
    const size_t smem = fused_contract_smem(N, Kd, p->R, n, gb);
    const int ntile = (a.Kn4 >> 2) * (a.C4 >> 2);
    const int nt = (ntile + FC_THREADS - 1) / FC_THREADS;
#define RTR_FC(NT_)                                                                                       \
    if (nt <= NT_) {                                                                                      \
        RTR_SMEM(fused_contract_kernel<NT_>, smem);                                                        \
        fused_contract_kernel<NT_><<<(unsigned)gx, FC_THREADS, smem, s>>>(a);                             \
    } else
    RTR_FC(1) RTR_FC(2) RTR_FC(4) { return rtr_set_error(RTR_EINVAL, "TR-ALS: fused contraction too wide"); }
#undef RTR_FC
    RTR_LAUNCH_CHECK("fused_contract_kernel");
    fused_reduce_kernel<<<(unsigned)rtr_ceil_div(count, 32), 256, 0, s>>>(p->partial, (int)gx, count, W);
    RTR_LAUNCH_CHECK("fused_reduce_kernel");
    return RTR_OK;
}

// Build subchain products over `cores` in ring order start, start+1, ...,
// start+count-1 (indices mod N); writes the product slices for every
// multi-index (row-major) as rows x Rfirst x Rlast into one of two buffers,
// returns the buffer holding the result.  final_tr permutes rows as above.
template <typename T, typename TZ = double>
T* build_chain(int N, const int64_t* dims, const int* R, const TZ* const* Z, int start, int count,
               T* buf0, T* buf1, int final_tr, int64_t Aa, int64_t Bb, cudaStream_t s, int* status) {
    T* cur = nullptr;
    T* bufs[2] = {buf0, buf1};
    int which = 0;
    int64_t Jp = 1;
    const int Rfirst = R[start % N];
    const TZ* zfirst = nullptr;
    int t0 = 0;
    if (count >= 2) {          // fold the first core into the first product
        zfirst = Z[start % N];
        Jp = dims[start % N];
        t0 = 1;
    }
    for (int t = t0; t < count; ++t) {
        const int m = (start + t) % N;
        const int Km = (int)dims[m];
        const int Rc = R[m], Rd = R[(m + 1) % N];
        T* out = bufs[which];
        const int fin = (t == count - 1) ? final_tr : 0;
        const int64_t total = Jp * Km * Rfirst * Rd;
        // 32-bit decode when the output (and so every index) stays below 2^31;
        // four consecutive gamma per thread (shared loads of the previous level)
        const int64_t outsz = std::max<int64_t>(total, Aa * Bb * Rfirst * Rd);
        const int64_t nthr = Jp * Km * Rfirst * ((Rd + 3) / 4);
        if (outsz < ((int64_t)1 << 31))
            subchain_step_kernel<T, TZ, uint32_t, 4><<<grid_for(nthr), 256, 0, s>>>(
                cur, Jp, Rfirst, Rc, Z[m], Km, Rd, out, fin, Aa, Bb, t == t0 ? zfirst : nullptr);
        else
            subchain_step_kernel<T, TZ, int64_t, 4><<<grid_for(nthr), 256, 0, s>>>(
                cur, Jp, Rfirst, Rc, Z[m], Km, Rd, out, fin, Aa, Bb, t == t0 ? zfirst : nullptr);
        rtr_count_launch();
        if (cudaGetLastError() != cudaSuccess) { *status = RTR_ECUDA; return nullptr; }
        cur = out;
        which ^= 1;
        Jp *= Km;
    }
    return cur;
}

int launch_gram_inverse(const float* G, int C, float* Ginv, int* need_slow, cudaStream_t s) {
    if (C <= 64) gram_inverse_kernel<4><<<1, 256, 0, s>>>(G, C, Ginv, need_slow);
    else if (C <= 112) gram_inverse_kernel<7><<<1, 256, 0, s>>>(G, C, Ginv, need_slow);
    else gram_inverse_kernel<9><<<1, 256, 0, s>>>(G, C, Ginv, need_slow);
    RTR_LAUNCH_CHECK("gram_inverse_kernel");
    return RTR_OK;
}

template <typename T>
int als_impl(rtr_plan* p, const T* P, double* const* Z, int init_given, double* err, cudaStream_t s) {
    const int N = p->N;
    const int is_f64 = std::is_same<T, double>::value;
    int64_t Kd[RTR_MAXN];
    for (int n = 0; n < N; ++n) Kd[n] = p->K[n];
    double* ws = p->als_ws;
    const int64_t ESZ = 256 * 256;
    double* E[RTR_MAXN];
    for (int n = 0; n < N; ++n) E[n] = ws + n * ESZ;
    double* Mp[2] = {ws + RTR_MAXN * ESZ, ws + (RTR_MAXN + 1) * ESZ};
    // prefix products A_n = E_{n+1} ... E_{n-2} of the Gram chains (ping-pong)
    double* Ab[2] = {ws + (RTR_MAXN + 2) * ESZ, ws + (RTR_MAXN + 3) * ESZ};
    // Mp[1] serves the start's transfer products only; during the sweeps it
    // holds the float32 inverse of the current Gram matrix
    float* Ginv = reinterpret_cast<float*>(Mp[1]);
    float* Gf = Ginv + 160 * 160;                    // float32 copy of the Gram matrix (hi part)
    float* Gfl = Gf + 160 * 160;                     // and its low part
    double* W = ws + (RTR_MAXN + 4) * ESZ;
    double* Wz = W + p->als_wmax;
    double* jac = Wz + p->als_wmax;              // 2 * 144^2 for the pinv fallback
    double* zw = jac + 2 * 144 * 144;            // z_i . w_i per slice (max K_n)
    int* need_slow = reinterpret_cast<int*>(p->scal + 24);
    double* normP2 = p->scal + 1;
    double* normTR2 = p->scal + 2;

    for (int n = 0; n < N; ++n)
        if (p->R[n] * p->R[(n + 1) % N] > 144)
            return rtr_set_error(RTR_EUNSUPPORTED, "TR-ALS: R_%d R_%d = %d > 144", n, (n + 1) % N,
                                 p->R[n] * p->R[(n + 1) % N]);
    int st = launch_sumsq(P, is_f64, p->pnumel, p->partial, 1024, normP2, p->flags, s);
    if (st) return st;

    auto transfer = [&](int m) -> int {
        const int Ra = p->R[m], Rb = p->R[(m + 1) % N];
        transfer_kernel<<<grid_for((int64_t)Ra * Ra * Rb * Rb, 64), 64, 0, s>>>(Z[m], Ra, (int)Kd[m], Rb, E[m]);
        RTR_LAUNCH_CHECK("transfer_kernel");
        return RTR_OK;
    };
    // product E_start ... E_{start+count-1} (mod N) into one of Mp; returns pointer
    auto eprod = [&](int start, int count, double** res) -> int {
        double* cur = E[start % N];
        int rows = p->R[start % N] * p->R[start % N];
        int which = 0;
        for (int t = 1; t < count; ++t) {
            const int m = (start + t) % N;
            const int k = p->R[m] * p->R[m];
            const int cols = p->R[(m + 1) % N] * p->R[(m + 1) % N];
            matmul_f64_kernel<<<dim3((unsigned)rtr_ceil_div(cols, 8), (unsigned)rtr_ceil_div(rows, 8)), 64, 0, s>>>(
                cur, E[m], Mp[which], rows, k, cols);
            RTR_LAUNCH_CHECK("matmul_f64_kernel");
            cur = Mp[which];
            which ^= 1;
        }
        *res = cur;
        return RTR_OK;
    };

    if (!init_given) {
        for (int n = 0; n < N; ++n) {
            const int64_t cnt = (int64_t)p->R[n] * Kd[n] * p->R[(n + 1) % N];
            init_core_kernel<<<grid_for(cnt), 256, 0, s>>>(Z[n], cnt, p->params.seed, n, p->tab64);
            RTR_LAUNCH_CHECK("init_core_kernel");
        }
        for (int n = 0; n < N; ++n) if ((st = transfer(n))) return st;
        double* full = nullptr;
        if ((st = eprod(0, N, &full))) return st;
        trace_kernel<<<1, 32, 0, s>>>(full, p->R[0] * p->R[0], normTR2);
        RTR_LAUNCH_CHECK("trace_kernel");
        for (int n = 0; n < N; ++n) {
            const int64_t cnt = (int64_t)p->R[n] * Kd[n] * p->R[(n + 1) % N];
            scale_cores_kernel<<<grid_for(cnt), 256, 0, s>>>(Z[n], cnt, normP2, normTR2, N);
            RTR_LAUNCH_CHECK("scale_cores_kernel");
        }
    }
    // transfer matrices of the start; the transfer of each updated core and
    // the Gram chain of the next update then run on the plan's side stream,
    // concurrently with the contraction on the caller's stream
    for (int n = 0; n < N; ++n) if ((st = transfer(n))) return st;

    // compute-type core copies read by the contraction (float32 shadows for
    // the FP32/BF16 plans; the FP64 plan reads its cores directly)
    const void* Zt[RTR_MAXN];
    float* Zf[RTR_MAXN] = {};
    if (!is_f64) {
        float* zf = reinterpret_cast<float*>(zw + p->als_maxK);
        for (int n = 0; n < N; ++n) {
            const int64_t cnt = (int64_t)p->R[n] * Kd[n] * p->R[(n + 1) % N];
            Zf[n] = zf;
            zf += (cnt + 3) & ~(int64_t)3;
            to_f32_kernel<<<grid_for(cnt), 256, 0, s>>>(Z[n], Zf[n], cnt);
            RTR_LAUNCH_CHECK("to_f32_kernel");
            Zt[n] = Zf[n];
        }
    } else {
        for (int n = 0; n < N; ++n) Zt[n] = Z[n];
    }
    cudaStream_t side = p->side, side2 = p->side2;
    // The Gram matrix of update n is G_n = A_n E_{n-1} (reindexed) with the
    // prefix A_n = E_{n+1} ... E_{n-2}, which does not involve the core updated
    // last: A_{n+1} is formed on a third stream during update n, as soon as
    // E_{n-1} is known, so that update n + 1's side chain holds one product.
    // (Order 3: A_n = E_{n+1}, no product.)
    // buf: the update's running number modulo 2 (consecutive updates alternate)
    auto prefix = [&](int n1, int buf, cudaStream_t st, double** res) -> int {
        if (N == 3) { *res = E[(n1 + 1) % N]; return RTR_OK; }
        GramChainArgs ga{};
        ga.cnt = N - 2;
        for (int t = 0; t < ga.cnt; ++t) {
            const int m = (n1 + 1 + t) % N;
            ga.F[t] = E[m];
            ga.dim[t] = p->R[m] * p->R[m];
        }
        const int ml = (n1 + N - 1) % N;
        ga.dim[ga.cnt] = p->R[ml] * p->R[ml];
        ga.out = Ab[buf];
        const int rows = p->R[(n1 + 1) % N] * p->R[(n1 + 1) % N];
        gram_chain_kernel<<<(unsigned)rows, GC_THREADS, 0, st>>>(ga);
        RTR_LAUNCH_CHECK("gram_chain_kernel");
        *res = Ab[buf];
        return RTR_OK;
    };
    double* Acur = nullptr;
    // A_0 of the first update, from the start's transfer matrices
    RTR_CUDA(cudaEventRecord(p->ev[4], s));
    RTR_CUDA(cudaStreamWaitEvent(side2, p->ev[4], 0));
    if ((st = prefix(0, 0, side2, &Acur))) return st;
    RTR_CUDA(cudaEventRecord(p->ev[5], side2));
    // the float plans form W without storing the subchain where the sizes allow
    int fused[RTR_MAXN] = {};
    for (int n = 0; n < N; ++n) fused[n] = !is_f64 && fused_contract_ok(p, n) == 0;
    // dynamic shared memory limits, set once for the largest update (a host
    // API call per launch would pace the whole chain of small kernels)
    {
        int cmax = 0;
        for (int n = 0; n < N; ++n) cmax = std::max(cmax, p->R[n] * p->R[(n + 1) % N]);
        RTR_SMEM(als_solve_inv_kernel, sizeof(double) * (size_t)cmax * (cmax + 1));
    }
    for (int sweep = 0; sweep < p->params.sweeps; ++sweep) {
        for (int n = 0; n < N; ++n) {
            const int Rn = p->R[n], Rn1 = p->R[(n + 1) % N];
            const int C = Rn * Rn1;
            int64_t A, I, B;
            rtr_mode_view(N, Kd, n, &A, &I, &B);
            // ---- side stream: E of the core updated last, then G = A_n E_{n-1}
            RTR_CUDA(cudaEventRecord(p->ev[0], s));
            RTR_CUDA(cudaStreamWaitEvent(side, p->ev[0], 0));
            const int ml = (n + N - 1) % N;
            if (sweep > 0 || n > 0) {
                const int Ra = p->R[ml], Rb = p->R[(ml + 1) % N];
                // 64-thread blocks: the float64 work spreads over every SM
                transfer_kernel<<<grid_for((int64_t)Ra * Ra * Rb * Rb, 64), 64, 0, side>>>(Z[ml], Ra, (int)Kd[ml], Rb, E[ml]);
                RTR_LAUNCH_CHECK("transfer_kernel");
            }
            RTR_CUDA(cudaEventRecord(p->ev[4], side));
            RTR_CUDA(cudaStreamWaitEvent(side, p->ev[5], 0));     // A_n formed
            GramChainArgs gc{};
            gc.cnt = 2;
            gc.F[0] = Acur; gc.F[1] = E[ml];
            gc.dim[0] = Rn1 * Rn1; gc.dim[1] = p->R[ml] * p->R[ml]; gc.dim[2] = Rn * Rn;
            gc.out = Mp[0];
            gc.reindex = 1; gc.Rb = Rn1; gc.Rn = Rn; gc.outf = Gf; gc.outl = Gfl;
            gram_chain_kernel<<<(unsigned)(Rn1 * Rn1), GC_THREADS, 0, side>>>(gc);
            RTR_LAUNCH_CHECK("gram_chain_kernel");
            if ((st = launch_gram_inverse(Gf, C, Ginv, need_slow, side))) return st;
            RTR_CUDA(cudaEventRecord(p->ev[1], side));
            // ---- third stream: A_{n+1} for the next update, once E_{n-1} is known
            RTR_CUDA(cudaStreamWaitEvent(side2, p->ev[4], 0));
            if ((st = prefix((n + 1) % N, (sweep * N + n + 1) & 1, side2, &Acur))) return st;
            RTR_CUDA(cudaEventRecord(p->ev[5], side2));
            // ---- caller's stream: W = P_<n> S, subchain generated in the contraction
            // ---- caller's stream: subchain S (natural row order), then W = P_<n> S
            if (!is_f64 && fused[n]) {
                if ((st = launch_fused_contract(p, reinterpret_cast<const float*>(P), Zf, n, W, s))) return st;
            } else {
            if ((size_t)(A * B) * (size_t)C * sizeof(T) > p->sub_bytes)
                return rtr_set_error(RTR_ENOMEM, "TR-ALS: subchain exceeds the plan workspace");
            const T* Zc[RTR_MAXN];
            for (int m = 0; m < N; ++m) Zc[m] = reinterpret_cast<const T*>(Zt[m]);
            int cst = RTR_OK;
            const T* Sn = build_chain<T, T>(N, Kd, p->R, Zc, n + 1, N - 1, reinterpret_cast<T*>(p->sub_ws[0]),
                                            reinterpret_cast<T*>(p->sub_ws[1]), 1, A, B, s, &cst);
            if (cst) return rtr_set_error(cst, "TR-ALS: subchain launch failed");
            {
                ContractArgs w{};
                w.X = P; w.A = A; w.I = I; w.B = B; w.C = C;
                w.gen = 0; w.M = Sn; w.ldm = C;
                w.Y = W; w.norm_out = nullptr;
                if ((st = launch_contract(p, is_f64, w, s))) return st;
            }
            }
            // ---- join, then solve G z_i = w_i for every slice
            RTR_CUDA(cudaStreamWaitEvent(s, p->ev[1], 0));
            double* G = Mp[0];
            // refinement: float64 accuracy for FP64 plans; for the float32 / BF16
            // plans one float64-residual correction after the float32 solve
            // (relative error ~(kappa 2^-24)^2)
            const float tol2 = is_f64 ? 1e-28f : 1e-18f;
            const int max_it = is_f64 ? 12 : 2;
            // dynamic shared memory: the float32 inverse, or the slow path's float64 Gram matrix
            const size_t gsmem = std::max(sizeof(float) * (size_t)C * C, sizeof(double) * (size_t)C * (C + 1));
            als_solve_inv_kernel<<<(unsigned)I, SOLVE_THREADS, gsmem, s>>>(Gf, Gfl, Ginv, Rn, Rn1, (int)I, W, Z[n],
                                                                          Zf[n], zw, need_slow, tol2, max_it, G, Wz,
                                                                          jac, p->flags);
            RTR_LAUNCH_CHECK("als_solve_inv_kernel");
            if (err && n == N - 1) {
                als_err_kernel<<<1, 32, 0, s>>>(zw, (int)I, normP2, err + sweep);
                RTR_LAUNCH_CHECK("als_err_kernel");
            }
        }
    }
    // the last prefix product (for an update that does not come) joins the caller's stream
    RTR_CUDA(cudaStreamWaitEvent(s, p->ev[5], 0));
    return RTR_OK;
}

template <typename T>
int reconstruct_impl(int N, const int64_t* dims, const int* R, const double* const* G, T* Xhat, void* work,
                     size_t work_bytes, cudaStream_t s) {
    const int h = N / 2;
    int64_t L = 1, Rr = 1;
    for (int n = 0; n < h; ++n) L *= dims[n];
    for (int n = h; n < N; ++n) Rr *= dims[n];
    const int R0 = R[0], Rh = R[h % N];
    const int64_t maxR = 16;
    const int64_t szL = L * maxR * maxR, szR = Rr * maxR * maxR;
    const int64_t sz = std::max(szL, szR);
    if (work_bytes < sizeof(T) * (size_t)(4 * sz)) return rtr_set_error(RTR_EINVAL, "reconstruct work buffer too small");
    T* w0 = (T*)work;
    T* w1 = w0 + sz;
    T* w2 = w1 + sz;
    T* w3 = w2 + sz;
    int st = 0;
    // left[l, alpha, gamma] = G_0(i_0)...G_{h-1}(i_{h-1})      (R0 x Rh)
    T* left = build_chain<T>(N, dims, R, G, 0, h, w0, w1, 0, 1, 1, s, &st);
    // right[r, gamma, alpha] = G_h(i_h)...G_{N-1}(i_{N-1})     (Rh x R0)
    T* right = build_chain<T>(N, dims, R, G, h, N - h, w2, w3, 0, 1, 1, s, &st);
    if (!left || !right) return rtr_set_error(RTR_ECUDA, "reconstruct chain launch failed");
    // rightT[r, alpha, gamma]
    T* rightT = (right == w2) ? w3 : w2;
    block_transpose_kernel<T><<<grid_for(Rr * R0 * Rh), 256, 0, s>>>(right, Rr, Rh, R0, rightT);
    RTR_LAUNCH_CHECK("block_transpose_kernel");
    dim3 grid((unsigned)rtr_ceil_div(Rr, 64), (unsigned)rtr_ceil_div(L, 64));
    if (grid.y > 65535) return rtr_set_error(RTR_EINVAL, "reconstruct: left extent too large");
    nt_gemm_kernel<T><<<grid, 256, 0, s>>>(left, rightT, Xhat, L, Rr, R0 * Rh);
    RTR_LAUNCH_CHECK("nt_gemm_kernel");
    return RTR_OK;
}

}  // namespace

size_t reconstruct_work_bytes(int N, const int64_t* dims, const int* R) {
    const int h = N / 2;
    int64_t L = 1, Rr = 1;
    for (int n = 0; n < h; ++n) L *= dims[n];
    for (int n = h; n < N; ++n) Rr *= dims[n];
    return sizeof(double) * (size_t)(4 * std::max(L, Rr) * 16 * 16);
}

int run_reconstruct(int N, const int64_t* dims, const int* R, const double* const* G, int out_prec, void* Xhat,
                    void* work, size_t work_bytes, cudaStream_t s) {
    if (out_prec == RTR_FP64) return reconstruct_impl<double>(N, dims, R, G, (double*)Xhat, work, work_bytes, s);
    return reconstruct_impl<float>(N, dims, R, G, (float*)Xhat, work, work_bytes, s);
}

static int als_eager(rtr_plan* p, const void* P, double* const* Z, int init_given, double* err, cudaStream_t s) {
    if (p->params.prec == RTR_FP64) return als_impl<double>(p, (const double*)P, Z, init_given, err, s);
    return als_impl<float>(p, (const float*)P, Z, init_given, err, s);
}

// The sweeps are a long chain of small dependent kernels on two streams; they
// are recorded once into a CUDA graph per argument set (P, Z, err,
// init_given) on the plan's own stream and replayed on the caller's stream,
// which removes the per-launch gaps.  A call made while the caller's stream is
// being captured runs eagerly (the caller's capture records it); if recording
// fails the call runs eagerly too.
int run_als(rtr_plan* p, const void* P, double* const* Z, int init_given, double* err, cudaStream_t s) {
    for (int n = 0; n < p->N; ++n) {
        if (p->R[n] * p->R[(n + 1) % p->N] > 144)
            return rtr_set_error(RTR_EUNSUPPORTED, "TR-ALS supports R_n R_{n+1} <= 144");
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RTR_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return als_eager(p, P, Z, init_given, err, s);
    bool same = p->als_exec != nullptr && p->als_key_P == P && p->als_key_err == err &&
                p->als_key_init == (init_given != 0);
    for (int n = 0; same && n < p->N; ++n) same = p->als_key_Z[n] == Z[n];
    if (!same) {
        if (p->als_exec) {
            // new arguments (rare): let any replay of the old graph finish first
            RTR_CUDA(cudaDeviceSynchronize());
            cudaGraphExecDestroy(p->als_exec);
            p->als_exec = nullptr;
        }
        const unsigned long long before = rtr_kernel_launches();
        RTR_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        const int st = als_eager(p, P, Z, init_given, err, p->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(p->cap, &g);
        const long long recorded = (long long)(rtr_kernel_launches() - before);
        rtr_count_launches(-recorded);              // recorded, not run
        cudaGraphExec_t ex = nullptr;
        if (st == RTR_OK && ee == cudaSuccess && g != nullptr &&
            cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
            p->als_exec = ex;
            p->als_kernels = recorded;
            p->als_key_P = P;
            p->als_key_err = err;
            p->als_key_init = (init_given != 0);
            for (int n = 0; n < p->N; ++n) p->als_key_Z[n] = Z[n];
        }
        if (g) cudaGraphDestroy(g);
        if (!p->als_exec) {
            cudaGetLastError();
            return als_eager(p, P, Z, init_given, err, s);
        }
    }
    RTR_CUDA(cudaGraphLaunch(p->als_exec, s));
    rtr_count_launches(p->als_kernels);
    return RTR_OK;
}

int run_backproject(rtr_plan* p, const double* const* Z, const double* const* Q, double* const* G, const int* ranks,
                    cudaStream_t s) {
    const int N = p->N;
    const int* R = ranks ? ranks : p->R;
    for (int n = 0; n < N; ++n) {
        if (!Z[n] || !Q[n] || !G[n]) return rtr_set_error(RTR_EINVAL, "backproject: NULL pointer for mode %d", n);
        const int Ra = R[n], Rb = R[(n + 1) % N];
        const int64_t total = (int64_t)Ra * p->dims[n] * Rb;
        backproject_kernel<<<grid_for(total), 256, 0, s>>>(Z[n], Q[n], G[n], Ra, p->K[n], (int)p->dims[n], Rb);
        RTR_LAUNCH_CHECK("backproject_kernel");
    }
    return RTR_OK;
}

int run_rse(rtr_plan* p, const void* P, const double* const* Z, const int* ranks, double* out, cudaStream_t s) {
    const int N = p->N;
    const int* R = ranks ? ranks : p->R;
    int64_t Kd[RTR_MAXN];
    for (int n = 0; n < N; ++n) Kd[n] = p->K[n];
    double* dense = (double*)p->chain[0];       // >= |P| doubles (ensured at plan creation)
    void* work = p->sub_ws[0];
    int st = run_reconstruct(N, Kd, R, Z, RTR_FP64, dense, work, p->sub_bytes * 2, s);
    if (st) return st;
    const int is_f64 = p->params.prec == RTR_FP64;
    if ((st = launch_sumsq(P, is_f64, p->pnumel, p->partial, 1024, p->scal + 1, p->flags, s))) return st;
    if (is_f64) sqdiff_kernel<double><<<1024, 256, 0, s>>>((const double*)P, dense, p->pnumel, p->partial);
    else sqdiff_kernel<float><<<1024, 256, 0, s>>>((const float*)P, dense, p->pnumel, p->partial);
    RTR_LAUNCH_CHECK("sqdiff_kernel");
    rse_final_kernel<<<1, 1024, 0, s>>>(p->partial, 1024, p->scal + 0, p->scal + 1, out);
    RTR_LAUNCH_CHECK("rse_final_kernel");
    return RTR_OK;
}

int run_draw_omega(rtr_plan* p, int mode, int64_t row0, int64_t nrows, int K, double* out, cudaStream_t s) {
    const int ncalls = (K + 19) / 20;
    draw_omega_kernel<<<grid_for(nrows * ncalls), 256, 0, s>>>(out, row0, nrows, K, p->params.seed, mode, p->tab64,
                                                               p->tab32,
                                                               p->params.prec == RTR_FP8 ? p->tab_e4m3 : nullptr,
                                                               p->params.prec == RTR_FP64);
    RTR_LAUNCH_CHECK("draw_omega_kernel");
    return RTR_OK;
}
