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
#include <type_traits>
#include "rtr_internal.cuh"
#include "dense.cuh"

size_t contract_partial_elems(int num_sms, int64_t I, int C);

namespace {

// ---- subchain products --------------------------------------------------------
// Sout[(j'*Km + i), beta, gamma] = sum_c Sprev[j', beta, c] * Z[c, i, gamma]
// (Sprev == nullptr: Sout[i, beta, gamma] = Z[beta, i, gamma]).
// With final_tr, row j = b*A + a of the cyclic order is stored at a*B + b.
template <typename T>
__global__ void subchain_step_kernel(const T* __restrict__ Sprev, int64_t Jp, int Rb, int Rc,
                                     const double* __restrict__ Z, int Km, int Rd, T* __restrict__ Sout,
                                     int final_tr, int64_t Aa, int64_t Bb) {
    const int64_t total = Jp * Km * Rb * Rd;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(e % Rd);
        const int be = (int)((e / Rd) % Rb);
        const int64_t j = e / ((int64_t)Rd * Rb);
        const int i = (int)(j % Km);
        const int64_t jp = j / Km;
        T v;
        if (Sprev == nullptr) {
            v = (T)Z[((int64_t)be * Km + i) * Rd + g];
        } else {
            T s = T(0);
            const T* sp = Sprev + (jp * Rb + be) * Rc;
            for (int c = 0; c < Rc; ++c) s = fma(sp[c], (T)Z[((int64_t)c * Km + i) * Rd + g], s);
            v = s;
        }
        int64_t r = j;
        if (final_tr) { const int64_t b = j / Aa, a = j % Aa; r = a * Bb + b; }
        Sout[(r * Rb + be) * Rd + g] = v;
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

// C (m x n) = A (m x k) B (k x n), float64, one output per thread.
__global__ void matmul_f64_kernel(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C,
                                  int m, int k, int n) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * n + j];
        C[e] = s;
    }
}

__global__ void trace_kernel(const double* __restrict__ M, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += M[i * n + i];
        *out = s;
    }
}

// Solve z_i G = w_i for all i (G from Mprod by the (beta,alpha) reindexing),
// write Z_n[alpha, i, beta] = z_i[beta*Rn + alpha]; err2 = ||P||^2 - sum z.w.
// G in dynamic shared memory; fallback: Jacobi pseudo-inverse in global memory.
__global__ void __launch_bounds__(512) als_solve_kernel(const double* __restrict__ Mprod, int Rn, int Rn1, int In,
                                                        double* __restrict__ W, double* __restrict__ Wz,
                                                        double* __restrict__ Zn, const double* __restrict__ normP2,
                                                        double* __restrict__ err_out, double* __restrict__ jac_ws,
                                                        int* __restrict__ flags) {
    extern __shared__ __align__(16) double Gs[];
    const int C = Rn * Rn1;
    const int ld = C + 1;
    __shared__ double red[32];
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
        const int c = e / C, c2 = e % C;
        const int be = c / Rn, al = c % Rn, be2 = c2 / Rn, al2 = c2 % Rn;
        Gs[c * ld + c2] = Mprod[((int64_t)be * Rn1 + be2) * (Rn * Rn) + al * Rn + al2];
    }
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
        for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
            const int c = e / C, c2 = e % C;
            const int be = c / Rn, al = c % Rn, be2 = c2 / Rn, al2 = c2 % Rn;
            Aj[e] = Mprod[((int64_t)be * Rn1 + be2) * (Rn * Rn) + al * Rn + al2];
        }
        __syncthreads();
        rtr::block_jacobi_eig(Aj, V, C, C, pairs, cs, 40);
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
    double zw = 0.0;
    for (int e = threadIdx.x; e < In * C; e += blockDim.x) {
        const int i = e / C, c = e % C;
        const int be = c / Rn, al = c % Rn;
        const double z = Wz[e];
        zw += z * W[e];
        Zn[((int64_t)al * In + i) * Rn1 + be] = z;
    }
    zw = rtr::block_sum(zw, red);
    if (err_out && threadIdx.x == 0) *err_out = sqrt(fmax(*normP2 - zw, 0.0));
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

__global__ void rse_final_kernel(const double* __restrict__ part, int nparts, const double* __restrict__ normX2,
                                 const double* __restrict__ normP2, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double e2 = 0.0;
        for (int i = 0; i < nparts; ++i) e2 += part[i];
        const double x2 = *normX2;
        *out = sqrt(fmax(x2 - *normP2 + e2, 0.0) / x2);
    }
}

__global__ void draw_omega_kernel(double* __restrict__ out, int64_t row0, int64_t nrows, int K, uint64_t seed,
                                  int mode, const double* __restrict__ tab64, const float* __restrict__ tab32,
                                  int use64) {
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
                out[rr * K + k] = use64 ? tab64[j] : (double)tab32[j];
            }
        }
    }
}

inline unsigned grid_for(int64_t n, int threads = 256, int64_t cap = 65535) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(rtr_ceil_div(n, threads), cap));
}

// Build subchain products over `cores` in ring order start, start+1, ...,
// start+count-1 (indices mod N); writes the product slices for every
// multi-index (row-major) as rows x Rfirst x Rlast into one of two buffers,
// returns the buffer holding the result.  final_tr permutes rows as above.
template <typename T>
T* build_chain(int N, const int64_t* dims, const int* R, const double* const* Z, int start, int count,
               T* buf0, T* buf1, int final_tr, int64_t Aa, int64_t Bb, cudaStream_t s, int* status) {
    T* cur = nullptr;
    T* bufs[2] = {buf0, buf1};
    int which = 0;
    int64_t Jp = 1;
    const int Rfirst = R[start % N];
    for (int t = 0; t < count; ++t) {
        const int m = (start + t) % N;
        const int Km = (int)dims[m];
        const int Rc = R[m], Rd = R[(m + 1) % N];
        T* out = bufs[which];
        const int fin = (t == count - 1) ? final_tr : 0;
        const int64_t total = Jp * Km * Rfirst * Rd;
        subchain_step_kernel<T><<<grid_for(total), 256, 0, s>>>(cur, Jp, Rfirst, Rc, Z[m], Km, Rd, out, fin, Aa, Bb);
        rtr_count_launch();
        if (cudaGetLastError() != cudaSuccess) { *status = RTR_ECUDA; return nullptr; }
        cur = out;
        which ^= 1;
        Jp *= Km;
    }
    return cur;
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
    double* W = ws + (RTR_MAXN + 2) * ESZ;
    double* Wz = W + p->als_wmax;
    double* jac = Wz + p->als_wmax;              // 2 * 144^2 for the pinv fallback
    double* normP2 = p->scal + 1;
    double* normTR2 = p->scal + 2;

    int st = launch_sumsq(P, is_f64, p->pnumel, p->partial, 1024, normP2, s);
    if (st) return st;

    auto transfer = [&](int m) -> int {
        const int Ra = p->R[m], Rb = p->R[(m + 1) % N];
        transfer_kernel<<<grid_for((int64_t)Ra * Ra * Rb * Rb), 256, 0, s>>>(Z[m], Ra, (int)Kd[m], Rb, E[m]);
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
            matmul_f64_kernel<<<grid_for((int64_t)rows * cols, 64), 64, 0, s>>>(cur, E[m], Mp[which], rows, k, cols);
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
    for (int n = 0; n < N; ++n) if ((st = transfer(n))) return st;

    T* sb0 = (T*)p->sub_ws[0];
    T* sb1 = (T*)p->sub_ws[1];
    for (int sweep = 0; sweep < p->params.sweeps; ++sweep) {
        for (int n = 0; n < N; ++n) {
            const int Rn = p->R[n], Rn1 = p->R[(n + 1) % N];
            const int C = Rn * Rn1;
            int64_t A, I, B;
            rtr_mode_view(N, Kd, n, &A, &I, &B);
            // subchain S (rows a*B + b, columns (beta, alpha))
            T* S = build_chain<T>(N, Kd, p->R, Z, n + 1, N - 1, sb0, sb1, 1, A, B, s, &st);
            if (!S) return rtr_set_error(RTR_ECUDA, "subchain kernel launch failed");
            ContractArgs ca{};
            ca.X = P; ca.A = A; ca.I = I; ca.B = B; ca.C = C;
            ca.gen = 0; ca.M = S; ca.ldm = C; ca.Y = W; ca.norm_out = nullptr;
            if ((st = launch_contract(p, is_f64, ca, s))) return st;
            double* Mprod = nullptr;
            if ((st = eprod(n + 1, N - 1, &Mprod))) return st;
            const size_t smem = sizeof(double) * (size_t)C * (C + 1);
            RTR_CUDA(cudaFuncSetAttribute(als_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            double* eo = (err && n == N - 1) ? err + sweep : nullptr;
            als_solve_kernel<<<1, 512, smem, s>>>(Mprod, Rn, Rn1, (int)I, W, Wz, Z[n], normP2, eo, jac, p->flags);
            RTR_LAUNCH_CHECK("als_solve_kernel");
            if ((st = transfer(n))) return st;
        }
    }
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

int run_als(rtr_plan* p, const void* P, double* const* Z, int init_given, double* err, cudaStream_t s) {
    for (int n = 0; n < p->N; ++n) {
        if (p->R[n] * p->R[(n + 1) % p->N] > 144)
            return rtr_set_error(RTR_EUNSUPPORTED, "TR-ALS supports R_n R_{n+1} <= 144");
    }
    if (p->params.prec == RTR_FP64) return als_impl<double>(p, (const double*)P, Z, init_given, err, s);
    return als_impl<float>(p, (const float*)P, Z, init_given, err, s);
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
    if ((st = launch_sumsq(P, is_f64, p->pnumel, p->partial, 1024, p->scal + 1, s))) return st;
    if (is_f64) sqdiff_kernel<double><<<1024, 256, 0, s>>>((const double*)P, dense, p->pnumel, p->partial);
    else sqdiff_kernel<float><<<1024, 256, 0, s>>>((const float*)P, dense, p->pnumel, p->partial);
    RTR_LAUNCH_CHECK("sqdiff_kernel");
    rse_final_kernel<<<1, 32, 0, s>>>(p->partial, 1024, p->scal + 0, p->scal + 1, out);
    RTR_LAUNCH_CHECK("rse_final_kernel");
    return RTR_OK;
}

int run_draw_omega(rtr_plan* p, int mode, int64_t row0, int64_t nrows, int K, double* out, cudaStream_t s) {
    const int ncalls = (K + 19) / 20;
    draw_omega_kernel<<<grid_for(nrows * ncalls), 256, 0, s>>>(out, row0, nrows, K, p->params.seed, mode, p->tab64,
                                                               p->tab32, p->params.prec == RTR_FP64);
    RTR_LAUNCH_CHECK("draw_omega_kernel");
    return RTR_OK;
}
