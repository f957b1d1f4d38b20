// TR-SVD on the projected tensor (Algorithm 1 step 9, second decomposer;
// Section 4.1 tolerance), float64.
//
// Step k works on the unfolding C_k (rows x cols, row-major float64):
//   C_0 = P as K_1 x (K_2 ... K_N)
//   SVD C_k = U S V^T: FP64 plans by a one-sided Jacobi SVD of C_k itself
//   (float64, one CTA per rotation pair); the float plans through the Gram
//   matrix of the smaller side (float64, many CTAs) and its float32 Jacobi
//   eigendecomposition (one CTA, in shared memory when it fits); each pair
//   (u_k, v_k) signed so that the entry of u_k largest in magnitude is
//   positive (the result of TR-SVD depends on these signs through the
//   reshapes between steps);
//   rank r_k = smallest r with sqrt(sum_{i>=r} s_i^2) <= threshold (sqrt(2)
//   delta for k = 0, delta after; delta = tol ||P|| / sqrt(N)), or forced;
//   core k = U_r reshaped, carry = S_r V_r^T = U_r^T C_k, which is reshaped
//   (and, after the first step, cyclically permuted) into C_{k+1}.
// The last core is the final carry.  Each rank decision is read back to the
// host (the next shapes depend on it).
#include <algorithm>
#include <cmath>
#include <vector>
#include "rtr_internal.cuh"
#include "dense.cuh"

namespace {

inline unsigned gridn(int64_t n, int t = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535));
}

// G = C C^T (left) or C^T C (right), m x m float64: one warp per output
// (i <= j), lanes split the long sum (every SM takes part: float64 work is
// slow on this GPU, so it is spread as widely as possible).
template <typename T>
__global__ void gram_kernel(const T* __restrict__ Cm, int64_t rows, int64_t cols, int left, double* __restrict__ G) {
    const int64_t m = left ? rows : cols;
    const int64_t len = left ? cols : rows;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < m * m; e += nw) {
        const int64_t i = e / m, j = e % m;
        if (j < i) continue;                           // uniform per warp
        double s = 0.0;
        if (left)
            for (int64_t l = lane; l < len; l += 32) s += (double)Cm[i * cols + l] * (double)Cm[j * cols + l];
        else
            for (int64_t l = lane; l < len; l += 32) s += (double)Cm[l * cols + i] * (double)Cm[l * cols + j];
        s = rtr::warp_sum(s);
        if (lane == 0) {
            G[i * m + j] = s;
            G[j * m + i] = s;
        }
    }
}

// Jacobi eigendecomposition of G (m x m, global memory) in one CTA, in the
// arithmetic type T (float64 for FP64 plans; float32 for the float plans,
// whose decomposition input P is float32 anyway: float64 rotations on this
// GPU cost about a hundred times more); then sort eigenpairs by decreasing
// eigenvalue into lam[m] and Vs (m x m, columns), both float64.
template <typename T>
__global__ void __launch_bounds__(1024) eig_kernel(double* __restrict__ G, T* __restrict__ A, T* __restrict__ V, int m,
                                                   double* __restrict__ lam, double* __restrict__ Vs,
                                                   int* __restrict__ order) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int np = (m + 1) / 2 + 1;
    T* cs = reinterpret_cast<T*>(smem_raw);                      // 2 np
    int* pairs = reinterpret_cast<int*>(cs + 2 * np);            // 2 np
    if ((void*)A != (void*)G)
        for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) A[e] = (T)G[e];
    __syncthreads();
    rtr::block_jacobi_eig<T>(A, V, m, m, pairs, cs, 60, sizeof(T) == 8 ? T(1e-30) : T(1e-13));
    __syncthreads();
    // rank sort by decreasing eigenvalue (ties keep index order; NaN last)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const T vi = A[(int64_t)i * m + i];
        const T ki = isnan(vi) ? -INFINITY : vi;
        int rk = 0;
        for (int j = 0; j < m; ++j) {
            const T vj = A[(int64_t)j * m + j];
            const T kj = isnan(vj) ? -INFINITY : vj;
            rk += (kj > ki) || (kj == ki && j < i);
        }
        order[rk] = i;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = (double)A[(int64_t)order[i] * m + order[i]];
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
        const int64_t r = e / m, c = e % m;
        Vs[e] = (double)V[r * m + order[c]];
    }
}

// Shared-memory form for m small enough that A (twice) and V fit in shared
// memory (block_jacobi_eig_db); ld = m | 1 keeps column accesses free of
// bank conflicts.  Eigenpairs are sorted by decreasing eigenvalue with a
// parallel rank sort (ties keep index order; NaN sorts last).
template <typename T>
__global__ void __launch_bounds__(1024) eig_smem_kernel(const double* __restrict__ G, int m, double* __restrict__ lam,
                                                        double* __restrict__ Vs, int max_sweeps, T off_tol) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = m | 1;
    const int np = (m + 1) / 2;
    T* A0 = reinterpret_cast<T*>(smem_raw);
    T* A1 = A0 + (size_t)m * ld;
    T* V = A1 + (size_t)m * ld;
    T* cs = V + (size_t)m * ld;                                   // 3 np
    int* pairs = reinterpret_cast<int*>(cs + 3 * np);             // 2 np
    int* order = pairs + 2 * np;                                  // m
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) A0[(e / m) * ld + e % m] = (T)G[e];
    __syncthreads();
    const T* A = rtr::block_jacobi_eig_db<T>(A0, A1, V, m, ld, pairs, cs, max_sweeps, off_tol);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const T vi = A[i * ld + i];
        const T ki = isnan(vi) ? -INFINITY : vi;
        int rk = 0;
        for (int j = 0; j < m; ++j) {
            const T vj = A[j * ld + j];
            const T kj = isnan(vj) ? -INFINITY : vj;
            rk += (kj > ki) || (kj == ki && j < i);
        }
        order[rk] = i;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = (double)A[order[i] * ld + order[i]];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e % m;
        Vs[e] = (double)V[r * ld + order[c]];
    }
}

template <typename T>
size_t eig_smem_bytes(int m) {
    const size_t ld = (size_t)(m | 1), np = (size_t)(m + 1) / 2;
    return sizeof(T) * (3 * (size_t)m * ld + 3 * np) + sizeof(int) * (2 * np + (size_t)m);
}

constexpr size_t EIG_SMEM_MAX = 227 * 1024;

// ---- one-sided Jacobi SVD (FP64 plans) ---------------------------------------
// The m vectors w_k of the smaller side (the rows of C when rows <= cols, its
// columns otherwise), each of length L, are copied to W (m x L row-major) and
// Jt (m x m) starts as the identity.  A sweep visits every pair once, in
// m' - 1 rounds of m'/2 disjoint pairs (circle schedule, m' = m rounded up to
// even; one CTA per pair), and rotates each pair (i, j) so that w_i . w_j = 0
// (Hestenes), applying the same rotation to rows i, j of Jt.  At convergence
// the w_k are orthogonal with sigma_k = ||w_k||, and J = Jt^T holds the
// eigenvectors of the Gram matrix of the smaller side (C C^T or C^T C) for
// the eigenvalues sigma_k^2, without that Gram matrix being formed: singular
// values and vectors carry errors of order u ||C|| instead of u ||C||^2.
template <typename T>
__global__ void jac_init_kernel(const T* __restrict__ Cm, int64_t rows, int64_t cols, int left, int m, int64_t L,
                                double* __restrict__ W, double* __restrict__ Jt) {
    const int64_t nw = (int64_t)m * L, total = nw + (int64_t)m * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nw) {
            const int64_t k = e / L, l = e % L;
            W[e] = (double)(left ? Cm[k * cols + l] : Cm[l * cols + k]);
        } else {
            const int64_t f = e - nw;
            Jt[f] = (f / m == f % m) ? 1.0 : 0.0;
        }
    }
}

// pair p of round t of the circle schedule over mp (even) indices: index 0
// stays, indices 1..mp-1 turn one place per round
__device__ __forceinline__ void jac_pair(int mp, int t, int p, int& i, int& j) {
    const int ring = mp - 1;
    if (p == 0) {
        i = 0;
        j = t % ring + 1;
    } else {
        i = (t + p) % ring + 1;
        j = (t + mp - 1 - p) % ring + 1;
    }
}

constexpr int JAC_THREADS = 256;

__global__ void __launch_bounds__(JAC_THREADS) jac_round_kernel(double* __restrict__ W, double* __restrict__ Jt, int m,
                                                                int64_t L, int mp, int t, double tol,
                                                                unsigned* __restrict__ nrot) {
    __shared__ double red[3][JAC_THREADS / 32];
    __shared__ double cs[2];
    int i, j;
    jac_pair(mp, t, blockIdx.x, i, j);
    if (i >= m || j >= m) return;                      // the odd index out: uniform per CTA
    double* wi = W + (int64_t)i * L;
    double* wj = W + (int64_t)j * L;
    double a = 0.0, b = 0.0, g = 0.0;
    for (int64_t l = threadIdx.x; l < L; l += JAC_THREADS) {
        const double x = wi[l], y = wj[l];
        a = fma(x, x, a);
        b = fma(y, y, b);
        g = fma(x, y, g);
    }
    a = rtr::warp_sum(a);
    b = rtr::warp_sum(b);
    g = rtr::warp_sum(g);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = a; red[1][w] = b; red[2][w] = g; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = g = 0.0;
        for (int q = 0; q < JAC_THREADS / 32; ++q) { a += red[0][q]; b += red[1][q]; g += red[2][q]; }
        double c = 1.0, sn = 0.0;
        if (a > 0.0 && b > 0.0 && fabs(g) > tol * sqrt(a) * sqrt(b)) {
            const double z = (b - a) / (2.0 * g);
            const double tn = copysign(1.0, z) / (fabs(z) + hypot(1.0, z));
            c = 1.0 / sqrt(1.0 + tn * tn);
            sn = c * tn;
            if (sn != 0.0) atomicAdd(nrot, 1u);
        }
        cs[0] = c;
        cs[1] = sn;
    }
    __syncthreads();
    const double c = cs[0], sn = cs[1];
    if (sn == 0.0) return;
    for (int64_t l = threadIdx.x; l < L; l += JAC_THREADS) {
        const double x = wi[l], y = wj[l];
        wi[l] = c * x - sn * y;
        wj[l] = sn * x + c * y;
    }
    double* ji = Jt + (int64_t)i * m;
    double* jj = Jt + (int64_t)j * m;
    for (int l = threadIdx.x; l < m; l += JAC_THREADS) {
        const double x = ji[l], y = jj[l];
        ji[l] = c * x - sn * y;
        jj[l] = sn * x + c * y;
    }
}

// lam (decreasing) = ||w_k||^2 and Vs (m x m, eigenvector columns in the same
// order) from a converged Jacobi; one CTA.  Ties keep index order; NaN last.
__global__ void __launch_bounds__(1024) jac_finish_kernel(const double* __restrict__ W, const double* __restrict__ Jt,
                                                          int m, int64_t L, double* __restrict__ lam,
                                                          double* __restrict__ Vs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* nrm = reinterpret_cast<double*>(smem_raw);         // m
    int* order = reinterpret_cast<int*>(nrm + m);               // m
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int k = threadIdx.x >> 5; k < m; k += nwarp) {
        double s = 0.0;
        for (int64_t l = lane; l < L; l += 32) s = fma(W[(int64_t)k * L + l], W[(int64_t)k * L + l], s);
        s = rtr::warp_sum(s);
        if (lane == 0) nrm[k] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double ki = isnan(nrm[i]) ? -INFINITY : nrm[i];
        int rk = 0;
        for (int j = 0; j < m; ++j) {
            const double kj = isnan(nrm[j]) ? -INFINITY : nrm[j];
            rk += (kj > ki) || (kj == ki && j < i);
        }
        order[rk] = i;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = nrm[order[i]];
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
        const int64_t r = e / m, c = e % m;
        Vs[e] = Jt[(int64_t)order[c] * m + r];
    }
}

// Sign rule of the singular pairs (the TR-SVD reading that makes its result
// unique): column k of U (rows x r) is negated unless its entry largest in
// magnitude (the first such entry on ties) is positive.  One warp per column;
// the carry U^T C formed afterwards follows the same signs.
__global__ void sign_kernel(double* __restrict__ U, int64_t rows, int r) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int k = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); k < r; k += nw) {
        double best = -1.0;
        int64_t bi = rows;
        for (int64_t i = lane; i < rows; i += 32) {
            const double v = fabs(U[i * r + k]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (bi < rows && U[bi * r + k] < 0.0)
            for (int64_t i = lane; i < rows; i += 32) U[i * r + k] = -U[i * r + k];
    }
}

constexpr int JAC_MAX_SWEEPS = 40;

// rank from the eigenvalue tail: smallest r >= 1 with sum_{i>=r} max(lam_i, 0)
// <= thr^2.  The tail is summed from the smallest eigenvalue up (never as the
// total minus the leading terms, whose cancellation error u ||C||^2 would hide
// thresholds below sqrt(u) ||C||).
__global__ void rank_kernel(const double* __restrict__ lam, int m, double thr2, int cap, int* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double tail = 0.0;
        int r = m;
        for (int i = m - 1; i >= 0; --i) {
            const double t = tail + fmax(lam[i], 0.0);
            if (!(t <= thr2)) break;
            tail = t;
            r = i;
        }
        r = max(r, 1);
        out[0] = min(r, cap);
        out[1] = r > cap;
    }
}

// left singular vectors: U[:, :r] for the left Gram: U = Vs[:, :r] (rows x r);
// for the right Gram: U = C Vs[:, :r] / s   (s = sqrt(lam)).
template <typename T>
__global__ void left_vectors_kernel(const T* __restrict__ Cm, int64_t rows, int64_t cols, int left,
                                    const double* __restrict__ Vs, const double* __restrict__ lam, int m, int r,
                                    double* __restrict__ U) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * r; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r, k = e % r;
        if (left) {
            U[e] = Vs[i * m + k];
        } else {
            double s = 0.0;
            for (int64_t l = 0; l < cols; ++l) s += (double)Cm[i * cols + l] * Vs[l * m + k];
            const double sg = sqrt(fmax(lam[k], 0.0));
            U[e] = sg > 0.0 ? s / sg : 0.0;
        }
    }
}

// carry = U^T C  (r x cols).  The sum over rows runs as four interleaved
// float64 chains (row i to chain i mod 4, chains added pairwise): a single
// chain is bound by the float64 add latency of this GPU.
template <typename T>
__global__ void carry_kernel(const T* __restrict__ Cm, int64_t rows, int64_t cols, const double* __restrict__ U, int r,
                             double* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)r * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / cols, j = e % cols;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t i = 0;
        for (; i + 4 <= rows; i += 4) {
            a0 = fma(U[i * r + k], (double)Cm[i * cols + j], a0);
            a1 = fma(U[(i + 1) * r + k], (double)Cm[(i + 1) * cols + j], a1);
            a2 = fma(U[(i + 2) * r + k], (double)Cm[(i + 2) * cols + j], a2);
            a3 = fma(U[(i + 3) * r + k], (double)Cm[(i + 3) * cols + j], a3);
        }
        if (i < rows) a0 = fma(U[i * r + k], (double)Cm[i * cols + j], a0);
        if (i + 1 < rows) a1 = fma(U[(i + 1) * r + k], (double)Cm[(i + 1) * cols + j], a1);
        if (i + 2 < rows) a2 = fma(U[(i + 2) * r + k], (double)Cm[(i + 2) * cols + j], a2);
        out[e] = (a0 + a1) + (a2 + a3);
    }
}

// core 0: U (K_0 x R0 R1) -> Z (R0, K_0, R1)
__global__ void core0_kernel(const double* __restrict__ U, int K0, int R0, int R1, double* __restrict__ Z) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K0 * R0 * R1; e += gridDim.x * blockDim.x) {
        const int b = e % R1, i = (e / R1) % K0, a = e / (R1 * K0);
        Z[e] = U[(int64_t)i * (R0 * R1) + a * R1 + b];
    }
}

// first carry (R0, R1, rest) -> (R1, rest, R0)
__global__ void permute_first_kernel(const double* __restrict__ in, int R0, int R1, int64_t rest,
                                     double* __restrict__ out) {
    const int64_t total = (int64_t)R0 * R1 * rest;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % R0);
        const int64_t x = (e / R0) % rest;
        const int b = (int)(e / ((int64_t)R0 * rest));
        out[e] = in[((int64_t)a * R1 + b) * rest + x];
    }
}

__global__ void copy_kernel(const double* __restrict__ in, int64_t n, double* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = in[e];
}

template <typename T>
__global__ void sumsq_svd_kernel(const T* __restrict__ X, int64_t n, double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        s += (double)X[e] * (double)X[e];
    s = rtr::block_sum(s, red);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

struct SvdWs {
    double *Cbuf0, *Cbuf1, *G, *V, *Vs, *U, *lam;
    int* iv;           // [0..1] rank, overflow; [2..] order (Gram route) or the Jacobi rotation count
    double* nrm;
    int jac_notconv = 0;
};

// Jacobi route of svd_step: W in w.G, Jt in w.V, then lam and Vs
template <typename T>
int jacobi_eig(const T* Cm, int64_t rows, int64_t cols, int left, int m, SvdWs& w, cudaStream_t s) {
    const int64_t L = left ? cols : rows;
    const int mp = m + (m & 1);
    unsigned* nrot = reinterpret_cast<unsigned*>(w.iv + 2);
    jac_init_kernel<T><<<gridn((int64_t)m * L + (int64_t)m * m), 256, 0, s>>>(Cm, rows, cols, left, m, L, w.G, w.V);
    RTR_LAUNCH_CHECK("jac_init_kernel");
    bool conv = false;
    for (int sweep = 0; sweep < JAC_MAX_SWEEPS && !conv; ++sweep) {
        RTR_CUDA(cudaMemsetAsync(nrot, 0, sizeof(unsigned), s));
        for (int t = 0; t < mp - 1; ++t) {
            jac_round_kernel<<<mp / 2, JAC_THREADS, 0, s>>>(w.G, w.V, m, L, mp, t, 1e-15, nrot);
            RTR_LAUNCH_CHECK("jac_round_kernel");
        }
        unsigned h = 0;
        RTR_CUDA(cudaMemcpyAsync(&h, nrot, sizeof(h), cudaMemcpyDeviceToHost, s));
        RTR_CUDA(cudaStreamSynchronize(s));
        conv = h == 0;
    }
    if (!conv) w.jac_notconv = 1;
    const size_t smem = (size_t)m * (sizeof(double) + sizeof(int));
    if (smem > EIG_SMEM_MAX) return rtr_set_error(RTR_EUNSUPPORTED, "TR-SVD: Gram side %d too large", m);
    RTR_SMEM(jac_finish_kernel, smem);
    jac_finish_kernel<<<1, 1024, smem, s>>>(w.G, w.V, m, L, w.lam, w.Vs);
    RTR_LAUNCH_CHECK("jac_finish_kernel");
    return RTR_OK;
}

template <typename T>
int svd_vectors(const T* Cm, int64_t rows, int64_t cols, int left, int m, double thr, int forced, int cap, SvdWs& w,
                int* r_out, int* overflow, cudaStream_t s);

// one truncated SVD of C (rows x cols); returns rank (host), writes U (rows x r,
// canonical signs) into ws
// eig32: the float plans: Gram matrix and its eigendecomposition in float32;
// otherwise (FP64 plans) the one-sided Jacobi SVD
template <typename T>
int svd_step(const T* Cm, int64_t rows, int64_t cols, double thr, int forced, int cap, SvdWs& w, int* r_out,
             int* overflow, bool eig32, cudaStream_t s) {
    const int left = rows <= cols;
    const int m = (int)(left ? rows : cols);
    if (!eig32) {
        const int st = jacobi_eig<T>(Cm, rows, cols, left, m, w, s);
        if (st) return st;
        return svd_vectors<T>(Cm, rows, cols, left, m, thr, forced, cap, w, r_out, overflow, s);
    }
    gram_kernel<T><<<gridn((int64_t)m * m * 32), 256, 0, s>>>(Cm, rows, cols, left, w.G);
    RTR_LAUNCH_CHECK("gram_kernel");
    const size_t np = (size_t)(m + 1) / 2 + 1;
    const size_t sm_bytes = eig32 ? eig_smem_bytes<float>(m) : eig_smem_bytes<double>(m);
    if (sm_bytes <= EIG_SMEM_MAX) {
        if (eig32)
            RTR_SMEM(eig_smem_kernel<float>, sm_bytes);
        else
            RTR_SMEM(eig_smem_kernel<double>, sm_bytes);
        if (eig32) eig_smem_kernel<float><<<1, 1024, sm_bytes, s>>>(w.G, m, w.lam, w.Vs, 60, 1e-13f);
        else eig_smem_kernel<double><<<1, 1024, sm_bytes, s>>>(w.G, m, w.lam, w.Vs, 60, 1e-30);
    } else if (!eig32) {
        const size_t smem = 2 * np * (sizeof(double) + sizeof(int));
        eig_kernel<double><<<1, 1024, smem, s>>>(w.G, w.G, w.V, m, w.lam, w.Vs, w.iv + 2);
    } else {
        // float32 working copies in the (float64-sized) V buffer
        float* A32 = reinterpret_cast<float*>(w.V);
        float* V32 = A32 + (size_t)m * m;
        const size_t smem = 2 * np * (sizeof(float) + sizeof(int));
        eig_kernel<float><<<1, 1024, smem, s>>>(w.G, A32, V32, m, w.lam, w.Vs, w.iv + 2);
    }
    RTR_LAUNCH_CHECK("eig_kernel");
    return svd_vectors<T>(Cm, rows, cols, left, m, thr, forced, cap, w, r_out, overflow, s);
}

// rank decision on lam, then U (rows x r) from Vs with canonical signs
template <typename T>
int svd_vectors(const T* Cm, int64_t rows, int64_t cols, int left, int m, double thr, int forced, int cap, SvdWs& w,
                int* r_out, int* overflow, cudaStream_t s) {
    int r = forced;
    if (forced <= 0) {
        rank_kernel<<<1, 32, 0, s>>>(w.lam, m, thr * thr, std::min(cap, m), w.iv);
        RTR_LAUNCH_CHECK("rank_kernel");
        int h[2];
        RTR_CUDA(cudaMemcpyAsync(h, w.iv, sizeof(h), cudaMemcpyDeviceToHost, s));
        RTR_CUDA(cudaStreamSynchronize(s));
        r = h[0];
        *overflow |= h[1];
    }
    if (r < 1 || r > m) return rtr_set_error(RTR_EINVAL, "TR-SVD rank %d outside [1, %d]", r, m);
    // 64-thread blocks: the float64 dot products spread over every SM
    left_vectors_kernel<T><<<gridn(rows * r, 64), 64, 0, s>>>(Cm, rows, cols, left, w.Vs, w.lam, m, r, w.U);
    RTR_LAUNCH_CHECK("left_vectors_kernel");
    sign_kernel<<<gridn((int64_t)r * 32), 256, 0, s>>>(w.U, rows, r);
    RTR_LAUNCH_CHECK("sign_kernel");
    *r_out = r;
    return RTR_OK;
}

template <typename T>
int trsvd_impl(rtr_plan* p, const T* P, double tol, double* const* Z, int* ranks, cudaStream_t s) {
    const int N = p->N;
    int64_t K[RTR_MAXN];
    for (int n = 0; n < N; ++n) K[n] = p->K[n];
    SvdWs w;
    w.Cbuf0 = p->svd_ws;
    w.Cbuf1 = w.Cbuf0 + p->svd_cbuf;
    w.G = w.Cbuf1 + p->svd_cbuf;
    w.V = w.G + p->svd_gmax * p->svd_gmax;
    w.Vs = w.V + p->svd_gmax * p->svd_gmax;
    w.lam = w.Vs + p->svd_gmax * p->svd_gmax;
    w.U = w.lam + p->svd_gmax;
    w.nrm = w.U + p->svd_umax;
    w.iv = reinterpret_cast<int*>(w.nrm + 2);
    const bool forced = ranks[0] > 0;
    // delta = tol ||P|| / sqrt(N)
    RTR_CUDA(cudaMemsetAsync(w.nrm, 0, sizeof(double), s));
    sumsq_svd_kernel<T><<<256, 256, 0, s>>>(P, p->pnumel, w.nrm);
    RTR_LAUNCH_CHECK("sumsq_svd_kernel");
    double nrm2 = 0.0;
    RTR_CUDA(cudaMemcpyAsync(&nrm2, w.nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    RTR_CUDA(cudaStreamSynchronize(s));
    const double delta = tol * std::sqrt(nrm2) / std::sqrt((double)N);
    int overflow = 0;
    int R[RTR_MAXN + 1];
    // ---- step 0: C_0 = P (K_0 x rest)
    int64_t rest = p->pnumel / K[0];
    int cap0 = p->R[0] * p->R[1];
    int r = 0;
    const bool eig32 = p->params.prec != RTR_FP64;
    int st = svd_step<T>(P, K[0], rest, std::sqrt(2.0) * delta, forced ? ranks[0] * ranks[1] : 0, cap0, w, &r,
                         &overflow, eig32, s);
    if (st) return st;
    int R0, R1;
    if (forced) { R0 = ranks[0]; R1 = ranks[1]; }
    else {
        R0 = 1;
        for (int d = 1; d * d <= r; ++d) if (r % d == 0) R0 = d;
        R1 = r / R0;
        if (R0 > p->R[0] || R1 > p->R[1]) {
            // the split does not fit the plan's core capacity: cap both factors
            R0 = std::min(R0, p->R[0]);
            R1 = std::min(R1, p->R[1]);
            r = R0 * R1;
            overflow = 1;
        }
    }
    R[0] = R0; R[1] = R1;
    core0_kernel<<<gridn((int64_t)K[0] * r), 256, 0, s>>>(w.U, (int)K[0], R0, R1, Z[0]);
    RTR_LAUNCH_CHECK("core0_kernel");
    carry_kernel<T><<<gridn((int64_t)r * rest, 64), 64, 0, s>>>(P, K[0], rest, w.U, r, w.Cbuf1);
    RTR_LAUNCH_CHECK("carry_kernel");
    permute_first_kernel<<<gridn((int64_t)r * rest), 256, 0, s>>>(w.Cbuf1, R0, R1, rest, w.Cbuf0);
    RTR_LAUNCH_CHECK("permute_first_kernel");
    double* Ccur = w.Cbuf0;
    double* Cnext = w.Cbuf1;
    // ---- steps 1 .. N-2
    for (int k = 1; k <= N - 2; ++k) {
        const int64_t rows = (int64_t)R[k] * K[k];
        const int64_t cols = (int64_t)r * rest / rows;       // total stays r * rest
        int rk = 0;
        const int cap = p->R[k + 1];
        st = svd_step<double>(Ccur, rows, cols, delta, forced ? ranks[k + 1] : 0, cap, w, &rk, &overflow, eig32, s);
        if (st) return st;
        R[k + 1] = rk;
        // core k = U reshaped (R_k, K_k, R_{k+1})
        copy_kernel<<<gridn(rows * rk), 256, 0, s>>>(w.U, rows * rk, Z[k]);
        RTR_LAUNCH_CHECK("copy_kernel");
        carry_kernel<double><<<gridn((int64_t)rk * cols, 64), 64, 0, s>>>(Ccur, rows, cols, w.U, rk, Cnext);
        RTR_LAUNCH_CHECK("carry_kernel");
        std::swap(Ccur, Cnext);
        r = rk;
        rest = cols;
    }
    // ---- last core: carry (R_{N-1} x K_{N-1} R_0)
    copy_kernel<<<gridn((int64_t)R[N - 1] * K[N - 1] * R0), 256, 0, s>>>(Ccur, (int64_t)R[N - 1] * K[N - 1] * R0,
                                                                          Z[N - 1]);
    RTR_LAUNCH_CHECK("copy_kernel");
    for (int n = 0; n < N; ++n) ranks[n] = R[n];
    if (overflow)
        return rtr_set_error(RTR_ENOTCONV, "TR-SVD: a chosen rank exceeded the plan's core capacity and was capped");
    if (w.jac_notconv)
        return rtr_set_error(RTR_ENOTCONV, "TR-SVD: a Jacobi SVD stopped after %d sweeps before every pair was "
                             "orthogonal to 1e-15", JAC_MAX_SWEEPS);
    return RTR_OK;
}

}  // namespace

size_t trsvd_ws_elems(int64_t pnumel, int64_t* cbuf, int64_t* gmax, int64_t* umax) {
    // every unfolding C_k has at most |P| entries (each carry has no more rows
    // than the unfolding it came from), the Gram side is <= sqrt(|C_k|), and
    // U_r (rows x r) fits in |P| entries
    *cbuf = std::max<int64_t>(pnumel, 1);
    int64_t g = 1;
    while (g * g < *cbuf) ++g;
    *gmax = g;
    *umax = *cbuf;
    return (size_t)(2 * *cbuf + 3 * *gmax * *gmax + *gmax + *umax + 4 + *gmax / 2 + 8);
}

int run_trsvd(rtr_plan* p, const void* P, double tol, double* const* Z, int* ranks, cudaStream_t s) {
    if (!(tol > 0.0)) return rtr_set_error(RTR_EINVAL, "TR-SVD tolerance must be positive");
    for (int n = 0; n < p->N; ++n) if (!Z[n]) return rtr_set_error(RTR_EINVAL, "Z[%d] is NULL", n);
    if (ranks[0] > 0) {
        for (int n = 0; n < p->N; ++n)
            if (ranks[n] < 1 || ranks[n] > p->R[n])
                return rtr_set_error(RTR_EINVAL, "forced rank %d of core %d outside [1, %d]", ranks[n], n, p->R[n]);
    }
    if (p->params.prec == RTR_FP64) return trsvd_impl<double>(p, (const double*)P, tol, Z, ranks, s);
    return trsvd_impl<float>(p, (const float*)P, tol, Z, ranks, s);
}
