// Block-level float64 dense kernels on shared-memory matrices (one CTA).
#pragma once
#include "rtr_internal.cuh"

namespace rtr {

// In-place lower Cholesky G = L L^T of an n x n SPD matrix (row-major, ld,
// n <= 256, blockDim.x a multiple of 16).  Returns false (uniformly across the
// block) if a pivot is not finite or not above rel_tol times the original
// diagonal entry (rel_tol = 0 is the LAPACK potrf failure condition, pivot <= 0).
// Right-looking, one barrier per column: step k updates the trailing matrix
// from the unscaled column k (scaled by 1/d_k), and scales column k-1 and
// writes its diagonal, which no thread reads during step k.
template <typename T>
__device__ inline bool block_cholesky(T* G, int n, int ld, double rel_tol = 0.0) {
    __shared__ T diag0[256];
    for (int k = threadIdx.x; k < n; k += blockDim.x) diag0[k] = G[k * ld + k];
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4, nty = blockDim.x >> 4;
    T inv_prev = T(0), sq_prev = T(0);
    for (int k = 0; k < n; ++k) {
        const T d = G[k * ld + k];
        // compared in T: a float64 conversion here would run on the slow
        // float64 pipe in every thread at every column
        if (!(d > (T)rel_tol * diag0[k]) || !(d > T(0)) || !isfinite(d)) return false;
        const T sq = sqrt(d);
        const T inv = T(1) / sq;
        const T inv2 = inv * inv;
        if (k > 0) {
            for (int i = k + threadIdx.x; i < n; i += blockDim.x) G[i * ld + k - 1] *= inv_prev;
            if (threadIdx.x == 0) G[(k - 1) * ld + k - 1] = sq_prev;
        }
        for (int i = k + 1 + ty; i < n; i += nty) {
            const T gik = G[i * ld + k] * inv2;
            for (int j = k + 1 + tx; j <= i; j += 16) G[i * ld + j] -= gik * G[j * ld + k];
        }
        inv_prev = inv;
        sq_prev = sq;
        __syncthreads();
    }
    if (threadIdx.x == 0 && n > 0) G[(n - 1) * ld + n - 1] = sq_prev;
    __syncthreads();
    return true;
}

// One warp solves L L^T z = w in place (w of length n in shared or global
// memory, stride 1), L lower from block_cholesky.  Column-oriented sweeps.
__device__ inline void warp_chol_solve(const double* L, int n, int ld, double* w) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < n; ++k) {             // forward: L y = w
        const double yk = w[k] / L[k * ld + k];
        __syncwarp();
        if (lane == 0) w[k] = yk;
        for (int l = k + 1 + lane; l < n; l += 32) w[l] -= L[l * ld + k] * yk;
        __syncwarp();
    }
    for (int k = n - 1; k >= 0; --k) {        // backward: L^T z = y
        const double zk = w[k] / L[k * ld + k];
        __syncwarp();
        if (lane == 0) w[k] = zk;
        for (int l = lane; l < k; l += 32) w[l] -= L[k * ld + l] * zk;
        __syncwarp();
    }
}

// Sum of v over the block, returned to every thread (fixed order: warp
// butterflies, then one butterfly over the warp sums).  Only warp 0 adds the
// warp sums: a float64 add in every thread would load GB300's narrow FP64 pipe.
__device__ inline double block_sum(double v, double* red /* >= 32 doubles */) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double s = lane < nw ? red[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    const double s = red[0];
    __syncthreads();
    return s;
}

// Cyclic Jacobi eigendecomposition of a symmetric n x n matrix A (row-major,
// ld) in memory visible to the block, parallel round-robin pairing (n/2
// disjoint rotations per step), in the arithmetic type T.  On return the
// diagonal of A holds the eigenvalues and the columns of V (n x n, ld) the
// eigenvectors.  `pairs` needs 2*((n+1)/2) ints, `cs` needs 2*((n+1)/2) T.
// A pair is rotated only while |a_pq| > eps_T sqrt(|a_pp a_qq|) (eps_T the
// unit roundoff of T; the relative rule of Demmel and Veselic, 1992) and
// |a_pq| > eps_T ||A||_F: entries below the second bound are rounding noise
// of the rotations themselves, which would otherwise keep a numerically
// singular block rotating forever in float32.  The iteration stops after the
// first sweep that rotates nothing, once the off-diagonal mass is at most
// off_tol times the total (block-wide reduction, every thread takes part),
// or after max_sweeps.
template <typename T>
__device__ inline void block_jacobi_eig(T* A, T* V, int n, int ld, int* pairs, T* cs, int max_sweeps,
                                        T off_tol) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * n; e += nt) V[(e / n) * ld + e % n] = (e / n == e % n) ? T(1) : T(0);
    __syncthreads();
    if (n < 2) return;
    const int m = (n + 1) & ~1;             // even player count (dummy = n when odd)
    const int np = m / 2;
    __shared__ T red_off[32], red_tot[32];
    const int lane = tid & 31, w = tid >> 5, nw = (nt + 31) >> 5;
    const T eps = sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // convergence test: off-diagonal mass relative to the whole
        T off = T(0), tot = T(0);
        for (int e = tid; e < n * n; e += nt) {
            const int i = e / n, j = e % n;
            const T a = A[i * ld + j];
            tot += a * a;
            if (i != j) off += a * a;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (lane == 0) { red_off[w] = off; red_tot[w] = tot; }
        __syncthreads();
        off = T(0); tot = T(0);
        for (int u = 0; u < nw; ++u) { off += red_off[u]; tot += red_tot[u]; }
        __syncthreads();
        if (!(off > off_tol * tot)) break;
        const T floor_abs = eps * sqrt(tot);
        int rotated = 0;
        for (int step = 0; step < m - 1; ++step) {
            // round-robin pairing: player 0 fixed, others rotate
            for (int k = tid; k < np; k += nt) {
                int p = (k == 0) ? 0 : 1 + (k - 1 + step) % (m - 1);
                int q = 1 + (m - 2 - k + step) % (m - 1);
                if (p > q) { const int t = p; p = q; q = t; }
                pairs[2 * k] = p; pairs[2 * k + 1] = q;
                T c = T(1), sn = T(0);
                if (q < n) {
                    const T apq = A[p * ld + q];
                    const T app = A[p * ld + p], aqq = A[q * ld + q];
                    if (fabs(apq) > eps * sqrt(fabs(app)) * sqrt(fabs(aqq)) && fabs(apq) > floor_abs) {
                        rotated = 1;
                        const T tau = (aqq - app) / (T(2) * apq);
                        const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
                        c = T(1) / sqrt(T(1) + t * t);
                        sn = t * c;
                    }
                }
                cs[2 * k] = c; cs[2 * k + 1] = sn;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < np * n; e += nt) {
                const int k = e / n, j = e % n;
                const int p = pairs[2 * k], q = pairs[2 * k + 1];
                if (q >= n) continue;
                const T c = cs[2 * k], sn = cs[2 * k + 1];
                const T ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - sn * aq;
                A[q * ld + j] = sn * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < np * n; e += nt) {
                const int k = e / n, i = e % n;
                const int p = pairs[2 * k], q = pairs[2 * k + 1];
                if (q >= n) continue;
                const T c = cs[2 * k], sn = cs[2 * k + 1];
                const T ap = A[i * ld + p], aq = A[i * ld + q];
                A[i * ld + p] = c * ap - sn * aq;
                A[i * ld + q] = sn * ap + c * aq;
                const T vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - sn * vq;
                V[i * ld + q] = sn * vp + c * vq;
            }
            __syncthreads();
        }
        if (!__syncthreads_or(rotated)) break;
    }
}

// Shared-memory form of the same cyclic Jacobi iteration (same pairing,
// thresholds and stopping rules as block_jacobi_eig).  A round applies the
// n/2 disjoint rotations from both sides at once: with pairs (p, q) and
// (r, u), block [p q] x [r u] of J^T A J is J_pq^T A[pq, ru] J_ru, so each
// thread reads one 2 x 2 block of the current buffer and writes it to the
// other (no read/write hazard: two barriers per round, one after the
// rotation parameters, one after the update).  Diagonal blocks take the
// classical update a_pp -= t a_pq, a_qq += t a_pq, a_pq = 0.
// A0 holds the input (n x n, ld), A1 and V are n x ld scratch; cs needs
// 3 * np T and pairs 2 * np ints (np = ceil(n / 2)).  Returns the buffer
// (A0 or A1) whose diagonal holds the eigenvalues; V's columns are the
// eigenvectors.
template <typename T>
__device__ inline T* block_jacobi_eig_db(T* A0, T* A1, T* V, int n, int ld, int* pairs, T* cs, int max_sweeps,
                                         T off_tol) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * n; e += nt) V[(e / n) * ld + e % n] = (e / n == e % n) ? T(1) : T(0);
    if (n < 2) { __syncthreads(); return A0; }
    const int m = (n + 1) & ~1;
    const int np = m / 2;
    __shared__ T red_off[32], red_tot[32];
    const int lane = tid & 31, w = tid >> 5, nw = (nt + 31) >> 5;
    const T eps = sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08);
    T* cur = A0;
    T* nxt = A1;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        T off = T(0), tot = T(0);
        __syncthreads();
        for (int e = tid; e < n * n; e += nt) {
            const int i = e / n, j = e % n;
            const T a = cur[i * ld + j];
            tot += a * a;
            if (i != j) off += a * a;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (lane == 0) { red_off[w] = off; red_tot[w] = tot; }
        __syncthreads();
        off = T(0); tot = T(0);
        for (int u = 0; u < nw; ++u) { off += red_off[u]; tot += red_tot[u]; }
        if (!(off > off_tol * tot)) break;
        const T floor_abs = eps * sqrt(tot);
        int rotated = 0;
        for (int step = 0; step < m - 1; ++step) {
            for (int k = tid; k < np; k += nt) {
                int p = (k == 0) ? 0 : 1 + (k - 1 + step) % (m - 1);
                int q = 1 + (m - 2 - k + step) % (m - 1);
                if (p > q) { const int t = p; p = q; q = t; }
                pairs[2 * k] = p; pairs[2 * k + 1] = q;
                T c = T(1), sn = T(0), tt = T(0);
                if (q < n) {
                    const T apq = cur[p * ld + q];
                    const T app = cur[p * ld + p], aqq = cur[q * ld + q];
                    if (fabs(apq) > eps * sqrt(fabs(app)) * sqrt(fabs(aqq)) && fabs(apq) > floor_abs) {
                        rotated = 1;
                        const T tau = (aqq - app) / (T(2) * apq);
                        tt = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
                        c = T(1) / sqrt(T(1) + tt * tt);
                        sn = tt * c;
                    }
                }
                cs[3 * k] = c; cs[3 * k + 1] = sn; cs[3 * k + 2] = tt;
            }
            __syncthreads();
            for (int e = tid; e < np * np; e += nt) {
                const int k = e / np, l = e % np;
                const int p = pairs[2 * k], q = pairs[2 * k + 1];
                const int r = pairs[2 * l], u = pairs[2 * l + 1];
                if (k == l) {
                    if (q < n) {
                        const T apq = cur[p * ld + q], t = cs[3 * k + 2];
                        nxt[p * ld + p] = cur[p * ld + p] - t * apq;
                        nxt[q * ld + q] = cur[q * ld + q] + t * apq;
                        nxt[p * ld + q] = T(0);
                        nxt[q * ld + p] = T(0);
                    } else {
                        nxt[p * ld + p] = cur[p * ld + p];
                    }
                    continue;
                }
                const T ck = cs[3 * k], sk = cs[3 * k + 1], cl = cs[3 * l], sl = cs[3 * l + 1];
                const bool qv = q < n, uv = u < n;
                const T xpr = cur[p * ld + r];
                const T xpu = uv ? cur[p * ld + u] : T(0);
                const T xqr = qv ? cur[q * ld + r] : T(0);
                const T xqu = (qv && uv) ? cur[q * ld + u] : T(0);
                const T ypr = ck * xpr - sk * xqr, yqr = sk * xpr + ck * xqr;
                const T ypu = ck * xpu - sk * xqu, yqu = sk * xpu + ck * xqu;
                nxt[p * ld + r] = cl * ypr - sl * ypu;
                if (uv) nxt[p * ld + u] = sl * ypr + cl * ypu;
                if (qv) nxt[q * ld + r] = cl * yqr - sl * yqu;
                if (qv && uv) nxt[q * ld + u] = sl * yqr + cl * yqu;
            }
            for (int e = tid; e < n * np; e += nt) {
                const int i = e / np, k = e % np;
                const int p = pairs[2 * k], q = pairs[2 * k + 1];
                if (q >= n) continue;
                const T c = cs[3 * k], sn = cs[3 * k + 1];
                const T vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - sn * vq;
                V[i * ld + q] = sn * vp + c * vq;
            }
            __syncthreads();
            T* t = cur; cur = nxt; nxt = t;
        }
        if (!__syncthreads_or(rotated)) break;
    }
    __syncthreads();
    return cur;
}

}  // namespace rtr
