// Grouped TR-ALS for a batch of small projected tensors P_t (Algorithm 1,
// step 9, for many tensors at once).
//
// The per-tensor path spends most of a small tensor's time in launch latency
// (seven launches per core update).  Here every stage of a core update runs
// as ONE launch over all tensors of the batch:
//   bgram     : the Gram matrix S^T S of the update from the transfer
//               matrices, one work item per (tensor, block of 16 output rows)
//               of the chain product E_{n+1} ... E_{n-1};
//   bcontract : W = P_<n> S (Eq. 2 subchain generated on the fly), work items
//               (tensor, range of subchain prefixes) sized for equal work, one
//               float64 partial per item;
//   bsolve    : one CTA per tensor: partials summed in a fixed order,
//               equilibrated Cholesky of the Gram matrix, the K_n normal
//               equations solved, the core written, and its transfer matrix
//               E_n refreshed for the next updates.
// All tensors share N and the sweep count, so a sweep of N core updates is
// 3N launches for the whole batch.  The compute type T is float64 for
// float64 tensors and float32 otherwise (Gram and solve included).
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>
#include "dense.cuh"
#include "als_tile.cuh"

namespace {

constexpr int CT_THREADS = 256;
constexpr int SV_THREADS = 512;
constexpr int LB = 32;              // last-mode indices per contraction block (K_n <= 64: at most 2)
constexpr int MAXC = 160;           // C = R_n R_{n+1} <= 144

template <typename T>
struct BTensor {
    const T* P;
    T* Zt[RTR_MAXN];                 // cores in the compute type
    double* Zo[RTR_MAXN];            // float64 output cores
    T* E[RTR_MAXN];                  // transfer matrices, E_m: R_m^2 x R_{m+1}^2
    T* G;                            // Gram matrix of the current update, C x C
    double* W;                       // K_n x C
    double* trace;                   // R_0^2 diagonal parts of the full chain
    double* scal;                    // [0] ||P||^2
    int64_t K[RTR_MAXN];
    int64_t stride[RTR_MAXN];
    int R[RTR_MAXN];
    int64_t part_off[RTR_MAXN];      // first partial of the update of mode n
    int nitems[RTR_MAXN];            // contraction items of the update of mode n
    int64_t numel;
    uint64_t seed;
};

struct CItem { int t; int64_t jp0, jp1; int64_t off; };
struct GItem { int t, r; };

template <typename T>
__device__ __forceinline__ T dfma(T a, T b, T c) { return fma(a, b, c); }

// ---- Gram rows: rows r0 .. r0 + 15 of E_start E_start+1 ... (cnt factors, cyclic)
// Each item carries a block of GB rows through the chain: V (GB x len) times
// E_m, with E_m staged in shared memory GB rows at a time, so that one load of
// E_m serves GB rows.
constexpr int GB = 16;

template <typename T>
__global__ void __launch_bounds__(CT_THREADS) bgram_kernel(const BTensor<T>* __restrict__ tens,
                                                           const GItem* __restrict__ items, int nitems, int N,
                                                           int start, int cnt, int trace_mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* V0 = reinterpret_cast<T*>(smem_raw);          // GB x 256
    T* V1 = V0 + GB * 256;                           // GB x 256
    T* Es = V1 + GB * 256;                           // GB x 256
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const GItem g = items[it];
        const BTensor<T>& b = tens[g.t];
        int m = start % N;
        const int rows = b.R[m] * b.R[m];
        const int nr = min(GB, rows - g.r);
        int len = b.R[(m + 1) % N] * b.R[(m + 1) % N];
        __syncthreads();
        for (int e = tid; e < nr * len; e += blockDim.x) {
            const int r = e / len, j = e % len;
            V0[r * 256 + j] = b.E[m][(int64_t)(g.r + r) * len + j];
        }
        T* cur = V0;
        T* nxt = V1;
        for (int s = 1; s < cnt; ++s) {
            m = (start + s) % N;
            const int cols = b.R[(m + 1) % N] * b.R[(m + 1) % N];
            const T* Em = b.E[m];
            const int nout = nr * cols;
            T acc[GB];
#pragma unroll
            for (int q = 0; q < GB; ++q) acc[q] = T(0);
            for (int k0 = 0; k0 < len; k0 += GB) {
                const int kb = min(GB, len - k0);
                __syncthreads();
                for (int e = tid; e < kb * cols; e += blockDim.x) {
                    const int kk = e / cols, j = e % cols;
                    Es[kk * 256 + j] = Em[(int64_t)(k0 + kk) * cols + j];
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < GB; ++q) {
                    const int e = tid + q * CT_THREADS;
                    if (e < nout) {
                        const int r = e / cols, j = e % cols;
                        T a = acc[q];
                        for (int kk = 0; kk < kb; ++kk) a = dfma(cur[r * 256 + k0 + kk], Es[kk * 256 + j], a);
                        acc[q] = a;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < GB; ++q) {
                const int e = tid + q * CT_THREADS;
                if (e < nout) nxt[(e / cols) * 256 + e % cols] = acc[q];
            }
            T* tmp = cur; cur = nxt; nxt = tmp;
            len = cols;
        }
        __syncthreads();
        if (trace_mode) {
            for (int r = tid; r < nr; r += blockDim.x) b.trace[g.r + r] = (double)cur[r * 256 + g.r + r];
        } else {
            // G[(beta, alpha), (beta', alpha')] = M[(beta, beta'), (alpha, alpha')]
            const int n = (start + N - 1) % N;              // the mode being updated
            const int Rn = b.R[n], Rb = b.R[(n + 1) % N];
            const int C = Rb * Rn;
            for (int e = tid; e < nr * len; e += blockDim.x) {
                const int r = e / len, j = e % len;
                const int rg = g.r + r;
                const int be = rg / Rb, be2 = rg % Rb;
                const int al = j / Rn, al2 = j % Rn;
                b.G[(int64_t)(be * Rn + al) * C + be2 * Rn + al2] = cur[r * 256 + j];
            }
        }
    }
}

// ---- W = P_<n> S: items of subchain prefixes --------------------------------
// One work item (tensor, prefix range) of the batched contraction, with the
// register tile depth IP (i values per thread) fixed at compile time: the
// accumulation loop then carries no per-k predicates.  A prefix fixes the
// indices of the cyclic modes c_1 .. c_{N-3} (none when N = 3); its product M
// (identity when empty) is extended once by every slice of mode c_{N-2}
// (M2[i2] = M Z_{c_{N-2}}(i2), in shared memory), and the subchain rows
// (i2, l) then stream through in blocks of LB: far fewer barriers per row
// than one prefix per (i2).  Thread mappings are computed once per item.
template <typename T, int IP>
__device__ __forceinline__ void bcontract_item(const CItem& ci, int N, int n, double* __restrict__ partial,
                                               const int* sK, const int* sR, const int* scyc, const int64_t* sstride,
                                               const T* const* Zc, const T* __restrict__ Pt, T* M0, T* M1, T* M2,
                                               T* S, T* Pv, const rtr::WTile& wt) {
    const int tid = threadIdx.x;
    const int ml = scyc[N - 1];
    const int m2 = scyc[N - 2];
    const int Rb = sR[(n + 1) % N], Rn = sR[n];
    const int C = Rb * Rn;
    const int Cp = rtr::tile_cp(C);
    const int Kn = sK[n];
    const int Kl = sK[ml];
    const int Rl = sR[ml];                      // right rank of mode c_{N-2} = left rank of the last
    const int K2 = sK[m2];
    const int R2 = sR[m2];                      // left rank of mode c_{N-2}
    const int64_t str_n = sstride[n], str_l = sstride[ml], str_2 = sstride[m2];
    const int nrows = K2 * Kl;
    // S rows: thread -> column c (fixed), rows q = l_s, l_s + s_pass, ...
    const int s_pass = max(1, CT_THREADS / Cp);
    const int sc = tid % Cp, l_s = tid / Cp;
    const bool s_on = l_s < s_pass;
    const int s_be = (sc < C) ? sc / Rn : 0, s_al = (sc < C) ? sc % Rn : 0;
    // P rows: thread -> i (fixed), rows q = l_p, l_p + p_pass, ...
    const int p_pass = max(1, CT_THREADS / Kn);
    const int pi = tid % Kn, l_p = tid / Kn;
    const bool p_on = l_p < p_pass;
    const int zst = Kl * Rn;
    T acc[IP][4];
#pragma unroll
    for (int k = 0; k < IP; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = T(0);
    for (int64_t jp = ci.jp0; jp < ci.jp1; ++jp) {
        // prefix decode in 32 bits (a 64-bit division is a long sequence)
        uint32_t rem = (uint32_t)jp;
        int64_t base = 0;
        int idx[RTR_MAXN];
        for (int t = N - 3; t >= 1; --t) {
            const int m = scyc[t];
            const uint32_t km = (uint32_t)sK[m];
            idx[t] = (int)(rem % km);
            rem /= km;
            base += idx[t] * sstride[m];
        }
        __syncthreads();
        // M = Z_{c_1}(i_1) ... Z_{c_{N-3}}(i_{N-3})  (Rb x R2; the identity when N = 3)
        if (N == 3) {
            for (int e = tid; e < Rb * Rb; e += blockDim.x) {
                const int be = e / Rb, gg = e % Rb;
                M0[be * RTR_MAX_RANK + gg] = (be == gg) ? T(1) : T(0);
            }
        } else {
            const int m = scyc[1];
            const int Rc = sR[(m + 1) % N];
            const int Km = sK[m];
            for (int e = tid; e < Rb * Rc; e += blockDim.x) {
                const int be = e / Rc, gg = e % Rc;
                M0[be * RTR_MAX_RANK + gg] = Zc[m][(be * Km + idx[1]) * Rc + gg];
            }
        }
        T* cur = M0;
        T* nxt = M1;
        for (int t = 2; t <= N - 3; ++t) {
            __syncthreads();
            const int m = scyc[t];
            const int Rm = sR[m], Rc = sR[(m + 1) % N], Km = sK[m];
            const T* zm = Zc[m] + idx[t] * Rc;
            for (int e = tid; e < Rb * Rc; e += blockDim.x) {
                const int be = e / Rc, gg = e % Rc;
                T sum = T(0);
                for (int c = 0; c < Rm; ++c) sum = dfma(cur[be * RTR_MAX_RANK + c], zm[c * Km * Rc + gg], sum);
                nxt[be * RTR_MAX_RANK + gg] = sum;
            }
            T* tmp = cur; cur = nxt; nxt = tmp;
        }
        __syncthreads();
        // M2[i2][be][g] = sum_c M[be][c] Z_{c_{N-2}}[c, i2, g]
        for (int e = tid; e < K2 * Rb * Rl; e += blockDim.x) {
            const int g = e % Rl, be = (e / Rl) % Rb, i2 = e / (Rl * Rb);
            const T* z2 = Zc[m2] + i2 * Rl + g;
            T sum = T(0);
            for (int c = 0; c < R2; ++c) sum = dfma(cur[be * RTR_MAX_RANK + c], z2[c * K2 * Rl], sum);
            M2[(i2 * Rb + be) * RTR_MAX_RANK + g] = sum;
        }
        __syncthreads();
        for (int q0 = 0; q0 < nrows; q0 += LB) {
            const int lb = min(LB, nrows - q0);
            if (s_on) {
                // row q = q0 + l -> (i2, ll) = divmod(q, Kl), advanced by s_pass
                int i2 = (q0 + l_s) / Kl, ll = (q0 + l_s) - i2 * Kl;
                for (int l = l_s; l < lb; l += s_pass) {
                    T sum = T(0);
                    if (sc < C) {
                        const T* mrow = M2 + (i2 * Rb + s_be) * RTR_MAX_RANK;
                        const T* zl = Zc[ml] + ll * Rn + s_al;
                        for (int gg = 0; gg < Rl; ++gg) sum = dfma(mrow[gg], zl[gg * zst], sum);
                    }
                    S[l * Cp + sc] = sum;
                    ll += s_pass;
                    while (ll >= Kl) { ll -= Kl; ++i2; }
                }
            }
            if (p_on) {
                const T* prow = Pt + base + (int64_t)pi * str_n;
                int i2 = (q0 + l_p) / Kl, ll = (q0 + l_p) - i2 * Kl;
                for (int l = l_p; l < lb; l += p_pass) {
                    Pv[l * Kn + pi] = prow[(int64_t)i2 * str_2 + (int64_t)ll * str_l];
                    ll += p_pass;
                    while (ll >= Kl) { ll -= Kl; ++i2; }
                }
            }
            __syncthreads();
            if (wt.active) {
#pragma unroll 2
                for (int l = 0; l < lb; ++l) {
                    const T* srow = S + l * Cp + wt.c0;
                    T sv[4];
                    if constexpr (sizeof(T) == 4) {
                        const float4 v = *reinterpret_cast<const float4*>(srow);
                        sv[0] = v.x; sv[1] = v.y; sv[2] = v.z; sv[3] = v.w;
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) sv[j] = srow[j];
                    }
                    const T* prw = Pv + l * Kn;
#pragma unroll
                    for (int k = 0; k < IP; ++k) {
                        const int i = wt.ti + wt.Ti * k;
                        const T pv = (i < Kn) ? prw[i] : T(0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[k][j] = dfma(pv, sv[j], acc[k][j]);
                    }
                }
            }
            __syncthreads();
        }
    }
    if (wt.active) {
        double* out = partial + ci.off;
#pragma unroll
        for (int k = 0; k < IP; ++k) {
            const int i = wt.ti + wt.Ti * k;
            if (i < Kn) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = wt.c0 + j;
                    if (c < C) out[(int64_t)i * C + c] = (double)acc[k][j];
                }
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(CT_THREADS) bcontract_kernel(const BTensor<T>* __restrict__ tens,
                                                               const CItem* __restrict__ items, int nitems, int N,
                                                               int n, double* __restrict__ partial, int stage,
                                                               int k2max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* M0 = reinterpret_cast<T*>(smem_raw);          // 16 x 16
    T* M1 = M0 + RTR_MAX_RANK * RTR_MAX_RANK;        // 16 x 16
    T* S = M1 + RTR_MAX_RANK * RTR_MAX_RANK;         // LB x Cp (Cp <= 144)
    T* Pv = S + LB * 144;                            // LB x K_n (K_n <= 64)
    T* M2 = Pv + LB * 64;                            // k2max x 16 x 16
    T* Zs0 = M2 + (size_t)k2max * RTR_MAX_RANK * RTR_MAX_RANK;   // the other cores (if `stage`)
    // this item's tensor descriptor, cached in shared memory: reading it from
    // the global BTensor inside the loops would repeat dependent global loads
    __shared__ int sK[RTR_MAXN], sR[RTR_MAXN], scyc[RTR_MAXN];
    __shared__ int64_t sstride[RTR_MAXN];
    __shared__ const T* sZ[RTR_MAXN];
    __shared__ const T* sP;
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const CItem ci = items[it];
        __syncthreads();                             // previous item done with the shared state
        if (tid < N) {
            const BTensor<T>& b = tens[ci.t];
            sK[tid] = (int)b.K[tid];
            sR[tid] = b.R[tid];
            sstride[tid] = b.stride[tid];
            scyc[tid] = (n + tid) % N;
            sZ[tid] = b.Zt[tid];
            if (tid == 0) sP = b.P;
        }
        __syncthreads();
        // the other cores of this tensor, read many times per prefix: staged
        // in shared memory (if they fit) instead of dependent global loads
        const T* Zc[RTR_MAXN];
        {
            T* zs = Zs0;
            for (int t = 1; t < N; ++t) {
                const int m = scyc[t];
                if (stage) {
                    const int cnt = sR[m] * sK[m] * sR[(m + 1) % N];
                    for (int e = tid; e < cnt; e += blockDim.x) zs[e] = sZ[m][e];
                    Zc[m] = zs;
                    zs += cnt;
                } else {
                    Zc[m] = sZ[m];
                }
            }
        }
        const int C = sR[(n + 1) % N] * sR[n];
        const rtr::WTile wt = rtr::wtile(C, sK[n]);
        switch (wt.ip) {
#define RTR_IP_CASE(v) case v: bcontract_item<T, v>(ci, N, n, partial, sK, sR, scyc, sstride, Zc, sP, M0, M1, M2, S, Pv, wt); break;
            RTR_IP_CASE(1) RTR_IP_CASE(2) RTR_IP_CASE(3) RTR_IP_CASE(4) RTR_IP_CASE(5)
            RTR_IP_CASE(6) RTR_IP_CASE(7) RTR_IP_CASE(8) RTR_IP_CASE(9)
            default: bcontract_item<T, rtr::TILE_IP>(ci, N, n, partial, sK, sR, scyc, sstride, Zc, sP, M0, M1, M2, S, Pv, wt); break;
#undef RTR_IP_CASE
        }
    }
}

// E_m[(a, a'), (b, b')] = sum_i Z[a, i, b] Z[a', i, b']   (block-wide)
template <typename T>
__device__ void transfer_block(const T* __restrict__ Z, int Ra, int Km, int Rb, T* __restrict__ E) {
    const int total = Ra * Ra * Rb * Rb;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int col = e % (Rb * Rb), row = e / (Rb * Rb);
        const int a = row / Ra, a2 = row % Ra, bb = col / Rb, b2 = col % Rb;
        T s = T(0);
#pragma unroll 4
        for (int i = 0; i < Km; ++i) s = dfma(Z[((int64_t)a * Km + i) * Rb + bb], Z[((int64_t)a2 * Km + i) * Rb + b2], s);
        E[e] = s;
    }
}

// ---- start: ||P||^2, default start cores, their transfer matrices ------------
// Default start (the same as the single-tensor path): entry e of core m is the
// float64 table value picked by field e % 20 of Philox4x64-10 with counter
// (e / 20, 0, 0, 0) and key (seed + 1, 256 + m).
template <typename T>
__global__ void __launch_bounds__(SV_THREADS) binit_kernel(const BTensor<T>* __restrict__ tens, int N,
                                                           const double* __restrict__ tab) {
    __shared__ double red[32];
    const BTensor<T>& b = tens[blockIdx.x];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < b.numel; e += blockDim.x) {
        const double v = (double)b.P[e];
        s += v * v;
    }
    s = rtr::block_sum(s, red);
    if (threadIdx.x == 0) b.scal[0] = s;
    for (int m = 0; m < N; ++m) {
        const int64_t cnt = (int64_t)b.R[m] * b.K[m] * b.R[(m + 1) % N];
        for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
            uint64_t c0 = (uint64_t)(e / 20), c1 = 0, c2 = 0, c3 = 0;
            rtr::philox4x64_10(c0, c1, c2, c3, b.seed + 1, 256 + (uint64_t)m);
            const uint64_t w[4] = {c0, c1, c2, c3};
            b.Zt[m][e] = (T)tab[rtr::omega_field(w, (int)(e % 20))];
        }
    }
    __syncthreads();
    for (int m = 0; m < N; ++m) transfer_block<T>(b.Zt[m], b.R[m], (int)b.K[m], b.R[(m + 1) % N], b.E[m]);
}

// scale every core by (||P|| / ||TR(Z)||)^(1/N), ||TR(Z)||^2 = trace(E_0 ... E_{N-1})
template <typename T>
__global__ void __launch_bounds__(SV_THREADS) bscale_kernel(const BTensor<T>* __restrict__ tens, int N) {
    const BTensor<T>& b = tens[blockIdx.x];
    __shared__ double sc;
    if (threadIdx.x == 0) {
        double tr = 0.0;
        const int r0 = b.R[0] * b.R[0];
        for (int r = 0; r < r0; ++r) tr += b.trace[r];
        sc = pow(sqrt(b.scal[0]) / sqrt(fmax(tr, 1e-300)), 1.0 / N);
    }
    __syncthreads();
    const T s = (T)sc, s2 = (T)(sc * sc);
    for (int m = 0; m < N; ++m) {
        const int64_t cnt = (int64_t)b.R[m] * b.K[m] * b.R[(m + 1) % N];
        for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
            const T z = b.Zt[m][e] * s;
            b.Zt[m][e] = z;
            b.Zo[m][e] = (double)z;
        }
        const int64_t ecnt = (int64_t)b.R[m] * b.R[m] * b.R[(m + 1) % N] * b.R[(m + 1) % N];
        for (int64_t e = threadIdx.x; e < ecnt; e += blockDim.x) b.E[m][e] *= s2;
    }
}

// ---- solve the normal equations of core n, one CTA per tensor ---------------
template <typename T>
__global__ void __launch_bounds__(SV_THREADS) bsolve_kernel(const BTensor<T>* __restrict__ tens, int N, int n,
                                                            const double* __restrict__ partial, int sweep, int sweeps,
                                                            double* __restrict__ err, int* __restrict__ flags,
                                                            int cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ T sc[MAXC];
    __shared__ T invd[MAXC];
    const BTensor<T>& b = tens[blockIdx.x];
    const int Rn = b.R[n], Rb = b.R[(n + 1) % N];
    const int C = Rn * Rb;
    const int Kn = (int)b.K[n];
    const int KC = Kn * C;
    T* L = reinterpret_cast<T*>(smem_raw);           // C x C
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    // W = sum of this tensor's partials, fixed order
    const double* pp = partial + b.part_off[n];
    const int np = b.nitems[n];
    for (int e = tid; e < KC; e += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < np; ++q) s += pp[(int64_t)q * KC + e];
        b.W[e] = s;
    }
    // equilibrated Gram: D G D, D = diag(G)^-1/2
    for (int c = tid; c < C; c += blockDim.x) {
        const T d = b.G[(int64_t)c * C + c];
        sc[c] = (d > T(0)) ? T(1) / sqrt(d) : T(0);
    }
    __syncthreads();
    // ridges tried in turn (relative to the unit diagonal): the first is the
    // plain factorisation; float32 Gram matrices of nearly rank-deficient
    // subchains can lose positive definiteness to rounding
    bool ok = false;
    for (int attempt = 0; attempt < 5 && !ok; ++attempt) {
        const T ridge = attempt == 0 ? T(0)
                        : (std::is_same<T, double>::value ? T(pow(10.0, -12.0 + 4.0 * (attempt - 1)))
                                                          : T(pow(10.0, -6.0 + 2.0 * (attempt - 1))));
        for (int e = tid; e < C * C; e += blockDim.x) {
            const int c = e / C, c2 = e % C;
            L[e] = b.G[e] * sc[c] * sc[c2] + (c == c2 ? ridge : T(0));
        }
        __syncthreads();
        ok = rtr::block_cholesky<T>(L, C, C);
        if (!ok && attempt == 0 && tid == 0) atomicOr(flags, RTR_FLAG_GRAM_PINV);
    }
    if (!ok) {
        if (tid == 0) atomicOr(flags, RTR_FLAG_NONFINITE);
        return;
    }
    for (int c = tid; c < C; c += blockDim.x) invd[c] = T(1) / L[c * C + c];
    __syncthreads();
    // one warp per right-hand side i: (L L^T) y = D w_i, z_i = D y
    double zw = 0.0;
    for (int i = warp; i < Kn; i += nw) {
        T y[MAXC / 32];
        double wv[MAXC / 32];
#pragma unroll
        for (int q = 0; q < MAXC / 32; ++q) {
            const int j = lane + 32 * q;
            wv[q] = (j < C) ? b.W[(int64_t)i * C + j] : 0.0;
            y[q] = (j < C) ? (T)wv[q] * sc[j] : T(0);
        }
#pragma unroll
        for (int ks = 0; ks < MAXC / 32; ++ks) {
            for (int kk = 0; kk < 32; ++kk) {
                const int k = ks * 32 + kk;
                if (k >= C) break;
                const T yk = __shfl_sync(0xffffffffu, y[ks], kk) * invd[k];
                if (lane == kk) y[ks] = yk;
#pragma unroll
                for (int q = 0; q < MAXC / 32; ++q) {
                    const int j = lane + 32 * q;
                    if (j > k && j < C) y[q] -= L[j * C + k] * yk;
                }
            }
        }
#pragma unroll
        for (int ks = MAXC / 32 - 1; ks >= 0; --ks) {
            for (int kk = 31; kk >= 0; --kk) {
                const int k = ks * 32 + kk;
                if (k >= C) continue;
                const T xk = __shfl_sync(0xffffffffu, y[ks], kk) * invd[k];
                if (lane == kk) y[ks] = xk;
#pragma unroll
                for (int q = 0; q < MAXC / 32; ++q) {
                    const int j = lane + 32 * q;
                    if (j < k) y[q] -= L[k * C + j] * xk;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < MAXC / 32; ++q) {
            const int j = lane + 32 * q;
            if (j < C) {
                const T z = y[q] * sc[j];
                const int be = j / Rn, al = j % Rn;
                const int64_t o = ((int64_t)al * Kn + i) * Rb + be;
                b.Zt[n][o] = z;
                b.Zo[n][o] = (double)z;
                zw += (double)z * wv[q];
            }
        }
    }
    zw = rtr::block_sum(zw, red);
    if (err && n == N - 1 && tid == 0) err[(int64_t)blockIdx.x * sweeps + sweep] = sqrt(fmax(b.scal[0] - zw, 0.0));
    __syncthreads();
    // E_n of the new core, from a shared-memory copy of it (the Cholesky
    // factor's space is free now) when it fits
    const T* zsrc = b.Zt[n];
    if ((int64_t)C * Kn <= (int64_t)cap) {
        for (int e = tid; e < C * Kn; e += blockDim.x) L[e] = b.Zt[n][e];
        __syncthreads();
        zsrc = L;
    }
    transfer_block<T>(zsrc, Rn, Kn, Rb, b.E[n]);
}

template <typename T>
struct Impl {
    int count = 0, N = 0, sweeps = 0, num_sms = 0;
    BTensor<T>* d_tens = nullptr;
    std::vector<CItem*> d_citems;
    std::vector<int> n_citems;
    std::vector<GItem*> d_gitems;
    std::vector<int> n_gitems;
    GItem* d_titems = nullptr;
    int n_titems = 0;
    double* partial = nullptr;
    void* scratch = nullptr;
    int* flags = nullptr;
    const double* tab = nullptr;
    size_t ct_smem = 0, sv_smem = 0;
    int ct_stage = 0;
    int k2max = 1;                  // largest K of a mode streamed as c_{N-2} by the contraction
};

}  // namespace

struct BatchAls {
    int is_f64 = 0;
    void* impl = nullptr;
};

namespace {

template <typename T>
void free_impl(Impl<T>* m) {
    if (!m) return;
    cudaFree(m->d_tens);
    for (auto* p : m->d_citems) cudaFree(p);
    for (auto* p : m->d_gitems) cudaFree(p);
    cudaFree(m->d_titems);
    cudaFree(m->partial);
    cudaFree(m->scratch);
    cudaFree(m->flags);
    delete m;
}

template <typename T>
int create_impl(Impl<T>** out, int count, int N, const int64_t* K, const int* R, int sweeps, const uint64_t* seeds,
                const double* tab, const void* const* P, double* const* Z, int num_sms) {
    auto* m = new (std::nothrow) Impl<T>();
    if (!m) return rtr_set_error(RTR_ENOMEM, "host allocation failed");
    m->count = count; m->N = N; m->sweeps = sweeps; m->num_sms = num_sms; m->tab = tab;
    std::vector<BTensor<T>> h(count);
    // scratch layout per tensor (256-byte aligned pieces)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    std::vector<size_t> off(count);
    size_t total = 0;
    int64_t maxKn = 1;
    int cmax = 1;
    for (int t = 0; t < count; ++t) {
        const int64_t* k = K + (size_t)t * N;
        const int* r = R + (size_t)t * N;
        off[t] = total;
        size_t sz = 0, gmax = 0, wmax = 0;
        for (int n = 0; n < N; ++n) {
            const int rb = r[(n + 1) % N];
            sz += al(sizeof(T) * r[n] * k[n] * rb);                 // Zt
            sz += al(sizeof(T) * r[n] * r[n] * rb * rb);            // E
            gmax = std::max<size_t>(gmax, (size_t)r[n] * rb * r[n] * rb);
            wmax = std::max<size_t>(wmax, (size_t)k[n] * r[n] * rb);
            maxKn = std::max<int64_t>(maxKn, k[n]);
            cmax = std::max(cmax, r[n] * rb);
        }
        sz += al(sizeof(T) * gmax) + al(sizeof(double) * wmax) + al(sizeof(double) * r[0] * r[0]) + al(64);
        total += sz;
    }
    if (cudaMalloc(&m->scratch, std::max<size_t>(total, 256)) != cudaSuccess) {
        cudaGetLastError(); free_impl(m);
        return rtr_set_error(RTR_ENOMEM, "batch ALS scratch (%zu B) allocation failed", total);
    }
    uint8_t* base = reinterpret_cast<uint8_t*>(m->scratch);
    for (int t = 0; t < count; ++t) {
        const int64_t* k = K + (size_t)t * N;
        const int* r = R + (size_t)t * N;
        BTensor<T>& b = h[t];
        b = BTensor<T>{};
        uint8_t* q = base + off[t];
        size_t gmax = 0, wmax = 0;
        int64_t st = 1, numel = 1;
        for (int n = N - 1; n >= 0; --n) { b.stride[n] = st; st *= k[n]; }
        for (int n = 0; n < N; ++n) {
            const int rb = r[(n + 1) % N];
            b.K[n] = k[n];
            b.R[n] = r[n];
            numel *= k[n];
            b.Zt[n] = reinterpret_cast<T*>(q); q += al(sizeof(T) * r[n] * k[n] * rb);
            b.E[n] = reinterpret_cast<T*>(q);  q += al(sizeof(T) * r[n] * r[n] * rb * rb);
            b.Zo[n] = Z[(size_t)t * N + n];
            gmax = std::max<size_t>(gmax, (size_t)r[n] * rb * r[n] * rb);
            wmax = std::max<size_t>(wmax, (size_t)k[n] * r[n] * rb);
        }
        b.G = reinterpret_cast<T*>(q); q += al(sizeof(T) * gmax);
        b.W = reinterpret_cast<double*>(q); q += al(sizeof(double) * wmax);
        b.trace = reinterpret_cast<double*>(q); q += al(sizeof(double) * r[0] * r[0]);
        b.scal = reinterpret_cast<double*>(q);
        b.P = reinterpret_cast<const T*>(P[t]);
        b.numel = numel;
        b.seed = seeds[t];
    }
    // contraction items per mode: prefixes of tensor t split into chunks of
    // about equal work (target: 4 items per SM over the batch)
    int64_t part_max = 0;
    for (int n = 0; n < N; ++n) {
        std::vector<double> wpre(count);
        std::vector<int64_t> jpre(count);
        double wsum = 0.0;
        for (int t = 0; t < count; ++t) {
            const BTensor<T>& b = h[t];
            // a prefix fixes the cyclic modes n+1 .. n+N-3; the rows of one prefix
            // run over the last two (n+N-2, n+N-1)
            int64_t J = 1;
            for (int s = 1; s <= N - 3; ++s) J *= b.K[(n + s) % N];
            const int ml = (n + N - 1) % N, m2 = (n + N - 2) % N;
            const double C = (double)b.R[n] * b.R[(n + 1) % N];
            const double rows = (double)b.K[m2] * b.K[ml];
            const double per = rows * (C * b.R[ml] + (double)b.K[n] * C) +
                               (double)b.K[m2] * b.R[(n + 1) % N] * b.R[ml] * b.R[m2] + 4096.0;
            jpre[t] = J;
            wpre[t] = per;
            wsum += per * J;
        }
        const double target = std::max(1.0, wsum / (4.0 * num_sms));
        std::vector<CItem> items;
        int64_t poff = 0;
        for (int t = 0; t < count; ++t) {
            const int64_t chunk = std::max<int64_t>(1, (int64_t)std::floor(target / wpre[t]));
            const int64_t KC = h[t].K[n] * h[t].R[n] * h[t].R[(n + 1) % N];
            h[t].part_off[n] = poff;
            int cnt = 0;
            for (int64_t j = 0; j < jpre[t]; j += chunk) {
                items.push_back(CItem{t, j, std::min(jpre[t], j + chunk), poff});
                poff += KC;
                ++cnt;
            }
            h[t].nitems[n] = cnt;
        }
        part_max = std::max(part_max, poff);
        CItem* d = nullptr;
        if (cudaMalloc(&d, sizeof(CItem) * items.size()) != cudaSuccess) { cudaGetLastError(); free_impl(m); return rtr_set_error(RTR_ENOMEM, "item table allocation failed"); }
        m->d_citems.push_back(d);
        m->n_citems.push_back((int)items.size());
        RTR_CUDA(cudaMemcpy(d, items.data(), sizeof(CItem) * items.size(), cudaMemcpyHostToDevice));
        // Gram rows of the update of mode n: rows of E_{n+1}
        std::vector<GItem> g;
        for (int t = 0; t < count; ++t) {
            const int rr = h[t].R[(n + 1) % N];
            for (int r0 = 0; r0 < rr * rr; r0 += GB) g.push_back(GItem{t, r0});
        }
        GItem* dg = nullptr;
        if (cudaMalloc(&dg, sizeof(GItem) * g.size()) != cudaSuccess) { cudaGetLastError(); free_impl(m); return rtr_set_error(RTR_ENOMEM, "item table allocation failed"); }
        m->d_gitems.push_back(dg);
        m->n_gitems.push_back((int)g.size());
        RTR_CUDA(cudaMemcpy(dg, g.data(), sizeof(GItem) * g.size(), cudaMemcpyHostToDevice));
    }
    {
        std::vector<GItem> g;
        for (int t = 0; t < count; ++t)
            for (int r0 = 0; r0 < h[t].R[0] * h[t].R[0]; r0 += GB) g.push_back(GItem{t, r0});
        if (cudaMalloc(&m->d_titems, sizeof(GItem) * g.size()) != cudaSuccess) { cudaGetLastError(); free_impl(m); return rtr_set_error(RTR_ENOMEM, "item table allocation failed"); }
        m->n_titems = (int)g.size();
        RTR_CUDA(cudaMemcpy(m->d_titems, g.data(), sizeof(GItem) * g.size(), cudaMemcpyHostToDevice));
    }
    if (cudaMalloc(&m->partial, sizeof(double) * std::max<int64_t>(part_max, 1)) != cudaSuccess ||
        cudaMalloc(&m->d_tens, sizeof(BTensor<T>) * count) != cudaSuccess ||
        cudaMalloc(&m->flags, sizeof(int)) != cudaSuccess) {
        cudaGetLastError(); free_impl(m);
        return rtr_set_error(RTR_ENOMEM, "batch ALS allocation failed");
    }
    RTR_CUDA(cudaMemcpy(m->d_tens, h.data(), sizeof(BTensor<T>) * count, cudaMemcpyHostToDevice));
    RTR_CUDA(cudaMemset(m->flags, 0, sizeof(int)));
    // contraction: fixed part, plus the other cores of the largest update if
    // everything fits in 96 KB
    size_t zmax = 0;
    for (int t = 0; t < count; ++t)
        for (int n = 0; n < N; ++n) {
            size_t z = 0;
            for (int q = 1; q < N; ++q) {
                const int mm = (n + q) % N;
                z += (size_t)h[t].R[mm] * h[t].K[mm] * h[t].R[(mm + 1) % N];
            }
            zmax = std::max(zmax, z);
        }
    (void)maxKn;
    m->k2max = 1;
    for (int t = 0; t < count; ++t)
        for (int n = 0; n < N; ++n) m->k2max = std::max<int>(m->k2max, (int)h[t].K[(n + N - 2) % N]);
    m->ct_smem = sizeof(T) * (2 * RTR_MAX_RANK * RTR_MAX_RANK + LB * 144 + LB * 64 +
                              (size_t)m->k2max * RTR_MAX_RANK * RTR_MAX_RANK);
    m->ct_stage = (m->ct_smem + sizeof(T) * zmax <= 96 * 1024) ? 1 : 0;
    if (m->ct_stage) m->ct_smem += sizeof(T) * zmax;
    m->sv_smem = sizeof(T) * (size_t)cmax * cmax;
    *out = m;
    return RTR_OK;
}

template <typename T>
int run_impl(Impl<T>* m, double* err, cudaStream_t s) {
    const int N = m->N;
    auto gram = bgram_kernel<T>;
    auto contract = bcontract_kernel<T>;
    auto solve = bsolve_kernel<T>;
    RTR_SMEM(contract, m->ct_smem);
    RTR_SMEM(solve, m->sv_smem);
    const size_t gsmem = sizeof(T) * 3 * GB * 256;
    RTR_SMEM(gram, gsmem);
    binit_kernel<T><<<m->count, SV_THREADS, 0, s>>>(m->d_tens, N, m->tab);
    RTR_LAUNCH_CHECK("binit_kernel");
    gram<<<(unsigned)std::min(m->n_titems, 4 * m->num_sms), CT_THREADS, gsmem, s>>>(m->d_tens, m->d_titems,
                                                                                    m->n_titems, N, 0, N, 1);
    RTR_LAUNCH_CHECK("bgram_kernel");
    bscale_kernel<T><<<m->count, SV_THREADS, 0, s>>>(m->d_tens, N);
    RTR_LAUNCH_CHECK("bscale_kernel");
    for (int sw = 0; sw < m->sweeps; ++sw) {
        for (int n = 0; n < N; ++n) {
            gram<<<(unsigned)std::min(m->n_gitems[n], 4 * m->num_sms), CT_THREADS, gsmem, s>>>(
                m->d_tens, m->d_gitems[n], m->n_gitems[n], N, (n + 1) % N, N - 1, 0);
            RTR_LAUNCH_CHECK("bgram_kernel");
            contract<<<(unsigned)std::min(m->n_citems[n], 4 * m->num_sms), CT_THREADS, m->ct_smem, s>>>(
                m->d_tens, m->d_citems[n], m->n_citems[n], N, n, m->partial, m->ct_stage, m->k2max);
            RTR_LAUNCH_CHECK("bcontract_kernel");
            solve<<<m->count, SV_THREADS, m->sv_smem, s>>>(m->d_tens, N, n, m->partial, sw, m->sweeps, err,
                                                           m->flags, (int)(m->sv_smem / sizeof(T)));
            RTR_LAUNCH_CHECK("bsolve_kernel");
        }
    }
    return RTR_OK;
}

}  // namespace

int batch_als_create(BatchAls** out, int count, int N, const int64_t* K, const int* R, int is_f64, int sweeps,
                     const uint64_t* seeds, const double* tab, const void* const* P, double* const* Z, int num_sms) {
    *out = nullptr;
    for (int t = 0; t < count; ++t)
        for (int n = 0; n < N; ++n) {
            const int C = R[(size_t)t * N + n] * R[(size_t)t * N + (n + 1) % N];
            const int64_t k = K[(size_t)t * N + n];
            if (C > 144 || k > 64 || k * C > 10240)
                return rtr_set_error(RTR_EUNSUPPORTED, "grouped TR-ALS: tensor %d mode %d out of range", t, n);
        }
    auto* b = new (std::nothrow) BatchAls();
    if (!b) return rtr_set_error(RTR_ENOMEM, "host allocation failed");
    b->is_f64 = is_f64;
    int st;
    if (is_f64) {
        Impl<double>* m = nullptr;
        st = create_impl<double>(&m, count, N, K, R, sweeps, seeds, tab, P, Z, num_sms);
        b->impl = m;
    } else {
        Impl<float>* m = nullptr;
        st = create_impl<float>(&m, count, N, K, R, sweeps, seeds, tab, P, Z, num_sms);
        b->impl = m;
    }
    if (st) { delete b; return st; }
    *out = b;
    return RTR_OK;
}

void batch_als_destroy(BatchAls* b) {
    if (!b) return;
    if (b->is_f64) free_impl(static_cast<Impl<double>*>(b->impl));
    else free_impl(static_cast<Impl<float>*>(b->impl));
    delete b;
}

int batch_als_run(BatchAls* b, double* err, cudaStream_t s) {
    if (b->is_f64) return run_impl(static_cast<Impl<double>*>(b->impl), err, s);
    return run_impl(static_cast<Impl<float>*>(b->impl), err, s);
}

int batch_als_flags(BatchAls* b, int* flags) {
    int* d = b->is_f64 ? static_cast<Impl<double>*>(b->impl)->flags : static_cast<Impl<float>*>(b->impl)->flags;
    RTR_CUDA(cudaDeviceSynchronize());
    RTR_CUDA(cudaMemcpy(flags, d, sizeof(int), cudaMemcpyDeviceToHost));
    RTR_CUDA(cudaMemset(d, 0, sizeof(int)));
    return RTR_OK;
}
