// Register-tiled block update of the TR-ALS contraction (Eq. 2):
//     W[i, c] += sum_l Pv[l, i] S[l, c]     l < lb <= 16
// for one block of last-mode indices, with Pv (lb x K_n) and S (lb x Cp) in
// shared memory.  Each thread owns 4 consecutive c (S rows are padded to
// Cp = 4 ceil(C / 4) with zeros) times up to TILE_IP values of i spaced Ti
// apart, so one S quad and one Pv value feed 4 FMAs.
#pragma once
#include "rtr_internal.cuh"

namespace rtr {

constexpr int TILE_IP = 10;     // i values per thread: ceil(K_n / Ti) <= 10 for K_n <= 64, C <= 144

struct WTile {
    int Ti, ti, c0, ip;
    bool active;
};

__device__ __forceinline__ int tile_cp(int C) { return (C + 3) & ~3; }

__device__ __forceinline__ WTile wtile(int C, int Kn) {
    WTile w;
    const int Tc = (C + 3) >> 2;
    w.Ti = max(1, (int)blockDim.x / Tc);
    w.ti = (int)threadIdx.x / Tc;
    w.c0 = 4 * ((int)threadIdx.x % Tc);
    w.ip = (Kn + w.Ti - 1) / w.Ti;
    w.active = w.ti < w.Ti;
    return w;
}

template <typename T>
__device__ __forceinline__ void wtile_zero(T (&acc)[TILE_IP][4]) {
#pragma unroll
    for (int k = 0; k < TILE_IP; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = T(0);
}

template <typename T>
__device__ __forceinline__ void wtile_accum(T (&acc)[TILE_IP][4], const WTile& w, const T* Pv, int Kn, const T* S,
                                            int Cp, int lb) {
    if (!w.active) return;
#pragma unroll 2
    for (int l = 0; l < lb; ++l) {
        const T* srow = S + l * Cp + w.c0;
        T s[4];
        if constexpr (sizeof(T) == 4) {
            const float4 v = *reinterpret_cast<const float4*>(srow);
            s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
        } else {
            const double2 a = *reinterpret_cast<const double2*>(srow);
            const double2 b = *reinterpret_cast<const double2*>(srow + 2);
            s[0] = a.x; s[1] = a.y; s[2] = b.x; s[3] = b.y;
        }
        const T* prow = Pv + l * Kn;
#pragma unroll
        for (int k = 0; k < TILE_IP; ++k) {
            const int i = w.ti + w.Ti * k;
            if (k < w.ip && i < Kn) {
                const T p = prow[i];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[k][j] = fma(p, s[j], acc[k][j]);
            }
        }
    }
}

// out[i * C + c] = acc (converted to O), for the valid (i, c) of this thread
template <typename T, typename O>
__device__ __forceinline__ void wtile_store(const T (&acc)[TILE_IP][4], const WTile& w, int Kn, int C,
                                            O* __restrict__ out) {
    if (!w.active) return;
#pragma unroll
    for (int k = 0; k < TILE_IP; ++k) {
        const int i = w.ti + w.Ti * k;
        if (k < w.ip && i < Kn) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = w.c0 + j;
                if (c < C) out[(int64_t)i * C + c] = (O)acc[k][j];
            }
        }
    }
}

}  // namespace rtr
