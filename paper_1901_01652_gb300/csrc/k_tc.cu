// tcgen05 (5th-generation tensor core) Gaussian sketch, Algorithm 1 step 5:
//     Y_n[i, k] = sum_r X_(n)[i, r] Omega_n[r, k]
// with X float32 in HBM split in registers into bfloat16 hi + lo
// (x ~= hi + lo to ~2^-17 relative), Omega_n exactly bfloat16 (the
// bfloat16-rounded quantile table), FP32 accumulation in TMEM:
//     D[i, k] += A_hi[i, r] B[r, k] + A_lo[i, r] B[r, k].
//
// CTA = 11 warps, one CTA per SM (smem-bound), persistent over chunks of 64
// consecutive r (grid-stride):
//   warps 0-7  converters: vectorised global loads of X, hi/lo split, stores
//              into 128B-swizzled K-major tiles; then the epilogue (TMEM ->
//              float64 partials)
//   warps 8-9  Omega generators: Philox4x64-10 + table lookup into the B tile
//   warp 10    one elected lane issues tcgen05.mma and commits stage releases
// A ring of S stages (A_hi, A_lo, B per stage) is handed over with mbarriers;
// every wait is bounded (tc_common.cuh) and raises RTR_FLAG_TIMEOUT.
// The accumulators D (one 128 x N block per 128-row M tile) live in TMEM.
#include <algorithm>
#include <type_traits>
#include <cuda.h>
#include <cudaTypedefs.h>
#include "rtr_internal.cuh"
#include "tc_common.cuh"

namespace {

// Position of a role's local step t in a ring of S slots (slot = t mod S,
// use = t div S), advanced without divisions: 64-bit integer division is a
// long subroutine, far too slow for a per-chunk loop.
struct Ring {
    int slot = 0, S = 1;
    uint32_t use = 0;
    __device__ explicit Ring(int S_, int t0 = 0) : S(S_) { step(t0); }
    __device__ void step(int by) {
        slot += by;
        while (slot >= S) { slot -= S; ++use; }
    }
};

// (a, b-chunk) of chunk ch = a * nbc + bi, for ch = ch0, ch0 + stride, ...
struct ChunkPos {
    int64_t a, bi, qa, qb, nbc;
    __device__ ChunkPos(int64_t ch0, int64_t stride, int64_t nbc_) : nbc(nbc_) {
        a = ch0 / nbc; bi = ch0 % nbc; qa = stride / nbc; qb = stride % nbc;
    }
    __device__ void step() {
        bi += qb; a += qa;
        if (bi >= nbc) { bi -= nbc; ++a; }
    }
};

using namespace rtr::tc;

constexpr int CONV_WARPS = 8;
constexpr int RNG_WARPS = 2;
constexpr int MMA_WARP = CONV_WARPS + RNG_WARPS;
constexpr int NTHREADS = (CONV_WARPS + RNG_WARPS + 1) * 32;
constexpr int CONV_THREADS = CONV_WARPS * 32;
constexpr int RNG_THREADS = RNG_WARPS * 32;
constexpr int KC = 64;                       // reduction values per chunk (one 128-byte bf16 row)
constexpr uint32_t MTILE_BYTES = 128 * 128;  // 128 rows x 128 bytes

struct SketchTCArgs {
    const float* X;
    int64_t A, B;
    int I, K, N, MT, rows_cta, S;
    int64_t nchunks, nbc;
    int64_t aoff;                 // index of the view's first a in the whole tensor (slabs)
    uint64_t seed;
    int mode;
    int vec;                      // 1: 16-byte vector loads are legal
    int fp8;                      // 1: block-scaled float8 values, one MMA (last mode, vec only)
    const uint16_t* tab;          // bfloat16 table (global)
    double* partial;              // [gridDim.x][I][K]
    double* normp;                // [gridDim.y * gridDim.x] or null
    int* flags;
};

__global__ void __launch_bounds__(NTHREADS, 1) sketch_tc_kernel(const SketchTCArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    const uint32_t a_bytes = (uint32_t)p.MT * MTILE_BYTES;
    const uint32_t b_bytes = (uint32_t)p.N * 128u;
    const uint32_t stage_bytes = 2 * a_bytes + b_bytes;
    const int S = p.S;
    uint16_t* tab = reinterpret_cast<uint16_t*>(sm + S * stage_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tab + 4096);
    uint64_t* fullA = bars;
    uint64_t* fullB = bars + S;
    uint64_t* empty = bars + 2 * S;
    uint64_t* accf = bars + 3 * S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    double* nred = reinterpret_cast<double*>(bars + 3 * S + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = (uint32_t)(p.MT * p.N);

    // ---- set-up: zero all operand tiles (padding rows/columns stay zero), table, barriers, TMEM
    {
        const uint32_t base = smem_u32(sm);
        for (uint32_t off = tid * 16u; off < (uint32_t)S * stage_bytes; off += NTHREADS * 16u)
            asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(base + off), "r"(0) : "memory");
        for (int j = tid; j < 4096; j += NTHREADS) tab[j] = p.tab[j];
        if (tid == 0) {
            for (int s = 0; s < S; ++s) {
                mbar_init(&fullA[s], CONV_THREADS);
                mbar_init(&fullB[s], RNG_THREADS);
                mbar_init(&empty[s], 1);
            }
            mbar_init(accf, 1);
            *abort = 0;
            mbar_fence_init();
        }
        if (warp == MMA_WARP) tmem_alloc(tmem_slot, ncols);
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    const uint32_t tmem = *tmem_slot;
    const int rbeg = blockIdx.y * p.rows_cta;
    const int rows_valid = min(p.rows_cta, p.I - rbeg);
    const int64_t nloc = (blockIdx.x < p.nchunks) ? (p.nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t stage0 = smem_u32(sm);
    double nsum = 0.0;

    if (warp < CONV_WARPS) {
        // ================================================================ converters
        const int ct = tid;
        const bool want_norm = p.normp != nullptr;   // ||X||^2 only in the pass that records it
        Ring rg(S);
        ChunkPos cp(blockIdx.x, gridDim.x, p.nbc);
        for (int64_t t = 0; t < nloc; ++t, rg.step(1), cp.step()) {
            const int64_t ch = blockIdx.x + t * gridDim.x;
            const int s = rg.slot;
            const uint32_t u = rg.use;
            if (t >= S && !mbar_wait(&empty[s], (u - 1) & 1, abort, p.flags)) break;
            const uint32_t hi_base = stage0 + s * stage_bytes;
            const uint32_t lo_base = hi_base + a_bytes;
            float csum = 0.f;
            if (p.B > 1) {
                const int64_t a = cp.a, b0 = cp.bi * KC;
                const int len = (int)min((int64_t)KC, p.B - b0);
                const float* xrow0 = p.X + ((int64_t)a * p.I + rbeg) * p.B + b0;
                if (p.vec && len == KC) {
                    // piece = (row, 16-byte column group c4): 16 pieces per row
                    const int npieces = rows_valid * 16;
                    float4 v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int pc = ct + CONV_THREADS * j;
                        if (pc < npieces)
                            v[j] = __ldg(reinterpret_cast<const float4*>(xrow0 + (int64_t)(pc >> 4) * p.B) + (pc & 15));
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int pc = ct + CONV_THREADS * j;
                        if (pc < npieces) {
                            const int row = pc >> 4, c4 = pc & 15;
                            uint32_t h0, l0, h1, l1;
                            split2(v[j].x, v[j].y, h0, l0);
                            split2(v[j].z, v[j].w, h1, l1);
                            csum += v[j].x * v[j].x + v[j].y * v[j].y + v[j].z * v[j].z + v[j].w * v[j].w;
                            const uint32_t off = (uint32_t)(row >> 7) * MTILE_BYTES + sw128_off(row & 127, 4 * c4);
                            st_shared_v2(hi_base + off, h0, h1);
                            st_shared_v2(lo_base + off, l0, l1);
                        }
                    }
                } else {
                    for (int e = ct; e < rows_valid * (KC / 2); e += CONV_THREADS) {
                        const int row = e / (KC / 2), kp = e % (KC / 2);
                        const int k0 = 2 * kp;
                        const float x0 = (k0 < len) ? xrow0[(int64_t)row * p.B + k0] : 0.f;
                        const float x1 = (k0 + 1 < len) ? xrow0[(int64_t)row * p.B + k0 + 1] : 0.f;
                        uint32_t h, l;
                        split2(x0, x1, h, l);
                        csum += x0 * x0 + x1 * x1;
                        const uint32_t off = (uint32_t)(row >> 7) * MTILE_BYTES + sw128_off(row & 127, k0);
                        st_shared_u32(hi_base + off, h);
                        st_shared_u32(lo_base + off, l);
                    }
                }
            } else {
                // last mode: r = a; X[a, i] is contiguous along i, so the tile is
                // transposed on the way in: item = (pair q of r values, quad u of rows)
                const int64_t a0 = ch * KC;
                const int len = (int)min((int64_t)KC, p.A - a0);
                const float* xb = p.X + a0 * p.I + rbeg;
                if (p.vec && !p.fp8) {
                    // item = (quad u4 of rows, quad qq of r values): four coalesced
                    // float4 loads (lanes run along the contiguous i), a 4 x 4
                    // transpose in registers, then 8-byte stores of 4 consecutive r
                    const int U = rows_valid >> 2;
                    const int nitems = U * (KC / 4);
                    for (int it0 = 0; it0 < nitems; it0 += CONV_THREADS * 2) {
                        float4 x[2][4];
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int it = it0 + ct + CONV_THREADS * j;
                            const int u4 = it % U, qq = it / U;
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                x[j][t] = make_float4(0.f, 0.f, 0.f, 0.f);
                                if (it < nitems && 4 * qq + t < len)
                                    x[j][t] = __ldg(reinterpret_cast<const float4*>(xb + (int64_t)(4 * qq + t) * p.I + 4 * u4));
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int it = it0 + ct + CONV_THREADS * j;
                            if (it >= nitems) continue;
                            const int u4 = it % U, qq = it / U;
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                const float r0 = (&x[j][0].x)[v], r1 = (&x[j][1].x)[v];
                                const float r2 = (&x[j][2].x)[v], r3 = (&x[j][3].x)[v];
                                if (want_norm) csum += r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3;
                                uint32_t h0, l0, h1, l1;
                                split2(r0, r1, h0, l0);
                                split2(r2, r3, h1, l1);
                                const int row = 4 * u4 + v;
                                const uint32_t off = (uint32_t)(row >> 7) * MTILE_BYTES + sw128_off(row & 127, 4 * qq);
                                st_shared_v2(hi_base + off, h0, h1);
                                st_shared_v2(lo_base + off, l0, l1);
                            }
                        }
                    }
                } else if (p.vec) {
                    const int nitems = (rows_valid >> 2) * 32;
                    for (int it0 = 0; it0 < nitems; it0 += CONV_THREADS * 4) {
                        float4 x0[4], x1[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int it = it0 + ct + CONV_THREADS * j;
                            const int q = it & 31, u4 = it >> 5;
                            x0[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                            x1[j] = x0[j];
                            if (it < nitems) {
                                if (2 * q < len) x0[j] = __ldg(reinterpret_cast<const float4*>(xb + (int64_t)(2 * q) * p.I + 4 * u4));
                                if (2 * q + 1 < len) x1[j] = __ldg(reinterpret_cast<const float4*>(xb + (int64_t)(2 * q + 1) * p.I + 4 * u4));
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int it = it0 + ct + CONV_THREADS * j;
                            if (it >= nitems) continue;
                            const int q = it & 31, u4 = it >> 5;
                            const float a0v[4] = {x0[j].x, x0[j].y, x0[j].z, x0[j].w};
                            const float a1v[4] = {x1[j].x, x1[j].y, x1[j].z, x1[j].w};
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                const int row = 4 * u4 + v;
                                csum += a0v[v] * a0v[v] + a1v[v] * a1v[v];
                                const uint32_t off = (uint32_t)(row >> 7) * MTILE_BYTES + sw128_off(row & 127, 2 * q);
                                if (p.fp8) {
                                    // scale block = 32 consecutive r = a of this row: lanes
                                    // q = 0..15 hold r 0..31 of the chunk, q = 16..31 the rest
                                    // (the item test above is uniform per warp)
                                    const float m = group_max(fmaxf(fabsf(a0v[v]), fabsf(a1v[v])), 16);
                                    st_shared_u32(hi_base + off, mx_pair(a0v[v], a1v[v], mx_scale(m)));
                                    continue;
                                }
                                uint32_t h, l;
                                split2(a0v[v], a1v[v], h, l);
                                st_shared_u32(hi_base + off, h);
                                st_shared_u32(lo_base + off, l);
                            }
                        }
                    }
                } else {
                    for (int e = ct; e < rows_valid * (KC / 2); e += CONV_THREADS) {
                        const int q = e % (KC / 2), row = e / (KC / 2);
                        const float x0 = (2 * q < len) ? xb[(int64_t)(2 * q) * p.I + row] : 0.f;
                        const float x1 = (2 * q + 1 < len) ? xb[(int64_t)(2 * q + 1) * p.I + row] : 0.f;
                        uint32_t h, l;
                        split2(x0, x1, h, l);
                        csum += x0 * x0 + x1 * x1;
                        const uint32_t off = (uint32_t)(row >> 7) * MTILE_BYTES + sw128_off(row & 127, 2 * q);
                        st_shared_u32(hi_base + off, h);
                        st_shared_u32(lo_base + off, l);
                    }
                }
            }
            nsum += (double)csum;
            fence_proxy_async();
            mbar_arrive(&fullA[s]);
        }
    } else if (warp < MMA_WARP) {
        // ================================================================ Omega generators
        const int kk = tid - CONV_THREADS;            // 0..63: the r column this thread fills
        const int ncall = (p.K + 19) / 20;
        Ring rg(S);
        ChunkPos cp(blockIdx.x, gridDim.x, p.nbc);
        for (int64_t t = 0; t < nloc; ++t, rg.step(1), cp.step()) {
            const int64_t ch = blockIdx.x + t * gridDim.x;
            const int s = rg.slot;
            const uint32_t u = rg.use;
            int64_t r0;
            int len;
            if (p.B > 1) {
                const int64_t a = cp.a, b0 = cp.bi * KC;
                r0 = (a + p.aoff) * p.B + b0;
                len = (int)min((int64_t)KC, p.B - b0);
            } else {
                r0 = ch * KC;
                len = (int)min((int64_t)KC, p.A - r0);
                r0 += p.aoff;
            }
            if (t >= S && !mbar_wait(&empty[s], (u - 1) & 1, abort, p.flags)) break;
            const uint32_t bt = stage0 + s * stage_bytes + 2 * a_bytes;
            for (int cb = 0; cb < ncall; ++cb) {
                uint64_t w[4] = {0, 0, 0, 0};
                if (kk < len) rtr::omega_words(p.seed, p.mode, (uint64_t)(r0 + kk), (uint64_t)cb, w);
#pragma unroll
                for (int tt = 0; tt < 20; ++tt) {
                    const int k = cb * 20 + tt;
                    if (k < p.K) {
                        const uint16_t val = (kk < len) ? tab[rtr::omega_field(w, tt)] : (uint16_t)0;
                        st_shared_u16(bt + sw128_off(k, kk), val);
                    }
                }
            }
            fence_proxy_async();
            mbar_arrive(&fullB[s]);
        }
    } else {
        // ================================================================ MMA issuer
        const uint32_t idesc = idesc_bf16_f32(128, p.N);
        Ring rg(S);
        for (int64_t t = 0; t < nloc; ++t, rg.step(1)) {
            const int s = rg.slot;
            const uint32_t u = rg.use;
            if (!mbar_wait(&fullA[s], u & 1, abort, p.flags)) break;
            if (!mbar_wait(&fullB[s], u & 1, abort, p.flags)) break;
            tc_fence_after();
            if (lane == 0) {
                const uint32_t ahi = stage0 + s * stage_bytes, alo = ahi + a_bytes, bb = ahi + 2 * a_bytes;
                for (int m = 0; m < p.MT; ++m) {
                    const uint32_t d = tmem + (uint32_t)(m * p.N);
#pragma unroll
                    for (int j = 0; j < KC / 16; ++j) {
                        const uint64_t bd = sdesc_sw128(bb + 32u * j);
                        mma_bf16(d, sdesc_sw128(ahi + m * MTILE_BYTES + 32u * j), bd, idesc, (t > 0 || j > 0) ? 1u : 0u);
                        if (!p.fp8) mma_bf16(d, sdesc_sw128(alo + m * MTILE_BYTES + 32u * j), bd, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
            }
            __syncwarp();
        }
        if (lane == 0) mma_commit(accf);
        __syncwarp();
    }

    // ==================================================================== epilogue
    if (warp < CONV_WARPS) {
        const int m = warp >> 2;
        const bool have = nloc > 0;
        bool ok = true;
        if (have) {
            ok = mbar_wait(accf, 0, abort, p.flags);
            tc_fence_after();
        }
        if (m < p.MT) {
            const int row = m * 128 + 32 * (warp & 3) + lane;
            for (int c0 = 0; c0 < p.N; c0 += 32) {
                float v[32];
                if (have && ok) {
                    tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(m * p.N + c0), v);
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k) v[k] = 0.f;
                }
                if (row < rows_valid) {
                    double* dst = p.partial + ((int64_t)blockIdx.x * p.I + rbeg + row) * p.K;
#pragma unroll
                    for (int k = 0; k < 32; ++k)
                        if (c0 + k < p.K) dst[c0 + k] = (double)v[k];
                }
            }
        }
        if (p.normp) {
            nsum = rtr::warp_sum(nsum);
            if (lane == 0) nred[warp] = nsum;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (p.normp && tid == 0) {
        double s = 0.0;
        for (int w = 0; w < CONV_WARPS; ++w) s += nred[w];
        p.normp[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
    if (warp == MMA_WARP) tmem_dealloc(tmem, ncols);
}

// as reduce_partials_kernel: a non-finite norm total raises RTR_FLAG_NONFINITE
__global__ void tc_reduce_kernel(const double* __restrict__ partial, int nparts, int64_t count,
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

// ---- TMA-fed variant for modes with B > 1 ------------------------------------
// Same arithmetic as sketch_tc_kernel.  A CTA covers up to 256 rows of the
// (A, I, B) view (rows a*I + i with pitch B) as MT = 1 or 2 M tiles of 128
// rows that share one Omega tile, so Omega is generated once per chunk of kc
// consecutive b for all of them.  Ring slot layout (S slots):
//   [tile 0: 32 KB][tile 1: 32 KB, if MT = 2][B: N x 64 bf16, SW128]
// Each tile region receives a TMA box (128 rows x kc float32, dense rows) and
// is then converted IN PLACE into its bf16 operand tiles: hi in the first
// 16 KB, lo in the second (SW128 K-major, 128 rows x 64).  Every converter
// reads its pieces of a tile into registers, the converters meet at a named
// barrier, and only then write, so no value is overwritten before it is read.
// Without a separate operand ring the whole of shared memory holds staging
// slots: up to 192 KB of loads in flight per SM.
//   warps 0-7   converters, then warps 0 .. 4 MT - 1 drain the accumulators
//   warps 8-11  Omega generators (one Philox4x64-10 call per thread per chunk
//               for K <= 40; one Omega tile serves both M tiles)
//   warp 12     TMA producer (one lane)
//   warp 13     MMA issuer (one lane)
// (14 warps: at most four per SM sub-partition, so 128 registers a thread)
//
// The last mode (B = 1, rows a of I contiguous values) runs the same pipeline
// without a transpose: a chunk is 64 consecutive a, each 128-row M tile of i
// arrives as two TMA boxes of 64 a x 64 i (16 KB), converted in place into
// hi (8 KB) and lo (8 KB) tiles whose 128-byte rows hold 64 consecutive i.
// Read as the MMA's A operand these tiles are MN-major (M = i contiguous):
// 8-row groups of a (the K direction) 1024 B apart, the two 64-wide halves
// of the M tile 16 KB apart.
constexpr int TM_CONV_WARPS = 8;
constexpr int TM_RNG_GROUPS = 1;
constexpr int TM_RNG_WARPS = 4 * TM_RNG_GROUPS;
constexpr int TM_TMA_WARP = TM_CONV_WARPS + TM_RNG_WARPS;
constexpr int TM_MMA_WARP = TM_TMA_WARP + 1;
constexpr int TM_NTHREADS = (TM_MMA_WARP + 1) * 32;
constexpr int TM_CONV_THREADS = TM_CONV_WARPS * 32;
constexpr int TM_RNG_THREADS = 128;               // threads of one RNG group
constexpr uint32_t TM_TILE = 32768;               // one tile region: 128 x 64 float32 = hi + lo bf16
constexpr int TM_MAX_SLOTS = 6;

struct SketchTmaArgs {
    int64_t A, B;
    int I, K, N, MT, S;
    int kc;                       // chunk width along b: a multiple of 8 dividing B (or 64);
                                  // FP8: 64 or 32 (whole 32-value scale blocks)
    int fp8;                      // 1: block-scaled float8 values, one MMA (no lo part)
    int lm;                       // 1: the last mode (B = 1, BF16): boxes of 64 a x 64 i, A operand MN-major
    int64_t nchunks, nbc;
    int64_t aoff;                 // index of the view's first a in the whole tensor (slabs)
    uint64_t seed;
    int mode;
    const uint16_t* tab;
    double* partial;
    double* normp;
    int* flags;
};

// named barrier 1 among the converter threads only
__device__ __forceinline__ void conv_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(TM_CONV_THREADS) : "memory");
}
// the same barrier with an AND vote: every converter thread gets the same
// answer, so a bounded wait that gave up in one thread ends the loop in all
// of them (none is left waiting at a later conv_bar)
__device__ __forceinline__ bool conv_bar_and(bool v) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred pv, pr;\n\tsetp.ne.u32 pv, %1, 0;\n\tbar.red.and.pred pr, 1, %2, pv;\n\t"
                 "selp.u32 %0, 1, 0, pr;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v), "n"(TM_CONV_THREADS) : "memory");
    return r != 0;
}

// VAR: 1 = BF16 values in 64-wide chunks (every BF16 plan), 2 = float8 values
// in 64-wide chunks, each with the other form's code and the narrow-chunk
// code compiled out; 0 = any (FP8 in 32-wide chunks)
template <bool LM, int VAR>
__global__ void __launch_bounds__(TM_NTHREADS, 1) sketch_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                   const SketchTmaArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const bool fp8 = VAR == 1 ? false : VAR == 2 ? true : (p.fp8 != 0);
    const int kc = VAR != 0 ? 64 : p.kc;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    const int S = p.S, MT = p.MT;
    const uint32_t b_bytes = (uint32_t)p.N * 128u;
    const uint32_t slot_bytes = (uint32_t)MT * TM_TILE + b_bytes;
    const uint32_t sl0 = smem_u32(sm);
    uint16_t* tab = reinterpret_cast<uint16_t*>(sm + (size_t)S * slot_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tab + 4096);
    uint64_t* full = bars;                 // TMA landed (transaction bytes)
    uint64_t* conv = bars + S;             // operand tiles written (8 converter warps)
    uint64_t* fullB = bars + 2 * S;        // Omega tile written (4 generator warps)
    uint64_t* empty = bars + 3 * S;        // MMAs of the slot done (tcgen05.commit)
    uint64_t* accf = bars + 4 * S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    double* nred = reinterpret_cast<double*>(accf + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = (uint32_t)(p.N * MT);

    // zero every slot once: the Omega tiles' columns kc .. 63 are never written
    for (uint32_t off = tid * 16u; off < (uint32_t)S * slot_bytes; off += TM_NTHREADS * 16u)
        asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(sl0 + off), "r"(0) : "memory");
    for (int j = tid; j < 4096; j += TM_NTHREADS) tab[j] = p.tab[j];
    if (tid == 0) {
        // one arrival per warp (lane 0 after __syncwarp): same-address
        // arrivals from every thread serialise on the barrier word
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], TM_CONV_WARPS);
            mbar_init(&fullB[s], TM_RNG_THREADS / 32);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        *abort = 0;
        mbar_fence_init();
    }
    if (warp == TM_MMA_WARP) tmem_alloc(tmem_slot, ncols < 32 ? 32 : ncols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int rbeg = blockIdx.y * 256;
    const int rows_valid = min(128 * MT, p.I - rbeg);
    // each CTA takes a contiguous range of chunks (its successive boxes are
    // adjacent in b: 2% faster at 200^4 than a grid-stride assignment)
    const int64_t per_cta = p.nchunks / gridDim.x, rem_cta = p.nchunks % gridDim.x;
    const int64_t c0 = blockIdx.x * per_cta + min((int64_t)blockIdx.x, rem_cta);
    const int64_t nloc = per_cta + ((int64_t)blockIdx.x < rem_cta ? 1 : 0);
    const int ksteps = (kc + 15) >> 4;          // operand columns kc .. 16 ksteps - 1 are written as zeros
    double nsum = 0.0;

    if (warp < TM_CONV_WARPS) {
        // ================================================================ converters
        const int ct = tid;
        const bool want_norm = p.normp != nullptr;
        Ring r(S);
        for (int64_t t = 0; t < nloc; ++t, r.step(1)) {
            const int s = r.slot;
            const uint32_t u = r.use;
            if (!conv_bar_and(mbar_wait(&full[s], u & 1, abort, p.flags))) break;
            const uint32_t slot = sl0 + s * slot_bytes;
            float csum = 0.f;
            for (int m = 0; m < MT; ++m) {
                const uint32_t src = slot + m * TM_TILE;
                const uint32_t hi = src, lo = src + TM_TILE / 2;
                const int rows_m = min(128, rows_valid - 128 * m);
                auto piece = [&](const float4 v, uint32_t off) {
                    if (fp8) {
                        // a 32-value scale block is 8 consecutive pieces of one row,
                        // held by 8 consecutive lanes (kc = 32 or 64)
                        const float mx = group_max(fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))), 8);
                        const MxScale sc = mx_scale(mx);
                        st_shared_v2(hi + off, mx_pair(v.x, v.y, sc), mx_pair(v.z, v.w, sc));
                        return;
                    }
                    uint32_t h0, l0, h1, l1;
                    split2(v.x, v.y, h0, l0);
                    split2(v.z, v.w, h1, l1);
                    st_shared_v2(hi + off, h0, h1);
                    st_shared_v2(lo + off, l0, l1);
                };
                if constexpr (LM) {
                    // two boxes of 64 a (rows) x 64 i; piece j of this thread: box
                    // j >> 2, row (ct >> 4) + 16 (j & 3), column group ct & 15
                    float4 v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int row = (ct >> 4) + 16 * (j & 3);
                        v[j] = ld_shared_f4(src + (uint32_t)(j >> 2) * 16384u + (uint32_t)row * 256u +
                                            (uint32_t)(ct & 15) * 16u);
                        if (want_norm) csum += v[j].x * v[j].x + v[j].y * v[j].y + v[j].z * v[j].z + v[j].w * v[j].w;
                    }
                    conv_bar();
                    const uint32_t off0 = sw128_off((uint32_t)(ct >> 4), 4u * (uint32_t)(ct & 15));
                    if (fp8) {
                        // float8 scale blocks run along a: rows 0-31 and 32-63 of each
                        // column.  This thread's rows of block b are pieces 2b, 2b + 1;
                        // the partner lane (lane ^ 16) holds the next row; the other
                        // rows sit in the other 7 converter warps, met through the
                        // box's lo half (unused by the FP8 form) after the barrier above
                        float4 mx[2][2];
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int b = 0; b < 2; ++b) {
                                const float4 a0 = v[4 * h + 2 * b], a1 = v[4 * h + 2 * b + 1];
                                float4 m = make_float4(fmaxf(fabsf(a0.x), fabsf(a1.x)), fmaxf(fabsf(a0.y), fabsf(a1.y)),
                                                       fmaxf(fabsf(a0.z), fabsf(a1.z)), fmaxf(fabsf(a0.w), fabsf(a1.w)));
                                m.x = fmaxf(m.x, __shfl_xor_sync(0xffffffffu, m.x, 16));
                                m.y = fmaxf(m.y, __shfl_xor_sync(0xffffffffu, m.y, 16));
                                m.z = fmaxf(m.z, __shfl_xor_sync(0xffffffffu, m.z, 16));
                                m.w = fmaxf(m.w, __shfl_xor_sync(0xffffffffu, m.w, 16));
                                mx[h][b] = m;
                            }
                        // exchange slots: box h's lo half, [block][warp][64 columns] floats
                        if (lane < 16)
#pragma unroll
                            for (int h = 0; h < 2; ++h)
#pragma unroll
                                for (int b = 0; b < 2; ++b)
                                    st_shared_v4f(src + (uint32_t)h * 16384u + 8192u +
                                                      (uint32_t)((b * TM_CONV_WARPS + warp) * 64 + 4 * (ct & 15)) * 4u,
                                                  mx[h][b]);
                        conv_bar();
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int b = 0; b < 2; ++b) {
                                float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
                                for (int w = 0; w < TM_CONV_WARPS; ++w) {
                                    const float4 o = ld_shared_f4(src + (uint32_t)h * 16384u + 8192u +
                                                                  (uint32_t)((b * TM_CONV_WARPS + w) * 64 + 4 * (ct & 15)) * 4u);
                                    m = make_float4(fmaxf(m.x, o.x), fmaxf(m.y, o.y), fmaxf(m.z, o.z), fmaxf(m.w, o.w));
                                }
                                const MxScale s0 = mx_scale(m.x), s1 = mx_scale(m.y), s2 = mx_scale(m.z), s3 = mx_scale(m.w);
#pragma unroll
                                for (int jj = 0; jj < 2; ++jj) {
                                    const int j = 4 * h + 2 * b + jj;
                                    st_shared_v2(src + (uint32_t)h * 16384u + off0 + 2048u * (uint32_t)(j & 3),
                                                 mx_pair2(v[j].x, v[j].y, s0, s1), mx_pair2(v[j].z, v[j].w, s2, s3));
                                }
                            }
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const uint32_t bx = src + (uint32_t)(j >> 2) * 16384u;
                            uint32_t h0, l0, h1, l1;
                            split2(v[j].x, v[j].y, h0, l0);
                            split2(v[j].z, v[j].w, h1, l1);
                            const uint32_t off = off0 + 2048u * (uint32_t)(j & 3);
                            st_shared_v2(bx + off, h0, h1);
                            st_shared_v2(bx + 8192u + off, l0, l1);
                        }
                    }
                } else if (kc == 64) {
                    // piece j of this thread: row (ct >> 4) + 16 j, column group ct & 15
                    float4 v[8];
#pragma unroll
                    // rows past I were zero-filled by the TMA unit: every row is loaded
                    for (int j = 0; j < 8; ++j) {
                        const int row = (ct >> 4) + 16 * j;
                        v[j] = ld_shared_f4(src + (uint32_t)row * 256u + (uint32_t)(ct & 15) * 16u);
                        if (want_norm) csum += v[j].x * v[j].x + v[j].y * v[j].y + v[j].z * v[j].z + v[j].w * v[j].w;
                    }
                    conv_bar();                        // every piece of this tile is in registers
                    // the swizzle phase (row & 7) is the same for every j
                    const uint32_t off0 = sw128_off((uint32_t)(ct >> 4), 4u * (uint32_t)(ct & 15));
                    if (fp8) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) piece(v[j], off0 + 2048u * j);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            uint32_t h0, l0, h1, l1;
                            split2(v[j].x, v[j].y, h0, l0);
                            split2(v[j].z, v[j].w, h1, l1);
                            st_shared_v2(hi + off0 + 2048u * j, h0, h1);
                            st_shared_v2(lo + off0 + 2048u * j, l0, l1);
                        }
                    }
                } else {
                    // kc = 4 Q4 with Q4 a compile-time constant: row/column of a piece
                    // by multiply-shift; zero columns kc .. 16 ksteps - 1 afterwards
                    auto run = [&](auto q4c) {
                        constexpr int Q4 = decltype(q4c)::value;
                        constexpr int NP = (128 * Q4 + TM_CONV_THREADS - 1) / TM_CONV_THREADS;
                        float4 v[NP];
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            const int pc = ct + TM_CONV_THREADS * j;
                            const int row = pc / Q4;
                            v[j] = (pc < 128 * Q4 && row < rows_m)
                                       ? ld_shared_f4(src + (uint32_t)row * (uint32_t)(16 * Q4) + (uint32_t)(pc % Q4) * 16u)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                            if (want_norm) csum += v[j].x * v[j].x + v[j].y * v[j].y + v[j].z * v[j].z + v[j].w * v[j].w;
                        }
                        conv_bar();
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            const int pc = ct + TM_CONV_THREADS * j;
                            if (pc < 128 * Q4) piece(v[j], sw128_off(pc / Q4, 4 * (pc % Q4)));
                        }
                        constexpr int ZP = (4 * ((4 * Q4 + 15) / 16) - Q4);   // zero pieces per row
                        if constexpr (ZP > 0) {
                            for (int pc = ct; pc < 128 * ZP; pc += TM_CONV_THREADS) {
                                const uint32_t off = sw128_off(pc / ZP, 4 * (Q4 + pc % ZP));
                                st_shared_v2(hi + off, 0u, 0u);
                                if (!fp8) st_shared_v2(lo + off, 0u, 0u);
                            }
                        }
                    };
                    switch (kc >> 2) {
                        case 2: run(std::integral_constant<int, 2>{}); break;
                        case 4: run(std::integral_constant<int, 4>{}); break;
                        case 6: run(std::integral_constant<int, 6>{}); break;
                        case 8: run(std::integral_constant<int, 8>{}); break;
                        case 10: run(std::integral_constant<int, 10>{}); break;
                        case 12: run(std::integral_constant<int, 12>{}); break;
                        default: run(std::integral_constant<int, 14>{}); break;
                    }
                }
            }
            nsum += (double)csum;
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[s]);
        }
    } else if (warp < TM_TMA_WARP) {
        // ================================================================ Omega generators
        const int rt = (tid - TM_CONV_THREADS) % TM_RNG_THREADS;
        const int grp = (tid - TM_CONV_THREADS) / TM_RNG_THREADS;
        const int ncall = (p.K + 19) / 20;
        const int nitems = kc * ncall;              // <= 64 * 4 = 2 * TM_RNG_THREADS
        const int it0 = rt, it1 = rt + TM_RNG_THREADS;
        const int rr0 = it0 % kc, cb0 = it0 / kc, rr1 = it1 % kc, cb1 = it1 / kc;
        Ring r(S, grp);
        ChunkPos cp(c0 + grp, (int64_t)TM_RNG_GROUPS, p.nbc);
        for (int64_t t = grp; t < nloc; t += TM_RNG_GROUPS, r.step(TM_RNG_GROUPS), cp.step()) {
            const int s = r.slot;
            const uint32_t u = r.use;
            const int64_t a = cp.a, b0 = cp.bi * kc;
            // last mode: chunk a covers rows 64 a .. 64 a + 63 of the (A, I) view
            const int64_t r0 = LM ? 64 * a + p.aoff : (a + p.aoff) * p.B + b0;
            const int len = LM ? (int)min((int64_t)64, p.A - 64 * a) : (int)min((int64_t)kc, p.B - b0);
            if (t >= S && !mbar_wait(&empty[s], (u - 1) & 1, abort, p.flags)) break;
            const uint32_t bt = sl0 + s * slot_bytes + (uint32_t)MT * TM_TILE;
            for (int item = it0; item < nitems; item += TM_RNG_THREADS) {
                const int rr = item == it0 ? rr0 : rr1, cb = item == it0 ? cb0 : cb1;
                uint64_t w[4] = {0, 0, 0, 0};
                if (rr < len) rtr::omega_words(p.seed, p.mode, (uint64_t)(r0 + rr), (uint64_t)cb, w);
#pragma unroll
                for (int tt = 0; tt < 20; ++tt) {
                    const int k = cb * 20 + tt;
                    if (k < p.K) st_shared_u16(bt + sw128_off(k, rr), (rr < len) ? tab[rtr::omega_field(w, tt)] : (uint16_t)0);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&fullB[s]);
        }
    } else if (warp == TM_TMA_WARP) {
        // ================================================================ TMA producer
        if (lane == 0) {
            Ring r(S);
            ChunkPos cp(c0, 1, p.nbc);
            const uint32_t box_bytes = (uint32_t)(128 * 4 * kc);
            for (int64_t t = 0; t < nloc; ++t, r.step(1), cp.step()) {
                const int s = r.slot;
                const uint32_t u = r.use;
                if (t >= S && !mbar_wait(&empty[s], (u - 1) & 1, abort, p.flags)) break;
                const int64_t a = cp.a, b0 = cp.bi * kc;
                // the full boxes are always counted: out-of-range rows (i >= I) and
                // columns are zero-filled by the TMA unit without memory traffic
                mbar_arrive_expect_tx(&full[s], box_bytes * (uint32_t)MT);
                if constexpr (LM) {
                    // boxes {64 i, 64 a}: x = i, y = a
                    for (int m = 0; m < MT; ++m)
                        for (int h = 0; h < 2; ++h)
                            tma_load_2d(sl0 + s * slot_bytes + m * TM_TILE + h * 16384, &tmap, rbeg + 128 * m + 64 * h,
                                        (int)(64 * a), &full[s]);
                } else {
                    for (int m = 0; m < MT; ++m)
                        tma_load_3d(sl0 + s * slot_bytes + m * TM_TILE, &tmap, (int)b0, rbeg + 128 * m, (int)a,
                                    &full[s]);
                }
            }
        }
        __syncwarp();
    } else {
        // ================================================================ MMA issuer
        const uint32_t idesc = idesc_bf16_f32(128, p.N) | (LM ? IDESC_A_MN_MAJOR : 0u);
        Ring r(S);
        for (int64_t t = 0; t < nloc; ++t, r.step(1)) {
            const int s = r.slot;
            const uint32_t u = r.use;
            if (!mbar_wait(&conv[s], u & 1, abort, p.flags)) break;
            if (!mbar_wait(&fullB[s], u & 1, abort, p.flags)) break;
            tc_fence_after();
            if (lane == 0) {
                const uint32_t slot = sl0 + s * slot_bytes;
                const uint32_t bb = slot + (uint32_t)MT * TM_TILE;
                for (int m = 0; m < MT; ++m) {
                    const uint32_t d = tmem + (uint32_t)(m * p.N);
                    if constexpr (LM) {
                        // MN-major A: K step j = a rows 16 j .. 16 j + 15 (two 8-row groups)
                        const uint32_t ahi = slot + m * TM_TILE, alo = ahi + 8192u;
                        for (int j = 0; j < ksteps; ++j) {
                            const uint64_t bd = sdesc_sw128(bb + 32u * j);
                            mma_bf16(d, sdesc_sw128_mn(ahi + 2048u * j, 16384u), bd, idesc, (t > 0 || j > 0) ? 1u : 0u);
                            if (!fp8) mma_bf16(d, sdesc_sw128_mn(alo + 2048u * j, 16384u), bd, idesc, 1u);
                        }
                        continue;
                    }
                    const uint32_t ahi = slot + m * TM_TILE, alo = ahi + TM_TILE / 2;
                    for (int j = 0; j < ksteps; ++j) {
                        const uint64_t bd = sdesc_sw128(bb + 32u * j);
                        mma_bf16(d, sdesc_sw128(ahi + 32u * j), bd, idesc, (t > 0 || j > 0) ? 1u : 0u);
                        if (!fp8) mma_bf16(d, sdesc_sw128(alo + 32u * j), bd, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
            }
            __syncwarp();
        }
        if (lane == 0) mma_commit(accf);
        __syncwarp();
    }

    // ==================================================================== epilogue
    if (warp < 4 * MT) {
        const bool have = nloc > 0;
        bool ok = true;
        if (have) {
            ok = mbar_wait(accf, 0, abort, p.flags);
            tc_fence_after();
        }
        const int m = warp >> 2, q = warp & 3;
        const int row = 128 * m + 32 * q + lane;
        for (int c0 = 0; c0 < p.N; c0 += 32) {
            float v[32];
            if (have && ok) {
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(m * p.N + c0), v);
            } else {
#pragma unroll
                for (int k = 0; k < 32; ++k) v[k] = 0.f;
            }
            if (row < rows_valid) {
                double* dst = p.partial + ((int64_t)blockIdx.x * p.I + rbeg + row) * p.K;
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (c0 + k < p.K) dst[c0 + k] = (double)v[k];
            }
        }
    }
    if (warp < TM_CONV_WARPS && p.normp) {
        nsum = rtr::warp_sum(nsum);
        if (lane == 0) nred[warp] = nsum;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (p.normp && tid == 0) {
        double s = 0.0;
        for (int w = 0; w < TM_CONV_WARPS; ++w) s += nred[w];
        p.normp[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
    if (warp == TM_MMA_WARP) tmem_dealloc(tmem, ncols < 32 ? 32 : ncols);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

constexpr size_t SMEM_LIMIT = 232448;   // 227 KiB opt-in per CTA

int sketch_geometry(int64_t I, int K, int* MT, int* N, int* S, size_t* smem) {
    *N = (K <= 32) ? 32 : 64;
    *MT = (I > 128) ? 2 : 1;
    const size_t stage = 2 * (size_t)(*MT) * MTILE_BYTES + (size_t)(*N) * 128;
    const size_t fixed = 8192 + 64 * 8 + 1024;
    int s = (int)((SMEM_LIMIT - fixed) / stage);
    s = std::min(s, 4);
    if (s < 2) return 0;
    *S = s;
    *smem = fixed + (size_t)s * stage;
    return 1;
}

// ---- the last two modes in one read of X (BF16) ------------------------------
// Algorithm 1 step 5 for modes N-2 and N-1 together, X viewed as (A, I, J)
// with I = I_{N-2}, J = I_{N-1} and a the flat index of the leading modes:
//     Y_{N-2}[i, k] = sum_{a, j} X[a, i, j] Omega_{N-2}[a J + j, k]
//     Y_{N-1}[j, k] = sum_{a, i} X[a, i, j] Omega_{N-1}[a I + i, k]
// Both sums run over the same elements, so one tile of X in shared memory
// feeds both products and X is read once for the two modes.  A chunk is
// (a, jt, it): 128 rows of i (tile it) x 128 consecutive j (tile jt, the last
// one ragged), and a CTA walks a contiguous range of chunks in that order (it
// fastest).  A chunk arrives by TMA as two boxes of 128 i x 64 j float32 (32 KB
// each) and is converted in place into bf16 hi/lo tiles exactly as in
// sketch_tma_kernel (rows i, 64 j in each 128-byte SW128 row).  Read with a
// K-major descriptor the tiles are the A operand of mode N-2 (M = i, K = j, two
// K atoms); read with an MN-major descriptor the same bytes are the A operand
// of mode N-1 (M = j in two 64-wide halves 32 KB apart, K = i in eight steps
// of 16 rows).  The Omega tiles are drawn once per use group: the mode N-2
// tile of (a, jt) serves the consecutive chunks it = 0 .. nit - 1, and the
// mode N-1 tiles of a (all of i) serve every chunk of that a; each kind has a
// ring of two groups, released by the MMA of the group's last chunk.  So per
// element of X as many Omega rows are drawn as by the two one-mode passes.
// The quantile table is read through the L1 cache.  TMEM holds one mode N-2
// accumulator per i tile and one mode N-1 accumulator per j tile.
//   warps 0-7    converters; then warps 0-3 drain mode N-2, warps 4-7 mode N-1
//   warps 8-13   Omega generators (both modes)
//   warp 14      TMA producer (one lane)
//   warp 15      MMA issuer (one lane)
constexpr int PR_CONV_WARPS = TM_CONV_WARPS;
constexpr int PR_RNG_WARPS = 6;
constexpr int PR_TMA_WARP = PR_CONV_WARPS + PR_RNG_WARPS;
constexpr int PR_MMA_WARP = PR_TMA_WARP + 1;
constexpr int PR_NTHREADS = (PR_MMA_WARP + 1) * 32;
constexpr int PR_RNG_THREADS = PR_RNG_WARPS * 32;
constexpr uint32_t PR_XSLOT = 2 * TM_TILE;       // two boxes of 128 i x 64 j float32
constexpr int PR_MAX_XS = 3;                     // X slots

struct SketchPairArgs {
    int64_t A;
    int I, J, K2, K3, N2, N3, S, nit, njt;
    int64_t nchunks;              // A * njt * nit
    uint64_t seed;
    int mode2, mode3;             // N - 2, N - 1
    const uint16_t* tab;          // bfloat16 quantile table (global)
    double* part2;                // [gridDim.x][I][K2]
    double* part3;                // [gridDim.x][J][K3]
    double* normp;                // [gridDim.x] or null
    int* flags;
};

// 64-wide K atoms of a chunk that hold any j < J (1 or 2)
__device__ __forceinline__ int pair_atoms(int J, int jt) { return min(2, (J - 128 * jt + 63) >> 6); }

// (a, jt, it) of chunk c = (a njt + jt) nit + it, stepped without divisions
struct PairPos {
    int64_t a;
    int jt, it;
    __device__ PairPos(int64_t c, int nit, int njt) {
        it = (int)(c % nit);
        const int64_t q = c / nit;
        jt = (int)(q % njt);
        a = q / njt;
    }
    __device__ void step(int nit, int njt) {
        if (++it == nit) {
            it = 0;
            if (++jt == njt) { jt = 0; ++a; }
        }
    }
};

__global__ void __launch_bounds__(PR_NTHREADS, 1) sketch_pair_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                     const SketchPairArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    const int S = p.S, nit = p.nit, njt = p.njt;
    const uint32_t b2_tile = 2u * (uint32_t)p.N2 * 128u;            // 128 rows of reduction, two K atoms
    const uint32_t b3_tile = 2u * (uint32_t)p.N3 * 128u;
    const uint32_t b3_group = (uint32_t)nit * b3_tile;
    const uint32_t xs0 = smem_u32(sm);
    const uint32_t b2s0 = xs0 + (uint32_t)S * PR_XSLOT;             // ring of 2 mode N-2 tiles
    const uint32_t b3s0 = b2s0 + 2u * b2_tile;                      // ring of 2 groups of nit mode N-1 tiles
    const uint32_t total = (uint32_t)S * PR_XSLOT + 2u * b2_tile + 2u * b3_group;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + total);
    uint64_t* full = bars;                 // X boxes landed (transaction bytes)
    uint64_t* conv = bars + S;             // hi/lo tiles written (8 converter warps)
    uint64_t* empty = bars + 2 * S;        // MMAs reading the X slot done
    uint64_t* full2 = bars + 3 * S;        // mode N-2 Omega tile written (6 generator warps)
    uint64_t* empty2 = full2 + 2;          // MMAs of the tile's last chunk done
    uint64_t* full3 = full2 + 4;           // mode N-1 Omega group written
    uint64_t* empty3 = full2 + 6;
    uint64_t* accf = full2 + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    double* nred = reinterpret_cast<double*>(accf + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(nit * p.N2 + njt * p.N3)) ncols <<= 1;

    // zero every slot once: Omega columns k >= K are never written
    for (uint32_t off = tid * 16u; off < total; off += PR_NTHREADS * 16u)
        asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(xs0 + off), "r"(0) : "memory");
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], PR_CONV_WARPS);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full2[s], PR_RNG_WARPS);
            mbar_init(&empty2[s], 1);
            mbar_init(&full3[s], PR_RNG_WARPS);
            mbar_init(&empty3[s], 1);
        }
        mbar_init(accf, 1);
        *abort = 0;
        mbar_fence_init();
    }
    if (warp == PR_MMA_WARP) tmem_alloc(tmem_slot, ncols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t per_cta = p.nchunks / gridDim.x, rem_cta = p.nchunks % gridDim.x;
    const int64_t c0 = blockIdx.x * per_cta + min((int64_t)blockIdx.x, rem_cta);
    const int64_t nloc = per_cta + ((int64_t)blockIdx.x < rem_cta ? 1 : 0);
    double nsum = 0.0;

    if (warp < PR_CONV_WARPS) {
        // ================================================================ converters
        const int ct = tid;
        const bool want_norm = p.normp != nullptr;
        Ring r(S);
        PairPos pos(c0, nit, njt);
        for (int64_t t = 0; t < nloc; ++t, r.step(1), pos.step(nit, njt)) {
            const int s = r.slot;
            if (!conv_bar_and(mbar_wait(&full[s], r.use & 1, abort, p.flags))) break;
            const int nat = pair_atoms(p.J, pos.jt);
            float csum = 0.f;
            for (int h = 0; h < nat; ++h) {
                // box h: 128 rows of i x 64 j; piece j of this thread: row
                // (ct >> 4) + 16 j, column group ct & 15; rows past I and
                // columns past J were zero-filled by the TMA unit
                const uint32_t src = xs0 + s * PR_XSLOT + h * TM_TILE;
                float4 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int row = (ct >> 4) + 16 * j;
                    v[j] = ld_shared_f4(src + (uint32_t)row * 256u + (uint32_t)(ct & 15) * 16u);
                    if (want_norm) csum += v[j].x * v[j].x + v[j].y * v[j].y + v[j].z * v[j].z + v[j].w * v[j].w;
                }
                conv_bar();                        // every piece of this box is in registers
                const uint32_t off0 = sw128_off((uint32_t)(ct >> 4), 4u * (uint32_t)(ct & 15));
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint32_t h0, l0, h1, l1;
                    split2(v[j].x, v[j].y, h0, l0);
                    split2(v[j].z, v[j].w, h1, l1);
                    st_shared_v2(src + off0 + 2048u * j, h0, h1);
                    st_shared_v2(src + TM_TILE / 2 + off0 + 2048u * j, l0, l1);
                }
            }
            nsum += (double)csum;
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[s]);
        }
    } else if (warp < PR_TMA_WARP) {
        // ================================================================ Omega generators
        // A tile holds `nrows` reduction rows (128 per tile, tiles consecutive)
        // of Omega_mode from row `row0` on; rows at or past `lim` are zero.
        // Items: (rows 2 rp, 2 rp + 1, Philox call cb).  A thread draws both
        // rows, looks up all 40 table entries before its first store (the
        // stores are ordered asm, so a lookup placed between them would wait
        // out its full latency each time) and writes the pairs as 32-bit
        // words (adjacent rows are adjacent bf16).
        const int gt = tid - PR_CONV_WARPS * 32;
        auto draw = [&](uint32_t base, int nrows, int Nc, int K, int mode, uint64_t row0, int lim) {
            const int npair = nrows >> 1, items = npair * ((K + 19) / 20);
            for (int item = gt; item < items; item += PR_RNG_THREADS) {
                const int rp = item % npair, cb = item / npair;
                const int rr = 2 * rp;
                const uint32_t bt = base + (uint32_t)(rr >> 6) * (uint32_t)Nc * 128u;   // tiles, then atoms, consecutive
                uint64_t w0[4] = {0, 0, 0, 0}, w1[4] = {0, 0, 0, 0};
                if (rr < lim) rtr::omega_words(p.seed, mode, row0 + rr, (uint64_t)cb, w0);
                if (rr + 1 < lim) rtr::omega_words(p.seed, mode, row0 + rr + 1, (uint64_t)cb, w1);
                uint32_t v[20];
#pragma unroll
                for (int tt = 0; tt < 20; ++tt) {
                    const uint32_t e0 = rr < lim ? (uint32_t)__ldg(p.tab + rtr::omega_field(w0, tt)) : 0u;
                    const uint32_t e1 = rr + 1 < lim ? (uint32_t)__ldg(p.tab + rtr::omega_field(w1, tt)) : 0u;
                    v[tt] = e0 | (e1 << 16);
                }
#pragma unroll
                for (int tt = 0; tt < 20; ++tt) {
                    const int k = cb * 20 + tt;
                    if (k < K) st_shared_u32(bt + sw128_off(k, rr & 63), v[tt]);
                }
            }
            fence_proxy_async();
            __syncwarp();
        };
        PairPos pos(c0, nit, njt);
        int64_t g2 = -1, g3 = -1;
        for (int64_t t = 0; t < nloc; ++t, pos.step(nit, njt)) {
            if (t == 0 || (pos.jt == 0 && pos.it == 0)) {
                // a new a: the mode N-1 tiles of all of i
                ++g3;
                const int s3 = (int)(g3 & 1);
                if (g3 >= 2 && !mbar_wait(&empty3[s3], (uint32_t)((g3 >> 1) - 1) & 1, abort, p.flags)) break;
                draw(b3s0 + s3 * b3_group, 128 * nit, p.N3, p.K3, p.mode3, (uint64_t)(pos.a * p.I), p.I);
                if (lane == 0) mbar_arrive(&full3[s3]);
            }
            if (t == 0 || pos.it == 0) {
                // a new (a, jt): the mode N-2 tile of 128 j
                ++g2;
                const int s2 = (int)(g2 & 1);
                if (g2 >= 2 && !mbar_wait(&empty2[s2], (uint32_t)((g2 >> 1) - 1) & 1, abort, p.flags)) break;
                draw(b2s0 + s2 * b2_tile, 128, p.N2, p.K2, p.mode2, (uint64_t)(pos.a * p.J + 128 * pos.jt),
                     p.J - 128 * pos.jt);
                if (lane == 0) mbar_arrive(&full2[s2]);
            }
        }
    } else if (warp == PR_TMA_WARP) {
        // ================================================================ TMA producer
        if (lane == 0) {
            Ring r(S);
            PairPos pos(c0, nit, njt);
            for (int64_t t = 0; t < nloc; ++t, r.step(1), pos.step(nit, njt)) {
                const int s = r.slot;
                if (t >= S && !mbar_wait(&empty[s], (r.use - 1) & 1, abort, p.flags)) break;
                const int nat = pair_atoms(p.J, pos.jt);
                // a box past J is not loaded (its tiles are neither converted
                // nor read by the mode N-2 product)
                mbar_arrive_expect_tx(&full[s], (uint32_t)nat * TM_TILE);
                for (int h = 0; h < nat; ++h)
                    tma_load_3d(xs0 + s * PR_XSLOT + h * TM_TILE, &tmap, 128 * pos.jt + 64 * h, 128 * pos.it,
                                (int)pos.a, &full[s]);
            }
        }
        __syncwarp();
    } else {
        // ================================================================ MMA issuer
        const uint32_t id2 = idesc_bf16_f32(128, p.N2);
        const uint32_t id3 = idesc_bf16_f32(128, p.N3) | IDESC_A_MN_MAJOR;
        Ring r(S);
        PairPos pos(c0, nit, njt);
        int64_t g2 = -1, g3 = -1;
        uint64_t init = 0;           // bit it: mode N-2 tile it written; bit 32 + jt: mode N-1 tile jt
        for (int64_t t = 0; t < nloc; ++t, r.step(1), pos.step(nit, njt)) {
            const int s = r.slot;
            const bool new3 = t == 0 || (pos.jt == 0 && pos.it == 0), new2 = t == 0 || pos.it == 0;
            const bool last = t == nloc - 1;
            const bool last2 = last || pos.it == nit - 1, last3 = last || (pos.jt == njt - 1 && pos.it == nit - 1);
            if (new3) ++g3;
            if (new2) ++g2;
            const int s2 = (int)(g2 & 1), s3 = (int)(g3 & 1);
            if (!mbar_wait(&conv[s], r.use & 1, abort, p.flags)) break;
            if (new3 && !mbar_wait(&full3[s3], (uint32_t)(g3 >> 1) & 1, abort, p.flags)) break;
            if (new2 && !mbar_wait(&full2[s2], (uint32_t)(g2 >> 1) & 1, abort, p.flags)) break;
            tc_fence_after();
            if (lane == 0) {
                const uint32_t xa = xs0 + s * PR_XSLOT;
                const uint32_t b2 = b2s0 + s2 * b2_tile;
                const uint32_t b3 = b3s0 + s3 * b3_group + (uint32_t)pos.it * b3_tile;
                const int nat = pair_atoms(p.J, pos.jt);
                // mode N-2: D2[it][i, k] += A[i, j] B2[j, k], K atom h = j 64 h .. 64 h + 63
                const uint32_t d2 = tmem + (uint32_t)(pos.it * p.N2);
                const uint64_t bit2 = 1ull << pos.it;
                for (int h = 0; h < nat; ++h) {
                    const uint32_t ahi = xa + (uint32_t)h * TM_TILE, alo = ahi + TM_TILE / 2;
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t bd = sdesc_sw128(b2 + (uint32_t)h * (uint32_t)p.N2 * 128u + 32u * ks);
                        mma_bf16(d2, sdesc_sw128(ahi + 32u * ks), bd, id2, (init & bit2) ? 1u : 0u);
                        init |= bit2;
                        mma_bf16(d2, sdesc_sw128(alo + 32u * ks), bd, id2, 1u);
                    }
                }
                // mode N-1: D3[jt][j, k] += A[j, i] B3[i, k] on the same tiles read
                // MN-major: 8-row groups of i 1024 B apart, the two 64-wide halves
                // of j one box (32 KB) apart; K step kk = rows 16 kk .. 16 kk + 15
                const uint32_t d3 = tmem + (uint32_t)(nit * p.N2 + pos.jt * p.N3);
                const uint64_t bit3 = 1ull << (32 + pos.jt);
                for (int kk = 0; kk < 8; ++kk) {
                    const uint64_t bd = sdesc_sw128(b3 + (uint32_t)(kk >> 2) * (uint32_t)p.N3 * 128u + 32u * (kk & 3));
                    mma_bf16(d3, sdesc_sw128_mn(xa + 2048u * kk, TM_TILE), bd, id3, (init & bit3) ? 1u : 0u);
                    init |= bit3;
                    mma_bf16(d3, sdesc_sw128_mn(xa + TM_TILE / 2 + 2048u * kk, TM_TILE), bd, id3, 1u);
                }
                mma_commit(&empty[s]);
                if (last2) mma_commit(&empty2[s2]);
                if (last3) mma_commit(&empty3[s3]);
            }
            __syncwarp();
        }
        if (lane == 0) mma_commit(accf);
        __syncwarp();
    }

    // ==================================================================== epilogue
    if (warp < PR_CONV_WARPS) {
        const bool have = nloc > 0;
        bool ok = true;
        if (have) {
            ok = mbar_wait(accf, 0, abort, p.flags);
            tc_fence_after();
        }
        const int q = warp & 3;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        if (warp < 4) {
            // tile it was written iff the CTA's chunks c0 .. c0 + nloc - 1 include one with it
            const int it0 = (int)(c0 % nit);
            for (int it = 0; it < nit; ++it) {
                const bool touched = have && ok && (nloc >= nit || (it - it0 + nit) % nit < nloc);
                const int row = 128 * it + 32 * q + lane;
                for (int cc = 0; cc < p.N2; cc += 32) {
                    float v[32];
                    if (touched) {
                        tmem_ld32(tmem + lanes + (uint32_t)(it * p.N2 + cc), v);
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k) v[k] = 0.f;
                    }
                    if (row < p.I) {
                        double* dst = p.part2 + ((int64_t)blockIdx.x * p.I + row) * p.K2;
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            if (cc + k < p.K2) dst[cc + k] = (double)v[k];
                    }
                }
            }
        } else {
            // the chunks' (a, jt) groups q0 .. q1 are consecutive; tile jt was
            // written iff one of them has jt
            const int64_t q0 = c0 / nit, q1 = have ? (c0 + nloc - 1) / nit : q0 - 1;
            const int jt0 = (int)(q0 % njt);
            for (int jt = 0; jt < njt; ++jt) {
                const bool touched = have && ok && (q1 - q0 + 1 >= njt || (jt - jt0 + njt) % njt <= q1 - q0);
                const int j = 128 * jt + 32 * q + lane;
                for (int cc = 0; cc < p.N3; cc += 32) {
                    float v[32];
                    if (touched) {
                        tmem_ld32(tmem + lanes + (uint32_t)(nit * p.N2 + jt * p.N3 + cc), v);
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k) v[k] = 0.f;
                    }
                    if (j < p.J) {
                        double* dst = p.part3 + ((int64_t)blockIdx.x * p.J + j) * p.K3;
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            if (cc + k < p.K3) dst[cc + k] = (double)v[k];
                    }
                }
            }
        }
    }
    if (warp < PR_CONV_WARPS && p.normp) {
        nsum = rtr::warp_sum(nsum);
        if (lane == 0) nred[warp] = nsum;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (p.normp && tid == 0) {
        double s = 0.0;
        for (int w = 0; w < PR_CONV_WARPS; ++w) s += nred[w];
        p.normp[blockIdx.x] = s;
    }
    if (warp == PR_MMA_WARP) tmem_dealloc(tmem, ncols);
}

// Launch geometry of sketch_pair_kernel for plan p, or 0 when the plan does
// not take the two-mode pass (not BF16 or no RTR_PARAM_PAIR, one of the two modes
// not projected, J % 4 != 0, the accumulators, Omega rings or partial sums
// do not fit).
struct PairGeom {
    int64_t A, I, J;
    int N2, N3, S, nit, njt, gx;
    size_t smem;
};

int pair_geometry(const rtr_plan* p, PairGeom* g) {
    const int N = p->N;
    if (N < 3 || p->params.prec != RTR_BF16 || !(p->params.flags & RTR_PARAM_PAIR)) return 0;
    if (!p->proj[N - 2] || !p->proj[N - 1]) return 0;
    g->I = p->dims[N - 2];
    g->J = p->dims[N - 1];
    g->A = p->numel / (g->I * g->J);
    if (g->J % 4 != 0 || g->A >= ((int64_t)1 << 31) || g->I >= ((int64_t)1 << 30)) return 0;
    g->N2 = p->K[N - 2] <= 32 ? 32 : 64;
    g->N3 = p->K[N - 1] <= 32 ? 32 : 64;
    g->nit = (int)rtr_ceil_div(g->I, 128);
    g->njt = (int)rtr_ceil_div(g->J, 128);
    if (g->nit > 32 || g->njt > 32 || g->nit * g->N2 + g->njt * g->N3 > 512) return 0;
    const size_t omega = 2 * 256 * (size_t)g->N2 + 2 * (size_t)g->nit * 256 * g->N3;   // both rings
    const size_t fixed = (3 * PR_MAX_XS + 9 + 1) * 8 + 64 + 1024;                    // barriers, scalars, alignment
    if (SMEM_LIMIT < fixed + omega + 2 * (size_t)PR_XSLOT) return 0;
    g->S = (int)std::min<size_t>(PR_MAX_XS, (SMEM_LIMIT - fixed - omega) / PR_XSLOT);
    g->smem = fixed + (size_t)g->S * PR_XSLOT + omega;
    const int64_t nchunks = g->A * g->njt * g->nit;
    g->gx = (int)std::min<int64_t>(p->num_sms, nchunks);
    const size_t need = (size_t)g->gx * (g->I * p->K[N - 2] + g->J * p->K[N - 1]);
    if (need > p->partial_elems || (size_t)g->gx > p->normx_part_elems) return 0;
    return 1;
}

}  // namespace

size_t pair_partial_elems(int num_sms, int64_t I, int K2, int64_t J, int K3) {
    return (size_t)num_sms * ((size_t)I * K2 + (size_t)J * K3);
}

int sketch_passes(const rtr_plan* p) {
    PairGeom g;
    int n = 0;
    for (int m = 0; m < p->N; ++m) n += p->proj[m] ? 1 : 0;
    return pair_geometry(p, &g) ? n - 1 : n;
}

// Modes N-2 and N-1 of the BF16 sketch in one pass over X; *done = 0 (and
// nothing launched) when the plan does not take that pass.
int launch_sketch_pair(rtr_plan* p, const float* X, double* Y2, double* Y3, double* norm_out, cudaStream_t s,
                       int* done) {
    *done = 0;
    PairGeom g;
    if ((reinterpret_cast<uintptr_t>(X) & 15) != 0 || !tensor_map_encoder() || !pair_geometry(p, &g)) return RTR_OK;
    const int N = p->N;
    SketchPairArgs a{};
    a.A = g.A; a.I = (int)g.I; a.J = (int)g.J;
    a.K2 = p->K[N - 2]; a.K3 = p->K[N - 1]; a.N2 = g.N2; a.N3 = g.N3; a.S = g.S; a.nit = g.nit; a.njt = g.njt;
    a.nchunks = g.A * g.njt * g.nit;
    a.seed = p->params.seed; a.mode2 = N - 2; a.mode3 = N - 1;
    a.tab = p->tab_bf16; a.flags = p->flags;
    a.part2 = p->partial;
    a.part3 = p->partial + (size_t)g.gx * g.I * a.K2;
    a.normp = norm_out ? p->normx_part : nullptr;
    CUtensorMap tmap;
    const cuuint64_t gdim[3] = {(cuuint64_t)g.J, (cuuint64_t)g.I, (cuuint64_t)g.A};
    const cuuint64_t gstride[2] = {(cuuint64_t)g.J * 4, (cuuint64_t)g.I * g.J * 4};
    const cuuint32_t box[3] = {64, 128, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult cr = tensor_map_encoder()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(X), gdim,
                                             gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return rtr_set_error(RTR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    RTR_SMEM(sketch_pair_kernel, g.smem);
    sketch_pair_kernel<<<(unsigned)g.gx, PR_NTHREADS, g.smem, s>>>(tmap, a);
    RTR_LAUNCH_CHECK("sketch_pair_kernel");
    const int64_t c2 = g.I * a.K2, c3 = g.J * a.K3;
    tc_reduce_kernel<<<(unsigned)rtr_ceil_div(c2 * 32, 256), 256, 0, s>>>(a.part2, g.gx, c2, Y2, p->normx_part, g.gx,
                                                                        norm_out, p->flags);
    RTR_LAUNCH_CHECK("tc_reduce_kernel");
    tc_reduce_kernel<<<(unsigned)rtr_ceil_div(c3 * 32, 256), 256, 0, s>>>(a.part3, g.gx, c3, Y3, nullptr, 0,
                                                                        nullptr, p->flags);
    RTR_LAUNCH_CHECK("tc_reduce_kernel");
    *done = 1;
    return RTR_OK;
}

int launch_sketch_tma(rtr_plan* p, const float* X, int64_t A, int64_t I, int64_t B, int n, double* Y,
                      double* norm_out, cudaStream_t s, int64_t aoff) {
    const int K = p->K[n];
    SketchTmaArgs a{};
    a.A = A; a.B = B; a.I = (int)I; a.K = K; a.aoff = aoff;
    a.lm = B == 1 ? 1 : 0;
    a.N = (K <= 32) ? 32 : 64;
    a.fp8 = p->params.prec == RTR_FP8 ? 1 : 0;
    // chunk width 64: a ragged tail of each b-run is zero-filled by the TMA
    // unit (for B = 200 the slots then carry 200 of 256 values, against 40
    // of 64 for 40-wide chunks: 2.37 ms per 200^4 pass against 2.68 ms).
    // FP8 chunks hold whole 32-value scale blocks: 64, or 32 when B % 64 != 0.
    a.kc = 64;
    if (a.fp8 && B % 64 != 0) a.kc = 32;
    if (a.lm) {
        // the last mode: chunks of 64 consecutive a, boxes of 64 a x 64 i
        a.kc = 64;
        a.nbc = 1;
        a.nchunks = rtr_ceil_div(A, 64);
    } else {
        a.nbc = rtr_ceil_div(B, a.kc);
        a.nchunks = A * a.nbc;
    }
    a.seed = p->params.seed; a.mode = n;
    a.tab = a.fp8 ? p->tab_e4m3 : p->tab_bf16; a.flags = p->flags;
    // a CTA covers up to 256 rows: MT = 2 tiles of 128 when the view has more than 128
    a.MT = I > 128 ? 2 : 1;
    const size_t slot = (size_t)a.MT * TM_TILE + (size_t)a.N * 128;
    const size_t fixed = 8192 + (4 * TM_MAX_SLOTS + 2) * 8 + 64 + 1024;   // table, barriers, scalars, alignment
    a.S = (int)std::min<size_t>(TM_MAX_SLOTS, (SMEM_LIMIT - fixed) / slot);
    if (a.S < 2) return rtr_set_error(RTR_EUNSUPPORTED, "TMA sketch: no two slots fit in shared memory");
    const size_t smem = fixed + (size_t)a.S * slot;
    const int gy = (int)rtr_ceil_div(I, 256);
    int64_t gx = std::max<int64_t>(1, p->num_sms / gy);
    gx = std::min<int64_t>(gx, a.nchunks);
    if ((size_t)(gx * I * K) > p->partial_elems) return rtr_set_error(RTR_ENOMEM, "sketch partials exceed workspace");
    if ((size_t)(gx * gy) > p->normx_part_elems) return rtr_set_error(RTR_ENOMEM, "norm partials exceed workspace");
    a.partial = p->partial;
    a.normp = norm_out ? p->normx_part : nullptr;
    CUtensorMap tmap;
    CUresult cr;
    if (a.lm) {
        const cuuint64_t gdim[2] = {(cuuint64_t)I, (cuuint64_t)A};
        const cuuint64_t gstride[1] = {(cuuint64_t)I * 4};
        const cuuint32_t box[2] = {64, 64};
        const cuuint32_t estr[2] = {1, 1};
        cr = tensor_map_encoder()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), gdim, gstride, box,
                                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t gdim[3] = {(cuuint64_t)B, (cuuint64_t)I, (cuuint64_t)A};
        const cuuint64_t gstride[2] = {(cuuint64_t)B * 4, (cuuint64_t)I * B * 4};
        const cuuint32_t box[3] = {(cuuint32_t)a.kc, 128, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        cr = tensor_map_encoder()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(X), gdim, gstride, box,
                                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (cr != CUDA_SUCCESS) return rtr_set_error(RTR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    // one instantiation per (last mode, value form with 64-wide chunks)
    auto launch = [&](auto kern) -> int {
        RTR_SMEM(kern, smem);
        kern<<<dim3((unsigned)gx, (unsigned)gy), TM_NTHREADS, smem, s>>>(tmap, a);
        return RTR_OK;
    };
    const int var = a.kc != 64 ? 0 : a.fp8 ? 2 : 1;
    int lst;
    if (a.lm) lst = var == 1 ? launch(sketch_tma_kernel<true, 1>) : var == 2 ? launch(sketch_tma_kernel<true, 2>)
                                                                      : launch(sketch_tma_kernel<true, 0>);
    else lst = var == 1 ? launch(sketch_tma_kernel<false, 1>) : var == 2 ? launch(sketch_tma_kernel<false, 2>)
                                                                  : launch(sketch_tma_kernel<false, 0>);
    if (lst) return lst;
    RTR_LAUNCH_CHECK("sketch_tma_kernel");
    const int64_t count = I * K;
    tc_reduce_kernel<<<(unsigned)rtr_ceil_div(count * 32, 256), 256, 0, s>>>(p->partial, (int)gx, count, Y,
                                                                          p->normx_part, (int)(gx * gy), norm_out,
                                                                          p->flags);
    RTR_LAUNCH_CHECK("tc_reduce_kernel");
    return RTR_OK;
}

size_t tc_ws_bytes(const rtr_plan* p) { (void)p; return 0; }

// Tensor-core sketch of one mode of a float32 tensor viewed as (A, I, B)
// (X itself, or an intermediate of the sequential projection): Y = X_(n) Omega_n.
// norm_out (may be NULL) receives sum x^2 of the tensor.
int launch_sketch_tc_mode(rtr_plan* p, const float* X, int64_t A, int64_t I, int64_t B, int n, double* Y,
                          double* norm_out, cudaStream_t s, int64_t aoff) {
    const int K = p->K[n];
    const bool aligned16 = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    const bool fp8 = p->params.prec == RTR_FP8;
    if (B > 1 && B % 4 == 0 && aligned16 && A < ((int64_t)1 << 31) && tensor_map_encoder())
        return launch_sketch_tma(p, X, A, I, B, n, Y, norm_out, s, aoff);
    // the last mode on the same pipeline (BF16 and FP8)
    if (B == 1 && I % 4 == 0 && aligned16 && A < ((int64_t)1 << 31) && tensor_map_encoder())
        return launch_sketch_tma(p, X, A, I, B, n, Y, norm_out, s, aoff);
    // the FP8 form exists in the TMA kernel (B > 1) and in the vectorised
    // last-mode path of sketch_tc_kernel only
    if (fp8 && (B > 1 || !aligned16 || I % 4 != 0))
        return rtr_set_error(RTR_EUNSUPPORTED,
                             "FP8 sketch of mode %d needs a 16-byte aligned X and %s", n,
                             B > 1 ? "B % 4 == 0 (TMA path)" : "I_n % 4 == 0");
    int MT, N, S;
    size_t smem;
    if (!sketch_geometry(I, K, &MT, &N, &S, &smem))
        return rtr_set_error(RTR_EUNSUPPORTED, "tensor-core sketch: no stage fits in shared memory");
    SketchTCArgs a{};
    a.X = X; a.A = A; a.B = B; a.I = (int)I; a.K = K; a.N = N; a.MT = MT; a.rows_cta = MT * 128; a.S = S;
    if (B > 1) { a.nbc = rtr_ceil_div(B, KC); a.nchunks = A * a.nbc; }
    else { a.nbc = 1; a.nchunks = rtr_ceil_div(A, KC); }
    a.seed = p->params.seed; a.mode = n; a.aoff = aoff;
    a.vec = aligned16 && ((B > 1) ? (B % 4 == 0) : (I % 4 == 0)) ? 1 : 0;
    a.fp8 = fp8 ? 1 : 0;
    a.tab = fp8 ? p->tab_e4m3 : p->tab_bf16;
    a.flags = p->flags;
    const int gy = (int)rtr_ceil_div(I, a.rows_cta);
    int64_t gx = std::max<int64_t>(1, p->num_sms / gy);
    gx = std::min<int64_t>(gx, a.nchunks);
    if ((size_t)(gx * I * K) > p->partial_elems) return rtr_set_error(RTR_ENOMEM, "sketch partials exceed workspace");
    if ((size_t)(gx * gy) > p->normx_part_elems) return rtr_set_error(RTR_ENOMEM, "norm partials exceed workspace");
    a.partial = p->partial;
    a.normp = norm_out ? p->normx_part : nullptr;
    RTR_SMEM(sketch_tc_kernel, smem);
    sketch_tc_kernel<<<dim3((unsigned)gx, (unsigned)gy), NTHREADS, smem, s>>>(a);
    RTR_LAUNCH_CHECK("sketch_tc_kernel");
    const int64_t count = I * K;
    tc_reduce_kernel<<<(unsigned)rtr_ceil_div(count * 32, 256), 256, 0, s>>>(
        p->partial, (int)gx, count, Y, p->normx_part, (int)(gx * gy), norm_out, p->flags);
    RTR_LAUNCH_CHECK("tc_reduce_kernel");
    return RTR_OK;
}

int launch_sketch_tc(rtr_plan* p, const float* X, double* const* Y, cudaStream_t s) {
    bool norm_done = false;
    // modes N-2 and N-1 in one pass when the plan asks for it (BF16, RTR_PARAM_PAIR)
    int nmodes = p->N, pair = 0;
    if (p->N >= 3 && p->proj[p->N - 2] && p->proj[p->N - 1]) {
        const int st = launch_sketch_pair(p, X, Y[p->N - 2], Y[p->N - 1], p->scal + 0, s, &pair);
        if (st) return st;
        if (pair) { nmodes = p->N - 2; norm_done = true; }
    }
    for (int n = 0; n < nmodes; ++n) {
        if (!p->proj[n]) continue;
        int64_t A, I, B;
        rtr_mode_view(p->N, p->dims, n, &A, &I, &B);
        const int st = launch_sketch_tc_mode(p, X, A, I, B, n, Y[n], norm_done ? nullptr : p->scal + 0, s, 0);
        if (st) return st;
        norm_done = true;
    }
    if (!norm_done) return launch_sumsq(X, 0, p->numel, p->partial, 1024, p->scal + 0, p->flags, s);
    return RTR_OK;
}

// ---- tensor-core mode product of the last mode ------------------------------
// Algorithm 1 step 7 for the mode with B = 1 (X viewed as rows a of length I):
//     T[a, k] = sum_i X[a, i] Q[i, k]
// D += Xhi Qhi + Xlo Qhi + Xhi Qlo on tcgen05 (BF16 inputs, FP32 accumulation);
// Q (float64) is split once into resident bf16 hi/lo tiles.  Work unit = one
// 128-row tile of X and one 64-wide chunk of i, loaded by TMA as a box of
// 128 rows x 64 float32 into a ring slot and converted there in place into
// its hi (first 16 KB) and lo (second 16 KB) operand tiles, as in the sketch.
// Warps: 8 converters, 1 MMA issuer, 4 epilogue warps draining a
// double-buffered TMEM accumulator into T, 1 TMA producer.
namespace {

constexpr int TT_CONV_WARPS = 8;
constexpr int TT_MMA_WARP = TT_CONV_WARPS;
constexpr int TT_TMA_WARP = TT_CONV_WARPS + 1 + 4;
constexpr int TT_NTHREADS = (TT_TMA_WARP + 1) * 32;       // converters, MMA issuer, 4 epilogue warps, TMA
constexpr int TT_CONV_THREADS = TT_CONV_WARPS * 32;
constexpr int TT_PIECES = 128 * 32 / TT_CONV_THREADS;    // float4 pieces per converter thread per unit

struct TtmTCArgs {
    const double* Q;
    float* out;
    int64_t A;
    int I, K, N, NKC, S;          // NKC: 64-wide K atoms of I (Q tiles); a work unit holds two
    int NKU;                      // work units (128 columns of i) per 128-row tile
    int64_t ntiles;
    int* flags;
};

// named barrier 2 among the product's converter threads
__device__ __forceinline__ void tt_conv_bar() {
    asm volatile("bar.sync 2, %0;" ::"n"(TT_CONV_THREADS) : "memory");
}
__device__ __forceinline__ bool tt_conv_bar_and(bool v) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred pv, pr;\n\tsetp.ne.u32 pv, %1, 0;\n\tbar.red.and.pred pr, 2, %2, pv;\n\t"
                 "selp.u32 %0, 1, 0, pr;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v), "n"(TT_CONV_THREADS) : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(TT_NTHREADS, 1) ttm_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                               const TtmTCArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    const uint32_t btile = (uint32_t)p.N * 128u;
    const uint32_t b_bytes = 2u * p.NKC * btile;               // Q hi tiles, then Q lo tiles
    const uint32_t a_stage = 4u * MTILE_BYTES;                 // one box of 128 x 128 float32 = 2 x (X hi + X lo)
    const int S = p.S;
    const uint32_t bbase = smem_u32(sm);
    const uint32_t abase = bbase + b_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + b_bytes + S * a_stage);
    uint64_t* full = bars;              // TMA landed
    uint64_t* conv = bars + S;          // operand tiles written (8 converter warps)
    uint64_t* empty = bars + 2 * S;     // MMAs of the slot done
    uint64_t* accf = bars + 3 * S;      // [2]
    uint64_t* acce = bars + 3 * S + 2;  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 4);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = 2u * p.N;

    // ---- set-up: Q hi/lo tiles, barriers, TMEM
    for (int e = tid; e < p.NKC * p.N * 32; e += TT_NTHREADS) {
        const int c = e / (p.N * 32), rem = e % (p.N * 32);
        const int k = rem / 32, ip = rem % 32;          // bf16 pair (2 ip, 2 ip + 1) of chunk c, row k
        const int i0 = c * 64 + 2 * ip;
        const float q0 = (k < p.K && i0 < p.I) ? (float)p.Q[(int64_t)i0 * p.K + k] : 0.f;
        const float q1 = (k < p.K && i0 + 1 < p.I) ? (float)p.Q[(int64_t)(i0 + 1) * p.K + k] : 0.f;
        uint32_t h, l;
        split2(q0, q1, h, l);
        const uint32_t off = sw128_off(k, 2 * ip);
        st_shared_u32(bbase + c * btile + off, h);
        st_shared_u32(bbase + (p.NKC + c) * btile + off, l);
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], TT_CONV_WARPS);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 128);
        }
        *abort = 0;
        mbar_fence_init();
    }
    if (warp == TT_MMA_WARP) tmem_alloc(tmem_slot, ncols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t nloc = (blockIdx.x < p.ntiles) ? (p.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nunits = nloc * p.NKU;

    if (warp < TT_CONV_WARPS) {
        // ================================================================ converters
        // a unit is a box of 128 rows x 128 float32 (rows of 512 bytes); it becomes
        // K atom 0 (columns 0-63: hi at 0, lo at 16 KB) and atom 1 (columns 64-127:
        // hi at 32 KB, lo at 48 KB).  Thread ct takes column group ct & 31 of rows
        // (ct >> 5) + 8 q, so the swizzle phase (row & 7) is its warp's for every q.
        const int ct = tid;
        const int cg = ct & 31;
        const uint32_t off0 = (uint32_t)(cg >> 4) * (2u * MTILE_BYTES) +
                              sw128_off((uint32_t)(ct >> 5), 4u * (uint32_t)(cg & 15));
        Ring rg(S);
        for (int64_t u = 0; u < nunits; ++u, rg.step(1)) {
            const int s = rg.slot;
            if (!tt_conv_bar_and(mbar_wait(&full[s], rg.use & 1, abort, p.flags))) break;
            const uint32_t src = abase + s * a_stage;
            float4 v[TT_PIECES];
#pragma unroll
            for (int q = 0; q < TT_PIECES; ++q)
                v[q] = ld_shared_f4(src + (uint32_t)((ct >> 5) + 8 * q) * 512u + (uint32_t)cg * 16u);
            tt_conv_bar();                            // every piece of the box is in registers
#pragma unroll
            for (int q = 0; q < TT_PIECES; ++q) {
                uint32_t h0, l0, h1, l1;
                split2(v[q].x, v[q].y, h0, l0);
                split2(v[q].z, v[q].w, h1, l1);
                st_shared_v2(src + off0 + 1024u * q, h0, h1);
                st_shared_v2(src + MTILE_BYTES + off0 + 1024u * q, l0, l1);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[s]);
        }
    } else if (warp == TT_MMA_WARP) {
        // ================================================================ MMA issuer
        const uint32_t idesc = idesc_bf16_f32(128, p.N);
        bool ok = true;
        Ring rg(S);
        for (int64_t j = 0; j < nloc && ok; ++j) {
            const int buf = (int)(j & 1);
            if (j >= 2 && !mbar_wait(&acce[buf], (uint32_t)(((j >> 1) - 1) & 1), abort, p.flags)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(buf * p.N);
            for (int cu = 0; cu < p.NKU; ++cu, rg.step(1)) {
                const int s = rg.slot;
                if (!mbar_wait(&conv[s], rg.use & 1, abort, p.flags)) { ok = false; break; }
                tc_fence_after();
                if (lane == 0) {
                    for (int h = 0; h < 2; ++h) {
                        const int c = 2 * cu + h;             // K atom of I
                        if (c >= p.NKC) break;
                        const uint32_t ahi = abase + s * a_stage + (uint32_t)h * 2u * MTILE_BYTES, alo = ahi + MTILE_BYTES;
                        const uint32_t bhi = bbase + c * btile, blo = bbase + (p.NKC + c) * btile;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t dah = sdesc_sw128(ahi + 32u * kk), dal = sdesc_sw128(alo + 32u * kk);
                            const uint64_t dbh = sdesc_sw128(bhi + 32u * kk), dbl = sdesc_sw128(blo + 32u * kk);
                            mma_bf16(d, dah, dbh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                            mma_bf16(d, dal, dbh, idesc, 1u);
                            mma_bf16(d, dah, dbl, idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                __syncwarp();
            }
            if (ok && lane == 0) mma_commit(&accf[buf]);
            __syncwarp();
        }
    } else if (warp < TT_TMA_WARP) {
        // ================================================================ epilogue
        const int g = warp & 3;                       // TMEM lane group of this warp
        for (int64_t j = 0; j < nloc; ++j) {
            const int buf = (int)(j & 1);
            if (!mbar_wait(&accf[buf], (uint32_t)((j >> 1) & 1), abort, p.flags)) break;
            tc_fence_after();
            const int64_t a0 = (blockIdx.x + j * gridDim.x) * 128;
            const int64_t row = a0 + 32 * g + lane;
            for (int c0 = 0; c0 < p.N; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(buf * p.N + c0), v);
                if (row < p.A) {
                    float* dst = p.out + row * p.K;
#pragma unroll
                    for (int k = 0; k < 32; ++k)
                        if (c0 + k < p.K) dst[c0 + k] = v[k];
                }
            }
            tc_fence_before();
            mbar_arrive(&acce[buf]);
        }
    } else {
        // ================================================================ TMA producer
        if (lane == 0) {
            Ring rg(S);
            int64_t j = 0;
            int c = 0;
            for (int64_t u = 0; u < nunits; ++u, rg.step(1)) {
                const int s = rg.slot;
                if (u >= S && !mbar_wait(&empty[s], (rg.use - 1) & 1, abort, p.flags)) break;
                const int64_t a0 = (blockIdx.x + j * gridDim.x) * 128;
                // rows a >= A and columns i >= I are zero-filled without memory traffic
                mbar_arrive_expect_tx(&full[s], (uint32_t)a_stage);
                tma_load_2d(abase + s * a_stage, &tmap, c * 128, (int)a0, &full[s]);
                if (++c == p.NKU) { c = 0; ++j; }
            }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == TT_MMA_WARP) tmem_dealloc(tmem, ncols);
}

}  // namespace

int launch_ttm_tc(rtr_plan* p, const float* X, int64_t A, int64_t I, int64_t B, const double* Q, int K, float* out,
                  cudaStream_t s) {
    const bool tma_ok = (reinterpret_cast<uintptr_t>(X) & 15) == 0 && I % 4 == 0 && A < ((int64_t)1 << 31) &&
                        tensor_map_encoder();
    if (B != 1 || I > 256 || K > 64 || !tma_ok) {
        // other mode products of BF16 plans run on the SIMT FP32 kernel
        return launch_ttm(p, 0, X, A, I, B, Q, K, out, s);
    }
    TtmTCArgs a{};
    a.Q = Q; a.out = out; a.A = A; a.I = (int)I; a.K = K;
    a.N = (K <= 32) ? 32 : 64;
    a.NKC = (int)rtr_ceil_div(I, 64);
    a.NKU = (int)rtr_ceil_div(I, 128);
    a.ntiles = rtr_ceil_div(A, 128);
    a.flags = p->flags;
    const size_t bq = 2 * (size_t)a.NKC * a.N * 128;
    const size_t fixed = 1024 + 256;
    int S = (int)((SMEM_LIMIT - fixed - bq) / (4 * MTILE_BYTES));
    S = std::min(S, 6);
    if (S < 2) return launch_ttm(p, 0, X, A, I, B, Q, K, out, s);
    a.S = S;
    const size_t smem = fixed + bq + (size_t)S * 4 * MTILE_BYTES;
    CUtensorMap tmap;
    const cuuint64_t gdim[2] = {(cuuint64_t)I, (cuuint64_t)A};
    const cuuint64_t gstride[1] = {(cuuint64_t)I * 4};
    const cuuint32_t box[2] = {128, 128};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult cr = tensor_map_encoder()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), gdim,
                                             gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return rtr_set_error(RTR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(a.ntiles, p->num_sms));
    RTR_SMEM(ttm_tc_kernel, smem);
    ttm_tc_kernel<<<(unsigned)gx, TT_NTHREADS, smem, s>>>(tmap, a);
    RTR_LAUNCH_CHECK("ttm_tc_kernel");
    return RTR_OK;
}

// ---- test support: a bounded wait that runs out ------------------------------
namespace {

// One thread waits on a barrier of this CTA that expects one arrival and
// never gets it; the bounded wait gives up after limit_ns, raises
// RTR_FLAG_TIMEOUT in *flags, and the kernel returns normally.
__global__ void expired_wait_kernel(uint64_t limit_ns, int* flags) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        rtr::tc::mbar_init(&bar, 1);
        rtr::tc::mbar_fence_init();
        abort_flag = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) rtr::tc::mbar_wait(&bar, 0, (volatile int*)&abort_flag, flags, limit_ns);
}

}  // namespace

extern "C" int rtr_test_bounded_wait(int limit_us, int* flags, void* stream) {
    if (!flags) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (limit_us < 1 || limit_us > 2000000)
        return rtr_set_error(RTR_EINVAL, "wait limit %d us outside [1, 2000000]", limit_us);
    cudaStream_t s = (cudaStream_t)stream;
    expired_wait_kernel<<<1, 32, 0, s>>>((uint64_t)limit_us * 1000ull, flags);
    RTR_LAUNCH_CHECK("expired_wait_kernel");
    RTR_CUDA(cudaStreamSynchronize(s));
    int h = 0;
    RTR_CUDA(cudaMemcpy(&h, flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & RTR_FLAG_TIMEOUT)
        return rtr_set_error(RTR_ETIMEOUT, "a bounded device wait gave up after %d us", limit_us);
    return RTR_OK;
}
