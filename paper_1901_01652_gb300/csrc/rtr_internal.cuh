// Internal declarations of the rTRD CUDA library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "rtr.h"

#define RTR_MAXN 8
#define RTR_MAX_KSKETCH 64
#define RTR_MAX_RANK 16

struct rtr_plan {
    int N = 0;
    int64_t dims[RTR_MAXN] = {};
    int Kreq[RTR_MAXN] = {};
    int K[RTR_MAXN] = {};        // effective projection size
    int R[RTR_MAXN] = {};
    int proj[RTR_MAXN] = {};     // 1 if mode is projected (K < I)
    int order[RTR_MAXN] = {};    // chain order
    rtr_params params{};
    int device = 0;
    int num_sms = 0;
    int64_t numel = 0;           // |X|
    int64_t pnumel = 0;          // |P|

    // device Gaussian tables (4096 entries)
    double* tab64 = nullptr;     // float64 quantiles
    float* tab32 = nullptr;      // bfloat16-rounded quantiles as float
    uint16_t* tab_bf16 = nullptr;// bfloat16 bit patterns
    uint16_t* tab_e4m3 = nullptr;// e4m3-rounded quantiles as bfloat16 bit patterns (exact)

    // workspace
    double* partial = nullptr;   size_t partial_elems = 0;    // split-K partials
    double* normx_part = nullptr; size_t normx_part_elems = 0;
    double* scal = nullptr;      // scalars: [0] ||X||^2 [1] ||P||^2 [2..] misc
    void* chain[2] = {nullptr, nullptr}; size_t chain_bytes[2] = {0, 0};
    double* qr_ws = nullptr;     size_t qr_ws_elems = 0;      // orth workspace
    double* als_ws = nullptr;    size_t als_ws_elems = 0;     // FP64 ALS workspace
    size_t als_wmax = 0;         // max K_n R_n R_{n+1}
    size_t als_maxK = 0;         // max K_n
    cudaStream_t side = nullptr; // second stream for work that overlaps the caller's stream
    cudaStream_t side2 = nullptr;// third stream (TR-ALS: prefix products of the Gram chains)
    cudaEvent_t ev[6] = {};
    // TR-ALS replay: the sweeps of rtr_als recorded once (on `cap`, a stream of
    // the plan) per argument set and replayed on the caller's stream
    cudaStream_t cap = nullptr;
    cudaGraphExec_t als_exec = nullptr;
    const void* als_key_P = nullptr;
    double* als_key_Z[RTR_MAXN] = {};
    double* als_key_err = nullptr;
    int als_key_init = -1;
    long long als_kernels = 0;   // kernels in the recorded graph (counted at each replay)
    void* sub_ws[2] = {nullptr, nullptr}; size_t sub_bytes = 0;  // subchain ping-pong
    int* flags = nullptr;
    void* tc_ws = nullptr;       size_t tc_ws_bytes = 0;       // tensor-core path workspace
    void* ttm_q = nullptr;       size_t ttm_q_bytes = 0;       // mode-product Q in the compute type
    double* svd_ws = nullptr;    int64_t svd_cbuf = 0, svd_gmax = 0, svd_umax = 0;  // TR-SVD workspace
    // power iterations: Q of the current mode (I_n x K_n float64) and
    // T = X x_n Q^T in the compute type (max_n |X| K_n / I_n values)
    double* pow_q = nullptr;
    void* pow_t = nullptr;       size_t pow_t_bytes = 0;
    double* acc_y = nullptr;     // one slab's Y_n (max I_n x 64) before it is added in (rtr_project_host)
};

// ---- error reporting (rtr_api.cu) -------------------------------------------
int rtr_set_error(int code, const char* fmt, ...);
int rtr_cuda_check(cudaError_t e, const char* what);
#define RTR_CUDA(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return rtr_cuda_check(e_, #call); } while (0)
// every kernel launch of the library is followed by this check, which also
// counts the launch (rtr_kernel_launches)
void rtr_count_launch();
void rtr_count_launches(long long delta);
#define RTR_LAUNCH_CHECK(what) do { rtr_count_launch(); cudaError_t e_ = cudaGetLastError(); if (e_ != cudaSuccess) return rtr_cuda_check(e_, what); } while (0)

static inline int64_t rtr_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Dynamic shared memory of a kernel: the first call for a kernel on a device
// raises its limit to the device's opt-in maximum (less the kernel's static
// shared memory); every call checks that `bytes` fits.  The limit is a
// property of the kernel that is read when a launch runs, also when a CUDA
// graph replays a recorded launch: setting it to each launch's own size
// would let a later, smaller launch of the same kernel lower it below what a
// recorded graph node needs.
int rtr_smem_limit(const void* kernel, size_t bytes);
#define RTR_SMEM(kernel, bytes) do { const int st_ = rtr_smem_limit((const void*)(kernel), (size_t)(bytes)); if (st_) return st_; } while (0)

// host copies of the Gaussian quantile table: float64 and bfloat16-rounded
void rtr_host_tables(double* t64, float* t32);

// mode view (A, I, B) of a shape
static inline void rtr_mode_view(int N, const int64_t* dims, int n, int64_t* A, int64_t* I, int64_t* B) {
    int64_t a = 1, b = 1;
    for (int m = 0; m < n; ++m) a *= dims[m];
    for (int m = n + 1; m < N; ++m) b *= dims[m];
    *A = a; *I = dims[n]; *B = b;
}

// ---- launchers implemented in the kernel translation units -------------------
// k_sketch.cu: generic split-K "mode contraction"
//   Y[i, c] = sum_{a,b} X[a, i, b] * M[r(a,b), c]     (i < I, c < C)
// with M either generated (Gaussian test matrix Omega_n, r = a*B + b) or read
// from memory (row r = a*B + b, leading dimension ldm).  Writes FP64 partials
// and reduces them deterministically into Y (ldy = C).
struct ContractArgs {
    const void* X; int64_t A; int64_t I; int64_t B;
    int C;
    // generated operand; aoff: index of the view's first a in the whole tensor
    // (Omega_n row r = (a + aoff) * B + b), 0 unless X is a slab
    int gen; uint64_t seed; int mode; const void* table; int64_t aoff;
    // stored operand (gen == 0), same element type as X: row r = a*B + b at
    // M[r * ldm + c] (makb = 0), or M laid out (A, C, B), entry (a, c, b) at
    // M[(a * C + c) * B + b] (makb = 1: the output of a mode product)
    const void* M; int64_t ldm; int makb;
    double* Y;                  // I x C float64 output
    double* norm_out;           // optional: receives sum x^2 (float64) of X
};
int launch_contract(rtr_plan* p, int is_f64, const ContractArgs& a, cudaStream_t s);

// k_ttm.cu: out[a, k, b] = sum_i X[a, i, b] * Q[i, k]   (Q: I x K float64)
int launch_ttm(rtr_plan* p, int is_f64, const void* X, int64_t A, int64_t I, int64_t B,
               const double* Q, int K, void* out, cudaStream_t s);

// k_linalg.cu
int launch_orth(rtr_plan* p, const double* const* Y, double* const* Q, cudaStream_t s);
// the modes whose bit is set in `mask` only (Y, Q: arrays of N pointers)
int launch_orth_mask(rtr_plan* p, const double* const* Y, double* const* Q, unsigned mask, cudaStream_t s);
// *out = sum of squares of X[0 .. n); a non-finite result raises
// RTR_FLAG_NONFINITE in *flags (when flags is not NULL)
int launch_sumsq(const void* X, int is_f64, int64_t n, double* part, int nparts, double* out, int* flags,
                 cudaStream_t s);

// y[0 .. n) += x[0 .. n) (float64 or float32)
int launch_add(void* y, const void* x, int64_t n, int is_f64, cudaStream_t s);

// k_als.cu
int run_als(rtr_plan* p, const void* P, double* const* Z, int init_given, double* err,
            cudaStream_t s);
int run_backproject(rtr_plan* p, const double* const* Z, const double* const* Q,
                    double* const* G, const int* ranks, cudaStream_t s);
int run_reconstruct(int N, const int64_t* dims, const int* R, const double* const* G,
                    int out_prec, void* Xhat, void* work, size_t work_bytes, cudaStream_t s);
size_t reconstruct_work_bytes(int N, const int64_t* dims, const int* R);
int run_rse(rtr_plan* p, const void* P, const double* const* Z, const int* ranks, double* out,
            cudaStream_t s);
int run_draw_omega(rtr_plan* p, int mode, int64_t row0, int64_t nrows, int K, double* out,
                   cudaStream_t s);

// k_als_batch.cu: grouped TR-ALS over a batch of projected tensors of the
// same order (default start, `sweeps` sweeps).  K, R: count*N effective
// sizes and ranks; P, Z: per-tensor device buffers fixed at creation.
struct BatchAls;
int batch_als_create(BatchAls** out, int count, int N, const int64_t* K, const int* R, int is_f64, int sweeps,
                     const uint64_t* seeds, const double* tab, const void* const* P, double* const* Z, int num_sms);
void batch_als_destroy(BatchAls* b);
int batch_als_run(BatchAls* b, double* err, cudaStream_t s);
int batch_als_flags(BatchAls* b, int* flags);

// k_tc.cu: tensor-core sketch (BF16/FP8 plans) of one mode of a float32
// tensor viewed as (A, I, B), and of every projected mode of X; the
// tensor-core product of the last mode (B = 1), other views fall back to launch_ttm
// aoff: index of the view's first a in the whole tensor (0 unless X is a slab)
int launch_sketch_tc_mode(rtr_plan* p, const float* X, int64_t A, int64_t I, int64_t B, int n, double* Y,
                          double* norm_out, cudaStream_t s, int64_t aoff);
int launch_sketch_tc(rtr_plan* p, const float* X, double* const* Y, cudaStream_t s);
// modes N-2 and N-1 of the BF16 sketch in one pass over X (*done = 0: not taken)
int launch_sketch_pair(rtr_plan* p, const float* X, double* Y2, double* Y3, double* norm_out, cudaStream_t s,
                       int* done);
// partial-sum elements that pass needs (at most)
size_t pair_partial_elems(int num_sms, int64_t I, int K2, int64_t J, int K3);
// reads of a 16-byte aligned X by rtr_sketch (one per projected mode, one
// less when the last two modes share a pass: RTR_PARAM_PAIR)
int sketch_passes(const rtr_plan* p);
int launch_ttm_tc(rtr_plan* p, const float* X, int64_t A, int64_t I, int64_t B, const double* Q, int K, float* out,
                  cudaStream_t s);

// k_trsvd.cu
int run_trsvd(rtr_plan* p, const void* P, double tol, double* const* Z, int* ranks, cudaStream_t s);

// ---- device helpers ----------------------------------------------------------
#ifdef __CUDACC__
namespace rtr {

// Philox4x64-10 (Salmon et al., SC'11): 256-bit counter, 128-bit key.
__device__ __forceinline__ void philox4x64_10(uint64_t& c0, uint64_t& c1, uint64_t& c2, uint64_t& c3,
                                              uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
}

// The 20 table indices of one Philox call for Omega_n row r, column block cb:
// index t (0..19) is bits 12*(t%5).. of word t/5.
__device__ __forceinline__ void omega_words(uint64_t seed, int mode, uint64_t r, uint64_t cb,
                                            uint64_t w[4]) {
    uint64_t c0 = r, c1 = cb, c2 = 0, c3 = 0;
    philox4x64_10(c0, c1, c2, c3, seed, (uint64_t)mode);
    w[0] = c0; w[1] = c1; w[2] = c2; w[3] = c3;
}
__device__ __forceinline__ int omega_field(const uint64_t w[4], int t) {
    return (int)((w[t / 5] >> (12 * (t % 5))) & 0xFFFull);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace rtr
#endif
