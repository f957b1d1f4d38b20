/*
 * rtr.h - C ABI of the GB300 randomized tensor-ring decomposition library.
 *
 * Method: Yuan, Li, Cao, Zhao, "Randomized Tensor Ring Decomposition and Its
 * Application to Large-scale Data Reconstruction" (arXiv:1901.01652),
 * Algorithm 1 (rTRD), Eq. 1-4.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status (RTR_OK = 0).  On failure
 *    rtr_last_error() returns a message for the calling host thread.
 *  - Tensors are dense, row-major, last mode fastest.  dims[] has N entries,
 *    3 <= N <= 8 for the decomposition entry points (rtr_reconstruct also
 *    accepts N = 2).  Mode numbers are 0-based (the paper counts from 1).
 *  - TR cores are float64, core n of shape R_n x I_n x R_{n+1} row-major,
 *    with R_{N+1} = R_1 (Section 2.2).
 *  - All data pointers are DEVICE pointers owned by the caller; arrays of
 *    pointers (double* const* Y, ...) are HOST arrays of N device pointers.
 *    The library allocates device memory only in rtr_plan_create (its
 *    workspace and tables) and frees it in rtr_plan_destroy.
 *  - Every compute call takes a cudaStream_t (passed as void*; NULL = the
 *    legacy default stream), is asynchronous on that stream and does not
 *    synchronise.  Calls on one plan must not overlap in time (the plan's
 *    workspace is shared by its calls); use one plan per concurrent stream.
 *  - Input-dependent numerical events (non-finite values, a Cholesky that
 *    fell back) are recorded in device flags that rtr_plan_flags() reads.
 */
#ifndef RTR_H
#define RTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RTR_OK            0
#define RTR_EINVAL        1   /* bad argument (null pointer, size, rank, precision) */
#define RTR_ENOMEM        2   /* workspace allocation failed */
#define RTR_ECUDA         3   /* a CUDA call failed (message has the CUDA error) */
#define RTR_ENONFINITE    4   /* non-finite values met (device flag) */
#define RTR_ENOTCONV      5   /* warning: a fallback path was taken; results written */
#define RTR_ETIMEOUT      6   /* a bounded device wait gave up (device flag) */
#define RTR_EUNSUPPORTED  7   /* valid request this build does not implement */

/* arithmetic of the sketch and mode-product chain (Algorithm 1, steps 5, 7) */
#define RTR_FP64  0   /* X float64; every step float64                            */
#define RTR_FP32  1   /* X float32; SIMT float32 sketch / chain, float64 QR & solves */
#define RTR_BF16  2   /* X float32; tcgen05 BF16 (hi+lo split) sketch / chain      */
#define RTR_FP8   3   /* X float32; the sketch reads a block-scaled float8 copy of X:
                         e4m3 values with one power-of-two scale per block of 32
                         (blocks run along b of each (a, i) fibre of the (A, I_n, B)
                         mode view, along a when B = 1; scale exponent
                         max(floor(log2 amax) - 8, -120); round to nearest even,
                         saturate at 448) against the e4m3-rounded quantile table.
                         The dequantised values are exact in bfloat16, so one BF16
                         tcgen05 MMA per step forms the same products with FP32
                         accumulation.  Quantisation happens in the kernel's
                         registers (X stays float32 in memory).  Everything after
                         the sketch runs as for RTR_BF16. */

/* rtr_params.flags bits */
#define RTR_PARAM_NO_GRAPH     1   /* rtr_batch_run: always run eagerly, never capture a graph */
#define RTR_PARAM_PAIR         2   /* rtr_sketch (BF16): sketch the last two modes from the same
                                      tiles of X, one pass for both, instead of one pass per mode
                                      (same products, other summation order; off by default: on
                                      GB300 at 200^4 the shared pass takes 3.8 ms against 3.4 ms
                                      for the two single-mode passes) */

/* device flag bits (rtr_plan_flags) */
#define RTR_FLAG_NONFINITE     1   /* NaN/Inf met in an input or a reduction */
#define RTR_FLAG_QR_FALLBACK   2   /* CholeskyQR2 failed; Gram-Schmidt applied twice used */
#define RTR_FLAG_GRAM_PINV     4   /* an ALS Gram matrix was not SPD; pseudo-inverse used */
#define RTR_FLAG_TIMEOUT       8   /* a bounded device wait gave up */

typedef struct rtr_plan rtr_plan;

typedef struct {
    int      prec;            /* RTR_FP64 / RTR_FP32 / RTR_BF16 / RTR_FP8 */
    uint64_t seed;            /* seed of the Gaussian test matrices Omega_n */
    int      sweeps;          /* TR-ALS sweeps (each updates cores 1..N once) */
    double   tol;             /* TR-SVD relative tolerance epsilon */
    int      flags;           /* RTR_PARAM_* bits, 0 = defaults */
    int      chain_order[8];  /* order of the mode products of step 7; all -1 = default
                                 (largest I_n/K_n first; among equal ratios the last
                                 mode first, then increasing mode order) */
    int      power_iters;     /* q >= 0 power iterations per sketch (the remark after
                                 Algorithm 1): rtr_sketch returns Y_n after q times
                                 Y <- X_(n) (X_(n)^T orth(Y)); 0 = the plain sketch */
} rtr_params;

/* Fill *p with defaults: FP32, seed 0, 20 sweeps, tol 1e-2, default chain order,
   no power iterations. */
void rtr_params_default(rtr_params* p);

/* Message of the last failed call on this host thread ("" if none). */
const char* rtr_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
   (all threads; for accounting launches inside a timed region). */
unsigned long long rtr_kernel_launches(void);

/*
 * Create a plan for an order-N tensor of shape dims[N] with projection sizes
 * K[N] (Algorithm 1, input [K_n]) and TR ranks R[N] (input R_1..R_N).
 * A mode with K_n >= I_n is not projected: Q_n = I and K_n := I_n (the
 * paper keeps such a mode whole in Section 4.1).  Limits: 1 <= K_n <= 64
 * for projected modes, 1 <= R_n <= 16.  Allocates the workspace on the
 * current device.  The plan is owned by the caller; free with rtr_plan_destroy.
 */
int rtr_plan_create(rtr_plan** plan, int N, const int64_t* dims, const int* K,
                    const int* R, const rtr_params* params);
int rtr_plan_destroy(rtr_plan* plan);

/* Effective K_n (after the K_n >= I_n rule) and the chain order the plan uses. */
int rtr_plan_info(const rtr_plan* plan, int* K_eff, int* chain_order);

/* Read and clear the device flags (synchronises the device). */
int rtr_plan_flags(rtr_plan* plan, int* flags);

/* Number of passes over a 16-byte aligned X that rtr_sketch makes (Algorithm 1
   step 5): one per projected mode, one less when a BF16 plan sketches its last
   two modes from the same tiles of X (RTR_PARAM_PAIR, both projected,
   I_N % 4 == 0, the accumulators fit).  Host only, no device work. */
int rtr_plan_sketch_passes(const rtr_plan* plan, int* passes);

/*
 * Algorithm 1, steps 4-5: for every projected mode n,
 *     Y_n = X_(n) Omega_n        (I_n x K_n, float64, row-major)
 * X: dims, float64 for RTR_FP64 plans, float32 otherwise.  Omega_n is never
 * stored: entry (r, k) is generated in the kernel from Philox4x64-10 with key
 * (seed, n) and counter (r, k/20, 0, 0) mapped through the 4096-level Gaussian
 * quantile table (float64 values for RTR_FP64, bfloat16-rounded values for
 * RTR_FP32 and RTR_BF16, e4m3-rounded values for RTR_FP8); r is the row-major
 * index of the other modes.  RTR_FP8 plans sketch the block-scaled float8 copy
 * of X described at RTR_FP8; they need a 16-byte aligned X and, per projected
 * mode, B % 4 == 0 (B > 1) or I_n % 4 == 0 (B = 1), else RTR_EUNSUPPORTED.
 * Y[n] may be NULL for modes that are not projected.  Also records ||X||_F^2
 * (of X itself, not of its float8 copy) in the plan for rtr_rse; a NaN or Inf
 * in X makes that sum non-finite and raises RTR_FLAG_NONFINITE (rtr_plan_flags).
 *
 * With params.power_iters = q > 0 (Section 3.2, the remark after Algorithm 1:
 * power iterations, citing Halko et al.) every projected mode then runs q
 * times  Q = orth(Y_n);  T = X x_n Q^T;  Y_n = X_(n) T_(n)^T,  i.e. Y_n <-
 * X_(n) X_(n)^T orth(Y_n), on X itself (also for RTR_FP8): the mode product
 * of rtr_project (tensor cores for the last mode of BF16/FP8 plans) and the
 * split-K contraction with a stored operand (float32 SIMT for the float
 * plans, float64 for RTR_FP64).  Each iteration reads X twice per mode and
 * uses a plan buffer of max_n |X| K_n / I_n values.
 */
int rtr_sketch(rtr_plan* plan, const void* X, double* const* Y, void* stream);

/*
 * Sequential form of Algorithm 1 steps 3-8 (not the paper's: its step 5
 * sketches every mode from X itself): the modes are taken in the plan's chain
 * order and mode n is sketched from the tensor the earlier modes have already
 * shrunk,
 *     Y_n = P_(n) Omega_n,   Q_n = orth(Y_n),   P <- P x_n Q_n^T,
 * with Omega_n as in rtr_sketch (key (seed, n)) but with one row per entry of
 * the other modes of the current P (row-major index).  Outputs as rtr_sketch
 * (Y) and rtr_project (Q, P); records ||X||^2 for rtr_rse.  X is read twice
 * (its sketch and its product); every later step reads only intermediates.
 * power_iters must be 0.  RTR_FP8 plans need every sketched intermediate to
 * meet the FP8 alignment rule of rtr_sketch, else RTR_EUNSUPPORTED.
 */
int rtr_project_sequential(rtr_plan* plan, const void* X, double* const* Y, double* const* Q, void* P,
                           void* stream);

/*
 * Algorithm 1, steps 6-7 (Eq. 3): Q_n = orth(Y_n) (economy QR with diag(R) > 0,
 * CholeskyQR2 in float64; a mode whose Cholesky meets a pivot below 1e-14 of
 * its diagonal falls back to classical Gram-Schmidt applied twice), then
 *     P = X x_{pi_1} Q_{pi_1}^T ... x_{pi_N} Q_{pi_N}^T
 * in the plan's chain order.  Y[n]: I_n x K_n float64 (ignored for modes that
 * are not projected).  Q[n]: I_n x K_n float64 output (identity written for
 * unprojected modes).  P: K_1 x ... x K_N output, float64 for RTR_FP64 plans,
 * float32 otherwise.  X is read once by the first product; later products read
 * the plan's intermediates.
 */
int rtr_project(rtr_plan* plan, const void* X, const double* const* Y,
                double* const* Q, void* P, void* stream);

/*
 * Out-of-core form of Algorithm 1 steps 3-8 for a tensor in HOST memory (one
 * larger than the GPU's, or one that should not be copied whole): X is
 * streamed to the GPU in slabs of slab_rows indices of mode 0 (contiguous in
 * row-major order), twice.  Pass 1 sketches every projected mode slab by slab:
 * a slab holds whole rows of Y_0, and adds its part of Y_n = X_(n) Omega_n for
 * the other modes, the test-matrix rows counted over the whole tensor, so Y is
 * rtr_sketch's up to summation order; ||X||^2 is recorded for rtr_rse.  Then
 * Q_n = orth(Y_n) as in rtr_project, and pass 2 applies every mode product but
 * mode 0's to each slab and adds the slab's share of the mode-0 product into
 * P, P = sum over slabs of T_slab x_0 Q_0[slab rows]^T (Eq. 3: the products
 * commute, and mode 0's splits over its rows).  The plan's chain order must
 * end with mode 0; power_iters must be 0.
 * X_host: HOST pointer to X (page-locked memory lets the copies overlap the
 * kernels); it must stay valid until `stream` has passed this call's work.
 * stage[2]: caller-owned DEVICE buffers of stage_bytes each, at least
 * slab_rows * prod_{m>0} I_m elements (float64 for RTR_FP64 plans, float32
 * otherwise).  The copies run on a stream of the plan, overlapped with the
 * kernels on `stream` through events.  Y, Q, P as in rtr_sketch and
 * rtr_project.  RTR_FP8 plans with several slabs need slab_rows x
 * prod(I_1 .. I_{N-2}) to be a multiple of 32 (whole scale blocks of the last
 * mode's sketch), else RTR_EUNSUPPORTED.
 */
int rtr_project_host(rtr_plan* plan, const void* X_host, int64_t slab_rows, void* const* stage, size_t stage_bytes,
                     double* const* Y, double* const* Q, void* P, void* stream);

/*
 * Algorithm 1, step 9 with TR-ALS: fit cores Z_n (R_n x K_n x R_{n+1},
 * float64) to P by `sweeps` sweeps of exact least-squares core updates
 * (Eq. 2: P_<n> = Z_{n,(2)} S^T, S the subchain; Z_{n,(2)} = P_<n> S (S^T S)^-1,
 * the Gram S^T S formed from float64 transfer matrices and solved to float64
 * accuracy: a float32 inverse refined with double-float residuals).
 * Z: in/out.  If init_given != 0 the Z buffers hold the starting cores;
 * otherwise the library writes its default start (discrete-Gaussian cores
 * from Philox4x64-10 with key (seed + 1, 256 + n), scaled so ||TR(Z)|| = ||P||).
 * err: device float64[sweeps] (may be NULL) receives ||P - TR(Z)||_F after
 * each sweep.  Requires R_n R_{n+1} <= 144 for every n (else
 * RTR_EUNSUPPORTED).  The first call with a given (P, Z, err, init_given)
 * records the sweeps into a CUDA graph on a stream of the plan and later calls
 * with the same pointers replay it on `stream` (a call while `stream` is being
 * captured runs eagerly and is recorded by the caller's capture); calling with
 * new pointers synchronises the device once and records again.
 */
int rtr_als(rtr_plan* plan, const void* P, double* const* Z, int init_given,
            double* err, void* stream);

/*
 * Algorithm 1, step 9 with TR-SVD (Section 4.1 tolerance): sequential
 * truncated SVDs of P with delta = tol ||P|| / sqrt(N) (sqrt(2) delta for the
 * first, whose rank is split R_1 R_2 with R_1 the largest divisor <= sqrt).
 * ranks: host int[N]; if ranks[0] > 0 on entry the ranks are forced, else they
 * are chosen and written back.  Z: device buffers, each of capacity
 * R_max(n) x K_n x R_max(n+1) float64 with the plan's R as capacity.
 * (Returns RTR_EUNSUPPORTED in builds without the TR-SVD kernels.)
 */
int rtr_svd(rtr_plan* plan, const void* P, double tol, double* const* Z,
            int* ranks, void* stream);

/*
 * Algorithm 1, step 11 (read as the mode-2 product of the order-3 core):
 *     G_n = Z_n x_2 Q_n,   G_n[a, i, b] = sum_k Z_n[a, k, b] Q_n[i, k]
 * Z[n]: R_n x K_n x R_{n+1}; Q[n]: I_n x K_n; G[n]: R_n x I_n x R_{n+1}; all float64.
 * ranks: host int[N] ranks of Z (NULL = the plan's R).
 */
int rtr_backproject(rtr_plan* plan, const double* const* Z, const double* const* Q,
                    double* const* G, const int* ranks, void* stream);

/*
 * Psi([G_n]) of Eq. 4: the dense tensor of a TR (Eq. 1),
 *     Xhat(i_1..i_N) = Trace(G_1(i_1) ... G_N(i_N)).
 * N >= 2; G[n]: R[n] x dims[n] x R[(n+1)%N] float64.  out_prec RTR_FP64 writes
 * float64, RTR_FP32 writes float32 (accumulated in float32).  Allocates
 * nothing: the caller passes `work` (device, at least rtr_reconstruct_work_bytes
 * bytes).  No plan needed.
 */
size_t rtr_reconstruct_work_bytes(int N, const int64_t* dims, const int* R);
int rtr_reconstruct(int N, const int64_t* dims, const int* R, const double* const* G,
                    int out_prec, void* Xhat, void* work, size_t work_bytes, void* stream);

/*
 * RSE of Section 4 without forming the large tensor:
 *     ||X - Psi(G)||^2 = ||X||^2 - ||P||^2 + ||P - TR(Z)||^2
 * (Eq. 3 with orthonormal Q_n).  ||X||^2 is the value recorded by the plan's
 * last rtr_sketch; P and Z as given to rtr_als / rtr_svd (ranks NULL = plan R).
 * out: device float64[1].
 */
int rtr_rse(rtr_plan* plan, const void* P, const double* const* Z, const int* ranks,
            double* out, void* stream);

/*
 * Test support: write rows row0..row0+nrows-1 of Omega_n (K columns, float64
 * values of the table the plan's precision uses) to out (device, nrows x K).
 */
int rtr_draw_omega(rtr_plan* plan, int mode, int64_t row0, int64_t nrows, int K,
                   double* out, void* stream);

/* Test support: the Gaussian table of a precision as float64 values (host out[4096]). */
int rtr_gaussian_table(int prec, double* out);

/*
 * Test support for the device watchdog (no counterpart in the paper): one
 * thread waits, with the bounded mbarrier wait every tensor-core kernel of
 * the library uses, on a barrier that nothing completes, with a limit of
 * limit_us microseconds (1 .. 2e6) instead of the kernels' 2 s.  The wait
 * gives up, ORs RTR_FLAG_TIMEOUT into *flags (a caller-owned device int) and
 * the kernel returns normally, so the context stays usable.  Synchronises
 * `stream`; returns RTR_ETIMEOUT when the flag was raised, RTR_OK otherwise.
 */
int rtr_test_bounded_wait(int limit_us, int* flags, void* stream);

/*
 * Allocation-free sketch of one mode (the paper has no counterpart; this is a
 * deployment variant of rtr_sketch for callers that cannot call cudaMalloc,
 * e.g. code embedded in a framework that owns all device memory, or a
 * service that must not grow its device footprint after start-up).
 *     Y = X_(n) Omega_n     for X viewed as (A, I, B), i.e. I = I_n,
 *                           A = prod of the modes before n, B = after n
 * prec: RTR_FP64 (X float64) or RTR_FP32 (X float32, bfloat16-valued Omega).
 * seed, mode: the key (seed, n) of Omega_n, as in rtr_sketch.  X and Y
 * (I x K float64) are caller-owned device buffers; no plan is needed.
 * Scratch: a file-scope device array of 2^21 float64 (16 MiB) plus the two
 * Gaussian tables (48 KiB), held on every GPU that loads the library until
 * the process exits.  Requires I*K <= 2^21 and 1 <= K <= 64, else RTR_EINVAL.
 * The first call on a device performs set-up on the current device
 * (resolves the arrays' device addresses, copies the tables with synchronous
 * cudaMemcpy); make that first call before any stream capture.  It calls no
 * cudaMalloc/cudaFree.  Every call shares the one scratch array (each call
 * overwrites every partial it reads, so nothing needs clearing); calls that
 * overlap on the GPU (other streams, other threads) race on it.
 */
int rtr_sketch_mode_noalloc(int prec, const void* X, int64_t A, int64_t I, int64_t B, int K,
                            uint64_t seed, int mode, double* Y, void* stream);

/*
 * Batched form: Algorithm 1 (sketch, orthonormal bases, projection chain,
 * TR-ALS with the default start, back-projection, RSE) for `count` tensors of
 * uneven shapes, run as one unit.
 *
 * rtr_batch_create: count >= 1 tensors of the same order N.  dims, K, R are
 * HOST arrays of count*N entries (tensor t's entries at [t*N, t*N+N)), with
 * the meaning they have in rtr_plan_create.  params applies to every tensor
 * except the seed: tensor t uses seed params->seed + t (its own Omega_n and
 * start cores); params->chain_order must be all -1 (each tensor takes its
 * own default order).  nstreams (1..64): worker streams over which the
 * tensors are spread (tensor t on worker t % nstreams).  The batch owns one
 * plan and the step buffers (Y_n, Q_n, P, Z_n) per tensor.
 *
 * rtr_batch_run: X is a HOST array of count device pointers (tensor t:
 * float64 for RTR_FP64, float32 otherwise, row-major of its dims); G a HOST
 * array of count*N device float64 pointers (G[t*N+n]: R_n x I_n x R_{n+1});
 * rse (may be NULL) a device float64[count] for the RSE of Section 4 of each
 * tensor.  The first run with a given set of pointers executes eagerly
 * (the mode-product autotuner times tile variants for shape classes it has
 * not seen) and captures the same schedule into a CUDA graph; later runs
 * with the same pointers replay that graph with one launch (with
 * RTR_PARAM_NO_GRAPH in params->flags every run is eager and nothing is
 * captured, for one-shot batches).  Asynchronous on
 * `stream` (ordered after the work already on it), except that the first run
 * with new pointers synchronises once before capturing.  Runs of one batch
 * must not overlap in time.
 */
typedef struct rtr_batch rtr_batch;
int rtr_batch_create(rtr_batch** batch, int count, int N, const int64_t* dims, const int* K,
                     const int* R, const rtr_params* params, int nstreams);
int rtr_batch_destroy(rtr_batch* batch);
int rtr_batch_run(rtr_batch* batch, const void* const* X, double* const* G, double* rse, void* stream);
/* device flags (RTR_FLAG_*) raised by the batch's runs so far, ORed over its
 * tensors; synchronises the device and clears them */
int rtr_batch_flags(rtr_batch* batch, int* flags);
/* number of kernel launches in the batch's captured graph (0 before the first run) */
int rtr_batch_graph_kernels(const rtr_batch* batch, uint64_t* n);

/*
 * Learned proposer of the sketch sizes K_n and TR ranks R_n.  The paper sets
 * K_n and R_n by hand for each experiment (Section 4); this is the library's
 * own addition (it has no counterpart in the paper): a perceptron reads the
 * singular-value spectra of the sketches Y_n = X_(n) Omega_n (Algorithm 1,
 * step 5) and outputs (K_n, R_n) for up to 5 modes.
 *
 * Features (rtr_spectrum_features): for mode n < N, with s_0 >= s_1 >= ...
 * the singular values of Y_n (I_n x Kf_n float64 row-major, device; 1 <=
 * Kf_n <= 64), f[64 n + i] = max(0, 1 + log10(s_i / s_0) / 6) for
 * i < min(I_n, Kf_n), else 0; rows n in [N, 5) are 0.  f: device float[320]
 * (one feature row).  1 <= N <= 5.  The spectrum is taken from the
 * eigenvalues of the float64 Gram matrix Y_n^T Y_n.
 *
 * Network: 320 -> 128 -> 128 -> 128 -> 10 with GELU (x Phi(x)) after the
 * hidden layers.  theta: device float32[rtr_mlp_param_count()] =
 * [W1 (128 x 320 row-major), b1[128], W2 (128 x 128), b2, W3 (128 x 128), b3,
 * W4 (10 x 128), b4[10]] (float32 master weights).  Every matrix product
 * rounds both operands to bfloat16 and accumulates in float32 on the tensor
 * cores.  F: device float[batch x 320]; out: device float[batch x 10];
 * 1 <= batch <= 65536.  work: device scratch of rtr_mlp_work_bytes(batch)
 * bytes, owned by the caller; its first int holds status flags and must be
 * zero before the first call (rtr_mlp_status clears it).
 *
 * rtr_mlp_grad: loss = 0.5 * sum(M .* (out - T)^2) / sum(M) for targets T
 * and a 0/1 mask M (device float[batch x 10] each), written to *loss (device
 * double, may be NULL); grad (device float, theta's layout) = d loss / d theta
 * (no accumulation: overwritten).
 * rtr_mlp_adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at step
 * number `step` >= 1 on theta with moments m, v (device float, theta's
 * layout, zero before step 1).
 * rtr_mlp_status: synchronises the device, returns the work area's flags
 * (RTR_FLAG_TIMEOUT if a bounded wait of a product gave up) and clears them.
 * rtr_propose (host): out = one network output row (HOST float[10]) ->
 * K_n = clamp(round(64 out[2n]), 1, min(I_n, 64)), R_n = clamp(round(16
 * out[2n+1]), 1, r_max) for n < N (r_max <= 16), rounding half to even.
 */
size_t rtr_mlp_param_count(void);
size_t rtr_mlp_work_bytes(int batch);
int rtr_spectrum_features(int N, const int64_t* dims, const int* Kf, const double* const* Y, float* f,
                          void* stream);
int rtr_mlp_forward(const float* theta, const float* F, int batch, float* out, void* work, size_t work_bytes,
                    void* stream);
int rtr_mlp_grad(const float* theta, const float* F, const float* T, const float* M, int batch, float* grad,
                 double* loss, void* work, size_t work_bytes, void* stream);
int rtr_mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, void* stream);
int rtr_mlp_status(void* work, int* flags);
int rtr_propose(const float* out, int N, const int64_t* dims, int r_max, int* K, int* R);

#ifdef __cplusplus
}
#endif
#endif /* RTR_H */
