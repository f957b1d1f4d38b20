// C ABI of the rTRD library: plans, workspace, Gaussian tables, dispatch of
// Algorithm 1's steps to the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include "rtr_internal.cuh"

size_t contract_partial_elems(int num_sms, int64_t I, int C);
size_t contract_norm_elems(int num_sms, int64_t I, int C);
size_t orth_ws_elems(int num_sms, int64_t maxI);
size_t tc_ws_bytes(const rtr_plan* p);
size_t trsvd_ws_elems(int64_t pnumel, int64_t* cbuf, int64_t* gmax, int64_t* umax);

namespace {
thread_local char g_err[1024] = "";

// ---- Gaussian quantile table (library's own copy) ------------------------------
// T[j] = Phi^{-1}((j + 1/2) / 4096): lower half by bisection on
// Phi(x) = erfc(-x / sqrt 2) / 2 (accurate in relative terms for x < 0) with
// a Newton polish, upper half by the symmetry of N(0, 1).
double phi_lower(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

double inv_phi_lower(double p) {
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 2000; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (phi_lower(mid) < p) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 2; ++it) {
        const double f = phi_lower(x) - p;
        const double d = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
        x -= f / d;
    }
    return x;
}

void gaussian_table64(double* t) {
    for (int j = 0; j < 2048; ++j) {
        const double v = inv_phi_lower((j + 0.5) / 4096.0);
        t[j] = v;
        t[4095 - j] = -v;
    }
}

// round a double to 8 significant bits, ties to even, as a bfloat16 pattern
uint16_t bf16_bits(double x) {
    if (x == 0.0) return std::signbit(x) ? 0x8000 : 0;
    int e;
    const double m = std::frexp(x, &e);               // |m| in [0.5, 1)
    const double r = std::ldexp(std::nearbyint(std::ldexp(m, 8)), e - 8);
    const float f = (float)r;                          // exact
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}
// round a double to the nearest float8 e4m3 value: 4 significant bits, ties
// to even, spacing 2^-9 below the smallest normal 2^-6, saturated at 448
double e4m3_value(double x) {
    const double a = std::fabs(x);
    double q;
    if (a < 0.015625) {
        q = std::ldexp(std::nearbyint(std::ldexp(a, 9)), -9);
    } else {
        int e;
        const double m = std::frexp(a, &e);               // m in [0.5, 1)
        q = std::ldexp(std::nearbyint(std::ldexp(m, 4)), e - 4);
    }
    q = std::min(q, 448.0);
    return std::copysign(q, x);
}
float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int choose_order(rtr_plan* p) {
    const rtr_params& pr = p->params;
    bool given = true;
    for (int n = 0; n < p->N; ++n) if (pr.chain_order[n] < 0) given = false;
    if (given) {
        int seen[RTR_MAXN] = {};
        for (int n = 0; n < p->N; ++n) {
            const int m = pr.chain_order[n];
            if (m >= p->N || seen[m]) return rtr_set_error(RTR_EINVAL, "chain_order is not a permutation");
            seen[m] = 1;
            p->order[n] = m;
        }
        return RTR_OK;
    }
    // largest shrink first (smallest K_n / I_n); among equal ratios the last
    // mode first, then increasing mode order
    int idx[RTR_MAXN];
    for (int n = 0; n < p->N; ++n) idx[n] = n;
    const int last = p->N - 1;
    std::stable_sort(idx, idx + p->N, [&](int a, int b) {
        const double ra = (double)p->K[a] / (double)p->dims[a], rb = (double)p->K[b] / (double)p->dims[b];
        if (ra != rb) return ra < rb;
        if ((a == last) != (b == last)) return a == last;
        return a < b;
    });
    for (int n = 0; n < p->N; ++n) p->order[n] = idx[n];
    return RTR_OK;
}

void free_plan(rtr_plan* p) {
    if (!p) return;
    cudaFree(p->tab64); cudaFree(p->tab32); cudaFree(p->tab_bf16); cudaFree(p->tab_e4m3);
    cudaFree(p->partial); cudaFree(p->normx_part); cudaFree(p->scal);
    cudaFree(p->chain[0]); cudaFree(p->chain[1]);
    cudaFree(p->qr_ws); cudaFree(p->als_ws); cudaFree(p->sub_ws[0]);
    cudaFree(p->flags); cudaFree(p->tc_ws); cudaFree(p->svd_ws); cudaFree(p->ttm_q);
    cudaFree(p->pow_q); cudaFree(p->pow_t); cudaFree(p->acc_y);
    for (int e = 0; e < 6; ++e) if (p->ev[e]) cudaEventDestroy(p->ev[e]);
    if (p->als_exec) cudaGraphExecDestroy(p->als_exec);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->side2) cudaStreamDestroy(p->side2);
    delete p;
}

template <typename T>
int dalloc(T** ptr, size_t elems) {
    cudaError_t e = cudaMalloc((void**)ptr, std::max<size_t>(elems, 1) * sizeof(T));
    if (e != cudaSuccess) { cudaGetLastError(); return rtr_set_error(RTR_ENOMEM, "cudaMalloc(%zu B) failed: %s", elems * sizeof(T), cudaGetErrorString(e)); }
    return RTR_OK;
}
}  // namespace

int rtr_set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}
void rtr_host_tables(double* t64, float* t32) {
    gaussian_table64(t64);
    for (int j = 0; j < 4096; ++j) t32[j] = bf16_value(bf16_bits(t64[j]));
}

static std::atomic<unsigned long long> g_launches{0};
void rtr_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void rtr_count_launches(long long delta) { g_launches.fetch_add((unsigned long long)delta, std::memory_order_relaxed); }

int rtr_cuda_check(cudaError_t e, const char* what) {
    return rtr_set_error(RTR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static std::mutex g_smem_mu;
static std::map<std::pair<const void*, int>, size_t> g_smem_max;   // (kernel, device) -> dynamic limit

int rtr_smem_limit(const void* kernel, size_t bytes) {
    int dev = 0;
    RTR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_smem_mu);
    auto it = g_smem_max.find({kernel, dev});
    if (it == g_smem_max.end()) {
        int optin = 0;
        RTR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cudaFuncAttributes fa{};
        RTR_CUDA(cudaFuncGetAttributes(&fa, kernel));
        const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        RTR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
        it = g_smem_max.emplace(std::make_pair(kernel, dev), lim).first;
    }
    if (bytes > it->second)
        return rtr_set_error(RTR_EINVAL, "a kernel needs %zu B of dynamic shared memory, the device allows %zu",
                             bytes, it->second);
    return RTR_OK;
}

extern "C" {

const char* rtr_last_error(void) { return g_err; }

unsigned long long rtr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void rtr_params_default(rtr_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->prec = RTR_FP32;
    p->seed = 0;
    p->sweeps = 20;
    p->tol = 1e-2;
    for (int n = 0; n < 8; ++n) p->chain_order[n] = -1;
}

int rtr_gaussian_table(int prec, double* out) {
    if (!out) return rtr_set_error(RTR_EINVAL, "out is NULL");
    double t[4096];
    gaussian_table64(t);
    for (int j = 0; j < 4096; ++j) {
        if (prec == RTR_FP64) out[j] = t[j];
        else if (prec == RTR_FP32 || prec == RTR_BF16) out[j] = (double)bf16_value(bf16_bits(t[j]));
        else if (prec == RTR_FP8) out[j] = e4m3_value(t[j]);
        else return rtr_set_error(RTR_EINVAL, "unknown precision %d", prec);
    }
    return RTR_OK;
}

int rtr_plan_create(rtr_plan** plan, int N, const int64_t* dims, const int* K, const int* R,
                    const rtr_params* params) {
    if (!plan || !dims || !K || !R || !params) return rtr_set_error(RTR_EINVAL, "NULL argument");
    *plan = nullptr;
    if (N < 3 || N > RTR_MAXN) return rtr_set_error(RTR_EINVAL, "order N=%d outside [3, 8]", N);
    if (params->prec != RTR_FP64 && params->prec != RTR_FP32 && params->prec != RTR_BF16 &&
        params->prec != RTR_FP8)
        return rtr_set_error(RTR_EINVAL, "unknown precision %d", params->prec);
    if (params->sweeps < 0) return rtr_set_error(RTR_EINVAL, "sweeps < 0");
    if (params->power_iters < 0 || params->power_iters > 16)
        return rtr_set_error(RTR_EINVAL, "power_iters = %d outside [0, 16]", params->power_iters);
    rtr_plan* p = new (std::nothrow) rtr_plan();
    if (!p) return rtr_set_error(RTR_ENOMEM, "host allocation failed");
    p->N = N;
    p->params = *params;
    p->numel = 1;
    p->pnumel = 1;
    for (int n = 0; n < N; ++n) {
        if (dims[n] < 1) { delete p; return rtr_set_error(RTR_EINVAL, "dims[%d] = %lld < 1", n, (long long)dims[n]); }
        if (K[n] < 1) { delete p; return rtr_set_error(RTR_EINVAL, "K[%d] = %d < 1", n, K[n]); }
        if (R[n] < 1 || R[n] > RTR_MAX_RANK) { delete p; return rtr_set_error(RTR_EINVAL, "R[%d] = %d outside [1, 16]", n, R[n]); }
        p->dims[n] = dims[n];
        p->Kreq[n] = K[n];
        p->proj[n] = (int64_t)K[n] < dims[n];
        p->K[n] = p->proj[n] ? K[n] : (int)std::min<int64_t>(dims[n], 1 << 30);
        if (p->proj[n] && K[n] > RTR_MAX_KSKETCH) { delete p; return rtr_set_error(RTR_EINVAL, "K[%d] = %d > 64", n, K[n]); }
        if (!p->proj[n] && dims[n] > 4096) { delete p; return rtr_set_error(RTR_EINVAL, "unprojected mode %d longer than 4096", n); }
        p->R[n] = R[n];
        p->numel *= dims[n];
        p->pnumel *= p->K[n];
    }
    int st = choose_order(p);
    if (st) { delete p; return st; }
    cudaError_t ce = cudaGetDevice(&p->device);
    if (ce != cudaSuccess) { delete p; return rtr_cuda_check(ce, "cudaGetDevice"); }
    ce = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (ce != cudaSuccess) { delete p; return rtr_cuda_check(ce, "cudaDeviceGetAttribute"); }
    const bool f64 = params->prec == RTR_FP64;
    const size_t esz = f64 ? 8 : 4;

    // ---- workspace sizes
    size_t part = 1024, normp = 1024;
    int64_t maxI = 1, maxJ = 1;
    int maxR = 1;
    for (int n = 0; n < N; ++n) {
        maxR = std::max(maxR, R[n]);
        if (p->proj[n]) {
            part = std::max(part, contract_partial_elems(p->num_sms, dims[n], p->K[n]));
            normp = std::max(normp, contract_norm_elems(p->num_sms, dims[n], p->K[n]));
            maxI = std::max<int64_t>(maxI, dims[n]);
        }
        // the BF16 sketch of the last two modes in one pass (mode N-2 partials
        // per CTA column, mode N-1 partials per CTA)
        if (n == N - 1 && N >= 3 && p->params.prec == RTR_BF16 && p->proj[N - 2] && p->proj[N - 1])
            part = std::max(part, pair_partial_elems(p->num_sms, dims[N - 2], p->K[N - 2], dims[N - 1], p->K[N - 1]));
        const int C = R[n] * R[(n + 1) % N];
        part = std::max(part, contract_partial_elems(p->num_sms, p->K[n], C));
        maxJ = std::max<int64_t>(maxJ, p->pnumel / p->K[n]);
    }
    // chain intermediates (ping-pong); the last product goes straight to P
    int64_t cdims[RTR_MAXN];
    for (int n = 0; n < N; ++n) cdims[n] = dims[n];
    int nsteps = 0;
    for (int s = 0; s < N; ++s) if (p->proj[p->order[s]]) ++nsteps;
    size_t chain_elems[2] = {0, 0};
    int step = 0;
    for (int s = 0; s < N; ++s) {
        const int n = p->order[s];
        if (!p->proj[n]) continue;
        cdims[n] = p->K[n];
        int64_t sz = 1;
        for (int m = 0; m < N; ++m) sz *= cdims[m];
        if (step < nsteps - 1) chain_elems[step & 1] = std::max<size_t>(chain_elems[step & 1], (size_t)sz);
        ++step;
    }
    size_t chain_bytes0 = std::max(chain_elems[0] * esz, (size_t)p->pnumel * 8);
    size_t chain_bytes1 = chain_elems[1] * esz;
    // subchain buffers (>= J x R^2 per level) and reconstruct work for rtr_rse
    size_t sub_bytes = esz * (size_t)maxJ * (size_t)(maxR * maxR);
    int64_t kd[RTR_MAXN];
    for (int n = 0; n < N; ++n) kd[n] = p->K[n];
    sub_bytes = std::max(sub_bytes, (reconstruct_work_bytes(N, kd, R) + 1) / 2);
    sub_bytes = (sub_bytes + 255) & ~(size_t)255;

    // ---- allocations
    double t64[4096];
    gaussian_table64(t64);
    float t32[4096];
    uint16_t tb[4096], t8[4096];
    for (int j = 0; j < 4096; ++j) {
        tb[j] = bf16_bits(t64[j]);
        t32[j] = bf16_value(tb[j]);
        t8[j] = bf16_bits(e4m3_value(t64[j]));     // exact: 4 significant bits
    }
#define RTR_TRY(x) do { int s_ = (x); if (s_) { free_plan(p); return s_; } } while (0)
#define RTR_TRYC(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { free_plan(p); return rtr_cuda_check(e_, #x); } } while (0)
    RTR_TRY(dalloc(&p->tab64, 4096));
    RTR_TRY(dalloc(&p->tab32, 4096));
    RTR_TRY(dalloc(&p->tab_bf16, 4096));
    RTR_TRYC(cudaMemcpy(p->tab64, t64, sizeof(t64), cudaMemcpyHostToDevice));
    RTR_TRYC(cudaMemcpy(p->tab32, t32, sizeof(t32), cudaMemcpyHostToDevice));
    RTR_TRYC(cudaMemcpy(p->tab_bf16, tb, sizeof(tb), cudaMemcpyHostToDevice));
    if (params->prec == RTR_FP8) {
        RTR_TRY(dalloc(&p->tab_e4m3, 4096));
        RTR_TRYC(cudaMemcpy(p->tab_e4m3, t8, sizeof(t8), cudaMemcpyHostToDevice));
    }
    RTR_TRY(dalloc(&p->partial, part)); p->partial_elems = part;
    RTR_TRY(dalloc(&p->normx_part, normp)); p->normx_part_elems = normp;
    RTR_TRY(dalloc(&p->scal, 64));
    RTR_TRYC(cudaMemset(p->scal, 0, 64 * sizeof(double)));
    {
        char* c0 = nullptr;
        char* c1 = nullptr;
        RTR_TRY(dalloc(&c0, chain_bytes0)); p->chain[0] = c0; p->chain_bytes[0] = chain_bytes0;
        RTR_TRY(dalloc(&c1, std::max<size_t>(chain_bytes1, 256))); p->chain[1] = c1; p->chain_bytes[1] = chain_bytes1;
    }
    p->qr_ws_elems = orth_ws_elems(p->num_sms, maxI);
    RTR_TRY(dalloc(&p->qr_ws, p->qr_ws_elems));
    p->als_wmax = 0;
    for (int n = 0; n < N; ++n)
        p->als_wmax = std::max<size_t>(p->als_wmax, (size_t)p->K[n] * R[n] * R[(n + 1) % N]);
    int64_t maxK = 1, core_elems = 0;
    for (int n = 0; n < N; ++n) {
        maxK = std::max<int64_t>(maxK, p->K[n]);
        core_elems += (((int64_t)R[n] * p->K[n] * R[(n + 1) % N]) + 3) & ~(int64_t)3;
    }
    p->als_maxK = (size_t)maxK;
    p->als_ws_elems = (size_t)(RTR_MAXN + 4) * 256 * 256 + 2 * p->als_wmax + 2 * 144 * 144 + (size_t)maxK +
                      (size_t)(core_elems / 2 + 8);   // float32 core shadows
    RTR_TRY(dalloc(&p->als_ws, p->als_ws_elems));
    {
        char* sb = nullptr;
        RTR_TRY(dalloc(&sb, 2 * sub_bytes));
        p->sub_ws[0] = sb; p->sub_ws[1] = sb + sub_bytes; p->sub_bytes = sub_bytes;
    }
    RTR_TRYC(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    RTR_TRYC(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    RTR_TRYC(cudaStreamCreateWithFlags(&p->side2, cudaStreamNonBlocking));
    for (int e = 0; e < 6; ++e) RTR_TRYC(cudaEventCreateWithFlags(&p->ev[e], cudaEventDisableTiming));
    RTR_TRY(dalloc(&p->flags, 4));
    RTR_TRYC(cudaMemset(p->flags, 0, 4 * sizeof(int)));
    RTR_TRY(dalloc(&p->svd_ws, trsvd_ws_elems(p->pnumel, &p->svd_cbuf, &p->svd_gmax, &p->svd_umax)));
    {
        // mode-product Q converted to the compute type: I_n rows of at most 64 values
        char* q = nullptr;
        p->ttm_q_bytes = (size_t)maxI * 64 * esz;
        RTR_TRY(dalloc(&q, p->ttm_q_bytes));
        p->ttm_q = q;
    }
    RTR_TRY(dalloc(&p->acc_y, (size_t)maxI * 64));
    if (params->power_iters > 0) {
        // Q of one mode and T = X x_n Q^T for the largest K_n / I_n
        size_t tmax = 1;
        for (int n = 0; n < N; ++n)
            if (p->proj[n]) tmax = std::max<size_t>(tmax, (size_t)(p->numel / dims[n]) * (size_t)p->K[n]);
        RTR_TRY(dalloc(&p->pow_q, (size_t)maxI * 64));
        char* t = nullptr;
        p->pow_t_bytes = tmax * esz;
        RTR_TRY(dalloc(&t, p->pow_t_bytes));
        p->pow_t = t;
    }
    p->tc_ws_bytes = tc_ws_bytes(p);
    if (p->tc_ws_bytes) {
        char* t = nullptr;
        RTR_TRY(dalloc(&t, p->tc_ws_bytes));
        p->tc_ws = t;
    }
#undef RTR_TRY
#undef RTR_TRYC
    *plan = p;
    return RTR_OK;
}

int rtr_plan_destroy(rtr_plan* plan) {
    free_plan(plan);
    return RTR_OK;
}

int rtr_plan_info(const rtr_plan* p, int* K_eff, int* chain_order) {
    if (!p) return rtr_set_error(RTR_EINVAL, "plan is NULL");
    for (int n = 0; n < p->N; ++n) {
        if (K_eff) K_eff[n] = p->K[n];
        if (chain_order) chain_order[n] = p->order[n];
    }
    return RTR_OK;
}

int rtr_plan_sketch_passes(const rtr_plan* p, int* passes) {
    if (!p || !passes) return rtr_set_error(RTR_EINVAL, "NULL argument");
    *passes = sketch_passes(p);
    return RTR_OK;
}

int rtr_plan_flags(rtr_plan* p, int* flags) {
    if (!p || !flags) return rtr_set_error(RTR_EINVAL, "NULL argument");
    RTR_CUDA(cudaDeviceSynchronize());
    RTR_CUDA(cudaMemcpy(flags, p->flags, sizeof(int), cudaMemcpyDeviceToHost));
    RTR_CUDA(cudaMemset(p->flags, 0, sizeof(int)));
    return RTR_OK;
}

namespace {

// Power iterations of rtr_sketch: q times, for every projected mode,
// Q = orth(Y_n); T = X x_n Q^T (A x K x B); Y_n = X_(n) T_(n)^T.
int power_iterations(rtr_plan* p, const void* X, double* const* Y, cudaStream_t s) {
    const int f64 = p->params.prec == RTR_FP64;
    const bool tc = p->params.prec == RTR_BF16 || p->params.prec == RTR_FP8;
    for (int it = 0; it < p->params.power_iters; ++it) {
        for (int n = 0; n < p->N; ++n) {
            if (!p->proj[n]) continue;
            int64_t A, I, B;
            rtr_mode_view(p->N, p->dims, n, &A, &I, &B);
            const int K = p->K[n];
            if ((size_t)(A * B) * (size_t)K * (f64 ? 8 : 4) > p->pow_t_bytes)
                return rtr_set_error(RTR_ENOMEM, "power iteration buffer too small");
            const double* Yarr[RTR_MAXN] = {};
            double* Qarr[RTR_MAXN] = {};
            Yarr[n] = Y[n];
            Qarr[n] = p->pow_q;
            int st = launch_orth_mask(p, Yarr, Qarr, 1u << n, s);
            if (st) return st;
            st = tc ? launch_ttm_tc(p, (const float*)X, A, I, B, p->pow_q, K, (float*)p->pow_t, s)
                    : launch_ttm(p, f64, X, A, I, B, p->pow_q, K, p->pow_t, s);
            if (st) return st;
            ContractArgs a{};
            a.X = X; a.A = A; a.I = I; a.B = B; a.C = K;
            a.gen = 0; a.M = p->pow_t; a.ldm = K; a.makb = 1;
            a.Y = Y[n]; a.norm_out = nullptr;
            if ((st = launch_contract(p, f64, a, s))) return st;
        }
    }
    return RTR_OK;
}

}  // namespace

int rtr_sketch(rtr_plan* p, const void* X, double* const* Y, void* stream) {
    if (!p || !X || !Y) return rtr_set_error(RTR_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int n = 0; n < p->N; ++n)
        if (p->proj[n] && !Y[n]) return rtr_set_error(RTR_EINVAL, "Y[%d] is NULL", n);
    int st = RTR_OK;
    if (p->params.prec == RTR_BF16 || p->params.prec == RTR_FP8) {
        st = launch_sketch_tc(p, (const float*)X, Y, s);
    } else {
        const int f64 = p->params.prec == RTR_FP64;
        bool norm_done = false;
        for (int n = 0; n < p->N; ++n) {
            if (!p->proj[n]) continue;
            ContractArgs a{};
            int64_t A, I, B;
            rtr_mode_view(p->N, p->dims, n, &A, &I, &B);
            a.X = X; a.A = A; a.I = I; a.B = B; a.C = p->K[n];
            a.gen = 1; a.seed = p->params.seed; a.mode = n;
            a.table = f64 ? (const void*)p->tab64 : (const void*)p->tab32;
            a.Y = Y[n];
            a.norm_out = norm_done ? nullptr : p->scal + 0;
            st = launch_contract(p, f64, a, s);
            if (st) return st;
            norm_done = true;
        }
        if (!norm_done) st = launch_sumsq(X, f64, p->numel, p->partial, 1024, p->scal + 0, p->flags, s);
    }
    if (st) return st;
    if (p->params.power_iters > 0) return power_iterations(p, X, Y, s);
    return RTR_OK;
}

int rtr_project_sequential(rtr_plan* p, const void* X, double* const* Y, double* const* Q, void* P, void* stream) {
    if (!p || !X || !Y || !Q || !P) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (p->params.power_iters != 0)
        return rtr_set_error(RTR_EINVAL, "the sequential projection takes no power iterations");
    cudaStream_t s = (cudaStream_t)stream;
    const int f64 = p->params.prec == RTR_FP64;
    const bool tc = p->params.prec == RTR_BF16 || p->params.prec == RTR_FP8;
    const size_t esz = f64 ? 8 : 4;
    unsigned keep = 0;
    for (int n = 0; n < p->N; ++n) {
        if (!Q[n]) return rtr_set_error(RTR_EINVAL, "Q[%d] is NULL", n);
        if (p->proj[n] && !Y[n]) return rtr_set_error(RTR_EINVAL, "Y[%d] is NULL", n);
        if (!p->proj[n]) keep |= 1u << n;
    }
    int st = RTR_OK;
    if (keep && (st = launch_orth_mask(p, Y, Q, keep, s))) return st;       // Q_n = I
    int64_t cd[RTR_MAXN];
    for (int n = 0; n < p->N; ++n) cd[n] = p->dims[n];
    int nsteps = 0;
    for (int i = 0; i < p->N; ++i) if (p->proj[p->order[i]]) ++nsteps;
    if (nsteps == 0) {
        RTR_CUDA(cudaMemcpyAsync(P, X, (size_t)p->numel * esz, cudaMemcpyDeviceToDevice, s));
        return launch_sumsq(X, f64, p->numel, p->partial, 1024, p->scal + 0, p->flags, s);
    }
    const void* cur = X;
    int step = 0;
    for (int i = 0; i < p->N; ++i) {
        const int n = p->order[i];
        if (!p->proj[n]) continue;
        int64_t A, I, B;
        rtr_mode_view(p->N, cd, n, &A, &I, &B);
        // the first sketch reads X itself and records ||X||^2
        double* norm = step == 0 ? p->scal + 0 : nullptr;
        if (tc) {
            st = launch_sketch_tc_mode(p, (const float*)cur, A, I, B, n, Y[n], norm, s, 0);
        } else {
            ContractArgs a{};
            a.X = cur; a.A = A; a.I = I; a.B = B; a.C = p->K[n];
            a.gen = 1; a.seed = p->params.seed; a.mode = n;
            a.table = f64 ? (const void*)p->tab64 : (const void*)p->tab32;
            a.Y = Y[n]; a.norm_out = norm;
            st = launch_contract(p, f64, a, s);
        }
        if (st) return st;
        if ((st = launch_orth_mask(p, Y, Q, 1u << n, s))) return st;
        void* out = (step == nsteps - 1) ? P : p->chain[step & 1];
        if (tc && step == 0) st = launch_ttm_tc(p, (const float*)cur, A, I, B, Q[n], p->K[n], (float*)out, s);
        else st = launch_ttm(p, f64, cur, A, I, B, Q[n], p->K[n], out, s);
        if (st) return st;
        cd[n] = p->K[n];
        cur = out;
        ++step;
    }
    return RTR_OK;
}

namespace {

// H2D copy of slab `sl` (rows r0 .. r0 + rows - 1 of mode 0) into its stage
// buffer on the plan's side stream, after the compute that last read that
// buffer; the caller's stream waits for the copy.
int stage_in(rtr_plan* p, const void* X_host, int64_t r0, int64_t rows, int64_t row_elems, size_t esz, int64_t sl,
             void* const* stage, cudaStream_t s) {
    const int b = sl & 1;
    cudaEvent_t copied = p->ev[b], done = p->ev[2 + b];
    if (sl >= 2) RTR_CUDA(cudaStreamWaitEvent(p->side, done, 0));
    RTR_CUDA(cudaMemcpyAsync(stage[b], static_cast<const char*>(X_host) + (size_t)(r0 * row_elems) * esz,
                             (size_t)(rows * row_elems) * esz, cudaMemcpyHostToDevice, p->side));
    RTR_CUDA(cudaEventRecord(copied, p->side));
    RTR_CUDA(cudaStreamWaitEvent(s, copied, 0));
    return RTR_OK;
}

}  // namespace

int rtr_project_host(rtr_plan* p, const void* X_host, int64_t slab_rows, void* const* stage, size_t stage_bytes,
                     double* const* Y, double* const* Q, void* P, void* stream) {
    if (!p || !X_host || !stage || !stage[0] || !stage[1] || !Y || !Q || !P)
        return rtr_set_error(RTR_EINVAL, "NULL argument");
    const int N = p->N;
    if (slab_rows < 1 || slab_rows > p->dims[0])
        return rtr_set_error(RTR_EINVAL, "slab_rows = %lld outside [1, %lld]", (long long)slab_rows,
                             (long long)p->dims[0]);
    if (p->order[N - 1] != 0)
        return rtr_set_error(RTR_EINVAL, "rtr_project_host needs a plan whose chain order ends with mode 0");
    if (p->params.power_iters != 0) return rtr_set_error(RTR_EINVAL, "rtr_project_host takes no power iterations");
    for (int n = 0; n < N; ++n) {
        if (!Q[n]) return rtr_set_error(RTR_EINVAL, "Q[%d] is NULL", n);
        if (p->proj[n] && !Y[n]) return rtr_set_error(RTR_EINVAL, "Y[%d] is NULL", n);
    }
    const int f64 = p->params.prec == RTR_FP64;
    const bool tc = p->params.prec == RTR_BF16 || p->params.prec == RTR_FP8;
    const size_t esz = f64 ? 8 : 4;
    const int64_t row_elems = p->numel / p->dims[0];
    if (stage_bytes < (size_t)(slab_rows * row_elems) * esz)
        return rtr_set_error(RTR_EINVAL, "stage buffers of %zu B hold fewer than slab_rows = %lld rows", stage_bytes,
                             (long long)slab_rows);
    const int64_t nslabs = rtr_ceil_div(p->dims[0], slab_rows);
    if (p->params.prec == RTR_FP8 && p->proj[N - 1] && nslabs > 1) {
        // the last mode's float8 scale blocks run along a: a slab must hold whole blocks
        int64_t mid = 1;
        for (int m = 1; m < N - 1; ++m) mid *= p->dims[m];
        if ((slab_rows * mid) % 32 != 0)
            return rtr_set_error(RTR_EUNSUPPORTED, "FP8: slab_rows x prod(I_1..I_{N-2}) must be a multiple of 32");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the copies start after the work already queued on the caller's stream
    RTR_CUDA(cudaEventRecord(p->ev[2], s));
    RTR_CUDA(cudaStreamWaitEvent(p->side, p->ev[2], 0));
    int st = RTR_OK;
    for (int n = 1; n < N; ++n)
        if (p->proj[n]) RTR_CUDA(cudaMemsetAsync(Y[n], 0, (size_t)p->dims[n] * p->K[n] * sizeof(double), s));
    RTR_CUDA(cudaMemsetAsync(p->scal + 0, 0, sizeof(double), s));

    // ---- pass 1: sketches, slab by slab
    for (int64_t sl = 0; sl < nslabs; ++sl) {
        const int64_t r0 = sl * slab_rows, rows = std::min<int64_t>(slab_rows, p->dims[0] - r0);
        void* buf = stage[sl & 1];
        if ((st = stage_in(p, X_host, r0, rows, row_elems, esz, sl, stage, s))) return st;
        int64_t sd[RTR_MAXN];
        for (int n = 0; n < N; ++n) sd[n] = p->dims[n];
        sd[0] = rows;
        bool norm_done = false;
        for (int n = 0; n < N; ++n) {
            if (!p->proj[n]) continue;
            int64_t A, I, B;
            rtr_mode_view(N, sd, n, &A, &I, &B);
            // mode 0: this slab's rows of Y_0 are whole; other modes: this
            // slab's part of the sum, the test matrix rows counted globally
            const int64_t aoff = n == 0 ? 0 : r0 * (A / rows);
            double* ydst = n == 0 ? Y[0] + r0 * p->K[0] : p->acc_y;
            double* norm = norm_done ? nullptr : p->scal + 2;
            if (tc) {
                st = launch_sketch_tc_mode(p, (const float*)buf, A, I, B, n, ydst, norm, s, aoff);
            } else {
                ContractArgs a{};
                a.X = buf; a.A = A; a.I = I; a.B = B; a.C = p->K[n];
                a.gen = 1; a.seed = p->params.seed; a.mode = n; a.aoff = aoff;
                a.table = f64 ? (const void*)p->tab64 : (const void*)p->tab32;
                a.Y = ydst; a.norm_out = norm;
                st = launch_contract(p, f64, a, s);
            }
            if (st) return st;
            if (n > 0 && (st = launch_add(Y[n], p->acc_y, I * p->K[n], 1, s))) return st;
            if (!norm_done) {
                if ((st = launch_add(p->scal + 0, p->scal + 2, 1, 1, s))) return st;
                norm_done = true;
            }
        }
        if (!norm_done) {
            if ((st = launch_sumsq(buf, f64, rows * row_elems, p->partial, 1024, p->scal + 2, p->flags, s))) return st;
            if ((st = launch_add(p->scal + 0, p->scal + 2, 1, 1, s))) return st;
        }
        RTR_CUDA(cudaEventRecord(p->ev[2 + (sl & 1)], s));
    }
    if ((st = launch_orth(p, Y, Q, s))) return st;

    // ---- pass 2: every product but mode 0's per slab, then the slab's rows of
    // the mode-0 product added into P
    if (p->proj[0]) RTR_CUDA(cudaMemsetAsync(P, 0, (size_t)p->pnumel * esz, s));
    int64_t prest = 1;
    for (int n = 1; n < N; ++n) prest *= p->K[n];
    for (int64_t sl = 0; sl < nslabs; ++sl) {
        const int64_t r0 = sl * slab_rows, rows = std::min<int64_t>(slab_rows, p->dims[0] - r0);
        const int64_t gsl = nslabs + sl;          // copies so far: pass 1 used nslabs
        void* buf = stage[gsl & 1];
        if ((st = stage_in(p, X_host, r0, rows, row_elems, esz, gsl, stage, s))) return st;
        int64_t cd[RTR_MAXN];
        for (int n = 0; n < N; ++n) cd[n] = p->dims[n];
        cd[0] = rows;
        const void* cur = buf;
        int step = 0;
        for (int i = 0; i < N - 1; ++i) {
            const int n = p->order[i];
            if (!p->proj[n]) continue;
            int64_t A, I, B;
            rtr_mode_view(N, cd, n, &A, &I, &B);
            void* out = p->chain[step & 1];
            st = (tc && step == 0) ? launch_ttm_tc(p, (const float*)cur, A, I, B, Q[n], p->K[n], (float*)out, s)
                                   : launch_ttm(p, f64, cur, A, I, B, Q[n], p->K[n], out, s);
            if (st) return st;
            cd[n] = p->K[n];
            cur = out;
            ++step;
        }
        if (p->proj[0]) {
            // the stage buffer is free once the first product has read it
            void* tmp = step == 0 ? p->chain[0] : buf;
            const size_t cap = step == 0 ? p->chain_bytes[0] : stage_bytes;
            if ((size_t)p->pnumel * esz > cap) return rtr_set_error(RTR_ENOMEM, "P does not fit the slab buffers");
            if ((st = launch_ttm(p, f64, cur, 1, rows, prest, Q[0] + r0 * p->K[0], p->K[0], tmp, s))) return st;
            if ((st = launch_add(P, tmp, p->pnumel, f64, s))) return st;
        } else {
            // mode 0 kept whole: this slab's rows of P are the intermediate
            RTR_CUDA(cudaMemcpyAsync(static_cast<char*>(P) + (size_t)(r0 * prest) * esz, cur,
                                     (size_t)(rows * prest) * esz, cudaMemcpyDeviceToDevice, s));
        }
        RTR_CUDA(cudaEventRecord(p->ev[2 + (gsl & 1)], s));
    }
    return RTR_OK;
}

int rtr_project(rtr_plan* p, const void* X, const double* const* Y, double* const* Q, void* P, void* stream) {
    if (!p || !X || !Y || !Q || !P) return rtr_set_error(RTR_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int st = launch_orth(p, Y, Q, s);
    if (st) return st;
    const int f64 = p->params.prec == RTR_FP64;
    const size_t esz = f64 ? 8 : 4;
    int64_t cd[RTR_MAXN];
    for (int n = 0; n < p->N; ++n) cd[n] = p->dims[n];
    int nsteps = 0;
    for (int i = 0; i < p->N; ++i) if (p->proj[p->order[i]]) ++nsteps;
    if (nsteps == 0) {
        RTR_CUDA(cudaMemcpyAsync(P, X, (size_t)p->numel * esz, cudaMemcpyDeviceToDevice, s));
        return RTR_OK;
    }
    const void* cur = X;
    int step = 0;
    for (int i = 0; i < p->N; ++i) {
        const int n = p->order[i];
        if (!p->proj[n]) continue;
        int64_t A, I, B;
        rtr_mode_view(p->N, cd, n, &A, &I, &B);
        void* out = (step == nsteps - 1) ? P : p->chain[step & 1];
        if ((p->params.prec == RTR_BF16 || p->params.prec == RTR_FP8) && step == 0)
            st = launch_ttm_tc(p, (const float*)cur, A, I, B, Q[n], p->K[n], (float*)out, s);
        else
            st = launch_ttm(p, f64, cur, A, I, B, Q[n], p->K[n], out, s);
        if (st) return st;
        cd[n] = p->K[n];
        cur = out;
        ++step;
    }
    return RTR_OK;
}

int rtr_als(rtr_plan* p, const void* P, double* const* Z, int init_given, double* err, void* stream) {
    if (!p || !P || !Z) return rtr_set_error(RTR_EINVAL, "NULL argument");
    for (int n = 0; n < p->N; ++n) if (!Z[n]) return rtr_set_error(RTR_EINVAL, "Z[%d] is NULL", n);
    return run_als(p, P, Z, init_given, err, (cudaStream_t)stream);
}

int rtr_svd(rtr_plan* p, const void* P, double tol, double* const* Z, int* ranks, void* stream) {
    if (!p || !P || !Z || !ranks) return rtr_set_error(RTR_EINVAL, "NULL argument");
    return run_trsvd(p, P, tol, Z, ranks, (cudaStream_t)stream);
}

int rtr_backproject(rtr_plan* p, const double* const* Z, const double* const* Q, double* const* G, const int* ranks,
                    void* stream) {
    if (!p || !Z || !Q || !G) return rtr_set_error(RTR_EINVAL, "NULL argument");
    return run_backproject(p, Z, Q, G, ranks, (cudaStream_t)stream);
}

size_t rtr_reconstruct_work_bytes(int N, const int64_t* dims, const int* R) {
    if (N < 2 || N > RTR_MAXN || !dims || !R) return 0;
    return reconstruct_work_bytes(N, dims, R);
}

int rtr_reconstruct(int N, const int64_t* dims, const int* R, const double* const* G, int out_prec, void* Xhat,
                    void* work, size_t work_bytes, void* stream) {
    if (N < 2 || N > RTR_MAXN) return rtr_set_error(RTR_EINVAL, "order N=%d outside [2, 8]", N);
    if (!dims || !R || !G || !Xhat || !work) return rtr_set_error(RTR_EINVAL, "NULL argument");
    for (int n = 0; n < N; ++n) {
        if (!G[n]) return rtr_set_error(RTR_EINVAL, "G[%d] is NULL", n);
        if (dims[n] < 1 || R[n] < 1 || R[n] > RTR_MAX_RANK) return rtr_set_error(RTR_EINVAL, "bad dims/R at mode %d", n);
    }
    if (out_prec != RTR_FP64 && out_prec != RTR_FP32) return rtr_set_error(RTR_EINVAL, "out_prec must be FP64 or FP32");
    return run_reconstruct(N, dims, R, G, out_prec, Xhat, work, work_bytes, (cudaStream_t)stream);
}

int rtr_rse(rtr_plan* p, const void* P, const double* const* Z, const int* ranks, double* out, void* stream) {
    if (!p || !P || !Z || !out) return rtr_set_error(RTR_EINVAL, "NULL argument");
    return run_rse(p, P, Z, ranks, out, (cudaStream_t)stream);
}

int rtr_draw_omega(rtr_plan* p, int mode, int64_t row0, int64_t nrows, int K, double* out, void* stream) {
    if (!p || !out) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (mode < 0 || mode >= p->N || row0 < 0 || nrows < 0 || K < 1) return rtr_set_error(RTR_EINVAL, "bad range");
    return run_draw_omega(p, mode, row0, nrows, K, out, (cudaStream_t)stream);
}

}  // extern "C"
