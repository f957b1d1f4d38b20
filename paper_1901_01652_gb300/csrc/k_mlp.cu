// Learned proposer of K_n and R_n: spectrum features of the sketches Y_n,
// a 320-128-128-128-10 GELU perceptron (forward, gradient, Adam) and the
// decoding of its output.  The paper fixes K_n and R_n by hand (Section 4);
// the proposer is this library's own addition, defined in rtr.h.
//
// Every matrix product of the network runs on the 5th-generation tensor
// cores: operands rounded to bfloat16 while they are staged into shared
// memory (128-byte swizzle, K-major), tcgen05.mma with float32 accumulation
// in tensor memory, and a fused epilogue (bias, GELU, GELU derivative).
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>
#include "dense.cuh"
#include "tc_common.cuh"

using namespace rtr::tc;

namespace {

constexpr int IN = 320, HID = 128, OUT = 10, SPEC = 64, MODES = 5;
constexpr int GT = 128;                       // GEMM threads (4 warps)
constexpr int A_BYTES = 128 * 128;            // 128 rows x 64 bf16
constexpr size_t PCOUNT = (size_t)HID * IN + HID + 2 * ((size_t)HID * HID + HID) + (size_t)OUT * HID + OUT;
constexpr size_t WORK_HEADER = 256;           // bytes: int status flags at offset 0

enum Epi { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

struct GemmArgs {
    // C[m, n] = sum_k A(m, k) B(n, k); A(m, k) = A[m * a_rs + k * a_ks], same for B
    const float* A; int64_t a_rs, a_ks;
    const float* B; int64_t b_rs, b_ks;
    int M, N, K, Np;
    int epi;
    const float* bias;                        // [N]
    const float* aux; int64_t aux_ld;         // GELU-backward: pre-activation Z[m * aux_ld + n]
    float* out0; int64_t c_rs, c_cs;          // C[m, n] -> out0[m * c_rs + n * c_cs]
    float* out1;                              // GELU forward: activation, same layout as out0
    int* flags;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ uint32_t pack_bf16(float x0, float x1) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Stage rows [r0, r0 + rows_tile) x k in [k0, k0 + 64) of a strided operand
// into a SW128 K-major bf16 tile (zero outside [0, nrows) x [0, K)).
__device__ __forceinline__ void stage_operand(uint32_t dst, const float* __restrict__ src, int64_t rs, int64_t ks,
                                              int r0, int nrows, int rows_tile, int k0, int K) {
    const int pairs = rows_tile * 32;
    for (int e = threadIdx.x; e < pairs; e += GT) {
        int r, kp;
        if (ks == 1) { r = e >> 5; kp = e & 31; }          // k fastest: coalesced along k
        else { r = e % rows_tile; kp = e / rows_tile; }    // rows fastest: coalesced along rows
        const int gr = r0 + r, k = k0 + 2 * kp;
        float x0 = 0.f, x1 = 0.f;
        if (gr < nrows) {
            const float* p = src + (int64_t)gr * rs;
            if (k < K) x0 = p[(int64_t)k * ks];
            if (k + 1 < K) x1 = p[(int64_t)(k + 1) * ks];
        }
        st_shared_u32(dst + sw128_off((uint32_t)r, (uint32_t)(2 * kp)), pack_bf16(x0, x1));
    }
}

__global__ void __launch_bounds__(GT) mlp_gemm_kernel(const GemmArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* sm = smem_raw + pad;
    const uint32_t b_bytes = (uint32_t)p.Np * 128u;
    const uint32_t stage_bytes = A_BYTES + ((b_bytes + 1023u) & ~1023u);
    const uint32_t base = smem_u32(sm);
    uint64_t* done = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)p.Np) ncols <<= 1;

    if (tid == 0) {
        mbar_init(&done[0], 1);
        mbar_init(&done[1], 1);
        *abort = 0;
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int m0 = blockIdx.x * 128;
    const int nchunks = (p.K + 63) / 64;
    const uint32_t idesc = idesc_bf16_f32(128, p.Np);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (c >= 2 && !mbar_wait(&done[s], (uint32_t)(((c - 2) >> 1) & 1), abort, p.flags)) { ok = false; break; }
        const uint32_t a_t = base + s * stage_bytes, b_t = a_t + A_BYTES;
        stage_operand(a_t, p.A, p.a_rs, p.a_ks, m0, p.M, 128, c * 64, p.K);
        stage_operand(b_t, p.B, p.b_rs, p.b_ks, 0, p.N, p.Np, c * 64, p.K);
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_bf16(tmem, sdesc_sw128(a_t + 32u * kk), sdesc_sw128(b_t + 32u * kk), idesc,
                         (c > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&done[s]);
        }
        __syncwarp();
    }
    if (ok && nchunks > 0) {
        const int L = nchunks - 1;
        ok = mbar_wait(&done[L & 1], (uint32_t)((L >> 1) & 1), abort, p.flags);
    }
    tc_fence_after();
    if (ok) {
        const int row = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < p.Np; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            if (row < p.M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = c0 + j;
                    if (n >= p.N) break;
                    const int64_t o = (int64_t)row * p.c_rs + (int64_t)n * p.c_cs;
                    float x = v[j];
                    if (p.epi == EPI_BIAS || p.epi == EPI_BIAS_GELU) x += p.bias[n];
                    if (p.epi == EPI_GELU_BWD) x *= gelu_grad_f(p.aux[(int64_t)row * p.aux_ld + n]);
                    p.out0[o] = x;
                    if (p.epi == EPI_BIAS_GELU) p.out1[o] = gelu_f(x);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

int gemm(GemmArgs a, cudaStream_t s) {
    if (a.M < 1 || a.N < 1 || a.N > 256 || a.K < 1) return rtr_set_error(RTR_EINVAL, "proposer GEMM shape");
    a.Np = std::max(16, (a.N + 15) / 16 * 16);
    const size_t stage = A_BYTES + (((size_t)a.Np * 128 + 1023) & ~(size_t)1023);
    const size_t smem = 1024 + 2 * stage + 64;
    RTR_SMEM(mlp_gemm_kernel, smem);
    mlp_gemm_kernel<<<(unsigned)rtr_ceil_div(a.M, 128), GT, smem, s>>>(a);
    RTR_LAUNCH_CHECK("mlp_gemm_kernel");
    return RTR_OK;
}

// masked squared error: dOut = M (out - T) / sum(M), loss = 0.5 sum(M (out - T)^2) / sum(M)
__global__ void __launch_bounds__(1024) mlp_loss_kernel(const float* __restrict__ out, const float* __restrict__ T,
                                                        const float* __restrict__ Mk, int64_t n, float* __restrict__ dout,
                                                        double* __restrict__ loss) {
    __shared__ double red[32];
    double c = 0.0, l = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const double d = (double)out[e] - (double)T[e];
        c += Mk[e];
        l += Mk[e] * d * d;
    }
    c = rtr::block_sum(c, red);
    l = rtr::block_sum(l, red);
    const float inv = c > 0.0 ? (float)(1.0 / c) : 0.f;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) dout[e] = Mk[e] * (out[e] - T[e]) * inv;
    if (threadIdx.x == 0 && loss) *loss = c > 0.0 ? 0.5 * l / c : 0.0;
}

// db[o] = sum_b dZ[b * ld + o]
__global__ void __launch_bounds__(256) bias_grad_kernel(const float* __restrict__ dZ, int64_t ld, int batch,
                                                        float* __restrict__ db) {
    __shared__ double red[32];
    float s = 0.f;
    for (int b = threadIdx.x; b < batch; b += blockDim.x) s += dZ[(int64_t)b * ld + blockIdx.x];
    const double t = rtr::block_sum((double)s, red);
    if (threadIdx.x == 0) db[blockIdx.x] = (float)t;
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float c1, float c2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = 0.9f * m[e] + 0.1f * ge;
        const float ve = 0.999f * v[e] + 0.001f * ge * ge;
        m[e] = me;
        v[e] = ve;
        th[e] -= lr * (me * c1) / (sqrtf(ve * c2) + 1e-8f);
    }
}

// One CTA per mode: Gram Y^T Y (float64), Jacobi eigenvalues, sorted
// descending; f[64 n + i] = max(0, 1 + log10(lambda_i / lambda_0) / 12)
// (= 1 + log10(s_i / s_0) / 6 for the singular values s of Y_n).
struct FeatArgs {
    const double* Y[MODES];
    int I[MODES], K[MODES];
    int N;
    float* f;
};

__global__ void __launch_bounds__(256) features_kernel(const FeatArgs p) {
    extern __shared__ __align__(16) double fsm[];
    const int n = blockIdx.x;
    const int tid = threadIdx.x;
    float* fo = p.f + (size_t)SPEC * n;
    if (n >= p.N) {
        for (int i = tid; i < SPEC; i += blockDim.x) fo[i] = 0.f;
        return;
    }
    const int K = p.K[n], I = p.I[n];
    const double* Y = p.Y[n];
    double* A = fsm;                 // K x K
    double* V = A + K * K;           // K x K
    double* cs = V + K * K;          // 2 * ((K + 1) / 2)
    int* pairs = reinterpret_cast<int*>(cs + 2 * ((K + 1) / 2 + 1));
    __shared__ double lam[SPEC];
    for (int e = tid; e < K * K; e += blockDim.x) {
        const int a = e / K, b = e % K;
        if (a > b) continue;
        double s = 0.0;
        for (int i = 0; i < I; ++i) s += Y[(int64_t)i * K + a] * Y[(int64_t)i * K + b];
        A[a * K + b] = s;
        A[b * K + a] = s;
    }
    __syncthreads();
    rtr::block_jacobi_eig<double>(A, V, K, K, pairs, cs, 40, 1e-30);
    __syncthreads();
    for (int i = tid; i < K; i += blockDim.x) lam[i] = A[i * K + i];
    __syncthreads();
    const int valid = min(I, K);
    for (int i = tid; i < SPEC; i += blockDim.x) {
        float out = 0.f;
        if (i < K) {
            // rank of lam[i] in descending order (ties by index)
            const double li = lam[i];
            int pos = 0;
            double l0 = lam[0];
            for (int j = 0; j < K; ++j) {
                const double lj = lam[j];
                if (lj > li || (lj == li && j < i)) ++pos;
                l0 = fmax(l0, lj);
            }
            double fv = 0.0;
            if (pos < valid && l0 > 0.0 && li > 0.0) fv = fmax(0.0, 1.0 + log10(li / l0) / 12.0);
            fo[pos] = (float)fv;
        } else {
            fo[i] = 0.f;
        }
    }
}

// network pointers inside theta
struct Net {
    const float* W[4];
    const float* b[4];
    int in[4], out[4];
};
Net net_of(const float* th) {
    Net n{};
    const int ins[4] = {IN, HID, HID, HID}, outs[4] = {HID, HID, HID, OUT};
    size_t off = 0;
    for (int l = 0; l < 4; ++l) {
        n.in[l] = ins[l];
        n.out[l] = outs[l];
        n.W[l] = th + off;
        off += (size_t)ins[l] * outs[l];
        n.b[l] = th + off;
        off += outs[l];
    }
    return n;
}

struct Work {
    int* flags;
    float* Z[3];
    float* H[3];
    float* out;
    float* dout;
    float* dZ[2];
};
size_t work_bytes_for(int batch) {
    return WORK_HEADER + sizeof(float) * (size_t)batch * (6 * HID + 2 * 16 + 2 * HID);
}
Work work_of(void* w, int batch) {
    Work k{};
    k.flags = reinterpret_cast<int*>(w);
    float* f = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(w) + WORK_HEADER);
    const size_t bh = (size_t)batch * HID;
    for (int l = 0; l < 3; ++l) { k.Z[l] = f; f += bh; k.H[l] = f; f += bh; }
    k.out = f; f += (size_t)batch * 16;
    k.dout = f; f += (size_t)batch * 16;
    k.dZ[0] = f; f += bh;
    k.dZ[1] = f;
    return k;
}

int forward(const Net& net, const float* F, int batch, float* out, const Work& w, cudaStream_t s) {
    const float* H = F;
    for (int l = 0; l < 4; ++l) {
        GemmArgs a{};
        a.A = H; a.a_rs = net.in[l]; a.a_ks = 1;
        a.B = net.W[l]; a.b_rs = net.in[l]; a.b_ks = 1;
        a.M = batch; a.N = net.out[l]; a.K = net.in[l];
        a.bias = net.b[l];
        a.flags = w.flags;
        if (l < 3) {
            a.epi = EPI_BIAS_GELU;
            a.out0 = w.Z[l]; a.out1 = w.H[l]; a.c_rs = HID; a.c_cs = 1;
        } else {
            a.epi = EPI_BIAS;
            a.out0 = out; a.c_rs = OUT; a.c_cs = 1;
        }
        int st = gemm(a, s);
        if (st) return st;
        H = w.H[l < 3 ? l : 0];
    }
    return RTR_OK;
}

int check_batch(int batch) {
    if (batch < 1 || batch > 65536) return rtr_set_error(RTR_EINVAL, "proposer batch %d outside [1, 65536]", batch);
    return RTR_OK;
}

}  // namespace

extern "C" {

size_t rtr_mlp_param_count(void) { return PCOUNT; }

size_t rtr_mlp_work_bytes(int batch) { return batch < 1 ? 0 : work_bytes_for(batch); }

int rtr_mlp_forward(const float* theta, const float* F, int batch, float* out, void* work, size_t work_bytes,
                    void* stream) {
    if (!theta || !F || !out || !work) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (int st = check_batch(batch)) return st;
    if (work_bytes < work_bytes_for(batch)) return rtr_set_error(RTR_ENOMEM, "proposer workspace too small");
    return forward(net_of(theta), F, batch, out, work_of(work, batch), (cudaStream_t)stream);
}

int rtr_mlp_grad(const float* theta, const float* F, const float* T, const float* M, int batch, float* grad,
                 double* loss, void* work, size_t work_bytes, void* stream) {
    if (!theta || !F || !T || !M || !grad || !work) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (int st = check_batch(batch)) return st;
    if (work_bytes < work_bytes_for(batch)) return rtr_set_error(RTR_ENOMEM, "proposer workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    const Net net = net_of(theta);
    const Work w = work_of(work, batch);
    int st = forward(net, F, batch, w.out, w, s);
    if (st) return st;
    mlp_loss_kernel<<<1, 1024, 0, s>>>(w.out, T, M, (int64_t)batch * OUT, w.dout, loss);
    RTR_LAUNCH_CHECK("mlp_loss_kernel");
    // gradient pointers: same layout as theta
    Net g = net_of(grad);
    const float* dZ = w.dout;
    int64_t dz_ld = OUT;
    for (int l = 3; l >= 0; --l) {
        const float* Hin = l > 0 ? w.H[l - 1] : F;
        const int64_t h_ld = net.in[l];
        // dW_l^T[i, o] = sum_b H_in[b, i] dZ[b, o]   (stored as dW_l[o, i])
        GemmArgs a{};
        a.A = Hin; a.a_rs = 1; a.a_ks = h_ld;
        a.B = dZ; a.b_rs = 1; a.b_ks = dz_ld;
        a.M = net.in[l]; a.N = net.out[l]; a.K = batch;
        a.epi = EPI_STORE;
        a.out0 = const_cast<float*>(g.W[l]); a.c_rs = 1; a.c_cs = net.in[l];
        a.flags = w.flags;
        if ((st = gemm(a, s))) return st;
        bias_grad_kernel<<<net.out[l], 256, 0, s>>>(dZ, dz_ld, batch, const_cast<float*>(g.b[l]));
        RTR_LAUNCH_CHECK("bias_grad_kernel");
        if (l == 0) break;
        // dZ_{l-1}[b, i] = (sum_o dZ[b, o] W_l[o, i]) * GELU'(Z_{l-1}[b, i])
        GemmArgs d{};
        d.A = dZ; d.a_rs = dz_ld; d.a_ks = 1;
        d.B = net.W[l]; d.b_rs = 1; d.b_ks = net.in[l];
        d.M = batch; d.N = net.in[l]; d.K = net.out[l];
        d.epi = EPI_GELU_BWD;
        d.aux = w.Z[l - 1]; d.aux_ld = HID;
        float* dst = w.dZ[l & 1];
        d.out0 = dst; d.c_rs = HID; d.c_cs = 1;
        d.flags = w.flags;
        if ((st = gemm(d, s))) return st;
        dZ = dst;
        dz_ld = HID;
    }
    return RTR_OK;
}

int rtr_mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, void* stream) {
    if (!theta || !grad || !m || !v) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (step < 1) return rtr_set_error(RTR_EINVAL, "Adam step %d < 1", step);
    const double c1 = 1.0 / (1.0 - std::pow(0.9, step)), c2 = 1.0 / (1.0 - std::pow(0.999, step));
    adam_kernel<<<(unsigned)rtr_ceil_div((int64_t)PCOUNT, 256), 256, 0, (cudaStream_t)stream>>>(
        theta, grad, m, v, (int64_t)PCOUNT, lr, (float)c1, (float)c2);
    RTR_LAUNCH_CHECK("adam_kernel");
    return RTR_OK;
}

int rtr_mlp_status(void* work, int* flags) {
    if (!work || !flags) return rtr_set_error(RTR_EINVAL, "NULL argument");
    RTR_CUDA(cudaDeviceSynchronize());
    RTR_CUDA(cudaMemcpy(flags, work, sizeof(int), cudaMemcpyDeviceToHost));
    RTR_CUDA(cudaMemset(work, 0, sizeof(int)));
    *flags &= RTR_FLAG_TIMEOUT;
    return *flags & RTR_FLAG_TIMEOUT ? RTR_ETIMEOUT : RTR_OK;
}

int rtr_spectrum_features(int N, const int64_t* dims, const int* Kf, const double* const* Y, float* f,
                          void* stream) {
    if (!dims || !Kf || !Y || !f) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (N < 1 || N > MODES) return rtr_set_error(RTR_EINVAL, "feature modes %d outside [1, 5]", N);
    FeatArgs a{};
    a.N = N;
    a.f = f;
    int kmax = 1;
    for (int n = 0; n < N; ++n) {
        if (!Y[n]) return rtr_set_error(RTR_EINVAL, "Y[%d] is NULL", n);
        if (Kf[n] < 1 || Kf[n] > SPEC) return rtr_set_error(RTR_EINVAL, "sketch width %d outside [1, 64]", Kf[n]);
        if (dims[n] < 1 || dims[n] > (1 << 30)) return rtr_set_error(RTR_EINVAL, "mode size out of range");
        a.Y[n] = Y[n];
        a.I[n] = (int)dims[n];
        a.K[n] = Kf[n];
        kmax = std::max(kmax, Kf[n]);
    }
    const size_t smem = sizeof(double) * (2 * (size_t)kmax * kmax + 2 * ((kmax + 1) / 2 + 1)) +
                        sizeof(int) * 2 * ((kmax + 1) / 2 + 1) + 16;
    RTR_SMEM(features_kernel, smem);
    features_kernel<<<MODES, 256, smem, (cudaStream_t)stream>>>(a);
    RTR_LAUNCH_CHECK("features_kernel");
    return RTR_OK;
}

int rtr_propose(const float* out, int N, const int64_t* dims, int r_max, int* K, int* R) {
    if (!out || !dims || !K || !R) return rtr_set_error(RTR_EINVAL, "NULL argument");
    if (N < 1 || N > MODES) return rtr_set_error(RTR_EINVAL, "proposal modes %d outside [1, 5]", N);
    if (r_max < 1 || r_max > RTR_MAX_RANK) return rtr_set_error(RTR_EINVAL, "r_max %d outside [1, 16]", r_max);
    for (int n = 0; n < N; ++n) {
        const double k = std::nearbyint((double)out[2 * n] * 64.0);
        const double r = std::nearbyint((double)out[2 * n + 1] * 16.0);
        const double kcap = (double)std::min<int64_t>(dims[n], SPEC);
        K[n] = (int)std::min(std::max(k, 1.0), kcap);
        R[n] = (int)std::min(std::max(r, 1.0), (double)r_max);
    }
    return RTR_OK;
}

}  // extern "C"
