// Batched randomized TR decomposition: many tensors of uneven shapes
// decomposed (Algorithm 1 with TR-ALS) as one unit.
//
// rtr_batch_create builds one plan per tensor plus its step buffers.  The
// first rtr_batch_run executes eagerly, the tensors spread over a pool of
// worker streams (work of small tensors overlaps), and meanwhile tunes any
// new mode-product shape class; it then captures the same schedule into one
// CUDA graph.  Later runs with the same buffers replay the graph with a
// single launch on the caller's stream.
#include <algorithm>
#include <new>
#include <vector>
#include "rtr_internal.cuh"

struct rtr_batch {
    int count = 0, N = 0, nstreams = 0;
    std::vector<rtr_plan*> plans;
    std::vector<double*> Y, Q, Z;      // count * N
    std::vector<void*> P;              // count
    std::vector<int64_t> dims;         // count * N
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> fork, join;
    cudaEvent_t start = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key_X;
    std::vector<double*> key_G;
    double* key_rse = nullptr;
    uint64_t graph_kernels = 0;        // kernel launches captured in `exec`
    bool no_graph = false;
    BatchAls* als = nullptr;           // grouped TR-ALS over all tensors (null: per-tensor ALS)
};

namespace {

void free_batch(rtr_batch* b) {
    if (!b) return;
    for (auto* p : b->plans) if (p) rtr_plan_destroy(p);
    for (auto* v : b->Y) cudaFree(v);
    for (auto* v : b->Q) cudaFree(v);
    for (auto* v : b->Z) cudaFree(v);
    for (auto* v : b->P) cudaFree(v);
    for (auto s : b->workers) cudaStreamDestroy(s);
    for (auto e : b->fork) cudaEventDestroy(e);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->start) cudaEventDestroy(b->start);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->als) batch_als_destroy(b->als);
    delete b;
}

// Enqueue Algorithm 1 for every tensor on the worker streams, forked from and
// joined back into `origin`.  With the grouped TR-ALS, the sketches and
// projection chains run per tensor on the workers, then one grouped ALS over
// all tensors on `origin`, then back-projection and RSE per tensor again.
int fork(rtr_batch* b) {
    for (int w = 0; w < b->nstreams; ++w) {
        RTR_CUDA(cudaEventRecord(b->fork[w], b->origin));
        RTR_CUDA(cudaStreamWaitEvent(b->workers[w], b->fork[w], 0));
    }
    return RTR_OK;
}
int join(rtr_batch* b) {
    for (int w = 0; w < b->nstreams; ++w) {
        RTR_CUDA(cudaEventRecord(b->join[w], b->workers[w]));
        RTR_CUDA(cudaStreamWaitEvent(b->origin, b->join[w], 0));
    }
    return RTR_OK;
}

int enqueue(rtr_batch* b, const void* const* X, double* const* G, double* rse) {
    const int N = b->N;
    int st = fork(b);
    if (st) return st;
    for (int t = 0; t < b->count; ++t) {
        rtr_plan* p = b->plans[t];
        void* s = b->workers[t % b->nstreams];
        double* const* Y = b->Y.data() + (size_t)t * N;
        double* const* Q = b->Q.data() + (size_t)t * N;
        double* const* Z = b->Z.data() + (size_t)t * N;
        st = rtr_sketch(p, X[t], Y, s);
        if (!st) st = rtr_project(p, X[t], Y, Q, b->P[t], s);
        if (!st && !b->als) st = rtr_als(p, b->P[t], Z, 0, nullptr, s);
        if (!st && !b->als) st = rtr_backproject(p, Z, Q, G + (size_t)t * N, nullptr, s);
        if (!st && !b->als && rse) st = rtr_rse(p, b->P[t], Z, nullptr, rse + t, s);
        if (st) return st;
    }
    if ((st = join(b))) return st;
    if (!b->als) return RTR_OK;
    if ((st = batch_als_run(b->als, nullptr, b->origin))) return st;
    if ((st = fork(b))) return st;
    for (int t = 0; t < b->count; ++t) {
        rtr_plan* p = b->plans[t];
        void* s = b->workers[t % b->nstreams];
        double* const* Q = b->Q.data() + (size_t)t * N;
        double* const* Z = b->Z.data() + (size_t)t * N;
        st = rtr_backproject(p, Z, Q, G + (size_t)t * N, nullptr, s);
        if (!st && rse) st = rtr_rse(p, b->P[t], Z, nullptr, rse + t, s);
        if (st) return st;
    }
    return join(b);
}

}  // namespace

extern "C" {

int rtr_batch_create(rtr_batch** out, int count, int N, const int64_t* dims, const int* K, const int* R,
                     const rtr_params* params, int nstreams) {
    if (!out || !dims || !K || !R || !params) return rtr_set_error(RTR_EINVAL, "NULL argument");
    *out = nullptr;
    if (count < 1) return rtr_set_error(RTR_EINVAL, "batch count %d < 1", count);
    if (nstreams < 1 || nstreams > 64) return rtr_set_error(RTR_EINVAL, "stream count %d outside [1, 64]", nstreams);
    rtr_batch* b = new (std::nothrow) rtr_batch();
    if (!b) return rtr_set_error(RTR_ENOMEM, "host allocation failed");
    b->count = count;
    b->N = N;
    b->nstreams = std::min(nstreams, count);
    b->no_graph = (params->flags & RTR_PARAM_NO_GRAPH) != 0;
    b->dims.assign(dims, dims + (size_t)count * N);
    const size_t esz = params->prec == RTR_FP64 ? 8 : 4;
#define B_TRY(x) do { int s_ = (x); if (s_) { free_batch(b); return s_; } } while (0)
#define B_CUDA(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { free_batch(b); return rtr_cuda_check(e_, #x); } } while (0)
    for (int n = 0; n < 8; ++n)
        if (params->chain_order[n] != -1) {
            free_batch(b);
            return rtr_set_error(RTR_EINVAL, "batch params must leave chain_order at its default");
        }
    for (int t = 0; t < count; ++t) {
        rtr_plan* p = nullptr;
        rtr_params pt = *params;
        pt.seed = params->seed + (uint64_t)t;
        B_TRY(rtr_plan_create(&p, N, dims + (size_t)t * N, K + (size_t)t * N, R + (size_t)t * N, &pt));
        b->plans.push_back(p);
        int64_t pn = 1;
        for (int n = 0; n < N; ++n) {
            const int64_t I = dims[(size_t)t * N + n];
            const int k = p->K[n];
            const int ra = R[(size_t)t * N + n], rb = R[(size_t)t * N + (n + 1) % N];
            double *y = nullptr, *q = nullptr, *z = nullptr;
            if (p->proj[n]) B_CUDA(cudaMalloc(&y, sizeof(double) * I * k));
            B_CUDA(cudaMalloc(&q, sizeof(double) * I * k));
            B_CUDA(cudaMalloc(&z, sizeof(double) * ra * k * rb));
            b->Y.push_back(y);
            b->Q.push_back(q);
            b->Z.push_back(z);
            pn *= k;
        }
        void* P = nullptr;
        B_CUDA(cudaMalloc(&P, esz * pn));
        b->P.push_back(P);
    }
    B_CUDA(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    B_CUDA(cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming));
    for (int w = 0; w < b->nstreams; ++w) {
        cudaStream_t s;
        cudaEvent_t e1, e2;
        B_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->workers.push_back(s);
        B_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
        b->fork.push_back(e1);
        B_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
        b->join.push_back(e2);
    }
    {
        // grouped TR-ALS when every tensor is within its limits (else per-tensor ALS)
        std::vector<int64_t> Ke((size_t)count * N);
        std::vector<uint64_t> seeds(count);
        for (int t = 0; t < count; ++t) {
            for (int n = 0; n < N; ++n) Ke[(size_t)t * N + n] = b->plans[t]->K[n];
            seeds[t] = params->seed + (uint64_t)t;
        }
        int dev = 0;
        B_CUDA(cudaGetDevice(&dev));
        int sms = 0;
        B_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int st = batch_als_create(&b->als, count, N, Ke.data(), R, params->prec == RTR_FP64,
                                        params->sweeps, seeds.data(), b->plans[0]->tab64,
                                        (const void* const*)b->P.data(), b->Z.data(), sms);
        if (st == RTR_EUNSUPPORTED) b->als = nullptr;
        else if (st) { free_batch(b); return st; }
    }
#undef B_TRY
#undef B_CUDA
    *out = b;
    return RTR_OK;
}

int rtr_batch_destroy(rtr_batch* b) {
    free_batch(b);
    return RTR_OK;
}

int rtr_batch_run(rtr_batch* b, const void* const* X, double* const* G, double* rse, void* stream) {
    if (!b || !X || !G) return rtr_set_error(RTR_EINVAL, "NULL argument");
    for (int t = 0; t < b->count; ++t) {
        if (!X[t]) return rtr_set_error(RTR_EINVAL, "X[%d] is NULL", t);
        for (int n = 0; n < b->N; ++n)
            if (!G[(size_t)t * b->N + n]) return rtr_set_error(RTR_EINVAL, "G[%d][%d] is NULL", t, n);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ng = (size_t)b->count * b->N;
    bool same = b->exec && b->key_rse == rse;
    for (int t = 0; same && t < b->count; ++t) same = b->key_X[t] == X[t];
    for (size_t i = 0; same && i < ng; ++i) same = b->key_G[i] == G[i];
    if (same) {
        RTR_CUDA(cudaGraphLaunch(b->exec, s));
        return RTR_OK;
    }
    // eager run (tunes new shape classes), ordered after the caller's stream
    RTR_CUDA(cudaEventRecord(b->start, s));
    RTR_CUDA(cudaStreamWaitEvent(b->origin, b->start, 0));
    int st = enqueue(b, X, G, rse);
    if (st) return st;
    RTR_CUDA(cudaEventRecord(b->start, b->origin));
    RTR_CUDA(cudaStreamWaitEvent(s, b->start, 0));
    if (b->no_graph) return RTR_OK;
    // capture the same schedule for the next runs with these buffers
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    RTR_CUDA(cudaStreamSynchronize(b->origin));
    cudaGraph_t graph = nullptr;
    const uint64_t l0 = rtr_kernel_launches();
    RTR_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
    st = enqueue(b, X, G, rse);
    b->graph_kernels = rtr_kernel_launches() - l0;
    cudaError_t ce = cudaStreamEndCapture(b->origin, &graph);
    if (st) { if (graph) cudaGraphDestroy(graph); return st; }
    if (ce != cudaSuccess) return rtr_cuda_check(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { b->exec = nullptr; return rtr_cuda_check(ce, "cudaGraphInstantiate"); }
    b->key_X.assign(X, X + b->count);
    b->key_G.assign(G, G + ng);
    b->key_rse = rse;
    return RTR_OK;
}

int rtr_batch_flags(rtr_batch* b, int* flags) {
    if (!b || !flags) return rtr_set_error(RTR_EINVAL, "NULL argument");
    int f = 0;
    for (auto* p : b->plans) {
        int pf = 0;
        const int st = rtr_plan_flags(p, &pf);
        if (st) return st;
        f |= pf;
    }
    if (b->als) {
        int af = 0;
        const int st = batch_als_flags(b->als, &af);
        if (st) return st;
        f |= af;
    }
    *flags = f;
    return RTR_OK;
}

int rtr_batch_graph_kernels(const rtr_batch* b, uint64_t* n) {
    if (!b || !n) return rtr_set_error(RTR_EINVAL, "NULL argument");
    *n = b->exec ? b->graph_kernels : 0;
    return RTR_OK;
}

}  // extern "C"
