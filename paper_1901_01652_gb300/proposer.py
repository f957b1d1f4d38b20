"""Learned proposer of the sketch sizes K_n and TR ranks R_n.

The paper sets K_n and R_n by hand (Section 4).  Here a perceptron
(``rtr_mlp_*`` in include/rtr.h) reads the singular-value spectra of 64-column
sketches Y_n = X_(n) Omega_n (``rtr_sketch_mode_noalloc`` +
``rtr_spectrum_features``) and proposes (K_n, R_n).  It is trained on labels
from rank sweeps of the plain method (``rank_sweep_labels``: the smallest R
whose decomposition reaches a target error against the clean signal); the
fixed choice stays the fallback.  Every numerical step runs in the library's
kernels; this module holds device buffers, the training loop and the sweep
bookkeeping.
"""
import math

import numpy as np
import torch

from . import rtr

KF = 64          # sketch width of the features
N_IN, N_OUT = 320, 10


def sketch_features(X, seed, out=None, stream=None):
    """Spectrum features (float32 CUDA tensor of 320) of a float32 CUDA tensor
    X with at most 5 modes.  The sketches use the allocation-free entry point,
    whose static scratch array is shared by every call: calls of this function
    must not overlap on the GPU (other streams or threads)."""
    dims = tuple(X.shape)
    N = len(dims)
    Ys = []
    for n in range(N):
        A = math.prod(dims[:n])
        B = math.prod(dims[n + 1:])
        Y = torch.empty((dims[n], KF), dtype=torch.float64, device=X.device)
        rtr.rtr_sketch_mode_noalloc("fp32", X, (A, dims[n], B), KF, seed, n, Y, stream)
        Ys.append(Y)
    f = torch.empty(N_IN, dtype=torch.float32, device=X.device) if out is None else out
    rtr.rtr_spectrum_features(dims, [KF] * N, Ys, f, stream)
    return f


def k_rule(R):
    """Sketch size tied to a TR rank in the sweeps: the unfolding of a TR
    tensor of ranks R has rank <= R^2, so K = R^2 + R (oversampled by R),
    at most 64."""
    return min(R * R + R, KF)


class Proposer:
    """Device state of the perceptron: float32 master weights and Adam moments."""

    def __init__(self, seed=0, device="cuda"):
        P = rtr.rtr_mlp_param_count()
        rng = np.random.default_rng(seed)
        parts = []
        for o, i in ((128, 320), (128, 128), (128, 128), (10, 128)):
            parts.append(rng.standard_normal(o * i) * math.sqrt(2.0 / i))   # He initialisation
            parts.append(np.zeros(o))
        self.theta = torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(device)
        assert self.theta.numel() == P
        self.m = torch.zeros(P, dtype=torch.float32, device=device)
        self.v = torch.zeros(P, dtype=torch.float32, device=device)
        self.grad = torch.zeros(P, dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.step = 0
        self.device = device

    def fit(self, F, T, M, steps, lr=1e-3, batch=None, seed=0, log_every=100):
        """Adam on the masked squared error; F, T, M device float32 tensors.
        Returns the losses at every log_every-th step."""
        n = F.shape[0]
        batch = n if batch is None else min(batch, n)
        work = torch.zeros(rtr.rtr_mlp_work_bytes(batch), dtype=torch.uint8, device=self.device)
        gen = torch.Generator(device="cpu")
        gen.manual_seed(seed)
        hist = []
        perm, pos = None, n
        for s in range(steps):
            if batch == n:
                Fb, Tb, Mb = F, T, M
            else:
                if pos + batch > n:
                    perm = torch.randperm(n, generator=gen).to(self.device)
                    pos = 0
                idx = perm[pos:pos + batch]
                pos += batch
                Fb, Tb, Mb = F[idx].contiguous(), T[idx].contiguous(), M[idx].contiguous()
            rtr.rtr_mlp_grad(self.theta, Fb, Tb, Mb, self.grad, self.loss, work)
            self.step += 1
            rtr.rtr_mlp_adam(self.theta, self.grad, self.m, self.v, self.step, lr)
            if log_every and (s % log_every == 0 or s == steps - 1):
                hist.append(float(self.loss.cpu()[0]))
        if rtr.rtr_mlp_status(work):
            raise RuntimeError("a bounded wait of the proposer GEMM gave up")
        return hist

    def predict(self, F):
        out = torch.empty((F.shape[0], N_OUT), dtype=torch.float32, device=self.device)
        work = torch.zeros(rtr.rtr_mlp_work_bytes(F.shape[0]), dtype=torch.uint8, device=self.device)
        rtr.rtr_mlp_forward(self.theta, F, out, work)
        return out

    def propose(self, F, shapes, r_max=16):
        """(K list, R list) per tensor for feature rows F and their shapes."""
        out = self.predict(F).cpu().numpy()
        return [rtr.rtr_propose(out[t], shapes[t], r_max) for t in range(len(shapes))]


def decompose_batch(Xs, Ks, Rs, prec="fp32", seed=0, sweeps=10, nstreams=16, graph=False):
    """rTR-ALS of every tensor through the batched entry point (one batch per
    tensor order); returns (batches, core lists per tensor)."""
    groups = {}
    for t, X in enumerate(Xs):
        groups.setdefault(X.dim(), []).append(t)
    G = [None] * len(Xs)
    batches = []
    for N, idx in sorted(groups.items()):
        shapes = [tuple(Xs[t].shape) for t in idx]
        params = rtr.make_params(prec, seed, sweeps)
        if not graph:
            params.flags = rtr.PARAM_NO_GRAPH
        b = rtr.rtr_batch_create(shapes, [Ks[t] for t in idx], [Rs[t] for t in idx], params, nstreams)
        Gs = [[torch.empty(Rs[t][n] * Xs[t].shape[n] * Rs[t][(n + 1) % N], dtype=torch.float64,
                           device=Xs[t].device) for n in range(N)] for t in idx]
        rtr.rtr_batch_run(b, [Xs[t] for t in idx], Gs, None)
        for t, g in zip(idx, Gs):
            G[t] = g
        batches.append(b)
    return batches, G


def errors_vs_clean(G, Rs, Ss):
    """||TR(G_t) - S_t|| / ||S_t|| per tensor (reconstruction by the library)."""
    errs = []
    for t, S in enumerate(Ss):
        dims = tuple(S.shape)
        Xh = torch.empty(dims, dtype=torch.float32, device=S.device)
        work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, Rs[t]), dtype=torch.uint8, device=S.device)
        rtr.rtr_reconstruct(dims, Rs[t], G[t], "fp32", Xh, work)
        errs.append(float(torch.linalg.vector_norm(Xh - S, dtype=torch.float64) /
                          torch.linalg.vector_norm(S, dtype=torch.float64)))
    return np.array(errs)


def rank_sweep_labels(Xs, Ss, R_values, target=1e-2, prec="fp32", seed=0, sweeps=10):
    """Label of every tensor: the smallest R in R_values (uniform TR ranks,
    K_n = min(I_n, k_rule(R))) whose decomposition by the plain method has
    error <= target against the clean signal (the largest R if none does).
    Returns (labels R, error table [len(R_values) x count])."""
    table = []
    for R in R_values:
        Ks = [tuple(min(d, k_rule(R)) for d in X.shape) for X in Xs]
        Rs = [(R,) * X.dim() for X in Xs]
        bs, G = decompose_batch(Xs, Ks, Rs, prec, seed, sweeps)
        table.append(errors_vs_clean(G, Rs, Ss))
        for b in bs:
            b.close()
    table = np.array(table)
    labels = []
    for t in range(len(Xs)):
        ok = np.nonzero(table[:, t] <= target)[0]
        labels.append(R_values[ok[0]] if ok.size else R_values[-1])
    return np.array(labels), table


def label_targets(labels, shapes):
    """Target and mask rows (count x 10) for uniform labels R: K_n = k_rule(R)."""
    T = np.zeros((len(labels), N_OUT), dtype=np.float32)
    M = np.zeros((len(labels), N_OUT), dtype=np.float32)
    for t, (R, dims) in enumerate(zip(labels, shapes)):
        for n in range(len(dims)):
            T[t, 2 * n] = k_rule(int(R)) / 64.0
            T[t, 2 * n + 1] = int(R) / 16.0
            M[t, 2 * n] = M[t, 2 * n + 1] = 1.0
    return T, M


def nested_rank_sweep(X, S, R_values, target=1e-2, prec="fp32", seed=0, sweeps=10):
    """Rank-sweep label of one tensor with few sketches (the prefix reuse of
    the sketch sizes) and every TR-ALS run on the small projected tensor only;
    the result is rank_sweep_labels' for a tensor decomposed with `seed`.

    R uses K_n = min(I_n, k_rule(R)).  A mode with k_rule(R) >= I_n is kept
    whole, so the R values are grouped by the set of projected modes (larger
    R keep more modes whole).  Within a group the test matrix of a smaller K
    is the first K columns of the group's largest one (Omega_n[r, k] depends on
    (r, k) only), its basis the first K columns of the largest basis (QR is
    nested in its columns), and its projection P_K the leading block of the
    largest projection.  So per group X is sketched and projected once and S
    (the clean signal) projected with the same bases; for every R the grouped
    TR-ALS of the batched form runs on P_K alone (the solver and start of
    rank_sweep_labels), and the error against the clean signal is
        ||Xhat - S||^2 = ||TR(Z)||^2 - 2 <TR(Z), P_S,K> + ||S||^2
    with Xhat = TR(Z) x_n Q_K (Eq. 3; Q_K orthonormal).
    Returns (label R, error per R)."""
    from .api import RTRD
    dims = tuple(X.shape)
    N = len(dims)
    nS2 = float(torch.linalg.vector_norm(S, dtype=torch.float64)) ** 2
    groups = {}
    for R in R_values:
        groups.setdefault(tuple(k_rule(R) < d for d in dims), []).append(R)
    errs = {}
    for pattern, Rg in groups.items():
        Kg = [max(k_rule(R) for R in Rg) if pr else d for pr, d in zip(pattern, dims)]
        eng = RTRD(dims, Kg, [1] * N, prec, seed, sweeps, device=X.device)
        eng.sketch(X)
        eng.project(X)
        PS = torch.empty_like(eng.P)
        rtr.rtr_project(eng.plan, S, eng.Y, [torch.empty_like(q) for q in eng.Q], PS)
        for R in Rg:
            idx = tuple(slice(0, min(d, k_rule(R))) for d in dims)
            PK, PSK = eng.P[idx].contiguous(), PS[idx].contiguous()
            K = tuple(PK.shape)
            Rl = (R,) * N
            params = rtr.make_params(prec, seed, sweeps)
            params.flags = rtr.PARAM_NO_GRAPH
            b = rtr.rtr_batch_create([K], [K], [Rl], params, 1)
            G = [torch.empty(R * k * R, dtype=torch.float64, device=X.device) for k in K]
            rtr.rtr_batch_run(b, [PK], [G], None)
            work = torch.empty(rtr.rtr_reconstruct_work_bytes(K, Rl), dtype=torch.uint8, device=X.device)
            T = torch.empty(K, dtype=torch.float64, device=X.device)
            rtr.rtr_reconstruct(K, Rl, G, "fp64", T, work)
            e2 = float((T * T).sum()) - 2.0 * float((T * PSK.double()).sum()) + nS2
            errs[R] = max(e2, 0.0) ** 0.5 / nS2 ** 0.5
            b.close()
        eng.plan.close()
    errs = np.array([errs[R] for R in R_values])
    ok = np.nonzero(errs <= target)[0]
    return (R_values[ok[0]] if ok.size else R_values[-1]), errs
