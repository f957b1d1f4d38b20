"""The learned proposer against the fixed choice K_n = 2R, R = 12: trained on
rank sweeps of the plain method, it must reach the error target on held-out
tensors about as often as the fixed choice, with far fewer TR parameters and
less GPU time."""
import time

import numpy as np
import pytest
import torch

from paper_1901_01652_gb300 import proposer as pp
from paper_1901_01652_gb300 import rtr, workloads

pytestmark = pytest.mark.gpu

TARGET = 1e-2          # error against the clean signal
N_TRAIN, N_TEST = 320, 96
R_SWEEP = list(range(1, 8))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()


def make_tensors(specs):
    """Clean TR tensors (library reconstruct of seeded cores) plus Gaussian
    noise at each tensor's SNR, as float32 CUDA tensors."""
    Xs, Ss = [], []
    for dims, r, snr, seed in specs:
        R = [r] * len(dims)
        cores = [torch.from_numpy(c).cuda() for c in workloads.tr_cores(dims, R, seed)]
        S = torch.empty(dims, dtype=torch.float32, device="cuda")
        work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, R), dtype=torch.uint8, device="cuda")
        rtr.rtr_reconstruct(dims, R, cores, "fp32", S, work)
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        nrm = float(torch.linalg.vector_norm(S, dtype=torch.float64))
        sigma = workloads.snr_sigma(nrm, S.numel(), snr)
        Xs.append(S + sigma * torch.randn(dims, generator=g, device="cuda"))
        Ss.append(S)
    return Xs, Ss


def tr_params(shape, R):
    N = len(shape)
    return sum(R[n] * shape[n] * R[(n + 1) % N] for n in range(N))


def timed_decomposition(Xs, Ks, Rs):
    """GPU seconds of the batched decomposition (graph replay, after a first
    run that captures it) and the cores."""
    bs, G = pp.decompose_batch(Xs, Ks, Rs, "fp32", 5, 10, graph=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in bs:
        xs = [X for X in Xs if X.dim() == b.N]
        gs = [g for X, g in zip(Xs, G) if X.dim() == b.N]
        rtr.rtr_batch_run(b, xs, gs, None)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, G, bs


def test_proposer_beats_the_fixed_choice():
    specs = workloads.proposer_shapes(N_TRAIN + N_TEST)
    Xs, Ss = make_tensors(specs)
    F = torch.stack([pp.sketch_features(X, 77) for X in Xs])
    labels, table = pp.rank_sweep_labels(Xs, Ss, R_SWEEP, TARGET, seed=5)
    shapes = [s[0] for s in specs]
    T, M = pp.label_targets(labels, shapes)
    tr = slice(0, N_TRAIN)
    prop = pp.Proposer(seed=11)
    hist = prop.fit(F[tr].contiguous(), torch.from_numpy(T[tr]).cuda(), torch.from_numpy(M[tr]).cuda(),
                    steps=3000, lr=1e-3, batch=64, seed=12)
    assert hist[-1] < 0.1 * hist[0]

    te = list(range(N_TRAIN, N_TRAIN + N_TEST))
    Xt, St, sh = [Xs[t] for t in te], [Ss[t] for t in te], [shapes[t] for t in te]
    props = prop.propose(F[N_TRAIN:].contiguous(), sh, r_max=12)
    Kp = [tuple(k) for k, _ in props]
    Rp = [tuple(r) for _, r in props]
    Kf = [tuple(min(d, 24) for d in s) for s in sh]
    Rf = [(12,) * len(s) for s in sh]
    t_prop, Gp, bp = timed_decomposition(Xt, Kp, Rp)
    e_prop = pp.errors_vs_clean(Gp, Rp, St)
    t_fix, Gf, bf = timed_decomposition(Xt, Kf, Rf)
    e_fix = pp.errors_vs_clean(Gf, Rf, St)
    # fallback rule: a proposal whose error misses the target is replaced by the fixed choice
    ok = e_prop <= TARGET
    p_prop = sum(tr_params(s, r) for s, r in zip(sh, Rp))
    p_fix = sum(tr_params(s, r) for s, r in zip(sh, Rf))
    r_true = np.array([specs[t][1] for t in te])
    r_prop = np.array([r[0] for r in Rp])
    print(f"\nproposer: target met {ok.mean():.3f} (fixed {np.mean(e_fix <= TARGET):.3f}); "
          f"TR parameters {p_prop} vs {p_fix} ({p_prop / p_fix:.3f}); GPU time {t_prop * 1e3:.1f} ms vs "
          f"{t_fix * 1e3:.1f} ms; label accuracy {np.mean(r_prop == labels[N_TRAIN:]):.3f}; "
          f"mean |R - r_true| {np.mean(np.abs(r_prop - r_true)):.2f}")
    # the gain: the target is met about as often as with the fixed choice (which
    # itself misses it where K_n = 24 < r^2 makes the projection lossy), with
    # at most half the TR parameters and less GPU time
    assert ok.mean() >= np.mean(e_fix <= TARGET) - 0.05
    assert p_prop <= 0.5 * p_fix
    assert t_prop < t_fix
    for b in bp + bf:
        b.close()
