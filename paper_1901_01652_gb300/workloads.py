"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests (which feed the oracle) and by the bench
(which feeds the CUDA library).  It draws random numbers and builds data
factors only: it holds none of the decomposition's arithmetic.  Consumers
assemble a TR tensor from the cores themselves (the oracle with its own
Eq. 1 expansion, the bench with the library's reconstruct).

The paper's data (an RGB image, CIFAR10, COIL100, a hyperspectral image) is
not available; the recipes below stand in for the shapes and structure of
those workloads (Section 4).
"""
import math

import numpy as np

# The five workloads, with the sizes they are measured at.
CONFIGS = {
    "c1_fp64_60x4": dict(dims=(60, 60, 60, 60), tr_rank=5, snr_db=40.0, K=15, R=5,
                         sweeps=20, prec="fp64", seed=1902),
    "c2_bf16_200x4": dict(dims=(200, 200, 200, 200), tr_rank=10, snr_db=30.0, K=25, R=10,
                          sweeps=30, prec="bf16", seed=1903),
    "c3_fp8_hsi": dict(dims=(1024, 1024, 256), n_sig=20, n_bumps=40, noise_rel=0.01,
                       K=(60, 60, 30), eps=1e-2, prec="fp8", seed=1904),
    # 256 image-like order-4 tensors (H, W, C, S), modes U{32..96}, TR rank
    # r ~ U{4..12} per tensor, K_n = min(I_n, 2r), R_n = r
    "c4_batch256": dict(count=256, lo=32, hi=96, rlo=4, rhi=12, sweeps=20, prec="bf16", seed=1905),
}


def tr_cores(dims, ranks, seed):
    """TR cores G_n of shape (R_n, I_n, R_{n+1}), R_{N+1} = R_1, entries
    i.i.d. N(0, 1) (float64)."""
    rng = np.random.default_rng(seed)
    N = len(dims)
    if np.isscalar(ranks):
        ranks = [int(ranks)] * N
    return [rng.standard_normal((ranks[n], dims[n], ranks[(n + 1) % N]))
            for n in range(N)]


def unit_noise(shape, seed):
    """i.i.d. N(0, 1) noise (float64)."""
    return np.random.default_rng(seed + 7919).standard_normal(shape)


def snr_sigma(signal_norm, numel, snr_db):
    """Noise standard deviation giving SNR_dB = 10 log10(||S||^2 / ||N||^2)
    in expectation for i.i.d. Gaussian noise on `numel` entries."""
    return signal_norm * 10.0 ** (-snr_db / 20.0) / math.sqrt(numel)


def als_init(dims, ranks, seed):
    """A seeded TR-ALS starting point (cores with N(0,1) entries)."""
    return tr_cores(dims, ranks, seed + 104729)


def hsi_factors(H, W, B, n_sig=20, n_bumps=40, seed=0):
    """Hyperspectral-shaped factors: `n_sig` abundance maps (H x W), each a sum
    of `n_bumps` separable Gaussian bumps (random centres, widths 10..80 px,
    amplitudes U(0,1)), and `n_sig` smooth spectral signatures of length B
    (natural cubic splines through 8 random knots on [0, B-1], values U(0,1)).
    The tensor is X(h, w, b) = sum_s A[h, w, s] * S[b, s] (plus noise)."""
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(seed)
    h = np.arange(H, dtype=np.float64)
    w = np.arange(W, dtype=np.float64)
    A = np.zeros((H, W, n_sig))
    for s in range(n_sig):
        ch = rng.uniform(0, H, n_bumps)
        cw = rng.uniform(0, W, n_bumps)
        wh = rng.uniform(10, 80, n_bumps)
        ww = rng.uniform(10, 80, n_bumps)
        amp = rng.uniform(0, 1, n_bumps)
        fh = np.exp(-0.5 * ((h[:, None] - ch[None]) / wh[None]) ** 2)   # (H, nb)
        fw = np.exp(-0.5 * ((w[:, None] - cw[None]) / ww[None]) ** 2)   # (W, nb)
        A[:, :, s] = (fh * amp[None]) @ fw.T
    knots = np.linspace(0, B - 1, 8)
    S = np.empty((B, n_sig))
    b = np.arange(B, dtype=np.float64)
    for s in range(n_sig):
        S[:, s] = CubicSpline(knots, rng.uniform(0, 1, 8), bc_type="natural")(b)
    return A, S


def batch_shapes(count=256, lo=32, hi=96, rlo=4, rhi=12, seed=1905):
    """Uneven order-4 shapes (H, W, C, S) with modes uniform on [lo, hi] and a
    per-tensor TR rank uniform on [rlo, rhi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dims = tuple(int(x) for x in rng.integers(lo, hi + 1, size=4))
        out.append((dims, int(rng.integers(rlo, rhi + 1))))
    return out


def smoothed_tr_cores(dims, r, seed, sigma=2.0, spatial=(0, 1)):
    """TR cores with N(0, 1) entries, those of the `spatial` modes smoothed
    along their index by a Gaussian filter (std `sigma` samples), so that the
    tensor varies smoothly along those modes like image rows and columns."""
    from scipy.ndimage import gaussian_filter1d
    cores = tr_cores(dims, r, seed)
    return [gaussian_filter1d(c, sigma, axis=1, mode="nearest") if n in spatial else c
            for n, c in enumerate(cores)]


def to_pixels(x):
    """Min-max map to [0, 255] and round to integers (numpy array or torch
    tensor, same type back)."""
    lo, hi = x.min(), x.max()
    return ((x - lo) * (255.0 / (hi - lo))).round()


def batch_ranks(dims, r):
    """Sketch sizes and TR ranks of one batch tensor: K_n = min(I_n, 2r), R_n = r."""
    return tuple(min(int(d), 2 * r) for d in dims), (r,) * len(dims)


def proposer_shapes(count, seed=1906, snr=(30.0, 50.0), rlo=1, rhi=6):
    """Training/evaluation tensors of the learned proposer: order 4 (modes
    U{16..36}) or order 5 (modes U{10..18}) with equal probability, uniform TR
    rank r ~ U{rlo..rhi}, SNR ~ U[snr] dB.  Returns (dims, r, snr_db, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        if rng.uniform() < 0.5:
            dims = tuple(int(x) for x in rng.integers(16, 37, size=4))
        else:
            dims = tuple(int(x) for x in rng.integers(10, 19, size=5))
        out.append((dims, int(rng.integers(rlo, rhi + 1)), float(rng.uniform(*snr)), seed + 7 * t + 1))
    return out
