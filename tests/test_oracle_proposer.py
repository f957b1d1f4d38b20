"""Pins of the proposer oracle (oracle/proposer.py) against closed forms,
finite differences and independent library routines (SciPy, PyTorch CPU)."""
import numpy as np
import pytest
import scipy.stats
import torch

from oracle import proposer as op


def rand_theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in op.LAYERS:
        parts.append(rng.standard_normal(o * i) * scale / np.sqrt(i))
        parts.append(rng.standard_normal(o) * 0.1)
    return np.concatenate(parts)


def test_param_layout():
    assert op.param_count() == 128 * 320 + 128 + 2 * (128 * 128 + 128) + 10 * 128 + 10
    th = np.arange(op.param_count(), dtype=np.float64)
    (W1, b1), (W2, _), _, (W4, b4) = op.unpack(th)
    assert W1.shape == (128, 320) and W1[0, 1] == 1 and b1[0] == 128 * 320
    assert W2[0, 0] == 128 * 320 + 128
    assert W4.shape == (10, 128) and b4[-1] == op.param_count() - 1


def test_gelu_closed_forms_and_library():
    x = np.linspace(-6, 6, 241)
    assert op.gelu(np.array([0.0]))[0] == 0.0
    # Phi(x) + Phi(-x) = 1  =>  GELU(x) - GELU(-x) = x
    assert np.allclose(op.gelu(x) - op.gelu(-x), x, atol=1e-14)
    assert np.allclose(op.gelu(x), x * scipy.stats.norm.cdf(x), rtol=1e-13, atol=1e-15)
    assert op.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    h = 1e-6
    fd = (op.gelu(x + h) - op.gelu(x - h)) / (2 * h)
    assert np.allclose(op.gelu_grad(x), fd, atol=1e-8)


def bf16(t):
    """torch's own bfloat16 rounding (float64 -> float32 -> bfloat16; the first
    step can double-round a value lying within 2^-24 of a bfloat16 halfway
    point, which the fixed seeds below never meet)."""
    return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def torch_forward(theta, F, rnd):
    """Independent forward: torch float64 Linear + GELU, bf16 via torch's own rounding."""
    th = torch.from_numpy(theta)
    H = torch.from_numpy(F)
    off = 0
    for l, (o, i) in enumerate(op.LAYERS):
        W = th[off:off + o * i].view(o, i)
        off += o * i
        b = th[off:off + o]
        off += o
        if rnd:
            Hr, Wr = bf16(H), bf16(W)
        else:
            Hr, Wr = H, W
        Z = torch.nn.functional.linear(Hr, Wr, b)
        H = torch.nn.functional.gelu(Z, approximate="none") if l < 3 else Z
    return H.numpy()


@pytest.mark.parametrize("rnd", [False, True])
def test_forward_matches_torch(rnd):
    rng = np.random.default_rng(3)
    F = rng.uniform(0, 1, (7, op.N_IN))
    th = rand_theta(4).astype(np.float32).astype(np.float64)    # float32 master weights
    out, _ = op.forward(th, F, rnd)
    ref = torch_forward(th, F, rnd)
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_gradient_matches_torch_autograd_and_finite_differences():
    rng = np.random.default_rng(5)
    B = 6
    F = rng.uniform(0, 1, (B, op.N_IN))
    T = rng.uniform(0, 1, (B, op.N_OUT))
    M = (rng.uniform(0, 1, (B, op.N_OUT)) < 0.7).astype(np.float64)
    th = rand_theta(6)
    loss, g = op.loss_and_grad(th, F, T, M, rnd=False)
    # autograd of an independent torch expression of the same loss
    tt = torch.from_numpy(th.copy()).requires_grad_(True)
    H = torch.from_numpy(F)
    off = 0
    for l, (o, i) in enumerate(op.LAYERS):
        W = tt[off:off + o * i].view(o, i)
        off += o * i
        b = tt[off:off + o]
        off += o
        Z = H @ W.T + b
        H = torch.nn.functional.gelu(Z) if l < 3 else Z
    Mt = torch.from_numpy(M)
    lt = 0.5 * (Mt * (H - torch.from_numpy(T)) ** 2).sum() / Mt.sum()
    lt.backward()
    assert loss == pytest.approx(float(lt.detach()), rel=1e-13)
    assert np.allclose(g, tt.grad.numpy(), rtol=1e-10, atol=1e-13)
    # central differences on a sample of coordinates (one per layer part)
    idx = [0, 5000, 128 * 320 + 3, 128 * 320 + 128 + 77, op.param_count() - 1290, op.param_count() - 1]
    for j in idx:
        h = 1e-6
        e = np.zeros_like(th)
        e[j] = h
        lp, _ = op.loss_and_grad(th + e, F, T, M, rnd=False)
        lm, _ = op.loss_and_grad(th - e, F, T, M, rnd=False)
        assert g[j] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9), j


def test_loss_mask_and_zero_residual():
    rng = np.random.default_rng(7)
    F = rng.uniform(0, 1, (4, op.N_IN))
    th = rand_theta(8)
    out, _ = op.forward(th, F)
    M = np.ones_like(out)
    M[:, 6:] = 0.0
    loss, g = op.loss_and_grad(th, F, out, M)
    assert loss == 0.0 and not np.any(g)
    T = out + 1.0
    T2 = T.copy()
    T2[:, 6:] += 100.0                  # masked entries do not matter
    l1, g1 = op.loss_and_grad(th, F, T, M)
    l2, g2 = op.loss_and_grad(th, F, T2, M)
    assert l1 == l2 and np.array_equal(g1, g2)
    assert l1 == pytest.approx(0.5, rel=1e-14)   # 0.5 * mean of 1^2


def test_adam_matches_torch_and_first_step_closed_form():
    rng = np.random.default_rng(9)
    th = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    p = torch.nn.Parameter(torch.from_numpy(th.copy()))
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    g0 = rng.standard_normal(50)
    t1, _, _ = op.adam_step(th, g0, m, v, 1, 1e-2)
    # first step: m_hat = g, v_hat = g^2  =>  step = lr * g / (|g| + eps)
    assert np.allclose(th - t1, 1e-2 * g0 / (np.abs(g0) + 1e-8), rtol=1e-12)
    cur = th
    for t in range(1, 6):
        g = rng.standard_normal(50)
        cur, m, v = op.adam_step(cur, g, m, v, t, 1e-2)
        p.grad = torch.from_numpy(g)
        opt.step()
    assert np.allclose(cur, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_spectrum_features_closed_form():
    rng = np.random.default_rng(11)
    s = np.array([10.0, 1.0, 1e-2, 1e-5, 1e-7])
    U, _ = np.linalg.qr(rng.standard_normal((30, 5)))
    V, _ = np.linalg.qr(rng.standard_normal((8, 5)))
    Y = (U * s) @ V.T                       # 30 x 8, singular values s then 0
    f = op.spectrum_features([Y, 3.0 * Y])
    want = np.maximum(1 + np.log10(s / s[0]) / 6, 0)   # [1, 5/6, 1/2, 0, 0]
    assert np.allclose(f[:5], want, atol=1e-9)
    assert np.allclose(f[5:8], 0, atol=1e-9)            # rank deficiency -> floor
    assert np.allclose(f[64:72], f[:8], atol=1e-9)      # scale invariance
    assert not np.any(f[8:64]) and not np.any(f[128:])  # beyond min(I, K) and N
    assert want[1] == pytest.approx(5 / 6) and want[2] == pytest.approx(0.5)


def test_decode_and_targets_round_trip():
    dims = (40, 20, 100, 64)
    K, R = [30, 20, 64, 17], [5, 9, 1, 16]
    T, M = op.targets(K, R)
    assert op.decode(T, dims) == (K, R)
    assert M.sum() == 8 and not np.any(M[8:])
    assert op.decode(np.full(10, 5.0), (10, 80, 3)) == ([10, 64, 3], [16, 16, 16])
    assert op.decode(np.full(10, -1.0), (10, 80, 3)) == ([1, 1, 1], [1, 1, 1])
