"""GPU kernels of the learned proposer (spectrum features, tensor-core MLP
forward and gradient, Adam) against the oracle in oracle/proposer.py."""
import numpy as np
import pytest
import torch

from oracle import proposer as op
from paper_1901_01652_gb300 import rtr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rand_theta(seed):
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in op.LAYERS:
        parts.append(rng.standard_normal(o * i) * np.sqrt(2.0 / i))
        parts.append(rng.standard_normal(o) * 0.1)
    return np.concatenate(parts).astype(np.float32)


def dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def test_param_count_matches_oracle():
    assert rtr.rtr_mlp_param_count() == op.param_count()


@pytest.mark.parametrize("shapes", [[(40, 64), (200, 64), (17, 64), (64, 64)], [(9, 64), (30, 5)],
                                    [(100, 64), (100, 64), (100, 64), (100, 64), (100, 64)]])
def test_spectrum_features_vs_oracle(shapes):
    rng = np.random.default_rng(len(shapes))
    Ys = []
    for I, K in shapes:
        # decaying spectrum over several decades plus a rank-deficient tail
        r = min(I, K)
        U, _ = np.linalg.qr(rng.standard_normal((I, r)))
        V, _ = np.linalg.qr(rng.standard_normal((K, r)))
        s = 10.0 ** (-np.linspace(0, 7, r)) * (1 + 0.1 * rng.uniform(size=r))
        Ys.append((U * s) @ V.T)
    f = torch.zeros(320, dtype=torch.float32, device="cuda")
    rtr.rtr_spectrum_features([I for I, _ in shapes], [K for _, K in shapes], [dev(Y, torch.float64) for Y in Ys], f)
    ref = op.spectrum_features(Ys)
    assert np.max(np.abs(f.cpu().numpy() - ref)) < 2e-5


@pytest.mark.parametrize("batch", [1, 77, 300])
def test_forward_vs_oracle(batch):
    th = rand_theta(1)
    F = np.random.default_rng(2).uniform(0, 1, (batch, op.N_IN)).astype(np.float32)
    out = torch.zeros((batch, 10), dtype=torch.float32, device="cuda")
    work = torch.zeros(rtr.rtr_mlp_work_bytes(batch), dtype=torch.uint8, device="cuda")
    rtr.rtr_mlp_forward(dev(th), dev(F), out, work)
    assert rtr.rtr_mlp_status(work) == 0
    ref, _ = op.forward(th.astype(np.float64), F.astype(np.float64), rnd=True)
    # bf16 operands are the same on both sides; float32 accumulation, and the
    # rare activation that float32 and float64 round to different bf16
    # neighbours, leave ~1e-5
    assert rel(out.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("batch", [5, 300])
def test_gradient_vs_oracle(batch):
    th = rand_theta(3)
    rng = np.random.default_rng(4)
    F = rng.uniform(0, 1, (batch, op.N_IN)).astype(np.float32)
    T = rng.uniform(0, 1, (batch, 10)).astype(np.float32)
    M = (rng.uniform(size=(batch, 10)) < 0.8).astype(np.float32)
    grad = torch.zeros(op.param_count(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    work = torch.zeros(rtr.rtr_mlp_work_bytes(batch), dtype=torch.uint8, device="cuda")
    rtr.rtr_mlp_grad(dev(th), dev(F), dev(T), dev(M), grad, loss, work)
    assert rtr.rtr_mlp_status(work) == 0
    lr_, gr = op.loss_and_grad(th.astype(np.float64), F.astype(np.float64), T.astype(np.float64),
                               M.astype(np.float64), rnd=True)
    assert float(loss.cpu()[0]) == pytest.approx(lr_, rel=1e-5)
    g = grad.cpu().numpy()
    off = 0
    for o, i in op.LAYERS:
        for n in (o * i, o):
            assert rel(g[off:off + n], gr[off:off + n]) < 2e-3, (o, i, n)
            off += n


def test_adam_vs_oracle():
    rng = np.random.default_rng(5)
    P = op.param_count()
    th = rng.standard_normal(P).astype(np.float32)
    tg, mg, vg = dev(th), torch.zeros(P, device="cuda"), torch.zeros(P, device="cuda")
    t64, m64, v64 = th.astype(np.float64), np.zeros(P), np.zeros(P)
    for step in range(1, 6):
        g = rng.standard_normal(P).astype(np.float32)
        rtr.rtr_mlp_adam(tg, dev(g), mg, vg, step, 1e-3)
        t64, m64, v64 = op.adam_step(t64, g.astype(np.float64), m64, v64, step, 1e-3)
    assert np.max(np.abs(tg.cpu().numpy() - t64)) < 1e-6
    assert rel(mg.cpu().numpy(), m64) < 1e-6 and rel(vg.cpu().numpy(), v64) < 1e-6


def test_training_lowers_the_loss_like_the_oracle():
    """Ten full-batch Adam steps on a fixed regression task: the GPU loss curve
    follows the oracle's (same data, same start) within bf16 tolerance."""
    th = rand_theta(6)
    rng = np.random.default_rng(7)
    B = 256
    F = rng.uniform(0, 1, (B, op.N_IN)).astype(np.float32)
    T = np.tanh(F[:, :10] * 2 - 1).astype(np.float32)
    M = np.ones((B, 10), dtype=np.float32)
    tg, mg, vg = dev(th), torch.zeros(th.size, device="cuda"), torch.zeros(th.size, device="cuda")
    grad = torch.zeros(th.size, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    work = torch.zeros(rtr.rtr_mlp_work_bytes(B), dtype=torch.uint8, device="cuda")
    Fd, Td, Md = dev(F), dev(T), dev(M)
    t64, m64, v64 = th.astype(np.float64), np.zeros(th.size), np.zeros(th.size)
    gl, ol = [], []
    for step in range(1, 11):
        rtr.rtr_mlp_grad(tg, Fd, Td, Md, grad, loss, work)
        gl.append(float(loss.cpu()[0]))
        rtr.rtr_mlp_adam(tg, grad, mg, vg, step, 1e-3)
        l64, g64 = op.loss_and_grad(t64, F.astype(np.float64), T.astype(np.float64), M.astype(np.float64))
        ol.append(l64)
        t64, m64, v64 = op.adam_step(t64, g64, m64, v64, step, 1e-3)
    assert gl[-1] < 0.5 * gl[0]
    assert np.allclose(gl, ol, rtol=2e-2)


def test_propose_decoding_matches_oracle():
    rng = np.random.default_rng(8)
    for _ in range(50):
        out = rng.uniform(-0.2, 1.3, 10).astype(np.float32)
        dims = tuple(int(x) for x in rng.integers(2, 120, size=int(rng.integers(3, 6))))
        assert rtr.rtr_propose(out, dims) == op.decode(out.astype(np.float64), dims)
