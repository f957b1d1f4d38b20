"""The pipelined end-to-end call (api.decompose_stream): several host tensors
with two in flight on their own plans and streams give, per tensor, the
result of the one-tensor call (api.decompose) and the oracle's within the
BF16 gate."""
import numpy as np
import pytest
import torch

from oracle import rtrd as orc
from oracle import tensor as ot
from paper_1901_01652_gb300 import rtr, workloads
from paper_1901_01652_gb300.api import decompose, decompose_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_decompose_stream_matches_decompose_and_oracle():
    dims, K, R, seed, sweeps = (24, 20, 22, 18), (8, 8, 8, 8), (3, 3, 3, 3), 21, 6
    Xs = []
    for t in range(3):
        S = ot.tr_full(workloads.tr_cores(dims, R, 40 + t))
        X = S + workloads.snr_sigma(ot.fro(S), S.size, 30.0) * workloads.unit_noise(dims, 40 + t)
        Xs.append(X.astype(np.float32))
    hosts = [torch.from_numpy(x).pin_memory() for x in Xs]
    out = decompose_stream(hosts, K, R, "als", "bf16", seed, sweeps, inflight=2)
    assert len(out) == 3
    for x, h, (G, rse) in zip(Xs, hosts, out):
        G1, rse1, eng = decompose(h, K, R, "als", "bf16", seed, sweeps)
        assert rtr.rtr_plan_flags(eng.plan) == 0
        # same plan parameters and kernels: the same result, and the same RSE
        for g, g1 in zip(G, G1):
            assert np.array_equal(g.numpy(), g1.numpy())
        assert rse == rse1
        ref = orc.rtrd(x.astype(np.float64), K, R, "als", seed=seed, prec="bf16", sweeps=sweeps)
        assert rel(ot.tr_full([g.numpy() for g in G]), ot.tr_full(ref["G"])) < 1e-3
