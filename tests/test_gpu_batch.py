"""Batched form of Algorithm 1 (many uneven tensors, one graph) against the
oracle, tensor by tensor."""
import numpy as np
import pytest
import torch

from oracle import rtrd as orc
from oracle import tensor as ot
from paper_1901_01652_gb300 import rtr, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small_batch(count, lo, hi, rlo, rhi, seed):
    """Image-like tensors of the batched workload's recipe at small sizes."""
    shapes = workloads.batch_shapes(count, lo, hi, rlo, rhi, seed)
    Xs, Ks, Rs = [], [], []
    for t, (dims, r) in enumerate(shapes):
        S = ot.tr_full(workloads.smoothed_tr_cores(dims, r, seed + 31 * t))
        Xs.append(workloads.to_pixels(S))
        K, R = workloads.batch_ranks(dims, r)
        Ks.append(K)
        Rs.append(R)
    return [s[0] for s in shapes], Xs, Ks, Rs


def run_batch(shapes, Xs, Ks, Rs, prec, seed, sweeps, nstreams, runs=1, refill=None):
    params = rtr.make_params(prec, seed, sweeps)
    b = rtr.rtr_batch_create(shapes, Ks, Rs, params, nstreams)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = [torch.from_numpy(np.ascontiguousarray(X)).to(dt).cuda() for X in Xs]
    N = len(shapes[0])
    G = [[torch.zeros(Rs[t][n] * shapes[t][n] * Rs[t][(n + 1) % N], dtype=torch.float64, device="cuda")
          for n in range(N)] for t in range(len(shapes))]
    rse = torch.zeros(len(shapes), dtype=torch.float64, device="cuda")
    outs = []
    for i in range(runs):
        if refill is not None and i == runs - 1:
            for t, X in enumerate(refill):
                Xd[t].copy_(torch.from_numpy(np.ascontiguousarray(X)).to(dt))
        rtr.rtr_batch_run(b, Xd, G, rse)
        torch.cuda.synchronize()
        cores = [[G[t][n].cpu().numpy().reshape(Rs[t][n], shapes[t][n], Rs[t][(n + 1) % N]) for n in range(N)]
                 for t in range(len(shapes))]
        outs.append((cores, rse.cpu().numpy().copy()))
    return b, outs


def oracle_batch(Xs, Ks, Rs, prec, seed, sweeps):
    refs = []
    for t, X in enumerate(Xs):
        Xo = X.astype(np.float32).astype(np.float64) if prec != "fp64" else X
        ref = orc.rtrd(Xo, Ks[t], Rs[t], "als", seed=seed + t, prec=prec, sweeps=sweeps)
        rse = orc.rse_identity(ot.fro(Xo) ** 2, ref["P"], ref["Z"])
        refs.append((ot.tr_full(ref["G"]), rse))
    return refs


def test_batch_fp64_uneven_vs_oracle():
    shapes, Xs, Ks, Rs = small_batch(7, 6, 15, 2, 3, 70)
    _, outs = run_batch(shapes, Xs, Ks, Rs, "fp64", 71, 6, nstreams=3)
    refs = oracle_batch(Xs, Ks, Rs, "fp64", 71, 6)
    cores, rse = outs[0]
    for t in range(len(shapes)):
        assert rel(ot.tr_full(cores[t]), refs[t][0]) <= 1e-10, t
        assert abs(rse[t] - refs[t][1]) <= 1e-9 * max(1.0, refs[t][1]), t


def test_batch_bf16_graph_replay_and_new_data():
    """First run eager + capture, second run replays the graph (bitwise the
    same results), third run replays on new contents of the same buffers."""
    shapes, Xs, Ks, Rs = small_batch(9, 8, 24, 2, 4, 80)
    # same shapes, new values
    Xs2 = [workloads.to_pixels(ot.tr_full(workloads.smoothed_tr_cores(X.shape, Rs[t][0], 900 + t)))
           for t, X in enumerate(Xs)]
    b, outs = run_batch(shapes, Xs, Ks, Rs, "bf16", 82, 8, nstreams=4, runs=3, refill=Xs2)
    assert rtr.rtr_batch_graph_kernels(b) > 0
    (c1, r1), (c2, r2), (c3, r3) = outs
    for t in range(len(shapes)):
        for n in range(4):
            assert np.array_equal(c1[t][n], c2[t][n]), (t, n)
    assert np.array_equal(r1, r2)
    for cores, rse, data in ((c1, r1, Xs), (c3, r3, Xs2)):
        refs = oracle_batch(data, Ks, Rs, "bf16", 82, 8)
        for t in range(len(shapes)):
            assert rel(ot.tr_full(cores[t]), refs[t][0]) <= 1e-3, t
            assert abs(rse[t] - refs[t][1]) <= 1e-3 * max(1e-3, refs[t][1]) + 1e-6, t


def test_batch_bf16_large_ranks_vs_oracle():
    """The batched workload's recipe at ranks 8..12 (Gram matrices up to
    144 x 144, K_n R_n R_{n+1} up to 3456): every tensor within 1e-3."""
    shapes, Xs, Ks, Rs = small_batch(4, 20, 30, 8, 12, 90)
    b, outs = run_batch(shapes, Xs, Ks, Rs, "bf16", 91, 5, nstreams=2)
    assert rtr.rtr_batch_flags(b) & ~rtr.FLAG_GRAM_PINV == 0
    refs = oracle_batch(Xs, Ks, Rs, "bf16", 91, 5)
    cores, rse = outs[0]
    for t in range(len(shapes)):
        assert rel(ot.tr_full(cores[t]), refs[t][0]) <= 1e-3, (t, shapes[t], Rs[t])
        assert abs(rse[t] - refs[t][1]) <= 1e-3 * refs[t][1] + 1e-6, t


def test_batch_argument_errors():
    params = rtr.make_params("fp32", 1, 2)
    with pytest.raises(ValueError):
        rtr.rtr_batch_create([(8, 8, 8)], [(4, 4)], [(2, 2, 2)], params)
    with pytest.raises(rtr.RtrError):
        rtr.rtr_batch_create([(8, 8, 8)], [(4, 4, 4)], [(2, 2, 2)], params, nstreams=0)
    params.chain_order[0] = 2
    with pytest.raises(rtr.RtrError):
        rtr.rtr_batch_create([(8, 8, 8)], [(4, 4, 4)], [(2, 2, 2)], params)


def _order_batch(order, count, lo, hi, rlo, rhi, seed):
    """Order-3 or order-5 TR tensors of the batched recipe (the contraction
    streams the last two cyclic modes of every update: an empty prefix for
    order 3, a one-product prefix chain for order 5)."""
    rng = np.random.default_rng(seed)
    shapes, Xs, Ks, Rs = [], [], [], []
    for t in range(count):
        dims = tuple(int(x) for x in rng.integers(lo, hi + 1, size=order))
        r = int(rng.integers(rlo, rhi + 1))
        S = ot.tr_full(workloads.smoothed_tr_cores(dims, r, seed + 31 * t))
        shapes.append(dims)
        Xs.append(workloads.to_pixels(S))
        K, R = workloads.batch_ranks(dims, r)
        Ks.append(K)
        Rs.append(R)
    return shapes, Xs, Ks, Rs


@pytest.mark.parametrize("order,prec", [(3, "fp64"), (5, "fp64"), (3, "bf16"), (5, "bf16")])
def test_batch_orders_3_and_5_vs_oracle(order, prec):
    lo, hi = (8, 20) if order == 3 else (5, 9)
    shapes, Xs, Ks, Rs = _order_batch(order, 5, lo, hi, 2, 3, 120 + order)
    _, outs = run_batch(shapes, Xs, Ks, Rs, prec, 121, 4, nstreams=2)
    cores, rse = outs[0]
    refs = oracle_batch(Xs, Ks, Rs, prec, 121, 4)
    tol = 1e-10 if prec == "fp64" else 1e-3
    for t in range(len(shapes)):
        assert rel(ot.tr_full(cores[t]), refs[t][0]) <= tol, (t, shapes[t], Rs[t])
