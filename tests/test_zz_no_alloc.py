"""The allocation-free one-mode sketch (rtr_sketch_mode_noalloc) against the
plan-based rtr_sketch and against the oracle's sketch.

Some callers cannot call cudaMalloc: code embedded in a framework that owns
all device memory, or a service that must not grow its device footprint once
running.  For them the library keeps the sketch's split-K scratch in a
file-scope device array.  This file is named to be collected last, so that a
run stopping at the first failure has run every other test first; it also
passes alone in a fresh process (the first call does the per-device set-up).
"""
import numpy as np
import pytest
import torch

from oracle import rtrd as orc
from paper_1901_01652_gb300 import rtr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()


def _views(dims):
    for n in range(len(dims)):
        A = int(np.prod(dims[:n], dtype=np.int64))
        B = int(np.prod(dims[n + 1:], dtype=np.int64))
        yield n, (A, dims[n], B)


def _x(dims, prec, seed=3):
    X = np.random.default_rng(seed).standard_normal(dims)
    if prec == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == "fp64" else torch.float32
    return X, torch.from_numpy(X).to(dt).cuda()


def _noalloc(prec, Xd, dims, n, K, seed):
    A = int(np.prod(dims[:n], dtype=np.int64))
    B = int(np.prod(dims[n + 1:], dtype=np.int64))
    Y = torch.full((dims[n], K), float("nan"), dtype=torch.float64, device="cuda")
    rtr.rtr_sketch_mode_noalloc(prec, Xd, (A, dims[n], B), K, seed, n, Y)
    torch.cuda.synchronize()
    return Y.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_noalloc_sketch_matches_plan_sketch_and_oracle_twice(prec, tol):
    dims, K, seed = (23, 150, 41, 9), (7, 20, 13, 5), 2024
    X, Xd = _x(dims, prec)
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2, 2), rtr.make_params(prec, seed))
    Yref = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    rtr.rtr_sketch(plan, Xd, Yref)
    torch.cuda.synchronize()
    Yor = orc.sketch(X, K, seed, prec)
    for call in range(2):                      # the scratch keeps the last call's contents
        for n, _ in _views(dims):
            got = _noalloc(prec, Xd, dims, n, K[n], seed)
            assert _rel(got, Yref[n].cpu().numpy()) <= tol, (call, n)
            assert _rel(got, Yor[n]) <= tol, (call, n)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("dims,n,K", [
    ((2, 32768, 3), 1, 64),      # I*K = 2^21, the scratch's limit: a single split-K CTA
    ((3, 1000, 5), 1, 20),       # I = 1000: several row blocks (grid.y > 1)
])
def test_noalloc_sketch_at_the_scratch_limit_and_with_row_blocks(prec, tol, dims, n, K):
    seed = 77
    X, Xd = _x(dims, prec, seed=4)
    Kp = [d if m != n else K for m, d in enumerate(dims)]     # only mode n projected
    plan = rtr.rtr_plan_create(dims, Kp, (1, 1, 1), rtr.make_params(prec, seed))
    Yref = [None if m != n else torch.zeros((dims[n], K), dtype=torch.float64, device="cuda") for m in range(3)]
    rtr.rtr_sketch(plan, Xd, Yref)
    torch.cuda.synchronize()
    ref = orc.sketch(X, Kp, seed, prec)[n]
    for call in range(2):
        got = _noalloc(prec, Xd, dims, n, K, seed)
        assert _rel(got, Yref[n].cpu().numpy()) <= tol, call
        assert _rel(got, ref) <= tol, call


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    X = torch.zeros(40000, dtype=torch.float32, device="cuda")
    Y = torch.zeros(40000 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_sketch_mode_noalloc("fp32", X, (1, 40000, 1), 64, 0, 0, Y)   # I*K = 2.56e6 > 2^21
    assert e.value.status == rtr.RTR_EINVAL and "static scratch" in str(e.value)
    with pytest.raises(rtr.RtrError):
        rtr.rtr_sketch_mode_noalloc("fp32", X[:4], (1, 4, 1), 65, 0, 0, Y[:4 * 65])
