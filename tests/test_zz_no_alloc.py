"""The allocation-free one-mode sketch (rtr_sketch_mode_noalloc) against the
plan-based rtr_sketch.

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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_noalloc_sketch_matches_plan_sketch_twice(prec, tol):
    dims, K, seed = (23, 150, 41, 9), (7, 20, 13, 5), 2024
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.randn(dims, dtype=torch.float64, generator=torch.Generator().manual_seed(3)).to(dt).cuda()
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2, 2), rtr.make_params(prec, seed))
    Yref = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    rtr.rtr_sketch(plan, X, Yref)
    torch.cuda.synchronize()
    for call in range(2):                      # the scratch keeps the last call's contents
        for n, view in _views(dims):
            Y = torch.full((dims[n], K[n]), float("nan"), dtype=torch.float64, device="cuda")
            rtr.rtr_sketch_mode_noalloc(prec, X, view, K[n], seed, n, Y)
            torch.cuda.synchronize()
            ref = Yref[n].cpu().numpy()
            got = Y.cpu().numpy()
            assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (call, n)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    X = torch.zeros(4, dtype=torch.float32, device="cuda")
    Y = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_sketch_mode_noalloc("fp32", X, (1, 40000, 1), 64, 0, 0, Y)   # I*K = 2.56e6 > 2^21
    assert e.value.status == rtr.RTR_EINVAL and "static scratch" in str(e.value)
    with pytest.raises(rtr.RtrError):
        rtr.rtr_sketch_mode_noalloc("fp32", X, (1, 4, 1), 65, 0, 0, Y)
