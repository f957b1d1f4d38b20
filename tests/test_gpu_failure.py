"""Failure detection on the GPU without a GPU fault.

* A bounded device wait that runs out: a test kernel waits on an mbarrier
  that nothing completes, with the library's own bounded wait and a 2 ms
  limit; the call returns RTR_ETIMEOUT, the device flag holds
  RTR_FLAG_TIMEOUT, and the context still runs a sketch correctly.
* Non-finite input: a NaN or an Inf in X makes ||X||^2 non-finite, which
  the sketch's norm reduction reports as RTR_FLAG_NONFINITE.
"""
import time

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _bf16_sketch_matches_oracle():
    dims, K = (20, 130, 36), (6, 8, 6)
    X32 = np.random.default_rng(5).standard_normal(dims).astype(np.float32)
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2), rtr.make_params("bf16", 11))
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    rtr.rtr_sketch(plan, torch.from_numpy(X32).cuda(), Y)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    ref = orc.sketch(X32.astype(np.float64), K, 11, "bf16")
    for n in range(3):
        assert rel(Y[n].cpu().numpy(), ref[n]) < 2e-5, n


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    st = rtr.rtr_test_bounded_wait(2000, flags)
    el = time.perf_counter() - t
    assert st == rtr.RTR_ETIMEOUT
    assert int(flags.cpu()[0]) & rtr.FLAG_TIMEOUT
    assert el < 1.0                     # the 2 ms limit, not the kernels' 2 s
    # the context is intact: tensor-core kernels (with their own bounded
    # waits) still give the oracle's sketch, and raise no flag
    _bf16_sketch_matches_oracle()
    # a second expiry behaves the same
    flags.zero_()
    assert rtr.rtr_test_bounded_wait(500, flags) == rtr.RTR_ETIMEOUT


def test_bounded_wait_rejects_bad_limits():
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert rtr.rtr_test_bounded_wait(0, flags) == rtr.RTR_EINVAL
    assert rtr.rtr_test_bounded_wait(3000000, flags) == rtr.RTR_EINVAL
    assert int(flags.cpu()[0]) == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp8"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_nonfinite_x_raises_the_flag(prec, bad):
    dims, K = (24, 40, 32), (5, 6, 4)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.from_numpy(np.random.default_rng(6).standard_normal(dims)).to(dt).cuda()
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2), rtr.make_params(prec, 3))
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    rtr.rtr_sketch(plan, X, Y)
    assert rtr.rtr_plan_flags(plan) == 0          # a clean X raises nothing
    X[3, 17, 9] = bad
    rtr.rtr_sketch(plan, X, Y)
    assert rtr.rtr_plan_flags(plan) & rtr.FLAG_NONFINITE
    assert rtr.rtr_plan_flags(plan) == 0          # reading clears the flags
