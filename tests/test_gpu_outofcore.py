"""The out-of-core projection (rtr_project_host: X in host memory, streamed
in slabs of mode 0, twice) against the in-memory path and the oracle."""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _order_mode0_last(dims, K):
    o = [n for n in orc.default_chain_order(dims, K) if n != 0]
    return o + [0]


def _buffers(dims, K):
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    Q = [torch.zeros((d, min(k, d)), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    return Y, Q


@pytest.mark.parametrize("prec,slab,tolY,tolP", [
    ("fp64", 8, 1e-12, 1e-11),     # 37 = 4 x 8 + 5: a ragged last slab
    ("fp64", 37, 1e-12, 1e-11),    # one slab
    ("fp32", 7, 2e-6, 2e-6),
    ("bf16", 8, 2e-5, 3e-5),       # tensor-core sketches of the slabs (TMA and last-mode paths)
    ("fp8", 8, 2e-5, 3e-5),        # 8 x 20 x 18 = 2880 = 90 whole scale blocks per slab
])
def test_project_host_vs_in_memory_and_oracle(prec, slab, tolY, tolP):
    dims, K = (37, 20, 18, 24), (6, 5, 4, 7)
    X = np.random.default_rng(70).standard_normal(dims)
    if prec != "fp64":
        X = X.astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == "fp64" else torch.float32
    order = _order_mode0_last(dims, K)
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2, 2), rtr.make_params(prec, 71, chain_order=order))
    Xh = torch.from_numpy(X).to(dt).pin_memory()
    row = int(np.prod(dims[1:]))
    stage = [torch.empty(slab * row, dtype=dt, device="cuda") for _ in range(2)]
    Y, Q = _buffers(dims, K)
    P = torch.zeros(K, dtype=dt, device="cuda")
    rtr.rtr_project_host(plan, Xh, slab, stage, Y, Q, P)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    # the same plan in memory
    Xd = Xh.cuda()
    Y2, Q2 = _buffers(dims, K)
    P2 = torch.zeros(K, dtype=dt, device="cuda")
    rtr.rtr_sketch(plan, Xd, Y2)
    rtr.rtr_project(plan, Xd, Y2, Q2, P2)
    torch.cuda.synchronize()
    tab = {"fp64": "fp64", "fp32": "fp32", "bf16": "bf16", "fp8": "fp8"}[prec]
    Yr = orc.sketch(X, K, 71, tab)
    for n in range(4):
        assert rel(Y[n].cpu().numpy(), Y2[n].cpu().numpy()) < tolY, n
        assert rel(Y[n].cpu().numpy(), Yr[n]) < tolY, n
    Pr = orc.project(X, [orc.orth(y) for y in Yr], order)
    assert rel(P.cpu().numpy(), P2.cpu().numpy()) < tolP
    assert rel(P.cpu().numpy(), Pr) < tolP


def test_project_host_unprojected_mode0_and_rse():
    """Mode 0 kept whole (K_0 >= I_0): the slabs' rows of P are their
    intermediates; the recorded ||X||^2 feeds the RSE identity."""
    dims, K, R = (9, 26, 20, 24), (12, 6, 5, 6), (2, 2, 2, 2)
    S = ot.tr_full(workloads.tr_cores(dims, R, 72))
    X = S + workloads.snr_sigma(ot.fro(S), S.size, 30.0) * workloads.unit_noise(dims, 72)
    order = _order_mode0_last(dims, K)
    plan = rtr.rtr_plan_create(dims, K, R, rtr.make_params("fp64", 73, 5, chain_order=order))
    Xh = torch.from_numpy(X).pin_memory()
    stage = [torch.empty(4 * 26 * 20 * 24, dtype=torch.float64, device="cuda") for _ in range(2)]
    Y, Q = _buffers(dims, K)
    Keff = orc.effective_K(dims, K)
    P = torch.zeros(Keff, dtype=torch.float64, device="cuda")
    rtr.rtr_project_host(plan, Xh, 4, stage, Y, Q, P)
    torch.cuda.synchronize()
    Yr = orc.sketch(X, K, 73)
    Qr = [np.eye(9)] + [orc.orth(y) for y in Yr[1:]]
    Pr = orc.project(X, Qr, order)
    assert rel(P.cpu().numpy(), Pr) < 1e-11
    init = workloads.als_init(Keff, R, 74)
    Z = [torch.from_numpy(z).cuda() for z in init]
    rtr.rtr_als(plan, P, Z, True)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rtr.rtr_rse(plan, P, Z, out)
    torch.cuda.synchronize()
    ref = orc.tr_als(Pr, R, 5, init=init)[0]
    assert abs(float(out.cpu()[0]) - orc.rse_identity(ot.fro(X) ** 2, Pr, ref)) < 1e-9


def test_project_host_rejects_bad_arguments():
    dims, K = (10, 12, 9), (3, 3, 3)
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2), rtr.make_params("fp64", 1, chain_order=(0, 1, 2)))
    Xh = torch.zeros(dims, dtype=torch.float64)
    stage = [torch.empty(4 * 12 * 9, dtype=torch.float64, device="cuda") for _ in range(2)]
    Y, Q = _buffers(dims, K)
    P = torch.zeros(K, dtype=torch.float64, device="cuda")
    with pytest.raises(rtr.RtrError) as e:           # chain order does not end with mode 0
        rtr.rtr_project_host(plan, Xh, 4, stage, Y, Q, P)
    assert e.value.status == rtr.RTR_EINVAL
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2), rtr.make_params("fp64", 1, chain_order=(1, 2, 0)))
    with pytest.raises(rtr.RtrError):                # stage buffers too small for 5 rows
        rtr.rtr_project_host(plan, Xh, 5, stage, Y, Q, P)
