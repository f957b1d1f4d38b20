"""GPU parity of the variants of the projection step against the oracle:
power iterations on the sketch (the remark after Algorithm 1) and the
sequential projection."""
import numpy as np
import pytest
import torch

from oracle import rtrd as orc
from oracle import tensor as ot
from paper_1901_01652_gb300 import rtr, workloads
from paper_1901_01652_gb300.api import RTRD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def noisy_tr(dims, R, snr, seed):
    S = ot.tr_full(workloads.tr_cores(dims, R, seed))
    return S + workloads.snr_sigma(ot.fro(S), S.size, snr) * workloads.unit_noise(dims, seed)


@pytest.mark.parametrize("q", [1, 2])
def test_power_iterations_fp64_vs_oracle(q):
    dims, K = (20, 24, 18, 22), (5, 6, 4, 5)
    X = noisy_tr(dims, (2, 3, 2, 2), 20.0, 50)
    plan = rtr.rtr_plan_create(dims, K, (2, 3, 2, 2), rtr.make_params("fp64", 51, power=q))
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    rtr.rtr_sketch(plan, torch.from_numpy(X).cuda(), Y)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    ref = orc.sketch_power(X, K, 51, q)
    for n in range(4):
        assert rel(Y[n].cpu().numpy(), ref[n]) < 1e-11, n


def test_power_iterations_fp64_end_to_end_and_unprojected_mode():
    dims, K, R = (16, 20, 6, 18), (5, 6, 8, 5), (2, 2, 2, 2)      # mode 2 kept whole
    X = noisy_tr(dims, R, 25.0, 52)
    init = workloads.als_init(orc.effective_K(dims, K), R, 53)
    ref = orc.rtrd(X, K, R, "als", seed=54, sweeps=6, init=init, power=1)
    eng = RTRD(dims, K, R, "fp64", 54, 6, power=1)
    eng.run(torch.from_numpy(X).cuda(), "als", init=[torch.from_numpy(z) for z in init])
    Xh = eng.reconstruct("fp64").cpu().numpy()
    assert rel(Xh, ot.tr_full(ref["G"])) < 1e-10


def test_power_iteration_bf16_end_to_end_vs_oracle():
    """BF16 plan, q = 1: the first sketch on the tensor cores, the power
    iteration's products (tensor-core last mode, SIMT others) and its
    contraction in float32; the reconstruction within the 1e-3 gate."""
    dims, K, R = (48, 40, 44, 52), (10, 10, 10, 10), (3, 3, 3, 3)
    X32 = noisy_tr(dims, R, 20.0, 55).astype(np.float32)
    X = X32.astype(np.float64)
    init = workloads.als_init(K, R, 56)
    ref = orc.rtrd(X, K, R, "als", seed=57, prec="bf16", sweeps=8, init=init, power=1)
    eng = RTRD(dims, K, R, "bf16", 57, 8, chain_order=orc.default_chain_order(dims, K), power=1)
    eng.run(torch.from_numpy(X32).cuda(), "als", init=[torch.from_numpy(z) for z in init])
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(eng.plan) == 0
    Xh = eng.reconstruct("fp64").cpu().numpy()
    assert rel(Xh, ot.tr_full(ref["G"])) <= 1e-3
    # and q = 1 is closer to X than the plain sketch at the same K (20 dB noise)
    ref0 = orc.rtrd(X, K, R, "als", seed=57, prec="bf16", sweeps=8, init=init)
    assert rel(ot.tr_full(ref["G"]), X) <= rel(ot.tr_full(ref0["G"]), X) + 1e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 3e-5), ("bf16", 5e-5)])
def test_sequential_projection_vs_oracle(prec, tol):
    dims, K = (30, 26, 20, 36), (6, 5, 4, 7)
    order = (3, 0, 2, 1)
    X = noisy_tr(dims, (2, 2, 2, 2), 20.0, 58)
    if prec != "fp64":
        X = X.astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2, 2), rtr.make_params(prec, 59, chain_order=order))
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    Q = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    P = torch.zeros(K, dtype=dt, device="cuda")
    rtr.rtr_project_sequential(plan, torch.from_numpy(X).to(dt).cuda(), Y, Q, P)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    Yr, Qr, Pr = orc.project_sequential(X, K, 59, order, "fp32" if prec != "fp64" else "fp64")
    for n in range(4):
        assert rel(Y[n].cpu().numpy(), Yr[n]) < tol, n
        Qg = Q[n].cpu().numpy()
        assert np.abs(Qg @ Qg.T - Qr[n] @ Qr[n].T).max() < 10 * tol, n
    assert rel(P.cpu().numpy(), Pr) < 10 * tol


def test_sequential_projection_bf16_end_to_end_and_rse():
    dims, K, R = (48, 40, 44, 52), (10, 10, 10, 10), (3, 3, 3, 3)
    X32 = noisy_tr(dims, R, 30.0, 60).astype(np.float32)
    X = X32.astype(np.float64)
    init = workloads.als_init(K, R, 61)
    order = orc.default_chain_order(dims, K)
    ref = orc.rtrd(X, K, R, "als", seed=62, prec="bf16", sweeps=8, init=init, sequential=True, order=order)
    eng = RTRD(dims, K, R, "bf16", 62, 8, chain_order=order, sequential=True)
    eng.run(torch.from_numpy(X32).cuda(), "als", init=[torch.from_numpy(z) for z in init])
    eng.compute_rse()
    torch.cuda.synchronize()
    Xh = eng.reconstruct("fp64").cpu().numpy()
    assert rel(Xh, ot.tr_full(ref["G"])) <= 1e-3
    # the RSE identity holds for the sequential projection too (orthonormal Q_n)
    assert abs(float(eng.rse.cpu()[0]) - rel(Xh, X)) < 1e-4


def test_sequential_projection_rejects_power_iterations():
    dims, K = (10, 12, 9), (3, 3, 3)
    plan = rtr.rtr_plan_create(dims, K, (2, 2, 2), rtr.make_params("fp64", 1, power=1))
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    Q = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(dims, K)]
    P = torch.zeros(K, dtype=torch.float64, device="cuda")
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_project_sequential(plan, torch.zeros(dims, dtype=torch.float64, device="cuda"), Y, Q, P)
    assert e.value.status == rtr.RTR_EINVAL
