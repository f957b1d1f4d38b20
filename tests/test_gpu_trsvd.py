"""GPU TR-SVD (Algorithm 1 step 9, second decomposer) against the oracle."""
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


def noisy_tr(dims, R, snr_db, seed):
    S = ot.tr_full(workloads.tr_cores(dims, R, seed))
    return S + workloads.snr_sigma(ot.fro(S), S.size, snr_db) * workloads.unit_noise(dims, seed)


def gpu_trsvd(P, eps, prec, cap, ranks=None):
    dims = P.shape
    N = len(dims)
    plan = rtr.rtr_plan_create(dims, dims, cap, rtr.make_params(prec, 1, 1, eps))
    dt = torch.float64 if prec == "fp64" else torch.float32
    Z = [torch.zeros(cap[n] * dims[n] * cap[(n + 1) % N], dtype=torch.float64, device="cuda") for n in range(N)]
    try:
        rk = rtr.rtr_svd(plan, torch.from_numpy(np.ascontiguousarray(P)).to(dt).cuda(), eps, Z, ranks)
    except rtr.RtrError as e:
        raise
    torch.cuda.synchronize()
    cores = [Z[n][: rk[n] * dims[n] * rk[(n + 1) % N]].cpu().numpy().reshape(rk[n], dims[n], rk[(n + 1) % N])
             for n in range(N)]
    return cores, rk


# Parity of the cores' reconstruction needs a spectral gap at every chosen
# rank (otherwise the retained subspace is not determined by the data and two
# correct SVDs may differ): near-noiseless TR tensors give that gap.
@pytest.mark.parametrize("dims,R,eps", [((12, 10, 9), (2, 3, 2), 1e-3), ((7, 8, 6, 5), (2, 2, 3, 2), 1e-3),
                                        ((20, 16, 12), (2, 2, 2), 1e-3), ((10, 12, 8, 6), (2, 2, 2, 2), 1e-3)])
def test_trsvd_fp64_free_ranks_vs_oracle(dims, R, eps):
    P = noisy_tr(dims, R, 100.0, 40)
    Zr, rr = orc.tr_svd(P, eps)
    assert max(rr) <= 16, rr            # the case must fit the plan's core capacity
    Zg, rg = gpu_trsvd(P, eps, "fp64", [16] * len(dims))
    assert rg == rr
    Xg, Xr = ot.tr_full(Zg), ot.tr_full(Zr)
    # FP64 plans: one-sided Jacobi SVD on the GPU, LAPACK in the oracle, the
    # same sign rule on both sides; the FP64 gate
    assert rel(Xg, Xr) < 1e-10
    assert ot.fro(P - Xg) <= eps * ot.fro(P) * (1 + 1e-9)


@pytest.mark.parametrize("dims,R,eps,snr", [((12, 10, 9), (2, 3, 2), 0.05, 35.0), ((7, 8, 6, 5), (2, 2, 3, 2), 0.1, 35.0)])
def test_trsvd_noisy_meets_the_published_bound(dims, R, eps, snr):
    """Without a spectral gap only the guarantee ||P - TR(Z)|| <= eps ||P|| and
    the rank choice are comparable."""
    P = noisy_tr(dims, R, snr, 40)
    _, rr = orc.tr_svd(P, eps)
    Zg, rg = gpu_trsvd(P, eps, "fp64", [16] * len(dims))
    assert rg == rr
    assert ot.fro(P - ot.tr_full(Zg)) <= eps * ot.fro(P) * (1 + 1e-9)


def test_trsvd_forced_ranks_and_fp32():
    dims, R = (16, 12, 10, 8), (2, 3, 2, 2)
    P = noisy_tr(dims, R, 100.0, 41)
    Zr, rr = orc.tr_svd(P, 1e-3)
    Zg, rg = gpu_trsvd(P, 1e-3, "fp64", [16] * 4, ranks=rr)
    assert rg == rr
    assert rel(ot.tr_full(Zg), ot.tr_full(Zr)) < 1e-10
    P32 = P.astype(np.float32)
    Zr32, rr32 = orc.tr_svd(P32.astype(np.float64), 1e-3)
    Zg32, _ = gpu_trsvd(P32, 1e-3, "fp32", [16] * 4, ranks=rr32)
    assert rel(ot.tr_full(Zg32), ot.tr_full(Zr32)) < 1e-5


def test_trsvd_large_gram_side_both_eigen_paths():
    """A 120-long first mode: 120 vectors in the FP64 plan's Jacobi SVD (60
    rotation pairs per round) and a 120 x 120 Gram matrix in the float plan's
    shared-memory float32 eigensolver."""
    dims, R = (120, 24, 20), (2, 3, 2)
    P = noisy_tr(dims, R, 100.0, 43)
    Zr, rr = orc.tr_svd(P, 1e-3)
    Zg, rg = gpu_trsvd(P, 1e-3, "fp64", [16] * 3)
    assert rg == rr
    assert rel(ot.tr_full(Zg), ot.tr_full(Zr)) < 1e-10
    P32 = P.astype(np.float32)
    Zr32, rr32 = orc.tr_svd(P32.astype(np.float64), 1e-3)
    Zg32, _ = gpu_trsvd(P32, 1e-3, "fp32", [16] * 3, ranks=rr32)
    assert rel(ot.tr_full(Zg32), ot.tr_full(Zr32)) < 1e-4


def test_trsvd_exact_recovery_small_rank():
    """A noiseless TR: the Jacobi SVD leaves singular values of about u ||P||
    in the null space, so a tolerance of 1e-9 (far below sqrt(u)) still finds
    the exact ranks, and the reconstruction is P to float64 accuracy."""
    dims, R = (9, 8, 7), (2, 2, 2)
    P = ot.tr_full(workloads.tr_cores(dims, R, 42))
    Zr, rr = orc.tr_svd(P, 1e-9)
    Zg, rg = gpu_trsvd(P, 1e-9, "fp64", [8, 8, 8])
    assert rg == rr and rg[0] * rg[1] == 4
    assert rel(ot.tr_full(Zg), P) < 1e-12
    assert rel(ot.tr_full(Zg), ot.tr_full(Zr)) < 1e-10


def test_rtrsvd_bf16_end_to_end_hsi_shaped():
    """rTR-SVD on a small hyperspectral-shaped tensor: BF16 sketch/chain, TR-SVD
    with the oracle's ranks forced, reconstruction vs the oracle <= 1e-3."""
    A, S = workloads.hsi_factors(64, 48, 32, n_sig=6, n_bumps=8, seed=43)
    X = np.einsum("hws,bs->hwb", A, S)
    X = X + 0.01 * ot.fro(X) / np.sqrt(X.size) * workloads.unit_noise(X.shape, 44)
    X32 = X.astype(np.float32)
    K = (12, 12, 8)
    ref = orc.rtrd(X32.astype(np.float64), K, None, "svd", seed=45, prec="bf16", eps=0.005)
    assert ref["ranks"] == [1, 2, 4]
    from paper_1901_01652_gb300.api import RTRD
    eng = RTRD(X.shape, K, (16, 16, 16), "bf16", 45, 1, 0.005, chain_order=orc.default_chain_order(X.shape, K))
    eng.run(torch.from_numpy(X32).cuda(), "svd", ranks=ref["ranks"])
    Xh = eng.reconstruct("fp64").cpu().numpy()
    assert rel(Xh, ot.tr_full(ref["G"])) <= 1e-3
