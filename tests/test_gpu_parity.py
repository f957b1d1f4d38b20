"""GPU parity: every step of Algorithm 1 through the C ABI against the FP64
oracle on the same seeded inputs (SIMT FP64 and FP32 paths)."""
import numpy as np
import pytest
import torch

from oracle import omega as oom
from oracle import rtrd as orc
from oracle import tensor as ot
from paper_1901_01652_gb300 import rtr, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()
    torch.cuda.init()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def noisy_tr(dims, R, snr_db, seed):
    S = ot.tr_full(workloads.tr_cores(dims, R, seed))
    return S + workloads.snr_sigma(ot.fro(S), S.size, snr_db) * workloads.unit_noise(dims, seed)


def make_plan(dims, K, R, prec, seed=7, sweeps=5, order=None):
    if order is None:
        order = orc.default_chain_order(dims, K)
    return rtr.rtr_plan_create(dims, K, R, rtr.make_params(prec, seed, sweeps, 1e-2, order))


def gpu_sketch(plan, X):
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") if pr else None
         for d, k, pr in zip(plan.dims, plan.K, plan.projected)]
    rtr.rtr_sketch(plan, X, Y)
    torch.cuda.synchronize()
    return [None if y is None else y.cpu().numpy() for y in Y]


# ------------------------------------------------------------------ Omega

@pytest.mark.parametrize("prec,tabprec", [("fp64", "fp64"), ("fp32", "bf16")])
def test_omega_bit_exact(prec, tabprec):
    plan = make_plan((50, 40, 30), (43, 7, 20), (2, 2, 2), prec, seed=123456789)
    for mode, row0, nrows, K in ((0, 0, 1200, 43), (2, 100, 500, 7), (1, 1499, 1, 20)):
        out = torch.empty((nrows, K), dtype=torch.float64, device="cuda")
        rtr.rtr_draw_omega(plan, mode, row0, nrows, K, out)
        ref = oom.omega(123456789, mode, nrows, K, tabprec, row0=row0)
        got = out.cpu().numpy()
        if tabprec == "bf16":
            assert np.array_equal(got, ref)
        else:
            # the two float64 tables are computed independently and agree to
            # ~1 ulp; adjacent table entries are >= 6e-4 apart, so this bound
            # also proves every Philox index matches
            assert np.max(np.abs(got - ref)) < 2e-15


def test_default_chain_order_matches_rule():
    for dims, K in (((200, 200, 200, 200), (25,) * 4), ((1024, 1024, 256), (60, 60, 30)), ((9, 5, 7), (3, 9, 2))):
        plan = rtr.rtr_plan_create(dims, K, (2,) * len(dims), rtr.make_params("fp64"))
        assert list(plan.order) == orc.default_chain_order(dims, K)
        assert list(plan.K) == orc.effective_K(dims, K)


# ------------------------------------------------------------------ sketch

SKETCH_CASES = [
    ((7, 37, 5, 11), (3, 5, 2, 4)),          # ragged, below one tile
    ((33, 65, 3), (5, 9, 64)),               # last mode unprojected (K >= I)
    ((3, 4, 300, 5, 2), (2, 3, 40, 2, 1)),   # order 5, K spanning 2 Philox calls
    ((257, 19, 6), (64, 7, 5)),              # I > one row tile (two CTA rows), K = 64
]


@pytest.mark.parametrize("dims,K", SKETCH_CASES)
def test_sketch_fp64_vs_oracle(dims, K):
    X = np.random.default_rng(1).standard_normal(dims)
    plan = make_plan(dims, K, (2,) * len(dims), "fp64", seed=11)
    Y = gpu_sketch(plan, dev(X))
    ref = orc.sketch(X, K, 11, "fp64")
    for n in range(len(dims)):
        if ref[n] is None:
            assert Y[n] is None
        else:
            assert rel(Y[n], ref[n]) < 1e-13, n


def test_sketch_fp64_60x4():
    X = noisy_tr((60, 60, 60, 60), 5, 40.0, 1902)
    plan = make_plan(X.shape, (15,) * 4, (5,) * 4, "fp64", seed=1902)
    Y = gpu_sketch(plan, dev(X))
    ref = orc.sketch(X, (15,) * 4, 1902, "fp64")
    for n in range(4):
        assert rel(Y[n], ref[n]) < 1e-13


@pytest.mark.parametrize("dims,K", SKETCH_CASES[:3] + [((40, 48, 44, 52), (10, 10, 10, 10))])
def test_sketch_fp32_vs_oracle(dims, K):
    X32 = np.random.default_rng(2).standard_normal(dims).astype(np.float32)
    plan = make_plan(dims, K, (2,) * len(dims), "fp32", seed=5)
    Y = gpu_sketch(plan, dev(X32, torch.float32))
    ref = orc.sketch(X32.astype(np.float64), K, 5, "fp32")
    for n in range(len(dims)):
        if ref[n] is not None:
            assert rel(Y[n], ref[n]) < 2e-6, n


def test_sketch_is_linear_and_scales():
    dims, K = (20, 30, 25), (6, 6, 6)
    rng = np.random.default_rng(3)
    X1, X2 = rng.standard_normal(dims), rng.standard_normal(dims)
    plan = make_plan(dims, K, (2, 2, 2), "fp64", seed=9)
    Ya = gpu_sketch(plan, dev(2.0 * X1 - 3.0 * X2))
    Y1 = gpu_sketch(plan, dev(X1))
    Y2 = gpu_sketch(plan, dev(X2))
    for n in range(3):
        assert rel(Ya[n], 2.0 * Y1[n] - 3.0 * Y2[n]) < 1e-13


# ------------------------------------------------------------------ QR + chain

def run_project(plan, X, Y):
    Yd = [None if y is None else dev(y) for y in Y]
    Q = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(plan.dims, plan.K)]
    P = torch.zeros(plan.K, dtype=plan.x_dtype, device="cuda")
    rtr.rtr_project(plan, X, Yd, Q, P)
    torch.cuda.synchronize()
    return [q.cpu().numpy() for q in Q], P.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dims,K", SKETCH_CASES + [((60, 60, 60, 60), (15,) * 4)])
def test_orth_and_chain_fp64(dims, K):
    X = np.random.default_rng(4).standard_normal(dims)
    plan = make_plan(dims, K, (2,) * len(dims), "fp64", seed=3)
    Yr = orc.sketch(X, K, 3, "fp64")
    Q, P = run_project(plan, dev(X), Yr)
    Qr = [np.eye(d) if y is None else orc.orth(y) for d, y in zip(dims, Yr)]
    for n in range(len(dims)):
        assert np.abs(Q[n] - Qr[n]).max() < 1e-12, n
        assert np.abs(Q[n].T @ Q[n] - np.eye(Q[n].shape[1])).max() < 1e-13
    Pr = orc.project(X, Qr, orc.default_chain_order(dims, K))
    assert rel(P, Pr) < 1e-12


def test_chain_order_does_not_change_P():
    dims, K = (30, 20, 25, 10), (7, 5, 6, 3)
    X = np.random.default_rng(5).standard_normal(dims)
    Yr = orc.sketch(X, K, 1, "fp64")
    ref = None
    for order in ([3, 2, 1, 0], [0, 1, 2, 3], [2, 0, 3, 1]):
        plan = make_plan(dims, K, (2,) * 4, "fp64", seed=1, order=order)
        _, P = run_project(plan, dev(X), Yr)
        ref = P if ref is None else ref
        assert rel(P, ref) < 1e-13


def test_orth_fallback_on_rank_deficient_sketch():
    rng = np.random.default_rng(6)
    dims, K = (40, 30, 20), (12, 5, 5)
    Y0 = rng.standard_normal((40, 4)) @ rng.standard_normal((4, 12))     # rank 4 < K = 12
    Yr = [Y0, rng.standard_normal((30, 5)), rng.standard_normal((20, 5))]
    plan = make_plan(dims, K, (2, 2, 2), "fp64")
    X = np.zeros(dims)
    Q, _ = run_project(plan, dev(X), Yr)
    flags = rtr.rtr_plan_flags(plan)
    assert flags & rtr.FLAG_QR_FALLBACK
    assert np.abs(Q[0].T @ Q[0] - np.eye(12)).max() < 1e-12
    assert np.linalg.norm(Y0 - Q[0] @ (Q[0].T @ Y0)) < 1e-12 * np.linalg.norm(Y0)
    assert np.abs(Q[1] - orc.orth(Yr[1])).max() < 1e-12


@pytest.mark.parametrize("dims,K", [((40, 48, 44, 52), (10, 10, 10, 10)), ((257, 19, 6), (64, 7, 5))])
def test_chain_fp32_vs_oracle(dims, K):
    X32 = np.random.default_rng(7).standard_normal(dims).astype(np.float32)
    X = X32.astype(np.float64)
    plan = make_plan(dims, K, (2,) * len(dims), "fp32", seed=2)
    Yr = orc.sketch(X, K, 2, "fp32")
    Q, P = run_project(plan, dev(X32, torch.float32), Yr)
    Qr = [orc.orth(y) for y in Yr]
    Pr = orc.project(X, Qr, orc.default_chain_order(dims, K))
    assert rel(P, Pr) < 2e-6


# ------------------------------------------------------------------ ALS

def run_als(plan, P, init, sweeps):
    Pd = dev(P, plan.x_dtype)
    Z = [dev(z) for z in init] if init is not None else \
        [torch.zeros((plan.R[n], plan.K[n], plan.R[(n + 1) % plan.N]), dtype=torch.float64, device="cuda")
         for n in range(plan.N)]
    err = torch.zeros(sweeps, dtype=torch.float64, device="cuda")
    rtr.rtr_als(plan, Pd, Z, init is not None, err)
    torch.cuda.synchronize()
    return [z.cpu().numpy() for z in Z], err.cpu().numpy()


@pytest.mark.parametrize("dims,R", [((15, 15, 15, 15), (5, 5, 5, 5)), ((9, 7, 8), (2, 3, 4)),
                                    ((6, 5, 7, 4, 5), (2, 2, 3, 2, 1)), ((25, 25, 25, 25), (10,) * 4)])
def test_als_fp64_vs_oracle(dims, R):
    P = noisy_tr(dims, R, 30.0, 8)
    init = workloads.als_init(dims, R, 9)
    sweeps = 4
    plan = make_plan(dims, dims, R, "fp64", sweeps=sweeps)
    Z, err = run_als(plan, P, init, sweeps)
    Zr, errs = orc.tr_als(P, R, sweeps, init=init)
    assert rel(ot.tr_full(Z), ot.tr_full(Zr)) < 1e-10
    assert np.max(np.abs(err - np.array(errs)) / np.array(errs)) < 1e-8


def test_als_default_init_vs_oracle():
    dims, R = (10, 9, 8, 7), (3, 2, 3, 2)
    P = noisy_tr(dims, R, 20.0, 10)
    plan = make_plan(dims, dims, R, "fp64", seed=42, sweeps=3)
    Z, _ = run_als(plan, P, None, 3)
    Zr, _ = orc.tr_als(P, R, 3, seed=42)
    assert rel(ot.tr_full(Z), ot.tr_full(Zr)) < 1e-10


def test_als_fp32_contraction_vs_oracle():
    dims, R = (25, 25, 25, 25), (10,) * 4
    P32 = noisy_tr(dims, R, 30.0, 11).astype(np.float32)
    init = workloads.als_init(dims, R, 12)
    plan = make_plan(dims, dims, R, "fp32", sweeps=5)
    Z, err = run_als(plan, P32, init, 5)
    Zr, errs = orc.tr_als(P32.astype(np.float64), R, 5, init=init)
    assert rel(ot.tr_full(Z), ot.tr_full(Zr)) < 1e-4
    assert np.max(np.abs(err - np.array(errs)) / np.array(errs)) < 1e-3


@pytest.mark.parametrize("dims,R", [
    ((12, 11, 13), (2, 3, 5)),                # order 3 (one outer core): R_{n+1} R_n = 15, 10, 6
    ((9, 8, 7, 10, 6), (2, 3, 2, 3, 1)),      # order 5: three outer cores per update
    ((40, 33, 37, 35), (12, 6, 9, 7)),        # K_n up to 40, R_{n+1} R_n up to 108 (eight items a thread)
    ((64, 20, 64, 5), (4, 16, 4, 3)),         # K_n = 64, R = 16
])
def test_als_fp32_fused_contraction_orders(dims, R):
    """The float32 plans form W = P_<n> S without storing the subchain; the
    TR-ALS result follows the oracle's for orders 3-5 and rank products
    that are not multiples of 4."""
    P32 = noisy_tr(dims, R, 30.0, 16).astype(np.float32)
    init = workloads.als_init(dims, R, 17)
    sweeps = 3
    plan = make_plan(dims, dims, R, "fp32", sweeps=sweeps)
    Z, err = run_als(plan, P32, init, sweeps)
    assert rtr.rtr_plan_flags(plan) & ~rtr.FLAG_GRAM_PINV == 0
    Zr, errs = orc.tr_als(P32.astype(np.float64), R, sweeps, init=init)
    assert rel(ot.tr_full(Z), ot.tr_full(Zr)) < 1e-4
    assert np.max(np.abs(err - np.array(errs)) / np.array(errs)) < 1e-3


# ------------------------------------------------------------------ back-projection, Psi, RSE

def test_backproject_and_reconstruct_vs_oracle():
    dims, K, R = (20, 17, 13), (6, 5, 4), (2, 3, 2)
    rng = np.random.default_rng(13)
    Zs = workloads.tr_cores(K, R, 14)
    Qs = [np.linalg.qr(rng.standard_normal((d, k)))[0] for d, k in zip(dims, K)]
    plan = make_plan(dims, K, R, "fp64")
    G = [torch.zeros((R[n], dims[n], R[(n + 1) % 3]), dtype=torch.float64, device="cuda") for n in range(3)]
    rtr.rtr_backproject(plan, [dev(z) for z in Zs], [dev(q) for q in Qs], G)
    Gr = orc.backproject(Zs, Qs)
    for g, gr in zip(G, Gr):
        assert np.abs(g.cpu().numpy() - gr).max() < 1e-13
    for out_prec, tol in (("fp64", 1e-13), ("fp32", 2e-6)):
        Xh = torch.zeros(dims, dtype=torch.float64 if out_prec == "fp64" else torch.float32, device="cuda")
        work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, R), dtype=torch.uint8, device="cuda")
        rtr.rtr_reconstruct(dims, R, [dev(g) for g in Gr], out_prec, Xh, work)
        assert rel(Xh.cpu().numpy(), ot.tr_full(Gr)) < tol


@pytest.mark.parametrize("dims,R", [((8, 9), (3, 2)), ((5, 6, 7, 4, 3), (2, 3, 1, 2, 2)), ((60, 60, 60, 60), (5,) * 4)])
def test_reconstruct_orders(dims, R):
    Gr = workloads.tr_cores(dims, R, 15)
    Xh = torch.zeros(dims, dtype=torch.float64, device="cuda")
    work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, R), dtype=torch.uint8, device="cuda")
    rtr.rtr_reconstruct(dims, R, [dev(g) for g in Gr], "fp64", Xh, work)
    assert rel(Xh.cpu().numpy(), ot.tr_full(Gr)) < 1e-13


# ------------------------------------------------------------------ end to end

def run_pipeline(X, K, R, prec, seed, sweeps, init):
    from paper_1901_01652_gb300.api import RTRD
    eng = RTRD(X.shape, K, R, prec, seed, sweeps, chain_order=orc.default_chain_order(X.shape, K))
    Xd = dev(X, eng.plan.x_dtype)
    eng.run(Xd, "als", init=[torch.from_numpy(z) for z in init])
    eng.compute_rse()
    Xh = eng.reconstruct("fp64").cpu().numpy()
    return eng, Xh


def test_end_to_end_fp64_60x4():
    """Config: 60^4 TR ranks 5, 40 dB, K = 15, R = 5, 20 sweeps, FP64: <= 1e-10."""
    cfg = workloads.CONFIGS["c1_fp64_60x4"]
    X = noisy_tr(cfg["dims"], cfg["tr_rank"], cfg["snr_db"], cfg["seed"])
    K, R = (cfg["K"],) * 4, (cfg["R"],) * 4
    init = workloads.als_init(orc.effective_K(X.shape, K), R, cfg["seed"])
    ref = orc.rtrd(X, K, R, "als", seed=cfg["seed"], sweeps=cfg["sweeps"], init=init)
    eng, Xh = run_pipeline(X, K, R, "fp64", cfg["seed"], cfg["sweeps"], init)
    Xr = ot.tr_full(ref["G"])
    assert rel(Xh, Xr) <= 1e-10
    rse_ref = orc.rse_identity(ot.fro(X) ** 2, ref["P"], ref["Z"])
    assert abs(float(eng.rse.cpu()[0]) - rse_ref) < 1e-9
    assert abs(orc.rse(X, Xr) - rse_ref) < 1e-9
    assert rtr.rtr_plan_flags(eng.plan) == 0


def test_end_to_end_fp32_40x4():
    dims, K, R = (40, 44, 36, 40), (10, 10, 10, 10), (3, 3, 3, 3)
    X32 = noisy_tr(dims, R, 30.0, 16).astype(np.float32)
    X = X32.astype(np.float64)
    init = workloads.als_init(K, R, 17)
    ref = orc.rtrd(X, K, R, "als", seed=18, prec="fp32", sweeps=10, init=init)
    eng, Xh = run_pipeline(X32, K, R, "fp32", 18, 10, init)
    assert rel(Xh, ot.tr_full(ref["G"])) <= 1e-3


# ------------------------------------------------------------------ argument errors

def test_argument_errors_are_reported():
    plan = make_plan((10, 11, 12), (3, 3, 3), (2, 2, 2), "fp64")
    X = torch.zeros((10, 11, 12), dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        rtr.rtr_sketch(plan, X.float(), [None] * 3)
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_sketch(plan, X, [None, None, None])
    assert e.value.status == rtr.RTR_EINVAL
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_draw_omega(plan, 5, 0, 1, 1, torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert e.value.status == rtr.RTR_EINVAL
