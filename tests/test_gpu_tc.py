"""GPU parity of the BF16 (tcgen05, hi+lo split) path against the FP64 oracle.

X is float32 on both sides; Omega is the bfloat16-rounded table on both
sides.  The only differences are the hi+lo representation of X (relative
error <= 2^-16 per element) and FP32 accumulation, so the sketch matches the
oracle to ~1e-5 and the end-to-end reconstruction to the 1e-3 gate."""
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


TC_CASES = [
    ((40, 48, 44, 52), (10, 10, 10, 10)),     # vector paths; last mode transposed (I % 4 == 0)
    ((257, 19, 6), (64, 7, 5)),              # I > 256: two row groups; K = 64; B % 4 != 0 (scalar)
    ((9, 130, 7, 33), (5, 40, 3, 20)),       # ragged chunks (B < 64), I = 130 (two M tiles, one partial)
    ((6, 5, 301), (3, 4, 21)),               # last mode with I % 4 != 0 (scalar transpose path)
    ((3, 128, 512), (2, 32, 31)),            # B % 64 == 0 vector path, exactly one M tile
    ((5, 300, 36), (3, 40, 7)),              # TMA path: I = 300 (three row groups), B = 36 < 64 (ragged)
]


LAST_MODE_CASES = [
    ((300, 200), (7, 25)),                    # I = 200: two M tiles, the second ragged; A = 300 (ragged chunk)
    ((2, 3, 5, 64), (1, 2, 4, 20)),           # I = 64: one M tile, half of it past I; A = 30 < 64
    ((97, 300), (5, 33)),                     # I = 300: two row blocks (256 + 44), N = 64
    ((130, 128), (9, 64)),                    # I = 128 exactly one M tile, K = 64
]


PAIR = [pytest.param(rtr.PARAM_PAIR, id="pair"), pytest.param(0, id="per_mode")]


@pytest.mark.parametrize("flags", PAIR)
@pytest.mark.parametrize("dims,K", LAST_MODE_CASES)
def test_bf16_last_mode_tma_sketch_vs_oracle(dims, K, flags):
    """The last mode through the TMA sketch with an MN-major operand: boxes of
    64 rows x 64 columns, zero-filled past I and past A (per_mode), or from the
    tiles of the two-mode pass (pair)."""
    dims = tuple(dims)
    full = dims if len(dims) >= 3 else (1,) + dims
    Kf = K if len(K) >= 3 else (1,) + tuple(K)
    X32 = np.random.default_rng(25).standard_normal(full).astype(np.float32)
    plan = rtr.rtr_plan_create(full, Kf, (2,) * len(full), rtr.make_params("bf16", 79, flags=flags))
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") if pr else None
         for d, k, pr in zip(plan.dims, plan.K, plan.projected)]
    rtr.rtr_sketch(plan, torch.from_numpy(X32).cuda(), Y)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    ref = orc.sketch(X32.astype(np.float64), Kf, 79, "bf16")
    n = len(full) - 1
    assert rel(Y[n].cpu().numpy(), ref[n]) < 2e-5


@pytest.mark.parametrize("flags", PAIR)
@pytest.mark.parametrize("dims,K", TC_CASES)
def test_bf16_sketch_vs_oracle(dims, K, flags):
    X32 = np.random.default_rng(21).standard_normal(dims).astype(np.float32)
    plan = rtr.rtr_plan_create(dims, K, (2,) * len(dims),
                               rtr.make_params("bf16", 77, 3, 1e-2, orc.default_chain_order(dims, K), flags=flags))
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") if pr else None
         for d, k, pr in zip(plan.dims, plan.K, plan.projected)]
    rtr.rtr_sketch(plan, torch.from_numpy(X32).cuda(), Y)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    ref = orc.sketch(X32.astype(np.float64), K, 77, "bf16")
    for n in range(len(dims)):
        if ref[n] is not None:
            assert rel(Y[n].cpu().numpy(), ref[n]) < 2e-5, n


def test_bf16_sketch_records_norm():
    dims, K = (40, 48, 44, 52), (10, 10, 10, 10)
    X32 = np.random.default_rng(22).standard_normal(dims).astype(np.float32)
    from paper_1901_01652_gb300.api import RTRD
    eng = RTRD(dims, K, (2,) * 4, "bf16", 5, 2)
    Xd = torch.from_numpy(X32).cuda()
    eng.sketch(Xd)
    eng.project(Xd)
    eng.als()
    eng.compute_rse()
    torch.cuda.synchronize()
    # rse^2 = (||X||^2 - ||P||^2 + e^2)/||X||^2 must be a valid fraction
    r = float(eng.rse.cpu()[0])
    assert 0.0 < r <= 1.0


def test_bf16_end_to_end_vs_oracle():
    dims, K, R = (48, 40, 44, 52), (10, 10, 10, 10), (3, 3, 3, 3)
    S = ot.tr_full(workloads.tr_cores(dims, R, 31))
    X32 = (S + workloads.snr_sigma(ot.fro(S), S.size, 30.0) * workloads.unit_noise(dims, 31)).astype(np.float32)
    init = workloads.als_init(K, R, 32)
    ref = orc.rtrd(X32.astype(np.float64), K, R, "als", seed=33, prec="bf16", sweeps=10, init=init)
    from paper_1901_01652_gb300.api import RTRD
    eng = RTRD(dims, K, R, "bf16", 33, 10, chain_order=orc.default_chain_order(dims, K))
    eng.run(torch.from_numpy(X32).cuda(), "als", init=[torch.from_numpy(z) for z in init])
    Xh = eng.reconstruct("fp64").cpu().numpy()
    assert rel(Xh, ot.tr_full(ref["G"])) <= 1e-3


@pytest.mark.parametrize("dims,K", [((40, 48, 44, 52), (10, 10, 10, 10)),   # last mode first, vector loads
                                    ((7, 9, 11, 203), (3, 4, 5, 60)),        # I = 203 (scalar path), N = 64
                                    ((30, 17, 256), (5, 6, 25)),             # I = 256: two full 128-wide units
                                    ((12, 10, 132), (5, 4, 20)),             # I = 132: three K atoms, the last unit half empty
                                    ((9, 8, 5, 100), (4, 4, 3, 30)),         # I = 100: one unit, two atoms
                                    ((16, 12, 200), (6, 5, 40))])            # I = 200, K = 40 (N = 64: two slots)
def test_bf16_chain_vs_oracle(dims, K):
    """rtr_project on a BF16 plan (tensor-core first product) from the oracle's Y."""
    X32 = np.random.default_rng(23).standard_normal(dims).astype(np.float32)
    X = X32.astype(np.float64)
    order = orc.default_chain_order(dims, K)
    plan = rtr.rtr_plan_create(dims, K, (2,) * len(dims), rtr.make_params("bf16", 3, 2, 1e-2, order))
    Yr = orc.sketch(X, K, 3, "bf16")
    Yd = [None if y is None else torch.from_numpy(y).cuda() for y in Yr]
    Q = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(plan.dims, plan.K)]
    P = torch.zeros(plan.K, dtype=torch.float32, device="cuda")
    rtr.rtr_project(plan, torch.from_numpy(X32).cuda(), Yd, Q, P)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    Pr = orc.project(X, [orc.orth(y) for y in Yr], order)
    assert rel(P.cpu().numpy(), Pr) < 3e-5


def test_bf16_sketch_and_chain_at_the_200x4_kernel_configurations():
    """The kernels of the 200^4 benchmark at its own launch configurations, on
    a 200 x 8 x 200 x 200 tensor (K = 25; mode 1, I = 8 < K, is kept whole):
    mode 0 (view 1 x 200 x 320000) runs the TMA sketch with two M tiles and
    full 64-wide chunks, as modes 0 and 1 of 200^4 do; mode 2 (1600 x 200 x
    200) runs it with 64-wide chunks whose last one per b-run is ragged (8 of
    64), as mode 2 of 200^4 does; mode 3 runs the last-mode TMA sketch (MN-major
    operand) at I = 200; the chain starts with the last mode's product on the
    tensor cores at I = 200, K = 25."""
    dims, K = (200, 8, 200, 200), (25, 25, 25, 25)
    X32 = np.random.default_rng(24).standard_normal(dims).astype(np.float32)
    X = X32.astype(np.float64)
    order = orc.default_chain_order(dims, K)
    assert order[0] == 3
    plan = rtr.rtr_plan_create(dims, K, (10,) * 4, rtr.make_params("bf16", 1903, 3, 1e-2, order))
    Xd = torch.from_numpy(X32).cuda()
    Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") if pr else None
         for d, k, pr in zip(plan.dims, plan.K, plan.projected)]
    rtr.rtr_sketch(plan, Xd, Y)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    Yr = orc.sketch(X, K, 1903, "bf16")
    assert Yr[1] is None
    for n in (0, 2, 3):
        assert rel(Y[n].cpu().numpy(), Yr[n]) < 2e-5, n
    # the chain from the oracle's sketches
    Yd = [None if y is None else torch.from_numpy(y).cuda() for y in Yr]
    Q = [torch.zeros((d, k), dtype=torch.float64, device="cuda") for d, k in zip(plan.dims, plan.K)]
    P = torch.zeros(plan.K, dtype=torch.float32, device="cuda")
    rtr.rtr_project(plan, Xd, Yd, Q, P)
    torch.cuda.synchronize()
    assert rtr.rtr_plan_flags(plan) == 0
    Pr = orc.project(X, [np.eye(d) if y is None else orc.orth(y) for d, y in zip(dims, Yr)], order)
    assert rel(P.cpu().numpy(), Pr) < 3e-5


PAIR_CASES = [
    ((7, 200, 200), (5, 25, 25)),            # I = J = 200: two i tiles and two j tiles, both ragged
    ((3, 130, 180), (2, 40, 20)),            # second i tile 2 rows; last j tile 52 wide (one box); N = 64 / 32
    ((2, 2, 64, 1024), (1, 1, 30, 31)),      # eight j tiles, 32 chunks: one chunk per CTA
    ((40, 36, 44), (5, 9, 11)),              # one i tile of 36 rows, one box of 44 j
    ((5, 4, 136, 200), (3, 3, 64, 64)),      # K = 64 for both (two X slots, 96 KB of Omega rings)
    ((4, 300, 100), (3, 20, 12)),            # three i tiles (the mode N-1 Omega group holds 384 rows)
    ((1000, 20, 8), (9, 7, 5)),              # many chunks per CTA, J = 8
]


@pytest.mark.parametrize("dims,K", PAIR_CASES)
def test_bf16_pair_sketch_vs_oracle(dims, K):
    """The last two modes from one pass over X (sketch_pair_kernel) against the
    oracle, and against the per-mode passes on the GPU; the pass count says
    which path ran."""
    X32 = np.random.default_rng(31).standard_normal(dims).astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    out = {}
    for flags in (rtr.PARAM_PAIR, 0):
        plan = rtr.rtr_plan_create(dims, K, (2,) * len(dims), rtr.make_params("bf16", 83, flags=flags))
        nproj = sum(plan.projected)
        assert rtr.rtr_plan_sketch_passes(plan) == (nproj - 1 if flags else nproj)
        Y = [torch.zeros((d, k), dtype=torch.float64, device="cuda") if pr else None
             for d, k, pr in zip(plan.dims, plan.K, plan.projected)]
        rtr.rtr_sketch(plan, Xd, Y)
        torch.cuda.synchronize()
        assert rtr.rtr_plan_flags(plan) == 0
        out[flags] = [y.cpu().numpy() if y is not None else None for y in Y]
    ref = orc.sketch(X32.astype(np.float64), K, 83, "bf16")
    for n in range(len(dims)):
        if ref[n] is None:
            continue
        assert rel(out[rtr.PARAM_PAIR][n], ref[n]) < 2e-5, n
        assert rel(out[rtr.PARAM_PAIR][n], out[0][n]) < 1e-5, n


def test_sketch_passes_by_precision():
    """Only BF16 plans that ask for it take the two-mode pass; FP32, FP64 and
    FP8 plans read X once per projected mode, and so does a BF16 plan without
    the flag or whose last mode is whole or has I_N % 4 != 0."""
    dims, K, pair = (30, 40, 48), (10, 10, 10), rtr.PARAM_PAIR
    for prec, flags, want in (("bf16", pair, 2), ("bf16", 0, 3), ("fp32", pair, 3), ("fp64", pair, 3),
                              ("fp8", pair, 3)):
        plan = rtr.rtr_plan_create(dims, K, (2, 2, 2), rtr.make_params(prec, 1, flags=flags))
        assert rtr.rtr_plan_sketch_passes(plan) == want, (prec, flags)
    assert rtr.rtr_plan_sketch_passes(rtr.rtr_plan_create((30, 40, 48), (10, 10, 48), (2, 2, 2),
                                                          rtr.make_params("bf16", 1, flags=pair))) == 2
    assert rtr.rtr_plan_sketch_passes(rtr.rtr_plan_create((30, 40, 50), (10, 10, 10), (2, 2, 2),
                                                          rtr.make_params("bf16", 1, flags=pair))) == 3
