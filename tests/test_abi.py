"""C-ABI library: loads, exports every declared entry point, validates
arguments on the host, and its host-side Gaussian table equals the oracle's.
No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtr.h")


@pytest.fixture(scope="module")
def L():
    from paper_1901_01652_gb300 import build, rtr
    build.build()
    return rtr.lib()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rtr_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_entry_points():
    from paper_1901_01652_gb300 import rtr
    assert set(_declared()) == set(rtr.ENTRY_POINTS)


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_library_links_no_oracle_or_python():
    lib = os.path.join(ROOT, "paper_1901_01652_gb300", "librtr.so")
    data = open(lib, "rb").read()
    assert b"oracle" not in data
    assert b"libpython" not in data


def test_params_default(L):
    from paper_1901_01652_gb300 import rtr
    p = rtr.rtr_params_default()
    assert p.prec == rtr.RTR_FP32 and p.sweeps == 20 and abs(p.tol - 1e-2) < 1e-15
    assert list(p.chain_order) == [-1] * 8


def test_plan_create_rejects_bad_arguments_on_host(L):
    from paper_1901_01652_gb300 import rtr
    p = rtr.make_params("fp64")
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_plan_create((10, 10), (3, 3), (2, 2), p)            # N < 3
    assert e.value.status == rtr.RTR_EINVAL and "order" in str(e.value)
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_plan_create((10, 10, 10), (3, 3, 3), (2, 0, 2), p)  # rank 0
    assert e.value.status == rtr.RTR_EINVAL
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_plan_create((100, 100, 100), (65, 3, 3), (2, 2, 2), p)  # K > 64
    assert e.value.status == rtr.RTR_EINVAL
    bad = rtr.make_params("fp64")
    bad.prec = 9
    with pytest.raises(rtr.RtrError):
        rtr.rtr_plan_create((10, 10, 10), (3, 3, 3), (2, 2, 2), bad)
    bad = rtr.make_params("fp64", chain_order=[0, 0, 1])
    with pytest.raises(rtr.RtrError):
        rtr.rtr_plan_create((10, 10, 10), (3, 3, 3), (2, 2, 2), bad)


def test_library_table_equals_oracle_table(L):
    """The library computes its own quantile table (bisection on erfc); it must
    agree with the oracle's (scipy ndtri): float64 to rounding, bfloat16 exactly."""
    from oracle import omega
    from paper_1901_01652_gb300 import rtr
    t64 = rtr.rtr_gaussian_table("fp64")
    ref = omega.gaussian_table_fp64()
    # near the median x = Phi^-1(p) is ill-conditioned in relative terms, so the
    # two computations agree to rounding in absolute terms (entries are O(1))
    assert np.max(np.abs(t64 - ref)) < 2e-15
    assert np.array_equal(rtr.rtr_gaussian_table("bf16"), omega.gaussian_table("bf16"))
    assert np.array_equal(rtr.rtr_gaussian_table("fp32"), omega.gaussian_table("fp32"))
    # e4m3 rounding (subnormal grid below 2^-6, ties to even) written
    # independently on both sides
    assert np.array_equal(rtr.rtr_gaussian_table("fp8"), omega.gaussian_table("fp8"))


def test_propose_decoding_matches_oracle(L):
    """rtr_propose is host code: its decoding of a network output equals the
    oracle's (round half to even, clamps to [1, min(I_n, 64)] and [1, r_max])."""
    from oracle import proposer as op
    from paper_1901_01652_gb300 import rtr
    rng = np.random.default_rng(8)
    for _ in range(200):
        out = rng.uniform(-0.2, 1.3, 10).astype(np.float32)
        dims = tuple(int(x) for x in rng.integers(2, 120, size=int(rng.integers(3, 6))))
        assert rtr.rtr_propose(out, dims) == op.decode(out.astype(np.float64), dims)
    half = np.array([2.5 / 64, 0.5 / 16] * 5, dtype=np.float32)    # exact halves -> even
    assert rtr.rtr_propose(half, (100, 100, 100)) == op.decode(half.astype(np.float64), (100, 100, 100))
    with pytest.raises(rtr.RtrError):
        rtr.rtr_propose(half, (10,) * 6)                            # more than 5 modes


def test_proposer_sizes(L):
    from oracle import proposer as op
    from paper_1901_01652_gb300 import rtr
    assert rtr.rtr_mlp_param_count() == op.param_count()
    assert rtr.rtr_mlp_work_bytes(0) == 0
    assert rtr.rtr_mlp_work_bytes(100) >= 100 * (6 * 128 + 20) * 4


def test_batch_create_rejects_bad_arguments_on_host(L):
    from paper_1901_01652_gb300 import rtr
    p = rtr.make_params("fp32", 1, 2)
    with pytest.raises(ValueError):
        rtr.rtr_batch_create([], [], [], p)
    with pytest.raises(rtr.RtrError) as e:
        rtr.rtr_batch_create([(8, 8, 8)], [(4, 4, 4)], [(2, 2, 2)], p, nstreams=65)
    assert e.value.status == rtr.RTR_EINVAL
    p.chain_order[1] = 0
    with pytest.raises(rtr.RtrError):
        rtr.rtr_batch_create([(8, 8, 8)], [(4, 4, 4)], [(2, 2, 2)], p)


def test_noalloc_wrapper_refuses_a_view_that_does_not_match_the_buffers():
    """The C entry point cannot see buffer sizes: the binding checks the view
    (A, I, B) against X and I*K against Y before any launch."""
    import torch
    from paper_1901_01652_gb300 import rtr
    X = torch.zeros(4, dtype=torch.float32)
    Y = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="does not match X"):
        rtr.rtr_sketch_mode_noalloc("fp32", X, (1, 40000, 1), 64, 0, 0, Y)
    with pytest.raises(ValueError, match="I\\*K"):
        rtr.rtr_sketch_mode_noalloc("fp32", X, (1, 4, 1), 3, 0, 0, Y)


def test_host_queries_reject_null_arguments(L):
    """The host-only plan queries refuse a NULL plan or output pointer with
    RTR_EINVAL before touching the device."""
    from paper_1901_01652_gb300 import rtr
    n = ctypes.c_int(-1)
    assert L.rtr_plan_sketch_passes(None, ctypes.byref(n)) == rtr.RTR_EINVAL
    assert n.value == -1
    assert L.rtr_plan_info(None, None, None) == rtr.RTR_EINVAL
    assert rtr.PARAM_PAIR == 2 and rtr.PARAM_NO_GRAPH == 1
    assert rtr.make_params("bf16", 1, flags=rtr.PARAM_PAIR).flags == rtr.PARAM_PAIR
    assert rtr.make_params("bf16", 1).flags == 0
