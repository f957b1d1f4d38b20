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
