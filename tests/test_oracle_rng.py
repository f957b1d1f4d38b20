"""Pins for the oracle's random test matrices (Algorithm 1, step 4)."""
import os

import numpy as np
import pytest
import torch

from oracle import omega
from oracle.philox import philox4x64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_kat.txt")


def _words(x):
    return [np.uint64((x >> (64 * i)) & ((1 << 64) - 1)) for i in range(4)]


def test_philox_matches_numpy_bit_generator():
    # numpy.random.Philox is an independent Philox4x64-10 implementation; it
    # increments its 256-bit counter before each block.
    rng = np.random.default_rng(5)
    for _ in range(20):
        key = int(rng.integers(0, 2**63)) | (int(rng.integers(0, 2**63)) << 64)
        ctr = int(rng.integers(0, 2**62))
        ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
        c = _words(ctr + 1)
        k = (np.uint64(key & ((1 << 64) - 1)), np.uint64(key >> 64))
        got = philox4x64(c, k)
        assert [int(g) for g in got] == [int(r) for r in ref]


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 2
    for r in rows:
        v = [np.uint64(int(x, 16)) for x in r]
        got = philox4x64(v[0:4], v[4:6])
        assert [int(g) for g in got] == [int(x) for x in v[6:10]]


def test_philox_vectorised_equals_scalar():
    rows = np.arange(1000, 1100, dtype=np.uint64)
    z = np.zeros_like(rows)
    vec = philox4x64((rows, z + np.uint64(3), z, z), (np.uint64(9), np.uint64(2)))
    for i in (0, 17, 99):
        sc = philox4x64((rows[i], np.uint64(3), np.uint64(0), np.uint64(0)),
                        (np.uint64(9), np.uint64(2)))
        assert [int(v[i]) for v in vec] == [int(s) for s in sc]


def test_gaussian_table_quantiles():
    from scipy.special import ndtr
    T = omega.gaussian_table_fp64()
    j = np.arange(4096)
    # forward CDF (a different routine) maps the table back to its midpoints
    assert np.max(np.abs(ndtr(T) - (j + 0.5) / 4096)) < 1e-15
    assert np.all(np.diff(T) > 0)
    assert np.array_equal(T, -T[::-1])                 # symmetry of N(0,1)
    assert abs(T.mean()) < 1e-15
    # midpoint-quantile law: variance just below 1
    assert 0.998 < np.mean(T ** 2) < 1.0


def _nearest_even(x, grid, grid_codes):
    """Brute-force round-to-nearest-even on an explicit sorted value grid."""
    out = np.empty_like(x)
    for t, v in enumerate(x):
        d = np.abs(grid - v)
        m = d.min()
        cand = np.nonzero(d == m)[0]
        if cand.size > 1:                       # tie: even code wins
            cand = [c for c in cand if grid_codes[c] % 2 == 0]
        out[t] = grid[cand[0]]
    return out


def test_bf16_rounding_is_nearest_even():
    T = omega.gaussian_table_fp64()
    codes = np.arange(0, 1 << 16, dtype=np.uint32)
    with np.errstate(invalid="ignore"):
        vals = (codes << 16).view(np.float32).astype(np.float64)
    ok = np.isfinite(vals) & (np.abs(vals) < 8)
    grid, gcodes = vals[ok], codes[ok]
    order = np.argsort(grid, kind="stable")
    grid, gcodes = grid[order], gcodes[order]
    sample = np.concatenate([T[:64], T[2016:2080], T[-64:], T[::97]])
    assert np.array_equal(omega.to_bf16(sample), _nearest_even(sample, grid, gcodes))


def test_e4m3_rounding_is_nearest_even():
    T = omega.gaussian_table_fp64()
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    vals = codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()
    ok = np.isfinite(vals)
    grid, gcodes = vals[ok], codes.numpy().astype(np.int64)[ok]
    # keep one code per value (+0 and -0 both map to 0.0; 0 is even)
    uniq, idx = np.unique(grid, return_index=True)
    sample = np.concatenate([T[:40], T[2000:2096], T[-40:], T[::61]])
    assert np.array_equal(omega.to_e4m3(sample), _nearest_even(sample, uniq, gcodes[idx]))


def test_omega_prefix_and_offset_consistency():
    a = omega.omega(11, 2, 300, 45, "fp64")
    b = omega.omega(11, 2, 100, 7, "fp64", row0=150)
    assert np.array_equal(a[150:250, :7], b)
    c = omega.omega(11, 2, 300, 20, "fp64")
    assert np.array_equal(a[:, :20], c)
    assert not np.array_equal(omega.omega(12, 2, 10, 5, "fp64"), a[:10, :5])
    assert not np.array_equal(omega.omega(11, 3, 10, 5, "fp64"), a[:10, :5])


def test_omega_field_layout_against_scalar_draws():
    # entry (r, k): call (r, k // 20), word (k % 20) // 5, bits 12*(k % 5)
    seed, n = 77, 1
    Om = omega.omega(seed, n, 5, 43, "fp64")
    T = omega.gaussian_table_fp64()
    for r in range(5):
        for k in (0, 4, 5, 19, 20, 33, 42):
            w = philox4x64((np.uint64(r), np.uint64(k // 20), np.uint64(0), np.uint64(0)),
                           (np.uint64(seed), np.uint64(n)))
            word = int(w[(k % 20) // 5])
            j = (word >> (12 * (k % 5))) & 0xFFF
            assert Om[r, k] == T[j]


def test_omega_moments_and_independence():
    Om = omega.omega(3, 0, 200000, 8, "bf16")
    n = Om.size
    var_t = np.mean(omega.gaussian_table("bf16") ** 2)
    assert abs(Om.mean()) < 4 / np.sqrt(n)
    assert abs(np.mean(Om ** 2) - var_t) < 4 * np.sqrt(2.0 / n) * var_t
    C = np.corrcoef(Om.T)
    off = C[~np.eye(8, dtype=bool)]
    assert np.max(np.abs(off)) < 4 / np.sqrt(Om.shape[0])
    # the 12-bit indices are uniform
    idx = omega.table_indices(3, 0, np.arange(50000, dtype=np.uint64), 20).ravel()
    hist = np.bincount(idx, minlength=4096)
    expect = idx.size / 4096
    chi2 = np.sum((hist - expect) ** 2 / expect)
    assert chi2 < 4096 + 6 * np.sqrt(2 * 4096)
