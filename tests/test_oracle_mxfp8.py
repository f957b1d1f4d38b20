"""Pins for the oracle's block-scaled float8 quantisation (the FP8 sketch's X~).

The quantiser is checked against torch's float8_e4m3fn conversion (a library
routine with round-to-nearest-even), a scalar loop restatement of the block
rule on tiny tensors, closed-form cases (saturation, scale choice, all-zero
and tiny blocks) and invariants (power-of-two equivariance, idempotence,
error bound, block locality).
"""
import itertools
import math

import numpy as np
import pytest
import torch

from oracle import mxfp8, omega, rtrd
from oracle.philox import philox4x64


def _scalar_e4m3(v):
    """Nearest e4m3 value by explicit grid search over the 127 finite
    non-negative codes (ties to the even code); the grid ends at 448, so
    larger values land on 448 (saturation)."""
    a = abs(v)
    grid = []
    for code in range(0, 127):            # 0x00..0x7E: all finite non-negative e4m3 codes
        e, m = code >> 3, code & 7
        val = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
        grid.append((val, code))
    best = min(grid, key=lambda g: (abs(g[0] - a), g[1] & 1))
    return math.copysign(best[0], v)


def _scalar_quantize_mode(X, n):
    """The block rule written as loops over elements (tiny tensors only)."""
    shape = X.shape
    A = int(np.prod(shape[:n], dtype=np.int64))
    I = shape[n]
    B = int(np.prod(shape[n + 1:], dtype=np.int64))
    V = X.reshape(A, I, B)
    out = np.zeros_like(V)
    for a in range(A):
        for i in range(I):
            for b in range(B):
                if B > 1:
                    members = [V[a, i, bb] for bb in range(B) if bb // 32 == b // 32]
                else:
                    members = [V[aa, i, 0] for aa in range(A) if aa // 32 == a // 32]
                amax = max(abs(m) for m in members)
                if amax > 0:
                    e = max(math.frexp(amax)[1] - 1 - 8, -120)     # floor(log2 amax) - 8
                else:
                    e = -120
                out[a, i, b] = _scalar_e4m3(V[a, i, b] * 2.0 ** -e) * 2.0 ** e
    return out.reshape(shape)


def test_element_rounding_matches_torch_e4m3():
    rng = np.random.default_rng(0)
    V = rng.standard_normal((50, 96)) * np.exp(rng.uniform(-6, 6, (50, 1)))
    V[:, 5] = 0.0
    V[3, :] *= 1e-3
    Xq, e = mxfp8.quantize_blocks(V)
    s = np.repeat(np.ldexp(1.0, e), 32, axis=1)
    scaled = V / s
    ok = np.abs(scaled) < 464.0                     # torch turns larger values into NaN
    t = torch.from_numpy(scaled).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert ok.mean() > 0.9
    assert np.array_equal((Xq / s)[ok], t[ok])
    assert np.all(np.abs(Xq / s) <= 448.0)


def test_scalar_loop_restatement_on_tiny_tensors():
    rng = np.random.default_rng(1)
    for shape in [(3, 2, 70), (2, 5, 3, 4), (70, 3), (33, 2, 1, 5)]:
        X = rng.standard_normal(shape) * rng.choice([1e-3, 1.0, 300.0], size=shape)
        for n in range(len(shape)):
            assert np.array_equal(mxfp8.quantize_for_mode(X, n), _scalar_quantize_mode(X, n)), (shape, n)


def test_saturation_and_scale_closed_forms():
    # amax 1.99 -> e = 0 - 8; 1.99 * 256 = 509.44 rounds to 512 -> saturates to 448
    v = np.zeros((1, 32))
    v[0, 0] = 1.99
    v[0, 1] = 470.0 / 256          # rounds to 480 -> saturates
    v[0, 2] = 460.0 / 256          # rounds to 448
    v[0, 3] = 100.3 / 256          # grid spacing 8 in [64, 128): 104
    v[0, 4] = 0.9 / 256 * 2 ** -6  # subnormal range: spacing 2^-9 -> 2^-9 * round(0.9 * 8) = 7 * 2^-9
    Xq, e = mxfp8.quantize_blocks(v)
    assert e[0, 0] == -8
    assert Xq[0, 0] == 448.0 / 256 and Xq[0, 1] == 448.0 / 256 and Xq[0, 2] == 448.0 / 256
    assert Xq[0, 3] == 104.0 / 256
    assert Xq[0, 4] == 7 * 2.0 ** -9 / 256
    # an all-zero block and a tiny block use the floor exponent -120
    z, ez = mxfp8.quantize_blocks(np.zeros((1, 32)))
    assert ez[0, 0] == -120 and not z.any()
    t, et = mxfp8.quantize_blocks(np.full((1, 32), 2.0 ** -115))
    assert et[0, 0] == -120 and np.all(t == 2.0 ** -115)
    # the block amax lands in [256, 512) before saturation
    rng = np.random.default_rng(2)
    V = rng.standard_normal((200, 32)) * np.exp(rng.uniform(-20, 20, (200, 1)))
    _, e = mxfp8.quantize_blocks(V)
    am = np.max(np.abs(V), axis=1) * np.ldexp(1.0, -e[:, 0])
    assert np.all((am >= 256) & (am < 512))


def test_blocks_are_local_and_follow_the_mode_view():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 3, 5, 40))           # mode 1: B = 200 (ragged last block of 8)
    base = mxfp8.quantize_for_mode(X, 1)
    Xb = X.copy()
    Xb[2, 1, 4, 39] = 1e4                            # b = 4*40 + 39 = 199: block b in [192, 200)
    q = mxfp8.quantize_for_mode(Xb, 1).reshape(4, 3, 200)
    bq = base.reshape(4, 3, 200)
    changed = np.argwhere(q != bq)
    assert len(changed) > 0
    assert all(a == 2 and i == 1 and 192 <= b < 200 for a, i, b in changed)
    # last mode (B = 1): blocks run along a
    X2 = rng.standard_normal((70, 6))
    Xc = X2.copy()
    Xc[40, 2] = 1e4                                   # a = 40: block a in [32, 64) of column i = 2
    d = np.argwhere(mxfp8.quantize_for_mode(Xc, 1) != mxfp8.quantize_for_mode(X2, 1))
    assert len(d) > 0 and all(32 <= a < 64 and i == 2 for a, i in d)


def test_equivariance_idempotence_and_error_bound():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((6, 7, 64)) * np.exp(rng.uniform(-3, 3, (6, 7, 1)))
    for n in range(3):
        Q = mxfp8.quantize_for_mode(X, n)
        for k in (-5, 3, 17):
            assert np.array_equal(mxfp8.quantize_for_mode(np.ldexp(X, k), n), np.ldexp(Q, k))
        assert np.array_equal(mxfp8.quantize_for_mode(Q, n), Q)
    Xq, e = mxfp8.quantize_blocks(X.reshape(-1, 64))
    V = X.reshape(-1, 64)
    s = np.repeat(np.ldexp(1.0, e), 32, axis=1)
    sat = np.abs(V / s) >= 464.0                 # rounds past 448: clipped
    normal = (np.abs(V / s) >= 2.0 ** -6) & ~sat
    err = np.abs(Xq - V)
    assert sat.any() and np.all(err[sat] <= (np.abs(V[sat]) - 448.0 * s[sat]) + 1e-300)
    assert np.all(err[normal] <= 2.0 ** -4 * np.abs(V[normal]))
    sub = np.abs(V / s) < 2.0 ** -6
    assert np.all(err[sub] <= 2.0 ** -10 * s[sub])


def test_fp8_sketch_bruteforce_loop():
    """Y_n[i,k] of the FP8 form = sum over the other indices of X~ * Omega_n,
    Omega_n entries drawn one by one and looked up in the e4m3 table."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, 4, 40))
    K = [2, 3, 4]
    seed = 9
    Tab = omega.gaussian_table("fp8")
    Y = rtrd.sketch(X, K, seed, "fp8")
    for n in range(3):
        Xq = _scalar_quantize_mode(X, n)
        others = [m for m in range(3) if m != n]
        Yb = np.zeros((X.shape[n], K[n]))
        for idx in itertools.product(*(range(s) for s in X.shape)):
            r = 0
            for m in others:
                r = r * X.shape[m] + idx[m]
            for k in range(K[n]):
                w = philox4x64((np.uint64(r), np.uint64(k // 20), np.uint64(0), np.uint64(0)),
                               (np.uint64(seed), np.uint64(n)))
                j = (int(w[(k % 20) // 5]) >> (12 * (k % 5))) & 0xFFF
                Yb[idx[n], k] += Xq[idx] * Tab[j]
        assert np.allclose(Y[n], Yb, rtol=1e-13, atol=1e-13)


def test_fp8_sketch_close_to_exact_sketch():
    """The FP8 sketch differs from the float64 one by the quantisation error
    only: at most a few per cent of ||X_(n)|| ||Omega_n||."""
    rng = np.random.default_rng(6)
    X = rng.standard_normal((20, 24, 36))
    Y8 = rtrd.sketch(X, [5, 5, 5], 3, "fp8")
    Y64 = rtrd.sketch(X, [5, 5, 5], 3, "fp64")
    for a, b in zip(Y8, Y64):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert 1e-4 < rel < 0.05
