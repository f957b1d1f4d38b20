"""Block-scaled float8 (e4m3) quantisation of X for the FP8 sketch (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper computes the sketch Y_n = X_(n) Omega_n (Algorithm 1, step 5) in
unstated, presumably float64, arithmetic.  The FP8 form of this build runs
the sketch on a float8 copy of X with one power-of-two scale per block of 32
values, the layout of the OCP microscaling (MX) formats.  Reading used
(the paper has no FP8 form, so all of it is a definition of this build):

* Blocks.  For the mode-n sketch X is viewed as (A, I_n, B).  When B > 1 a
  block is 32 consecutive b of one (a, i) fibre, b in [32j, 32j + 32); the
  last block of a fibre is short when 32 does not divide B.  When B = 1 (the
  last mode) a block is 32 consecutive a of one i, a in [32j, 32j + 32).
  Either way a block is 32 consecutive columns r = a*B + b of one row of the
  unfolding X_(n), never crossing a change of a when B > 1.
* Scale.  amax = max |x| over the block; e = floor(log2 amax) - 8 (8 is the
  exponent of the largest power of two in e4m3), raised to -120 if lower,
  and e = -120 for an all-zero block.  The floor at -120 keeps every
  dequantised value exactly representable in bfloat16.
* Elements.  q = x * 2^-e rounded to the nearest e4m3 value (4 significant
  bits, ties to even; subnormal spacing 2^-9 below 2^-6), then saturated to
  +-448 (the largest finite e4m3 value); the dequantised value is
  x~ = q * 2^e.

The sketch of the FP8 form is then Y_n = X~_(n) Omega_n with Omega_n taken
from the e4m3-rounded quantile table (``omega.gaussian_table("fp8")``).
"""
import numpy as np

from .omega import round_significand

E4M3_MAX = 448.0
E4M3_EMAX = 8            # largest power of two representable in e4m3
BLOCK = 32
SCALE_EXP_MIN = -120


def e4m3_round_sat(v):
    """Nearest e4m3 value of float64 ``v`` (ties to even, subnormals below
    2^-6 on the 2^-9 grid), saturated to [-448, 448]."""
    q = round_significand(v, 4, min_normal_exp=-6)
    return np.clip(q, -E4M3_MAX, E4M3_MAX)


def block_scale_exponents(amax):
    """Scale exponent e of each block from its amax (float64 array)."""
    amax = np.asarray(amax, dtype=np.float64)
    _, ex = np.frexp(amax)                 # amax = m 2^ex, 0.5 <= m < 1 -> floor(log2) = ex - 1
    e = ex.astype(np.int64) - 1 - E4M3_EMAX
    e = np.maximum(e, SCALE_EXP_MIN)
    return np.where(amax > 0, e, SCALE_EXP_MIN)


def quantize_blocks(V):
    """Quantise the last axis of V in blocks of 32 (the last block may be
    short).  Returns (x~, e) with e the scale exponent per block."""
    V = np.asarray(V, dtype=np.float64)
    L = V.shape[-1]
    nb = -(-L // BLOCK)
    pad = nb * BLOCK - L
    Vp = np.concatenate([V, np.zeros(V.shape[:-1] + (pad,))], axis=-1) if pad else V
    Vb = Vp.reshape(V.shape[:-1] + (nb, BLOCK))
    e = block_scale_exponents(np.max(np.abs(Vb), axis=-1))
    s = np.ldexp(1.0, e)[..., None]
    Xq = e4m3_round_sat(Vb / s) * s
    return Xq.reshape(Vp.shape)[..., :L], e


def quantize_for_mode(X, n):
    """X~ for the mode-n sketch (blocks as in the module docstring), same
    shape as X, float64."""
    shape = X.shape
    A = int(np.prod(shape[:n], dtype=np.int64))
    I = int(shape[n])
    B = int(np.prod(shape[n + 1:], dtype=np.int64))
    V = np.asarray(X, dtype=np.float64).reshape(A, I, B)
    if B > 1:
        Xq, _ = quantize_blocks(V)                          # blocks along b
    else:
        Xq, _ = quantize_blocks(V[:, :, 0].T)               # (I, A): blocks along a
        Xq = Xq.T[:, :, None]
    return Xq.reshape(shape)
