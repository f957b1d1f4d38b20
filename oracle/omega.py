"""Gaussian test matrices Omega_n of Algorithm 1, step 4 (oracle side).

Algorithm 1, step 4 asks for a matrix M in R^{prod_{i!=n} I_i x K_n} "following
the Gaussian distribution"; the paper names no mean, variance or generator.
Reading used here (the same definition the CUDA library implements on its
own):

* Distribution: the 4096-level midpoint-quantile discretisation of N(0, 1),
  T[j] = Phi^{-1}((j + 1/2) / 4096), j = 0..4095 (a discrete symmetric law with
  variance within 1e-3 of 1, support |x| <= 3.6).  Scaling Omega leaves Q_n
  unchanged, so only the shape of the law matters.
* Precision: the table is stored at the precision of the path that consumes
  it: float64 for the FP64 path, rounded to bfloat16 (round to nearest even)
  for the FP32 and BF16 paths, to float8 e4m3 for the FP8 path.  The oracle
  consumes those exact values in float64.
* Indexing: Omega_n[r, k] with r the row-major linear index of the remaining
  indices (i_1..i_{n-1}, i_{n+1}..i_N), i.e. r = a*B + b for the (A, I_n, B)
  view of X.  One Philox4x64-10 call with key (seed, n) and counter
  (r, k // 20, 0, 0) yields four 64-bit words; word q = (k % 20) // 5 holds five
  12-bit fields and field f = k % 5 (bits 12f..12f+11) is the table index.
"""
import numpy as np
from scipy.special import ndtri

from .philox import philox4x64

LEVELS = 4096
COLS_PER_CALL = 20


def gaussian_table_fp64():
    """T[j] = Phi^{-1}((j + 1/2)/4096) in float64 (scipy's ndtri)."""
    j = np.arange(LEVELS, dtype=np.float64)
    return ndtri((j + 0.5) / LEVELS)


def round_significand(x, bits, min_normal_exp=None):
    """Round float64 values to `bits` significant bits, ties to even.

    With ``min_normal_exp`` set, values below 2**min_normal_exp are rounded to
    the subnormal grid of spacing 2**(min_normal_exp - bits + 1).
    """
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)               # x = m * 2**e, 0.5 <= |m| < 1
    e = e.astype(np.int64)
    if min_normal_exp is not None:
        # normal numbers have exponent e-1 >= min_normal_exp
        e = np.maximum(e, min_normal_exp + 1)
    scale = np.ldexp(1.0, (bits - e))
    return np.rint(x * scale) / scale


def to_bf16(x):
    """float64 -> nearest bfloat16 value (8 significant bits), as float64."""
    return round_significand(x, 8)


def to_e4m3(x):
    """float64 -> nearest float8 e4m3 value (4 significant bits, min normal
    2**-6, subnormal spacing 2**-9), as float64.  Inputs here stay below 448."""
    return round_significand(x, 4, min_normal_exp=-6)


def gaussian_table(prec):
    t = gaussian_table_fp64()
    if prec == "fp64":
        return t
    if prec in ("fp32", "bf16"):
        return to_bf16(t)
    if prec == "fp8":
        return to_e4m3(t)
    raise ValueError(prec)


def table_indices(seed, n, rows, K):
    """12-bit table indices j[r, k] for rows `rows` (uint64 array) of Omega_n."""
    rows = np.asarray(rows, dtype=np.uint64)
    ncall = (K + COLS_PER_CALL - 1) // COLS_PER_CALL
    out = np.empty((rows.size, ncall * COLS_PER_CALL), dtype=np.int64)
    key = (np.uint64(seed), np.uint64(n))
    zero = np.zeros_like(rows)
    for c in range(ncall):
        words = philox4x64((rows, zero + np.uint64(c), zero, zero), key)
        for q in range(4):
            for f in range(5):
                out[:, c * 20 + q * 5 + f] = ((words[q] >> np.uint64(12 * f))
                                              & np.uint64(0xFFF)).astype(np.int64)
    return out[:, :K]


def omega(seed, n, nrows, K, prec, row0=0):
    """Rows row0..row0+nrows-1 of Omega_n (float64 values of the table)."""
    rows = np.arange(row0, row0 + nrows, dtype=np.uint64)
    return gaussian_table(prec)[table_indices(seed, n, rows, K)]


def init_core_values(seed, n, count):
    """Default TR-ALS initial core entries (flat, float64).

    Reading (the paper does not state an initialisation): entry e of core n is
    T_fp64 at the field (e % 20) of Philox4x64-10 with key (seed + 1, 256 + n)
    and counter (e // 20, 0, 0, 0), i.e. the same discrete Gaussian as Omega.
    """
    e = np.arange(count, dtype=np.uint64)
    blocks = e // np.uint64(COLS_PER_CALL)
    fld = (e % np.uint64(COLS_PER_CALL)).astype(np.int64)
    zero = np.zeros_like(blocks)
    words = philox4x64((blocks, zero, zero, zero),
                       (np.uint64(seed + 1), np.uint64(256 + n)))
    w = np.stack(words, axis=1)                       # (count, 4)
    q = fld // 5
    f = fld % 5
    sel = w[np.arange(count), q]
    j = ((sel >> (np.uint64(12) * f.astype(np.uint64))) & np.uint64(0xFFF)).astype(np.int64)
    return gaussian_table_fp64()[j]
