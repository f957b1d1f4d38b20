"""Algorithm 1 (randomized TR decomposition) and the decomposers it calls.

Oracle side, float64 throughout.  Each function follows the step of the paper
it names; the readings taken where the paper is silent or garbled are stated
in the docstrings.
"""
import numpy as np
import scipy.linalg

from . import mxfp8 as _mxfp8
from . import omega as _omega
from .tensor import (core_matrix, fro, mode_product, mode_view, subchain_matrix,
                     tr_full, tr_unfold, unfold)


# ----------------------------------------------------------------------------
# Algorithm 1, steps 3-8: tensor random projection (Eq. 3)
# ----------------------------------------------------------------------------

def effective_K(dims, K):
    """Reading of Section 4.1 ("the order-3 of the tensor remains as 3"): a
    mode with K_n >= I_n is not projected; its Q_n is the identity and its
    effective K_n is I_n."""
    return [min(int(k), int(i)) for k, i in zip(K, dims)]


def projected(dims, K):
    return [int(k) < int(i) for k, i in zip(K, dims)]


def sketch(X, K, seed, prec="fp64"):
    """Algorithm 1, steps 4-5: Y_n = X_(n) M with M the Gaussian test matrix
    Omega_n (see ``oracle.omega``).  Returns [Y_n] (None for modes that are
    not projected).  With prec="fp8" the sketch of mode n reads the
    block-scaled float8 copy of X defined in ``oracle.mxfp8`` (the rest of
    the algorithm still uses X itself)."""
    Y = []
    for n, k in enumerate(K):
        A, I, B = mode_view(X.shape, n)
        if k >= I:
            Y.append(None)
            continue
        Om = _omega.omega(seed, n, A * B, k, prec)
        Xs = _mxfp8.quantize_for_mode(X, n) if prec == "fp8" else X
        Y.append(unfold(Xs, n) @ Om)
    return Y


def orth(Y):
    """Algorithm 1, step 6: economy QR of Y (LAPACK Householder), with the
    reading that the column signs make diag(R) > 0 so that Q_n is unique when
    Y has full column rank."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def bases(X, K, seed, prec="fp64"):
    """Q_n for every mode (identity for unprojected modes)."""
    Ys = sketch(X, K, seed, prec)
    Qs = []
    for n, Y in enumerate(Ys):
        Qs.append(np.eye(X.shape[n]) if Y is None else orth(Y))
    return Ys, Qs


def default_chain_order(dims, K):
    """Order in which the mode products of step 7 are applied.  The products
    commute (Eq. 3), so the order only changes rounding; the rule is: largest
    shrink factor I_n/K_n first; among equal factors the last mode first, then
    the others in increasing mode order (after the last mode, the next product
    then runs over the longest contiguous runs of the intermediate)."""
    Ke = effective_K(dims, K)
    N = len(dims)
    return sorted(range(N), key=lambda n: (Ke[n] / dims[n], 0 if n == N - 1 else 1, n))


def project(X, Qs, order=None):
    """Algorithm 1, step 7, read cumulatively: P = X x_1 Q_1^T ... x_N Q_N^T,
    the K_1 x ... x K_N tensor of Eq. 3 (every sketch uses the original X)."""
    if order is None:
        order = range(X.ndim)
    P = X
    for n in order:
        P = mode_product(P, Qs[n].T, n)     # identity Q_n leaves P exactly as is
    return P


def backproject(Zs, Qs):
    """Algorithm 1, step 11, read as G_n = Z_n x_2 Q_n (the printed x_n is
    taken to mean the middle mode of the order-3 core)."""
    return [mode_product(Z, Q, 1) for Z, Q in zip(Zs, Qs)]


# ----------------------------------------------------------------------------
# Variants of the projection step (Section 3.2, the remark after Algorithm 1,
# and the sequential form)
# ----------------------------------------------------------------------------

def power_iterate(X, n, Y, q):
    """Power iterations on the sketch of mode n, which the remark after
    Algorithm 1 names as a way to make the spectrum of the projected unfolding
    decay faster (citing Halko et al.): q times
        Y <- X_(n) (X_(n)^T orth(Y)),
    i.e. Y spans (X_(n) X_(n)^T)^q X_(n) Omega_n in exact arithmetic.
    Reading: Y is orthonormalised (``orth``) before every application of
    X_(n) X_(n)^T, which keeps the iteration well conditioned; the Y returned
    is not orthonormalised (step 6 does that, as for q = 0)."""
    Xn = unfold(X, n)
    for _ in range(q):
        Q = orth(Y)
        Y = Xn @ (Xn.T @ Q)
    return Y


def sketch_power(X, K, seed, q, prec="fp64"):
    """Algorithm 1 steps 4-5 followed by q power iterations per mode: [Y_n]
    (None for modes that are not projected).  The iterations use X itself
    (for prec="fp8" only the first sketch reads the float8 copy)."""
    return [None if Y is None else power_iterate(X, n, Y, q) for n, Y in enumerate(sketch(X, K, seed, prec))]


def project_sequential(X, K, seed, order=None, prec="fp64"):
    """Sequential form of the projection step (not the paper's Algorithm 1,
    whose step 5 sketches every mode from X itself): the modes are taken in
    `order`, and mode n is sketched from the tensor the earlier modes have
    already shrunk,
        Y_n = P_(n) Omega_n,  Q_n = orth(Y_n),  P <- P x_n Q_n^T,
    with Omega_n drawn as in ``oracle.omega`` (key (seed, n)) with one row per
    entry of the other modes of the current P (row-major index).  A mode with
    K_n >= I_n is kept whole (Q_n = I).  Returns (Ys, Qs, P), Ys[n] None for
    unprojected modes."""
    N = X.ndim
    if order is None:
        order = default_chain_order(X.shape, K)
    Ys, Qs = [None] * N, [None] * N
    P = X
    for n in order:
        A, I, B = mode_view(P.shape, n)
        if K[n] >= I:
            Qs[n] = np.eye(I)
            continue
        Om = _omega.omega(seed, n, A * B, K[n], prec)
        Ps = _mxfp8.quantize_for_mode(P, n) if prec == "fp8" else P
        Ys[n] = unfold(Ps, n) @ Om
        Qs[n] = orth(Ys[n])
        P = mode_product(P, Qs[n].T, n)
    return Ys, Qs, P


# ----------------------------------------------------------------------------
# TR-ALS (cited by the paper, Algorithm 1 step 9; restated from Eq. 2)
# ----------------------------------------------------------------------------

def init_cores(P, R, seed):
    """Default TR-ALS start (the paper is silent): discrete-Gaussian cores from
    ``omega.init_core_values``, all scaled by one factor so that
    ||TR(Z)|| = ||P||."""
    dims = P.shape
    N = len(dims)
    Zs = []
    for n in range(N):
        shp = (R[n], dims[n], R[(n + 1) % N])
        Zs.append(_omega.init_core_values(seed, n, int(np.prod(shp))).reshape(shp))
    from .tensor import tr_norm
    s = (fro(P) / tr_norm(Zs)) ** (1.0 / N)
    return [Z * s for Z in Zs]


def gram_solve(G, W):
    """Solve Z G = W for Z (G symmetric positive semidefinite).

    Cholesky in float64; if it fails, the eigen-pseudoinverse with cutoff
    1e-13 * lambda_max (reading: the paper does not say how a singular Gram
    matrix is treated)."""
    try:
        c = scipy.linalg.cho_factor(G, lower=True, check_finite=True)
        return scipy.linalg.cho_solve(c, W.T).T, True
    except np.linalg.LinAlgError:
        w, V = np.linalg.eigh(G)
        cut = 1e-13 * max(w.max(), 0.0)
        inv = np.where(w > cut, 1.0 / np.where(w > cut, w, 1.0), 0.0)
        return (W @ V) * inv @ V.T, False


def als_update(P, Zs, n):
    """One TR-ALS core update: with the other cores fixed, Eq. 2 makes
    P_<n> ~= Z_{n,(2)} S^T linear in core n, whose least-squares solution is
    Z_{n,(2)} = P_<n> S (S^T S)^{-1}, S = G_{!=n,<2>}."""
    Pn = tr_unfold(P, n)
    S = subchain_matrix(Zs, n)
    W = Pn @ S
    G = S.T @ S
    Zmat, chol_ok = gram_solve(G, W)
    Rn, I, Rn1 = Zs[n].shape
    Zs[n] = np.transpose(Zmat.reshape(I, Rn, Rn1), (1, 0, 2)).copy()
    return chol_ok


def tr_als(P, R, sweeps, init=None, seed=0, tol=None):
    """TR-ALS [Zhao et al. 2016] on P: each sweep updates cores 1..N in turn
    (Gauss-Seidel), and records ||P - TR(Z)||_F after the sweep.  A fixed
    number of sweeps; with `tol`, stops once the relative change of the error
    is below tol."""
    Zs = [np.array(Z, dtype=np.float64, copy=True) for Z in init] if init is not None \
        else init_cores(P, R, seed)
    errs = []
    for s in range(sweeps):
        for n in range(P.ndim):
            als_update(P, Zs, n)
        errs.append(fro(P - tr_full(Zs)))
        if tol is not None and s > 0 and abs(errs[-2] - errs[-1]) <= tol * errs[-2]:
            break
    return Zs, errs


# ----------------------------------------------------------------------------
# TR-SVD (cited by the paper, Algorithm 1 step 9; Section 4.1 tolerance)
# ----------------------------------------------------------------------------

def trunc_rank(s, thr):
    """Smallest r with sqrt(sum_{i>r} s_i^2) <= thr (ties keep the smaller r),
    at least 1."""
    tail = np.sqrt(np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]]))
    r = int(np.argmax(tail <= thr))
    return max(r, 1)


def split_rank(r):
    """Reading for the first TR-SVD step: r = R_1 * R_2 with R_1 the largest
    divisor of r not above sqrt(r)."""
    best = 1
    d = 1
    while d * d <= r:
        if r % d == 0:
            best = d
        d += 1
    return best, r // best


def _svd(C):
    """Thin SVD of C (LAPACK)."""
    return np.linalg.svd(C, full_matrices=False)


def canonical_signs(U, Vt):
    """Reading for TR-SVD (the paper cites it without stating it): the sign of
    each singular pair (u_k, v_k) is free, yet through the reshapes between
    steps (the split r = R_1 R_2 of the first step in particular) it changes
    which tail the next truncation drops.  The result is made unique by
    flipping each pair so that the entry of u_k largest in magnitude (the
    first such entry on ties) is positive."""
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s, Vt * s[:, None]


def tr_svd(P, eps, ranks=None):
    """TR-SVD [Zhao et al. 2016] with relative tolerance eps on P.

    delta = eps ||P|| / sqrt(N); the first step truncates at sqrt(2) delta and
    splits its rank into R_1 R_2, later steps truncate at delta.  With `ranks`
    (R_1..R_N) given, the ranks are forced instead of chosen ("forced" mode,
    used for parity where a rank decision sits on the threshold).
    Every SVD's singular pairs take the signs of ``canonical_signs``.
    Guarantees ||P - TR(Z)|| <= eps ||P|| in free mode.
    Returns (cores, ranks).
    """
    dims = P.shape
    N = len(dims)
    delta = eps * fro(P) / np.sqrt(N)
    Zs = []
    C = P.reshape(dims[0], -1)
    U, s, Vt = _svd(C)
    U, Vt = canonical_signs(U, Vt)
    if ranks is None:
        r = trunc_rank(s, np.sqrt(2.0) * delta)
        R0, R1 = split_rank(r)
    else:
        R0, R1 = int(ranks[0]), int(ranks[1])
        r = R0 * R1
    Rk = [R0, R1]
    Zs.append(np.transpose(U[:, :r].reshape(dims[0], R0, R1), (1, 0, 2)))
    C = (s[:r, None] * Vt[:r]).reshape(R0, R1, -1)       # (R0, R1, rest)
    C = np.transpose(C, (1, 2, 0))                         # (R1, rest, R0)
    for k in range(1, N - 1):
        C = C.reshape(Rk[k] * dims[k], -1)
        U, s, Vt = _svd(C)
        U, Vt = canonical_signs(U, Vt)
        if ranks is None:
            rk = trunc_rank(s, delta)
        else:
            rk = int(ranks[k + 1])
        Rk.append(rk)
        Zs.append(U[:, :rk].reshape(Rk[k], dims[k], rk))
        C = s[:rk, None] * Vt[:rk]
    Zs.append(C.reshape(Rk[N - 1], dims[N - 1], R0))
    return Zs, Rk[:N]


# ----------------------------------------------------------------------------
# Section 4: error measures; Algorithm 1 driver
# ----------------------------------------------------------------------------

def rse(X, Y):
    """RSE = ||X - Y||_F / ||X||_F (Section 4; the formula has no square)."""
    return fro(X - Y) / fro(X)


def rse_identity(normX2, P, Zs):
    """||X - TR(G)||^2 = ||X||^2 - ||P||^2 + ||P - TR(Z)||^2 (Eq. 3 with
    orthonormal Q_n), returned as the RSE."""
    e2 = normX2 - fro(P) ** 2 + fro(P - tr_full(Zs)) ** 2
    return float(np.sqrt(max(e2, 0.0) / normX2))


def rtrd(X, K, R, method="als", seed=0, prec="fp64", sweeps=20, init=None,
         eps=None, ranks=None, order=None, power=0, sequential=False):
    """Algorithm 1 end to end.  Returns a dict with Y, Q, P, Z, G, errors.
    power = q > 0 adds q power iterations to every sketch
    (``power_iterate``); sequential=True takes the sequential projection
    (``project_sequential``) instead of steps 3-8."""
    dims = X.shape
    if order is None:
        order = default_chain_order(dims, K)
    if sequential:
        Ys, Qs, P = project_sequential(X, K, seed, order, prec)
    else:
        Ys = sketch_power(X, K, seed, power, prec) if power else sketch(X, K, seed, prec)
        Qs = [np.eye(X.shape[n]) if Y is None else orth(Y) for n, Y in enumerate(Ys)]
        P = project(X, Qs, order)
    out = {"Y": Ys, "Q": Qs, "P": P, "order": list(order)}
    if method == "als":
        Zs, errs = tr_als(P, R, sweeps, init=init, seed=seed)
        out["als_err"] = errs
    elif method == "svd":
        Zs, Rk = tr_svd(P, eps, ranks=ranks)
        out["ranks"] = Rk
    else:
        raise ValueError(method)
    out["Z"] = Zs
    out["G"] = backproject(Zs, Qs)
    return out
