"""Pins for the oracle's Algorithm 1, TR-ALS and TR-SVD."""
import itertools

import numpy as np
import pytest

from oracle import omega, rtrd
from oracle import tensor as T
from oracle.philox import philox4x64
from paper_1901_01652_gb300 import workloads


def _noiseless(dims, R, seed):
    cores = workloads.tr_cores(dims, R, seed)
    return T.tr_full(cores), cores


# --------------------------------------------------------------- sketch / QR

def test_sketch_bruteforce_loop():
    """Y_n[i,k] = sum over all other indices of X * Omega_n, with every Omega
    entry drawn one by one from Philox (no vectorisation, no unfolding)."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3, 4, 5))
    K = [2, 3, 2]
    seed = 21
    Tab = omega.gaussian_table_fp64()
    Y = rtrd.sketch(X, K, seed)
    for n in range(3):
        others = [m for m in range(3) if m != n]
        Yb = np.zeros((X.shape[n], K[n]))
        for idx in itertools.product(*(range(s) for s in X.shape)):
            r = 0
            for m in others:                      # row-major over the other modes
                r = r * X.shape[m] + idx[m]
            for k in range(K[n]):
                w = philox4x64((np.uint64(r), np.uint64(k // 20), np.uint64(0), np.uint64(0)),
                               (np.uint64(seed), np.uint64(n)))
                j = (int(w[(k % 20) // 5]) >> (12 * (k % 5))) & 0xFFF
                Yb[idx[n], k] += X[idx] * Tab[j]
        assert np.allclose(Y[n], Yb, rtol=1e-13, atol=1e-13)


def test_sketch_linearity_and_unprojected_modes():
    rng = np.random.default_rng(1)
    X1 = rng.standard_normal((6, 5, 7))
    X2 = rng.standard_normal((6, 5, 7))
    K = [3, 5, 2]                  # mode 1: K >= I, not projected
    Ya = rtrd.sketch(2.0 * X1 - 0.5 * X2, K, 4, "bf16")
    Y1 = rtrd.sketch(X1, K, 4, "bf16")
    Y2 = rtrd.sketch(X2, K, 4, "bf16")
    assert Ya[1] is None
    for n in (0, 2):
        assert np.allclose(Ya[n], 2.0 * Y1[n] - 0.5 * Y2[n], rtol=1e-12, atol=1e-12)


def test_orth_properties():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((40, 7)) @ np.diag(np.logspace(0, -4, 7))
    Q = rtrd.orth(Y)
    assert np.abs(Q.T @ Q - np.eye(7)).max() < 1e-14
    assert np.linalg.norm(Y - Q @ (Q.T @ Y)) <= 1e-13 * np.linalg.norm(Y)
    R = Q.T @ Y
    assert np.allclose(np.tril(R, -1), 0, atol=1e-12)    # triangular factor
    assert np.all(np.diag(R) > 0)                         # sign reading
    # scaling the test matrix (hence Y) leaves Q unchanged
    assert np.abs(rtrd.orth(3.7 * Y) - Q).max() < 1e-13


def test_orth_equals_gram_schmidt():
    """diag(R) > 0 makes Q unique: it must equal modified Gram-Schmidt."""
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((12, 4))
    Qg = np.zeros_like(Y)
    for k in range(4):
        v = Y[:, k].copy()
        for j in range(k):
            v -= (Qg[:, j] @ v) * Qg[:, j]
        Qg[:, k] = v / np.linalg.norm(v)
    assert np.abs(rtrd.orth(Y) - Qg).max() < 1e-13


# --------------------------------------------------------------- projection

def test_exact_recovery_when_K_covers_the_unfolding_rank():
    dims, R = (8, 9, 7, 6), (2, 2, 2, 2)
    X, _ = _noiseless(dims, R, 10)
    K = [4, 4, 4, 4]                               # = R_n R_{n+1}
    _, Qs = rtrd.bases(X, K, seed=5)
    Xp = X
    for n in range(4):
        Xp = T.mode_product(Xp, Qs[n] @ Qs[n].T, n)
    assert T.fro(X - Xp) <= 1e-12 * T.fro(X)


def test_chain_order_invariance_and_norm_bound():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((7, 6, 8, 5))
    _, Qs = rtrd.bases(X, [3, 2, 4, 3], seed=6)
    P0 = rtrd.project(X, Qs, [0, 1, 2, 3])
    for order in ([3, 2, 1, 0], [1, 3, 0, 2]):
        assert np.allclose(rtrd.project(X, Qs, order), P0, rtol=1e-13, atol=1e-13)
    assert P0.shape == (3, 2, 4, 3)
    assert T.fro(P0) <= T.fro(X)


def test_default_chain_order_rule():
    assert rtrd.default_chain_order((200, 200, 200, 200), [25] * 4) == [3, 0, 1, 2]
    assert rtrd.default_chain_order((1024, 1024, 256), [60, 60, 30]) == [0, 1, 2]
    assert rtrd.default_chain_order((1024, 1024, 256), [60, 60, 15]) == [2, 0, 1]
    assert rtrd.default_chain_order((60, 50, 3), [15, 25, 5]) == [0, 1, 2]


def test_pythagoras_identity_dense():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((6, 7, 5))
    _, Qs = rtrd.bases(X, [3, 4, 2], seed=8)
    P = rtrd.project(X, Qs)
    Zs = workloads.tr_cores(P.shape, 2, seed=9)
    Gs = rtrd.backproject(Zs, Qs)
    lhs = T.fro(X - T.tr_full(Gs)) ** 2
    rhs = T.fro(X) ** 2 - T.fro(P) ** 2 + T.fro(P - T.tr_full(Zs)) ** 2
    assert abs(lhs - rhs) < 1e-11 * T.fro(X) ** 2
    assert abs(rtrd.rse_identity(T.fro(X) ** 2, P, Zs) - rtrd.rse(X, T.tr_full(Gs))) < 1e-12


def test_backprojection_is_multilinear():
    """TR(Z_n x_2 Q_n) = TR(Z) x_1 Q_1 ... x_N Q_N (second line of Eq. 3)."""
    rng = np.random.default_rng(10)
    Zs = workloads.tr_cores((3, 4, 2), (2, 3, 2), seed=11)
    Qs = [np.linalg.qr(rng.standard_normal((d, k)))[0] for d, k in ((7, 3), (9, 4), (5, 2))]
    lhs = T.tr_full(rtrd.backproject(Zs, Qs))
    rhs = T.tr_full(Zs)
    for n in range(3):
        rhs = T.mode_product(rhs, Qs[n], n)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------- TR-ALS

def _err(P, Zs):
    return T.fro(P - T.tr_full(Zs))


def test_als_each_update_is_non_increasing():
    rng = np.random.default_rng(12)
    P = rng.standard_normal((5, 6, 4, 5))
    Zs = workloads.tr_cores(P.shape, 3, seed=13)
    prev = _err(P, Zs)
    for sweep in range(4):
        for n in range(4):
            rtrd.als_update(P, Zs, n)
            e = _err(P, Zs)
            assert e <= prev * (1 + 1e-12)
            prev = e


def test_als_update_satisfies_normal_equations():
    rng = np.random.default_rng(14)
    P = rng.standard_normal((4, 5, 6))
    Zs = workloads.tr_cores(P.shape, (2, 3, 2), seed=15)
    rtrd.als_update(P, Zs, 1)
    S = T.subchain_matrix(Zs, 1)
    resid = T.tr_unfold(P, 1) - T.core_matrix(Zs[1]) @ S.T
    assert np.abs(resid @ S).max() < 1e-11 * np.abs(T.tr_unfold(P, 1) @ S).max()


def test_als_exact_recovery_from_perturbed_truth():
    dims, R = (6, 7, 5, 6), (2, 2, 2, 2)
    P, cores = _noiseless(dims, R, 16)
    rng = np.random.default_rng(17)
    init = [c + 1e-3 * rng.standard_normal(c.shape) for c in cores]
    Zs, errs = rtrd.tr_als(P, R, 30, init=init)
    assert errs[-1] <= 1e-8 * T.fro(P)


def test_als_is_orthogonally_equivariant():
    """TR-ALS on P = X x_n U^T (U orthogonal) with the rotated start equals
    TR-ALS on X rotated afterwards: checks the unfolding/transposition logic."""
    rng = np.random.default_rng(18)
    X = rng.standard_normal((5, 6, 4))
    U = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    init = workloads.tr_cores(X.shape, (2, 3, 2), seed=19)
    Za, _ = rtrd.tr_als(X, None, 3, init=init)
    P = T.mode_product(X, U.T, 1)
    init_r = [c.copy() for c in init]
    init_r[1] = T.mode_product(init_r[1], U.T, 1)
    Zb, _ = rtrd.tr_als(P, None, 3, init=init_r)
    Zb[1] = T.mode_product(Zb[1], U, 1)
    assert np.allclose(T.tr_full(Za), T.tr_full(Zb), rtol=1e-9, atol=1e-9)


def test_gram_solve_pinv_fallback_on_singular_gram():
    rng = np.random.default_rng(20)
    B = rng.standard_normal((6, 3))
    G = B @ B.T                                     # rank 3 of 6
    W = rng.standard_normal((4, 3)) @ B.T           # consistent right-hand sides
    Z, ok = rtrd.gram_solve(G, W)
    assert not ok
    assert np.abs(Z @ G - W).max() < 1e-10 * np.abs(W).max()
    assert np.abs(Z - W @ np.linalg.pinv(G)).max() < 1e-8


def test_default_init_is_scaled_to_norm_of_P():
    rng = np.random.default_rng(21)
    P = rng.standard_normal((4, 5, 3))
    Zs = rtrd.init_cores(P, (2, 2, 3), seed=3)
    assert abs(T.fro(T.tr_full(Zs)) - T.fro(P)) < 1e-12 * T.fro(P)


# --------------------------------------------------------------- TR-SVD

def test_trsvd_error_bound():
    rng = np.random.default_rng(22)
    P = rng.standard_normal((6, 5, 7, 4))
    for eps in (0.3, 0.6, 0.9):
        Zs, _ = rtrd.tr_svd(P, eps)
        assert T.fro(P - T.tr_full(Zs)) <= eps * T.fro(P) * (1 + 1e-12)


def test_trsvd_exact_recovery_and_ranks():
    dims, R = (6, 7, 8), (2, 3, 2)
    P, _ = _noiseless(dims, R, 23)
    Zs, ranks = rtrd.tr_svd(P, 1e-12)
    assert T.fro(P - T.tr_full(Zs)) <= 1e-11 * T.fro(P)
    assert ranks[0] * ranks[1] == 6        # rank of P_(1) = R_1 R_2


def test_trsvd_order2_is_eckart_young():
    rng = np.random.default_rng(24)
    M = rng.standard_normal((9, 7))
    s = np.linalg.svd(M, compute_uv=False)
    Zs, ranks = rtrd.tr_svd(M, 0.5)
    r = ranks[0] * ranks[1]
    assert abs(T.fro(M - T.tr_full(Zs)) - np.sqrt(np.sum(s[r:] ** 2))) < 1e-12
    # r is the smallest rank meeting sqrt(2) * delta (delta = eps ||M|| / sqrt 2)
    thr = 0.5 * np.linalg.norm(M)
    assert np.sqrt(np.sum(s[r:] ** 2)) <= thr < np.sqrt(np.sum(s[r - 1:] ** 2))


def test_trsvd_forced_ranks_reproduce_free_ranks():
    rng = np.random.default_rng(25)
    P = rng.standard_normal((5, 6, 4))
    Za, ra = rtrd.tr_svd(P, 0.4)
    Zb, rb = rtrd.tr_svd(P, 0.4, ranks=ra)
    assert ra == rb
    assert np.allclose(T.tr_full(Za), T.tr_full(Zb), rtol=1e-13, atol=1e-13)


def test_canonical_signs_are_independent_of_the_svd_signs():
    """Each pair (u_k, v_k) leaves canonical_signs with the same sign whatever
    sign it came in with, and the product U S Vt is unchanged."""
    rng = np.random.default_rng(29)
    M = rng.standard_normal((7, 11))
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    Uc, Vc = rtrd.canonical_signs(U, Vt)
    D = rng.choice([-1.0, 1.0], size=s.size)
    Uf, Vf = rtrd.canonical_signs(U * D, Vt * D[:, None])
    assert np.array_equal(Uf, Uc) and np.array_equal(Vf, Vc)
    assert np.allclose((Uc * s) @ Vc, M, atol=1e-13)
    for k in range(s.size):
        i = int(np.argmax(np.abs(Uc[:, k])))
        assert Uc[i, k] > 0


def test_trsvd_does_not_depend_on_the_svd_signs(monkeypatch):
    """TR-SVD with every SVD's singular pairs flipped at random gives the same
    cores: a step that skipped the sign rule would reshape a differently
    signed carry and truncate a different tail at the next step."""
    rng = np.random.default_rng(30)
    S = T.tr_full([rng.standard_normal((r0, i, r1)) for r0, i, r1 in ((2, 9, 3), (3, 8, 2), (2, 7, 2), (2, 6, 2))])
    P = S + 1e-3 * T.fro(S) / np.sqrt(S.size) * rng.standard_normal(S.shape)
    Za, ra = rtrd.tr_svd(P, 1e-2)
    raw = rtrd._svd
    flips = np.random.default_rng(31)

    def flipped(C):
        U, s, Vt = raw(C)
        D = flips.choice([-1.0, 1.0], size=s.size)
        return U * D, s, Vt * D[:, None]

    monkeypatch.setattr(rtrd, "_svd", flipped)
    Zb, rb = rtrd.tr_svd(P, 1e-2)
    assert ra == rb
    for a, b in zip(Za, Zb):
        assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(a).max())


def test_split_rank_reading():
    assert rtrd.split_rank(12) == (3, 4)
    assert rtrd.split_rank(16) == (4, 4)
    assert rtrd.split_rank(7) == (1, 7)
    assert rtrd.split_rank(1) == (1, 1)


# --------------------------------------------------------------- end to end

def test_algorithm1_tiny_end_to_end_exact_recovery():
    """4x5x3x4 noiseless TR of ranks 2 with K_n = min(I_n, R^2): Algorithm 1
    with TR-ALS from the projected truth (slightly perturbed) recovers X."""
    dims, R = (4, 5, 3, 4), (2, 2, 2, 2)
    X, cores = _noiseless(dims, R, 26)
    K = [4, 4, 4, 4]
    _, Qs = rtrd.bases(X, K, seed=27)
    rng = np.random.default_rng(28)
    init = [T.mode_product(c, Q.T, 1) + 1e-4 * rng.standard_normal((c.shape[0], Q.shape[1], c.shape[2]))
            for c, Q in zip(cores, Qs)]
    out = rtrd.rtrd(X, K, R, "als", seed=27, sweeps=40, init=init)
    Xh = T.tr_full(out["G"])
    assert rtrd.rse(X, Xh) < 1e-8
    assert abs(rtrd.rse_identity(T.fro(X) ** 2, out["P"], out["Z"]) - rtrd.rse(X, Xh)) < 1e-7
    assert out["P"].shape == (4, 4, 3, 4)     # mode 3 (I=3 <= K) kept whole
