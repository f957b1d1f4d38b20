"""Pins for the oracle's variants of the projection step: power iterations
on the sketch (the remark after Algorithm 1) and the sequential projection."""
import itertools

import numpy as np

from oracle import omega, rtrd
from oracle import tensor as T
from oracle.philox import philox4x64
from paper_1901_01652_gb300 import workloads


def _projector(Y):
    Q = rtrd.orth(Y)
    return Q @ Q.T


def _gapped(shape, n, k, gap, seed):
    """A tensor whose mode-n unfolding has k singular values 1..2 and the rest
    `gap` times smaller (a clear spectral gap after the k-th)."""
    rng = np.random.default_rng(seed)
    I = shape[n]
    J = int(np.prod(shape)) // I
    U, _ = np.linalg.qr(rng.standard_normal((I, I)))
    V, _ = np.linalg.qr(rng.standard_normal((J, I)))
    s = np.concatenate([np.linspace(2.0, 1.0, k), gap * rng.uniform(0.5, 1.0, I - k)])
    Xn = (U * s) @ V.T
    perm = [n] + [m for m in range(len(shape)) if m != n]
    X = np.transpose(Xn.reshape([shape[m] for m in perm]), np.argsort(perm))
    return np.ascontiguousarray(X), U[:, :k]


def test_power_iterations_converge_to_the_dominant_subspace():
    """Subspace iteration: many iterations turn span(Y) into the span of the k
    leading left singular vectors of X_(n) (compared with LAPACK's SVD).  A
    missing re-orthonormalisation collapses the columns onto the top singular
    vector and fails this; so does a transposed product."""
    for n in range(3):
        X, Uk = _gapped((9, 10, 11), n, 4, 0.3, 40 + n)
        Y0 = rtrd.sketch(X, [4 if m == n else 99 for m in range(3)], 7)[n]
        Y = rtrd.power_iterate(X, n, Y0, 60)
        assert np.abs(_projector(Y) - Uk @ Uk.T).max() < 1e-10
        # q = 0 is the plain sketch
        assert np.array_equal(rtrd.power_iterate(X, n, Y0, 0), Y0)


def test_power_iterations_stay_in_the_range_of_the_unfolding():
    """Y_q = (X X^T)^q X Omega has its columns in range(X_(n)): for a
    low-rank unfolding (a noiseless TR, rank <= R_n R_{n+1} < I_n) the part
    of Y_q outside that range is at rounding level."""
    X, _ = workloads.tr_cores((12, 10, 11), (2, 2, 2), 3), None
    X = T.tr_full(X)
    for n in range(3):
        U, s, _ = np.linalg.svd(T.unfold(X, n), full_matrices=False)
        r = int(np.sum(s > 1e-10 * s[0]))
        assert r == 4
        Ur = U[:, :r]
        Y = rtrd.sketch_power(X, [6] * 3, 5, 2)[n]
        assert np.linalg.norm(Y - Ur @ (Ur.T @ Y)) <= 1e-12 * np.linalg.norm(Y)
        # and the single iteration equals the closed form X X^T X Omega up to span
        Y1 = rtrd.sketch_power(X, [6] * 3, 5, 1)[n]
        Xn = T.unfold(X, n)
        Yc = Xn @ (Xn.T @ rtrd.sketch(X, [6] * 3, 5)[n])
        assert np.abs(_projector(Y1[:, :r]) - _projector(Yc[:, :r])).max() < 1e-9


def test_power_iterations_improve_the_projection_of_a_flat_spectrum():
    """On a slowly decaying spectrum the projection error ||X - X x_n QQ^T||
    falls with q and approaches the optimal tail (Eckart-Young)."""
    rng = np.random.default_rng(9)
    I, J, k = 40, 300, 8
    U, _ = np.linalg.qr(rng.standard_normal((I, I)))
    V, _ = np.linalg.qr(rng.standard_normal((J, I)))
    s = 1.0 / np.arange(1, I + 1) ** 0.5
    X = ((U * s) @ V.T).reshape(I, 15, 20)
    Y0 = rtrd.sketch(X, [k, 99, 99], 11)[0]
    errs = []
    for q in (0, 1, 2, 4):
        Q = rtrd.orth(rtrd.power_iterate(X, 0, Y0, q))
        Xn = T.unfold(X, 0)
        errs.append(np.linalg.norm(Xn - Q @ (Q.T @ Xn)))
    best = np.sqrt(np.sum(s[k:] ** 2))
    assert errs[0] > errs[1] > errs[2] > errs[3] >= best * (1 - 1e-12)
    assert errs[3] < 1.05 * best


def test_power_iterations_exact_recovery():
    dims, R = (7, 8, 6, 9), (2, 2, 2, 2)
    X = T.tr_full(workloads.tr_cores(dims, R, 12))
    K = [4, 4, 4, 4]
    for q in (1, 2):
        Ys = rtrd.sketch_power(X, K, 13, q)
        Qs = [rtrd.orth(Y) for Y in Ys]
        Xh = X
        for n in range(4):
            Xh = T.mode_product(Xh, Qs[n] @ Qs[n].T, n)
        assert T.fro(X - Xh) <= 1e-12 * T.fro(X)


def _back(P, Qs):
    for n, Q in enumerate(Qs):
        P = T.mode_product(P, Q, n)
    return P


def test_sequential_projection_error_is_the_sum_of_the_step_errors():
    """Sequential orthogonal projections: with P_0 = X and P_j the tensor
    after the j-th mode in the order, ||X - P x_1 Q_1 ... x_N Q_N||^2 equals
    the sum over the steps of ||P_{j-1} - P_{j-1} x_n Q_n Q_n^T||^2 (each
    step's error is orthogonal to what the later steps keep)."""
    rng = np.random.default_rng(14)
    X = rng.standard_normal((9, 7, 8, 6))
    K = [4, 3, 5, 2]
    order = [2, 0, 3, 1]
    Ys, Qs, P = rtrd.project_sequential(X, K, 15, order)
    assert P.shape == (4, 3, 5, 2)
    total = T.fro(X - _back(P, Qs)) ** 2
    steps = 0.0
    cur = X
    for n in order:
        steps += T.fro(cur - T.mode_product(cur, Qs[n] @ Qs[n].T, n)) ** 2
        cur = T.mode_product(cur, Qs[n].T, n)
    assert abs(total - steps) <= 1e-12 * T.fro(X) ** 2
    assert np.allclose(cur, P, rtol=0, atol=1e-13)
    # the first mode of the order is sketched from X itself, as in Algorithm 1
    assert np.array_equal(Ys[order[0]], rtrd.sketch(X, K, 15)[order[0]])
    # every Q_n is orthonormal
    for Q in Qs:
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-13


def test_sequential_sketch_bruteforce_loop():
    """Each later sketch, entry by entry: Y_n[i, k] = sum over the other
    indices of the current (shrunk) P times Omega_n[r, k], r the row-major
    index of the other modes of P and every Omega entry drawn alone from
    Philox.  P is rebuilt here from the returned Q's by explicit sums."""
    rng = np.random.default_rng(20)
    X = rng.standard_normal((5, 4, 6))
    K = [3, 2, 4]
    order = [2, 0, 1]
    seed = 23
    Tab = omega.gaussian_table_fp64()
    Ys, Qs, P = rtrd.project_sequential(X, K, seed, order)
    cur = X.copy()
    for n in order:
        others = [m for m in range(3) if m != n]
        Yb = np.zeros((cur.shape[n], K[n]))
        for idx in itertools.product(*(range(s) for s in cur.shape)):
            r = 0
            for m in others:
                r = r * cur.shape[m] + idx[m]
            for k in range(K[n]):
                w = philox4x64((np.uint64(r), np.uint64(k // 20), np.uint64(0), np.uint64(0)),
                               (np.uint64(seed), np.uint64(n)))
                j = (int(w[(k % 20) // 5]) >> (12 * (k % 5))) & 0xFFF
                Yb[idx[n], k] += cur[idx] * Tab[j]
        assert np.allclose(Ys[n], Yb, rtol=1e-13, atol=1e-13), n
        # P <- P x_n Q_n^T by explicit sums
        shp = list(cur.shape)
        shp[n] = K[n]
        nxt = np.zeros(shp)
        for idx in itertools.product(*(range(s) for s in shp)):
            src = list(idx)
            acc = 0.0
            for i in range(cur.shape[n]):
                src[n] = i
                acc += cur[tuple(src)] * Qs[n][i, idx[n]]
            nxt[idx] = acc
        cur = nxt
    assert np.allclose(P, cur, rtol=1e-13, atol=1e-13)


def test_sequential_projection_later_sketches_see_the_shrunk_tensor():
    """Mode n later in the order is sketched from P with a test matrix of
    prod(current sizes of the other modes) rows: Y_n = P_(n) Omega_n, so
    Y_n^T Y_n-related spans lie in the range of the current unfolding."""
    X = T.tr_full(workloads.tr_cores((10, 9, 8), (2, 3, 2), 16))
    K = [6, 6, 6]
    order = [0, 1, 2]
    Ys, Qs, P = rtrd.project_sequential(X, K, 17, order)
    cur = T.mode_product(X, Qs[0].T, 0)
    U, s, _ = np.linalg.svd(T.unfold(cur, 1), full_matrices=False)
    r = int(np.sum(s > 1e-10 * s[0]))
    assert Ys[1].shape == (9, 6)
    assert np.linalg.norm(Ys[1] - U[:, :r] @ (U[:, :r].T @ Ys[1])) <= 1e-12 * np.linalg.norm(Ys[1])


def test_sequential_projection_exact_recovery():
    dims, R = (8, 9, 7, 6), (2, 2, 2, 2)
    X = T.tr_full(workloads.tr_cores(dims, R, 18))
    Ys, Qs, P = rtrd.project_sequential(X, [4, 4, 4, 4], 19)
    assert T.fro(X - _back(P, Qs)) <= 1e-12 * T.fro(X)
    out = rtrd.rtrd(X, [4, 4, 4, 4], R, "svd", seed=19, eps=1e-10, sequential=True)
    assert T.fro(X - T.tr_full(out["G"])) <= 1e-9 * T.fro(X)
