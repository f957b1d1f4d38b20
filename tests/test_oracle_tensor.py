"""Pins for the oracle's tensor algebra (Section 2: unfoldings, Eq. 1, Eq. 2)."""
import itertools

import numpy as np

from oracle import tensor as T
from paper_1901_01652_gb300 import workloads


def test_unfold_index_map_bruteforce():
    X = np.random.default_rng(0).standard_normal((3, 4, 2, 5))
    for n in range(4):
        U = T.unfold(X, n)
        A, I, B = T.mode_view(X.shape, n)
        Xv = X.reshape(A, I, B)
        for a, i, b in itertools.product(range(A), range(I), range(B)):
            assert U[i, a * B + b] == Xv[a, i, b]


def test_mode_product_bruteforce():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, 4, 5))
    U = rng.standard_normal((2, 4))
    Y = T.mode_product(X, U, 1)
    assert Y.shape == (3, 2, 5)
    for a, j, b in itertools.product(range(3), range(2), range(5)):
        assert abs(Y[a, j, b] - sum(X[a, i, b] * U[j, i] for i in range(4))) < 1e-14


def test_eq1_bruteforce_equals_tr_full():
    for dims, R in (((3, 4, 5), (2, 3, 2)), ((2, 3, 4, 3), (3, 1, 2, 2))):
        rng = np.random.default_rng(2)
        cores = [rng.standard_normal((R[n], dims[n], R[(n + 1) % len(dims)]))
                 for n in range(len(dims))]
        assert np.allclose(T.tr_full_bruteforce(cores), T.tr_full(cores), rtol=1e-13, atol=1e-13)


def test_eq2_expansion_equals_eq1_bruteforce():
    """tr_full_unfolded (Eq. 2, longest mode first, order undone) against the
    element-by-element trace of Eq. 1, with the longest mode in every place."""
    for dims, R in (((3, 4, 5), (2, 3, 2)), ((6, 3, 4, 3), (3, 1, 2, 2)), ((2, 3, 7, 4), (2, 2, 3, 1)),
                    ((2, 3, 4, 5, 2), (1, 2, 2, 3, 2))):
        rng = np.random.default_rng(4)
        cores = [rng.standard_normal((R[n], dims[n], R[(n + 1) % len(dims)]))
                 for n in range(len(dims))]
        X = T.tr_full_unfolded(cores)
        assert X.shape == dims and X.flags.c_contiguous
        assert np.allclose(X, T.tr_full_bruteforce(cores), rtol=1e-13, atol=1e-13)


def test_cyclic_shift_of_cores_permutes_modes():
    cores = workloads.tr_cores((3, 4, 5, 2), (2, 3, 2, 4), seed=3)
    X = T.tr_full(cores)
    Xs = T.tr_full(cores[1:] + cores[:1])
    assert np.allclose(Xs, np.transpose(X, (1, 2, 3, 0)), rtol=1e-12, atol=1e-12)


def test_gauge_transform_leaves_tensor_unchanged():
    rng = np.random.default_rng(4)
    dims, R = (3, 4, 5), (2, 3, 2)
    cores = [rng.standard_normal((R[n], dims[n], R[(n + 1) % 3])) for n in range(3)]
    M = [rng.standard_normal((r, r)) + 3 * np.eye(r) for r in R]
    g = []
    for n in range(3):
        Minv = np.linalg.inv(M[n])
        g.append(np.einsum("ab,bic,cd->aid", Minv, cores[n], M[(n + 1) % 3]))
    assert np.allclose(T.tr_full(g), T.tr_full(cores), rtol=1e-11, atol=1e-11)


def test_rank_one_ring_is_outer_product():
    rng = np.random.default_rng(5)
    vs = [rng.standard_normal(d) for d in (3, 4, 5)]
    cores = [v.reshape(1, -1, 1) for v in vs]
    assert np.allclose(T.tr_full(cores), np.einsum("i,j,k->ijk", *vs), rtol=1e-14)


def test_eq2_tr_unfolding_factorises():
    cores = workloads.tr_cores((3, 4, 5, 2), (2, 3, 2, 4), seed=6)
    X = T.tr_full(cores)
    for n in range(4):
        lhs = T.tr_unfold(X, n)
        rhs = T.core_matrix(cores[n]) @ T.subchain_matrix(cores, n).T
        assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_tr_unfold_index_map_bruteforce():
    X = np.random.default_rng(7).standard_normal((2, 3, 4))
    U = T.tr_unfold(X, 1)       # I_2 x I_3 I_1, columns (i3, i1) row-major
    for i1, i2, i3 in itertools.product(range(2), range(3), range(4)):
        assert U[i2, i3 * 2 + i1] == X[i1, i2, i3]


def test_tr_inner_matches_dense():
    a = workloads.tr_cores((3, 4, 5), (2, 3, 2), seed=8)
    b = workloads.tr_cores((3, 4, 5), (3, 1, 2), seed=9)
    dense = float(np.sum(T.tr_full(a) * T.tr_full(b)))
    assert abs(T.tr_inner(a, b) - dense) < 1e-11 * (1 + abs(dense))
    assert abs(T.tr_norm(a) - T.fro(T.tr_full(a))) < 1e-11 * T.fro(T.tr_full(a))
