"""Tensor algebra of Section 2 (oracle side, float64).

Conventions: tensors are NumPy arrays in row-major order (last mode fastest).
Modes are numbered 0..N-1 in code and 1..N in the paper.
"""
import itertools

import numpy as np


def mode_view(shape, n):
    """(A, I_n, B) with A = prod(shape[:n]) and B = prod(shape[n+1:])."""
    A = int(np.prod(shape[:n], dtype=np.int64))
    B = int(np.prod(shape[n + 1:], dtype=np.int64))
    return A, int(shape[n]), B


def unfold(X, n):
    """Mode-n unfolding X_(n) (Section 2.1), I_n x prod_{i!=n} I_i.

    Column order: row-major linear index of the remaining indices in
    increasing mode order, r = a*B + b.  (The paper takes Kolda's order; any
    fixed bijection of the columns is equivalent for the method because the
    test matrix rows are i.i.d., and this one is the order Omega_n is indexed
    by.)
    """
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1)


def mode_product(X, U, n):
    """Mode-n product X x_n U (Kolda): contracts mode n of X with the columns
    of U (J x I_n); the result has J in place of I_n."""
    return np.moveaxis(np.tensordot(U, X, axes=(1, n)), 0, n)


def fro(X):
    """Frobenius norm sqrt(<X, X>) (Section 2.1)."""
    return float(np.sqrt(np.sum(np.asarray(X, dtype=np.float64) ** 2)))


def tr_element(cores, idx):
    """Eq. 1: X(i_1..i_N) = Trace(prod_n G_n(i_n)), G_n(i_n) = G_n[:, i_n, :]."""
    M = cores[0][:, idx[0], :]
    for G, i in zip(cores[1:], idx[1:]):
        M = M @ G[:, i, :]
    return float(np.trace(M))


def tr_full_bruteforce(cores):
    """Eq. 1 evaluated element by element (tiny tensors only)."""
    shape = tuple(G.shape[1] for G in cores)
    X = np.empty(shape)
    for idx in itertools.product(*(range(s) for s in shape)):
        X[idx] = tr_element(cores, idx)
    return X


def tr_full(cores):
    """Psi([G_n]): the full tensor of a TR, by contracting the ring core by
    core and tracing the two open rank indices (the closed form of Eq. 1)."""
    T = cores[0]
    for G in cores[1:]:
        T = np.tensordot(T, G, axes=([-1], [0]))
    return np.trace(T, axis1=0, axis2=-1)


def tr_full_unfolded(cores):
    """Psi([G_n]) through Eq. 2 for tensors too large for ``tr_full``'s
    open-index contraction (which holds R_1^2 |X| values): with n the longest
    mode, X_<n> = G_{n,(2)} G_{!=n,<2>}^T as one matrix product, then the
    cyclic mode order of X_<n> undone."""
    N = len(cores)
    dims = [G.shape[1] for G in cores]
    n = int(np.argmax(dims))
    Xn = core_matrix(cores[n]) @ subchain_matrix(cores, n).T
    perm = cyclic_order(N, n)
    X = Xn.reshape([dims[m] for m in perm])
    return np.ascontiguousarray(np.transpose(X, np.argsort(perm)))


def cyclic_order(N, n):
    """Mode order n, n+1, ..., N-1, 0, ..., n-1 of the TR unfolding X_<n>."""
    return [(n + m) % N for m in range(N)]


def tr_unfold(X, n):
    """TR unfolding X_<n> (Section 2.1), I_n x I_{n+1}..I_N I_1..I_{n-1},
    columns in row-major order of the cyclic index sequence."""
    perm = cyclic_order(X.ndim, n)
    return np.transpose(X, perm).reshape(X.shape[n], -1)


def subchain(cores, n):
    """Subchain G_{!=n} of Eq. 2: for every column j of X_<n> the product
    G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1}), returned as (J, R_{n+1}, R_n)."""
    N = len(cores)
    S = cores[(n + 1) % N]
    for m in range(2, N):
        S = np.tensordot(S, cores[(n + m) % N], axes=([-1], [0]))
    R1, Rn = S.shape[0], S.shape[-1]
    S = S.reshape(R1, -1, Rn)
    return np.transpose(S, (1, 0, 2))


def core_matrix(Z):
    """G_{n,(2)}: core R_n x I_n x R_{n+1} as I_n x (R_n R_{n+1}),
    column (alpha, beta) = alpha * R_{n+1} + beta."""
    Rn, I, Rn1 = Z.shape
    return np.transpose(Z, (1, 0, 2)).reshape(I, Rn * Rn1)


def subchain_matrix(cores, n):
    """G_{!=n,<2>}: J x (R_n R_{n+1}) with column (alpha, beta) holding
    S_j[beta, alpha], so that X_<n> = G_{n,(2)} G_{!=n,<2>}^T (Eq. 2)."""
    S = subchain(cores, n)                   # (J, R_{n+1}, R_n)
    J = S.shape[0]
    return np.transpose(S, (0, 2, 1)).reshape(J, -1)


def tr_inner(coresA, coresB):
    """<TR(A), TR(B)> = Trace(prod_n sum_i A_n(i) (x) B_n(i)) (transfer
    matrices; used only for large tensors, tests pin it against tr_full)."""
    E = None
    for A, B in zip(coresA, coresB):
        Ra, I, Ra1 = A.shape
        Rb, _, Rb1 = B.shape
        En = np.einsum("aib,cid->acbd", A, B).reshape(Ra * Rb, Ra1 * Rb1)
        E = En if E is None else E @ En
    return float(np.trace(E))


def tr_norm(cores):
    return float(np.sqrt(max(tr_inner(cores, cores), 0.0)))
