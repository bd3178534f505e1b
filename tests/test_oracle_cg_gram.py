"""Pins of the oracle's Gram-matrix block CG (O'Leary's block CG in the
conjugacy form of Sec. 5.1, Alg. "CG", with m×m matrices for the scalars).

Pinned against facts that do not come from the oracle itself:
* m = 1 gives the scalar recurrences of Alg. "CG" (iterate by iterate);
* block CG minimises the A-norm error of every column over the block Krylov
  space, which contains that column's own Krylov space, so after j steps no
  column is worse than scalar CG after j steps;
* in exact arithmetic it terminates after at most ceil(n/m) steps;
* a dense Cholesky solve of Â X = B;
* rank-deficient right-hand sides (repeated, dependent, zero columns) are
  handled by deflation; <p, Ap> <= 0 is a breakdown.
"""
import math

import numpy as np
import scipy.linalg as sla

from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def _spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ Q.T


def test_single_column_is_scalar_cg():
    A = _spd(200, 1e3, 0)
    b = gaussian_rhs(200, 1, 3)
    for k in (1, 5, 17):
        g = O.block_cg_gram(lambda X: A @ X, b, tol=0.0, max_iter=k)
        c = O.block_cg(lambda X: A @ X, b, tol=0.0, max_iter=k)
        assert g.iterations == c.iterations == k
        assert np.linalg.norm(g.X - c.X) <= 1e-11 * np.linalg.norm(c.X)


def test_no_column_worse_than_scalar_cg_in_a_norm():
    A = _spd(300, 1e4, 1)
    B = gaussian_rhs(300, 6, 4)
    Xs = np.linalg.solve(A, B)

    def anorm_err(X):
        E = X - Xs
        return np.sqrt(np.einsum("ij,ij->j", E, A @ E))

    for k in (2, 6, 15, 40):
        g = O.block_cg_gram(lambda X: A @ X, B, tol=0.0, max_iter=k)
        c = O.block_cg(lambda X: A @ X, B, tol=0.0, max_iter=k)
        eg, ec = anorm_err(g.X), anorm_err(c.X)
        assert np.all(eg <= ec * (1 + 1e-8) + 1e-12), (k, eg / ec)
    # and clearly better once the block space has grown (ratio ≈ 0.34 here)
    assert np.all(eg < 0.5 * ec)


def test_finite_termination():
    n, m = 48, 8
    A = _spd(n, 10.0, 2)
    B = gaussian_rhs(n, m, 5)
    r = O.block_cg_gram(lambda X: A @ X, B, tol=1e-12, max_iter=100)
    assert r.status == "converged"
    assert r.iterations <= math.ceil(n / m) + 1
    assert np.linalg.norm(r.X - np.linalg.solve(A, B)) <= 1e-10 * np.linalg.norm(r.X)


def test_matches_dense_cholesky_solve_on_h2_matrix():
    H = O.H2Matrix(sphere_points(1500, 2), q=3, leaf_size=48, eta=2.0, sigma=1e-2)
    A = O.dense_expand(H)
    B = gaussian_rhs(1500, 8, 1)
    r = O.block_cg_gram(lambda X: O.h2mm(H, 1.0, X), B, tol=1e-8)
    assert r.status == "converged"
    Xc = sla.cho_solve(sla.cho_factor(A), B)
    assert np.linalg.norm(r.X - Xc) <= 1e-6 * np.linalg.norm(Xc)
    true = np.linalg.norm(B - A @ r.X, axis=0) / np.linalg.norm(B, axis=0)
    assert true.max() <= 1.05e-8
    cw = O.block_cg(lambda X: A @ X, B, tol=1e-8)
    assert r.iterations < cw.iterations


def test_rank_deficient_blocks_deflate():
    A = _spd(120, 1e3, 3)
    B = gaussian_rhs(120, 5, 6)
    B[:, 1] = B[:, 0]                  # repeated
    B[:, 3] = 2.0 * B[:, 0] - B[:, 2]  # dependent
    B[:, 4] = 0.0                      # zero column: converged from the start
    r = O.block_cg_gram(lambda X: A @ X, B, tol=1e-10, max_iter=500)
    assert r.status == "converged"
    Xs = np.linalg.solve(A, B)
    assert np.linalg.norm(r.X - Xs) <= 1e-7 * np.linalg.norm(Xs)
    assert np.all(r.X[:, 4] == 0.0) and r.col_iterations[4] == 0


def test_breakdown_on_negative_curvature():
    A = np.diag([1.0, 2.0, -3.0, 4.0])
    B = np.zeros((4, 2))
    B[2, 0] = 1.0
    B[0, 1] = 1.0
    r = O.block_cg_gram(lambda X: A @ X, B, tol=1e-10, max_iter=10)
    assert r.status == "breakdown"


def test_chol_deflate_is_a_cholesky_on_full_rank():
    G = _spd(10, 50.0, 7)
    L, K, broke = O._chol_deflate(G, list(range(10)))
    assert not broke and K == list(range(10))
    assert np.allclose(L, np.linalg.cholesky(G), rtol=1e-12, atol=1e-12)
    w = np.arange(10.0)
    assert np.allclose(O._chol_solve(L, K, w), np.linalg.solve(G, w), rtol=1e-10)


def test_chol_deflate_drops_dependent_directions():
    rng = np.random.default_rng(8)
    V = rng.standard_normal((30, 6))
    V[:, 2] = V[:, 0] + 1e-7 * rng.standard_normal(30)  # repeat up to 1e-7 (pivot ~1e-14 of its diagonal)
    V[:, 4] = V[:, 1] - 0.5 * V[:, 3]                   # exact combination
    G = V.T @ V
    L, K, broke = O._chol_deflate(G, list(range(6)))
    assert not broke and K == [0, 1, 3, 5]
    # on K the factor is the Cholesky factor of G_KK
    assert np.allclose(L[np.ix_(K, K)], np.linalg.cholesky(G[np.ix_(K, K)]), rtol=1e-12, atol=1e-12)
    # a direction with <p, Ap> <= 0 is a breakdown
    G2 = G.copy()
    G2[5, 5] = -1.0
    assert O._chol_deflate(G2, list(range(6)))[2]


def test_preconditioned_gram_single_column_is_pcg():
    """With m = 1 the preconditioned Gram form is Alg. "pcg block"."""
    H = O.H2Matrix(sphere_points(800, 3), q=3, leaf_size=48, eta=2.0, sigma=1e-2)
    A = O.dense_expand(H)
    Minv = O.block_jacobi(H)
    b = gaussian_rhs(800, 1, 9)
    for k in (1, 4, 9):
        g = O.block_cg_gram(lambda X: A @ X, b, tol=0.0, max_iter=k, apply_Minv=Minv)
        c = O.block_pcg(lambda X: A @ X, Minv, b, tol=0.0, max_iter=k)
        assert np.linalg.norm(g.X - c.X) <= 1e-10 * np.linalg.norm(c.X), k


def test_preconditioned_gram_solves_with_fewer_iterations():
    H = O.H2Matrix(sphere_points(1500, 2), q=3, leaf_size=48, eta=2.0, sigma=1e-2)
    A = O.dense_expand(H)
    B = gaussian_rhs(1500, 8, 1)
    r = O.block_cg_gram(lambda X: A @ X, B, tol=1e-8, apply_Minv=O.block_jacobi(H))
    g = O.block_cg_gram(lambda X: A @ X, B, tol=1e-8)
    assert r.status == "converged"
    Xc = sla.cho_solve(sla.cho_factor(A), B)
    assert np.linalg.norm(r.X - Xc) <= 1e-6 * np.linalg.norm(Xc)
    assert r.iterations < g.iterations
