"""Pins of the oracle's block GMRES (Sec. 5.2, Alg. "pgmres block"), from
facts that do not come from the oracle: the minimal-residual property over the
Krylov space (least squares on an explicit Krylov basis), the Givens residual
equal to the true residual, dense solves of non-symmetric systems (including
an H² matrix with asymmetrically perturbed couplings), restarts, column
independence and the block-Jacobi preconditioner."""
import numpy as np
import scipy.linalg as sla

from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def _nonsym(n, seed):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 3.0 + rng.standard_normal((n, n)) / np.sqrt(n)


def test_minimal_residual_over_krylov_space():
    A = _nonsym(120, 0)
    b = gaussian_rhs(120, 1, 1)
    for k in (1, 3, 6):
        r = O.block_gmres(lambda X: A @ X, b, tol=0.0, restart=50, max_iter=k)
        # least squares over K_k(A, b) with an orthonormal basis of [b, Ab, …]
        K = np.empty((120, k))
        v = b[:, 0] / np.linalg.norm(b)
        for j in range(k):
            K[:, j] = v
            v = A @ v
            v /= np.linalg.norm(v)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, b[:, 0], rcond=None)
        best = np.linalg.norm(b[:, 0] - A @ (Q @ y))
        got = np.linalg.norm(b[:, 0] - A @ r.X[:, 0])
        assert abs(got - best) <= 1e-10 * np.linalg.norm(b), (k, got, best)
        # the reported residual is the true one of the returned iterate
        assert abs(r.rel_residual[0] - got / np.linalg.norm(b)) <= 1e-10


def test_nonsymmetric_dense_solve_and_restarts():
    A = _nonsym(200, 2)
    B = gaussian_rhs(200, 4, 3)
    Xs = np.linalg.solve(A, B)
    for restart in (40, 7):
        r = O.block_gmres(lambda X: A @ X, B, tol=1e-10, restart=restart)
        assert r.status == "converged"
        assert np.linalg.norm(r.X - Xs) <= 1e-8 * np.linalg.norm(Xs)
        if restart == 7:
            assert r.cycles > 1


def test_columns_are_independent():
    A = _nonsym(150, 4)
    B = gaussian_rhs(150, 3, 5)
    r = O.block_gmres(lambda X: A @ X, B, tol=1e-9, restart=10)
    for i in range(3):
        ri = O.block_gmres(lambda X: A @ X, B[:, i:i + 1], tol=1e-9, restart=10)
        assert ri.col_iterations[0] == r.col_iterations[i]
        assert np.linalg.norm(ri.X[:, 0] - r.X[:, i]) <= 1e-12 * np.linalg.norm(r.X[:, i])


def test_nonsymmetric_h2_matrix():
    """Perturb every coupling matrix asymmetrically: CG no longer applies,
    GMRES solves the system the product defines."""
    H = O.H2Matrix(sphere_points(1200, 1), q=3, leaf_size=48, eta=2.0, sigma=1e-1)
    rng = np.random.default_rng(6)
    O.set_coupling(H, {(b.t.id, b.s.id): b.S * (1.0 + 0.05 * rng.standard_normal(b.S.shape)) for b in H.adm})
    A = O.dense_expand(H)
    assert np.abs(A - A.T).max() > 1e-3
    B = gaussian_rhs(1200, 3, 7)
    r = O.block_gmres(lambda X: O.h2mm(H, 1.0, X), B, tol=1e-9, restart=30, max_iter=3000)
    assert r.status == "converged"
    Xs = np.linalg.solve(A, B)
    assert np.linalg.norm(r.X - Xs) <= 1e-6 * np.linalg.norm(Xs)


def test_block_jacobi_preconditioned_gmres():
    H = O.H2Matrix(sphere_points(1500, 2), q=3, leaf_size=48, eta=2.0, sigma=1e-2)
    A = O.dense_expand(H)
    B = gaussian_rhs(1500, 4, 1)
    M = O.block_jacobi(H)
    r = O.block_gmres(lambda X: A @ X, B, tol=1e-9, restart=40, max_iter=4000, apply_Minv=M)
    p = O.block_gmres(lambda X: A @ X, B, tol=1e-9, restart=40, max_iter=4000)
    assert r.status == p.status == "converged"
    Xs = sla.cho_solve(sla.cho_factor(A), B)
    assert np.linalg.norm(r.X - Xs) <= 1e-6 * np.linalg.norm(Xs)
    assert r.iterations < p.iterations


def test_lucky_breakdown_is_exact():
    """b in a 2-dimensional invariant subspace: GMRES ends after two steps."""
    A = np.diag(np.arange(1.0, 11.0))
    b = np.zeros((10, 1))
    b[2, 0], b[5, 0] = 1.0, 2.0
    r = O.block_gmres(lambda X: A @ X, b, tol=1e-14, restart=10)
    assert r.status == "converged" and r.col_iterations[0] == 2
    assert np.allclose(A @ r.X, b, atol=1e-13)
