"""Pins of the oracle's block CG (Sec. 5.1, Alg. "CG" and Alg. "block CG"):
dense Cholesky solves (scipy), the textbook Hestenes–Stiefel recurrences,
column independence, and honest failure on an indefinite H² matrix."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


@pytest.fixture(scope="module")
def spd_case():
    pts = sphere_points(1024, 0)
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    A = O.dense_expand(H)
    return H, A


def test_block_cg_matches_cholesky_solve(spd_case):
    H, A = spd_case
    B = gaussian_rhs(1024, 6, 1)
    res = O.block_cg(lambda X: A @ X, B, tol=1e-8, max_iter=5000)
    assert res.status == "converged"
    Xc = sla.cho_solve(sla.cho_factor(A), B)
    assert np.linalg.norm(res.X - Xc) / np.linalg.norm(Xc) <= 1e-6
    true_rel = np.linalg.norm(B - A @ res.X, axis=0) / np.linalg.norm(B, axis=0)
    assert true_rel.max() <= 2e-8
    assert res.rel_residual.max() <= 1e-8
    assert res.iterations == res.col_iterations.max()


def test_block_cg_with_h2mm_operator(spd_case):
    H, A = spd_case
    B = gaussian_rhs(1024, 2, 3)
    res = O.block_cg(lambda X: O.h2mm(H, 1.0, X), B, tol=1e-8, max_iter=5000)
    ref = O.block_cg(lambda X: A @ X, B, tol=1e-8, max_iter=5000)
    assert res.status == "converged"
    assert np.linalg.norm(res.X - ref.X) / np.linalg.norm(ref.X) < 1e-7


def test_paper_cg_form_equals_textbook_cg(spd_case):
    """Alg. "CG" (γ = <Ap, r>/<p, Ap>, p = r - γ p) equals Hestenes–Stiefel
    (β = |r_new|²/|r|², p = r + β p) in exact arithmetic; compare early iterates."""
    _, A = spd_case
    b = gaussian_rhs(1024, 1, 9)[:, 0]
    x = np.zeros(1024)
    r = b.copy()
    p = r.copy()
    for _ in range(12):
        a = A @ p
        al = (r @ r) / (p @ a)
        x = x + al * p
        rn = r - al * a
        p = rn + ((rn @ rn) / (r @ r)) * p
        r = rn
    res = O.block_cg(lambda X: A @ X, b[:, None], tol=0.0, max_iter=12)
    assert res.iterations == 12 and res.status == "noconverge"
    assert np.linalg.norm(res.X[:, 0] - x) <= 1e-10 * np.linalg.norm(x)


def test_columns_are_independent(spd_case):
    _, A = spd_case
    B = gaussian_rhs(1024, 3, 4)
    B[:, 1] *= 1e3

    def colwise(X):  # same rounding for a column alone and inside a block
        return np.stack([A @ X[:, j] for j in range(X.shape[1])], axis=1)

    res = O.block_cg(colwise, B, tol=1e-8, max_iter=5000)
    for j in range(3):
        rj = O.block_cg(colwise, B[:, j:j + 1], tol=1e-8, max_iter=5000)
        assert rj.col_iterations[0] == res.col_iterations[j]
        assert np.array_equal(rj.X[:, 0], res.X[:, j])


def test_zero_column_and_initial_guess(spd_case):
    _, A = spd_case
    B = gaussian_rhs(1024, 2, 5)
    B[:, 0] = 0.0
    Xc = sla.cho_solve(sla.cho_factor(A), B)
    x0 = Xc + 1e-3 * gaussian_rhs(1024, 2, 6)
    x0[:, 0] = 0.0
    res = O.block_cg(lambda X: A @ X, B, X0=x0, tol=1e-8, max_iter=5000)
    assert res.status == "converged" and res.col_iterations[0] == 0
    assert np.all(res.X[:, 0] == 0.0)
    cold = O.block_cg(lambda X: A @ X, B, tol=1e-8, max_iter=5000)
    assert res.col_iterations[1] <= cold.col_iterations[1]


def test_indefinite_h2_matrix_is_reported_not_hidden():
    """At n = 2048 the q = 2 approximation has negative eigenvalues; block CG
    must end in breakdown or non-convergence, never report success."""
    pts = sphere_points(2048, 0)
    A = O.dense_expand(O.H2Matrix(pts, q=2, leaf_size=64, eta=2.0, sigma=1e-2))
    assert np.linalg.eigvalsh(A)[0] < 0
    B = gaussian_rhs(2048, 4, 1)
    res = O.block_cg(lambda X: A @ X, B, tol=1e-8, max_iter=3000)
    assert res.status in ("breakdown", "noconverge")


def test_breakdown_on_negative_curvature():
    A = np.diag([1.0, 2.0, -3.0, 4.0])
    B = np.array([[0.0], [0.0], [1.0], [0.0]])
    res = O.block_cg(lambda X: A @ X, B, tol=1e-10, max_iter=10)
    assert res.status == "breakdown"
