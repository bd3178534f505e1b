"""Pins of the oracle's preconditioned block CG (Sec. 5.1, Alg. "pcg block")
with the block-Jacobi preconditioner on the diagonal nearfield blocks."""
import numpy as np
import scipy.linalg as sla

from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def _case(n=1500, m=3):
    H = O.H2Matrix(sphere_points(n, 2), q=3, leaf_size=48, eta=2.0, sigma=1e-2)
    return H, O.dense_expand(H), gaussian_rhs(n, m, 1)


def test_block_jacobi_is_the_block_diagonal_inverse():
    H, A, B = _case()
    Minv = O.block_jacobi(H)
    # build the block-diagonal part of A from the leaves and invert it densely
    D = np.zeros_like(A)
    for c in H.clusters:
        if c.is_leaf:
            D[np.ix_(c.idx, c.idx)] = A[np.ix_(c.idx, c.idx)]
    Z = np.linalg.solve(D, B)
    assert np.allclose(Minv(B), Z, rtol=1e-10, atol=1e-10 * np.abs(Z).max())


def test_pcg_identity_preconditioner_is_cg():
    H, A, B = _case(800, 2)
    a = O.block_pcg(lambda X: A @ X, lambda R: R, B, tol=1e-9, max_iter=5000)
    b = O.block_cg(lambda X: A @ X, B, tol=1e-9, max_iter=5000)
    assert a.status == b.status == "converged"
    assert abs(a.iterations - b.iterations) <= 2
    assert np.linalg.norm(a.X - b.X) <= 1e-7 * np.linalg.norm(b.X)


def test_pcg_matches_textbook_pcg_iterates():
    """The paper's form (γ = <Ap, q>/<p, Ap>, p = q - γp) equals the textbook
    PCG (β = <r', z'>/<r, z>, p = z + βp) in exact arithmetic."""
    H, A, B = _case(800, 1)
    Minv = O.block_jacobi(H)
    b = B[:, 0]
    x = np.zeros_like(b)
    r = b.copy()
    z = Minv(r[:, None])[:, 0]
    p = z.copy()
    for _ in range(10):
        a = A @ p
        al = (r @ z) / (p @ a)
        x = x + al * p
        rn = r - al * a
        zn = Minv(rn[:, None])[:, 0]
        p = zn + ((rn @ zn) / (r @ z)) * p
        r, z = rn, zn
    res = O.block_pcg(lambda X: A @ X, Minv, B, tol=0.0, max_iter=10)
    assert np.linalg.norm(res.X[:, 0] - x) <= 1e-9 * np.linalg.norm(x)


def test_pcg_solves_and_needs_fewer_iterations():
    H, A, B = _case()
    Minv = O.block_jacobi(H)
    res = O.block_pcg(lambda X: A @ X, Minv, B, tol=1e-8, max_iter=5000)
    cg = O.block_cg(lambda X: A @ X, B, tol=1e-8, max_iter=5000)
    assert res.status == "converged"
    Xc = sla.cho_solve(sla.cho_factor(A), B)
    assert np.linalg.norm(res.X - Xc) <= 1e-6 * np.linalg.norm(Xc)
    assert res.iterations < cg.iterations
