"""Pins of the oracle's H² × dense-block product (Sec. 3 Alg. "H2_mvm" with the
k×m coefficient blocks of Sec. 4): brute force against the kernel matrix where
interpolation is exact, the dense expansion, Y += α A X semantics, linearity,
transposition and relabelling invariance.  The last test plants mistakes in a
copy of the oracle and checks that the pins catch each one."""
import numpy as np
import pytest

from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def _poly_kernel(x, y):
    s = x[..., 0] * y[..., 0] + x[..., 1] * y[..., 1] + x[..., 2] * y[..., 2]
    return (1.0 + s) ** 2 + 0.3 * x[..., 0] * y[..., 1]


def _poly_case(n=700, m=5, seed=8):
    pts = sphere_points(n, seed) * np.array([1.2, 0.8, 1.0])
    H = O.H2Matrix(pts, q=3, leaf_size=25, eta=2.0, kernel=_poly_kernel, sigma=0.5)
    X = gaussian_rhs(n, m, seed + 1)
    Y0 = gaussian_rhs(n, m, seed + 2)
    return pts, H, X, Y0


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_h2mm_equals_brute_force_for_exactly_interpolated_kernel():
    pts, H, X, Y0 = _poly_case()
    K = O.kernel_matrix(pts, _poly_kernel, 0.5)
    alpha = -0.75
    Y = O.h2mm(H, alpha, X, Y0)
    assert _rel(Y, Y0 + alpha * (K @ X)) < 1e-12
    # the non-symmetric polynomial kernel also pins the transposed product
    Yt = O.h2mm(H, alpha, X, Y0, transposed=True)
    assert _rel(Yt, Y0 + alpha * (K.T @ X)) < 1e-12


@pytest.mark.parametrize("q,m", [(3, 8), (4, 3), (2, 1)])
def test_h2mm_equals_dense_expansion(q, m):
    pts = sphere_points(2048, 0)
    H = O.H2Matrix(pts, q=q, leaf_size=64, eta=2.0, sigma=1e-2)
    X = gaussian_rhs(2048, m, 1)
    A = O.dense_expand(H)
    assert _rel(O.h2mm(H, 1.0, X), A @ X) < 1e-13


def test_linearity_and_columns():
    pts = sphere_points(1024, 6)
    H = O.H2Matrix(pts, q=3, leaf_size=32, sigma=1e-2)
    X = gaussian_rhs(1024, 4, 2)
    Y = O.h2mm(H, 2.5, X)
    for j in range(4):
        yj = O.h2mm(H, 2.5, X[:, j])
        assert _rel(Y[:, j], yj) < 1e-14
    Z = O.h2mm(H, 1.0, 3.0 * X[:, :2] - X[:, 2:])
    assert _rel(Z, (3.0 * Y[:, :2] - Y[:, 2:]) / 2.5) < 1e-13


def test_symmetry_and_adjoint_identity():
    pts = sphere_points(1024, 7)
    H = O.H2Matrix(pts, q=3, leaf_size=32, sigma=1e-2)
    X = gaussian_rhs(1024, 3, 3)
    # the construction is symmetric: Aᵀ X == A X
    assert _rel(O.h2mm(H, 1.0, X, transposed=True), O.h2mm(H, 1.0, X)) < 1e-13
    # perturb coupling matrices asymmetrically: <Y, A X> == <Aᵀ Y, X>
    rng = np.random.default_rng(0)
    for b in H.adm:
        b.S = b.S + 0.1 * rng.standard_normal(b.S.shape)
    Yv = gaussian_rhs(1024, 3, 4)
    lhs = np.sum(Yv * O.h2mm(H, 1.0, X))
    rhs = np.sum(O.h2mm(H, 1.0, Yv, transposed=True) * X)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert _rel(O.h2mm(H, 1.0, X, transposed=True), O.h2mm(H, 1.0, X)) > 1e-3


def test_result_independent_of_point_labels():
    pts = sphere_points(1500, 12)
    X = gaussian_rhs(1500, 3, 5)
    H = O.H2Matrix(pts, q=3, leaf_size=48, sigma=1e-2)
    Y = O.h2mm(H, 1.0, X)
    p = np.random.default_rng(1).permutation(1500)
    H2 = O.H2Matrix(pts[p], q=3, leaf_size=48, sigma=1e-2)
    Y2 = O.h2mm(H2, 1.0, X[p])
    assert _rel(Y2, Y[p]) < 1e-13


def test_single_cluster_is_dense():
    pts = sphere_points(50, 1)
    H = O.H2Matrix(pts, q=3, leaf_size=64, sigma=0.1)
    assert len(H.clusters) == 1 and len(H.adm) == 0 and len(H.near) == 1
    X = gaussian_rhs(50, 2, 1)
    K = O.kernel_matrix(pts, O.exp_kernel(0.5), 0.1)
    assert _rel(O.h2mm(H, 1.0, X), K @ X) < 1e-14


# ---------------------------------------------------------------------------
# Planted mistakes: each mutation of the oracle must fail a pin above.
# ---------------------------------------------------------------------------
def _mut_forward_no_transpose(H, s, X, xhat):
    if s.is_leaf:
        xhat[s.id] = H.V[s.id].T @ X[s.idx]
    else:
        acc = np.zeros((H.k, X.shape[1]))
        for s2 in s.sons:
            _mut_forward_no_transpose(H, s2, X, xhat)
            acc = acc + H.E[s2.id] @ xhat[s2.id]  # planted: E instead of Eᵀ
        xhat[s.id] = acc


def _mut_backward_skip_transfer(H, t, Y, yhat):
    if t.is_leaf:
        Y[t.idx] += H.V[t.id] @ yhat[t.id]
    else:
        for t2 in t.sons:  # planted: transfer term dropped
            _mut_backward_skip_transfer(H, t2, Y, yhat)


def _mut_addeval_wrong_side(H, alpha, b, xhat, yhat, X, Y, transposed):
    if b.kind == "adm":
        yhat[b.t.id] += alpha * (b.S.T @ xhat[b.s.id])  # planted: S_bᵀ
    elif b.kind == "near":
        Y[b.t.idx] += alpha * (b.G @ X[b.s.idx])
    else:
        for b2 in b.sons:
            _mut_addeval_wrong_side(H, alpha, b2, xhat, yhat, X, Y, transposed)


def _mut_tensor_nodes(nodes):
    q = nodes.shape[1]
    out = np.empty((q ** 3, 3))
    for nz in range(q):
        for ny in range(q):
            for nx in range(q):
                out[nx + q * ny + q * q * nz] = (nodes[0, ny], nodes[1, nx], nodes[2, nz])  # planted swap
    return out


@pytest.mark.parametrize("name,target,mutant", [
    ("forward E not transposed", "_forward", _mut_forward_no_transpose),
    ("backward transfer dropped", "_backward", _mut_backward_skip_transfer),
    ("coupling transposed", "_fast_addeval", _mut_addeval_wrong_side),
    ("tensor index order swapped", "tensor_nodes", _mut_tensor_nodes),
])
def test_pins_catch_planted_mistakes(monkeypatch, name, target, mutant):
    monkeypatch.setattr(O, target, mutant)
    pts, H, X, Y0 = _poly_case(n=500, m=3, seed=21)
    K = O.kernel_matrix(pts, _poly_kernel, 0.5)
    Y = O.h2mm(H, 1.0, X, Y0)
    assert _rel(Y, Y0 + K @ X) > 1e-6, name
