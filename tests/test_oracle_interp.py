"""Pins of the oracle's interpolation-based cluster bases (Sec. 2, Def.
"Cluster basis", Eq. (h2_admissible)): closed forms, exact polynomial
reproduction, the nesting identity checked by direct evaluation, and the decay
of the approximation error in q."""
import math

import numpy as np
import pytest

from oracle import h2_oracle as O
from workloads import sphere_points


def _box_cluster(lo, hi):
    return O.Cluster(np.arange(1), np.array(lo, float), np.array(hi, float), 0, 0, None)


def test_chebyshev_nodes_closed_form():
    c = _box_cluster([-1, -1, -1], [1, 1, 1])
    nd = O.cluster_nodes(c, 3)
    for d in range(3):
        assert np.allclose(nd[d], [math.sqrt(3) / 2, 0.0, -math.sqrt(3) / 2], atol=1e-15)
    c2 = _box_cluster([2, 0, -4], [4, 1, -2])
    nd2 = O.cluster_nodes(c2, 2)
    h = math.sqrt(0.5)
    assert np.allclose(nd2[0], [3 + h, 3 - h]) and np.allclose(nd2[1], [0.5 + 0.5 * h, 0.5 - 0.5 * h])
    assert np.allclose(nd2[2], [-3 + h, -3 - h])


def test_lagrange_q2_closed_form_and_cardinality():
    # q = 2 on [-1, 1]: nodes ±1/√2, L_0(x) = (x + 1/√2)/√2, L_1(x) = (1/√2 - x)/√2
    nodes = np.array([math.sqrt(0.5), -math.sqrt(0.5)])
    x = np.linspace(-1, 1, 7)
    L = O.lagrange_1d(nodes, x)
    assert np.allclose(L[:, 0], (x + math.sqrt(0.5)) / math.sqrt(2), atol=1e-15)
    assert np.allclose(L[:, 1], (math.sqrt(0.5) - x) / math.sqrt(2), atol=1e-15)
    for q in (1, 3, 4, 5):
        nd = O.cluster_nodes(_box_cluster([0.3, -2, 5], [1.7, 0.5, 5.2]), q)
        T = O.tensor_nodes(nd)
        Lt = O.tensor_lagrange(nd, T)
        assert np.allclose(Lt, np.eye(q ** 3), atol=1e-12)


@pytest.mark.parametrize("q", [2, 3, 4])
def test_lagrange_reproduces_polynomials(q):
    """Tensor interpolation of order q is exact on polynomials of degree <= q-1 per variable."""
    rng = np.random.default_rng(q)
    nd = O.cluster_nodes(_box_cluster([-0.2, 0.1, 0.4], [0.3, 0.9, 0.6]), q)
    T = O.tensor_nodes(nd)
    x = rng.uniform([-0.2, 0.1, 0.4], [0.3, 0.9, 0.6], size=(50, 3))
    ex = rng.integers(0, q, size=3)

    def p(z):
        return (1 + z[:, 0]) ** ex[0] * (2 - z[:, 1]) ** ex[1] * (0.5 + z[:, 2]) ** ex[2]

    interp = O.tensor_lagrange(nd, x) @ p(T)
    assert np.allclose(interp, p(x), rtol=1e-12, atol=1e-12)
    assert np.allclose(O.tensor_lagrange(nd, x).sum(1), 1.0, atol=1e-12)


def test_nesting_identity_by_direct_evaluation():
    """Def. "Cluster basis": V_t|_{t̂'×k} = V_{t'} E_{t'}; V_t of an inner cluster is
    evaluated here directly (Lagrange polynomials of t at the points of t̂)."""
    H = O.H2Matrix(sphere_points(1500, 2), q=3, leaf_size=40)
    for c in H.clusters:
        direct = O.tensor_lagrange(H.nodes[c.id], H.points[c.idx])
        expanded = O._expanded_basis(H, c)
        assert np.allclose(expanded, direct, rtol=1e-11, atol=1e-11), c.id
    for cid, E in H.E.items():
        assert np.allclose(E.sum(1), 1.0, atol=1e-12)
    for cid, V in H.V.items():
        assert np.allclose(V.sum(1), 1.0, atol=1e-12)


def test_h2_matrix_reproduces_polynomial_kernel_exactly():
    """For g(x, y) = (1 + x·y)² (degree <= 2 in every coordinate of x and of y),
    q = 3 interpolation is exact, so the dense expansion equals the kernel matrix."""
    def g(x, y):
        s = x[..., 0] * y[..., 0] + x[..., 1] * y[..., 1] + x[..., 2] * y[..., 2]
        return (1.0 + s) ** 2

    pts = sphere_points(900, 4) * np.array([1.0, 0.7, 1.3])
    H = O.H2Matrix(pts, q=3, leaf_size=30, eta=2.0, kernel=g, sigma=0.25)
    A = O.dense_expand(H)
    K = O.kernel_matrix(pts, g, 0.25)
    assert len(H.adm) > 100
    assert np.abs(A - K).max() <= 1e-12 * np.abs(K).max()


def test_interpolation_error_decays_with_q():
    """Relative Frobenius error of Â against the exact exp kernel matrix falls by
    at least 4x per extra order (Chebyshev interpolation of a smooth kernel)."""
    pts = sphere_points(2048, 0)
    g = O.exp_kernel(0.5)
    K = O.kernel_matrix(pts, g, 1e-2)
    errs = []
    for q in (2, 3, 4, 5):
        A = O.dense_expand(O.H2Matrix(pts, q=q, leaf_size=64, eta=2.0, sigma=1e-2))
        errs.append(np.linalg.norm(A - K) / np.linalg.norm(K))
    for a, b in zip(errs, errs[1:]):
        assert b * 4 <= a, errs
    assert errs[-1] < 1e-4


def test_planar_points_degenerate_box():
    """Points in the plane z = 0: the degenerate side is widened, nodes stay
    distinct, and polynomial kernels are still reproduced."""
    rng = np.random.default_rng(9)
    pts = np.zeros((500, 3))
    pts[:, :2] = rng.uniform(-1, 1, size=(500, 2))

    def g(x, y):
        return 1.0 + x[..., 0] * y[..., 0] + 0.5 * x[..., 1] * y[..., 1]

    H = O.H2Matrix(pts, q=2, leaf_size=20, kernel=g)
    A = O.dense_expand(H)
    K = O.kernel_matrix(pts, g)
    assert np.abs(A - K).max() <= 1e-11
