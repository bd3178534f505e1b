"""Pins of the oracle's row-by-row product for large n (H2Rows) against the
full oracle product, which the other oracle tests pin against the dense
expansion and brute force; and of its coupling gradients against
adjoint_grads."""
import numpy as np

from _helpers import rel_fro
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def test_rows_equal_full_product():
    pts = sphere_points(3000, 4)
    H = O.H2Matrix(pts, q=3, leaf_size=48, eta=2.0, sigma=1e-2)
    R = O.H2Rows(pts, q=3, leaf_size=48, eta=2.0, sigma=1e-2)
    assert (R.n_adm, R.n_near) == (len(H.adm), len(H.near))
    X = gaussian_rhs(3000, 5, 2)
    Y = O.h2mm(H, 0.7, X)
    rows = np.random.default_rng(0).choice(3000, 40, replace=False)
    got = R.rows(0.7, X, rows)
    assert np.abs(got - Y[rows]).max() <= 1e-12 * np.abs(Y).max()


def test_forward_equals_full_forward():
    pts = sphere_points(2000, 5)
    H = O.H2Matrix(pts, q=2, leaf_size=32, eta=2.0)
    R = O.H2Rows(pts, q=2, leaf_size=32, eta=2.0)
    X = gaussian_rhs(2000, 3, 3)
    a = R.forward(X)
    b = {}
    O._forward(H, H.root, X, b)
    for cid in b:
        assert np.allclose(a[cid], b[cid], rtol=1e-13, atol=1e-13 * np.abs(b[cid]).max())


def test_coupling_grads_equal_adjoint_grads():
    pts = sphere_points(1500, 6)
    H = O.H2Matrix(pts, q=2, leaf_size=32, eta=2.0, sigma=1e-2)
    R = O.H2Rows(pts, q=2, leaf_size=32, eta=2.0, sigma=1e-2)
    L, X = gaussian_rhs(1500, 2, 7), gaussian_rhs(1500, 2, 8)
    dS, _ = O.adjoint_grads(H, L, X)
    pairs = list(dS)[:25]
    got = R.coupling_grads(L, X, pairs)
    for p in pairs:
        assert np.allclose(got[p], dS[p], rtol=1e-12, atol=1e-12 * np.abs(dS[p]).max())


def test_rows_match_the_full_complex_product():
    """K = C (the regularised Helmholtz kernel): complex rows, complex α."""
    pts = sphere_points(1500, 4)
    g = O.helmholtz_kernel(1.0, 0.05)
    H = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, kernel=g, sigma=1e-2)
    R = O.H2Rows(pts, q=3, leaf_size=32, eta=2.0, sigma=1e-2, kernel=g)
    X = gaussian_rhs(1500, 3, 8) + 1j * gaussian_rhs(1500, 3, 9)
    rows = [0, 17, 640, 999, 1499]
    full = O.h2mm(H, 0.3 - 0.2j, X)
    got = R.rows(0.3 - 0.2j, X, rows)
    assert np.iscomplexobj(got)
    assert rel_fro(got, full[rows]) <= 1e-13
