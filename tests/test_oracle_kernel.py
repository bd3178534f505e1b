"""Pins of the kernel function g and the diagonal shift (Sec. 2: the matrix
entries g(x_i, x_j) of the inadmissible blocks and the nodes' values in the
coupling matrices), against values worked out by hand, not by the oracle.

The construction reads g(x, y) = exp(-|x - y|_2 / l) with l = 0.5 and the
shift sigma on the diagonal only.  A misread length scale (exp(-r·l),
exp(-r²/l), exp(-r/(2l))), a norm other than the Euclidean one, or sigma
added off the diagonal each fail one of these."""
import math

import numpy as np

from oracle import h2_oracle as O


def test_exp_kernel_at_hand_computed_pairs():
    g = O.exp_kernel(0.5)
    # |(0.3, 0.4, 0)| = 0.5 (a 3-4-5 triangle), so g = exp(-0.5 / 0.5) = e^-1
    assert abs(float(g(np.zeros(3), np.array([0.3, 0.4, 0.0]))) - math.exp(-1.0)) <= 1e-16
    # |(1, 2, 2)| = 3, so g = exp(-3 / 0.5) = e^-6; the kernel depends on x - y only
    x, y = np.array([1.0, -1.0, 0.5]), np.array([0.0, -3.0, -1.5])
    assert abs(float(g(x, y)) - math.exp(-6.0)) <= 1e-18
    assert float(g(x, y)) == float(g(y, x))
    # coincident points: g = 1
    assert float(g(x, x)) == 1.0
    # another length scale: l = 0.25 at distance 0.5 gives e^-2
    assert abs(float(O.exp_kernel(0.25)(np.zeros(3), np.array([0.0, 0.0, 0.5]))) - math.exp(-2.0)) <= 1e-17


def test_exp_kernel_broadcasts_over_leading_axes():
    g = O.exp_kernel(0.5)
    a = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    K = g(a[:, None, :], a[None, :, :])
    want = np.array([[1.0, math.exp(-1.0)], [math.exp(-1.0), 1.0]])
    assert np.allclose(K, want, rtol=0, atol=1e-16)


def test_shift_lives_on_the_diagonal_only():
    # two points at distance 0.5: K = [[1 + s, e^-1], [e^-1, 1 + s]]
    pts = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    K = O.kernel_matrix(pts, O.exp_kernel(0.5), sigma=0.125)
    want = np.array([[1.125, math.exp(-1.0)], [math.exp(-1.0), 1.125]])
    assert np.allclose(K, want, rtol=0, atol=1e-16)


def test_h2_matrix_entries_use_the_kernel_and_shift_as_stated():
    """A single-cluster H² matrix (n <= leaf size) is one inadmissible block:
    its dense expansion is exactly [g(x_i, x_j)] + sigma I.  Points on a line
    at spacing 0.25 give g = exp(-|i - j| / 2) for l = 0.5."""
    n = 6
    pts = np.zeros((n, 3))
    pts[:, 0] = 0.25 * np.arange(n)
    H = O.H2Matrix(pts, q=2, leaf_size=64, eta=2.0, sigma=0.01, length=0.5)
    A = O.dense_expand(H)
    i = np.arange(n)
    want = np.exp(-np.abs(i[:, None] - i[None, :]) / 2.0) + 0.01 * np.eye(n)
    assert np.allclose(A, want, rtol=0, atol=1e-15)
    # the product applies the shift once: A·e_0 is the first column
    e0 = np.zeros(n)
    e0[0] = 1.0
    assert np.allclose(O.h2mm(H, 1.0, e0), want[:, 0], rtol=0, atol=1e-15)


def test_coupling_matrices_are_the_kernel_at_the_nodes():
    """S_b[ν, μ] = g(ξ_{t,ν}, ξ_{s,μ}) (Eq. (h2_admissible)): every entry of
    a stored coupling matrix is exp(-r/l) at the Euclidean distance r of the
    two tensor nodes, computed here with math.dist / math.exp."""
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1.0, 1.0, size=(400, 3))
    H = O.H2Matrix(pts, q=2, leaf_size=16, eta=2.0, sigma=0.0, length=0.5)
    assert H.adm, "the point set must produce admissible blocks"
    for b in H.adm[:5]:
        xt, xs = H.tnodes[b.t.id], H.tnodes[b.s.id]
        for nu in range(H.k):
            for mu in range(H.k):
                r = math.dist(tuple(xt[nu]), tuple(xs[mu]))
                assert abs(b.S[nu, mu] - math.exp(-r / 0.5)) <= 1e-15
