"""Pins of the oracle's complex case (K = C, Sec. 2: the Helmholtz kernel
g_κ(x, y) = exp(iκ|x - y|) / (4π|x - y|), here regularised at r = 0 as
exp(iκr) / (4π sqrt(r² + δ²))).

* the kernel at pairs worked out by hand, its δ = 0 and κ = 0 limits, its
  symmetry (g(x, y) = g(y, x), not conjugate-symmetric);
* the complex product against brute force: a complex kernel that tensor
  interpolation of order q reproduces exactly gives A = K + σI, so h2mm
  must equal (K + σI)·X for complex X and complex α;
* the complex product against the (separately pinned) real one: the bases
  are real, so the H² matrix of g is the H² matrix of Re g plus i times
  that of Im g, and (A_re + i A_im)(X_re + i X_im) splits into four real
  products; a wrong sign, a conjugation or swapped real and imaginary parts
  anywhere in the complex path fails this;
* Aᵀ = A for the symmetric kernel (no conjugation), and the interpolation
  error against the dense kernel matrix falls with q."""
import math

import numpy as np
import pytest

from _helpers import rel_fro
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def test_helmholtz_kernel_at_hand_computed_pairs():
    # |(0.3, 0.4, 0)| = 0.5; δ = 0: e^{0.5 i} / (4π·0.5)
    g0 = O.helmholtz_kernel(kappa=1.0, delta=0.0)
    v = complex(g0(np.zeros(3), np.array([0.3, 0.4, 0.0])))
    assert abs(v - complex(math.cos(0.5), math.sin(0.5)) / (2.0 * math.pi)) <= 1e-16
    # |(1, 2, 2)| = 3, κ = 2: e^{6i} / (12π); depends on x - y only
    g2 = O.helmholtz_kernel(kappa=2.0, delta=0.0)
    x = np.array([0.5, -1.0, 2.0])
    v = complex(g2(x, x + np.array([1.0, 2.0, 2.0])))
    assert abs(v - complex(math.cos(6.0), math.sin(6.0)) / (12.0 * math.pi)) <= 1e-16
    # regularised: r = |(0.18, 0.24, 0)| = 0.3 and δ = 0.4 give sqrt(r² + δ²) = 0.5
    gd = O.helmholtz_kernel(kappa=1.0, delta=0.4)
    v = complex(gd(np.zeros(3), np.array([0.18, 0.24, 0.0])))
    assert abs(v - complex(math.cos(0.3), math.sin(0.3)) / (4.0 * math.pi * 0.5)) <= 1e-16
    # the diagonal is 1 / (4π δ), real
    v = complex(gd(x, x))
    assert v.imag == 0.0 and abs(v.real - 1.0 / (1.6 * math.pi)) <= 1e-16


def test_helmholtz_kernel_limits_and_symmetry():
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((50, 3)), rng.standard_normal((50, 3))
    r = np.linalg.norm(x - y, axis=1)
    # κ = 0: the (regularised) Laplace kernel, real
    g = O.helmholtz_kernel(kappa=0.0, delta=0.05)(x, y)
    assert np.all(g.imag == 0.0)
    assert np.allclose(g.real, 1.0 / (4.0 * np.pi * np.sqrt(r * r + 0.0025)), rtol=1e-15, atol=0)
    # symmetric, and not conjugate-symmetric
    h = O.helmholtz_kernel(kappa=1.0, delta=0.05)
    assert np.array_equal(h(x, y), h(y, x))
    assert np.abs(h(x, y).imag).max() > 0.1 / (4 * np.pi * r.max())


def _bilinear_complex_kernel(x, y):
    """Degree <= 2 per coordinate: reproduced exactly by tensor interpolation with q >= 3."""
    dot = (x[..., 0] * y[..., 0] + x[..., 1] * y[..., 1]) + x[..., 2] * y[..., 2]
    return (1.0 + 2.0j) * dot + (0.5 - 1.0j) * (x[..., 0] * x[..., 0]) * y[..., 2] + 0.25j


@pytest.mark.parametrize("transposed", [False, True])
def test_complex_product_reproduces_an_interpolable_kernel(transposed):
    pts = sphere_points(700, 5)
    H = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, kernel=_bilinear_complex_kernel, sigma=0.3)
    assert np.dtype(H.dtype).kind == "c" and len(H.adm) > 0
    K = O.kernel_matrix(pts, _bilinear_complex_kernel, sigma=0.3)
    X = gaussian_rhs(700, 3, 1) + 1j * gaussian_rhs(700, 3, 2)
    Y0 = gaussian_rhs(700, 3, 3) - 0.5j * gaussian_rhs(700, 3, 4)
    alpha = 0.7 - 1.3j
    got = O.h2mm(H, alpha, X, Y0, transposed=transposed)
    ref = Y0 + alpha * ((K.T if transposed else K) @ X)
    assert rel_fro(got, ref) <= 1e-12
    assert rel_fro(O.dense_expand(H), K) <= 1e-12


def test_complex_product_splits_into_real_products():
    pts = sphere_points(1500, 7)
    kap, dl, sig = 1.0, 0.05, 0.02
    g = O.helmholtz_kernel(kap, dl)
    Hc = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, kernel=g, sigma=sig)
    Hr = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, kernel=lambda x, y: g(x, y).real, sigma=sig)
    Hi = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, kernel=lambda x, y: g(x, y).imag, sigma=0.0)
    assert np.dtype(Hr.dtype).kind == "f" and np.dtype(Hi.dtype).kind == "f"
    Xr, Xi = gaussian_rhs(1500, 4, 11), gaussian_rhs(1500, 4, 12)
    got = O.h2mm(Hc, 1.0, Xr + 1j * Xi)
    re = O.h2mm(Hr, 1.0, Xr) - O.h2mm(Hi, 1.0, Xi)
    im = O.h2mm(Hr, 1.0, Xi) + O.h2mm(Hi, 1.0, Xr)
    assert rel_fro(got, re + 1j * im) <= 1e-13
    # α enters as one complex factor
    a = -0.4 + 2.5j
    assert rel_fro(O.h2mm(Hc, a, Xr + 1j * Xi), a * got) <= 1e-14


def test_complex_symmetric_kernel_gives_a_symmetric_matrix():
    pts = sphere_points(900, 9)
    H = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, kernel=O.helmholtz_kernel(1.0, 0.05), sigma=0.01)
    X = gaussian_rhs(900, 2, 5) + 1j * gaussian_rhs(900, 2, 6)
    assert rel_fro(O.h2mm(H, 1.0, X, transposed=True), O.h2mm(H, 1.0, X)) <= 1e-13
    A = O.dense_expand(H)
    assert rel_fro(A, A.T) <= 1e-13
    assert rel_fro(A, A.conj().T) > 1e-3  # symmetric, not Hermitian


def test_helmholtz_interpolation_error_falls_with_q():
    pts = sphere_points(1200, 13)
    g = O.helmholtz_kernel(1.0, 0.05)
    K = O.kernel_matrix(pts, g)
    errs = []
    for q in (2, 3, 4):
        H = O.H2Matrix(pts, q=q, leaf_size=32, eta=2.0, kernel=g)
        errs.append(rel_fro(O.dense_expand(H), K))
    assert errs[0] > 3 * errs[1] > 9 * errs[2], errs


def _mut_addeval_conj(H, alpha, b, xhat, yhat, X, Y, transposed):
    if b.kind == "adm":
        yhat[b.t.id] += alpha * (b.S.conj() @ xhat[b.s.id])  # planted: conjugated coupling
    elif b.kind == "near":
        Y[b.t.idx] += alpha * (b.G @ X[b.s.idx])
    else:
        for b2 in b.sons:
            _mut_addeval_conj(H, alpha, b2, xhat, yhat, X, Y, transposed)


def _mut_addeval_near_conj(H, alpha, b, xhat, yhat, X, Y, transposed):
    if b.kind == "adm":
        yhat[b.t.id] += alpha * (b.S @ xhat[b.s.id])
    elif b.kind == "near":
        Y[b.t.idx] += alpha * (b.G.conj() @ X[b.s.idx])  # planted: conjugated nearfield
    else:
        for b2 in b.sons:
            _mut_addeval_near_conj(H, alpha, b2, xhat, yhat, X, Y, transposed)


def _mut_forward_real_part(H, s, X, xhat):
    if s.is_leaf:
        xhat[s.id] = H.V[s.id].T @ X[s.idx].real  # planted: imaginary part of X dropped
    else:
        acc = np.zeros((H.k, X.shape[1]), dtype=X.dtype)
        for s2 in s.sons:
            _mut_forward_real_part(H, s2, X, xhat)
            acc = acc + H.E[s2.id].T @ xhat[s2.id]
        xhat[s.id] = acc


@pytest.mark.parametrize("name,target,mutant", [
    ("coupling conjugated", "_fast_addeval", _mut_addeval_conj),
    ("nearfield conjugated", "_fast_addeval", _mut_addeval_near_conj),
    ("imaginary part of X dropped in the forward pass", "_forward", _mut_forward_real_part),
])
def test_complex_pins_catch_planted_mistakes(monkeypatch, name, target, mutant):
    pts = sphere_points(700, 5)
    H = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, kernel=_bilinear_complex_kernel, sigma=0.3)
    K = O.kernel_matrix(pts, _bilinear_complex_kernel, sigma=0.3)
    X = gaussian_rhs(700, 3, 1) + 1j * gaussian_rhs(700, 3, 2)
    monkeypatch.setattr(O, target, mutant)
    assert rel_fro(O.h2mm(H, 1.0, X), K @ X) > 1e-6, name
