"""Pins of the oracle's adjoint gradients: central finite differences of a
loss through a dense solve of the same H² matrix, and the dense formula
V_tᵀ(−Λ Xᵀ)|_{t̂×ŝ} V_s built from independently expanded bases."""
import numpy as np
import scipy.linalg as sla

from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def _setup(n=600, m=3):
    pts = sphere_points(n, 4)
    H = O.H2Matrix(pts, q=3, leaf_size=32, eta=2.0, sigma=0.05)
    B = gaussian_rhs(n, m, 1)
    Xt = gaussian_rhs(n, m, 2)
    return H, B, Xt


def _loss(H, B, Xt):
    A = O.dense_expand(H)
    X = np.linalg.solve(A, B)
    return float(np.sum((X - Xt) ** 2)), A, X


def test_adjoint_matches_dense_formula():
    H, B, Xt = _setup()
    _, A, X = _loss(H, B, Xt)
    Lam = np.linalg.solve(A.T, 2 * (X - Xt))
    dS, dsig = O.adjoint_grads(H, Lam, X)
    dA = -Lam @ X.T
    for b in H.adm[:40]:
        Vt = O.tensor_lagrange(H.nodes[b.t.id], H.points[b.t.idx])  # direct evaluation, not the nesting
        Vs = O.tensor_lagrange(H.nodes[b.s.id], H.points[b.s.idx])
        ref = Vt.T @ dA[np.ix_(b.t.idx, b.s.idx)] @ Vs
        assert np.allclose(dS[(b.t.id, b.s.id)], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert abs(dsig - float(np.trace(dA))) <= 1e-10 * abs(dsig)


def test_adjoint_matches_finite_differences():
    H, B, Xt = _setup()
    L0, A, X = _loss(H, B, Xt)
    Lam = np.linalg.solve(A.T, 2 * (X - Xt))
    dS, dsig = O.adjoint_grads(H, Lam, X)
    # shift
    h = 1e-6
    H.sigma += h
    Lp = _loss(H, B, Xt)[0]
    H.sigma -= 2 * h
    Lm = _loss(H, B, Xt)[0]
    H.sigma += h
    assert abs((Lp - Lm) / (2 * h) - dsig) <= 1e-6 * abs(dsig)
    # right-hand side (dL/dB = Λ)
    D = gaussian_rhs(H.n, B.shape[1], 9)
    hb = 1e-5
    fd = (_loss(H, B + hb * D, Xt)[0] - _loss(H, B - hb * D, Xt)[0]) / (2 * hb)
    assert abs(fd - float(np.sum(Lam * D))) <= 1e-6 * abs(fd)
    # coupling matrices: a random direction on a few blocks
    rng = np.random.default_rng(3)
    blocks = [H.adm[i] for i in rng.choice(len(H.adm), 6, replace=False)]
    dirs = {(b.t.id, b.s.id): rng.standard_normal(b.S.shape) for b in blocks}
    base = {(b.t.id, b.s.id): b.S.copy() for b in H.adm}
    hs = 1e-5

    def loss_at(eps):
        S = dict(base)
        for key, d in dirs.items():
            S[key] = base[key] + eps * d
        O.set_coupling(H, S)
        return _loss(H, B, Xt)[0]

    fd = (loss_at(hs) - loss_at(-hs)) / (2 * hs)
    O.set_coupling(H, base)
    pred = sum(float(np.sum(dS[key] * d)) for key, d in dirs.items())
    assert abs(fd - pred) <= 1e-6 * abs(fd)
