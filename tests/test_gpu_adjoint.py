"""GPU adjoint through the C ABI: Aᵀ solve, ∂L/∂S_b = −λ̂_t x̂_sᵀ and
∂L/∂σ = −<Λ, X>_F against the oracle, and the torch.autograd wrapper against
central finite differences of the loss L = |X − X_target|_F² evaluated with
dense solves of the same H² matrix (n = 4096, q = 3, FP64)."""
import numpy as np
import pytest
import scipy.linalg as sla

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu

N, M = 4096, 4


@pytest.fixture(scope="module")
def case():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    pts = sphere_points(N, 0)
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    T = P.h2_tree_build(pts, leaf_size=64, eta=2.0)
    pairs = [(t, int(T["adm_col"][j])) for t in range(T["n_clusters"])
             for j in range(T["adm_rowptr"][t], T["adm_rowptr"][t + 1])]
    return P, H, G, pairs


def test_adjoint_grads_match_oracle(case):
    torch = require_cuda()
    P, H, G, pairs = case
    A = O.dense_expand(H)
    B = gaussian_rhs(N, M, 1)
    Xt = gaussian_rhs(N, M, 2)
    X = np.ascontiguousarray(sla.cho_solve(sla.cho_factor(A), B))
    Lam = np.ascontiguousarray(sla.cho_solve(sla.cho_factor(A.T), 2 * (X - Xt)))
    dS, dsig = P.h2_adjoint_grads(G.handle, torch.from_numpy(Lam).cuda(), torch.from_numpy(X).cuda())
    dS = dS.cpu().numpy()
    ref, ref_sig = O.adjoint_grads(H, Lam, X)
    assert len(pairs) == len(ref) == dS.shape[0]
    num = sum(np.sum((dS[j] - ref[p]) ** 2) for j, p in enumerate(pairs))
    den = sum(np.sum(ref[p] ** 2) for p in pairs)
    assert np.sqrt(num / den) <= 1e-12
    assert abs(dsig - ref_sig) <= 1e-12 * abs(ref_sig)


def test_transposed_solve(case):
    torch = require_cuda()
    P, H, G, pairs = case
    A = O.dense_expand(H)
    B = gaussian_rhs(N, M, 3)
    Xd = torch.zeros(N, M, dtype=torch.float64, device="cuda")
    res = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=1e-10, transposed=True)
    assert res.status == 0
    Xref = np.linalg.solve(A.T, B)
    assert rel_fro(Xd.cpu().numpy(), Xref) <= 1e-8


def test_autograd_matches_finite_differences(case):
    torch = require_cuda()
    P, H, G, pairs = case
    B0 = gaussian_rhs(N, M, 5)
    Xt = gaussian_rhs(N, M, 6)
    S0 = P.h2_coupling_get(G.handle, torch.zeros((len(pairs), 27, 27), dtype=torch.float64, device="cuda"))
    B = torch.from_numpy(B0).cuda().requires_grad_(True)
    sigma = torch.tensor(1e-2, dtype=torch.float64, device="cuda", requires_grad=True)
    S = S0.clone().requires_grad_(True)
    X = P.h2_solve(B, sigma, S, G, tol=1e-12)
    loss = ((X - torch.from_numpy(Xt).cuda()) ** 2).sum()
    loss.backward()
    gB, gsig, gS = B.grad.cpu().numpy(), float(sigma.grad), S.grad.cpu().numpy()

    base_S = {(b.t.id, b.s.id): b.S.copy() for b in H.adm}

    def dense_loss(Bm, sig, dS_dir=None, eps=0.0):
        S = dict(base_S)
        if dS_dir is not None:
            for j, d in dS_dir.items():
                S[pairs[j]] = base_S[pairs[j]] + eps * d
        O.set_coupling(H, S)
        H.sigma = sig
        A = O.dense_expand(H)
        # LU, not Cholesky: perturbing one S_b makes A non-symmetric
        X = np.linalg.solve(A, Bm)
        return float(np.sum((X - Xt) ** 2))

    # ∂L/∂σ
    h = 1e-7
    fd = (dense_loss(B0, 1e-2 + h) - dense_loss(B0, 1e-2 - h)) / (2 * h)
    assert abs(fd - gsig) <= 1e-6 * abs(fd)
    # ∂L/∂B along a random direction
    D = gaussian_rhs(N, M, 7)
    hb = 1e-6
    fd = (dense_loss(B0 + hb * D, 1e-2) - dense_loss(B0 - hb * D, 1e-2)) / (2 * hb)
    assert abs(fd - float(np.sum(gB * D))) <= 1e-6 * abs(fd)
    # ∂L/∂S along a random direction on a few blocks
    rng = np.random.default_rng(1)
    dirs = {int(j): rng.standard_normal((27, 27)) for j in rng.choice(len(pairs), 8, replace=False)}
    hs = 1e-6
    fd = (dense_loss(B0, 1e-2, dirs, hs) - dense_loss(B0, 1e-2, dirs, -hs)) / (2 * hs)
    pred = sum(float(np.sum(gS[j] * d)) for j, d in dirs.items())
    assert abs(fd - pred) <= 1e-6 * abs(fd)
    O.set_coupling(H, base_S)
    H.sigma = 1e-2
