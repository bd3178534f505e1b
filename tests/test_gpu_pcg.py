"""GPU preconditioned block CG (Sec. 5.1, Alg. "pcg block") with the
block-Jacobi preconditioner on the diagonal nearfield blocks, through the C
ABI, against the oracle's block_pcg and a dense Cholesky solve."""
import numpy as np
import pytest
import scipy.linalg as sla

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


@pytest.fixture(scope="module")
def case4096(P):
    pts = sphere_points(4096, 0)
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    A = O.dense_expand(H)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    return H, A, sla.cho_factor(A), G


def _true_rel(A, B, X):
    return np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)


def test_pcg_fp64_matches_oracle_and_dense_solve(case4096):
    torch = require_cuda()
    H, A, cf, G = case4096
    B = gaussian_rhs(4096, 8, 1)
    Xd = torch.zeros(4096, 8, dtype=torch.float64, device="cuda")
    res = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=1e-8, max_iter=5000, dtype="f64", precond="block_jacobi")
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert _true_rel(A, B, X).max() <= 1.5e-8  # dense recomputation in another rounding order
    assert res.rel_residual.max() <= 1e-8  # the solver confirms convergence on this FP64 residual
    assert rel_fro(X, sla.cho_solve(cf, B)) <= 1e-6
    ref = O.block_pcg(lambda Z: A @ Z, O.block_jacobi(H), B, tol=1e-8, max_iter=5000)
    assert ref.status == "converged"
    assert abs(res.iterations - ref.iterations) <= max(5, ref.iterations // 20), (res.iterations, ref.iterations)
    plain = O.block_cg(lambda Z: A @ Z, B, tol=1e-8, max_iter=5000)
    assert res.iterations < plain.iterations


def test_pcg_iterates_match_oracle(case4096):
    torch = require_cuda()
    H, A, cf, G = case4096
    B = gaussian_rhs(4096, 3, 2)
    Minv = O.block_jacobi(H)
    for k in (1, 4):
        Xd = torch.zeros(4096, 3, dtype=torch.float64, device="cuda")
        res = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=0.0, max_iter=k, dtype="f64", precond="block_jacobi")
        assert res.iterations == k
        ref = O.block_pcg(lambda Z: A @ Z, Minv, B, tol=0.0, max_iter=k)
        assert rel_fro(Xd.cpu().numpy(), ref.X) <= 1e-10, k


@pytest.mark.parametrize("refine", [1, 2])
def test_pcg_mixed_precision(case4096, refine):
    torch = require_cuda()
    H, A, cf, G = case4096
    B = gaussian_rhs(4096, 70, 3)  # more than one 64-column chunk of the apply pass
    Xd = torch.zeros(4096, 70, dtype=torch.float64, device="cuda")
    res = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=1e-8, max_iter=5000, dtype="f32", refine=refine,
                     inner_tol=0.1 if refine == 2 else 1e-4, precond="block_jacobi", check_every=2)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert _true_rel(A, B, X).max() <= 1.5e-8  # dense recomputation in another rounding order
    assert res.rel_residual.max() <= 1e-8  # the solver confirms convergence on this FP64 residual
    assert rel_fro(X, sla.cho_solve(cf, B)) <= 1e-6
    if refine == 2:
        # the low-precision iterations apply M⁻¹ in FP32: no more iterations than
        # the FP64 solve with the FP64 apply, within a margin
        X64 = torch.zeros_like(Xd)
        r64 = G.block_cg(torch.from_numpy(B).cuda(), X64, tol=1e-8, max_iter=5000, dtype="f64",
                         precond="block_jacobi", check_every=2)
        assert r64.status == 0
        assert res.iterations <= 1.2 * r64.iterations + 10, (res.iterations, r64.iterations)


def test_pcg_shift_change_refactors(case4096, P):
    """The factors are formed for the current σ: after h2_shift_set the
    preconditioned solve still solves the shifted system."""
    torch = require_cuda()
    H, A, cf, G = case4096
    B = gaussian_rhs(4096, 2, 4)
    P.h2_shift_set(G.handle, 5e-2)
    try:
        Xd = torch.zeros(4096, 2, dtype=torch.float64, device="cuda")
        res = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=1e-9, max_iter=5000, dtype="f64",
                         precond="block_jacobi")
        assert res.status == 0
        A2 = A + (5e-2 - 1e-2) * np.eye(4096)
        assert rel_fro(Xd.cpu().numpy(), np.linalg.solve(A2, B)) <= 1e-6
    finally:
        P.h2_shift_set(G.handle, 1e-2)


def test_pcg_unsupported_combinations(case4096, P):
    torch = require_cuda()
    H, A, cf, G = case4096
    B = torch.zeros(4096, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.H2Error) as e:
        G.block_cg(B, torch.zeros_like(B), precond="block_jacobi", transposed=True)
    assert e.value.code == P.H2_E_UNSUPPORTED


@pytest.mark.parametrize("dtype,refine", [("f64", 0), ("f32", 2)])
def test_preconditioned_gram(case4096, dtype, refine):
    """Gram-matrix block CG with the block-Jacobi preconditioner: the oracle's
    block_cg_gram(apply_Minv=...) iteration count within 20 % (FP64) and the
    FP64 tolerance for the mixed solve."""
    torch = require_cuda()
    H, A, cf, G = case4096
    B = gaussian_rhs(4096, 32, 5)
    Xd = torch.zeros(4096, 32, dtype=torch.float64, device="cuda")
    res = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=1e-8, max_iter=5000, dtype=dtype, refine=refine,
                     inner_tol=0.1, variant="gram", precond="block_jacobi", check_every=1)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert _true_rel(A, B, X).max() <= 1.5e-8  # dense recomputation in another rounding order
    assert res.rel_residual.max() <= 1e-8  # the solver confirms convergence on this FP64 residual
    assert rel_fro(X, sla.cho_solve(cf, B)) <= 1e-6
    if dtype == "f64":
        ref = O.block_cg_gram(lambda Z: A @ Z, B, tol=1e-8, max_iter=5000, apply_Minv=O.block_jacobi(H))
        assert abs(res.iterations - ref.iterations) <= max(5, ref.iterations // 5), (res.iterations, ref.iterations)
