"""GPU Gram-matrix block CG (variant H2_CG_GRAM: O'Leary's block CG with FP64
Gram matrices and a deflating Cholesky) through the C ABI, against the oracle's
block_cg_gram and a dense Cholesky solve of the same H² matrix."""
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
    cf = sla.cho_factor(A)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    return A, cf, G


def _true_rel(A, B, X):
    return np.linalg.norm(B - A @ X, axis=0) / np.maximum(np.linalg.norm(B, axis=0), 1e-300)


@pytest.mark.parametrize("m", [8, 17, 64])
def test_gram_fp64_matches_oracle_and_dense_solve(case4096, m):
    torch = require_cuda()
    A, cf, G = case4096
    B = gaussian_rhs(4096, m, 1)
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    res = G.block_cg(Bd, Xd, tol=1e-8, max_iter=5000, dtype="f64", variant="gram", check_every=1)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert _true_rel(A, B, X).max() <= 1.5e-8  # dense recomputation in another rounding order
    assert res.rel_residual.max() <= 1e-8  # the solver confirms convergence on this FP64 residual
    assert rel_fro(X, sla.cho_solve(cf, B)) <= 1e-6
    ref = O.block_cg_gram(lambda Z: A @ Z, B, tol=1e-8, max_iter=5000)
    assert ref.status == "converged"
    # Same recurrences, different rounding order.  Block CG on this matrix is
    # sensitive to rounding: perturbing the oracle's products by 1e-15 moves its
    # count by up to 12 % (m = 64: 66..81), and the count on another host's BLAS
    # differs as much, so the counts agree within 20 %.
    assert abs(res.iterations - ref.iterations) <= max(5, ref.iterations // 5), (res.iterations, ref.iterations)
    cw = O.block_cg(lambda Z: A @ Z, B, tol=1e-8, max_iter=5000)
    assert res.iterations < cw.iterations


def test_gram_iterates_match_oracle(case4096):
    """A fixed number of steps (tol = 0) from the same start: the GPU iterate
    equals the oracle's.  Rounding differences grow fast once Ritz values
    converge (oracle vs oracle with another product order: 1e-14 after 5 steps,
    3e-10 after 8, 1e-6 after 10), so the comparison stops at 5 steps."""
    torch = require_cuda()
    A, cf, G = case4096
    B = gaussian_rhs(4096, 5, 3)
    for k, tol in ((1, 1e-12), (3, 1e-11), (5, 1e-9)):
        Xd = torch.zeros(4096, 5, dtype=torch.float64, device="cuda")
        res = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=0.0, max_iter=k, dtype="f64", variant="gram")
        assert res.iterations == k
        ref = O.block_cg_gram(lambda Z: A @ Z, B, tol=0.0, max_iter=k)
        assert rel_fro(Xd.cpu().numpy(), ref.X) <= tol, k


@pytest.mark.parametrize("refine", [1, 2])
def test_gram_mixed_precision_reaches_fp64_tolerance(case4096, refine):
    torch = require_cuda()
    A, cf, G = case4096
    B = gaussian_rhs(4096, 16, 4)
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    res = G.block_cg(Bd, Xd, tol=1e-8, max_iter=5000, dtype="f32", variant="gram", refine=refine,
                     inner_tol=0.1 if refine == 2 else 1e-4, check_every=2)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert _true_rel(A, B, X).max() <= 1.5e-8
    assert res.rel_residual.max() <= 1e-8  # the solver decides on this FP64 residual
    assert rel_fro(X, sla.cho_solve(cf, B)) <= 1e-6
    assert res.outer_steps >= 1


def test_gram_single_column_is_scalar_cg(case4096):
    torch = require_cuda()
    A, cf, G = case4096
    B = gaussian_rhs(4096, 1, 5)
    it = {}
    for var in ("gram", "columnwise"):
        Xd = torch.zeros(4096, 1, dtype=torch.float64, device="cuda")
        r = G.block_cg(torch.from_numpy(B).cuda(), Xd, tol=1e-8, max_iter=5000, dtype="f64", variant=var)
        assert r.status == 0
        it[var] = r.iterations
    # equal in exact arithmetic; rounding moves the counts by a few per cent
    assert abs(it["gram"] - it["columnwise"]) <= max(5, it["columnwise"] // 20), it


def test_gram_rank_deficient_rhs(case4096):
    torch = require_cuda()
    A, cf, G = case4096
    B = gaussian_rhs(4096, 6, 6)
    B[:, 1] = B[:, 0]
    B[:, 3] = 2.0 * B[:, 0] - B[:, 2]
    B[:, 5] = 0.0
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    res = G.block_cg(Bd, Xd, tol=1e-8, max_iter=5000, dtype="f64", variant="gram")
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert np.all(X[:, 5] == 0.0)
    assert _true_rel(A, B[:, :5], X[:, :5]).max() <= 1.5e-8
    assert rel_fro(X, sla.cho_solve(cf, B)) <= 1e-6


def test_gram_too_many_columns_rejected(case4096, P):
    torch = require_cuda()
    A, cf, G = case4096
    B = torch.zeros(4096, 65, dtype=torch.float64, device="cuda")
    with pytest.raises(P.H2Error) as e:
        G.block_cg(B, torch.zeros_like(B), variant="gram")
    assert e.value.code == P.H2_E_UNSUPPORTED


def test_gram_indefinite_matrix_reported(P):
    """q = 2 at n = 4096 is indefinite (32 negative eigenvalues of Â): the
    solve ends with breakdown or no convergence, never a hang."""
    torch = require_cuda()
    pts = sphere_points(4096, 0)
    G = P.H2Matrix(pts, q=2, leaf_size=64, eta=2.0, sigma=1e-2)
    B = torch.from_numpy(gaussian_rhs(4096, 4, 1)).cuda()
    res = G.block_cg(B, torch.zeros_like(B), tol=1e-10, max_iter=3000, dtype="f64", variant="gram")
    assert res.status in (P.H2_E_BREAKDOWN, P.H2_E_NOCONVERGE)
