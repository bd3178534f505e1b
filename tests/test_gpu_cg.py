"""GPU block CG (Sec. 5.1, Alg. "block CG") through the C ABI: FP64 and the
mixed-precision refinement against a dense Cholesky solve of the same H²
matrix (oracle), and honest failure on an indefinite matrix."""
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
    B = gaussian_rhs(4096, 8, 1)
    Xc = sla.cho_solve(sla.cho_factor(A), B)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    return A, B, Xc, G


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_block_cg_matches_dense_solve(case4096, inner):
    torch = require_cuda()
    A, B, Xc, G = case4096
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    res = G.block_cg(Bd, Xd, tol=1e-8, max_iter=20000, dtype=inner, inner_tol=1e-4)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    true_rel = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert true_rel.max() <= 1e-8 * 1.5, true_rel
    assert res.rel_residual.max() <= 1e-8  # the solver confirms convergence on this FP64 residual
    assert rel_fro(X, Xc) <= 1e-6
    if inner == "f64":
        ref = O.block_cg(lambda Z: A @ Z, B, tol=1e-8, max_iter=20000)
        # same recurrences on the same matrix, different rounding order (H² product on
        # the GPU, dense product in the oracle): iteration counts agree within 5 %
        assert abs(res.iterations - ref.iterations) <= max(10, ref.iterations // 20)
    else:
        assert res.outer_steps >= 1


def test_mixed_solve_with_reliable_updates(case4096):
    """refine=2: one FP32-product block CG whose recurrence residuals are
    replaced by the FP64 residual B - A X; reaches the FP64 tolerance."""
    torch = require_cuda()
    A, B, Xc, G = case4096
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    res = G.block_cg(Bd, Xd, tol=1e-8, max_iter=20000, dtype="f32", refine=2, inner_tol=0.1)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    true_rel = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert true_rel.max() <= 1e-8 * 1.5, true_rel
    assert res.rel_residual.max() <= 1e-8  # the solver decides on this FP64 residual
    assert rel_fro(X, Xc) <= 1e-6
    assert res.outer_steps >= 1  # at least one reliable update
    # the FP32 operator costs some iterations against FP64 CG (loss of
    # conjugacy); bounded here at 2x
    plain = O.block_cg(lambda Z: A @ Z, B, tol=1e-8, max_iter=20000)
    assert res.iterations <= 2 * plain.iterations


def test_block_cg_host_buffers_and_initial_guess(case4096):
    A, B, Xc, G = case4096
    X0 = Xc + 1e-4 * gaussian_rhs(4096, 8, 2)
    X = X0.copy()
    res = G.block_cg(B, X, tol=1e-8, dtype="f64")
    assert res.status == 0
    assert rel_fro(X, Xc) <= 1e-6
    cold = np.zeros_like(B)
    res_cold = G.block_cg(B, cold, tol=1e-8, dtype="f64")
    assert res.iterations <= res_cold.iterations


def test_zero_rhs_column(case4096):
    A, B, Xc, G = case4096
    B2 = B.copy()
    B2[:, 3] = 0.0
    X = np.zeros_like(B2)
    res = G.block_cg(B2, X, tol=1e-8)
    assert res.status == 0
    assert np.all(X[:, 3] == 0.0) and res.col_iterations[3] == 0


def test_indefinite_matrix_reported(P):
    pts = sphere_points(2048, 0)
    G = P.H2Matrix(pts, q=2, leaf_size=64, eta=2.0, sigma=1e-2, precisions=())
    B = gaussian_rhs(2048, 4, 1)
    X = np.zeros_like(B)
    res = G.block_cg(B, X, tol=1e-8, max_iter=3000)
    assert res.status in (P.H2_E_BREAKDOWN, P.H2_E_NOCONVERGE)


def test_max_iter_cap(case4096, P):
    A, B, Xc, G = case4096
    X = np.zeros_like(B)
    res = G.block_cg(B, X, tol=1e-8, max_iter=10)
    assert res.status == P.H2_E_NOCONVERGE and res.iterations == 10
