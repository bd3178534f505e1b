"""GPU block GMRES (Sec. 5.2, Alg. "pgmres block") through the C ABI against
the oracle's block_gmres and dense solves: the symmetric sphere matrix, a
non-symmetric one (coupling matrices perturbed asymmetrically on both sides),
the block-Jacobi preconditioner and the mixed-precision solve."""
import numpy as np
import pytest
import scipy.linalg as sla

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu
N = 4096


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


@pytest.fixture(scope="module")
def case(P):
    pts = sphere_points(N, 0)
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    T = P.h2_tree_build(pts, leaf_size=64, eta=2.0)
    pairs = [(t, int(T["adm_col"][j])) for t in range(T["n_clusters"])
             for j in range(T["adm_rowptr"][t], T["adm_rowptr"][t + 1])]
    return H, G, pairs


def _true_rel(A, B, X):
    return np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)


def test_gmres_fp64_matches_oracle(case):
    torch = require_cuda()
    H, G, pairs = case
    A = O.dense_expand(H)
    B = gaussian_rhs(N, 6, 1)
    Xd = torch.zeros(N, 6, dtype=torch.float64, device="cuda")
    res = G.block_gmres(torch.from_numpy(B).cuda(), Xd, tol=1e-8, restart=30, max_iter=5000)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert _true_rel(A, B, X).max() <= 1.5e-8
    assert rel_fro(X, sla.cho_solve(sla.cho_factor(A), B)) <= 1e-6
    ref = O.block_gmres(lambda Z: A @ Z, B, tol=1e-8, restart=30, max_iter=5000)
    assert ref.status == "converged"
    # same recurrences, different rounding order
    assert abs(res.iterations - ref.iterations) <= max(5, ref.iterations // 10), (res.iterations, ref.iterations)


def test_gmres_steps_match_oracle_iterates(case):
    """A fixed number of Arnoldi steps inside one cycle: the iterate after the
    cycle's update equals the oracle's."""
    torch = require_cuda()
    H, G, pairs = case
    A = O.dense_expand(H)
    B = gaussian_rhs(N, 3, 2)
    for k in (1, 5):
        Xd = torch.zeros(N, 3, dtype=torch.float64, device="cuda")
        res = G.block_gmres(torch.from_numpy(B).cuda(), Xd, tol=0.0, restart=30, max_iter=k)
        assert res.status == -3  # H2_E_NOCONVERGE: the step cap ended the solve
        ref = O.block_gmres(lambda Z: A @ Z, B, tol=0.0, restart=30, max_iter=k)
        assert rel_fro(Xd.cpu().numpy(), ref.X) <= 1e-10, k


@pytest.fixture(scope="module")
def nonsym(P):
    """σ = 0.5 and every coupling matrix perturbed entrywise by 5 %: a
    non-symmetric, well-conditioned H² matrix (restarted GMRES converges in
    about 160 steps in the oracle)."""
    torch = require_cuda()
    pts = sphere_points(N, 0)
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=0.5)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=0.5, precisions=("f32",))
    T = P.h2_tree_build(pts, leaf_size=64, eta=2.0)
    pairs = [(t, int(T["adm_col"][j])) for t in range(T["n_clusters"])
             for j in range(T["adm_rowptr"][t], T["adm_rowptr"][t + 1])]
    S0 = P.h2_coupling_get(G.handle, torch.zeros((len(pairs), 27, 27), dtype=torch.float64, device="cuda"))
    rng = np.random.default_rng(3)
    S1 = S0.cpu().numpy() * (1.0 + 0.05 * rng.standard_normal(tuple(S0.shape)))
    P.h2_coupling_set(G.handle, torch.from_numpy(S1).cuda())
    O.set_coupling(H, {p: S1[j] for j, p in enumerate(pairs)})
    return H, G


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_gmres_nonsymmetric(nonsym, dtype):
    torch = require_cuda()
    H, G = nonsym
    A = O.dense_expand(H)
    assert np.abs(A - A.T).max() > 1e-2
    B = gaussian_rhs(N, 4, 4)
    Xd = torch.zeros(N, 4, dtype=torch.float64, device="cuda")
    res = G.block_gmres(torch.from_numpy(B).cuda(), Xd, tol=1e-8, restart=40, max_iter=3000, dtype=dtype)
    assert res.status == 0, res
    X = Xd.cpu().numpy()
    assert _true_rel(A, B, X).max() <= 1.5e-8
    assert rel_fro(X, np.linalg.solve(A, B)) <= 1e-7
    if dtype == "f64":
        ref = O.block_gmres(lambda Z: A @ Z, B, tol=1e-8, restart=40, max_iter=3000)
        assert abs(res.iterations - ref.iterations) <= max(5, ref.iterations // 10), (res.iterations, ref.iterations)
    else:
        assert res.outer_steps >= 2  # the FP64 restarts refine the FP32 cycles


def test_gmres_transposed(nonsym):
    """Aᵀ X = B through the transposed products."""
    torch = require_cuda()
    H, G = nonsym
    A = O.dense_expand(H)
    B = gaussian_rhs(N, 3, 8)
    Xd = torch.zeros(N, 3, dtype=torch.float64, device="cuda")
    res = G.block_gmres(torch.from_numpy(B).cuda(), Xd, tol=1e-9, restart=40, max_iter=3000, transposed=True)
    assert res.status == 0, res
    assert rel_fro(Xd.cpu().numpy(), np.linalg.solve(A.T, B)) <= 1e-7


def test_gmres_block_jacobi(case):
    torch = require_cuda()
    H, G, pairs = case
    A = O.dense_expand(H)
    B = gaussian_rhs(N, 5, 6)
    out = {}
    for pc in (None, "block_jacobi"):
        Xd = torch.zeros(N, 5, dtype=torch.float64, device="cuda")
        res = G.block_gmres(torch.from_numpy(B).cuda(), Xd, tol=1e-9, restart=30, max_iter=5000, precond=pc)
        assert res.status == 0, res
        assert rel_fro(Xd.cpu().numpy(), sla.cho_solve(sla.cho_factor(A), B)) <= 1e-6
        out[pc] = res.iterations
    assert out["block_jacobi"] < out[None]
    ref = O.block_gmres(lambda Z: A @ Z, B, tol=1e-9, restart=30, max_iter=5000, apply_Minv=O.block_jacobi(H))
    assert abs(out["block_jacobi"] - ref.iterations) <= max(5, ref.iterations // 10)


def test_gmres_argument_errors(case, P):
    torch = require_cuda()
    H, G, pairs = case
    B = torch.zeros(N, 2, dtype=torch.float64, device="cuda")
    for kw in ({"restart": 0}, {"restart": 65}):
        with pytest.raises(P.H2Error) as e:
            G.block_gmres(B, torch.zeros_like(B), **kw)
        assert e.value.code == P.H2_E_BADARG
    with pytest.raises(P.H2Error) as e:
        G.block_gmres(np.zeros((N, 2)), np.zeros((N, 2)))
    assert e.value.code == P.H2_E_BADARG
