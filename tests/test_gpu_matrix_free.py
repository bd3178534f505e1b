"""Matrix-free coupling (dtype "f32mf"): the tensor-core coupling kernel
evaluates S_b[ν, μ] = g(ξ_{t,ν}, ξ_{s,μ}) (Eq. (h2_admissible)) from the
Chebyshev nodes instead of reading the stored S_b.  The product must match the
FP64 oracle to the FP32 tolerance (1e-5), and the stored FP32 product to the
accuracy of the FP32 kernel evaluation; it refuses Aᵀ and couplings replaced
through h2_coupling_set."""
import numpy as np
import pytest

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import ellipsoid_points, gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu

TOL_ORACLE = 1e-5
TOL_STORED = 2e-6  # FP32 exp/sqrt of the kernel against the FP64-built, FP32-rounded S_b


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


def _apply(G, X, Y0, alpha, dtype):
    torch = require_cuda()
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y0).cuda()
    G.matmul(Xd, Yd, alpha=alpha, dtype=dtype)
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


@pytest.fixture(scope="module", params=[(3, "sphere"), (4, "ellipsoid")])
def case(P, request):
    q, shape = request.param
    n = 6000
    pts = sphere_points(n, 1) if shape == "sphere" else ellipsoid_points(n, (0.6, 1.9, 1.2), 2)
    H = O.H2Matrix(pts, q=q, leaf_size=64, eta=2.0, sigma=1e-2, length=0.5)
    G = P.H2Matrix(pts, q=q, leaf_size=64, eta=2.0, sigma=1e-2, length=0.5, precisions=("f32",))
    return n, H, G


@pytest.mark.parametrize("m", [1, 8, 20, 32, 64, 70])
def test_matrix_free_matches_oracle_and_stored(case, m):
    n, H, G = case
    X = gaussian_rhs(n, m, 30 + m)
    Y0 = gaussian_rhs(n, m, 40 + m)
    alpha = 0.75
    want = O.h2mm(H, alpha, X, Y0)
    got = _apply(G, X, Y0, alpha, "f32mf")
    stored = _apply(G, X, Y0, alpha, "f32")
    assert rel_fro(got, want) <= TOL_ORACLE
    assert rel_fro(got - Y0, stored - Y0) <= TOL_STORED


def test_matrix_free_is_deterministic(case):
    n, H, G = case
    X = gaussian_rhs(n, 32, 5)
    Y0 = np.zeros((n, 32))
    a = _apply(G, X, Y0, 1.0, "f32mf")
    b = _apply(G, X, Y0, 1.0, "f32mf")
    assert np.array_equal(a, b)


def test_matrix_free_refuses_transposed(P, case):
    n, H, G = case
    torch = require_cuda()
    X = torch.zeros(n, 4, dtype=torch.float64, device="cuda")
    Y = torch.zeros(n, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(P.H2Error):
        G.matmul_transposed(X, Y, dtype="f32mf")


def test_matrix_free_refuses_replaced_couplings(P):
    pts = sphere_points(3000, 3)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, length=0.5, precisions=("f32",))
    torch = require_cuda()
    X = torch.from_numpy(gaussian_rhs(3000, 4, 1)).cuda()
    Y = torch.zeros_like(X)
    G.matmul(X, Y, dtype="f32mf")  # allowed before any replacement
    S = P.h2_coupling_get(G.handle)
    P.h2_coupling_set(G.handle, S)
    with pytest.raises(P.H2Error):
        G.matmul(X, Y, dtype="f32mf")
