"""The q = 4 transfer passes with the transfer matrices as Kronecker products
(E_c = F_z ⊗ F_y ⊗ F_x of 4×4 factors, the 1-D Lagrange polynomials of the
father's nodes at the son's nodes: three 4×4 mode products instead of a
64×64 product) against the FP64 oracle and against the dense passes
(H2_KRON=0): the FP32 subtree passes (downward above 16 columns per chunk;
upward inner steps and climb), the FP64 one-launch passes, for 3 to 96
columns (one and two chunks), leaves on several levels, and repeated
products (bit for bit).  The oracle uses the dense E_c, so this also checks
that tensor Chebyshev interpolation makes E_c exactly that product."""
import numpy as np
import pytest

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import ellipsoid_points, gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


@pytest.fixture(scope="module")
def mp_module():
    mp = pytest.MonkeyPatch()
    yield mp
    mp.undo()


CASES = {
    "sphere20000_q4": (lambda: sphere_points(20000, 41), 4, 64),
    "ellipsoid_leaf20_q4": (lambda: ellipsoid_points(5000, (0.7, 1.6, 1.0), 43), 4, 20),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(P, request, mp_module):
    make, q, leaf = CASES[request.param]
    pts = make()
    H = O.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2)
    G = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("f32",))
    mp_module.setenv("H2_KRON", "0")
    G0 = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("f32",))
    mp_module.delenv("H2_KRON")
    yield request.param, pts.shape[0], H, G, G0
    G.close()
    G0.close()


def _apply(G, X, Y0, alpha):
    torch = require_cuda()
    Yd = torch.from_numpy(Y0).cuda()
    G.matmul(torch.from_numpy(X).cuda(), Yd, alpha=alpha, dtype="f32")
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


@pytest.mark.parametrize("m", [4, 8, 12, 32, 36, 64, 96])
def test_kron_down_matches_oracle_and_the_cuda_core_pass(pair, m):
    name, n, H, G, G0 = pair
    X, Y0 = gaussian_rhs(n, m, 60 + m), gaussian_rhs(n, m, 70 + m)
    ref = O.h2mm(H, 1.25, X, Y0)
    got = _apply(G, X, Y0, 1.25)
    plain = _apply(G0, X, Y0, 1.25)
    assert rel_fro(got, ref) <= 1e-5, (name, m)
    assert rel_fro(plain, ref) <= 1e-5, (name, m)
    assert rel_fro(got, plain) <= 5e-6, (name, m)


def test_kron_down_repeats_bit_for_bit(pair):
    name, n, H, G, G0 = pair
    X = gaussian_rhs(n, 16, 3)
    a = _apply(G, X, np.zeros_like(X), 1.0)
    b = _apply(G, X, np.zeros_like(X), 1.0)
    assert np.array_equal(a, b), name


@pytest.mark.parametrize("m", [3, 16, 40])
def test_kron_fp64_passes(P, pair, m):
    """The FP64 product's one-launch transfer passes take the Kronecker factors
    too (against H2_KRON=0 and the oracle)."""
    torch = require_cuda()
    name, n, H, G, G0 = pair
    X, Y0 = gaussian_rhs(n, m, 80 + m), gaussian_rhs(n, m, 90 + m)
    ref = O.h2mm(H, -0.5, X, Y0)
    for Gx in (G, G0):
        Yd = torch.from_numpy(Y0).cuda()
        Gx.matmul(torch.from_numpy(X).cuda(), Yd, alpha=-0.5, dtype="f64")
        torch.cuda.synchronize()
        assert rel_fro(Yd.cpu().numpy(), ref) <= 1e-12, (name, m)
