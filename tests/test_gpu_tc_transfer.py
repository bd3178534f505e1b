"""The transfer passes of Alg. "forward/backward" on the tensor cores (the FP32
product's upward and downward pass as work lists of 3xTF32 MMAs in dependency
order, each cluster's result released to the next by a ready flag; the
coupling result enters the downward pass through an identity tile) against
the FP64 oracle, and against the same product with the CUDA-core transfer
passes (H2_TC_TRANSFER=0 at build).  Shapes: q = 4 (k = 64), q = 3 (k = 27)
and q = 2 (k = 8, padded tiles), leaves on several levels, column counts
below, at and above the 64-column chunk, ragged ones included, and A as well
as Aᵀ."""
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


def _apply(G, X, Y0, alpha, transposed=False):
    torch = require_cuda()
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y0).cuda()
    (G.matmul_transposed if transposed else G.matmul)(Xd, Yd, alpha=alpha, dtype="f32")
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


CASES = {
    "sphere3000_q4": (lambda: sphere_points(3000, 21), 4, 64),
    "sphere20000_q4": (lambda: sphere_points(20000, 22), 4, 64),
    "sphere5000_q2": (lambda: sphere_points(5000, 23), 2, 64),
    "sphere4096_q3": (lambda: sphere_points(4096, 26), 3, 64),
    "ellipsoid_leaf17_q4": (lambda: ellipsoid_points(4000, (0.6, 1.9, 1.2), 24), 4, 17),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(P, request, monkeypatch_module):
    make, q, leaf = CASES[request.param]
    pts = make()
    H = O.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2)
    G = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("f32",))
    monkeypatch_module.setenv("H2_TC_TRANSFER", "0")
    G0 = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("f32",))
    monkeypatch_module.delenv("H2_TC_TRANSFER")
    yield request.param, pts.shape[0], H, G, G0
    G.close()
    G0.close()


@pytest.fixture(scope="module")
def monkeypatch_module():
    mp = pytest.MonkeyPatch()
    yield mp
    mp.undo()


@pytest.mark.parametrize("m", [1, 6, 32, 64, 70, 128])
@pytest.mark.parametrize("transposed", [False, True])
def test_tc_transfer_passes_match_oracle(pair, m, transposed):
    name, n, H, G, G0 = pair
    X = gaussian_rhs(n, m, 100 + m)
    Y0 = gaussian_rhs(n, m, 200 + m)
    want = O.h2mm(H, -0.75, X, Y0, transposed=transposed)
    got = _apply(G, X, Y0, -0.75, transposed)
    ref = _apply(G0, X, Y0, -0.75, transposed)
    assert rel_fro(got, want) <= 1e-5, (name, m)
    assert rel_fro(ref, want) <= 1e-5, (name, m)
    # both FP32 products carry FP32 rounding only: they agree far inside the tolerance
    assert rel_fro(got, ref) <= 3e-6, (name, m)


def test_tc_transfer_repeated_products_are_identical(P):
    """Each product clears its ready flags first: the same call twice gives the
    same bits, and a product of other columns in between does not leak."""
    pts = sphere_points(6000, 25)
    G = P.H2Matrix(pts, q=4, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    X = gaussian_rhs(6000, 16, 1)
    Z = gaussian_rhs(6000, 40, 2)
    a = _apply(G, X, np.zeros_like(X), 1.0)
    _apply(G, Z, np.zeros_like(Z), 1.0)
    b = _apply(G, X, np.zeros_like(X), 1.0)
    assert np.array_equal(a, b)
    G.close()
