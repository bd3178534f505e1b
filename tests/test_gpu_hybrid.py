"""The hybrid upward pass of the FP32 and BF16 tensor-core products: the CUDA-core
subtree pass stops at its cut, and the clusters above the cut (x̂_t =
E_s0ᵀ x̂_s0 + E_s1ᵀ x̂_s1, Alg. "forward/backward") are transfer items of the
coupling launch, waiting for their sons' ready flags, with the coupling items
that read them waiting in turn.  Checked against the FP64 oracle and the
same product without it (H2_TC_HYBRID=0), for shapes where the subtree passes
apply (k a multiple of 8: q = 2 and 4; columns a multiple of 4 per 64-column
chunk), one, two and three chunks, leaves on several levels, cut targets
moved by the tuner, and repeated products (bit for bit).  The BF16 product's
transfer items take E_sᵀ as a BF16 tile and its BF16 remainder, so they add
next to nothing to the BF16 coupling's error: against the oracle within the
BF16 tolerance, against the BF16 product without them within 2e-4."""
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
    "sphere20000_q4": (lambda: sphere_points(20000, 31), 4, 64),
    "sphere6000_q2": (lambda: sphere_points(6000, 32), 2, 64),
    "ellipsoid_leaf24_q4": (lambda: ellipsoid_points(5000, (0.5, 1.8, 1.1), 33), 4, 24),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(P, request, mp_module):
    make, q, leaf = CASES[request.param]
    pts = make()
    H = O.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2)
    mp_module.setenv("H2_TC_HYBRID", "1")
    G = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("f32",))
    mp_module.setenv("H2_TC_HYBRID", "0")
    G0 = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("f32",))
    mp_module.delenv("H2_TC_HYBRID")
    yield request.param, pts.shape[0], H, G, G0
    G.close()
    G0.close()


def _apply(G, X, Y0, alpha, dtype="f32"):
    torch = require_cuda()
    Yd = torch.from_numpy(Y0).cuda()
    G.matmul(torch.from_numpy(X).cuda(), Yd, alpha=alpha, dtype=dtype)
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


@pytest.mark.parametrize("m", [4, 8, 32, 64, 72, 132])
def test_hybrid_matches_oracle_and_the_plain_chain(pair, m):
    name, n, H, G, G0 = pair
    X, Y0 = gaussian_rhs(n, m, 40 + m), gaussian_rhs(n, m, 50 + m)
    ref = O.h2mm(H, -0.75, X, Y0)
    got = _apply(G, X, Y0, -0.75)
    plain = _apply(G0, X, Y0, -0.75)
    assert rel_fro(got, ref) <= 1e-5, (name, m)
    assert rel_fro(plain, ref) <= 1e-5, (name, m)
    assert rel_fro(got, plain) <= 5e-6, (name, m)


def test_hybrid_repeats_bit_for_bit(pair):
    name, n, H, G, G0 = pair
    X = gaussian_rhs(n, 32, 7)
    a = _apply(G, X, np.zeros_like(X), 1.0)
    b = _apply(G, X, np.zeros_like(X), 1.0)
    assert np.array_equal(a, b), name


def test_hybrid_follows_the_tuned_cut(P, pair):
    name, n, H, G, G0 = pair
    r = P.h2_autotune_ex(G.handle, 32, "f32")
    assert 5 in [c["path"] for c in r["candidates"]], r
    X, Y0 = gaussian_rhs(n, 32, 9), gaussian_rhs(n, 32, 10)
    assert rel_fro(_apply(G, X, Y0, 0.5), O.h2mm(H, 0.5, X, Y0)) <= 1e-5, (name, r["path"], r["up_target"])


@pytest.fixture(scope="module", params=sorted(CASES))
def pair16(P, request, mp_module):
    make, q, leaf = CASES[request.param]
    pts = make()
    H = O.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2)
    mp_module.setenv("H2_TC_HYBRID", "1")
    G = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("bf16",))
    mp_module.setenv("H2_TC_HYBRID", "0")
    G0 = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=1e-2, precisions=("bf16",))
    mp_module.delenv("H2_TC_HYBRID")
    yield request.param, pts.shape[0], H, G, G0
    G.close()
    G0.close()


@pytest.mark.parametrize("m", [4, 8, 32, 64, 72])
def test_bf16_hybrid_matches_oracle_and_the_plain_chain(pair16, m):
    name, n, H, G, G0 = pair16
    X, Y0 = gaussian_rhs(n, m, 60 + m), gaussian_rhs(n, m, 70 + m)
    ref = O.h2mm(H, 1.25, X, Y0)
    got = _apply(G, X, Y0, 1.25, "bf16")
    plain = _apply(G0, X, Y0, 1.25, "bf16")
    assert rel_fro(got, ref) <= 3e-3, (name, m)
    assert rel_fro(got, plain) <= 2e-4, (name, m)


def test_bf16_hybrid_repeats_bit_for_bit_and_is_tuned(P, pair16):
    name, n, H, G, G0 = pair16
    X = gaussian_rhs(n, 32, 8)
    a = _apply(G, X, np.zeros_like(X), 1.0, "bf16")
    b = _apply(G, X, np.zeros_like(X), 1.0, "bf16")
    assert np.array_equal(a, b), name
    r = P.h2_autotune_ex(G.handle, 32, "bf16")
    assert 5 in [c["path"] for c in r["candidates"]], r
    assert rel_fro(_apply(G, X, np.zeros_like(X), 1.0, "bf16"), O.h2mm(H, 1.0, X, np.zeros_like(X))) <= 3e-3
