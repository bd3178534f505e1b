"""GPU parity of the H² product through the C ABI against the FP64 oracle.

Tolerances (relative Frobenius error of Y_out = Y + α A X): FP64 1e-12,
FP32 1e-5.  Sizes span several tiles and ragged tails (m not a multiple of
the 16/32/64-column tiles, leaves of uneven size, trees whose leaves sit on
several levels)."""
import numpy as np
import pytest

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import ellipsoid_points, gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-3}


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


def _pair(P, pts, q, leaf=64, eta=2.0, sigma=1e-2, length=0.5):
    H = O.H2Matrix(pts, q=q, leaf_size=leaf, eta=eta, sigma=sigma, length=length)
    prec = ("f32", "bf16") if q <= 4 else ("f32",)
    G = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=eta, sigma=sigma, length=length, precisions=prec)
    return H, G


def _gpu_apply(G, X, Y0, alpha, dtype, transposed=False):
    torch = require_cuda()
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y0).cuda()
    if transposed:
        G.matmul_transposed(Xd, Yd, alpha=alpha, dtype=dtype)
    else:
        G.matmul(Xd, Yd, alpha=alpha, dtype=dtype)
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


@pytest.fixture(scope="module")
def sphere4096(P):
    return _pair(P, sphere_points(4096, 0), q=3)


def test_counts_match_oracle(sphere4096):
    H, G = sphere4096
    c = H.counts()
    for key in ("n_clusters", "n_leaves", "n_adm", "n_near", "nnz_near", "depth"):
        assert G.info[key] == c[key], key


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m", [1, 3, 8, 17, 40, 64, 65, 130])
def test_matmul_matches_oracle(sphere4096, dtype, m):
    H, G = sphere4096
    X = gaussian_rhs(4096, m, 10 + m)
    Y0 = gaussian_rhs(4096, m, 20 + m)
    alpha = -0.625
    want = O.h2mm(H, alpha, X, Y0)
    got = _gpu_apply(G, X, Y0, alpha, dtype)
    assert rel_fro(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m", [5, 40, 70])
def test_transposed_matches_oracle(sphere4096, dtype, m):
    H, G = sphere4096
    X = gaussian_rhs(4096, m, 3)
    Y0 = gaussian_rhs(4096, m, 4)
    want = O.h2mm(H, 1.5, X, Y0, transposed=True)
    got = _gpu_apply(G, X, Y0, 1.5, dtype, transposed=True)
    assert rel_fro(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_transposed_of_a_nonsymmetric_matrix(P, dtype):
    """After the couplings are replaced by non-symmetric ones (S_(s,t) no longer
    S_(t,s)ᵀ), Aᵀ differs from A; the tensor-core product with Aᵀ (S_bᵀ tiles,
    column-cluster lists) must follow, including the tiles rebuilt by
    h2_coupling_set.  A q = 4 tree so the subtree-owning transfer passes run."""
    torch = require_cuda()
    pts = sphere_points(3000, 11)
    H, G = _pair(P, pts, q=4)
    X = gaussian_rhs(3000, 24, 1)
    Y0 = gaussian_rhs(3000, 24, 2)
    _gpu_apply(G, X, Y0, 1.0, dtype, transposed=True)  # build the Aᵀ tiles before the change
    rng = np.random.default_rng(5)
    S = P.h2_coupling_get(G.handle)  # host copy, list order
    S = np.ascontiguousarray(S * (1.0 + 0.3 * rng.standard_normal(S.shape)))
    P.h2_coupling_set(G.handle, torch.from_numpy(S).cuda())
    T = P.h2_tree_build(pts, leaf_size=64, eta=2.0, q=4)
    order = [(t, int(T["adm_col"][j])) for t in range(T["n_clusters"])
             for j in range(T["adm_rowptr"][t], T["adm_rowptr"][t + 1])]
    O.set_coupling(H, {pair: S[j] for j, pair in enumerate(order)})
    for trans in (False, True):
        want = O.h2mm(H, -0.5, X, Y0, transposed=trans)
        got = _gpu_apply(G, X, Y0, -0.5, dtype, transposed=trans)
        assert rel_fro(got, want) <= TOL[dtype], trans
    assert rel_fro(O.h2mm(H, 1.0, X, transposed=True), O.h2mm(H, 1.0, X)) > 1e-2



def test_host_buffers_and_leading_dimension(P, sphere4096):
    torch = require_cuda()
    H, G = sphere4096
    X = gaussian_rhs(4096, 12, 5)
    Y0 = gaussian_rhs(4096, 12, 6)
    want = O.h2mm(H, 2.0, X[:, 2:9], Y0[:, 1:8])
    # host numpy views with ld = 12 > m = 7
    Yh = Y0.copy()
    G.matmul(X[:, 2:9], Yh[:, 1:8], alpha=2.0)
    assert rel_fro(Yh[:, 1:8], want) <= 1e-12
    assert np.array_equal(Yh[:, 0], Y0[:, 0]) and np.array_equal(Yh[:, 8:], Y0[:, 8:])
    # device views with ld = 12
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y0).cuda()
    G.matmul(Xd[:, 2:9], Yd[:, 1:8], alpha=2.0)
    out = Yd.cpu().numpy()
    assert rel_fro(out[:, 1:8], want) <= 1e-12
    assert np.array_equal(out[:, 0], Y0[:, 0]) and np.array_equal(out[:, 8:], Y0[:, 8:])
    # m = 0 is a no-op
    G.matmul(np.zeros((4096, 0)), np.zeros((4096, 0)))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_pinned_host_buffers_in_place(P, dtype):
    """Pinned host X and Y (device-mapped) are read and updated where they are;
    the result equals the product on device copies, columns outside the views
    untouched.  A q = 4 tree, so the FP32 and BF16 products take the
    subtree-owning transfer passes."""
    torch = require_cuda()
    n = 3000
    pts = sphere_points(n, 8)
    G = P.H2Matrix(pts, q=4, leaf_size=64, eta=2.0, sigma=1e-2, length=0.5, precisions=("f32", "bf16"))
    X = gaussian_rhs(n, 40, 7)
    Y0 = gaussian_rhs(n, 40, 8)
    Xh = torch.from_numpy(X).pin_memory()
    Yh = torch.from_numpy(Y0).pin_memory()
    G.matmul(Xh[:, 3:35], Yh[:, 5:37], alpha=0.5, dtype=dtype)  # ld = 40 > m = 32
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y0).cuda()
    G.matmul(Xd[:, 3:35], Yd[:, 5:37], alpha=0.5, dtype=dtype)
    torch.cuda.synchronize()
    got, ref = Yh.numpy(), Yd.cpu().numpy()
    assert np.array_equal(got, ref)
    assert np.array_equal(got[:, :5], Y0[:, :5]) and np.array_equal(got[:, 37:], Y0[:, 37:])


@pytest.mark.parametrize("case", ["n1", "n64", "n65", "coincident", "planar", "q1", "q2", "q4", "q5",
                                  "ellipsoid_leaf17"])
def test_edge_cases(P, case):
    q, leaf, eta = 3, 64, 2.0
    if case == "n1":
        pts = sphere_points(1, 1)
    elif case == "n64":
        pts = sphere_points(64, 1)
    elif case == "n65":
        pts = sphere_points(65, 1)
    elif case == "coincident":
        pts = np.vstack([np.full((150, 3), 0.3), sphere_points(200, 2)])
    elif case == "planar":
        pts = sphere_points(3000, 3)
        pts[:, 2] = 0.0
    elif case.startswith("q"):
        q = int(case[1])
        pts = sphere_points(2500, 4)
    else:
        pts = ellipsoid_points(3000, (0.6, 1.9, 1.2), 5)
        leaf, eta = 17, 1.0
    H, G = _pair(P, pts, q=q, leaf=leaf, eta=eta)
    n = pts.shape[0]
    X = gaussian_rhs(n, 6, 7)
    Y0 = gaussian_rhs(n, 6, 8)
    for dtype in ("f64", "f32", "bf16"):
        if dtype == "bf16" and q > 4:
            continue
        want = O.h2mm(H, 0.75, X, Y0)
        got = _gpu_apply(G, X, Y0, 0.75, dtype)
        assert rel_fro(got, want) <= TOL[dtype], (case, dtype)
        want_t = O.h2mm(H, 0.75, X, Y0, transposed=True)
        got_t = _gpu_apply(G, X, Y0, 0.75, dtype, transposed=True)
        assert rel_fro(got_t, want_t) <= TOL[dtype], (case, dtype, "T")


def test_fp32_cuda_core_path_matches_oracle(P, monkeypatch):
    """The FP32 product on the CUDA cores (the tensor-core path is disabled with
    H2_FORCE_SIMT=1 at build time) against the oracle."""
    monkeypatch.setenv("H2_FORCE_SIMT", "1")
    pts = sphere_points(3000, 9)
    H, G = _pair(P, pts, q=3)
    X = gaussian_rhs(3000, 20, 1)
    Y0 = gaussian_rhs(3000, 20, 2)
    want = O.h2mm(H, -1.25, X, Y0)
    assert rel_fro(_gpu_apply(G, X, Y0, -1.25, "f32"), want) <= TOL["f32"]


def test_precision_workload_full_size(P):
    """n = 65536 sphere, q = 4, m = 32: the full product against the oracle."""
    pts = sphere_points(65536, 0)
    H, G = _pair(P, pts, q=4)
    X = gaussian_rhs(65536, 32, 1)
    Y0 = np.zeros((65536, 32))
    want = O.h2mm(H, 1.0, X, Y0)
    for dtype in ("f64", "f32", "bf16"):
        got = _gpu_apply(G, X, Y0, 1.0, dtype)
        assert rel_fro(got, want) <= TOL[dtype], dtype


def test_errors(P, sphere4096):
    _, G = sphere4096
    X = np.zeros((4096, 2))
    G32 = P.H2Matrix(sphere_points(1000, 3), q=3, precisions=("f32",))
    with pytest.raises(P.H2Error) as e:
        G32.matmul(np.zeros((1000, 2)), np.zeros((1000, 2)), dtype="bf16")
    assert e.value.code == P.H2_E_UNSUPPORTED
    with pytest.raises(P.H2Error) as e:
        P.h2_build(sphere_points(1000, 3), q=5, precisions=("bf16",))
    assert e.value.code == P.H2_E_UNSUPPORTED
    with pytest.raises(P.H2Error) as e:
        G.matmul(X, X.copy(), dtype=7)
    assert e.value.code == P.H2_E_BADARG
    with pytest.raises(ValueError):
        G.matmul(np.zeros((4095, 2)), np.zeros((4095, 2)))
    with pytest.raises(P.H2Error) as e:
        P.h2_build(np.zeros((0, 3)))
    assert e.value.code == P.H2_E_BADARG
