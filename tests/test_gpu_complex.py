"""The complex product (K = C, Sec. 2: the Helmholtz kernel, regularised at
r = 0 as exp(iκr)/(4π sqrt(r² + δ²))) against the oracle's complex product,
element by element, through h2_matmul_complex:

* FP64 within 1e-12 and FP32 within 1e-5 (relative Frobenius), complex α,
  Y accumulated, on device tensors and on host arrays (the staged path);
* column counts that fill no tile exactly (1, 5, 17, 33, 70), q = 2, 3, 4,
  a ragged leaf size and an odd n;
* the precision workload's size (n = 65536, q = 4, m = 32) on sampled rows;
* the FP32 product on the split-TF32 tensor cores (S_im and G_im terms whose
  activation columns the epilogue swaps and negates) and on the CUDA cores;
* the entry points that compute over R refuse a complex matrix, and the
  complex product refuses a real one, BF16 and a transposed request."""
import numpy as np
import pytest

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu

KAPPA, DELTA, SIGMA = 1.0, 0.05, 1e-2
TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


def _cx(n, m, seed):
    return gaussian_rhs(n, m, seed) + 1j * gaussian_rhs(n, m, seed + 500)


_CASES = {}


def _case(P, n, q, leaf):
    key = (n, q, leaf)
    if key not in _CASES:
        pts = sphere_points(n, 3)
        G = P.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, sigma=SIGMA, precisions=("f32",), kernel="helmholtz",
                       kappa=KAPPA, delta=DELTA)
        H = O.H2Matrix(pts, q=q, leaf_size=leaf, eta=2.0, kernel=O.helmholtz_kernel(KAPPA, DELTA), sigma=SIGMA)
        _CASES[key] = (G, H)
    return _CASES[key]


@pytest.mark.parametrize("n,q,leaf", [(4096, 3, 64), (3001, 4, 64), (2500, 2, 17)])
@pytest.mark.parametrize("m", [1, 5, 17, 33, 70])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_complex_product_matches_oracle(P, n, q, leaf, m, dtype):
    torch = require_cuda()
    G, H = _case(P, n, q, leaf)
    X, Y0 = _cx(n, m, 10 + m), _cx(n, m, 20 + m)
    alpha = 0.7 - 1.3j
    ref = O.h2mm(H, alpha, X, Y0)
    Yd = torch.from_numpy(Y0.copy()).cuda()
    G.matmul_complex(torch.from_numpy(X).cuda(), Yd, alpha=alpha, dtype=dtype)
    torch.cuda.synchronize()
    assert rel_fro(Yd.cpu().numpy(), ref) <= TOL[dtype], (n, q, m, dtype)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_complex_product_on_host_arrays(P, dtype):
    require_cuda()
    G, H = _case(P, 4096, 3, 64)
    X, Y0 = _cx(4096, 8, 31), _cx(4096, 8, 32)
    ref = O.h2mm(H, -0.25 + 2j, X, Y0)
    Y = Y0.copy()
    G.matmul_complex(X, Y, alpha=-0.25 + 2j, dtype=dtype)
    assert rel_fro(Y, ref) <= TOL[dtype]
    # a strided view (leading dimension larger than m) is read and written in place
    Xw, Yw = np.zeros((4096, 11), complex), np.zeros((4096, 11), complex)
    Xw[:, 2:10], Yw[:, 2:10] = X, Y0
    G.matmul_complex(Xw[:, 2:10], Yw[:, 2:10], alpha=-0.25 + 2j, dtype=dtype)
    assert rel_fro(Yw[:, 2:10], ref) <= TOL[dtype]
    assert not Yw[:, :2].any() and not Yw[:, 10:].any()


def test_complex_product_full_size_sampled_rows(P):
    torch = require_cuda()
    n, m = 65536, 32
    pts = sphere_points(n, 0)
    G = P.H2Matrix(pts, q=4, leaf_size=64, eta=2.0, sigma=SIGMA, precisions=("f32",), kernel="helmholtz",
                   kappa=KAPPA, delta=DELTA)
    R = O.H2Rows(pts, q=4, leaf_size=64, eta=2.0, sigma=SIGMA, kernel=O.helmholtz_kernel(KAPPA, DELTA))
    X = _cx(n, m, 1)
    rows = np.random.default_rng(7).choice(n, 48, replace=False)
    ref = R.rows(1.0 - 0.5j, X, rows)
    Xd = torch.from_numpy(X).cuda()
    for dtype in ("f64", "f32"):
        Yd = torch.zeros_like(Xd)
        G.matmul_complex(Xd, Yd, alpha=1.0 - 0.5j, dtype=dtype)
        torch.cuda.synchronize()
        assert rel_fro(Yd.cpu().numpy()[rows], ref) <= TOL[dtype], dtype
    G.close()


def test_complex_and_real_entry_points_refuse_each_other(P):
    torch = require_cuda()
    G, _ = _case(P, 4096, 3, 64)
    Xr = torch.zeros(4096, 2, dtype=torch.float64, device="cuda")
    for call in (lambda: G.matmul(Xr, Xr.clone()), lambda: G.matmul_transposed(Xr, Xr.clone()),
                 lambda: P.h2_matmul_noalloc(G.handle, 1.0, Xr, Xr.clone()),
                 lambda: G.block_cg(Xr, Xr.clone()), lambda: P.h2_coupling_get(G.handle),
                 lambda: P.h2_autotune_ex(G.handle, 8)):
        with pytest.raises(P.H2Error) as e:
            call()
        assert e.value.code == P.H2_E_UNSUPPORTED and "complex" in str(e.value)
    Xc = torch.zeros(4096, 2, dtype=torch.complex128, device="cuda")
    with pytest.raises(P.H2Error) as e:
        G.matmul_complex(Xc, Xc.clone(), dtype="bf16")
    assert e.value.code == P.H2_E_UNSUPPORTED
    real = P.H2Matrix(sphere_points(2000, 1), q=3, precisions=("f32",))
    with pytest.raises(P.H2Error) as e:
        real.matmul_complex(torch.zeros(2000, 2, dtype=torch.complex128, device="cuda"),
                            torch.zeros(2000, 2, dtype=torch.complex128, device="cuda"))
    assert e.value.code == P.H2_E_UNSUPPORTED and "real kernel" in str(e.value)
    real.close()
    with pytest.raises(P.H2Error) as e:
        P.H2Matrix(sphere_points(2000, 1), q=3, precisions=("bf16",), kernel="helmholtz")
    assert e.value.code == P.H2_E_UNSUPPORTED


def test_complex_product_repeats_bit_for_bit(P):
    torch = require_cuda()
    G, _ = _case(P, 4096, 3, 64)
    Xd = torch.from_numpy(_cx(4096, 12, 5)).cuda()
    outs = []
    for _ in range(2):
        Yd = torch.zeros_like(Xd)
        G.matmul_complex(Xd, Yd, alpha=1.0, dtype="f32")
        outs.append(Yd.cpu())
    assert torch.equal(outs[0], outs[1])


def test_complex_product_on_the_cuda_cores_too(P, monkeypatch):
    """The FP32 complex product takes split-TF32 tensor cores where their tiles
    were built; with H2_FORCE_SIMT=1 at build it runs on the CUDA cores.  Both
    against the oracle, and against each other."""
    torch = require_cuda()
    _, H = _case(P, 4096, 3, 64)
    pts = sphere_points(4096, 3)
    monkeypatch.setenv("H2_FORCE_SIMT", "1")
    Gs = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=SIGMA, precisions=("f32",), kernel="helmholtz",
                    kappa=KAPPA, delta=DELTA)
    monkeypatch.delenv("H2_FORCE_SIMT")
    Gt, _ = _case(P, 4096, 3, 64)
    X, Y0 = _cx(4096, 20, 61), _cx(4096, 20, 62)
    ref = O.h2mm(H, 0.3 + 0.9j, X, Y0)
    outs = []
    for G in (Gs, Gt):
        Yd = torch.from_numpy(Y0.copy()).cuda()
        G.matmul_complex(torch.from_numpy(X).cuda(), Yd, alpha=0.3 + 0.9j, dtype="f32")
        torch.cuda.synchronize()
        outs.append(Yd.cpu().numpy())
        assert rel_fro(outs[-1], ref) <= TOL["f32"]
    assert rel_fro(outs[0], outs[1]) <= 5e-6
    Gs.close()
