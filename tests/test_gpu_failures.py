"""Failure paths reported as statuses, each provoked from the host (no GPU
fault, no wait that cannot end):

* a NaN in one right-hand side: block CG reports a breakdown (a non-finite
  <p, Ap>, Sec. 5.1 Alg. "block CG"), for the paper's column-wise form, the
  Gram form and the mixed-precision refinement;
* the library's device-allocation cap: h2_build reports H2_E_OOM and leaves
  no device memory behind;
* the device-side flag waits of the FP64 downward pass told to give up at
  once: the next call reports H2_E_TIMEOUT, and the call after that is
  correct again."""
import numpy as np
import pytest

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
def case(P):
    pts = sphere_points(4096, 0)
    G = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    return pts, G


@pytest.mark.parametrize("variant,dtype,refine", [("columnwise", "f64", 0), ("gram", "f64", 0),
                                                   ("columnwise", "f32", 2), ("columnwise", "f32", 1)])
def test_nan_in_rhs_reports_breakdown(P, case, variant, dtype, refine):
    torch = require_cuda()
    _, G = case
    B = gaussian_rhs(4096, 4, 1)
    B[17, 2] = np.nan
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    res = G.block_cg(Bd, Xd, tol=1e-8, max_iter=300, dtype=dtype, variant=variant, refine=refine,
                     inner_tol=0.1 if refine == 2 else 1e-4)
    assert res.status == P.H2_E_BREAKDOWN, res
    # the matrix is still usable: a clean solve of the other columns converges
    Bc = torch.from_numpy(np.delete(B, 2, axis=1)).cuda()
    Xc = torch.zeros_like(Bc)
    ok = G.block_cg(Bc, Xc, tol=1e-8, max_iter=5000, dtype="f64", variant=variant)
    assert ok.status == 0, ok


def test_alloc_cap_reports_oom_and_leaks_nothing(P, case):
    torch = require_cuda()
    pts, _ = case
    torch.cuda.synchronize()
    held = P.h2_alloc_bytes()
    free0 = torch.cuda.mem_get_info()[0]
    P.h2_set_alloc_limit(held + (1 << 20))  # 1 MiB more than the live matrices hold
    try:
        with pytest.raises(P.H2Error) as e:
            P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
        assert e.value.code == P.H2_E_OOM
        assert "cap" in str(e.value)
        assert P.h2_alloc_bytes() == held
    finally:
        P.h2_set_alloc_limit(0)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (4 << 20)
    with pytest.raises(P.H2Error) as e:
        P.h2_set_alloc_limit(-1)
    assert e.value.code == P.H2_E_BADARG
    # without the cap the same build succeeds and is counted while it lives
    G2 = P.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    assert P.h2_alloc_bytes() > held
    G2.close()
    assert P.h2_alloc_bytes() == held


def test_flag_wait_gives_up_then_reports_timeout(P, case):
    torch = require_cuda()
    pts, G = case
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    X = gaussian_rhs(4096, 6, 3)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.zeros_like(Xd)
    P.h2_set_wait_limit(-1)
    try:
        G.matmul(Xd, Yd, dtype="f64")  # its downward pass gives up on every flag it must wait for
        torch.cuda.synchronize()
    finally:
        P.h2_set_wait_limit(0)
    with pytest.raises(P.H2Error) as e:
        G.matmul(Xd, Yd, dtype="f64")
    assert e.value.code == P.H2_E_TIMEOUT
    # the flag was cleared by the report; the next product is correct
    Yd.zero_()
    G.matmul(Xd, Yd, dtype="f64")
    torch.cuda.synchronize()
    assert rel_fro(Yd.cpu().numpy(), O.h2mm(H, 1.0, X)) <= 1e-12
