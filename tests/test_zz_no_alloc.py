"""h2_matmul_noalloc: the product for callers that cannot allocate device
memory at call time (a process whose GPU memory belongs to another
framework's allocator under a fixed budget, or a hot path that cannot take
cudaMalloc's implicit synchronisation).  It must give the same result as
h2_matmul, call after call, using only the library's fixed scratch array.

This file is collected last on purpose (tests/test_zz_*), so a run that stops
at the first failure has already run every other test."""
import numpy as np
import pytest

from _helpers import rel_fro, require_cuda
from workloads import gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def setup():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    G = P.H2Matrix(sphere_points(4096, 0), q=3, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
    return P, G


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_h2_matmul_on_consecutive_calls(setup, dtype):
    torch = require_cuda()
    P, G = setup
    for call in range(2):  # the second call reuses the scratch the first one left behind
        m = 8 if call == 0 else 5
        X = torch.from_numpy(gaussian_rhs(4096, m, 40 + call)).cuda()
        Y0 = torch.from_numpy(gaussian_rhs(4096, m, 50 + call)).cuda()
        Y_ref = Y0.clone()
        Y_new = Y0.clone()
        P.h2_matmul(G.handle, -0.5, X, Y_ref, dtype=dtype)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        P.h2_matmul_noalloc(G.handle, -0.5, X, Y_new, dtype=dtype)
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the module that holds the scratch array
            assert torch.cuda.mem_get_info()[0] == free0, "the product allocated device memory"
        assert rel_fro(Y_new.cpu().numpy(), Y_ref.cpu().numpy()) <= TOL[dtype], (dtype, call)


def test_noalloc_rejects_what_it_cannot_do(setup):
    torch = require_cuda()
    P, G = setup
    too_many_cols = 4096  # n·m·8 alone is 128 MiB > the 32 MiB scratch
    X = torch.zeros(4096, too_many_cols, dtype=torch.float64, device="cuda")
    with pytest.raises(P.H2Error) as e:
        P.h2_matmul_noalloc(G.handle, 1.0, X, X.clone())
    assert e.value.code == P.H2_E_UNSUPPORTED and "scratch" in str(e.value)
    Xh = np.zeros((4096, 2))
    with pytest.raises(P.H2Error) as e:
        P.h2_matmul_noalloc(G.handle, 1.0, Xh, Xh.copy())
    assert e.value.code == P.H2_E_BADARG
    Xd = torch.zeros(4096, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.H2Error) as e:
        P.h2_matmul_noalloc(G.handle, 1.0, Xd, Xd.clone(), dtype="bf16")
    assert e.value.code == P.H2_E_UNSUPPORTED
    # more than 2^20 columns is refused before any size arithmetic (a huge m
    # could otherwise wrap the scratch size); the buffers are never touched
    big = (1 << 20) + 1
    L = P.lib()
    assert L.h2_matmul_noalloc(G.handle, 1.0, Xd.data_ptr(), big, Xd.data_ptr(), big, big, P.H2_F64,
                               None) == P.H2_E_BADARG
