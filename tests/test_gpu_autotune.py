"""The product autotuner (h2_autotune_ex): it times the product paths (tensor
cores with the CUDA-core or the tensor-core transfer passes, the latter alone
or sharing the coupling and leaf launches, and the CUDA cores), then stage
counts, then the cut targets of the subtree passes, and keeps the fastest.
Every candidate it leaves behind must still compute the same product: the
tuned products are checked against the FP64 oracle, for FP32 and BF16, and
for column counts in different classes."""
import numpy as np
import pytest

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    pts = sphere_points(12000, 31)
    H = O.H2Matrix(pts, q=4, leaf_size=64, eta=2.0, sigma=1e-2)
    G = P.H2Matrix(pts, q=4, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32", "bf16"))
    yield P, H, G
    G.close()


@pytest.mark.parametrize("dtype,m", [("f32", 32), ("f32", 6), ("f32", 64), ("bf16", 24)])
def test_tuned_products_stay_correct(case, dtype, m):
    torch = require_cuda()
    P, H, G = case
    r = P.h2_autotune_ex(G.handle, m, dtype)
    assert r["candidates"], r
    times = [c["ms"] for c in r["candidates"]]
    assert all(t > 0 for t in times)
    assert r["ms"] == min(times)
    chosen = [c for c in r["candidates"] if c["ms"] == r["ms"]][0]
    assert (chosen["path"], chosen["stages"], chosen["up_target"], chosen["down_target"]) == \
        (r["path"], r["stages"], r["up_target"], r["down_target"])
    if dtype == "bf16":
        # the BF16 product: the subtree passes, with or without the hybrid upward pass
        assert 1 in {c["path"] for c in r["candidates"]} <= {1, 5}
    else:
        assert {1, 4} <= {c["path"] for c in r["candidates"]}
    X = gaussian_rhs(12000, m, 7 + m)
    Y0 = gaussian_rhs(12000, m, 8 + m)
    want = O.h2mm(H, 0.5, X, Y0)
    Yd = torch.from_numpy(Y0).cuda()
    G.matmul(torch.from_numpy(X).cuda(), Yd, alpha=0.5, dtype=dtype)
    torch.cuda.synchronize()
    assert rel_fro(Yd.cpu().numpy(), want) <= (1e-5 if dtype == "f32" else 3e-3)


def test_tuning_rejects_bad_arguments(case):
    P, H, G = case
    with pytest.raises(P.H2Error) as e:
        P.h2_autotune_ex(G.handle, 0, "f32")
    assert e.value.code == P.H2_E_BADARG
    with pytest.raises(P.H2Error) as e:
        P.h2_autotune_ex(G.handle, 8, "f64")
    assert e.value.code == P.H2_E_BADARG
