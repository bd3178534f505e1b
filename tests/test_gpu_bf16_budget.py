"""The BF16 product's error against the FP64 oracle, predicted by the
oracle's BF16 error budget (``h2mm_bf16``: operands rounded to bfloat16,
FP32 accumulation) within a factor of 2, at n = 4096 and n = 65536.

The tensor-core product keeps in BF16 exactly what its matrices store in
BF16: the coupling matrices S_b, the nearfield blocks G_b and the leaf bases
of the backward transformation; X and the coefficient blocks enter its MMAs
as BF16 pairs (high and low parts, 16 significant bits) and the transfer
passes run in FP32.  The budget with those three operands rounded is the
prediction; the budget with every operand rounded (the plain reading of
"BF16 operands") is an upper estimate and must not be exceeded by much."""
import numpy as np
import pytest

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu

STORED_BF16 = ("S", "G", "Vb")


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


@pytest.mark.parametrize("n,q,m", [(4096, 3, 8), (4096, 4, 32), (65536, 4, 32)])
def test_bf16_error_within_2x_of_the_budget(P, n, q, m):
    torch = require_cuda()
    pts = sphere_points(n, 0)
    H = O.H2Matrix(pts, q=q, leaf_size=64, eta=2.0, sigma=1e-2)
    G = P.H2Matrix(pts, q=q, leaf_size=64, eta=2.0, sigma=1e-2, precisions=("bf16",))
    X = gaussian_rhs(n, m, 1)
    exact = O.h2mm(H, 1.0, X)
    Yd = torch.zeros(n, m, dtype=torch.float64, device="cuda")
    G.matmul(torch.from_numpy(X).cuda(), Yd, dtype="bf16")
    torch.cuda.synchronize()
    err = rel_fro(Yd.cpu().numpy(), exact)
    predicted = rel_fro(O.h2mm_bf16(H, 1.0, X, rounded=STORED_BF16), exact)
    upper = rel_fro(O.h2mm_bf16(H, 1.0, X), exact)
    G.close()
    print(f"n={n} q={q} m={m}: GPU {err:.3e}, budget {predicted:.3e}, all operands {upper:.3e}")
    assert predicted / 2 <= err <= 2 * predicted, (err, predicted)
    assert err <= 2 * upper
    assert err <= 3e-3
