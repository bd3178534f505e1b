"""Batches of independent systems (uneven n, m and q) through the C ABI: one
graph launch per batched product equals the per-system products; batched
mixed-precision block CG reaches the FP64 tolerance for every system; the
autotuner keeps products correct."""
import numpy as np
import pytest
import scipy.linalg as sla

from _helpers import rel_fro, require_cuda
from oracle import h2_oracle as O
from workloads import batch_specs, ellipsoid_points, gaussian_rhs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    specs = batch_specs(count=6, seed=3, n_lo=800, n_hi=4000)
    mats, pts = [], []
    for sp in specs:
        x = ellipsoid_points(sp["n"], sp["axes"], sp["point_seed"])
        pts.append(x)
        mats.append(P.H2Matrix(x, q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32", "bf16")))
    return P, specs, pts, mats


def test_batched_product_equals_single_products(batch):
    torch = require_cuda()
    P, specs, pts, mats = batch
    B = P.H2Batch(mats)
    # FP32: the batch runs every system's product in two multi-system launches; the
    # single products may take other (equally accurate) paths, so they agree to a few
    # FP32 roundings
    for dtype, tol in (("f64", 1e-12), ("f32", 3e-6)):
        Xs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], 10 + i)).cuda() for i, sp in enumerate(specs)]
        Ys = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], 20 + i)).cuda() for i, sp in enumerate(specs)]
        ref = [y.clone() for y in Ys]
        for mm, x, y in zip(mats, Xs, ref):
            mm.matmul(x, y, alpha=0.5, dtype=dtype)
        B.matmul(Xs, Ys, alpha=0.5, dtype=dtype)  # capture + launch
        torch.cuda.synchronize()
        for y, r in zip(Ys, ref):
            assert rel_fro(y.cpu().numpy(), r.cpu().numpy()) <= tol
        # replay the cached graph on new contents of the same buffers
        for i, x in enumerate(Xs):
            x.copy_(torch.from_numpy(gaussian_rhs(x.shape[0], x.shape[1], 30 + i)))
        ref = [y.clone() for y in Ys]
        for mm, x, y in zip(mats, Xs, ref):
            mm.matmul(x, y, alpha=0.5, dtype=dtype)
        B.matmul(Xs, Ys, alpha=0.5, dtype=dtype)
        torch.cuda.synchronize()
        for y, r in zip(Ys, ref):
            assert rel_fro(y.cpu().numpy(), r.cpu().numpy()) <= tol
    B.close()


def test_batched_block_cg(batch):
    torch = require_cuda()
    P, specs, pts, mats = batch
    B = P.H2Batch(mats)
    Bs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], 40 + i)).cuda() for i, sp in enumerate(specs)]
    Xs = [torch.zeros_like(b) for b in Bs]
    res = B.block_cg(Bs, Xs, tol=1e-8, max_iter=20000, dtype="f32", inner_tol=0.1, check_every=4)
    for sp, x, b, r, p in zip(specs, Xs, Bs, res, pts):
        assert r.status == 0, (sp, r)
        assert r.rel_residual.max() <= 1e-8  # the solver decides on this FP64 residual
        H = O.H2Matrix(p, q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2)
        A = O.dense_expand(H)
        bn = b.cpu().numpy()
        Xc = np.linalg.solve(A, bn)
        assert rel_fro(x.cpu().numpy(), Xc) <= 1e-6
    B.close()


def test_autotune_keeps_products_correct(batch):
    torch = require_cuda()
    P, specs, pts, mats = batch
    sp, mm = specs[0], mats[0]
    t_tc, t_simt = P.h2_autotune(mm.handle, sp["m"])
    assert t_simt > 0 and (t_tc > 0 or t_tc == -1.0)
    H = O.H2Matrix(pts[0], q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2)
    X = gaussian_rhs(sp["n"], sp["m"], 1)
    want = O.h2mm(H, 1.0, X)
    Yd = torch.zeros(sp["n"], sp["m"], dtype=torch.float64, device="cuda")
    mm.matmul(torch.from_numpy(X).cuda(), Yd, dtype="f32")
    assert rel_fro(Yd.cpu().numpy(), want) <= 1e-5


def test_batched_block_cg_gram(batch):
    """The Gram-matrix variant inside the batched graph: every system reaches
    the FP64 tolerance with the FP32 product and reliable updates."""
    torch = require_cuda()
    P, specs, pts, mats = batch
    B = P.H2Batch(mats)
    Bs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], 50 + i)).cuda() for i, sp in enumerate(specs)]
    Xs = [torch.zeros_like(b) for b in Bs]
    res = B.block_cg(Bs, Xs, tol=1e-8, max_iter=20000, dtype="f32", inner_tol=0.1, check_every=4, variant="gram")
    for sp, x, b, r, p in zip(specs, Xs, Bs, res, pts):
        assert r.status == 0, (sp, r)
        assert r.rel_residual.max() <= 1e-8  # the solver decides on this FP64 residual
        H = O.H2Matrix(p, q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2)
        A = O.dense_expand(H)
        Xc = np.linalg.solve(A, b.cpu().numpy())
        assert rel_fro(x.cpu().numpy(), Xc) <= 1e-6
    B.close()


def test_multi_system_launches_match_single_products_bit_for_bit():
    """With the tensor-core transfer passes on every matrix, a single product runs
    the same items (upward+coupling, downward+leaf work lists) as the batch's two
    multi-system launches, each with the same terms in the same order: the results
    agree bit for bit, and with the FP64 oracle to the FP32 tolerance.  Column
    counts 1..64 across the systems (R from 16 to 128 in one launch), q = 3 and 4."""
    torch = require_cuda()
    import os
    import paper_2509_17257_gb300 as P
    specs = batch_specs(count=7, seed=11, n_lo=700, n_hi=5000)
    specs[0]["m"], specs[1]["m"], specs[2]["m"] = 1, 64, 33
    os.environ["H2_TC_TRANSFER"] = "1"
    try:
        pts = [ellipsoid_points(sp["n"], sp["axes"], sp["point_seed"]) for sp in specs]
        mats = [P.H2Matrix(x, q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",))
                for x, sp in zip(pts, specs)]
    finally:
        del os.environ["H2_TC_TRANSFER"]
    B = P.H2Batch(mats)
    Xs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], 60 + i)).cuda() for i, sp in enumerate(specs)]
    Y0 = [gaussian_rhs(sp["n"], sp["m"], 70 + i) for i, sp in enumerate(specs)]
    for rep in range(2):  # capture, then replay
        Ys = [torch.from_numpy(y).cuda() for y in Y0]
        ref = [torch.from_numpy(y).cuda() for y in Y0]
        B.matmul(Xs, Ys, alpha=-0.25, dtype="f32")
        for mm, x, y in zip(mats, Xs, ref):
            mm.matmul(x, y, alpha=-0.25, dtype="f32")
        torch.cuda.synchronize()
        for i, (y, r) in enumerate(zip(Ys, ref)):
            assert torch.equal(y, r), (rep, i)
    for sp, p, x, y, y0 in zip(specs, pts, Xs, Ys, Y0):
        H = O.H2Matrix(p, q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2)
        assert rel_fro(y.cpu().numpy(), O.h2mm(H, -0.25, x.cpu().numpy(), y0)) <= 1e-5, sp
    B.close()
    for mm in mats:
        mm.close()

