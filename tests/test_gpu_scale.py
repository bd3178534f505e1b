"""The full-size workloads through the C ABI, against the oracle on sampled
outputs (H2Rows assembles single rows of the product from the definition of
the H² matrix) and, where the oracle cannot follow, against properties that
hold at any size (the solver's FP64 true residual).

* differentiation workload: n = 262144 sphere, q = 4, m = 16 — products in
  FP64/FP32/BF16, coupling gradients for sampled blocks; the system is
  indefinite (a Lanczos certificate), and the solvers say so;
* scale workload: n = 1048576 sphere, q = 4, m = 64 — FP64 and FP32 products,
  the mixed-precision solve reports its outcome;
* batch workload: 64 ellipsoid systems, n log-uniform in [2048, 32768],
  m in {1..64}, q in {3, 4} — the batched FP32 product and the batched mixed
  solve.
"""
import numpy as np
import pytest

from _helpers import require_cuda
from oracle import h2_oracle as O
from workloads import CONFIGS, batch_specs, ellipsoid_points, gaussian_rhs, sphere_points

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-3}


@pytest.fixture(scope="module")
def P():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


def _sample_rows(R, count, seed):
    """`count` random rows plus every row of one leaf (a whole leaf block)."""
    rng = np.random.default_rng(seed)
    rows = list(rng.choice(R.n, count, replace=False))
    leaf = R.by_id[int(R.leaf_of[rows[0]])]
    return np.array(sorted(set(rows) | set(int(i) for i in leaf.idx)))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def diff_case(P):
    cfg = CONFIGS["diff_n262144"]
    pts = sphere_points(cfg["n"], cfg["point_seed"])
    R = O.H2Rows(pts, q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"], sigma=cfg["sigma"])
    G = P.H2Matrix(pts, q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"], sigma=cfg["sigma"],
                   precisions=("f32", "bf16"))
    return cfg, R, G


def test_diff_workload_products(diff_case):
    torch = require_cuda()
    cfg, R, G = diff_case
    n, m = cfg["n"], cfg["m"]
    X = gaussian_rhs(n, m, cfg["rhs_seed"])
    Y0 = gaussian_rhs(n, m, 99)
    rows = _sample_rows(R, 48, 1)
    want = Y0[rows] + R.rows(0.5, X, rows)
    for dtype in ("f64", "f32", "bf16"):
        Yd = torch.from_numpy(Y0).cuda()
        G.matmul(torch.from_numpy(X).cuda(), Yd, alpha=0.5, dtype=dtype)
        got = Yd.cpu().numpy()[rows]
        # the error is measured on the product term, Y0 only checks the += semantics
        assert _rel(got - Y0[rows], want - Y0[rows]) <= TOL[dtype], dtype


def test_diff_workload_coupling_gradients(diff_case, P):
    torch = require_cuda()
    cfg, R, G = diff_case
    n, m = cfg["n"], cfg["m"]
    L, X = gaussian_rhs(n, m, 11), gaussian_rhs(n, m, 12)
    dS, dsig = P.h2_adjoint_grads(G.handle, torch.from_numpy(L).cuda(), torch.from_numpy(X).cuda())
    T = P.h2_tree_build(R.points, leaf_size=cfg["leaf"], eta=cfg["eta"])
    pairs = [(t, int(T["adm_col"][j])) for t in range(T["n_clusters"])
             for j in range(T["adm_rowptr"][t], T["adm_rowptr"][t + 1])]
    assert len(pairs) == R.n_adm == dS.shape[0]
    pick = np.random.default_rng(2).choice(len(pairs), 64, replace=False)
    ref = R.coupling_grads(L, X, [pairs[j] for j in pick])
    dSh = dS.cpu().numpy()
    num = sum(np.sum((dSh[j] - ref[pairs[j]]) ** 2) for j in pick)
    den = sum(np.sum(ref[pairs[j]] ** 2) for j in pick)
    assert np.sqrt(num / den) <= 1e-12
    ref_sig = -float(np.sum(L * X))
    assert abs(dsig - ref_sig) <= 1e-12 * abs(ref_sig)


def test_diff_workload_is_indefinite(diff_case):
    """At n = 2¹⁸ the q = 4 interpolant of the exponential kernel plus σ = 1e-2
    is not positive definite: Lanczos with the FP64 product finds a Ritz value
    below zero.  A Ritz value is the Rayleigh quotient of a vector of the
    Krylov space, so a negative one (by far more than the product's rounding,
    |A|·1e-15 ≈ 3e-11) certifies vᵀ(Â + σI)v < 0 for some v; CG does not apply
    to this system."""
    torch = require_cuda()
    cfg, R, G = diff_case
    n = cfg["n"]
    rng = np.random.default_rng(0)
    steps = 400
    Q = torch.zeros(n, steps + 1, dtype=torch.float64, device="cuda")
    v = torch.from_numpy(rng.standard_normal(n)).cuda()
    Q[:, 0] = v / v.norm()
    al, be = [], []
    for j in range(steps):
        y = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
        G.matmul(Q[:, j:j + 1].contiguous(), y, dtype="f64")
        w = y[:, 0]
        al.append(float(torch.dot(w, Q[:, j])))
        for _ in range(2):  # full reorthogonalisation
            w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        be.append(float(w.norm()))
        Q[:, j + 1] = w / be[-1]
    T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    theta, U = np.linalg.eigh(T)
    assert theta[0] < -1e-3, theta[:4]
    # the Ritz vector itself: its Rayleigh quotient through one more product
    x = (Q[:, :steps] @ torch.from_numpy(U[:, 0]).cuda()).contiguous()
    y2 = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    G.matmul(x[:, None].contiguous(), y2, dtype="f64")
    rq = float(torch.dot(x, y2[:, 0]) / torch.dot(x, x))
    assert rq < -1e-3, rq


def test_diff_workload_solves_fail_honestly(diff_case, P):
    """On the indefinite system every solver ends with a status that says so
    (breakdown or no convergence) — never H2_OK with a residual above tol."""
    torch = require_cuda()
    cfg, R, G = diff_case
    n, m = cfg["n"], cfg["m"]
    rhs = 2.0 * (gaussian_rhs(n, m, 21) - gaussian_rhs(n, m, 22))
    for kw in (dict(dtype="f64", variant="gram", transposed=True, max_iter=400),
               dict(dtype="f32", refine=2, inner_tol=0.1, variant="gram", precond="block_jacobi", max_iter=2000)):
        X = torch.zeros(n, m, dtype=torch.float64, device="cuda")
        res = G.block_cg(torch.from_numpy(rhs).cuda(), X, tol=1e-8, check_every=4, **kw)
        if res.status == 0:
            assert res.rel_residual.max() <= 1e-8 * 1.05
        else:
            assert res.status in (P.H2_E_BREAKDOWN, P.H2_E_NOCONVERGE), res


@pytest.fixture(scope="module")
def scale_case(P):
    cfg = CONFIGS["scale_n1048576"]
    pts = sphere_points(cfg["n"], cfg["point_seed"])
    G = P.H2Matrix(pts, q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"], sigma=cfg["sigma"],
                   precisions=("f32",))
    return cfg, pts, G


def test_scale_workload_products(scale_case):
    torch = require_cuda()
    cfg, pts, G = scale_case
    n, m = cfg["n"], cfg["m"]
    R = O.H2Rows(pts, q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"], sigma=cfg["sigma"])
    X = gaussian_rhs(n, m, cfg["rhs_seed"])
    rows = _sample_rows(R, 32, 3)
    want = R.rows(1.0, X, rows)
    Xd = torch.from_numpy(X).cuda()
    for dtype in ("f64", "f32"):
        Yd = torch.zeros(n, m, dtype=torch.float64, device="cuda")
        G.matmul(Xd, Yd, dtype=dtype)
        assert _rel(Yd.cpu().numpy()[rows], want) <= TOL[dtype], dtype


def test_scale_workload_mixed_solve_reports_its_outcome(scale_case, P):
    """n = 2²⁰: the system is indefinite like the n = 2¹⁸ one (more so:
    the interpolation error grows ∝ n while σ stays 1e-2).  The mixed solve
    (preconditioned Gram variant, FP32 tensor-core product, FP64 residuals)
    either reaches the FP64 tolerance or says that it did not."""
    torch = require_cuda()
    cfg, pts, G = scale_case
    n, m = cfg["n"], cfg["m"]
    B = torch.from_numpy(gaussian_rhs(n, m, cfg["rhs_seed"])).cuda()
    X = torch.zeros_like(B)
    res = G.block_cg(B, X, tol=1e-8, max_iter=400, dtype="f32", refine=2, inner_tol=0.1, variant="gram",
                     precond="block_jacobi", check_every=4)
    if res.status == 0:
        assert res.rel_residual.max() <= 1e-8 * 1.05
    else:
        assert res.status in (P.H2_E_BREAKDOWN, P.H2_E_NOCONVERGE), res


@pytest.fixture(scope="module")
def batch_case(P):
    specs = batch_specs(64, 3, 2048, 32768)
    mats, pts = [], []
    for sp in specs:
        x = ellipsoid_points(sp["n"], sp["axes"], sp["point_seed"])
        pts.append(x)
        mats.append(P.H2Matrix(x, q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2, precisions=("f32",)))
    return specs, pts, mats


def test_batch_workload_products(batch_case, P):
    torch = require_cuda()
    specs, pts, mats = batch_case
    Bt = P.H2Batch(mats)
    Xs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], sp["rhs_seed"])).cuda() for sp in specs]
    Ys = [torch.zeros_like(x) for x in Xs]
    Bt.matmul(Xs, Ys, dtype="f32")
    torch.cuda.synchronize()
    for sp, x, y, p in zip(specs, Xs, Ys, pts):
        R = O.H2Rows(p, q=sp["q"], leaf_size=64, eta=2.0, sigma=1e-2)
        rows = _sample_rows(R, 16, sp["index"])
        want = R.rows(1.0, x.cpu().numpy(), rows)
        assert _rel(y.cpu().numpy()[rows], want) <= TOL["f32"], sp
    Bt.close()


def test_batch_workload_mixed_solve(batch_case, P):
    """All 64 systems in one graph per iteration (Gram variant, FP32 product,
    reliable FP64 updates).  Every SPD system reaches 1e-8; interpolation order
    q = 3 loses definiteness as n grows (λ_min(Â) < 0 from n ≈ 16K on the
    sphere), so a q = 3 system with n > 12000 may instead end in breakdown or
    no convergence — never a wrong "ok"."""
    torch = require_cuda()
    specs, pts, mats = batch_case
    Bt = P.H2Batch(mats)
    Bs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], sp["rhs_seed"] + 7)).cuda() for sp in specs]
    Xs = [torch.zeros_like(b) for b in Bs]
    res = Bt.block_cg(Bs, Xs, tol=1e-8, max_iter=3000, dtype="f32", inner_tol=0.1, check_every=4, variant="gram")
    bad = []
    for sp, r in zip(specs, res):
        if r.status == 0:
            assert r.rel_residual.max() <= 1e-8 * 1.05, sp
        else:
            bad.append(sp)
            assert r.status in (P.H2_E_BREAKDOWN, P.H2_E_NOCONVERGE)
            assert sp["q"] == 3 and sp["n"] > 12000, sp
    assert len(bad) <= 12
    Bt.close()
