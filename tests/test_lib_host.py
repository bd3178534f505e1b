"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host topology (cluster tree, block tree, row-cluster lists of Alg.
"prepare_addeval") equals the oracle's, decision for decision."""
import json
import os

import numpy as np
import pytest

from _helpers import header_symbols
from oracle import h2_oracle as O
from workloads import ellipsoid_points, sphere_points


@pytest.fixture(scope="module")
def h2lib():
    import paper_2509_17257_gb300.build as bld
    bld.build()
    import paper_2509_17257_gb300 as P
    return P


def test_library_exports_every_declared_symbol(h2lib):
    L = h2lib.lib()
    names = header_symbols()
    assert "h2_matmul" in names and "h2_block_cg" in names
    for name in names:
        assert hasattr(L, name), name
    assert set(h2lib.EXPORTS) <= set(names)
    assert L.h2_version().startswith(b"h2bcg")


def _oracle_topology(pts, leaf, eta):
    root = O.build_cluster_tree(pts, leaf)
    cl = O.clusters_preorder(root)
    adm, near = O.leaf_blocks(O.build_block_tree(root, root, eta))
    return root, cl, adm, near


def _compare(h2lib, pts, leaf=64, eta=2.0):
    T = h2lib.h2_tree_build(pts, leaf_size=leaf, eta=eta)
    root, cl, adm, near = _oracle_topology(pts, leaf, eta)
    assert np.array_equal(T["perm"], root.idx)
    assert T["n_clusters"] == len(cl)
    for c in cl:
        assert T["offset"][c.id] == c.offset and T["size"][c.id] == c.size
        assert T["level"][c.id] == c.level
        assert T["parent"][c.id] == (c.parent.id if c.parent is not None else -1)
        assert np.array_equal(T["box"][c.id], np.concatenate([c.lo, c.hi]))
        if c.sons:
            assert (T["son0"][c.id], T["son1"][c.id]) == (c.sons[0].id, c.sons[1].id)
        else:
            assert T["son0"][c.id] == -1
    lib_adm = {(t, int(T["adm_col"][j])) for t in range(T["n_clusters"])
               for j in range(T["adm_rowptr"][t], T["adm_rowptr"][t + 1])}
    lib_near = {(t, int(T["near_col"][j])) for t in range(T["n_clusters"])
                for j in range(T["near_rowptr"][t], T["near_rowptr"][t + 1])}
    assert len(lib_adm) == T["n_adm"] and len(lib_near) == T["n_near"]
    assert lib_adm == {(b.t.id, b.s.id) for b in adm}
    assert lib_near == {(b.t.id, b.s.id) for b in near}
    return T


@pytest.mark.parametrize("n,seed", [(1, 0), (64, 1), (65, 2), (4096, 0), (20000, 3)])
def test_topology_matches_oracle_sphere(h2lib, n, seed):
    _compare(h2lib, sphere_points(n, seed))


def test_topology_matches_oracle_ellipsoid_and_degenerate(h2lib):
    _compare(h2lib, ellipsoid_points(5000, (0.5, 1.7, 1.1), 4), leaf=40)
    _compare(h2lib, np.full((300, 3), 0.25), leaf=64)
    pl = sphere_points(3000, 5)
    pl[:, 2] = 0.0
    _compare(h2lib, pl, leaf=17, eta=1.0)


def test_topology_golden_tiny_line(h2lib):
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tiny_line_blocks.json")))
    pts = np.zeros((6, 3))
    pts[:, 0] = d["points_x"]
    T = _compare(h2lib, pts, leaf=d["leaf_size"], eta=d["eta"])
    assert T["perm"].tolist() == d["perm"]
    assert T["n_adm"] == len(d["admissible"]) and T["n_near"] == len(d["inadmissible"])


def test_each_leaf_block_in_exactly_one_list(h2lib):
    pts = sphere_points(6000, 9)
    T = h2lib.h2_tree_build(pts, leaf_size=32, eta=2.0)
    n = T["n"]
    # expand every block of the row-cluster lists to its index rectangle; the
    # rectangles must tile I × I exactly once (checked on a sampled row set)
    rows = np.random.default_rng(0).choice(n, 200, replace=False)
    pos = np.empty(n, dtype=np.int64)
    pos[T["perm"]] = np.arange(n)
    cover = np.zeros((len(rows), n), dtype=np.int32)
    prow = pos[rows]
    for kind in ("adm", "near"):
        rp, col = T[kind + "_rowptr"], T[kind + "_col"]
        for t in range(T["n_clusters"]):
            o, s = T["offset"][t], T["size"][t]
            sel = np.nonzero((prow >= o) & (prow < o + s))[0]
            if sel.size == 0:
                continue
            for j in range(rp[t], rp[t + 1]):
                c = col[j]
                cover[np.ix_(sel, np.arange(T["offset"][c], T["offset"][c] + T["size"][c]))] += 1
    assert cover.min() == 1 and cover.max() == 1


def test_tree_argument_errors(h2lib):
    with pytest.raises(h2lib.H2Error) as e:
        h2lib.h2_tree_build(np.zeros((0, 3)))
    assert e.value.code == h2lib.H2_E_BADARG
    bad = sphere_points(100, 1)
    bad[5, 1] = np.nan
    with pytest.raises(h2lib.H2Error) as e:
        h2lib.h2_tree_build(bad)
    assert e.value.code == h2lib.H2_E_BADARG
    with pytest.raises(h2lib.H2Error) as e:
        h2lib.h2_tree_build(sphere_points(100, 1), q=6)
    assert e.value.code == h2lib.H2_E_UNSUPPORTED
    with pytest.raises(h2lib.H2Error) as e:
        h2lib.h2_tree_build(sphere_points(100, 1), leaf_size=65)
    assert e.value.code == h2lib.H2_E_UNSUPPORTED
    with pytest.raises(h2lib.H2Error) as e:
        h2lib.h2_tree_build(sphere_points(100, 1), eta=0.0)
    assert e.value.code == h2lib.H2_E_BADARG


def test_every_export_has_argtypes():
    """ctypes passes untyped Python ints as 32-bit C ints: every entry point
    that takes arguments declares them."""
    import paper_2509_17257_gb300.h2 as H
    L = H.lib()
    missing = [name for name in H.EXPORTS
               if name not in ("h2_last_error_string", "h2_version") and getattr(L, name).argtypes is None]
    assert not missing, missing


def test_matrix_entry_points_reject_bad_arguments_before_any_device_work(h2lib):
    """Null handles, bad sizes and bad parameters come back as statuses (and a
    message), checked before any CUDA call, so this runs without a GPU."""
    import ctypes as C

    import paper_2509_17257_gb300.h2 as H
    L = H.lib()
    BAD, UNSUP = h2lib.H2_E_BADARG, h2lib.H2_E_UNSUPPORTED
    x = np.zeros((4, 2))
    for f in (L.h2_matmul, L.h2_matmul_transposed):
        assert f(None, 1.0, x.ctypes.data, 2, x.ctypes.data, 2, 2, h2lib.H2_F64, None) == BAD
    assert L.h2_info(None, C.byref(H.Info())) == BAD
    assert L.h2_timing_enable(None, 1) == BAD
    cp = H.CGParams(1e-8, 100, h2lib.H2_CG_COLUMNWISE, h2lib.H2_F64, 0, 0.1, 10, 1, 0, h2lib.H2_PRECOND_NONE, None)
    res = H.CGResult()
    assert L.h2_block_cg(None, x.ctypes.data, 2, x.ctypes.data, 2, 2, C.byref(cp), C.byref(res)) == BAD
    gp = H.GMRESParams(1e-8, 100, 30, h2lib.H2_F64, h2lib.H2_PRECOND_NONE, 0, None)
    assert L.h2_block_gmres(None, x.ctypes.data, 2, x.ctypes.data, 2, 2, C.byref(gp), C.byref(res)) == BAD
    assert "null" in L.h2_last_error_string().decode()
    assert L.h2_matmul_complex(None, 1.0, 0.0, x.ctypes.data, 1, x.ctypes.data, 1, 1, h2lib.H2_F64, None) == BAD
    pts = np.ascontiguousarray(sphere_points(50, 1))
    h = C.c_void_p()
    for params, code in ((H.BuildParams(3, 64, 0.0, 0.5, 0.0, 1, None), BAD),       # eta
                         (H.BuildParams(3, 64, 2.0, -1.0, 0.0, 1, None), BAD),      # length
                         (H.BuildParams(3, 64, 2.0, 0.5, np.nan, 1, None), BAD),    # sigma
                         (H.BuildParams(6, 64, 2.0, 0.5, 0.0, 1, None), UNSUP),     # q
                         (H.BuildParams(3, 65, 2.0, 0.5, 0.0, 1, None), UNSUP),     # leaf size
                         (H.BuildParams(3, 64, 2.0, 0.5, 0.0, 1, None, 2, 1.0, 0.05), BAD),        # kernel
                         (H.BuildParams(3, 64, 2.0, 0.5, 0.0, 1, None, 1, np.inf, 0.05), BAD),     # kappa
                         (H.BuildParams(3, 64, 2.0, 0.5, 0.0, 1, None, 1, 1.0, 0.0), BAD),         # delta
                         (H.BuildParams(3, 64, 2.0, 0.5, 0.0, 1 << h2lib.H2_BF16, None, 1, 1.0, 0.05),
                          UNSUP)):                                                   # BF16 of a complex kernel
        assert L.h2_build(C.byref(params), pts.ctypes.data, 50, C.byref(h)) == code
        assert not h.value
    ok = H.BuildParams(3, 64, 2.0, 0.5, 0.0, 1, None)
    assert L.h2_build(C.byref(ok), None, 50, C.byref(h)) == BAD
    assert L.h2_build(C.byref(ok), pts.ctypes.data, 0, C.byref(h)) == BAD
    assert L.h2_build(C.byref(ok), pts.ctypes.data, 50, None) == BAD
