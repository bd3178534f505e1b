"""Host logic of the subtree-owning transfer passes (no GPU): the schedules
that h2_build hands to the upward and downward pass kernels, replayed in
numpy exactly as the kernels walk them, against a plain level-by-level pass
(Sec. 3, Alg. "fast_addeval": x̂_t = Σ E_{t'}ᵀ x̂_{t'} upwards, ŷ_{t'} += E_{t'} ŷ_t
downwards), with random transfer matrices.

Downward: a task loads the root's ŷ, recomputes the path to its cut cluster
and walks the cut cluster's subtree; every leaf must be stored exactly once,
with the value of the level-by-level pass, bit for bit (the same operations in
the same order).  Upward: every cluster below the cut is evaluated exactly once
in a post-order whose stack entries hold the sons when their father reads
them; the clusters above the cut are the climb's."""
import numpy as np
import pytest

import paper_2509_17257_gb300 as P
from workloads import ellipsoid_points, sphere_points

LOAD, STORE = 1, 2


def _tree(pts, q):
    return P.h2_tree_build(pts, leaf_size=64, eta=2.0, q=q)


CASES = [
    ("sphere20000", lambda: sphere_points(20000, 0), 3),
    ("sphere65536", lambda: sphere_points(65536, 0), 4),
    ("ellipsoid9000", lambda: ellipsoid_points(9000, (0.6, 1.9, 1.2), 5), 3),
    ("tiny", lambda: sphere_points(100, 7), 2),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    _, gen, q = request.param
    pts = gen()
    return pts, q, _tree(pts, q)


def _rand(rng, nc, k, m):
    E = rng.standard_normal((nc, k, k)) / np.sqrt(k)
    Y = rng.standard_normal((nc, k, m))
    return E, Y


def test_downward_schedule_reproduces_the_level_pass(case):
    pts, q, T = case
    nc = T["n_clusters"]
    par, son0 = T["parent"], T["son0"]
    sch = P.h2_tree_schedule(pts, "down", q=q)
    if nc <= 1:
        assert len(sch["task_ptr"]) == 1
        return
    k, m = 3, 2
    rng = np.random.default_rng(11)
    E, Yc = _rand(rng, nc, k, m)
    # level-by-level: clusters in pre-order have their father first
    ref = Yc.copy()
    for c in range(1, nc):
        ref[c] = Yc[c] + E[c] @ ref[par[c]]
    leaves = np.flatnonzero(son0 < 0)
    stored = {}
    ptr, steps, ent = sch["task_ptr"], sch["steps"], sch["entries"]
    for t in range(len(ptr) - 1):
        stack = [None] * ent
        who = [None] * ent  # which cluster's final ŷ each entry holds
        for c, rd, wr, fl in steps[ptr[t]:ptr[t + 1]]:
            assert 0 <= wr < ent
            if fl & LOAD:
                assert c == 0 and rd == -1
                stack[wr], who[wr] = Yc[0].copy(), 0
                continue
            assert 0 <= rd < ent and who[rd] == par[c], "the read entry must hold the father's ŷ"
            v = Yc[c] + E[c] @ stack[rd]
            stack[wr], who[wr] = v, c
            if fl & STORE:
                assert son0[c] < 0, "only leaves are stored"
                assert c not in stored, "every leaf is stored once"
                stored[c] = v
    assert sorted(stored) == sorted(leaves.tolist())
    for c, v in stored.items():
        assert np.array_equal(v, ref[c])


def test_upward_schedule_covers_the_tree_once(case):
    pts, q, T = case
    nc = T["n_clusters"]
    par, son0, son1, level = T["parent"], T["son0"], T["son1"], T["level"]
    sch = P.h2_tree_schedule(pts, "up", q=q)
    k, m = 3, 2
    rng = np.random.default_rng(12)
    E, Xl = _rand(rng, nc, k, m)  # Xl[c] stands for V_cᵀ X|_ĉ at a leaf
    ref = np.zeros_like(Xl)
    for c in range(nc - 1, -1, -1):  # sons after their father in pre-order: reverse is post-order
        ref[c] = Xl[c] if son0[c] < 0 else E[son0[c]].T @ ref[son0[c]] + E[son1[c]].T @ ref[son1[c]]
    got = {}
    roots = []
    ptr, steps, ent = sch["task_ptr"], sch["steps"], sch["entries"]
    assert ent >= 3
    lp = {c: i for i, c in enumerate(np.flatnonzero(son0 < 0))}
    for t in range(len(ptr) - 1):
        stack = [None] * ent
        who = [None] * ent
        for c, rd0, rd1, wr in steps[ptr[t]:ptr[t + 1]]:
            assert 0 <= wr < ent
            if rd0 < 0:
                assert son0[c] < 0 and rd1 == lp[c], "a leaf step carries the leaf's position"
                v = Xl[c].copy()
            else:
                assert who[rd0] == son0[c] and who[rd1] == son1[c], "entries hold the sons"
                v = E[son0[c]].T @ stack[rd0] + E[son1[c]].T @ stack[rd1]
            assert c not in got, "every cluster below the cut is evaluated once"
            stack[wr], who[wr] = v, c
            got[c] = v
        roots.append(steps[ptr[t + 1] - 1][0])
    # the cut: no task root lies inside another task's subtree, and the clusters
    # no task evaluated are exactly the strict ancestors of task roots
    above = set()
    for r in roots:
        a = par[r]
        while a >= 0:
            above.add(a)
            a = par[a]
    assert above.isdisjoint(got)
    assert set(got) | above == set(range(nc))
    for c, v in got.items():
        assert np.allclose(v, ref[c], rtol=1e-12, atol=1e-12)
    # the climb: the later brother adds the two contributions E_sᵀ x̂_s
    for c in sorted(above, key=lambda c: -level[c]):
        got[c] = E[son0[c]].T @ got[son0[c]] + E[son1[c]].T @ got[son1[c]]
        assert np.allclose(got[c], ref[c], rtol=1e-12, atol=1e-12)


def test_schedule_limits(case):
    pts, q, T = case
    down = P.h2_tree_schedule(pts, "down", q=q)
    up = P.h2_tree_schedule(pts, "up", q=q)
    # stack sizes and step counts the kernels' shared memory is sized for
    assert down["entries"] <= 8
    assert up["entries"] <= 5
    if len(down["task_ptr"]) > 1:
        assert np.diff(down["task_ptr"]).max() <= 192
    assert np.diff(up["task_ptr"]).max() <= 64
    # longest tasks first (the kernels claim tasks in order)
    for s in (down, up):
        lens = np.diff(s["task_ptr"])
        assert np.all(lens[:-1] >= lens[1:])


def test_schedule_argument_errors():
    import ctypes as C

    import paper_2509_17257_gb300.h2 as H
    L = H.lib()
    pts = np.ascontiguousarray(sphere_points(500, 3))
    bp = H.BuildParams(3, 64, 2.0, 0.5, 0.0, 0, None)
    h = C.c_void_p()
    assert L.h2_tree_build(C.byref(bp), pts.ctypes.data, pts.shape[0], C.byref(h)) == 0
    try:
        nt, ns, ent = C.c_int32(), C.c_int32(), C.c_int32()
        assert L.h2_tree_schedule(h, 2, C.byref(nt), C.byref(ns), C.byref(ent), None, None) == P.H2_E_BADARG
        assert L.h2_tree_schedule(None, 0, C.byref(nt), C.byref(ns), C.byref(ent), None, None) == P.H2_E_BADARG
        assert L.h2_tree_schedule(h, 0, None, C.byref(ns), C.byref(ent), None, None) == P.H2_E_BADARG
        # sizes first, then the arrays: both calls agree
        assert L.h2_tree_schedule(h, 1, C.byref(nt), C.byref(ns), C.byref(ent), None, None) == 0
        ptr = np.zeros(nt.value + 1, dtype=np.int32)
        steps = np.zeros((ns.value, 4), dtype=np.int32)
        nt2, ns2 = C.c_int32(), C.c_int32()
        assert L.h2_tree_schedule(h, 1, C.byref(nt2), C.byref(ns2), C.byref(ent), ptr.ctypes.data,
                                  steps.ctypes.data) == 0
        assert (nt2.value, ns2.value) == (nt.value, ns.value)
        assert ptr[0] == 0 and ptr[-1] == ns.value and np.all(np.diff(ptr) > 0)
    finally:
        L.h2_tree_free(h)
