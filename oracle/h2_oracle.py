"""Plain, slow FP64 CPU oracle for the H²-matrix × dense-block product and block CG.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this module.  The
library in ``paper_2509_17257_gb300`` never imports, links or calls it, and
this module imports nothing from the library: the two share no code.

What it follows (arXiv 2509.17257, "On efficient block Krylov solvers for
H²-matrices"):

* Sec. 2, Def. "Cluster tree"          -> :func:`build_cluster_tree`
* Sec. 2, Def. "Block tree"            -> :func:`build_block_tree`
* Sec. 2, Eq. (admiss)                 -> :func:`admissible`
* Sec. 2, Eq. (h2_admissible) and Def. "Cluster basis" (nested bases with
  transfer matrices E), built here by tensor Chebyshev interpolation, one of
  the constructions Sec. 2 names   -> :class:`H2Matrix`
* Sec. 3, Alg. "H2_mvm" (forward transformation, multiplication phase
  "fast_addeval", backward transformation) with the coefficient blocks of
  Sec. 4 (x̂_s, ŷ_t in K^{k×m})  -> :func:`h2mm`, over K = R and, for the
  complex Helmholtz kernel of Sec. 2 (with a smooth regularisation at
  r = 0), over K = C                       -> :func:`helmholtz_kernel`
* the same product with BF16 operands and FP32 accumulation, the error
  budget of the BF16 product (not in the paper) -> :func:`h2mm_bf16`
* Sec. 5.1, Alg. "block CG" (per-column α_i, β_i, γ_i) -> :func:`block_cg`
* the same recurrences with m×m Gram matrices in place of the per-column
  scalars (O'Leary's block CG; not in the paper)      -> :func:`block_cg_gram`
* Sec. 5.1, Alg. "pcg block" with a block-Jacobi M  -> :func:`block_pcg`
* Sec. 5.2, Alg. "pgmres block" (restarted, per column) -> :func:`block_gmres`

Readings where the paper is silent (split rule, diam/dist of point boxes,
interpolation nodes, kernel, shift, stopping rule) are the ones stated in the
docstrings below.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force or library routines (see each test).  The
interpolation *accuracy* against the exact kernel has no number in the paper
to compare with; it is pinned only by its decay in q.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Cluster",
    "Block",
    "build_cluster_tree",
    "clusters_preorder",
    "diam",
    "dist",
    "admissible",
    "build_block_tree",
    "leaf_blocks",
    "exp_kernel",
    "helmholtz_kernel",
    "cluster_nodes",
    "tensor_nodes",
    "lagrange_1d",
    "tensor_lagrange",
    "H2Matrix",
    "h2mm",
    "dense_expand",
    "kernel_matrix",
    "block_cg",
    "CGResult",
    "adjoint_grads",
    "set_coupling",
    "block_jacobi",
    "block_pcg",
    "block_cg_gram",
    "GRAM_DEFLATE",
    "H2Rows",
    "block_gmres",
    "GMRESResult",
    "round_bf16",
    "BF16_OPERANDS",
    "h2mm_bf16",
]


# ---------------------------------------------------------------------------
# Cluster tree (Sec. 2, Def. "Cluster tree")
# ---------------------------------------------------------------------------
class Cluster:
    """A node t of the cluster tree T_I.

    ``idx``  : original point indices of the label t̂, in pre-order (the
               concatenation of the sons' labels), so t̂ is the contiguous range
               [offset, offset + size) of the permutation ``root.idx``.
    ``lo/hi``: the tight axis-aligned bounding box of the points of t̂.
    """

    __slots__ = ("idx", "lo", "hi", "sons", "level", "offset", "parent", "id")

    def __init__(self, idx, lo, hi, level, offset, parent):
        self.idx = idx
        self.lo = lo
        self.hi = hi
        self.sons = []
        self.level = level
        self.offset = offset
        self.parent = parent
        self.id = -1

    @property
    def size(self) -> int:
        return int(self.idx.shape[0])

    @property
    def is_leaf(self) -> bool:
        return not self.sons


def build_cluster_tree(points: np.ndarray, leaf_size: int) -> Cluster:
    """Recursive geometric bisection (Sec. 2: split into non-overlapping parts
    until each cluster is small).

    Split rule (the paper gives none; this is the reading used on both sides):
    a cluster with more than ``leaf_size`` points is split; its box is the
    tight AABB of its points; the longest side (ties -> lowest axis) is cut at
    its midpoint ``(lo + hi) * 0.5``; points with coordinate <= midpoint form
    son 0, the rest son 1, both in their current order.  If one side would be
    empty (coincident points), the index range is halved instead: the first
    ``size // 2`` points form son 0.
    """
    points = np.asarray(points, dtype=np.float64)
    n = points.shape[0]
    if n < 1:
        raise ValueError("empty point set")

    def rec(idx, level, offset, parent):
        pts = points[idx]
        lo = pts.min(axis=0)
        hi = pts.max(axis=0)
        c = Cluster(idx, lo, hi, level, offset, parent)
        if idx.shape[0] > leaf_size:
            w = hi - lo
            d = int(np.argmax(w))  # first maximal side
            mid = (lo[d] + hi[d]) * 0.5
            mask = pts[:, d] <= mid
            i0 = idx[mask]
            i1 = idx[~mask]
            if i0.shape[0] == 0 or i1.shape[0] == 0:
                h = idx.shape[0] // 2
                i0, i1 = idx[:h], idx[h:]
            s0 = rec(i0, level + 1, offset, c)
            s1 = rec(i1, level + 1, offset + i0.shape[0], c)
            c.sons = [s0, s1]
            c.idx = np.concatenate([s0.idx, s1.idx])
        return c

    root = rec(np.arange(n, dtype=np.int64), 0, 0, None)
    for i, c in enumerate(clusters_preorder(root)):
        c.id = i
    return root


def clusters_preorder(root: Cluster):
    """All clusters in pre-order (parent before sons, son 0 before son 1)."""
    out = []
    stack = [root]
    while stack:
        c = stack.pop()
        out.append(c)
        stack.extend(reversed(c.sons))
    return out


# ---------------------------------------------------------------------------
# Admissibility (Sec. 2, Eq. (admiss))
# ---------------------------------------------------------------------------
def diam(c: Cluster) -> float:
    """Euclidean length of the box diagonal, sqrt((w0² + w1²) + w2²)."""
    w0 = float(c.hi[0] - c.lo[0])
    w1 = float(c.hi[1] - c.lo[1])
    w2 = float(c.hi[2] - c.lo[2])
    return math.sqrt((w0 * w0 + w1 * w1) + w2 * w2)


def dist(t: Cluster, s: Cluster) -> float:
    """Euclidean distance between the two boxes (0 when they touch or overlap)."""
    g = []
    for d in range(3):
        a = float(s.lo[d] - t.hi[d])
        b = float(t.lo[d] - s.hi[d])
        g.append(max(a, b, 0.0))
    return math.sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2])


def admissible(t: Cluster, s: Cluster, eta: float) -> bool:
    """Eq. (admiss): max{diam t, diam s} <= eta·dist(t, s), with dist > 0 required."""
    dd = dist(t, s)
    if not dd > 0.0:
        return False
    return max(diam(t), diam(s)) <= eta * dd


# ---------------------------------------------------------------------------
# Block tree (Sec. 2, Def. "Block tree")
# ---------------------------------------------------------------------------
@dataclass(eq=False)
class Block:
    t: Cluster
    s: Cluster
    kind: str  # "adm" (L+), "near" (L-), or "inner"
    sons: list = field(default_factory=list)


def build_block_tree(root_t: Cluster, root_s: Cluster, eta: float) -> Block:
    """Block tree from (root, root) with the sons rule of Def. "Block tree".

    Stopping (the paper gives only the sons rule): a block is a leaf iff it is
    admissible (L+) or both clusters are leaves (then it is in L-).
    """

    def rec(t, s):
        if admissible(t, s, eta):
            return Block(t, s, "adm")
        if t.is_leaf and s.is_leaf:
            return Block(t, s, "near")
        b = Block(t, s, "inner")
        if t.is_leaf:
            b.sons = [rec(t, s2) for s2 in s.sons]
        elif s.is_leaf:
            b.sons = [rec(t2, s) for t2 in t.sons]
        else:
            b.sons = [rec(t2, s2) for t2 in t.sons for s2 in s.sons]
        return b

    return rec(root_t, root_s)


def leaf_blocks(b: Block):
    """The leaves L_{I×J} of a block tree, split into (admissible, inadmissible)."""
    adm, near = [], []
    stack = [b]
    while stack:
        x = stack.pop()
        if x.kind == "adm":
            adm.append(x)
        elif x.kind == "near":
            near.append(x)
        else:
            stack.extend(reversed(x.sons))
    return adm, near


# ---------------------------------------------------------------------------
# Kernel function g and tensor Chebyshev interpolation (Sec. 2)
# ---------------------------------------------------------------------------
def exp_kernel(length: float = 0.5):
    """g(x, y) = exp(-||x - y||_2 / length), broadcasting over leading axes."""

    def g(x, y):
        d = x - y
        r = np.sqrt((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2])
        return np.exp(-r / length)

    return g


def helmholtz_kernel(kappa: float = 1.0, delta: float = 0.05):
    """The Helmholtz kernel of Sec. 2 (K = C), g(x, y) = exp(i κ r) / (4π r) with
    r = ||x - y||_2, regularised at r = 0 as

        g_{κ,δ}(x, y) = exp(i κ r) / (4π sqrt(r² + δ²)),

    which is smooth everywhere (the diagonal entries are 1 / (4π δ)) and equals
    the paper's kernel up to a relative O(δ²/r²) away from the diagonal; δ = 0
    gives the paper's kernel for r > 0.  Broadcasts over leading axes."""

    def g(x, y):
        d = x - y
        r = np.sqrt((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2])
        return np.exp(1j * kappa * r) / (4.0 * np.pi * np.sqrt(r * r + delta * delta))

    return g


def cluster_nodes(c: Cluster, q: int) -> np.ndarray:
    """Chebyshev points of the first kind mapped to the cluster's box, shape (3, q).

    node_{d,i} = center_d + half_d · cos((2i+1)π / (2q)).  A degenerate side
    (half-width below 1e-8 × the largest half-width) is widened to that floor so
    the nodes stay distinct; a box with no extent at all gets half-widths 1e-8.
    """
    center = (c.lo + c.hi) * 0.5
    half = (c.hi - c.lo) * 0.5
    hmax = float(half.max())
    floor = 1e-8 * hmax if hmax > 0.0 else 1e-8
    half = np.maximum(half, floor)
    ref = np.cos((2.0 * np.arange(q) + 1.0) * math.pi / (2.0 * q))
    return center[:, None] + half[:, None] * ref[None, :]


def tensor_nodes(nodes: np.ndarray) -> np.ndarray:
    """The k = q³ tensor nodes, shape (k, 3), with index ν = ν_x + q·ν_y + q²·ν_z."""
    q = nodes.shape[1]
    out = np.empty((q ** 3, 3))
    for nz in range(q):
        for ny in range(q):
            for nx in range(q):
                nu = nx + q * ny + q * q * nz
                out[nu] = (nodes[0, nx], nodes[1, ny], nodes[2, nz])
    return out


def lagrange_1d(nodes_1d: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L_i(x) = prod_{j != i} (x - ξ_j) / (ξ_i - ξ_j); returns shape (len(x), q)."""
    x = np.asarray(x, dtype=np.float64)
    q = nodes_1d.shape[0]
    out = np.ones((x.shape[0], q))
    for i in range(q):
        for j in range(q):
            if j != i:
                out[:, i] *= (x - nodes_1d[j]) / (nodes_1d[i] - nodes_1d[j])
    return out


def tensor_lagrange(nodes: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Tensor Lagrange polynomials L_ν(x) = L_{ν_x}(x_0) L_{ν_y}(x_1) L_{ν_z}(x_2), shape (len(pts), k)."""
    q = nodes.shape[1]
    lx = lagrange_1d(nodes[0], pts[:, 0])
    ly = lagrange_1d(nodes[1], pts[:, 1])
    lz = lagrange_1d(nodes[2], pts[:, 2])
    out = np.empty((pts.shape[0], q ** 3))
    for nz in range(q):
        for ny in range(q):
            for nx in range(q):
                out[:, nx + q * ny + q * q * nz] = lx[:, nx] * ly[:, ny] * lz[:, nz]
    return out


# ---------------------------------------------------------------------------
# The H² matrix (Sec. 2, Def. "H²-matrix"; W = V since I = J and the bases are real)
# ---------------------------------------------------------------------------
class H2Matrix:
    """Interpolation-based H² matrix A = Â + σI for a point cloud.

    * leaf matrices   V_t[i, ν] = L_{t,ν}(x_i), t leaf (Def. "Cluster basis")
    * transfer        E_{t'}[μ, ν] = L_{t,ν}(ξ_{t',μ}), t = father of t', so
                      that V_t|_{t̂'×k} = V_{t'} E_{t'}
    * coupling        S_b[ν, μ] = g(ξ_{t,ν}, ξ_{s,μ}), b = (t, s) ∈ L+ (Eq. (h2_admissible))
    * nearfield       G_b[i, j] = g(x_i, x_j), b ∈ L-  (stored explicitly, Sec. 2)
    * shift           σ on the diagonal only, applied separately.

    Over R the paper's W_s* and E* become transposes, and W = V.  With a
    complex kernel (K = C) the bases stay real (Lagrange polynomials of real
    nodes), S_b and G_b are complex, and the product is A X, not A* X; the
    transposed product is Aᵀ X (no conjugation).  ``dtype`` is float64 or
    complex128, the type of the stored entries.
    """

    def __init__(self, points, q=3, leaf_size=64, eta=2.0, kernel=None, sigma=0.0, length=0.5):
        self.points = np.ascontiguousarray(points, dtype=np.float64)
        self.n = self.points.shape[0]
        self.q = q
        self.k = q ** 3
        self.eta = eta
        self.sigma = float(sigma)
        self.g = kernel if kernel is not None else exp_kernel(length)
        self.root = build_cluster_tree(self.points, leaf_size)
        self.clusters = clusters_preorder(self.root)
        self.perm = self.root.idx
        self.btree = build_block_tree(self.root, self.root, eta)
        self.adm, self.near = leaf_blocks(self.btree)
        self.nodes = {c.id: cluster_nodes(c, q) for c in self.clusters}
        self.tnodes = {c.id: tensor_nodes(self.nodes[c.id]) for c in self.clusters}
        self.V = {}
        self.E = {}
        for c in self.clusters:
            if c.is_leaf:
                self.V[c.id] = tensor_lagrange(self.nodes[c.id], self.points[c.idx])
            if c.parent is not None:
                self.E[c.id] = tensor_lagrange(self.nodes[c.parent.id], self.tnodes[c.id])
        for b in self.adm:
            b.S = self.g(self.tnodes[b.t.id][:, None, :], self.tnodes[b.s.id][None, :, :])
        for b in self.near:
            b.G = self.g(self.points[b.t.idx][:, None, :], self.points[b.s.idx][None, :, :])
        self.dtype = np.result_type(np.float64, *[b.S.dtype for b in self.adm], *[b.G.dtype for b in self.near])

    # -- sizes -----------------------------------------------------------
    def counts(self):
        leaves = [c for c in self.clusters if c.is_leaf]
        return dict(
            n=self.n,
            n_clusters=len(self.clusters),
            n_leaves=len(leaves),
            n_adm=len(self.adm),
            n_near=len(self.near),
            nnz_near=int(sum(b.t.size * b.s.size for b in self.near)),
            depth=max(c.level for c in self.clusters),
        )


# ---------------------------------------------------------------------------
# H² × dense block (Sec. 3 Alg. "H2_mvm" with the k×m blocks of Sec. 4)
# ---------------------------------------------------------------------------
def _forward(H: H2Matrix, s: Cluster, X: np.ndarray, xhat: dict):
    """Forward transformation: x̂_s = V_sᵀ x|_ŝ at leaves, x̂_s = Σ E_{s'}ᵀ x̂_{s'} above."""
    if s.is_leaf:
        xhat[s.id] = H.V[s.id].T @ X[s.idx]
    else:
        acc = np.zeros((H.k, X.shape[1]), dtype=X.dtype)
        for s2 in s.sons:
            _forward(H, s2, X, xhat)
            acc = acc + H.E[s2.id].T @ xhat[s2.id]
        xhat[s.id] = acc


def _fast_addeval(H, alpha, b: Block, xhat, yhat, X, Y, transposed):
    """Multiplication phase: ŷ_t += α S_b x̂_s on L+, y|_t̂ += α G_b x|_ŝ on L-."""
    if b.kind == "adm":
        if transposed:  # block (s, t) of Aᵀ is V_s S_bᵀ V_tᵀ
            yhat[b.s.id] += alpha * (b.S.T @ xhat[b.t.id])
        else:
            yhat[b.t.id] += alpha * (b.S @ xhat[b.s.id])
    elif b.kind == "near":
        if transposed:
            Y[b.s.idx] += alpha * (b.G.T @ X[b.t.idx])
        else:
            Y[b.t.idx] += alpha * (b.G @ X[b.s.idx])
    else:
        for b2 in b.sons:
            _fast_addeval(H, alpha, b2, xhat, yhat, X, Y, transposed)


def _backward(H: H2Matrix, t: Cluster, Y: np.ndarray, yhat: dict):
    """Backward transformation: ŷ_{t'} += E_{t'} ŷ_t downwards, y|_t̂ += V_t ŷ_t at leaves."""
    if t.is_leaf:
        Y[t.idx] += H.V[t.id] @ yhat[t.id]
    else:
        for t2 in t.sons:
            yhat[t2.id] = yhat[t2.id] + H.E[t2.id] @ yhat[t.id]
            _backward(H, t2, Y, yhat)


def h2mm(H: H2Matrix, alpha: float, X: np.ndarray, Y: np.ndarray | None = None,
         transposed: bool = False) -> np.ndarray:
    """Return Y + α·A·X (or Y + α·Aᵀ·X) for A = Â + σI; X, Y are n×m in the
    caller's point order.  Follows Alg. "H2_mvm": forward, fast_addeval,
    backward, then the diagonal shift.  The arithmetic is complex when the
    matrix, X, Y or α is (K = C), FP64 otherwise."""
    cplx = (np.dtype(H.dtype).kind == "c" or np.iscomplexobj(X) or np.iscomplexobj(alpha)
            or (Y is not None and np.iscomplexobj(Y)))
    dt = np.complex128 if cplx else np.float64
    X = np.asarray(X, dtype=dt)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    m = X.shape[1]
    Yo = np.zeros((H.n, m), dtype=dt) if Y is None else np.array(Y, dtype=dt).reshape(H.n, m)
    xhat = {}
    yhat = {c.id: np.zeros((H.k, m), dtype=dt) for c in H.clusters}
    _forward(H, H.root, X, xhat)
    _fast_addeval(H, alpha, H.btree, xhat, yhat, X, Yo, transposed)
    _backward(H, H.root, Yo, yhat)
    Yo += (alpha * H.sigma) * X
    return Yo[:, 0] if squeeze else Yo


# ---------------------------------------------------------------------------
# BF16 error budget: the same product with BF16 operands, FP32 accumulation
# ---------------------------------------------------------------------------
def round_bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 value, ties to even, returned as FP64.

    bfloat16 keeps 8 significant bits (the implicit leading one and seven
    stored ones) and the FP32 exponent range.  Writing a = f·2^e with
    0.5 <= |f| < 1, the rounded value is rint(f·2^8)·2^(e-8), where rint
    rounds half to even; a carry to 2^8 lands on the next power of two, as it
    should.  The value is rounded once, from FP64 (no FP32 step, whose own
    rounding could move a value onto a bfloat16 midpoint).  Valid for
    magnitudes in the normal range (>= 2^-126); zero stays zero."""
    a = np.asarray(a, dtype=np.float64)
    f, e = np.frexp(a)
    return np.ldexp(np.rint(np.ldexp(f, 8)), e - 8)


#: operands the BF16 error budget rounds by default: the leaf bases (forward
#: "Vf" and backward "Vb"), the transfer matrices "E", the couplings "S", the
#: nearfield blocks "G" and the input block "X"
BF16_OPERANDS = ("Vf", "Vb", "E", "S", "G", "X")


def h2mm_bf16(H: H2Matrix, alpha: float, X: np.ndarray, Y: np.ndarray | None = None,
              rounded=BF16_OPERANDS, transposed: bool = False) -> np.ndarray:
    """Y + α·A·X (or Aᵀ) with the named operands rounded to bfloat16 and every
    matrix product accumulated in FP32: the BF16 error budget of the product.

    The steps are those of :func:`h2mm` (Alg. "H2_mvm": forward
    transformation, coupling and nearfield blocks, backward transformation)
    on a plain per-operand reading of "BF16 operands, FP32 accumulation":

    * each operand named in ``rounded`` is rounded to BF16 once
      (:func:`round_bf16`); "V" names both "Vf" and "Vb";
    * the coefficient blocks x̂_s, ŷ_t and the leaf results stay FP32: they
      are the accumulators, not operands read from memory;
    * every product is a float32 matmul (a product of two BF16 values is
      exact in FP32; the sums round in FP32);
    * α is applied once at the end and the shift uses the FP64 X:
      Y + α·(Z + σX) in FP64, where Z is the FP32 result.

    With ``rounded=()`` this is the product in FP32 arithmetic."""
    ops = set()
    for name in rounded:
        ops.update(("Vf", "Vb") if name == "V" else (name,))
    unknown = ops - set(BF16_OPERANDS)
    if unknown:
        raise ValueError(f"unknown operand names {sorted(unknown)}")
    f32 = np.float32

    def op(name, a):
        return (round_bf16(a) if name in ops else np.asarray(a, dtype=np.float64)).astype(f32)

    X = np.asarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    m = X.shape[1]
    Xo = op("X", X)
    xhat = {}

    def forward(s):
        if s.is_leaf:
            xhat[s.id] = op("Vf", H.V[s.id]).T @ Xo[s.idx]
        else:
            acc = np.zeros((H.k, m), dtype=f32)
            for s2 in s.sons:
                forward(s2)
                acc = acc + op("E", H.E[s2.id]).T @ xhat[s2.id]
            xhat[s.id] = acc

    forward(H.root)
    yhat = {c.id: np.zeros((H.k, m), dtype=f32) for c in H.clusters}
    Z = np.zeros((H.n, m), dtype=f32)
    for b in H.adm:
        if transposed:
            yhat[b.s.id] = yhat[b.s.id] + op("S", b.S).T @ xhat[b.t.id]
        else:
            yhat[b.t.id] = yhat[b.t.id] + op("S", b.S) @ xhat[b.s.id]
    for b in H.near:
        if transposed:
            Z[b.s.idx] = Z[b.s.idx] + op("G", b.G).T @ Xo[b.t.idx]
        else:
            Z[b.t.idx] = Z[b.t.idx] + op("G", b.G) @ Xo[b.s.idx]

    def backward(t):
        if t.is_leaf:
            Z[t.idx] = Z[t.idx] + op("Vb", H.V[t.id]) @ yhat[t.id]
        else:
            for t2 in t.sons:
                yhat[t2.id] = yhat[t2.id] + op("E", H.E[t2.id]) @ yhat[t.id]
                backward(t2)

    backward(H.root)
    Yo = np.zeros((H.n, m)) if Y is None else np.array(Y, dtype=np.float64).reshape(H.n, m)
    Yo = Yo + alpha * (Z.astype(np.float64) + H.sigma * X)
    return Yo[:, 0] if squeeze else Yo


def _expanded_basis(H: H2Matrix, c: Cluster) -> np.ndarray:
    """V_t for any cluster via the nesting V_t|_{t̂'} = V_{t'} E_{t'} (Def. "Cluster basis")."""
    if c.is_leaf:
        return H.V[c.id]
    return np.vstack([_expanded_basis(H, c2) @ H.E[c2.id] for c2 in c.sons])


def dense_expand(H: H2Matrix) -> np.ndarray:
    """The dense n×n matrix Â + σI represented by H (caller's point order)."""
    A = np.zeros((H.n, H.n), dtype=H.dtype)
    cache = {}

    def vb(c):
        if c.id not in cache:
            cache[c.id] = _expanded_basis(H, c)
        return cache[c.id]

    for b in H.adm:
        A[np.ix_(b.t.idx, b.s.idx)] = vb(b.t) @ b.S @ vb(b.s).T
    for b in H.near:
        A[np.ix_(b.t.idx, b.s.idx)] = b.G
    A[np.diag_indices(H.n)] += H.sigma
    return A


def kernel_matrix(points: np.ndarray, g, sigma: float = 0.0) -> np.ndarray:
    """Brute-force K_ij = g(x_i, x_j) + σ δ_ij (the matrix the H² matrix approximates)."""
    K = g(points[:, None, :], points[None, :, :])
    K[np.diag_indices(points.shape[0])] += sigma
    return K


# ---------------------------------------------------------------------------
# Selected rows of the product for large n (same H² matrix, built lazily)
# ---------------------------------------------------------------------------
class H2Rows:
    """The H² matrix of :class:`H2Matrix` without its stored blocks, for sizes
    where those do not fit (n up to 2²⁰): the trees and nodes are built, the
    forward transformation of Alg. "forward/backward" is run with V_t and
    E_{t'} formed on the fly, and rows i of  α(Â + σI)X  are assembled one by
    one from the definition of Â (Def. "H²-matrix"):

        (ÂX)_i = Σ_{t ∋ i} V_t[i, :] Σ_{b=(t,s)∈L+} S_b x̂_s  +  Σ_{b=(t_i,s)∈L-} G_b[i, :] X|_ŝ,

    where t runs over the ancestors of the leaf t_i that holds i and
    V_t[i, :] = V_{t_i}[i, :] E_{t_i} E_{father(t_i)} … (the nesting
    V_t|_{t̂'} = V_{t'} E_{t'}).  S_b and G_b are formed only for the blocks
    that touch the requested rows.  ``kernel`` as for :class:`H2Matrix` (a
    complex kernel gives complex rows, K = C).
    """

    def __init__(self, points, q=3, leaf_size=64, eta=2.0, sigma=0.0, length=0.5, kernel=None):
        self.points = np.ascontiguousarray(points, dtype=np.float64)
        self.n = self.points.shape[0]
        self.q, self.k, self.eta, self.sigma = q, q ** 3, eta, float(sigma)
        self.g = kernel if kernel is not None else exp_kernel(length)
        self.root = build_cluster_tree(self.points, leaf_size)
        self.clusters = clusters_preorder(self.root)
        self.nodes = {c.id: cluster_nodes(c, q) for c in self.clusters}
        self.tnodes = {c.id: tensor_nodes(self.nodes[c.id]) for c in self.clusters}
        adm, near = leaf_blocks(build_block_tree(self.root, self.root, eta))
        self.adm_of, self.near_of = {}, {}
        for b in adm:
            self.adm_of.setdefault(b.t.id, []).append(b.s)
        for b in near:
            self.near_of.setdefault(b.t.id, []).append(b.s)
        self.n_adm, self.n_near = len(adm), len(near)
        # leaf holding each original index, and the position inside it
        self.leaf_of = np.empty(self.n, dtype=np.int64)
        self.pos_in_leaf = np.empty(self.n, dtype=np.int64)
        self.by_id = {c.id: c for c in self.clusters}
        for c in self.clusters:
            if c.is_leaf:
                self.leaf_of[c.idx] = c.id
                self.pos_in_leaf[c.idx] = np.arange(c.size)

    def V(self, c):
        return tensor_lagrange(self.nodes[c.id], self.points[c.idx])

    def E(self, c):
        return tensor_lagrange(self.nodes[c.parent.id], self.tnodes[c.id])

    def forward(self, X):
        """x̂_s for every cluster (Alg. "forward/backward", forward part)."""
        X = np.asarray(X)
        X = X.astype(np.complex128 if np.iscomplexobj(X) else np.float64)
        xhat = {}
        for c in reversed(self.clusters):  # sons before fathers
            if c.is_leaf:
                xhat[c.id] = self.V(c).T @ X[c.idx]
            else:
                acc = np.zeros((self.k, X.shape[1]), dtype=X.dtype)
                for c2 in c.sons:
                    acc += self.E(c2).T @ xhat[c2.id]
                xhat[c.id] = acc
        return xhat

    def rows(self, alpha, X, rows, xhat=None):
        """Rows ``rows`` (original indices) of α(Â + σI)X, shape (len(rows), m)."""
        X = np.asarray(X)
        X = X.astype(np.complex128 if np.iscomplexobj(X) else np.float64)
        if xhat is None:
            xhat = self.forward(X)
        gi = self.g(self.points[:1], self.points[:1])
        dt = np.result_type(X.dtype, gi.dtype, np.asarray(alpha).dtype, np.float64)
        out = np.zeros((len(rows), X.shape[1]), dtype=dt)
        for r, i in enumerate(rows):
            t = self.by_id[int(self.leaf_of[i])]
            a = int(self.pos_in_leaf[i])
            v = self.V(t)[a]  # V_t[i, :] at the leaf
            acc = np.zeros(X.shape[1], dtype=dt)
            for s in self.near_of.get(t.id, []):
                acc += self.g(self.points[i][None, :], self.points[s.idx]) @ X[s.idx]
            c = t
            while c is not None:
                for s in self.adm_of.get(c.id, []):
                    S = self.g(self.tnodes[c.id][:, None, :], self.tnodes[s.id][None, :, :])
                    acc += v @ (S @ xhat[s.id])
                if c.parent is not None:
                    v = v @ self.E(c)
                c = c.parent
            out[r] = alpha * (acc + self.sigma * X[i])
        return out

    def coupling_grads(self, Lam, X, pairs):
        """−λ̂_t x̂_sᵀ for the admissible pairs (t.id, s.id) (see adjoint_grads)."""
        lh, xh = self.forward(Lam), self.forward(X)
        return {(t, s): -(lh[t] @ xh[s].T) for t, s in pairs}


# ---------------------------------------------------------------------------
# Block CG (Sec. 5.1, Alg. "block CG"; Alg. "CG" for its scalar form)
# ---------------------------------------------------------------------------
@dataclass
class CGResult:
    X: np.ndarray
    iterations: int
    col_iterations: np.ndarray
    rel_residual: np.ndarray  # recurrence residual ||r_i|| / ||b_i|| at exit
    status: str  # "converged", "breakdown", "noconverge"


def block_cg(apply_A, B: np.ndarray, X0: np.ndarray | None = None, tol: float = 1e-8,
             max_iter: int = 10000) -> CGResult:
    """Alg. "block CG": each column keeps its own Krylov space; one block
    product a = A p per iteration; per column
    β_i = <p_i, a_i>, α_i = <p_i, r_i>/β_i, x_i += α_i p_i, r_i -= α_i a_i,
    γ_i = <a_i, r_i>/β_i, p_i = r_i - γ_i p_i.

    Stopping (readings): column i has converged once ||r_i||/||b_i|| <= tol
    (||b_i|| = 0 is read as 1); converged columns are frozen; the loop runs
    until every column has converged.  β_i <= 0 or a non-finite value on an
    unconverged column is a breakdown.
    """
    B = np.asarray(B, dtype=np.float64)
    n, m = B.shape
    # columns are stored contiguously so each column's arithmetic is the same
    # whether it is solved alone or inside a block
    X = np.zeros((n, m), order="F") if X0 is None else np.array(X0, dtype=np.float64, order="F")
    R = np.asfortranarray(B - apply_A(X))
    P = R.copy(order="F")
    bn = np.linalg.norm(B, axis=0)
    bn[bn == 0.0] = 1.0
    done = np.linalg.norm(R, axis=0) / bn <= tol
    col_it = np.zeros(m, dtype=np.int64)
    it = 0
    status = "converged"
    while not done.all():
        if it >= max_iter:
            status = "noconverge"
            break
        Aq = np.asfortranarray(apply_A(P))
        it += 1
        for i in range(m):
            if done[i]:
                continue
            p, a, r = P[:, i], Aq[:, i], R[:, i]
            beta = float(p @ a)
            if not (beta > 0.0) or not math.isfinite(beta):
                status = "breakdown"
                break
            alpha = float(p @ r) / beta
            X[:, i] += alpha * p
            r = r - alpha * a
            R[:, i] = r
            gamma = float(a @ r) / beta
            P[:, i] = r - gamma * p
            col_it[i] = it
            if not math.isfinite(alpha) or not math.isfinite(gamma):
                status = "breakdown"
                break
            if np.linalg.norm(r) / bn[i] <= tol:
                done[i] = True
        if status == "breakdown":
            break
    rel = np.linalg.norm(R, axis=0) / bn
    return CGResult(X=X, iterations=it, col_iterations=col_it, rel_residual=rel, status=status)


# ---------------------------------------------------------------------------
# Block CG with m×m Gram matrices (O'Leary's block CG, written in the same
# conjugacy form as Alg. "CG": the scalars become m×m matrices)
# ---------------------------------------------------------------------------
GRAM_DEFLATE = 1e-10  # a direction is dropped when its Cholesky pivot is below this fraction of its diagonal


def _chol_deflate(G: np.ndarray, cols):
    """Cholesky G_KK = L Lᵀ over the columns K ⊆ cols that survive deflation.

    Pivots are taken in index order.  Column j is kept when its Schur pivot
    d_j = G_jj − Σ_{k∈K, k<j} L_jk² exceeds GRAM_DEFLATE·G_jj (p_j is then not
    A-dependent on the directions kept before it); otherwise it is dropped.
    G_jj <= 0 (or non-finite) means <p_j, A p_j> <= 0: breakdown, as for the
    scalar CG.  Returns (L restricted to K as an m×m array with zeros
    elsewhere, K as a list, breakdown flag)."""
    m = G.shape[0]
    L = np.zeros((m, m))
    K = []
    for j in cols:
        gjj = G[j, j]
        if not (gjj > 0.0) or not math.isfinite(gjj):
            return L, K, True
        d = gjj - sum(L[j, k] ** 2 for k in K)
        if not (d > GRAM_DEFLATE * gjj):
            continue
        L[j, j] = math.sqrt(d)
        for i in range(j + 1, m):
            L[i, j] = (G[i, j] - sum(L[i, k] * L[j, k] for k in K)) / L[j, j]
        K.append(j)
    return L, K, False


def _chol_solve(L: np.ndarray, K, Wcol: np.ndarray) -> np.ndarray:
    """y = G_KK⁻¹ w_K by forward then backward substitution; zero off K."""
    m = L.shape[0]
    z = np.zeros(m)
    for a, j in enumerate(K):
        z[j] = (Wcol[j] - sum(L[j, k] * z[k] for k in K[:a])) / L[j, j]
    y = np.zeros(m)
    for a in range(len(K) - 1, -1, -1):
        j = K[a]
        y[j] = (z[j] - sum(L[k, j] * y[k] for k in K[a + 1:])) / L[j, j]
    return y


def block_cg_gram(apply_A, B: np.ndarray, X0: np.ndarray | None = None, tol: float = 1e-8,
                  max_iter: int = 10000, apply_Minv=None) -> CGResult:
    """Block CG with m×m Gram matrices (O'Leary 1980), the block form of the
    scalar recurrences of Alg. "CG":

        Q = A P,   G = Pᵀ Q,   W = Pᵀ R,   α = G⁻¹ W,
        X += P α,  R −= Q α,   Γ = G⁻¹ (Qᵀ R),   P = R − P Γ.

    G⁻¹ is applied through a Cholesky factor of G with deflation
    (:func:`_chol_deflate`): a direction that has become A-dependent on the
    others is dropped for this step.  The stopping rule is the one of
    :func:`block_cg`: column i leaves the active set 𝒜 once
    ||r_i||/||b_i|| <= tol and is frozen from then on (its columns of α and Γ
    are zero and its direction is zero).  With m = 1 this is Alg. "CG".

    With a preconditioner (apply_Minv: R ↦ M⁻¹R) the directions are built
    from Z = M⁻¹R as in Alg. "pcg block": P starts as Z, Γ = G⁻¹ (AP)ᵀ Z and
    P = Z − PΓ.
    """
    B = np.asarray(B, dtype=np.float64)
    n, m = B.shape
    X = np.zeros((n, m)) if X0 is None else np.array(X0, dtype=np.float64)
    R = B - apply_A(X)
    Minv = (lambda V: V) if apply_Minv is None else apply_Minv
    P = np.array(Minv(R), dtype=np.float64)
    bn = np.linalg.norm(B, axis=0)
    bn[bn == 0.0] = 1.0
    active = np.linalg.norm(R, axis=0) / bn > tol
    P[:, ~active] = 0.0
    col_it = np.zeros(m, dtype=np.int64)
    it = 0
    status = "converged"
    while active.any():
        if it >= max_iter:
            status = "noconverge"
            break
        Q = apply_A(P)
        it += 1
        cols = [j for j in range(m) if active[j]]
        G = P.T @ Q
        W = P.T @ R
        L, K, broke = _chol_deflate(G, cols)
        if broke or not np.all(np.isfinite(G)):
            status = "breakdown"
            break
        alpha = np.zeros((m, m))
        for j in cols:
            alpha[:, j] = _chol_solve(L, K, W[:, j])
        X += P @ alpha
        R -= Q @ alpha
        rn = np.linalg.norm(R, axis=0) / bn
        for j in cols:
            col_it[j] = it
            if rn[j] <= tol:
                active[j] = False
        Zr = R if apply_Minv is None else np.asarray(Minv(R), dtype=np.float64)
        C = Q.T @ Zr
        Gamma = np.zeros((m, m))
        for j in range(m):
            if active[j]:
                Gamma[:, j] = _chol_solve(L, K, C[:, j])
        Pn = Zr - P @ Gamma
        Pn[:, ~active] = 0.0
        P = Pn
        if not np.all(np.isfinite(P)):
            status = "breakdown"
            break
    rel = np.linalg.norm(R, axis=0) / bn
    return CGResult(X=X, iterations=it, col_iterations=col_it, rel_residual=rel, status=status)


# ---------------------------------------------------------------------------
# Block GMRES (Sec. 5.2, Alg. "pgmres block"): every column runs restarted
# GMRES(ℓ) on its own Krylov space; one block product per step
# ---------------------------------------------------------------------------
@dataclass
class GMRESResult:
    X: np.ndarray
    iterations: int            # Arnoldi steps, summed over restart cycles (max over columns)
    cycles: int
    col_iterations: np.ndarray
    rel_residual: np.ndarray   # |M⁻¹(b - Ax)| / |M⁻¹ b| estimate at exit (the Givens residual)
    status: str


def _givens(a: float, b: float):
    """(c, s) with [c s; -s c] [a; b] = [r; 0], r = hypot(a, b) ≥ 0."""
    if b == 0.0:
        return 1.0, 0.0
    r = math.hypot(a, b)
    return a / r, b / r


def block_gmres(apply_A, B: np.ndarray, X0: np.ndarray | None = None, tol: float = 1e-8, restart: int = 30,
                max_iter: int = 10000, apply_Minv=None) -> GMRESResult:
    """Alg. "pgmres block": left-preconditioned GMRES(ℓ = restart) per column.

    One cycle, for every column i at once (the block product a = M⁻¹A q is
    the only coupling):  r = M⁻¹(b − Ax), β_i = |r_i|, q_0 = r/β, r̂ = β e_1;
    for k = 0, 1, …:  a = M⁻¹A q_k;  h_{0..k} = V_kᵀ a (all at once, as
    printed: classical Gram–Schmidt);  a −= V_k h;  h_{k+1,k} = |a|;
    q_{k+1} = a / h_{k+1,k};  the earlier Givens rotations are applied to the
    new column of H, a new rotation G_k removes h_{k+1,k} and is applied to r̂.
    The cycle ends after ℓ steps or when every column has |r̂_{k+1}| ≤ tol·|r̂⁰|
    (reading of the stopping test: relative to the column's initial
    preconditioned residual of the first cycle, the GMRES analogue of the CG
    rule); then x_i += V y_i with R y_i = r̂ (back substitution), and the
    next cycle restarts from the new x.  Columns that met the tolerance stop
    expanding their basis (frozen), as in block CG.  A zero h_{k+1,k} is a
    lucky breakdown: the column's Krylov space is invariant and its solution
    exact after the update.
    """
    B = np.asarray(B, dtype=np.float64)
    n, m = B.shape
    Minv = (lambda V: V) if apply_Minv is None else apply_Minv
    X = np.zeros((n, m)) if X0 is None else np.array(X0, dtype=np.float64)
    bn = np.linalg.norm(np.asarray(Minv(B)), axis=0)
    bn[bn == 0.0] = 1.0
    col_it = np.zeros(m, dtype=np.int64)
    done = np.zeros(m, dtype=bool)
    rel = np.ones(m)
    total, cycles = 0, 0
    status = "converged"
    while True:
        R = np.asarray(Minv(B - apply_A(X)), dtype=np.float64)
        beta = np.linalg.norm(R, axis=0)
        rel = beta / bn
        done = rel <= tol
        if done.all():
            break
        if total >= max_iter:
            status = "noconverge"
            break
        cycles += 1
        V = np.zeros((restart + 1, n, m))
        H = np.zeros((restart + 1, restart, m))
        cs = np.zeros((restart, m))
        sn = np.zeros((restart, m))
        rh = np.zeros((restart + 1, m))
        act = ~done
        for i in range(m):
            if act[i]:
                V[0, :, i] = R[:, i] / beta[i]
                rh[0, i] = beta[i]
        steps = np.zeros(m, dtype=np.int64)
        k = 0
        while k < restart and act.any() and total < max_iter:
            Q = np.where(act[None, :], V[k], 0.0)
            Aq = np.asarray(Minv(apply_A(Q)), dtype=np.float64)
            total += 1
            for i in range(m):
                if not act[i]:
                    continue
                a = Aq[:, i].copy()
                h = V[:k + 1, :, i] @ a            # all inner products first (CGS)
                a -= V[:k + 1, :, i].T @ h
                hn = float(np.linalg.norm(a))
                H[:k + 1, k, i] = h
                H[k + 1, k, i] = hn
                if hn > 0.0:
                    V[k + 1, :, i] = a / hn
                for j in range(k):                 # earlier rotations on the new column
                    t = cs[j, i] * H[j, k, i] + sn[j, i] * H[j + 1, k, i]
                    H[j + 1, k, i] = -sn[j, i] * H[j, k, i] + cs[j, i] * H[j + 1, k, i]
                    H[j, k, i] = t
                c, s_ = _givens(H[k, k, i], H[k + 1, k, i])
                cs[k, i], sn[k, i] = c, s_
                H[k, k, i] = c * H[k, k, i] + s_ * H[k + 1, k, i]
                H[k + 1, k, i] = 0.0
                rh[k + 1, i] = -s_ * rh[k, i]
                rh[k, i] = c * rh[k, i]
                steps[i] = k + 1
                col_it[i] += 1
                if abs(rh[k + 1, i]) / bn[i] <= tol or hn == 0.0:
                    act[i] = False
            k += 1
        for i in range(m):
            kk = int(steps[i])
            if kk == 0:
                continue
            y = np.zeros(kk)
            for j in range(kk - 1, -1, -1):        # R y = r̂ (upper triangular)
                y[j] = (rh[j, i] - H[j, j + 1:kk, i] @ y[j + 1:kk]) / H[j, j, i]
            X[:, i] += V[:kk, :, i].T @ y
    return GMRESResult(X=X, iterations=int(col_it.max()) if m else 0, cycles=cycles, col_iterations=col_it,
                       rel_residual=rel, status=status)


# ---------------------------------------------------------------------------
# Adjoint: gradients of a loss through X = A⁻¹B (not in the paper; the chain
# rule applied to the H² representation of Sec. 2)
# ---------------------------------------------------------------------------
def adjoint_grads(H: H2Matrix, Lam: np.ndarray, X: np.ndarray):
    """Given Λ = A⁻ᵀ ∂L/∂X and X, return ({(t.id, s.id): ∂L/∂S_b}, ∂L/∂σ).

    ∂L/∂A = −Λ Xᵀ; an admissible block is V_t S_b V_sᵀ, so
    ∂L/∂S_b = V_tᵀ(−Λ Xᵀ)|_{t̂×ŝ} V_s = −λ̂_t x̂_sᵀ with λ̂, x̂ the forward
    transformations of Λ and X; σ enters as σI, so ∂L/∂σ = −<Λ, X>_F.
    """
    Lam = np.asarray(Lam, dtype=np.float64).reshape(H.n, -1)
    X = np.asarray(X, dtype=np.float64).reshape(H.n, -1)
    lhat, xhat = {}, {}
    _forward(H, H.root, Lam, lhat)
    _forward(H, H.root, X, xhat)
    dS = {(b.t.id, b.s.id): -(lhat[b.t.id] @ xhat[b.s.id].T) for b in H.adm}
    return dS, -float(np.sum(Lam * X))


def set_coupling(H: H2Matrix, S_by_pair: dict):
    """Replace the coupling matrices S_b, keyed by (t.id, s.id)."""
    for b in H.adm:
        b.S = np.array(S_by_pair[(b.t.id, b.s.id)], dtype=np.float64)


# ---------------------------------------------------------------------------
# Preconditioned block CG (Sec. 5.1, Alg. "pcg block") with a block-Jacobi M
# ---------------------------------------------------------------------------
def block_jacobi(H: H2Matrix):
    """M = blockdiag over the leaves t of D_t = G_{(t,t)} + σI (the diagonal
    inadmissible blocks with the shift).  Returns a function r ↦ M⁻¹ r."""
    diag = {}
    for b in H.near:
        if b.t.id == b.s.id:
            D = b.G + H.sigma * np.eye(b.t.size)
            diag[b.t.id] = (b.t.idx, np.linalg.inv(D))

    def apply(R):
        R = np.asarray(R, dtype=np.float64)
        Z = np.zeros_like(R)
        for idx, Dinv in diag.values():
            Z[idx] = Dinv @ R[idx]
        return Z

    return apply


def block_pcg(apply_A, apply_Minv, B: np.ndarray, X0: np.ndarray | None = None, tol: float = 1e-8,
              max_iter: int = 10000) -> CGResult:
    """Alg. "pcg block": r = b - Ax, q = M⁻¹r, p = q (the listing's initial
    p ← r is read as p ← q, the standard start); per iteration a = Ap,
    β_i = <p_i, a_i>, α_i = <p_i, r_i>/β_i, x_i += α_i p_i, r_i -= α_i a_i,
    q = M⁻¹ r, γ_i = <a_i, q_i>/β_i, p_i = q_i - γ_i p_i.  Stopping as in
    block_cg (relative residual per column, converged columns frozen)."""
    B = np.asarray(B, dtype=np.float64)
    n, m = B.shape
    X = np.zeros((n, m), order="F") if X0 is None else np.array(X0, dtype=np.float64, order="F")
    R = np.asfortranarray(B - apply_A(X))
    Q = np.asfortranarray(apply_Minv(R))
    P = Q.copy(order="F")
    bn = np.linalg.norm(B, axis=0)
    bn[bn == 0.0] = 1.0
    done = np.linalg.norm(R, axis=0) / bn <= tol
    col_it = np.zeros(m, dtype=np.int64)
    it = 0
    status = "converged"
    while not done.all():
        if it >= max_iter:
            status = "noconverge"
            break
        Aq = np.asfortranarray(apply_A(P))
        it += 1
        alpha = np.zeros(m)
        beta = np.ones(m)
        for i in range(m):
            if done[i]:
                continue
            beta[i] = float(P[:, i] @ Aq[:, i])
            if not (beta[i] > 0.0) or not math.isfinite(beta[i]):
                status = "breakdown"
                break
            alpha[i] = float(P[:, i] @ R[:, i]) / beta[i]
            X[:, i] += alpha[i] * P[:, i]
            R[:, i] -= alpha[i] * Aq[:, i]
            col_it[i] = it
        if status == "breakdown":
            break
        Q = np.asfortranarray(apply_Minv(R))
        for i in range(m):
            if done[i]:
                continue
            gamma = float(Aq[:, i] @ Q[:, i]) / beta[i]
            P[:, i] = Q[:, i] - gamma * P[:, i]
            if np.linalg.norm(R[:, i]) / bn[i] <= tol:
                done[i] = True
    rel = np.linalg.norm(R, axis=0) / bn
    return CGResult(X=X, iterations=it, col_iterations=col_it, rel_residual=rel, status=status)
