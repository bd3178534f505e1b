// Host construction of the cluster tree, block tree and row-cluster block
// lists.  Compiled with -ffp-contract=off: the split and admissibility
// decisions are exact IEEE double expressions (no fused multiply-add), the
// same on x86-64 and aarch64.
#include "h2_tree.hpp"

#include <algorithm>
#include <cmath>
#include <utility>

namespace h2 {

namespace {

// Deeper trees only arise from pathological point sets (e.g. geometric
// sequences); they are rejected instead of overflowing the host stack.
constexpr int32_t kMaxDepth = 2048;

struct Builder {
    const double* pts;
    int32_t leaf_size;
    Tree& T;
    std::vector<int64_t> tmp;
    bool too_deep = false;

    // Sec. 2 Def. "Cluster tree".  Split rule: cut the longest side of the
    // tight bounding box (first maximum) at (lo + hi) * 0.5; coordinates <=
    // the cut go to son 0, both sons keep their relative order; if a side
    // would be empty the index range is halved.
    int32_t cluster(int64_t off, int64_t sz, int32_t level, int32_t parent) {
        const int32_t id = (int32_t)T.off.size();
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = pts[3 * T.perm[off] + d];
            hi[d] = lo[d];
        }
        for (int64_t i = off + 1; i < off + sz; ++i) {
            const double* p = pts + 3 * T.perm[i];
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], p[d]);
                hi[d] = std::max(hi[d], p[d]);
            }
        }
        T.off.push_back(off);
        T.size.push_back(sz);
        T.level.push_back(level);
        T.parent.push_back(parent);
        T.son0.push_back(-1);
        T.son1.push_back(-1);
        for (int d = 0; d < 3; ++d) T.box.push_back(lo[d]);
        for (int d = 0; d < 3; ++d) T.box.push_back(hi[d]);
        if (level > T.depth) T.depth = level;
        if (sz <= leaf_size) return id;
        if (level >= kMaxDepth) { too_deep = true; return id; }

        const double w0 = hi[0] - lo[0], w1 = hi[1] - lo[1], w2 = hi[2] - lo[2];
        int d = 0;
        double wd = w0;
        if (w1 > wd) { d = 1; wd = w1; }
        if (w2 > wd) { d = 2; }
        const double mid = (lo[d] + hi[d]) * 0.5;
        int64_t n0 = 0;
        for (int64_t i = off; i < off + sz; ++i)
            if (pts[3 * T.perm[i] + d] <= mid) ++n0;
        if (n0 > 0 && n0 < sz) {
            tmp.resize((size_t)sz);
            int64_t a = 0, b = n0;
            for (int64_t i = off; i < off + sz; ++i) {
                const int64_t p = T.perm[i];
                if (pts[3 * p + d] <= mid) tmp[a++] = p; else tmp[b++] = p;
            }
            std::copy(tmp.begin(), tmp.begin() + sz, T.perm.begin() + off);
        } else {
            n0 = sz / 2;
        }
        const int32_t s0 = cluster(off, n0, level + 1, id);
        const int32_t s1 = cluster(off + n0, sz - n0, level + 1, id);
        T.son0[id] = s0;
        T.son1[id] = s1;
        return id;
    }
};

inline double diam_of(const double* b) {
    const double w0 = b[3] - b[0], w1 = b[4] - b[1], w2 = b[5] - b[2];
    return std::sqrt((w0 * w0 + w1 * w1) + w2 * w2);
}

inline double dist_of(const double* t, const double* s) {
    double g[3];
    for (int d = 0; d < 3; ++d) {
        const double a = s[d] - t[3 + d];
        const double b = t[d] - s[3 + d];
        g[d] = std::max(std::max(a, b), 0.0);
    }
    return std::sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
}

// Eq. (admiss): max{diam t, diam s} <= eta·dist(t, s), dist > 0 required.
inline bool admissible(const Tree& T, int32_t t, int32_t s, double eta) {
    const double* bt = &T.box[6 * (size_t)t];
    const double* bs = &T.box[6 * (size_t)s];
    const double dd = dist_of(bt, bs);
    if (!(dd > 0.0)) return false;
    return std::max(diam_of(bt), diam_of(bs)) <= eta * dd;
}

struct BlockBuilder {
    const Tree& T;
    double eta;
    std::vector<std::pair<int32_t, int32_t>> adm, near;

    // Sec. 2 Def. "Block tree": a block is a leaf iff admissible or leaf × leaf;
    // otherwise its sons are {t}×sons(s), sons(t)×{s} or sons(t)×sons(s).
    void rec(int32_t t, int32_t s) {
        if (admissible(T, t, s, eta)) { adm.emplace_back(t, s); return; }
        const bool lt = T.is_leaf(t), ls = T.is_leaf(s);
        if (lt && ls) { near.emplace_back(t, s); return; }
        if (lt) {
            rec(t, T.son0[s]);
            rec(t, T.son1[s]);
        } else if (ls) {
            rec(T.son0[t], s);
            rec(T.son1[t], s);
        } else {
            rec(T.son0[t], T.son0[s]);
            rec(T.son0[t], T.son1[s]);
            rec(T.son1[t], T.son0[s]);
            rec(T.son1[t], T.son1[s]);
        }
    }
};

// Alg. "prepare_addeval": every leaf block goes to the list of its row
// cluster; a stable counting sort keeps the traversal order inside a list.
void to_csr(const std::vector<std::pair<int32_t, int32_t>>& blocks, int64_t nc,
            std::vector<int64_t>& rowptr, std::vector<int32_t>& col) {
    rowptr.assign((size_t)nc + 1, 0);
    for (auto& b : blocks) rowptr[(size_t)b.first + 1]++;
    for (int64_t i = 0; i < nc; ++i) rowptr[(size_t)i + 1] += rowptr[(size_t)i];
    std::vector<int64_t> pos(rowptr.begin(), rowptr.end() - 1);
    col.assign(blocks.size(), 0);
    for (auto& b : blocks) col[(size_t)pos[(size_t)b.first]++] = b.second;
}

}  // namespace

std::string build_tree(const double* pts, int64_t n, int32_t leaf_size, double eta, Tree& T) {
    if (n < 1) return "n must be >= 1";
    if (n > (int64_t)INT32_MAX) return "n must be < 2^31";
    if (leaf_size < 1) return "leaf_size must be >= 1";
    if (!(eta > 0.0) || !std::isfinite(eta)) return "eta must be finite and > 0";
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!std::isfinite(pts[i])) return "non-finite point coordinate";
    T = Tree();
    T.n = n;
    T.leaf_size = leaf_size;
    T.eta = eta;
    T.perm.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) T.perm[(size_t)i] = i;
    Builder B{pts, leaf_size, T, {}, false};
    B.cluster(0, n, 0, -1);
    if (B.too_deep) return "cluster tree deeper than 2048 levels (degenerate point set)";
    BlockBuilder BB{T, eta, {}, {}};
    BB.rec(0, 0);
    to_csr(BB.adm, T.n_clusters(), T.adm_rowptr, T.adm_col);
    to_csr(BB.near, T.n_clusters(), T.near_rowptr, T.near_col);
    return std::string();
}

}  // namespace h2
