// Host-side topology of the H² matrix: cluster tree, block tree and the
// per-row-cluster block lists (Sec. 2 Def. "Cluster tree", Def. "Block tree",
// Eq. (admiss); Sec. 3 Alg. "prepare_addeval").
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace h2 {

struct Tree {
    int64_t n = 0;
    int32_t leaf_size = 0;
    double eta = 0;
    int32_t depth = 0;
    // point index at each position of the pre-order cluster order
    std::vector<int64_t> perm;
    // clusters in pre-order
    std::vector<int64_t> off, size;
    std::vector<int32_t> level, parent, son0, son1;
    std::vector<double> box;  // 6 per cluster: lo xyz, hi xyz
    // leaf blocks grouped by row cluster (CSR over clusters)
    std::vector<int64_t> adm_rowptr;
    std::vector<int32_t> adm_col;
    std::vector<int64_t> near_rowptr;
    std::vector<int32_t> near_col;

    int64_t n_clusters() const { return (int64_t)off.size(); }
    int64_t n_adm() const { return (int64_t)adm_col.size(); }
    int64_t n_near() const { return (int64_t)near_col.size(); }
    bool is_leaf(int32_t c) const { return son0[c] < 0; }
};

// Builds the topology; returns an empty string on success, else an error text.
std::string build_tree(const double* pts, int64_t n, int32_t leaf_size, double eta, Tree& T);

}  // namespace h2
