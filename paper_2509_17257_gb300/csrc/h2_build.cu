// Device construction of the H² matrix entries (Sec. 2): leaf matrices V_t,
// transfer matrices E_t', coupling matrices S_b and nearfield blocks G_b from
// tensor Chebyshev interpolation of g(x, y) = exp(-|x - y| / length), plus the
// typed low-precision copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "h2_async.cuh"
#include "h2_internal.cuh"

namespace h2 {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Chebyshev points of the first kind on each side of the cluster box:
// node_{d,i} = center_d + half_d·cos((2i+1)π/(2q)); a side narrower than
// 1e-8 × the widest half-width is widened to that floor (1e-8 absolute for a
// box without extent).
__global__ void k_nodes(const double* __restrict__ box, int nc, int q, double* __restrict__ nodes) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const double* b = box + 6 * (size_t)c;
    double half[3], center[3];
    double hmax = 0.0;
    for (int d = 0; d < 3; ++d) {
        center[d] = (b[d] + b[3 + d]) * 0.5;
        half[d] = (b[3 + d] - b[d]) * 0.5;
        hmax = fmax(hmax, half[d]);
    }
    const double floor_h = hmax > 0.0 ? 1e-8 * hmax : 1e-8;
    for (int d = 0; d < 3; ++d) {
        const double h = fmax(half[d], floor_h);
        for (int i = 0; i < q; ++i)
            nodes[((size_t)c * 3 + d) * q + i] = center[d] + h * cos((2.0 * i + 1.0) * kPi / (2.0 * q));
    }
}

// Lagrange polynomial L_i of the q nodes nd at x.
__device__ __forceinline__ double lagrange(const double* nd, int q, int i, double x) {
    double v = 1.0;
    for (int j = 0; j < q; ++j)
        if (j != i) v *= (x - nd[j]) / (nd[i] - nd[j]);
    return v;
}

// L_ν(x) = L_{ν_x}(x_0) L_{ν_y}(x_1) L_{ν_z}(x_2), ν = ν_x + q ν_y + q² ν_z.
__device__ __forceinline__ double tensor_lagrange(const double* nodes3, int q, int nu, const double* x) {
    const int nx = nu % q, ny = (nu / q) % q, nz = nu / (q * q);
    return lagrange(nodes3, q, nx, x[0]) * lagrange(nodes3 + q, q, ny, x[1]) *
           lagrange(nodes3 + 2 * q, q, nz, x[2]);
}

__device__ __forceinline__ void tensor_node(const double* nodes3, int q, int mu, double* out) {
    out[0] = nodes3[mu % q];
    out[1] = nodes3[q + (mu / q) % q];
    out[2] = nodes3[2 * q + mu / (q * q)];
}

__device__ __forceinline__ double kernel_g(const double* x, const double* y, double inv_len) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    return exp(-sqrt((d0 * d0 + d1 * d1) + d2 * d2) * inv_len);
}

// The kernel of a build: exp(-r / length) (real), or the Helmholtz kernel of
// Sec. 2 regularised at r = 0, exp(i κ r) / (4π sqrt(r² + δ²)) (complex).
struct KernelSpec {
    int cplx;
    double inv_len, kappa, delta;
};

// g(x, y) into (re, im); im = 0 for the real kernel.
__device__ __forceinline__ void kernel_eval(const KernelSpec& ks, const double* x, const double* y, double* re,
                                            double* im) {
    if (!ks.cplx) {
        *re = kernel_g(x, y, ks.inv_len);
        *im = 0.0;
        return;
    }
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r2 = (d0 * d0 + d1 * d1) + d2 * d2;
    const double r = sqrt(r2);
    double sn, cs;
    sincos(ks.kappa * r, &sn, &cs);
    const double scale = 1.0 / (4.0 * 3.141592653589793 * sqrt(r2 + ks.delta * ks.delta));
    *re = cs * scale;
    *im = sn * scale;
}

// V_t[i, ν] = L_{t,ν}(x_i) for the points i of leaf t (one CTA per leaf).
__global__ void k_leaf_basis(const int32_t* __restrict__ leaves, const int32_t* __restrict__ cl_off,
                             const int32_t* __restrict__ cl_size, const double* __restrict__ pts,
                             const double* __restrict__ nodes, int q, double* __restrict__ V) {
    const int t = leaves[blockIdx.x];
    const int off = cl_off[t], sz = cl_size[t];
    const int k = q * q * q;
    const double* nd = nodes + (size_t)t * 3 * q;
    for (int e = threadIdx.x; e < sz * k; e += blockDim.x) {
        const int i = e / k, nu = e % k;
        V[(size_t)(off + i) * k + nu] = tensor_lagrange(nd, q, nu, pts + 3 * (size_t)(off + i));
    }
}

// E_{t'}[μ, ν] = L_{t,ν}(ξ_{t',μ}), t = parent of t' (one CTA per cluster).
__global__ void k_transfer(const int32_t* __restrict__ parent, const double* __restrict__ nodes, int q,
                           double* __restrict__ E) {
    const int c = blockIdx.x;
    const int p = parent[c];
    if (p < 0) return;
    const int k = q * q * q;
    const double* ndc = nodes + (size_t)c * 3 * q;
    const double* ndp = nodes + (size_t)p * 3 * q;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int mu = e / k, nu = e % k;
        double xi[3];
        tensor_node(ndc, q, mu, xi);
        E[(size_t)c * k * k + e] = tensor_lagrange(ndp, q, nu, xi);
    }
}

// The Kronecker factors of E_c (q = 4): F_a[μ][ν] = L_ν(ξ_{c,a,μ}), the 1-D Lagrange
// polynomials of the father's nodes on axis a at the son's nodes on that axis, so
// E_c[μ, ν] = F_x[μ_x][ν_x] F_y[μ_y][ν_y] F_z[μ_z][ν_z] (k_transfer's entries are
// these products); in FP32, 48 per cluster (zero for the root).
template <typename T>
__global__ void k_kron_factors(const int32_t* __restrict__ parent, const double* __restrict__ nodes, int64_t nc,
                               T* __restrict__ F) {
    const int q = 4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * 48; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / 48;
        const int r = (int)(e % 48), a = r / 16, mu = (r % 16) / 4, nu = r % 4;
        const int p = parent[c];
        F[e] = p < 0 ? T(0)
                     : (T)lagrange(nodes + ((size_t)p * 3 + a) * q, q, nu, nodes[((size_t)c * 3 + a) * q + mu]);
    }
}

// S_b[ν, μ] = g(ξ_{t,ν}, ξ_{s,μ}) for admissible blocks in list order (a complex
// kernel: imaginary parts in a second plane, n_adm·k² elements further on).
__global__ void k_coupling_entries(const int32_t* __restrict__ adm_row, const int32_t* __restrict__ adm_col,
                                   int64_t n_adm, const double* __restrict__ nodes, int q, KernelSpec ks,
                                   double* __restrict__ S) {
    const int k = q * q * q;
    for (int64_t j = blockIdx.x; j < n_adm; j += gridDim.x) {
        const double* nt = nodes + (size_t)adm_row[j] * 3 * q;
        const double* ns = nodes + (size_t)adm_col[j] * 3 * q;
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int nu = e / k, mu = e % k;
            double a[3], b[3];
            tensor_node(nt, q, nu, a);
            tensor_node(ns, q, mu, b);
            double re, im;
            kernel_eval(ks, a, b, &re, &im);
            S[(size_t)j * k * k + e] = re;
            if (ks.cplx) S[((size_t)n_adm + j) * k * k + e] = im;
        }
    }
}

// FP32 tensor nodes for the matrix-free coupling: nodes4[c·KP + ν] = ξ_{c,ν}
// (x, y, z, 0) for ν < k, zero for k <= ν < KP.
__global__ void k_nodes4(const double* __restrict__ nodes, int64_t nc, int q, int KP, float4* __restrict__ nodes4) {
    const int k = q * q * q;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * KP; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / KP;
        const int nu = (int)(e % KP);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (nu < k) {
            double x[3];
            tensor_node(nodes + (size_t)c * 3 * q, q, nu, x);
            v = make_float4((float)x[0], (float)x[1], (float)x[2], 0.f);
        }
        nodes4[e] = v;
    }
}

// G_b[i, j] = g(x_i, x_j) for inadmissible blocks (a complex kernel: imaginary
// parts in a second plane, im_off = nnz_near elements further on).
__global__ void k_near_entries(const int32_t* __restrict__ near_row, const int32_t* __restrict__ near_col,
                               const int64_t* __restrict__ near_off, int64_t n_near,
                               const int32_t* __restrict__ cl_off, const int32_t* __restrict__ cl_size,
                               const double* __restrict__ pts, KernelSpec ks, int64_t im_off,
                               double* __restrict__ G) {
    for (int64_t j = blockIdx.x; j < n_near; j += gridDim.x) {
        const int t = near_row[j], s = near_col[j];
        const int ot = cl_off[t], nt = cl_size[t], os = cl_off[s], ns = cl_size[s];
        double* g = G + near_off[j];
        for (int e = threadIdx.x; e < nt * ns; e += blockDim.x) {
            const int r = e / ns, c = e % ns;
            double re, im;
            kernel_eval(ks, pts + 3 * (size_t)(ot + r), pts + 3 * (size_t)(os + c), &re, &im);
            g[e] = re;
            if (ks.cplx) g[im_off + e] = im;
        }
    }
}

__global__ void k_cast_f32(const double* __restrict__ in, float* __restrict__ out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

}  // namespace

int cast_f32(const double* src, float* dst, int64_t count, cudaStream_t st) {
    if (count <= 0) return 0;
    k_cast_f32<<<1216, 256, 0, st>>>(src, dst, count);
    H2_LAUNCH_CHECK();
    return 0;
}

namespace {

template <typename T>
int upload(h2_matrix* A, T** dst, const std::vector<T>& src, cudaStream_t st) {
    void* p = nullptr;
    const size_t bytes = src.size() * sizeof(T);
    int rc = device_alloc(A, &p, bytes > 0 ? bytes : sizeof(T));
    if (rc) return rc;
    if (bytes) H2_CUDA_TRY(cudaMemcpyAsync(p, src.data(), bytes, cudaMemcpyHostToDevice, st));
    *dst = (T*)p;
    return 0;
}

// Et[c][μ][ν] = E[c][ν][μ] in FP32, rows of kEtLd floats (k×kEtLd per cluster, zero
// past column k): one bulk copy lands a cluster's block with the row stride the
// downward pass's warp-MMA fragment loads want (≡ 8 mod 32, no bank conflicts).
__global__ void k_transpose_f32(const double* __restrict__ E, float* __restrict__ Et, int64_t nc, int k) {
    const int64_t per = (int64_t)k * kEtLd;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * per; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / per;
        const int q = (int)((e % per) / kEtLd), r = (int)(e % kEtLd);
        Et[e] = r < k ? (float)E[c * k * k + (int64_t)r * k + q] : 0.f;
    }
}

// Lays out a work list sorted by decreasing cost for a kernel whose CTA b
// takes positions b, b + G, b + 2G, ...: round r of G items goes to the CTAs
// in order for even r and in reverse for odd r (the last, partial round in
// order), so no CTA takes the largest item of every round.
void snake_order(std::vector<TcItem>& v, int G) {
    const size_t n = v.size();
    if (G < 2 || n <= (size_t)G) return;
    std::vector<TcItem> out(n);
    for (size_t i = 0; i < n; ++i) {
        const size_t r = i / G, j = i % G;
        const bool full = (r + 1) * G <= n;
        out[r * G + ((r & 1) && full ? G - 1 - j : j)] = v[i];
    }
    v.swap(out);
}

// A term's fixed cost in the balance of the tensor-core work lists, in units of
// tile elements (a full 64×64 tile adds a third of it): a term's copies and
// hand-offs take nearly as long whatever its tile's size.
constexpr int64_t kTermFixedCost = 3 * 64 * 64;

// Lays the items out for a launch of G CTAs, where position r·G + c runs on
// CTA c: the items, largest first, are dealt round by round, each round's
// largest to the CTA with the least work so far; the CTAs that receive an item
// in the last, partial round are numbered first.
template <class Cost>
void balance_order(std::vector<TcItem>& v, Cost cost, int G) {
    const size_t n = v.size();
    if (G < 2 || n <= (size_t)G) return;
    std::stable_sort(v.begin(), v.end(), [&](const TcItem& a, const TcItem& b) { return cost(a) > cost(b); });
    const size_t rounds = (n + G - 1) / G;
    std::vector<int64_t> load(G, 0);
    std::vector<std::vector<TcItem>> per(G);
    std::vector<int> idx(G);
    for (size_t r = 0; r < rounds; ++r) {
        for (int c = 0; c < G; ++c) idx[c] = c;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return load[a] < load[b]; });
        const size_t i0 = r * G, i1 = std::min(n, i0 + G);
        for (size_t i = i0; i < i1; ++i) {
            const int c = idx[i - i0];
            per[c].push_back(v[i]);
            load[c] += cost(v[i]);
        }
    }
    std::vector<int> order;
    for (int c = 0; c < G; ++c)
        if (per[c].size() == rounds) order.push_back(c);
    for (int c = 0; c < G; ++c)
        if (per[c].size() < rounds) order.push_back(c);
    std::vector<TcItem> out;
    out.reserve(n);
    for (size_t r = 0; r < rounds; ++r)
        for (int c = 0; c < G; ++c)
            if (per[order[c]].size() > r) out.push_back(per[order[c]][r]);
    v.swap(out);
}

int cast_copy(h2_matrix* A, const double* src, void** dst, int64_t count, cudaStream_t st) {
    int rc = device_alloc(A, dst, (size_t)(count > 0 ? count : 1) * sizeof(float));
    if (rc) return rc;
    if (count > 0) {
        k_cast_f32<<<1216, 256, 0, st>>>(src, (float*)*dst, count);
        H2_LAUNCH_CHECK();
    }
    return 0;
}

}  // namespace

// Schedule of the subtree-owning downward pass.  The tree is cut at level Ls:
// the cut clusters (level Ls, and leaves above it) are the tasks.  A task
// recomputes ŷ of the clusters on the path from the root to its cut cluster
// t (ŷ_a += E_a ŷ_parent(a) in path order; the sum is the same for every
// task that shares the path), then walks the subtree of t in pre-order (the
// contiguous cluster range t .. t + |subtree| - 1).  No task reads what
// another task writes, so the pass needs no synchronisation between CTAs.
// Stack entries 0 and 1 alternate along the path; a node of relative depth
// d >= 1 below t keeps its ŷ in entry d + 1 (its father's is in entry d, or
// in the entry holding t's for d = 1).  Ls is the shallowest level with at
// least `target` tasks whose subtrees are at most kMaxSubDepth deep and whose
// step lists fit kDownMaxSteps (at the deepest level every task is a leaf's
// path, at most depth + 1 steps).
void down_schedule(const Tree& T, int target, std::vector<int32_t>& task_ptr, std::vector<DownStep>& steps,
                   int32_t& ntasks, int32_t& entries) {
    constexpr int kMaxSubDepth = 6;
    const int64_t nc = T.n_clusters();
    task_ptr.assign(1, 0);
    steps.clear();
    ntasks = 0;
    entries = 2;
    if (nc <= 1) return;
    std::vector<int64_t> nsub(nc, 1);  // subtree sizes (pre-order: sons follow their father)
    std::vector<int32_t> hsub(nc, 0);  // subtree heights
    for (int64_t c = nc - 1; c >= 1; --c) {
        nsub[T.parent[c]] += nsub[c];
        hsub[T.parent[c]] = std::max(hsub[T.parent[c]], hsub[c] + 1);
    }
    int Ls = T.depth;
    for (int l = 1; l <= T.depth; ++l) {
        int64_t count = 0, size = 0;
        int32_t h = 0;
        for (int64_t c = 0; c < nc; ++c)
            if (T.level[c] == l || (T.level[c] < l && T.is_leaf((int32_t)c))) {
                ++count;
                h = std::max(h, hsub[c]);
                size = std::max(size, nsub[c]);
            }
        // a task has 1 + l + (subtree size - 1) steps
        if (count >= target && h <= kMaxSubDepth && l + size <= kDownMaxSteps) { Ls = l; break; }
    }
    std::vector<int32_t> cut;
    for (int64_t c = 0; c < nc; ++c)
        if (T.level[c] == Ls || (T.level[c] < Ls && T.level[c] > 0 && T.is_leaf((int32_t)c))) cut.push_back((int32_t)c);
    std::vector<std::vector<DownStep>> task_steps(cut.size());
    int32_t dmax = 0;
    for (size_t i = 0; i < cut.size(); ++i) {
        const int32_t t = cut[i];
        std::vector<DownStep>& v = task_steps[i];
        std::vector<int32_t> path;
        for (int32_t a = t; T.parent[a] >= 0; a = T.parent[a]) path.push_back(a);
        std::reverse(path.begin(), path.end());
        v.push_back(DownStep{0, -1, 0, kDownLoad});  // the root's ŷ is final after the coupling phase
        int cur = 0;
        for (int32_t a : path) {
            v.push_back(DownStep{a, cur, cur ^ 1, (a == t && T.is_leaf(a)) ? kDownStore : 0});
            cur ^= 1;
        }
        for (int64_t c = t + 1; c < t + nsub[t]; ++c) {
            const int32_t d = T.level[c] - T.level[t];
            dmax = std::max(dmax, d);
            v.push_back(DownStep{(int32_t)c, d == 1 ? cur : d, d + 1, T.is_leaf((int32_t)c) ? kDownStore : 0});
        }
    }
    // longest tasks first: CTAs claim them in this order
    std::vector<size_t> order(cut.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return task_steps[a].size() > task_steps[b].size(); });
    for (size_t i : order) {
        steps.insert(steps.end(), task_steps[i].begin(), task_steps[i].end());
        task_ptr.push_back((int32_t)steps.size());
    }
    ntasks = (int32_t)cut.size();
    entries = 2 + dmax;
}

// Schedule of the subtree-owning upward pass.  The tree is cut at level Lu as
// for the downward pass; a task evaluates the subtree of its cut cluster t in
// post-order (sons before their father), keeping each x̂ in a shared-memory
// stack entry until its father has used it (the father's x̂ then takes its
// first son's entry), so no step waits for another CTA.  Entries come from a
// free list (a subtree of height h needs h + 1); at least three exist, for the
// climb above the cut (own x̂, the brother's contribution, the father's x̂).  Lu is the shallowest
// level with at least `target` tasks whose step lists fit kUpMaxSteps and
// whose stacks fit kUpMaxEntries.
void up_schedule(const Tree& T, int target, std::vector<int32_t>& task_ptr, std::vector<UpStep>& steps,
                 int32_t& ntasks, int32_t& entries, int32_t* cut_level) {
    const int64_t nc = T.n_clusters();
    task_ptr.assign(1, 0);
    steps.clear();
    ntasks = 0;
    entries = 3;
    if (cut_level) *cut_level = 0;
    if (nc < 1) return;
    std::vector<int64_t> nsub(nc, 1);
    for (int64_t c = nc - 1; c >= 1; --c) nsub[T.parent[c]] += nsub[c];
    std::vector<int32_t> leaf_pos(nc, -1);  // position among the leaves in cluster order
    for (int64_t c = 0, lp = 0; c < nc; ++c)
        if (T.is_leaf((int32_t)c)) leaf_pos[c] = (int32_t)lp++;
    // post-order step list of the subtree of t and the number of entries it needs
    auto build = [&](int32_t t, std::vector<UpStep>& v) {
        v.clear();
        std::vector<int32_t> free_list;
        int32_t next_new = 0, used = 0, max_used = 0;
        auto take = [&]() {
            int32_t e;
            if (!free_list.empty()) { e = free_list.back(); free_list.pop_back(); }
            else e = next_new++;
            max_used = std::max(max_used, ++used);
            return e;
        };
        auto give = [&](int32_t e) { free_list.push_back(e); --used; };
        // iterative post-order over the pre-order range of t
        std::vector<std::pair<int32_t, int>> st{{t, 0}};
        std::vector<int32_t> entry_of;  // entry holding x̂ of the cluster at the same stack position
        std::vector<int32_t> done;      // x̂ entries waiting for their father, in order
        while (!st.empty()) {
            auto& [c, state] = st.back();
            if (!T.is_leaf(c) && state == 0) {
                state = 1;
                st.push_back({T.son0[c], 0});
                continue;
            }
            if (!T.is_leaf(c) && state == 1) {
                state = 2;
                st.push_back({T.son1[c], 0});
                continue;
            }
            if (T.is_leaf(c)) {
                const int32_t e = take();
                v.push_back(UpStep{c, -1, leaf_pos[c], e});
                done.push_back(e);
            } else {
                // the father's x̂ replaces its first son's (the kernel waits for
                // every read of both sons before it writes)
                const int32_t e1 = done.back(); done.pop_back();
                const int32_t e0 = done.back(); done.pop_back();
                v.push_back(UpStep{c, e0, e1, e0});
                give(e1);
                done.push_back(e0);
            }
            st.pop_back();
        }
        return std::max<int32_t>(max_used, 3);
    };
    std::vector<UpStep> tmp;
    int Lu = T.depth;
    for (int l = 0; l <= T.depth; ++l) {
        int64_t count = 0, size = 0;
        int32_t ent = 0;
        for (int64_t c = 0; c < nc; ++c)
            if (T.level[c] == l || (T.level[c] < l && T.is_leaf((int32_t)c))) {
                ++count;
                size = std::max(size, nsub[c]);
                ent = std::max(ent, build((int32_t)c, tmp));
            }
        if ((count >= target || l == T.depth) && size <= kUpMaxSteps && ent <= kUpMaxEntries) { Lu = l; break; }
    }
    if (cut_level) *cut_level = Lu;
    std::vector<std::vector<UpStep>> task_steps;
    for (int64_t c = 0; c < nc; ++c)
        if (T.level[c] == Lu || (T.level[c] < Lu && T.is_leaf((int32_t)c))) {
            task_steps.emplace_back();
            entries = std::max(entries, build((int32_t)c, task_steps.back()));
        }
    // longest tasks first
    std::vector<size_t> order(task_steps.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return task_steps[a].size() > task_steps[b].size(); });
    for (size_t i : order) {
        steps.insert(steps.end(), task_steps[i].begin(), task_steps[i].end());
        task_ptr.push_back((int32_t)steps.size());
    }
    ntasks = (int32_t)task_steps.size();
}

int build_device(h2_matrix* A, const double* pts_host, uint32_t precisions, cudaStream_t st) {
    const Tree& T = A->T;
    const int64_t n = A->n, nc = A->nc;
    const int q = A->q, k = A->k;

    // ---- host-side schedule ----
    std::vector<int32_t> perm32(n), off32(nc), size32(nc), parent32(nc), son0(nc), son1(nc);
    for (int64_t i = 0; i < n; ++i) perm32[i] = (int32_t)T.perm[i];
    for (int64_t c = 0; c < nc; ++c) {
        off32[c] = (int32_t)T.off[c];
        size32[c] = (int32_t)T.size[c];
        parent32[c] = T.parent[c];
        son0[c] = T.son0[c];
        son1[c] = T.son1[c];
    }
    const int L = A->depth;
    A->up_ptr.assign(L + 2, 0);
    A->down_ptr.assign(L + 2, 0);
    std::vector<int32_t> up_list, down_list;
    for (int l = 0; l <= L; ++l) {
        A->up_ptr[l] = (int64_t)up_list.size();
        A->down_ptr[l] = (int64_t)down_list.size();
        for (int64_t c = 0; c < nc; ++c) {
            if (T.level[c] != l) continue;
            if (!T.is_leaf((int32_t)c)) up_list.push_back((int32_t)c);
            if (T.parent[c] >= 0) down_list.push_back((int32_t)c);
        }
    }
    A->up_ptr[L + 1] = (int64_t)up_list.size();
    A->down_ptr[L + 1] = (int64_t)down_list.size();
    if (k <= 64) {
        // gather, forward transformation (one launch), coupling, downward pass (one launch), leaf phase
        A->launches_per_product = A->down_ptr[L + 1] > 0 ? 5 : 4;
    } else {
        A->launches_per_product = 4;  // gather, leaf forward, coupling, leaf backward, + one launch per level
        for (int l = 0; l <= L; ++l) {
            A->launches_per_product += A->up_ptr[l + 1] > A->up_ptr[l];
            A->launches_per_product += A->down_ptr[l + 1] > A->down_ptr[l];
        }
    }
    A->leaves.clear();
    std::vector<int32_t> leaf_pos(nc, -1);
    for (int64_t c = 0; c < nc; ++c)
        if (T.is_leaf((int32_t)c)) {
            leaf_pos[c] = (int32_t)A->leaves.size();
            A->leaves.push_back((int32_t)c);
        }

    // admissible lists by row cluster, and the transposed lists by column cluster
    std::vector<int32_t> adm_rowptr(nc + 1), adm_col(A->n_adm), adm_row(A->n_adm);
    for (int64_t c = 0; c <= nc; ++c) adm_rowptr[c] = (int32_t)T.adm_rowptr[c];
    for (int64_t t = 0; t < nc; ++t)
        for (int64_t j = T.adm_rowptr[t]; j < T.adm_rowptr[t + 1]; ++j) {
            adm_col[j] = T.adm_col[j];
            adm_row[j] = (int32_t)t;
        }
    std::vector<int32_t> admT_rowptr(nc + 1, 0), admT_row(A->n_adm), admT_blk(A->n_adm);
    for (int64_t j = 0; j < A->n_adm; ++j) admT_rowptr[adm_col[j] + 1]++;
    for (int64_t c = 0; c < nc; ++c) admT_rowptr[c + 1] += admT_rowptr[c];
    {
        std::vector<int32_t> pos(admT_rowptr.begin(), admT_rowptr.end() - 1);
        for (int64_t j = 0; j < A->n_adm; ++j) {
            const int32_t p = pos[adm_col[j]]++;
            admT_row[p] = adm_row[j];
            admT_blk[p] = (int32_t)j;
        }
    }
    // nearfield lists by row leaf position, offsets of the dense blocks
    const int64_t NL = (int64_t)A->leaves.size();
    std::vector<int32_t> near_ptr(NL + 1, 0), near_col(A->n_near), near_row(A->n_near);
    std::vector<int64_t> near_off(A->n_near);
    int64_t acc = 0;
    {
        int64_t j = 0;
        for (int64_t lp = 0; lp < NL; ++lp) {
            const int32_t t = A->leaves[lp];
            near_ptr[lp] = (int32_t)j;
            for (int64_t e = T.near_rowptr[t]; e < T.near_rowptr[t + 1]; ++e, ++j) {
                near_col[j] = T.near_col[e];
                near_row[j] = t;
                near_off[j] = acc;
                acc += T.size[t] * T.size[T.near_col[e]];
            }
        }
        near_ptr[NL] = (int32_t)j;
    }
    A->nnz_near = acc;
    // offset of the diagonal block G_(t,t) of every leaf (always inadmissible: dist = 0)
    std::vector<int64_t> near_diag(NL, -1);
    for (int64_t lp = 0; lp < NL; ++lp)
        for (int64_t j = near_ptr[lp]; j < near_ptr[lp + 1]; ++j)
            if (near_col[j] == A->leaves[lp]) near_diag[lp] = near_off[j];
    for (int64_t lp = 0; lp < NL; ++lp)
        if (near_diag[lp] < 0) { set_error("internal: leaf without a diagonal nearfield block"); return H2_E_CUDA; }
    std::vector<int32_t> nearT_ptr(NL + 1, 0), nearT_row(A->n_near), nearT_blk(A->n_near);
    for (int64_t j = 0; j < A->n_near; ++j) nearT_ptr[leaf_pos[near_col[j]] + 1]++;
    for (int64_t lp = 0; lp < NL; ++lp) nearT_ptr[lp + 1] += nearT_ptr[lp];
    {
        std::vector<int32_t> pos(nearT_ptr.begin(), nearT_ptr.end() - 1);
        for (int64_t j = 0; j < A->n_near; ++j) {
            const int32_t p = pos[leaf_pos[near_col[j]]]++;
            nearT_row[p] = near_row[j];
            nearT_blk[p] = (int32_t)j;
        }
    }
    std::vector<double> pts_p((size_t)n * 3);
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) pts_p[3 * i + d] = pts_host[3 * T.perm[i] + d];

    int rc = 0;
#define UP(dst, src) if ((rc = upload(A, &(dst), (src), st))) return rc
    UP(A->d_perm, perm32);
    UP(A->d_cl_off, off32);
    UP(A->d_cl_size, size32);
    UP(A->d_parent, parent32);
    UP(A->d_son0, son0);
    UP(A->d_son1, son1);
    UP(A->d_leaves, A->leaves);
    UP(A->d_up_list, up_list);
    UP(A->d_down_list, down_list);
    {
        std::vector<int32_t> task_ptr;
        std::vector<DownStep> dsteps;
        down_schedule(T, A->down_target, task_ptr, dsteps, A->dn_ntasks, A->dn_entries);
        UP(A->d_dn_task_ptr, task_ptr);
        UP(A->d_dn_steps, dsteps);
        std::vector<UpStep> usteps;
        up_schedule(T, A->up_target, task_ptr, usteps, A->up_ntasks, A->up_entries, &A->up_cut);
        UP(A->d_up_task_ptr, task_ptr);
        UP(A->d_up_steps, usteps);
    }
    UP(A->d_adm_rowptr, adm_rowptr);
    UP(A->d_adm_col, adm_col);
    UP(A->d_adm_row, adm_row);
    UP(A->d_admT_rowptr, admT_rowptr);
    UP(A->d_admT_row, admT_row);
    UP(A->d_admT_blk, admT_blk);
    UP(A->d_near_ptr, near_ptr);
    UP(A->d_near_col, near_col);
    UP(A->d_near_row, near_row);
    UP(A->d_near_off, near_off);
    UP(A->d_near_diag, near_diag);
    UP(A->d_nearT_ptr, nearT_ptr);
    UP(A->d_nearT_row, nearT_row);
    UP(A->d_nearT_blk, nearT_blk);
    UP(A->d_pts, pts_p);
    double* d_box = nullptr;
    UP(d_box, T.box);
#undef UP

    // ---- entries in FP64 ----
    void* p = nullptr;
    if ((rc = device_alloc(A, &p, (size_t)nc * 3 * q * sizeof(double)))) return rc;
    A->d_nodes = (double*)p;
    k_nodes<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(d_box, (int)nc, q, A->d_nodes);
    H2_LAUNCH_CHECK();

    const size_t bV = (size_t)n * k * sizeof(double);
    const size_t bE = (size_t)nc * k * k * sizeof(double);
    const size_t planes = A->cplx ? 2 : 1;  // complex S and nearfield: real and imaginary planes
    const size_t bS = planes * (size_t)A->n_adm * k * k * sizeof(double);
    const size_t bN = planes * (size_t)A->nnz_near * sizeof(double);
    if ((rc = device_alloc(A, &A->f64.V, bV))) return rc;
    if ((rc = device_alloc(A, &A->f64.E, bE))) return rc;
    if ((rc = device_alloc(A, &A->f64.S, bS > 0 ? bS : 8))) return rc;
    if ((rc = device_alloc(A, &A->f64.Near, bN > 0 ? bN : 8))) return rc;
    A->f64.bytes = (int64_t)(bV + bE + bS + bN);
    H2_CUDA_TRY(cudaMemsetAsync(A->f64.E, 0, bE, st));

    const KernelSpec ks{A->cplx ? 1 : 0, 1.0 / A->length, A->kappa, A->delta};
    k_leaf_basis<<<(unsigned)NL, 256, 0, st>>>(A->d_leaves, A->d_cl_off, A->d_cl_size, A->d_pts, A->d_nodes,
                                               q, (double*)A->f64.V);
    H2_LAUNCH_CHECK();
    k_transfer<<<(unsigned)nc, 256, 0, st>>>(A->d_parent, A->d_nodes, q, (double*)A->f64.E);
    H2_LAUNCH_CHECK();
    if (A->n_adm > 0) {
        const unsigned g = (unsigned)std::min<int64_t>(A->n_adm, 152 * 64);
        k_coupling_entries<<<g, 256, 0, st>>>(A->d_adm_row, A->d_adm_col, A->n_adm, A->d_nodes, q, ks,
                                              (double*)A->f64.S);
        H2_LAUNCH_CHECK();
    }
    if (A->n_near > 0) {
        const unsigned g = (unsigned)std::min<int64_t>(A->n_near, 152 * 64);
        k_near_entries<<<g, 256, 0, st>>>(A->d_near_row, A->d_near_col, A->d_near_off, A->n_near, A->d_cl_off,
                                          A->d_cl_size, A->d_pts, ks, A->nnz_near, (double*)A->f64.Near);
        H2_LAUNCH_CHECK();
    }
    A->f64.built = true;
    // q = 4: the Kronecker factors of the transfer matrices, E_c = F_z ⊗ F_y ⊗ F_x
    const unsigned gkf = (unsigned)std::min<int64_t>((nc * 48 + 255) / 256, 152 * 8);
    if (q == 4) {
        if ((rc = device_alloc(A, &A->f64.kron, (size_t)nc * 48 * sizeof(double)))) return rc;
        k_kron_factors<double><<<gkf, 256, 0, st>>>(A->d_parent, A->d_nodes, nc, (double*)A->f64.kron);
        H2_LAUNCH_CHECK();
        if ((rc = device_alloc(A, &A->f32.kron, (size_t)nc * 48 * sizeof(float)))) return rc;
        k_kron_factors<float><<<gkf, 256, 0, st>>>(A->d_parent, A->d_nodes, nc, (float*)A->f32.kron);
        H2_LAUNCH_CHECK();
    }

    if (precisions & (1u << H2_F32)) {
        if ((rc = cast_copy(A, (const double*)A->f64.V, &A->f32.V, (int64_t)n * k, st))) return rc;
        if ((rc = cast_copy(A, (const double*)A->f64.E, &A->f32.E, nc * k * k, st))) return rc;
        if ((rc = cast_copy(A, (const double*)A->f64.S, &A->f32.S, (int64_t)planes * A->n_adm * k * k, st)))
            return rc;
        if ((rc = cast_copy(A, (const double*)A->f64.Near, &A->f32.Near, (int64_t)planes * A->nnz_near, st)))
            return rc;
        A->f32.bytes = A->f64.bytes / 2;
        A->f32.built = true;
    }
    if (!A->err_host) {
        H2_CUDA_TRY(cudaHostAlloc((void**)&A->err_host, sizeof(int), cudaHostAllocMapped));
        *A->err_host = 0;
        H2_CUDA_TRY(cudaHostGetDevicePointer((void**)&A->err_dev, A->err_host, 0));
    }
    const bool want_bf16 = (precisions & (1u << H2_BF16)) != 0;
    // the complex product takes the TF32 tiles of both planes of S and G (no BF16, no
    // transfer-pass or matrix-free tiles)
    const bool want_tf32 = (precisions & (1u << H2_F32)) != 0 && k <= 64;
    if (want_bf16 && A->cplx) {
        set_error("a complex kernel has no BF16 product");
        return H2_E_UNSUPPORTED;
    }
    if (want_bf16 && k > 64) {
        set_error("the BF16 tensor-core product supports q <= 4 (k <= 64)");
        return H2_E_UNSUPPORTED;
    }
    if (want_bf16 || want_tf32) {
        if (!A->f32.built) {
            // the tensor-core products run their transfer passes on the FP32 copies of V and E
            if ((rc = cast_copy(A, (const double*)A->f64.V, &A->f32.V, (int64_t)n * k, st))) return rc;
            if ((rc = cast_copy(A, (const double*)A->f64.E, &A->f32.E, nc * k * k, st))) return rc;
        }
        if (k % 8 == 0 && k <= 64) {
            // transposed transfer matrices for the subtree-owning downward pass
            if ((rc = device_alloc(A, &A->f32.Et, (size_t)nc * k * kEtLd * sizeof(float)))) return rc;
            k_transpose_f32<<<1216, 256, 0, st>>>((const double*)A->f64.E, (float*)A->f32.Et, nc, k);
            H2_LAUNCH_CHECK();
        }

        if ((rc = build_tc(A, want_bf16, want_tf32, st))) return rc;
    }
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

// ---- the transfer passes of Alg. "forward/backward" on the tensor cores ----
// Every cluster is one item of a work list whose terms are matrix tile ×
// activation tile, as in the coupling phase:
//   upward:   x̂_t = V_tᵀ X|_t̂ (a leaf: V_tᵀ × the leaf's X tile) or
//             x̂_t = E_s0ᵀ x̂_s0 + E_s1ᵀ x̂_s1 (the sons' x̂ tiles);
//   downward: ŷ_s = I·ŷ_s + E_s ŷ_t: the coupling result enters through an
//             identity tile (the coupling writes its results as split tiles,
//             and zero tiles for clusters without couplings), t the father
//             (the root has no father term).
// Items are ordered so that every item's terms read tiles of earlier items;
// the kernel keeps every CTA's items in that order, and a term marked
// kTermWait waits for its source's ready flag.  With A the upward pass shares
// one launch with the coupling phase (f1: all upward items, then the coupling
// items) and the downward pass one with the leaf phase (f2: all downward
// items, then the leaf items, each with its nearfield terms first).
struct FlowTiles {
    std::vector<int64_t> et_off, vt_off, e_off;  // Eᵀ_c, V_tᵀ (by leaf position), E_c
    int64_t id_off = 0;                          // the identity tile
    std::vector<float> ident;
    int64_t n_et = 0, n_vt = 0, n_e = 0;
};

void flow_tiles(h2_matrix* A, std::vector<TcPackTile>& tiles, int64_t& off, FlowTiles& ft) {
    const Tree& T = A->T;
    const TcData& D = A->tc;
    const int k = A->k, KP = D.KP, NP = D.NP;
    const int64_t nc = A->nc, NL = (int64_t)A->leaves.size();
    auto add = [&](int64_t src, int n, int kk, int ld, int np, int kp, int tr) {
        tiles.push_back(TcPackTile{src, off, n, kk, ld, np, kp, tr});
        const int64_t b = (int64_t)np * kp * 2;
        off += b;
        return off - b;
    };
    ft.et_off.assign(nc, -1);
    ft.e_off.assign(nc, -1);
    ft.vt_off.assign(NL, -1);
    for (int64_t c = 1; c < nc; ++c) ft.et_off[c] = add(c * k * k, k, k, k, NP, KP, 1);  // row ν, column μ
    ft.n_et = nc - 1;
    for (int64_t lp = 0; lp < NL; ++lp) {                                              // row ν, column p
        const int32_t t = A->leaves[lp];
        ft.vt_off[lp] = add(T.off[t] * k, k, (int)T.size[t], k, NP, round16((int)T.size[t]), 1);
    }
    ft.n_vt = NL;
    for (int64_t c = 1; c < nc; ++c) ft.e_off[c] = add(c * k * k, k, k, k, NP, KP, 0);  // row μ, column ν
    ft.n_e = nc - 1;
    ft.id_off = off;
    ft.ident.assign((size_t)NP * KP, 0.f);
    for (int r = 0; r < k; ++r) ft.ident[(size_t)(cm_off(r, r, KP, 4) / 4)] = 1.f;
    off += (int64_t)NP * KP * 2;
}

// Items with their sort keys, dealt in snake order over the CTAs within each key.
struct KeyedItem {
    int32_t key;
    TcItem it;
};
void order_by_key(std::vector<KeyedItem>& v, std::vector<TcItem>& out) {
    std::stable_sort(v.begin(), v.end(), [](const KeyedItem& a, const KeyedItem& b) { return a.key < b.key; });
    out.clear();
    std::vector<TcItem> group;
    for (size_t i = 0; i < v.size();) {
        size_t j = i;
        group.clear();
        while (j < v.size() && v[j].key == v[i].key) group.push_back(v[j++].it);
        snake_order(group, kTcGrid);
        out.insert(out.end(), group.begin(), group.end());
        i = j;
    }
}

// Items of several work lists merged by key (snake order over the CTAs within a
// key), for the multi-system launches of h2_batch_matmul.
void merge_by_key(const std::vector<int32_t>& keys, const std::vector<TcItem>& items, std::vector<TcItem>& out) {
    std::vector<KeyedItem> v(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) v[i] = KeyedItem{keys[i], items[i]};
    order_by_key(v, out);
}

int flow_lists(h2_matrix* A, const FlowTiles& ft, const std::vector<int64_t>& s_off,
               const std::vector<int64_t>& v_off, const std::vector<int64_t>& g_off,
               const std::vector<int64_t>& xkoff, cudaStream_t st) {
    TcData& D = A->tc;
    const Tree& T = A->T;
    const int KP = D.KP, NP = D.NP;
    const int64_t nc = A->nc, NL = (int64_t)A->leaves.size();
    std::vector<int32_t> leaf_pos(nc, -1);
    for (int64_t lp = 0; lp < NL; ++lp) leaf_pos[A->leaves[lp]] = (int32_t)lp;
    std::vector<int32_t> height(nc, 0);
    for (int64_t c = nc - 1; c >= 0; --c)  // pre-order: sons follow their father
        if (!T.is_leaf((int32_t)c)) height[c] = 1 + std::max(height[T.son0[c]], height[T.son1[c]]);
    const int16_t kAct0Wait = (int16_t)(0 | kTermWait);
    auto np_role = [](int np, int32_t role) { return (int32_t)(np | (role << 16)); };
    // upward items (activations: act0 the x̂ tiles of this launch, act1 the X tiles)
    std::vector<TcTerm> up_terms;
    std::vector<KeyedItem> up_k;
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t e0 = (int32_t)up_terms.size();
        if (T.is_leaf((int32_t)c)) {
            const int32_t lp = leaf_pos[c];
            up_terms.push_back(TcTerm{ft.vt_off[lp], (int32_t)xkoff[lp], (int16_t)round16((int)T.size[c]), (int16_t)1});
        } else {
            for (int32_t s : {T.son0[c], T.son1[c]})
                up_terms.push_back(TcTerm{ft.et_off[s], (int32_t)((int64_t)s * KP), (int16_t)KP, kAct0Wait});
        }
        up_k.push_back(KeyedItem{height[c], TcItem{(int32_t)c, e0, (int32_t)up_terms.size(),
                                                       np_role(NP, kRoleTransfer)}});
    }
    // downward items (act0 the ŷ tiles of this launch, act1 the coupling results)
    std::vector<TcTerm> dn_terms;
    std::vector<KeyedItem> dn_k;
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t e0 = (int32_t)dn_terms.size();
        dn_terms.push_back(TcTerm{ft.id_off, (int32_t)((int64_t)c * KP), (int16_t)KP, (int16_t)1});
        if (c != 0)
            dn_terms.push_back(TcTerm{ft.e_off[c], (int32_t)((int64_t)T.parent[c] * KP), (int16_t)KP, kAct0Wait});
        dn_k.push_back(KeyedItem{T.level[c], TcItem{(int32_t)c, e0, (int32_t)dn_terms.size(),
                                                        np_role(NP, kRoleTransfer)}});
    }
    std::vector<TcItem> up_items, dn_items;
    order_by_key(up_k, up_items);
    order_by_key(dn_k, dn_items);
    // f1: every CTA takes its upward items first (they form the dependency chain),
    // then its coupling items, those whose sources are ready earliest first (keys
    // from kLateKey on; heights and levels stay below it, trees being shallower)
    constexpr int32_t kLateKey = 4096;
    std::vector<TcTerm> f1_terms = up_terms;
    std::vector<KeyedItem> f1_k = up_k;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t j0 = T.adm_rowptr[c], j1 = T.adm_rowptr[c + 1];
        if (j1 == j0) continue;
        const int32_t e0 = (int32_t)f1_terms.size();
        int32_t hmax = 0;
        for (int64_t j = j0; j < j1; ++j) {
            const int32_t sc = T.adm_col[j];
            hmax = std::max(hmax, height[sc]);
            f1_terms.push_back(TcTerm{s_off[j], (int32_t)((int64_t)sc * KP), (int16_t)KP, kAct0Wait});
        }
        f1_k.push_back(KeyedItem{kLateKey + hmax, TcItem{(int32_t)c, e0, (int32_t)f1_terms.size(),
                                                      np_role(NP, kRoleCoupling)}});
    }
    // f2: the downward items first, then the leaf items, shallow leaves (ready first)
    // first; a leaf item's nearfield terms come first (act2, the X tiles; no wait),
    // V_t ŷ_t last (act0, waits)
    std::vector<TcTerm> f2_terms = dn_terms;
    std::vector<KeyedItem> f2_k = dn_k;
    {
        int64_t j = 0;
        for (int64_t lp = 0; lp < NL; ++lp) {
            const int32_t t = A->leaves[lp];
            const int32_t e0 = (int32_t)f2_terms.size();
            for (int64_t e = T.near_rowptr[t]; e < T.near_rowptr[t + 1]; ++e, ++j) {
                const int32_t sc = T.near_col[e];
                f2_terms.push_back(TcTerm{g_off[j], (int32_t)xkoff[leaf_pos[sc]],
                                          (int16_t)round16((int)T.size[sc]), (int16_t)2});
            }
            f2_terms.push_back(TcTerm{v_off[lp], (int32_t)((int64_t)t * KP), (int16_t)KP, kAct0Wait});
            f2_k.push_back(KeyedItem{kLateKey + T.level[t], TcItem{(int32_t)lp, e0, (int32_t)f2_terms.size(),
                                                                np_role(round16((int)T.size[t]), kRoleLeaf)}});
        }
    }
    D.f1_keys.clear();
    D.f1_host.clear();
    for (const auto& ki : f1_k) { D.f1_keys.push_back(ki.key); D.f1_host.push_back(ki.it); }
    D.f2_keys.clear();
    D.f2_host.clear();
    for (const auto& ki : f2_k) { D.f2_keys.push_back(ki.key); D.f2_host.push_back(ki.it); }
    std::vector<TcItem> f1_items, f2_items;
    order_by_key(f1_k, f1_items);
    order_by_key(f2_k, f2_items);
    D.up_nitems = (int)up_items.size();
    D.dn_nitems = (int)dn_items.size();
    D.f1_nitems = (int)f1_items.size();
    D.f2_nitems = (int)f2_items.size();
    int rc = 0;
#define UP(dst, src) if ((rc = upload(A, &(dst), (src), st))) return rc
    UP(D.up_items, up_items);
    UP(D.up_terms, up_terms);
    UP(D.dn_items, dn_items);
    UP(D.dn_terms, dn_terms);
    UP(D.f1_items, f1_items);
    UP(D.f1_terms, f1_terms);
    UP(D.f2_items, f2_items);
    UP(D.f2_terms, f2_terms);
#undef UP
    D.flow = true;
    return 0;
}

// The coupling launch of the hybrid upward pass (k_tc_gemm<4, KIND>).  The CUDA-core
// subtree pass (k_up_own without its climb) computes every cluster at or below
// the cut level up_cut (and the leaves above it); the clusters above the cut,
// x̂_t = E_s0ᵀ x̂_s0 + E_s1ᵀ x̂_s1 (Alg. "forward/backward"), become transfer items
// of the coupling launch, each writing its split tile and ready flag.  A term
// whose source is above the cut waits for that flag: a transfer item for its
// sons, a coupling item for its source cluster.  Keys order the list so that
// every wait points to a strictly smaller key (each CTA takes its items in list
// order, so the item with the smallest unfinished key can always proceed):
//   transfer item at height h above the cut (h = 1 for fathers of task roots): 2h - 1;
//   coupling item reading only clusters at or below the cut: key 2r for the
//     rounds r < H between two heights, the smallest items first and about
//     kHybridRoundTerms terms per CTA per round (the time a transfer item takes
//     to become readable), the rest key 2H;
//   coupling item reading a cluster above the cut: key 2H too if its highest
//     source is at height H - 3 or below, else 2H + 1.
// Each of the last two groups is dealt largest first.  The transfer items thus
// run early, a few microseconds apart, and the coupling items that read them
// come with the bulk of the coupling work, those reading the top of the tree
// last.
constexpr int kHybridRoundTerms = 16;  // H2_HYBRID_ROUND_TERMS overrides it (1..64)
// The product takes the hybrid upward pass by default when the coupling work
// that reads no cluster above the cut gives every CTA at least this many terms
// per height above the cut: then the chain of transfer items (a few
// microseconds per height) runs under that work instead of after it.
constexpr int kHybridTermsPerHeight = 12;

int hybrid_lists(h2_matrix* A, cudaStream_t st) {
    TcData& D = A->tc;
    const Tree& T = A->T;
    const int KP = D.KP, NP = D.NP;
    const int64_t nc = A->nc;
    D.hybrid = false;
    D.hybrid_bf16 = false;
    D.h_default = false;
    // FP32 lists: the Eᵀ tiles of the tensor-core transfer passes; BF16 lists: the
    // split BF16 Eᵀ tiles
    const bool f32 = D.flow && D.et_off_host.size() == (size_t)nc;
    const bool b16 = D.ebh_off_host.size() == (size_t)nc && D.ebl_off_host.size() == (size_t)nc;
    if ((!f32 && !b16) || D.s_off_host.size() != (size_t)A->n_adm) return 0;
    // height above the cut: 0 for clusters at or below it and for leaves above it
    std::vector<int32_t> h(nc, 0);
    int32_t H = 0;
    for (int64_t c = nc - 1; c >= 0; --c)  // pre-order: sons follow their father
        if (!T.is_leaf((int32_t)c) && T.level[c] < A->up_cut) {
            h[c] = 1 + std::max(h[T.son0[c]], h[T.son1[c]]);
            H = std::max(H, h[c]);
        }
    const int16_t kWait = (int16_t)(0 | kTermWait);
    auto np_role = [](int np, int32_t role) { return (int32_t)(np | (role << 16)); };
    int round_terms = kHybridRoundTerms;
    if (const char* e = getenv("H2_HYBRID_ROUND_TERMS")) round_terms = std::min(64, std::max(1, atoi(e)));
    int64_t free_terms = 0;
    // The list of one kind: transfer terms E_sᵀ x̂_s from the tiles et (and, BF16, the
    // remainder tiles etl as a second term per son).
    auto build = [&](const std::vector<int64_t>& et, const std::vector<int64_t>* etl, TcItem** d_items,
                     TcTerm** d_terms, int* n_items) -> int {
        std::vector<TcTerm> terms;
        std::vector<KeyedItem> keyed;
        for (int64_t c = 0; c < nc; ++c) {
            if (h[c] == 0) continue;
            const int32_t e0 = (int32_t)terms.size();
            for (int32_t s : {T.son0[c], T.son1[c]}) {
                const int16_t w = h[s] > 0 ? kWait : (int16_t)0;
                terms.push_back(TcTerm{et[s], (int32_t)((int64_t)s * KP), (int16_t)KP, w});
                if (etl) terms.push_back(TcTerm{(*etl)[s], (int32_t)((int64_t)s * KP), (int16_t)KP, w});
            }
            keyed.push_back(
                KeyedItem{2 * h[c] - 1, TcItem{(int32_t)c, e0, (int32_t)terms.size(), np_role(NP, kRoleTransfer)}});
        }
        struct Free {
            int64_t cost;
            TcItem it;
            int32_t hs;  // largest height above the cut among the sources
        };
        std::vector<Free> free_items, late;
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t j0 = T.adm_rowptr[c], j1 = T.adm_rowptr[c + 1];
            if (j1 == j0) continue;
            const int32_t e0 = (int32_t)terms.size();
            int32_t hs = 0;
            for (int64_t j = j0; j < j1; ++j) {
                const int32_t sc = T.adm_col[j];
                hs = std::max(hs, h[sc]);
                terms.push_back(TcTerm{D.s_off_host[j], (int32_t)((int64_t)sc * KP), (int16_t)KP,
                                       h[sc] > 0 ? kWait : (int16_t)0});
            }
            const TcItem it{(int32_t)c, e0, (int32_t)terms.size(), np_role(NP, 0)};
            if (hs > 0) late.push_back(Free{j1 - j0, it, hs});
            else free_items.push_back(Free{j1 - j0, it, 0});
        }
        // smallest first into the rounds, each round up to kHybridRoundTerms terms per CTA
        std::stable_sort(free_items.begin(), free_items.end(),
                         [](const Free& a, const Free& b) { return a.cost < b.cost; });
        const int64_t budget = (int64_t)round_terms * kTcGrid;
        size_t i = 0;
        for (int32_t r = 0; r < H; ++r) {
            int64_t used = 0;
            while (i < free_items.size() && used + free_items[i].cost <= budget) {
                used += free_items[i].cost;
                keyed.push_back(KeyedItem{2 * r, free_items[i++].it});
            }
        }
        // the rest, and the coupling items that read clusters above the cut: largest
        // first (snake-dealt within the key)
        std::vector<Free> rest(free_items.begin() + (long)i, free_items.end());
        rest.insert(rest.end(), late.begin(), late.end());
        std::stable_sort(rest.begin(), rest.end(), [](const Free& a, const Free& b) { return a.cost > b.cost; });
        for (const Free& f : rest) keyed.push_back(KeyedItem{f.hs > H - 3 ? 2 * H + 1 : 2 * H, f.it});
        std::vector<TcItem> items;
        order_by_key(keyed, items);
        release_allocation(A, *d_items);
        release_allocation(A, *d_terms);
        *d_items = nullptr;
        *d_terms = nullptr;
        int rc = 0;
        if ((rc = upload(A, d_items, items, st)) || (rc = upload(A, d_terms, terms, st))) return rc;
        *n_items = (int)items.size();
        free_terms = 0;
        for (const Free& f : free_items) free_terms += f.cost;
        return 0;
    };
    int rc = 0;
    if (f32) {
        if ((rc = build(D.et_off_host, nullptr, &D.h_items, &D.h_terms, &D.h_nitems))) return rc;
        D.hybrid = true;
    }
    if (b16) {
        if ((rc = build(D.ebh_off_host, &D.ebl_off_host, &D.hb_items, &D.hb_terms, &D.hb_nitems))) return rc;
        D.hybrid_bf16 = true;
    }
    D.h_nabove = 0;
    for (int64_t c = 0; c < nc; ++c) D.h_nabove += h[c] > 0;
    D.h_default = free_terms >= (int64_t)kHybridTermsPerHeight * H * kTcGrid;
    return 0;
}

// Core-matrix copies of S, V and G for the tensor cores (BF16 and/or FP32 for
// the split-TF32 product), and the schedules of the two tcgen05 kernels
// (coupling over row clusters, leaf phase over row leaves).
int build_tc(h2_matrix* A, bool bf16, bool tf32, cudaStream_t st) {
    const Tree& T = A->T;
    const int k = A->k;
    const int KP = round16(k), NP = round16(k);
    TcData& D = A->tc;
    D.KP = KP;
    D.NP = NP;
    const int64_t nc = A->nc, NL = (int64_t)A->leaves.size();
    std::vector<int32_t> leaf_pos(nc, -1);
    for (int64_t lp = 0; lp < NL; ++lp) leaf_pos[A->leaves[lp]] = (int32_t)lp;

    // ---- tiles ----
    std::vector<TcPackTile> tiles;
    tiles.reserve(A->n_adm + NL + A->n_near);
    int64_t off = 0;
    auto add = [&](int64_t src, int n, int kk, int ld, int np, int kp) {
        tiles.push_back(TcPackTile{src, off, n, kk, ld, np, kp, 0});
        const int64_t b = (int64_t)np * kp * 2;
        off += b;
        return off - b;
    };
    std::vector<int64_t> s_off(A->n_adm), v_off(NL), g_off(A->n_near);
    // a complex matrix: the imaginary planes' tiles follow the real ones (S at
    // n_adm·k², G at nnz_near elements further on in the FP64 arrays)
    std::vector<int64_t> si_off(A->cplx ? A->n_adm : 0), gi_off(A->cplx ? A->n_near : 0);
    for (int64_t j = 0; j < A->n_adm; ++j) s_off[j] = add(j * k * k, k, k, k, NP, KP);
    if (A->cplx)
        for (int64_t j = 0; j < A->n_adm; ++j) si_off[j] = add((A->n_adm + j) * k * k, k, k, k, NP, KP);
    const int64_t nS = (int64_t)tiles.size();
    for (int64_t lp = 0; lp < NL; ++lp) {
        const int32_t t = A->leaves[lp];
        const int nt = (int)T.size[t];
        v_off[lp] = add(T.off[t] * k, nt, k, k, round16(nt), KP);
    }
    const int64_t nV = (int64_t)tiles.size() - nS;
    // nearfield blocks in the order of the row-leaf lists (the FP64 Near array order)
    std::vector<int32_t> l_np(NL);
    std::vector<int64_t> near_src(A->n_near);
    {
        int64_t j = 0, acc = 0;
        for (int64_t lp = 0; lp < NL; ++lp) {
            const int32_t t = A->leaves[lp];
            const int nt = (int)T.size[t];
            l_np[lp] = round16(nt);
            for (int64_t e = T.near_rowptr[t]; e < T.near_rowptr[t + 1]; ++e, ++j) {
                const int ns = (int)T.size[T.near_col[e]];
                near_src[j] = acc;
                g_off[j] = add(acc, nt, ns, ns, round16(nt), round16(ns));
                acc += (int64_t)nt * ns;
            }
        }
        if (A->cplx) {
            int64_t jj = 0;
            for (int64_t lp = 0; lp < NL; ++lp) {
                const int nt = (int)T.size[A->leaves[lp]];
                for (int64_t e = T.near_rowptr[A->leaves[lp]]; e < T.near_rowptr[A->leaves[lp] + 1]; ++e, ++jj) {
                    const int ns = (int)T.size[T.near_col[e]];
                    gi_off[jj] = add(near_src[jj] + A->nnz_near, nt, ns, ns, round16(nt), round16(ns));
                }
            }
        }
    }
    const int64_t nG = (int64_t)tiles.size() - nS - nV;
    D.bytes = off;  // BF16 bytes; the FP32 copy is twice that
    // the transfer passes' tiles follow in the FP32 copy only
    FlowTiles ft;
    const bool flow = tf32 && k <= 64 && T.leaf_size <= 64 && !A->cplx;
    if (flow) flow_tiles(A, tiles, off, ft);
    const int64_t off32 = off;
    // the BF16 hybrid lists' Eᵀ_c tiles (high part, then remainder) after the BF16
    // tiles of S, V and G, in the BF16 copy only
    std::vector<TcPackTile> tilesE;
    int64_t off16 = D.bytes;
    D.ebh_off_host.clear();
    D.ebl_off_host.clear();
    if (bf16 && k <= 64 && T.leaf_size <= 64 && !A->cplx && nc > 1) {
        D.ebh_off_host.assign(nc, -1);
        D.ebl_off_host.assign(nc, -1);
        for (int64_t c = 1; c < nc; ++c)
            for (int lo = 0; lo < 2; ++lo) {
                (lo ? D.ebl_off_host : D.ebh_off_host)[c] = off16;
                tilesE.push_back(TcPackTile{c * k * k, off16, k, k, k, NP, KP, 1 | (lo << 1)});  // row ν, column μ
                off16 += (int64_t)NP * KP * 2;
            }
    }
    int rc = 0;
    TcPackTile* d_tiles = nullptr;
    if ((rc = upload(A, &d_tiles, tiles, st))) return rc;
    D.d_tiles = d_tiles;
    D.n_s_tiles = nS;
    for (int es = 2; es <= 4; es += 2) {
        if ((es == 2 && !bf16) || (es == 4 && !tf32)) continue;
        void* pm = nullptr;
        const int64_t total = es == 4 ? off32 : off16;
        if ((rc = device_alloc(A, &pm, (size_t)std::max<int64_t>(total * (es / 2), 128)))) return rc;
        uint8_t* dst = (uint8_t*)pm;
        if ((rc = launch_pack_tiles(d_tiles, nS, (const double*)A->f64.S, dst, es, st))) return rc;
        if ((rc = launch_pack_tiles(d_tiles + nS, nV, (const double*)A->f64.V, dst, es, st))) return rc;
        if ((rc = launch_pack_tiles(d_tiles + nS + nV, nG, (const double*)A->f64.Near, dst, es, st))) return rc;
        if (es == 4 && flow) {
            const int64_t f0 = nS + nV + nG;
            if ((rc = launch_pack_tiles(d_tiles + f0, ft.n_et, (const double*)A->f64.E, dst, es, st))) return rc;
            if ((rc = launch_pack_tiles(d_tiles + f0 + ft.n_et, ft.n_vt, (const double*)A->f64.V, dst, es, st)))
                return rc;
            if ((rc = launch_pack_tiles(d_tiles + f0 + ft.n_et + ft.n_vt, ft.n_e, (const double*)A->f64.E, dst, es, st)))
                return rc;
            H2_CUDA_TRY(cudaMemcpyAsync(dst + ft.id_off * 2, ft.ident.data(), ft.ident.size() * sizeof(float),
                                        cudaMemcpyHostToDevice, st));
        }
        if (es == 2 && !tilesE.empty()) {
            TcPackTile* d_tilesE = nullptr;
            if ((rc = upload(A, &d_tilesE, tilesE, st))) return rc;
            if ((rc = launch_pack_tiles(d_tilesE, (int64_t)tilesE.size(), (const double*)A->f64.E, dst, es, st)))
                return rc;
        }
        if (es == 2) D.mat = dst; else D.mat32 = dst;
    }
    D.has_bf16 = bf16;
    D.has_tf32 = tf32;
    if (tf32 && !A->cplx) {
        if ((rc = device_alloc(A, (void**)&D.nodes4, (size_t)nc * KP * sizeof(float4)))) return rc;
        const unsigned g = (unsigned)std::min<int64_t>((nc * KP + 255) / 256, 152 * 16);
        k_nodes4<<<g, 256, 0, st>>>(A->d_nodes, nc, A->q, KP, D.nodes4);
        H2_LAUNCH_CHECK();
    }

    // ---- coupling schedule: outputs = clusters with at least one admissible block ----
    std::vector<int32_t> c_zero;
    std::vector<TcItem> c_items;
    // a complex matrix: two terms per block, S_re·x̂_s and S_im·(i·x̂_s)
    const int tpb = A->cplx ? 2 : 1;
    std::vector<TcTerm> c_terms(tpb * A->n_adm);
    for (int64_t j = 0; j < A->n_adm; ++j) {
        const int32_t ak = (int32_t)((int64_t)T.adm_col[j] * KP);
        c_terms[tpb * j] = TcTerm{s_off[j], ak, (int16_t)KP, (int16_t)0};
        if (A->cplx) c_terms[2 * j + 1] = TcTerm{si_off[j], ak, (int16_t)KP, kTermImag};
    }
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t e0 = (int32_t)T.adm_rowptr[c], e1 = (int32_t)T.adm_rowptr[c + 1];
        if (e1 > e0) c_items.push_back(TcItem{(int32_t)c, tpb * e0, tpb * e1, NP});
        else c_zero.push_back((int32_t)c);
    }
    // longest lists first, each to the CTA with the least work so far
    balance_order(c_items, [](const TcItem& a) { return (int64_t)(a.e1 - a.e0); }, kTcGrid);
    // ---- leaf schedule: outputs = leaf positions; terms = V_t ŷ_t, then G_b X|_ŝ ----
    std::vector<int64_t> xkoff(NL + 1, 0);
    std::vector<int32_t> leaf_base(NL), leaf_kdim(NL);
    for (int64_t lp = 0; lp < NL; ++lp) {
        const int32_t t = A->leaves[lp];
        leaf_base[lp] = (int32_t)T.off[t];
        leaf_kdim[lp] = (int32_t)T.size[t];
        xkoff[lp + 1] = xkoff[lp] + round16((int)T.size[t]);
    }
    std::vector<TcItem> l_items(NL);
    std::vector<TcTerm> l_terms;
    std::vector<int64_t> l_cost(NL, 0);
    {
        int64_t j = 0;
        for (int64_t lp = 0; lp < NL; ++lp) {
            const int32_t t = A->leaves[lp];
            const int32_t e0 = (int32_t)l_terms.size();
            l_terms.push_back(TcTerm{v_off[lp], (int32_t)((int64_t)t * KP), (int16_t)KP, (int16_t)1});
            l_cost[lp] += kTermFixedCost + (int64_t)l_np[lp] * KP;
            for (int64_t e = T.near_rowptr[t]; e < T.near_rowptr[t + 1]; ++e, ++j) {
                const int32_t sc = T.near_col[e];
                const int kps = round16((int)T.size[sc]);
                l_terms.push_back(TcTerm{g_off[j], (int32_t)xkoff[leaf_pos[sc]], (int16_t)kps, (int16_t)0});
                l_cost[lp] += kTermFixedCost + (int64_t)l_np[lp] * kps;
                if (A->cplx) {  // G_im·(i·X|_ŝ)
                    l_terms.push_back(TcTerm{gi_off[j], (int32_t)xkoff[leaf_pos[sc]], (int16_t)kps, kTermImag});
                    l_cost[lp] += kTermFixedCost + (int64_t)l_np[lp] * kps;
                }
            }
            l_items[lp] = TcItem{(int32_t)lp, e0, (int32_t)l_terms.size(), l_np[lp]};
        }
    }
    balance_order(l_items, [&](const TcItem& a) { return l_cost[a.id]; }, kTcGrid);
    D.s_off_host = s_off;
    D.et_off_host.clear();
    if (flow) {
        if ((rc = flow_lists(A, ft, s_off, v_off, g_off, xkoff, st))) return rc;
        D.et_off_host = ft.et_off;
    }
    if ((rc = hybrid_lists(A, st))) return rc;
    D.xk_total = xkoff[NL];
    D.c_nitems = (int)c_items.size();
    D.c_nzero = (int)c_zero.size();
    D.l_nitems = (int)NL;
#define UP(dst, src) if ((rc = upload(A, &(dst), (src), st))) return rc
    UP(D.c_items, c_items);
    UP(D.c_terms, c_terms);
    UP(D.c_zero, c_zero);
    UP(D.l_items, l_items);
    UP(D.l_terms, l_terms);
    UP(D.xkoff, xkoff);
    UP(D.leaf_base, leaf_base);
    UP(D.leaf_kdim, leaf_kdim);
#undef UP
    D.built = true;
    return 0;
}

// The tensor-core product with Aᵀ (Alg. "H2_mvm" with the roles of row and
// column clusters swapped: ŷ_s = Σ_{b=(t,s)} S_bᵀ x̂_t, and y|_ŝ += G_bᵀ x|_t̂ on
// the inadmissible blocks; W = V, so the transfer passes are those of A).  Its
// tiles hold S_bᵀ, V_t and G_bᵀ in the layout of build_tc (V repeated so one
// base pointer serves the leaf phase), its coupling list runs over column
// clusters and its leaf list over column leaves.
int build_tc_transposed(h2_matrix* A, cudaStream_t st) {
    TcData& D = A->tc;
    if (D.t_built) return 0;
    if (!D.built) { set_error("tensor-core tiles not built"); return H2_E_UNSUPPORTED; }
    const Tree& T = A->T;
    const int k = A->k, KP = D.KP, NP = D.NP;
    const int64_t nc = A->nc, NL = (int64_t)A->leaves.size();
    std::vector<int32_t> leaf_pos(nc, -1);
    for (int64_t lp = 0; lp < NL; ++lp) leaf_pos[A->leaves[lp]] = (int32_t)lp;
    std::vector<TcPackTile> tiles;
    tiles.reserve(A->n_adm + NL + A->n_near);
    int64_t off = 0;
    auto add = [&](int64_t src, int n, int kk, int ld, int np, int kp, int tr) {
        tiles.push_back(TcPackTile{src, off, n, kk, ld, np, kp, tr});
        const int64_t b = (int64_t)np * kp * 2;
        off += b;
        return off - b;
    };
    // S_bᵀ: tile row μ, contraction ν (S_b[ν][μ] at j·k² + ν·k + μ)
    std::vector<int64_t> s_off(A->n_adm), v_off(NL), g_off(A->n_near);
    for (int64_t j = 0; j < A->n_adm; ++j) s_off[j] = add(j * k * k, k, k, k, NP, KP, 1);
    const int64_t nS = (int64_t)tiles.size();
    for (int64_t lp = 0; lp < NL; ++lp) {
        const int32_t t = A->leaves[lp];
        v_off[lp] = add(T.off[t] * k, (int)T.size[t], k, k, round16((int)T.size[t]), KP, 0);
    }
    // G_bᵀ for b = (t, s): tile row j of ŝ, contraction over t̂ (G_b[i][j] at near_src + i·|ŝ| + j)
    std::vector<int32_t> near_t(A->n_near), near_s(A->n_near);
    {
        int64_t j = 0, acc = 0;
        for (int64_t lp = 0; lp < NL; ++lp) {
            const int32_t t = A->leaves[lp];
            const int nt = (int)T.size[t];
            for (int64_t e = T.near_rowptr[t]; e < T.near_rowptr[t + 1]; ++e, ++j) {
                const int32_t sc = T.near_col[e];
                const int ns = (int)T.size[sc];
                g_off[j] = add(acc, ns, nt, ns, round16(ns), round16(nt), 1);
                near_t[j] = t;
                near_s[j] = sc;
                acc += (int64_t)nt * ns;
            }
        }
    }
    int rc = 0;
    TcPackTile* d_tiles = nullptr;
    if ((rc = upload(A, &d_tiles, tiles, st))) return rc;
    D.d_tilesT = d_tiles;
    const int64_t nV = NL, nG = A->n_near;
    for (int es = 2; es <= 4; es += 2) {
        if ((es == 2 && !D.has_bf16) || (es == 4 && !D.has_tf32)) continue;
        void* pm = nullptr;
        if ((rc = device_alloc(A, &pm, (size_t)std::max<int64_t>(off * (es / 2), 128)))) return rc;
        uint8_t* dst = (uint8_t*)pm;
        if ((rc = launch_pack_tiles(d_tiles, nS, (const double*)A->f64.S, dst, es, st))) return rc;
        if ((rc = launch_pack_tiles(d_tiles + nS, nV, (const double*)A->f64.V, dst, es, st))) return rc;
        if ((rc = launch_pack_tiles(d_tiles + nS + nV, nG, (const double*)A->f64.Near, dst, es, st))) return rc;
        if (es == 2) D.matT = dst; else D.matT32 = dst;
    }
    // ---- coupling list over column clusters: item s, terms S_bᵀ x̂_t ----
    std::vector<std::vector<int64_t>> by_col(nc);
    for (int64_t t = 0; t < nc; ++t)
        for (int64_t j = T.adm_rowptr[t]; j < T.adm_rowptr[t + 1]; ++j) by_col[T.adm_col[j]].push_back(j);
    std::vector<TcItem> c_items;
    std::vector<TcTerm> c_terms;
    std::vector<int32_t> c_zero;
    c_terms.reserve(A->n_adm);
    {
        // the row cluster of every admissible block
        std::vector<int32_t> row_of(A->n_adm);
        for (int64_t t = 0; t < nc; ++t)
            for (int64_t j = T.adm_rowptr[t]; j < T.adm_rowptr[t + 1]; ++j) row_of[j] = (int32_t)t;
        for (int64_t sc = 0; sc < nc; ++sc) {
            const int32_t e0 = (int32_t)c_terms.size();
            for (int64_t j : by_col[sc])
                c_terms.push_back(TcTerm{s_off[j], (int32_t)((int64_t)row_of[j] * KP), (int16_t)KP, (int16_t)0});
            const int32_t e1 = (int32_t)c_terms.size();
            if (e1 > e0) c_items.push_back(TcItem{(int32_t)sc, e0, e1, NP});
            else c_zero.push_back((int32_t)sc);
        }
    }
    balance_order(c_items, [](const TcItem& a) { return (int64_t)(a.e1 - a.e0); }, kTcGrid);
    // ---- leaf list over column leaves: item s, terms V_s ŷ_s, then G_bᵀ x|_t̂ ----
    std::vector<int64_t> xkoff(NL + 1, 0);
    for (int64_t lp = 0; lp < NL; ++lp) xkoff[lp + 1] = xkoff[lp] + round16((int)T.size[A->leaves[lp]]);
    std::vector<std::vector<int64_t>> near_by_col(NL);
    for (int64_t j = 0; j < A->n_near; ++j) near_by_col[leaf_pos[near_s[j]]].push_back(j);
    std::vector<TcItem> l_items(NL);
    std::vector<TcTerm> l_terms;
    std::vector<int64_t> l_cost(NL, 0);
    for (int64_t lp = 0; lp < NL; ++lp) {
        const int32_t sc = A->leaves[lp];
        const int np = round16((int)T.size[sc]);
        const int32_t e0 = (int32_t)l_terms.size();
        l_terms.push_back(TcTerm{v_off[lp], (int32_t)((int64_t)sc * KP), (int16_t)KP, (int16_t)1});
        l_cost[lp] += kTermFixedCost + (int64_t)np * KP;
        for (int64_t j : near_by_col[lp]) {
            const int32_t t = near_t[j];
            const int kpt = round16((int)T.size[t]);
            l_terms.push_back(TcTerm{g_off[j], (int32_t)xkoff[leaf_pos[t]], (int16_t)kpt, (int16_t)0});
            l_cost[lp] += kTermFixedCost + (int64_t)np * kpt;
        }
        l_items[lp] = TcItem{(int32_t)lp, e0, (int32_t)l_terms.size(), np};
    }
    balance_order(l_items, [&](const TcItem& a) { return l_cost[a.id]; }, kTcGrid);
    D.ct_nitems = (int)c_items.size();
    D.ct_nzero = (int)c_zero.size();
    D.lt_nitems = (int)NL;
#define UP(dst, src) if ((rc = upload(A, &(dst), (src), st))) return rc
    UP(D.ct_items, c_items);
    UP(D.ct_terms, c_terms);
    UP(D.ct_zero, c_zero);
    UP(D.lt_items, l_items);
    UP(D.lt_terms, l_terms);
#undef UP
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    D.t_built = true;
    return 0;
}

// New cut targets for the subtree schedules of the CUDA-core transfer passes
// (h2_autotune): the schedules are rebuilt and replace the old ones, which are
// freed once the stream has finished with them.
int set_transfer_targets(h2_matrix* A, int up_target, int down_target, cudaStream_t st) {
    if (up_target == A->up_target && down_target == A->down_target) return 0;
    std::vector<int32_t> dptr, uptr;
    std::vector<DownStep> dsteps;
    std::vector<UpStep> usteps;
    int32_t dn_ntasks = 0, dn_entries = 0, up_ntasks = 0, up_entries = 0;
    down_schedule(A->T, down_target, dptr, dsteps, dn_ntasks, dn_entries);
    int32_t up_cut = 0;
    up_schedule(A->T, up_target, uptr, usteps, up_ntasks, up_entries, &up_cut);
    if (up_entries > kUpMaxEntries || dn_entries > 8) {
        set_error("transfer-pass schedule needs more stack entries than the kernels hold");
        return H2_E_UNSUPPORTED;
    }
    int32_t *d_dptr = nullptr, *d_uptr = nullptr;
    DownStep* d_ds = nullptr;
    UpStep* d_us = nullptr;
    int rc = 0;
    if ((rc = upload(A, &d_dptr, dptr, st)) || (rc = upload(A, &d_ds, dsteps, st)) || (rc = upload(A, &d_uptr, uptr, st)) ||
        (rc = upload(A, &d_us, usteps, st)))
        return rc;
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    release_allocation(A, A->d_dn_task_ptr);
    release_allocation(A, A->d_dn_steps);
    release_allocation(A, A->d_up_task_ptr);
    release_allocation(A, A->d_up_steps);
    A->d_dn_task_ptr = d_dptr;
    A->d_dn_steps = d_ds;
    A->dn_ntasks = dn_ntasks;
    A->dn_entries = dn_entries;
    A->d_up_task_ptr = d_uptr;
    A->d_up_steps = d_us;
    A->up_ntasks = up_ntasks;
    A->up_entries = up_entries;
    A->up_target = up_target;
    A->down_target = down_target;
    const bool cut_moved = up_cut != A->up_cut;
    A->up_cut = up_cut;
    if (cut_moved && A->tc.built) return hybrid_lists(A, st);
    return 0;
}

}  // namespace h2
