// Internal state of an h2_matrix and helpers shared by the CUDA sources.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/h2.h"
#include "h2_tree.hpp"

namespace h2 {

void set_error(const std::string& msg);

#define H2_CUDA_TRY(expr)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError(); /* do not leave it for the next launch check */            \
            ::h2::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));            \
            return e_ == cudaErrorMemoryAllocation ? H2_E_OOM : H2_E_CUDA;                 \
        }                                                                                  \
    } while (0)

#define H2_LAUNCH_CHECK()                                                                  \
    do {                                                                                   \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess) {                                                           \
            ::h2::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));       \
            return H2_E_CUDA;                                                              \
        }                                                                                  \
    } while (0)

// One typed copy of the matrix data (V leaf rows, transfer E, coupling S,
// nearfield G), row-major:
//   V    [n][k]         rows in cluster order (position i = point perm[i])
//   E    [n_c][k][k]    E[c][μ][ν], c != root (root slot unused)
//   S    [n_adm][k][k]  S[j][ν][μ] in row-cluster list order
//   Near concatenated  G_j[|t̂|][|ŝ|] blocks at near_off[j]
struct MatData {
    void* V = nullptr;
    void* E = nullptr;
    void* Et = nullptr;  // FP32 only, k % 8 == 0, k <= 64: E_{t'}ᵀ per cluster, rows of kEtLd floats
    void* kron = nullptr;  // q = 4: the 4×4 factors F_x, F_y, F_z of E_{t'} = F_z ⊗ F_y ⊗ F_x [n_c][48]
    void* S = nullptr;
    void* Near = nullptr;
    int64_t bytes = 0;
    bool built = false;
};

// Per-phase event timing of the product (h2_timing_enable / h2_timing_query).
struct TimingRecord {
    std::vector<cudaEvent_t> ev;       // phase boundaries (7 per product)
    cudaEvent_t k0 = nullptr, k1 = nullptr;  // around the coupling kernel launch alone
};
struct Timing {
    bool on = false;
    std::vector<cudaEvent_t> free_events;
    std::vector<TimingRecord> pending;
    double ms[H2_NPHASE] = {0};
    int64_t calls = 0;
};

// One tile to convert into the tcgen05 core-matrix BF16 layout: rows n of k
// FP64 values (leading dimension ld) at element offset src → np × kp tile at
// byte offset dst (zero padded).
struct TcPackTile {
    int64_t src, dst;
    int32_t n, k, ld, np, kp;
    int32_t tr;  // bit 0: the tile holds the transpose, row r column c = src[c·ld + r];
                 // bit 1 (BF16): the remainder v - bf16(v) instead of v
};

// One output tile of the tcgen05 segmented GEMM: output id, its terms
// [e0, e1), and the output width np (a multiple of 16) in the low 16 bits of
// np; in the transfer-pass launches (mode 3) bits 16-17 give the item's role:
// kRoleTransfer (split tile into out_act, then the ready flag), kRoleCoupling
// (split tile into out_act2) or kRoleLeaf (FP32 rows into zp).
struct TcItem {
    int32_t id, e0, e1, np;
};
constexpr int32_t kRoleTransfer = 1, kRoleCoupling = 2, kRoleLeaf = 3;
__host__ __device__ inline int32_t item_np(const TcItem& t) { return t.np & 0xFFFF; }
__host__ __device__ inline int32_t item_role(const TcItem& t) { return (t.np >> 16) & 3; }
// One term: an activation tile (act0, act1 or act2 by asrc & 3, at akoff·R·es
// bytes, kp contraction columns) times a matrix tile (at boff BF16-bytes, scaled
// by es/2).  In mode 3, asrc & kTermWait makes the copy wait for the ready flag
// of cluster akoff / KP.
struct TcTerm {
    int64_t boff;
    int32_t akoff;
    int16_t kp, asrc;
};
constexpr int16_t kTermWait = 4;
// The complex product (TcGemmParams::cplx): the term multiplies i·act instead of
// act, i.e. its activation columns come in (real, imaginary) pairs and column 2j
// takes -(column 2j + 1), column 2j + 1 takes column 2j (the epilogue applies
// the swap and the sign to the term's result).
constexpr int16_t kTermImag = 8;

// The per-system arguments of a multi-system launch of the tcgen05 segmented
// GEMM (one launch serving several H² matrices, h2_batch_matmul): an item's
// system index (item_sys) selects its terms, buffers and sizes.
struct TcSys {
    const TcTerm* terms;
    const uint8_t* act0;
    const uint8_t* act1;
    const uint8_t* act2;
    const uint8_t* bmat;
    uint8_t* out_act;
    uint8_t* out_act2;
    int* flag;
    float* zp;
    const int32_t* leaves;
    const int32_t* cl_off;
    const int32_t* cl_size;
    int R, mc, k, KP, ldc, pad;
};
__host__ __device__ inline int32_t item_sys(const TcItem& t) { return (int32_t)((uint32_t)t.np >> 18); }

// Arguments of the tcgen05 segmented GEMM (h2_tc.cu).  Items are processed in
// order, item w by CTA w mod gridDim.
struct TcGemmParams {
    int n_items;
    const TcItem* items;
    const TcTerm* terms;
    const uint8_t* act0;
    const uint8_t* act1;
    const uint8_t* act2;
    const uint8_t* bmat;
    int R, mc;
    float* yhat;  // coupling output [cluster][k][ldc]
    float* zp;    // leaf output in cluster order [point][ldc]
    int k, ldc;
    const int32_t* leaves;
    const int32_t* cl_off;
    const int32_t* cl_size;
    int* err;
    int a_stage_bytes, nstages;  // filled by launch_tc_gemm
    // transfer passes (modes 3 and 4): each item's result goes, split as the
    // activations are, into its tile of out_act (TF32 pairs); then flag[id] = epoch
    // tells the CTAs whose terms read that tile (mode 4 adds the coupling result
    // yhat[id] first).  A term with asrc == 0 waits for flag[akoff / KP].
    uint8_t* out_act;
    uint8_t* out_act2;  // kRoleCoupling items
    int* flag;
    int epoch;
    // mode 3 with several systems: per-system arguments (items carry their system in
    // bits 18.. of np); the launch-wide R is the largest system's
    const TcSys* sys;
    // matrix-free coupling (mode 2): Chebyshev nodes [cluster][KP] (x, y, z, 0) and
    // the kernel's 1/length; S_b[ν, μ] = exp(-|ξ_{t,ν} - ξ_{s,μ}| / length) for ν, μ < k
    const float4* nodes;
    float inv_len;
    int KP;
    // modes 0 and 1 of the complex product: terms marked kTermImag apply i·act
    int cplx;
};

// BF16 tensor-core copy of the matrix data and the schedules of its kernels.
struct TcData {
    bool built = false;
    int KP = 0, NP = 0;
    uint8_t* mat = nullptr;    // BF16 core-matrix tiles: S (list order), V (leaf order), G (near order)
    uint8_t* mat32 = nullptr;  // the same tiles in FP32 (offsets ×2), for the 3xTF32 product
    float4* nodes4 = nullptr;  // [n_clusters][KP] Chebyshev tensor nodes (x, y, z, 0), zero past k (matrix-free coupling)
    int64_t bytes = 0;
    bool has_bf16 = false, has_tf32 = false;
    // coupling: outputs are clusters with at least one admissible block
    TcItem* c_items = nullptr;
    TcTerm* c_terms = nullptr;
    int c_nitems = 0;
    int32_t* c_zero = nullptr;
    int c_nzero = 0;
    // leaf: outputs are leaf positions
    TcItem* l_items = nullptr;
    TcTerm* l_terms = nullptr;
    int l_nitems = 0;
    int64_t* xkoff = nullptr;   // [n_leaves+1] prefix sums of round16(|leaf|)
    int64_t xk_total = 0;
    int32_t* leaf_base = nullptr;  // first point position of each leaf
    int32_t* leaf_kdim = nullptr;  // points of each leaf
    TcPackTile* d_tiles = nullptr; // pack descriptors (S tiles first), kept to rebuild S
    int64_t n_s_tiles = 0;
    // the product with Aᵀ (built on its first use, build_tc_transposed): S_bᵀ, V and
    // G_bᵀ tiles in the same layout, a coupling list over column clusters and a leaf
    // list over column leaves
    bool t_built = false;
    uint8_t* matT = nullptr;
    uint8_t* matT32 = nullptr;
    TcPackTile* d_tilesT = nullptr;  // S_bᵀ tiles first (rebuilt with S)
    TcItem* ct_items = nullptr;
    TcTerm* ct_terms = nullptr;
    int ct_nitems = 0;
    int32_t* ct_zero = nullptr;
    int ct_nzero = 0;
    TcItem* lt_items = nullptr;
    TcTerm* lt_terms = nullptr;
    int lt_nitems = 0;
    // the transfer passes on the tensor cores (built with the TF32 copy, k <= 64):
    // Eᵀ_s, V_tᵀ, E_s and an identity tile appended to mat32, and work lists in
    // dependency order: the upward and the downward pass alone (used with Aᵀ),
    // the upward pass with the coupling phase (f1) and the downward pass with the
    // leaf phase (f2) in one launch each (used with A)
    bool flow = false;
    TcItem* up_items = nullptr;  // clusters by height above the leaves (sons first)
    TcTerm* up_terms = nullptr;
    int up_nitems = 0;
    TcItem* dn_items = nullptr;  // clusters by level (fathers first)
    TcTerm* dn_terms = nullptr;
    int dn_nitems = 0;
    TcItem* f1_items = nullptr;
    TcTerm* f1_terms = nullptr;
    int f1_nitems = 0;
    TcItem* f2_items = nullptr;
    TcTerm* f2_terms = nullptr;
    int f2_nitems = 0;
    // the f1 and f2 items with their sort keys, on the host, for the work lists of
    // launches that serve several matrices (h2_batch_matmul)
    std::vector<int32_t> f1_keys, f2_keys;
    std::vector<TcItem> f1_host, f2_host;
    // the coupling launch that also computes the clusters above the CUDA-core
    // upward pass's cut (k_tc_gemm<4, 1>; rebuilt with the cut): transfer items
    // for those clusters interleaved with the coupling items (hybrid_lists)
    bool hybrid = false;
    bool h_default = false;  // the built-in rule takes it (enough coupling work to hide the chain)
    int64_t h_nabove = 0;    // clusters above the cut (its transfer items)
    TcItem* h_items = nullptr;
    TcTerm* h_terms = nullptr;
    int h_nitems = 0;
    std::vector<int64_t> s_off_host, et_off_host;  // tile offsets of S_j and of Eᵀ_c in mat32 (elements)
    // The BF16 product's hybrid lists (k_tc_gemm<4, 0>): Eᵀ_c as two BF16 tiles, its
    // high part and the remainder (after the BF16 tiles of S, V and G in mat), so
    // the transfer items lose no accuracy to the rounding of E; two terms per son.
    bool hybrid_bf16 = false;
    TcItem* hb_items = nullptr;
    TcTerm* hb_terms = nullptr;
    int hb_nitems = 0;
    std::vector<int64_t> ebh_off_host, ebl_off_host;  // Eᵀ_c high and low tiles in mat (bytes)
};

// Inter-CTA bookkeeping of the one-launch transfer passes: arrival counters of
// the upward pass (self-resetting), ready flags of the downward pass and its
// claim tickets (both cleared before every downward pass, so a captured CUDA
// graph can replay the product).
// One step of the subtree-owning downward pass (k_down_own, h2_mm.cu): cluster c
// gets ŷ_c = ŷ_c + E_c ŷ_parent with ŷ_parent read from shared-memory stack
// entry rd and the result kept in entry wr; kDownLoad marks the first step of a
// task (entry wr ← the root's ŷ, no product), kDownStore a leaf whose ŷ goes
// back to global memory.
struct DownStep {
    int32_t c, rd, wr, flags;
};
constexpr int kDownLoad = 1, kDownStore = 2;
constexpr int kEtLd = 72;  // row stride of the FP32 Eᵀ blocks (≡ 8 mod 32)
constexpr int kTcGrid = 152;  // CTAs of the tensor-core kernels (one per SM); their work lists are laid out for it
constexpr int kDownMaxSteps = 192;  // steps of one task at most (the schedule keeps to it)

// One step of the subtree-owning upward pass (k_up_own, h2_mm.cu): a leaf c
// (rd0 < 0, rd1 = its position among the leaves) gets x̂_c = V_cᵀ X|_ĉ; an
// inner cluster gets x̂_c = E_s0ᵀ x̂_s0 + E_s1ᵀ x̂_s1 with the sons' x̂ in
// shared-memory stack entries rd0 and rd1.  x̂_c goes to global memory and to
// entry wr.
struct UpStep {
    int32_t c, rd0, rd1, wr;
};
constexpr int kUpMaxSteps = 64;    // steps of one task at most
// Task counts the cut levels aim at: the downward pass takes the shallowest level
// with at least kDownTasks subtrees; the upward pass, whose longest subtree bounds
// its task phase, about 1.7 tasks per CTA slot (two per SM)
constexpr int kDownTasks = 256, kUpTasks = 400;
constexpr int kUpMaxEntries = 5;   // stack entries at most (three of them serve the climb above the cut)

struct Tree;
// Transfer-pass schedules (h2_build.cu), host only
void down_schedule(const Tree& T, int target, std::vector<int32_t>& task_ptr, std::vector<DownStep>& steps,
                   int32_t& ntasks, int32_t& entries);
void up_schedule(const Tree& T, int target, std::vector<int32_t>& task_ptr, std::vector<UpStep>& steps,
                 int32_t& ntasks, int32_t& entries,
                 int32_t* cut_level = nullptr);

// Product variants the autotuner chooses among (h2_autotune).
enum ProductPath : int8_t {
    kPathDefault = 0,  // built-in rule: tensor cores where built; their transfer passes where the
                       // CUDA-core subtree passes do not apply (k % 8 != 0 or columns % 4 != 0)
    kPathTcOwn = 1,    // tensor cores, CUDA-core transfer passes
    kPathTcFlow = 2,   // tensor cores, tensor-core transfer passes, one launch per phase
    kPathTcFused = 3,  // tensor cores, transfer passes sharing launches with coupling and leaf phases
    kPathSimt = 4,     // CUDA cores only (FP32)
    kPathTcHybrid = 5  // tensor cores, CUDA-core subtree passes below the cut, the clusters above
                       // the upward cut as transfer items of the coupling launch
};
struct Tune {
    int8_t path = kPathDefault;
    int8_t stages = 0;  // pipeline stages of the tensor-core kernels (0: as many as fit)
};
inline int column_class(int mc) { return mc <= 8 ? 0 : (mc <= 16 ? 1 : (mc <= 32 ? 2 : 3)); }

struct SyncBufs {
    unsigned* cnt = nullptr;
    int* flag = nullptr;
    unsigned* claim = nullptr;
    int epoch = 0;
    int* err = nullptr;
    int* fflag = nullptr;  // [2 × n_clusters] ready flags of the tensor-core upward and downward passes
    unsigned* claim2 = nullptr;  // the tensor-core chain's downward-pass task counter (claim is the upward one)
};

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    double* stage_x = nullptr;  // host-pointer staging (n×m doubles each)
    double* stage_y = nullptr;
    size_t stage_bytes = 0;
    // a product on host blocks copies Y in on a side stream while it computes;
    // the pass that updates Y first waits for y_in (once, when y_wait is set)
    cudaStream_t side = nullptr;
    cudaEvent_t y_in = nullptr, st_mark = nullptr;
    bool y_wait = false;
};
// Make st wait for a pending copy of Y into its staging buffer (see Workspace).
inline int wait_y_staged(Workspace& ws, cudaStream_t st) {
    if (!ws.y_wait) return 0;
    ws.y_wait = false;
    return cudaStreamWaitEvent(st, ws.y_in, 0) == cudaSuccess ? 0 : H2_E_CUDA;
}

}  // namespace h2

struct h2_matrix {
    h2::Tree T;
    int q = 0, k = 0;
    double length = 0, sigma = 0;
    // kernel g: H2_KERNEL_EXP (real) or H2_KERNEL_HELMHOLTZ (complex; kappa, delta).  A
    // complex matrix (cplx) stores S and the nearfield blocks of f64 / f32 as two planes,
    // real parts then imaginary parts; V and E are real.
    int32_t kernel = 0;
    double kappa = 0, delta = 0;
    bool cplx = false;
    int64_t n = 0, nc = 0, n_leaves = 0, n_adm = 0, n_near = 0, nnz_near = 0;
    int32_t depth = 0;

    // host copies of the level schedule
    std::vector<int64_t> up_ptr;    // [depth+2] inner clusters of level l: up_list[up_ptr[l]..up_ptr[l+1])
    std::vector<int64_t> down_ptr;  // [depth+2] non-root clusters of level l
    std::vector<int32_t> leaves;    // leaf cluster ids in pre-order

    // device topology (int32 ids/positions; int64 element offsets)
    int32_t* d_perm = nullptr;       // [n]
    int32_t* d_cl_off = nullptr;     // [nc]
    int32_t* d_cl_size = nullptr;    // [nc]
    int32_t* d_parent = nullptr;     // [nc]
    int32_t* d_leaves = nullptr;     // [n_leaves]
    int32_t* d_up_list = nullptr;    // inner clusters by level
    int32_t* d_son0 = nullptr;       // [nc]
    int32_t* d_son1 = nullptr;       // [nc]
    int32_t* d_down_list = nullptr;  // non-root clusters by level
    // subtree-owning downward pass: task t runs steps dn_steps[dn_task_ptr[t]..dn_task_ptr[t+1])
    int32_t* d_dn_task_ptr = nullptr;
    h2::DownStep* d_dn_steps = nullptr;
    int32_t dn_ntasks = 0, dn_entries = 0;
    // subtree-owning upward pass: task t runs up_steps[up_task_ptr[t]..up_task_ptr[t+1]), then climbs
    int32_t* d_up_task_ptr = nullptr;
    h2::UpStep* d_up_steps = nullptr;
    int32_t up_ntasks = 0, up_entries = 0;
    int32_t* d_adm_rowptr = nullptr; // [nc+1] by row cluster
    int32_t* d_adm_col = nullptr;    // [n_adm]
    int32_t* d_adm_row = nullptr;    // [n_adm]
    int32_t* d_admT_rowptr = nullptr;// [nc+1] by column cluster (transposed product)
    int32_t* d_admT_row = nullptr;   // [n_adm] row cluster t of each entry
    int32_t* d_admT_blk = nullptr;   // [n_adm] index j of S_j
    int32_t* d_near_ptr = nullptr;   // [n_leaves+1] by row leaf position
    int32_t* d_near_col = nullptr;   // [n_near] column cluster id
    int32_t* d_near_row = nullptr;   // [n_near] row cluster id
    int64_t* d_near_off = nullptr;   // [n_near] element offset of G_j
    int64_t* d_near_diag = nullptr;  // [n_leaves] element offset of the diagonal block G_(t,t)
    int32_t* d_nearT_ptr = nullptr;  // [n_leaves+1] by column leaf position
    int32_t* d_nearT_row = nullptr;  // [n_near] row cluster t
    int32_t* d_nearT_blk = nullptr;  // [n_near] block index j
    double* d_pts = nullptr;         // [n][3] points in cluster order
    double* d_nodes = nullptr;       // [nc][3][q] Chebyshev nodes per cluster

    h2::MatData f64, f32;
    h2::TcData tc;
    h2::Workspace ws;
    h2::Timing timing;
    int32_t launches_per_product = 0;
    int* err_host = nullptr;  // mapped pinned flag: a bounded device-side wait gave up
    int* err_dev = nullptr;
    unsigned* sync_cnt = nullptr;  // [nc × sync_tiles]
    int* sync_flag = nullptr;      // [nc × sync_tiles]
    unsigned* sync_claim = nullptr;// [sync_tiles]
    int* sync_fflag = nullptr;     // [2 × nc] tensor-core transfer-pass flags
    int64_t sync_tiles = 0;
    bool force_simt = false;
    // H2_TC_TRANSFER at build: 1 forces the tensor-core transfer passes on the FP32
    // product, 0 the CUDA-core ones; unset leaves the choice to the tuning below
    int use_flow = -1;
    // choices of h2_autotune per precision (0: FP32, 1: BF16) and column class
    // (columns per 64-column chunk: <= 8, <= 16, <= 32, <= 64)
    h2::Tune tune[2][4];
    int32_t up_target = h2::kUpTasks, down_target = h2::kDownTasks;  // transfer-pass cut targets
    int32_t up_cut = 0;  // level of the upward pass's task roots (leaves above it are tasks too)
    // H2_TC_HYBRID at build: 1 / 0 force the hybrid upward pass on / off (unset: tuning or default)
    int use_hybrid = -1;
    // H2_KRON at build: 0 keeps the q = 4 transfer passes on the dense transfer matrices
    int use_kron = 1;
    bool s_replaced = false;  // h2_coupling_set was called: S_b are no longer g's values  // H2_FORCE_SIMT=1 at build: FP32 product on the CUDA cores only
    // block-Jacobi preconditioner (h2_precond.cu): (G_(t,t) + σI)⁻¹ per leaf, built on first use
    double* bj_inv = nullptr;     // concatenated n_t×n_t inverses, leaf order
    float* bj_inv32 = nullptr;    // the same rounded to FP32 (the low-precision iterations of mixed solves)
    int64_t bj_count = 0;         // entries of bj_inv
    int64_t* bj_off = nullptr;    // [n_leaves] element offset of leaf t's inverse
    double bj_sigma = 0.0;        // σ the inverses were formed with
    bool bj_valid = false;
    std::vector<std::pair<void*, size_t>> allocations;
    int64_t alloc_bytes = 0;  // bytes of `allocations` (counted against h2_set_alloc_limit)
};

namespace h2 {

// Per-column state of the device block CG (h2_cg.cu, h2_gram.cu).
struct CgDev {
    double* bnorm;   // [m] |b_i| (1 when 0)
    double* alpha;   // [m]
    double* beta;    // [m]
    double* gamma;   // [m]
    double* rnorm;   // [m] |r_i| after the last update
    int* active;     // [m] 1 while column i has not converged
    int* conv_iter;  // [m]
    int* summary;    // [0] = active columns, [1] = breakdown flag
    double* partial; // [kRowBlocks = 304][m][2]; the block-Jacobi apply uses it as [456][m]
    unsigned* ticket;// [ceil(m/32)]
};

// State of the Gram-matrix block CG (variant H2_CG_GRAM, h2_gram.cu); m <= 64.
struct GramDev {
    double* part;      // [kGramCtas][2m² + m] per-CTA partial sums
    double* G;         // [m×m] Pᵀ(AP)
    double* W;         // [m×m] PᵀR, then (AP)ᵀR after the update
    double* L;         // [m×m] Cholesky factor of G on the kept directions (lower triangle)
    double* alpha;     // [m×m] step  α = G⁻¹ PᵀR
    double* gamma;     // [m×m] direction coefficients  Γ = G⁻¹ (AP)ᵀR
    double* rr;        // [m] |r_j|² after the update
    int* kept;         // [m] direction j kept by the deflating Cholesky
    unsigned* ticket;  // [1]
};

// Block-Jacobi preconditioner M = blockdiag_t (G_(t,t) + σI) (h2_precond.cu).
int bj_prepare(h2_matrix* A, cudaStream_t st);
// Z = M⁻¹ R (n×m, ld m, caller's point order).  With AP != nullptr also
// d.gamma[i] = <AP_i, Z_i> / d.beta[i] for the active columns (fixed-order
// reduction).  `low`: FP32 arithmetic with the FP32-rounded inverses.
int bj_apply(h2_matrix* A, const double* R, double* Z, int64_t n, int m, const double* AP, const CgDev& d,
             cudaStream_t st, bool low = false);

constexpr int kGramMaxCols = 64;
size_t gram_scratch_bytes(int m);
void gram_carve(GramDev* g, void* base, int m);
int gram_prepare();
// P = R on active columns, 0 elsewhere (the first direction block).
int gram_start(double* P, const double* R, int64_t n, int m, const GramDev& g, const CgDev& d, cudaStream_t st);
// After AP = A P: G = PᵀAP, W = PᵀR, the deflating Cholesky of G and α = G⁻¹W.
int gram_alpha(const double* P, const double* AP, const double* R, int64_t n, int m, const GramDev& g,
               const CgDev& d, cudaStream_t st);
// X += Pα, R -= (AP)α, column norms and convergence, Γ = G⁻¹(AP)ᵀR, P = R - PΓ.
int gram_update_dir(double* X, int64_t ldx, double* P, const double* AP, double* R, int64_t n, int m, double tol,
                    const GramDev& g, const CgDev& d, cudaStream_t st);
// Preconditioned form: X += Pα, R -= (AP)α and |r_j|² only; then, with
// Z = M⁻¹R, Γ = G⁻¹(AP)ᵀZ and P = Z - PΓ.
int gram_update(double* X, int64_t ldx, const double* P, const double* AP, double* R, int64_t n, int m,
                const GramDev& g, cudaStream_t st);
int gram_gamma_dir_from(double* P, const double* AP, const double* Z, int64_t n, int m, double tol,
                        const GramDev& g, const CgDev& d, cudaStream_t st);
// Zero the directions of inactive columns (after a reliable update).
int gram_mask(double* P, int64_t n, int m, const CgDev& d, cudaStream_t st);

}  // namespace h2

// A group of independent systems (h2_batch.cu, h2_cg.cu).
struct h2_batch {
    std::vector<h2_matrix*> mats;
    std::vector<cudaStream_t> streams;  // one per system: branches of the captured graphs
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t origin = nullptr;  // non-blocking stream the graphs are captured on and launched from
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t mm_exec = nullptr;  // cached product graph
    std::vector<int64_t> mm_key;
    // FP32 products whose upward/coupling and downward/leaf phases run as one
    // launch each over the items of every system (multi-system work lists)
    bool multi_launch = true;  // H2_BATCH_MULTI=0 at h2_batch_create: one graph branch per system instead
    cudaGraphExec_t flow_exec = nullptr;
    std::vector<int64_t> flow_key;
    void* flow_mem = nullptr;  // merged item lists and system tables on the device
    size_t flow_bytes = 0;
};

namespace h2 {

// Capture body(i, stream_i) for every system i in `sys` as independent
// branches of one CUDA graph forked from and joined into `origin`.
int batch_capture(h2_batch* b, cudaStream_t origin, const std::vector<int>& sys,
                  int (*body)(void* ctx, int i, cudaStream_t st), void* ctx, cudaGraphExec_t* exec);
int batch_block_cg(h2_batch* b, const double* const* B, const int64_t* ldb, double* const* X, const int64_t* ldx,
                   const int64_t* m, const h2_cg_params* p, h2_cg_result* res);

// Entry points implemented in h2_build.cu / h2_mm.cu / h2_cg.cu.
int build_device(h2_matrix* A, const double* pts_host, uint32_t precisions, cudaStream_t st);
// With alpha_im (the complex product of a complex matrix, h2_matmul_complex) X and
// Y are interleaved complex blocks seen as doubles: m, ldx and ldy count doubles
// (twice the complex counts) and α = alpha + i·*alpha_im.  Without it the matrix
// must be real.
int matmul(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
           int64_t m, int32_t dtype, cudaStream_t st, bool transposed, const double* alpha_im = nullptr);
// H2_E_UNSUPPORTED (with a message naming `what`) for a complex matrix: the
// entry points other than h2_matmul_complex compute over R only.
int refuse_complex(const h2_matrix* A, const char* what);
// Device-pointer product used by the solvers: Y = overwrite ? alpha·A·X : Y + alpha·A·X.
int matmul_device(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y,
                  int64_t ldy, int64_t m, int32_t dtype, cudaStream_t st, bool transposed,
                  bool overwrite, const double* alpha_im = nullptr);
int block_cg(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
             const h2_cg_params* p, h2_cg_result* res);
int block_gmres(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
                const h2_gmres_params* p, h2_cg_result* res);

// Buffers of one matrix's FP32 tensor-core product of m <= 64 columns whose
// upward/coupling and downward/leaf phases run in multi-system launches
// (h2_batch_matmul): flow_prepare sizes them, flow_pre gathers X, packs its
// tiles and clears the flags, flow_post scatters Y += α(Z + σX).
struct FlowBufs {
    float* Xp;
    uint8_t *Xcm, *xcm, *ycm, *ycp;
    int* fflag;
    int R, mc;
};
bool flow_batchable(const h2_matrix* A, int64_t m);
void merge_by_key(const std::vector<int32_t>& keys, const std::vector<TcItem>& items, std::vector<TcItem>& out);
int flow_prepare(h2_matrix* A, int m, cudaStream_t st, FlowBufs* fb);
int flow_pre(h2_matrix* A, const double* X, int64_t ldx, const FlowBufs& fb, cudaStream_t st);
int flow_post(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy, const FlowBufs& fb,
              bool overwrite, cudaStream_t st);
// Multi-system FP32 products of a batch (h2_batch.cu): whether every system of
// sys can take them, their work lists and tables, and their graph capture.
bool flow_batch_ok(h2_batch* b, const std::vector<int>& sys, const int64_t* m, int32_t dtype);
int flow_tables(h2_batch* b, const std::vector<int>& sys, const std::vector<FlowBufs>& fb, void** mem, size_t* bytes,
                TcGemmParams* p1, TcGemmParams* p2, cudaStream_t st);
int flow_capture(h2_batch* b, const std::vector<int>& sys, const TcGemmParams& p1, const TcGemmParams& p2,
                 const std::function<int(int, cudaStream_t)>& pre, const std::function<int(int, cudaStream_t)>& post,
                 cudaGraphExec_t* exec);

// Bytes of scratch one product needs (gathered X, x̂, ŷ, transfer-pass
// bookkeeping), and the product run in caller-provided scratch of at least
// that size (device X and Y).
size_t product_scratch_bytes(const h2_matrix* A, int64_t m, int32_t dtype);
int matmul_in_scratch(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
                      int64_t m, int32_t dtype, cudaStream_t st, void* scratch);

// tcgen05 BF16 kernels (h2_tc.cu)
int tc_smem_bytes();
int tc_prepare();
// Allocate everything a product of m columns in dtype needs (workspace,
// transfer-pass bookkeeping, kernel attributes), so that the product itself
// allocates nothing (e.g. while it is captured into a CUDA graph).
int product_prepare(h2_matrix* A, int64_t m, int32_t dtype, cudaStream_t st);
int launch_tc_gemm(int mode, int kind, TcGemmParams p, int grid, cudaStream_t st, int stages = 0);
// Rebuild the subtree schedules of the CUDA-core transfer passes for other cut targets.
int set_transfer_targets(h2_matrix* A, int up_target, int down_target, cudaStream_t st);
// Work list of the coupling launch with the clusters above the upward cut (TcData::h_*).
int hybrid_lists(h2_matrix* A, cudaStream_t st);
int launch_pack_tiles(const TcPackTile* tiles, int64_t count, const double* src, uint8_t* dst, int es,
                      cudaStream_t st);
int launch_pack_act(const float* src, int64_t ld, int ids, const int32_t* idmap, const int32_t* base,
                    const int32_t* kdim, int kdim_fixed, const int64_t* koff, int kp_fixed, int mc, int R,
                    uint8_t* dst, int es, cudaStream_t st);
int launch_zero_clusters(const int32_t* ids, int count, float* yhat, int k, int ldc, int mc, cudaStream_t st);
int launch_zero_tiles(const int32_t* ids, int count, uint8_t* buf, int64_t tile_bytes, cudaStream_t st);
int build_tc(h2_matrix* A, bool bf16, bool tf32, cudaStream_t st);
// Tiles and work lists of the tensor-core product with Aᵀ (once per matrix; allocates).
int build_tc_transposed(h2_matrix* A, cudaStream_t st);


inline int round16(int x) { return (x + 15) & ~15; }

// Forward transformation in FP64 (gather + leaves + upward pass): xhat_out is
// n_c × k × m; Xp_scratch holds n × m doubles.
int forward_transform_f64(h2_matrix* A, const double* X, int64_t ldx, int64_t m, double* Xp_scratch,
                          double* xhat_out, cudaStream_t st);
int cast_f32(const double* src, float* dst, int64_t count, cudaStream_t st);

// Poll limit of the device-side waits on another CTA's ready flag (FP64
// downward pass); negative: give up at once (h2_set_wait_limit).
long long wait_limit();

bool is_device_pointer(const void* p);
// The stream is being captured into a CUDA graph (or its state cannot be read).
bool stream_capture_active(cudaStream_t st);
const void* mapped_host_pointer(const void* p);
int device_alloc(h2_matrix* A, void** ptr, size_t bytes);
// Free every device_alloc allocation of A (and take it off the library's count).
void release_allocations(h2_matrix* A);
// Free one of them (no-op for a pointer that is not one).
void release_allocation(h2_matrix* A, void* p);

}  // namespace h2
