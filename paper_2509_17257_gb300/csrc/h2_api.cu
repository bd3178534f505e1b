// The extern "C" entry points declared in include/h2.h.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "h2_internal.cuh"

namespace h2 {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

bool is_device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Pinned host memory the device can address (mapped): its device pointer, else nullptr.
const void* mapped_host_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

namespace {
constexpr long long kDefaultWaitLimit = 1ll << 24;
std::atomic<long long> g_wait_limit{kDefaultWaitLimit};
std::atomic<int64_t> g_alloc_limit{0};  // 0: no cap
std::atomic<int64_t> g_alloc_live{0};   // bytes held through device_alloc by live matrices
}  // namespace

long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

// Every allocation of a matrix's stored data (h2_build, the block-Jacobi
// factors) comes through here: it is counted against h2_set_alloc_limit and
// released with the matrix.
bool stream_capture_active(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown: take the path that is safe in a capture
    }
    return cs != cudaStreamCaptureStatusNone;
}

int device_alloc(h2_matrix* A, void** ptr, size_t bytes) {
    const int64_t cap = g_alloc_limit.load();
    const int64_t live = g_alloc_live.fetch_add((int64_t)bytes) + (int64_t)bytes;
    if (cap > 0 && live > cap) {
        g_alloc_live.fetch_sub((int64_t)bytes);
        set_error("device allocation of " + std::to_string(bytes) + " bytes refused: the library's cap of " +
                  std::to_string(cap) + " bytes (h2_set_alloc_limit) would be exceeded");
        return H2_E_OOM;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        g_alloc_live.fetch_sub((int64_t)bytes);
        cudaGetLastError();
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? H2_E_OOM : H2_E_CUDA;
    }
    A->allocations.push_back({p, bytes});
    A->alloc_bytes += (int64_t)bytes;
    *ptr = p;
    return 0;
}

void release_allocations(h2_matrix* A) {
    for (auto& a : A->allocations) cudaFree(a.first);
    A->allocations.clear();
    g_alloc_live.fetch_sub(A->alloc_bytes);
    A->alloc_bytes = 0;
}

void release_allocation(h2_matrix* A, void* p) {
    for (size_t i = 0; i < A->allocations.size(); ++i) {
        if (A->allocations[i].first != p) continue;
        cudaFree(p);
        A->alloc_bytes -= (int64_t)A->allocations[i].second;
        g_alloc_live.fetch_sub((int64_t)A->allocations[i].second);
        A->allocations.erase(A->allocations.begin() + (long)i);
        return;
    }
}

}  // namespace h2

struct h2_tree {
    h2::Tree T;
};

namespace {

int check_params(const h2_build_params* p) {
    if (!p) { h2::set_error("null params"); return H2_E_BADARG; }
    if (p->q < 1 || p->q > 5) { h2::set_error("q must be in [1, 5]"); return H2_E_UNSUPPORTED; }
    if (p->leaf_size < 1 || p->leaf_size > 64) { h2::set_error("leaf_size must be in [1, 64]"); return H2_E_UNSUPPORTED; }
    if (!(p->eta > 0.0) || !std::isfinite(p->eta)) { h2::set_error("eta must be finite and > 0"); return H2_E_BADARG; }
    if (!(p->length > 0.0) || !std::isfinite(p->length)) { h2::set_error("length must be finite and > 0"); return H2_E_BADARG; }
    if (!std::isfinite(p->sigma)) { h2::set_error("sigma must be finite"); return H2_E_BADARG; }
    if (p->kernel != H2_KERNEL_EXP && p->kernel != H2_KERNEL_HELMHOLTZ) {
        h2::set_error("kernel must be H2_KERNEL_EXP or H2_KERNEL_HELMHOLTZ");
        return H2_E_BADARG;
    }
    if (p->kernel == H2_KERNEL_HELMHOLTZ) {
        if (!std::isfinite(p->kappa)) { h2::set_error("kappa must be finite"); return H2_E_BADARG; }
        if (!(p->delta > 0.0) || !std::isfinite(p->delta)) {
            h2::set_error("delta must be finite and > 0 (the regularisation of the Helmholtz kernel at r = 0)");
            return H2_E_BADARG;
        }
    }
    return 0;
}

void free_matrix(h2_matrix* A) {
    if (!A) return;
    for (auto& r : A->timing.pending) {
        for (auto e : r.ev) cudaEventDestroy(e);
        if (r.k0) cudaEventDestroy(r.k0);
        if (r.k1) cudaEventDestroy(r.k1);
    }
    for (auto e : A->timing.free_events) cudaEventDestroy(e);
    h2::release_allocations(A);
    if (A->ws.base) cudaFree(A->ws.base);
    if (A->ws.stage_x) cudaFree(A->ws.stage_x);
    if (A->ws.stage_y) cudaFree(A->ws.stage_y);
    if (A->ws.side) cudaStreamDestroy(A->ws.side);
    if (A->ws.y_in) cudaEventDestroy(A->ws.y_in);
    if (A->ws.st_mark) cudaEventDestroy(A->ws.st_mark);

    if (A->err_host) cudaFreeHost(A->err_host);
    if (A->sync_cnt) cudaFree(A->sync_cnt);
    delete A;
}

}  // namespace

extern "C" {

const char* h2_last_error_string(void) { return h2::g_last_error.c_str(); }

const char* h2_version(void) { return "h2bcg 0.1 (sm_103a)"; }

int h2_tree_build(const h2_build_params* params, const double* pts, int64_t n, h2_tree** out) {
    if (!out) { h2::set_error("null out"); return H2_E_BADARG; }
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    if (!pts || n < 1) { h2::set_error("need n >= 1 host points"); return H2_E_BADARG; }
    h2_tree* T = new (std::nothrow) h2_tree();
    if (!T) { h2::set_error("host allocation failed"); return H2_E_OOM; }
    std::string err = h2::build_tree(pts, n, params->leaf_size, params->eta, T->T);
    if (!err.empty()) {
        delete T;
        h2::set_error(err);
        return H2_E_BADARG;
    }
    *out = T;
    return 0;
}

int h2_tree_view_get(const h2_tree* T, h2_tree_view* v) {
    if (!T || !v) { h2::set_error("null argument"); return H2_E_BADARG; }
    v->n = T->T.n;
    v->n_clusters = T->T.n_clusters();
    v->n_adm = T->T.n_adm();
    v->n_near = T->T.n_near();
    v->depth = T->T.depth;
    v->perm = T->T.perm.data();
    v->cl_offset = T->T.off.data();
    v->cl_size = T->T.size.data();
    v->cl_level = T->T.level.data();
    v->cl_parent = T->T.parent.data();
    v->cl_son0 = T->T.son0.data();
    v->cl_son1 = T->T.son1.data();
    v->cl_box = T->T.box.data();
    v->adm_rowptr = T->T.adm_rowptr.data();
    v->adm_col = T->T.adm_col.data();
    v->near_rowptr = T->T.near_rowptr.data();
    v->near_col = T->T.near_col.data();
    return 0;
}

int h2_tree_schedule(const h2_tree* T, int32_t which, int32_t* ntasks, int32_t* nsteps, int32_t* entries,
                     int32_t* task_ptr, int32_t* steps) {
    if (!T || !ntasks || !nsteps || !entries || (which != 0 && which != 1)) {
        h2::set_error("h2_tree_schedule: null argument or which not 0/1");
        return H2_E_BADARG;
    }
    std::vector<int32_t> ptr;
    std::vector<int32_t> flat;
    int32_t nt = 0, ent = 0;
    if (which == 0) {
        std::vector<h2::DownStep> v;
        h2::down_schedule(T->T, h2::kDownTasks, ptr, v, nt, ent);
        for (const auto& d : v) flat.insert(flat.end(), {d.c, d.rd, d.wr, d.flags});
    } else {
        std::vector<h2::UpStep> v;
        h2::up_schedule(T->T, h2::kUpTasks, ptr, v, nt, ent);
        for (const auto& u : v) flat.insert(flat.end(), {u.c, u.rd0, u.rd1, u.wr});
    }
    *ntasks = nt;
    *nsteps = (int32_t)(flat.size() / 4);
    *entries = ent;
    if (task_ptr) std::copy(ptr.begin(), ptr.end(), task_ptr);
    if (steps) std::copy(flat.begin(), flat.end(), steps);
    return 0;
}

int h2_tree_free(h2_tree* T) {
    delete T;
    return 0;
}

int h2_build(const h2_build_params* params, const double* pts, int64_t n, h2_matrix** out) {
    if (!out) { h2::set_error("null out"); return H2_E_BADARG; }
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    if (!pts || n < 1) { h2::set_error("need n >= 1 points"); return H2_E_BADARG; }
    if (params->kernel == H2_KERNEL_HELMHOLTZ && (params->precisions & (1u << H2_BF16))) {
        h2::set_error("a complex kernel has no BF16 product");
        return H2_E_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)params->stream;
    std::vector<double> host;
    const double* hp = pts;
    if (h2::is_device_pointer(pts)) {
        host.resize((size_t)n * 3);
        cudaError_t e = cudaMemcpy(host.data(), pts, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { h2::set_error(cudaGetErrorString(e)); return H2_E_CUDA; }
        hp = host.data();
    }
    h2_matrix* A = new (std::nothrow) h2_matrix();
    if (!A) { h2::set_error("host allocation failed"); return H2_E_OOM; }
    std::string err = h2::build_tree(hp, n, params->leaf_size, params->eta, A->T);
    if (!err.empty()) {
        delete A;
        h2::set_error(err);
        return H2_E_BADARG;
    }
    A->q = params->q;
    A->k = params->q * params->q * params->q;
    A->length = params->length;
    A->sigma = params->sigma;
    A->kernel = params->kernel;
    A->cplx = params->kernel == H2_KERNEL_HELMHOLTZ;
    A->kappa = A->cplx ? params->kappa : 0.0;
    A->delta = A->cplx ? params->delta : 0.0;
    A->n = n;
    A->nc = A->T.n_clusters();
    A->n_adm = A->T.n_adm();
    A->n_near = A->T.n_near();
    A->depth = A->T.depth;
    int64_t nl = 0;
    for (int64_t c = 0; c < A->nc; ++c) nl += A->T.is_leaf((int32_t)c);
    A->n_leaves = nl;
    const char* fs = getenv("H2_FORCE_SIMT");
    A->force_simt = fs && fs[0] == '1';
    const char* ft = getenv("H2_TC_TRANSFER");
    A->use_flow = ft && ft[0] == '1' ? 1 : (ft && ft[0] == '0' ? 0 : -1);
    const char* fh = getenv("H2_TC_HYBRID");
    A->use_hybrid = fh && fh[0] == '1' ? 1 : (fh && fh[0] == '0' ? 0 : -1);
    const char* fk = getenv("H2_KRON");
    A->use_kron = fk && fk[0] == '0' ? 0 : 1;
    rc = h2::build_device(A, hp, params->precisions, st);
    if (rc) {
        free_matrix(A);
        return rc;
    }
    *out = A;
    return 0;
}

int h2_free(h2_matrix* A) {
    free_matrix(A);
    return 0;
}

int h2_info(const h2_matrix* A, h2_info_t* info) {
    if (!A || !info) { h2::set_error("null argument"); return H2_E_BADARG; }
    info->n = A->n;
    info->k = A->k;
    info->n_clusters = A->nc;
    info->n_leaves = A->n_leaves;
    info->n_adm = A->n_adm;
    info->n_near = A->n_near;
    info->nnz_near = A->nnz_near;
    info->depth = A->depth;
    info->q = A->q;
    info->bytes_f64 = A->f64.bytes;
    info->bytes_f32 = A->f32.built ? A->f32.bytes : 0;
    info->bytes_bf16 = A->tc.has_bf16 ? A->tc.bytes : 0;
    const double k = (double)A->k;
    // leaf forward + leaf backward, up + down transfers, coupling, nearfield, shift
    info->flops_per_col = 2.0 * 2.0 * (double)A->n * k + 2.0 * 2.0 * (double)(A->nc - 1) * k * k +
                          2.0 * (double)A->n_adm * k * k + 2.0 * (double)A->nnz_near + 2.0 * (double)A->n;
    if (A->cplx)  // per complex column: real transfers on two real columns, 8 flops per complex multiply-add
        info->flops_per_col = 2.0 * (2.0 * 2.0 * (double)A->n * k + 2.0 * 2.0 * (double)(A->nc - 1) * k * k) +
                              8.0 * ((double)A->n_adm * k * k + (double)A->nnz_near) + 4.0 * (double)A->n;
    info->launches = A->launches_per_product;
    // tensor-core chain: gather, upward pass, coupling, downward pass, leaf phase, scatter into Y, + zeroing of
    // clusters without couplings (done by the gather with the hybrid upward pass); where the subtree-owning
    // transfer passes do not apply (k % 4 != 0 or k > 64) also the packing of X, x̂ and ŷ
    const bool own_passes = A->f32.Et && A->k % 8 == 0 && A->k <= 64;
    const bool hybrid_default = own_passes && (A->tc.hybrid || A->tc.hybrid_bf16) && A->tc.h_default;
    info->launches_tc = A->tc.built ? (own_passes ? 5 : 8) + (A->down_ptr.back() > 0 ? 1 : 0) +
                                          (A->tc.c_nzero > 0 && !hybrid_default ? 1 : 0)
                                    : 0;
    info->kernel = A->kernel;
    info->hybrid = (A->tc.hybrid || A->tc.hybrid_bf16) && A->tc.h_default ? 1 : 0;
    info->n_above_cut = A->tc.h_nabove;
    return 0;
}

int h2_timing_enable(h2_matrix* A, int32_t enable) {
    if (!A) { h2::set_error("null argument"); return H2_E_BADARG; }
    A->timing.on = enable != 0;
    return 0;
}

int h2_timing_query(h2_matrix* A, double* ms, int64_t* calls, int32_t reset) {
    if (!A) { h2::set_error("null argument"); return H2_E_BADARG; }
    auto& Tm = A->timing;
    for (auto& r : Tm.pending) {
        const auto& ev = r.ev;
        if (!ev.empty()) {
            cudaError_t e = cudaEventSynchronize(ev.back());
            if (e != cudaSuccess) { h2::set_error(cudaGetErrorString(e)); return H2_E_CUDA; }
        }
        for (size_t i = 0; i + 1 < ev.size() && i < 6; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) Tm.ms[i] += t;
        }
        if (r.k0 && r.k1) {
            float t = 0.f;
            if (cudaEventSynchronize(r.k1) == cudaSuccess && cudaEventElapsedTime(&t, r.k0, r.k1) == cudaSuccess)
                Tm.ms[6] += t;
        }
        for (auto e : ev) Tm.free_events.push_back(e);
        if (r.k0) Tm.free_events.push_back(r.k0);
        if (r.k1) Tm.free_events.push_back(r.k1);
        Tm.calls += 1;
    }
    Tm.pending.clear();
    if (ms) for (int i = 0; i < H2_NPHASE; ++i) ms[i] = Tm.ms[i];
    if (calls) *calls = Tm.calls;
    if (reset) {
        for (int i = 0; i < H2_NPHASE; ++i) Tm.ms[i] = 0.0;
        Tm.calls = 0;
    }
    return 0;
}

int h2_matmul(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
              int32_t dtype, void* stream) {
    return h2::matmul(A, alpha, X, ldx, Y, ldy, m, dtype, (cudaStream_t)stream, false);
}

int h2_matmul_transposed(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
                         int64_t m, int32_t dtype, void* stream) {
    return h2::matmul(A, alpha, X, ldx, Y, ldy, m, dtype, (cudaStream_t)stream, true);
}

int h2_matmul_complex(h2_matrix* A, double alpha_re, double alpha_im, const double* X, int64_t ldx, double* Y,
                      int64_t ldy, int64_t m, int32_t dtype, void* stream) {
    if (!A) { h2::set_error("null argument"); return H2_E_BADARG; }
    if (m < 0 || m > ((int64_t)1 << 19) || ldx < m || ldy < m || ldx > INT64_MAX / 2 || ldy > INT64_MAX / 2) {
        h2::set_error("h2_matmul_complex: bad m / leading dimension (m <= 2^19 complex columns)");
        return H2_E_BADARG;
    }
    if (dtype != H2_F64 && dtype != H2_F32) {
        h2::set_error("h2_matmul_complex: dtype H2_F64 or H2_F32");
        return H2_E_UNSUPPORTED;
    }
    if (!std::isfinite(alpha_re) || !std::isfinite(alpha_im)) {
        h2::set_error("h2_matmul_complex: alpha must be finite");
        return H2_E_BADARG;
    }
    // interleaved complex blocks as doubles: 2m real columns, leading dimensions 2·ld
    return h2::matmul(A, alpha_re, X, 2 * ldx, Y, 2 * ldy, 2 * m, dtype, (cudaStream_t)stream, false, &alpha_im);
}

int h2_block_cg(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
                const h2_cg_params* params, h2_cg_result* res) {
    if (int rc = h2::refuse_complex(A, "h2_block_cg")) return rc;
    return h2::block_cg(A, B, ldb, X, ldx, m, params, res);
}

int h2_set_alloc_limit(int64_t bytes) {
    if (bytes < 0) { h2::set_error("h2_set_alloc_limit: bytes must be >= 0"); return H2_E_BADARG; }
    h2::g_alloc_limit.store(bytes);
    return 0;
}

int h2_alloc_bytes(int64_t* bytes) {
    if (!bytes) { h2::set_error("h2_alloc_bytes: null argument"); return H2_E_BADARG; }
    *bytes = h2::g_alloc_live.load();
    return 0;
}

int h2_set_wait_limit(int64_t polls) {
    h2::g_wait_limit.store(polls == 0 ? h2::kDefaultWaitLimit : (long long)polls);
    return 0;
}

int h2_block_gmres(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
                   const h2_gmres_params* params, h2_cg_result* res) {
    if (int rc = h2::refuse_complex(A, "h2_block_gmres")) return rc;
    return h2::block_gmres(A, B, ldb, X, ldx, m, params, res);
}

}  // extern "C"
