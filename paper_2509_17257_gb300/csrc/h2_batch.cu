// Batches of independent systems: products captured into one CUDA graph with
// one branch per system, and the autotuner that picks the FP32 product path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "h2_internal.cuh"

namespace h2 {

int batch_capture(h2_batch* b, cudaStream_t origin, const std::vector<int>& sys,
                  int (*body)(void* ctx, int i, cudaStream_t st), void* ctx, cudaGraphExec_t* exec) {
    *exec = nullptr;
    H2_CUDA_TRY(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    cudaError_t e = cudaEventRecord(b->fork, origin);
    for (size_t j = 0; j < sys.size() && !rc && e == cudaSuccess; ++j) {
        const int i = sys[j];
        e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        if (e != cudaSuccess) break;
        rc = body(ctx, i, b->streams[i]);
        if (rc) break;
        e = cudaEventRecord(b->join[i], b->streams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, b->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(origin, &graph);
    if (rc || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (!rc) {
            set_error(std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ee));
            rc = H2_E_CUDA;
        }
        return rc;
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
        return H2_E_CUDA;
    }
    return 0;
}

namespace {

struct MmCtx {
    h2_batch* b;
    double alpha;
    const double* const* X;
    const int64_t* ldx;
    double* const* Y;
    const int64_t* ldy;
    const int64_t* m;
    int32_t dtype;
};

int mm_body(void* ctx, int i, cudaStream_t st) {
    MmCtx* c = (MmCtx*)ctx;
    return matmul_device(c->b->mats[i], c->alpha, c->X[i], c->ldx[i], c->Y[i], c->ldy[i], c->m[i], c->dtype, st,
                         false, false);
}

}  // namespace

}  // namespace h2

using namespace h2;

extern "C" {

int h2_batch_create(h2_matrix* const* mats, int32_t count, h2_batch** out) {
    if (!out || !mats || count < 1) { set_error("bad batch arguments"); return H2_E_BADARG; }
    *out = nullptr;
    h2_batch* b = new h2_batch();
    for (int i = 0; i < count; ++i) {
        if (!mats[i]) { delete b; set_error("null matrix in batch"); return H2_E_BADARG; }
        b->mats.push_back(mats[i]);
    }
    b->streams.resize(count, nullptr);
    b->join.resize(count, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        h2_batch_free(b);
        set_error(std::string("batch streams: ") + cudaGetErrorString(e));
        return H2_E_CUDA;
    }
    *out = b;
    return 0;
}

int h2_batch_free(h2_batch* b) {
    if (!b) return 0;
    if (b->mm_exec) cudaGraphExecDestroy(b->mm_exec);
    for (auto s : b->streams) if (s) cudaStreamDestroy(s);
    for (auto e : b->join) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
    return 0;
}

int h2_batch_matmul(h2_batch* b, double alpha, const double* const* X, const int64_t* ldx, double* const* Y,
                    const int64_t* ldy, const int64_t* m, int32_t dtype, void* stream) {
    if (!b || !X || !ldx || !Y || !ldy || !m) { set_error("null argument"); return H2_E_BADARG; }
    if (dtype != H2_F64 && dtype != H2_F32 && dtype != H2_BF16) { set_error("bad dtype"); return H2_E_BADARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const int count = (int)b->mats.size();
    std::vector<int64_t> key;
    std::vector<int> sys;
    int64_t abits;
    memcpy(&abits, &alpha, sizeof(abits));
    key.push_back(dtype);
    key.push_back(abits);
    for (int i = 0; i < count; ++i) {
        if (m[i] < 0 || ldx[i] < m[i] || ldy[i] < m[i]) { set_error("bad m / leading dimension"); return H2_E_BADARG; }
        if (m[i] == 0) continue;
        if (!X[i] || !Y[i] || !is_device_pointer(X[i]) || !is_device_pointer(Y[i])) {
            set_error("batched products take device X and Y");
            return H2_E_BADARG;
        }
        if (b->mats[i]->timing.on) { set_error("disable timing on batched matrices"); return H2_E_UNSUPPORTED; }
        sys.push_back(i);
        key.insert(key.end(), {i, (int64_t)(uintptr_t)X[i], ldx[i], (int64_t)(uintptr_t)Y[i], ldy[i], m[i]});
    }
    if (sys.empty()) return 0;
    // the graph runs on the batch's own stream, ordered after and before the caller's stream
    H2_CUDA_TRY(cudaEventRecord(b->ev_in, st));
    H2_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
    if (!b->mm_exec || key != b->mm_key) {
        if (b->mm_exec) { cudaGraphExecDestroy(b->mm_exec); b->mm_exec = nullptr; }
        for (int i : sys) {
            int rc = product_prepare(b->mats[i], m[i], dtype, b->origin);
            if (rc) return rc;
        }
        H2_CUDA_TRY(cudaStreamSynchronize(b->origin));
        MmCtx ctx{b, alpha, X, ldx, Y, ldy, m, dtype};
        int rc = batch_capture(b, b->origin, sys, mm_body, &ctx, &b->mm_exec);
        if (rc) return rc;
        b->mm_key = key;
    }
    H2_CUDA_TRY(cudaGraphLaunch(b->mm_exec, b->origin));
    H2_CUDA_TRY(cudaEventRecord(b->ev_out, b->origin));
    H2_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_out, 0));
    return 0;
}

int h2_batch_block_cg(h2_batch* b, const double* const* B, const int64_t* ldb, double* const* X, const int64_t* ldx,
                      const int64_t* m, const h2_cg_params* params, h2_cg_result* res) {
    return batch_block_cg(b, B, ldb, X, ldx, m, params, res);
}

namespace {

// Time one product variant (2 warm-up, 5 timed products on zero blocks).
int time_variant(h2_matrix* A, int64_t m, int32_t dtype, cudaStream_t st, double* Xb, double* Yb, cudaEvent_t e0,
                 cudaEvent_t e1, double* ms) {
    int rc = 0;
    for (int r = 0; r < 2 && !rc; ++r) rc = matmul_device(A, 1.0, Xb, m, Yb, m, m, dtype, st, false, true);
    if (rc) return rc;
    H2_CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < 5 && !rc; ++r) rc = matmul_device(A, 1.0, Xb, m, Yb, m, m, dtype, st, false, true);
    if (rc) return rc;
    H2_CUDA_TRY(cudaEventRecord(e1, st));
    H2_CUDA_TRY(cudaEventSynchronize(e1));
    float f = 0.f;
    H2_CUDA_TRY(cudaEventElapsedTime(&f, e0, e1));
    *ms = f / 5.0;
    return 0;
}

}  // namespace

int h2_autotune_ex(h2_matrix* A, int64_t m, int32_t dtype, void* stream, h2_tune_result* out) {
    if (!A || m < 1 || (dtype != H2_F32 && dtype != H2_BF16)) { set_error("h2_autotune_ex: bad argument"); return H2_E_BADARG; }
    if (dtype == H2_F32 && !A->f32.built) { set_error("FP32 copy not built"); return H2_E_UNSUPPORTED; }
    if (dtype == H2_BF16 && !A->tc.has_bf16) { set_error("BF16 copy not built"); return H2_E_UNSUPPORTED; }
    cudaStream_t st = (cudaStream_t)stream;
    if (stream_capture_active(st)) { set_error("h2_autotune_ex: not inside a stream capture"); return H2_E_BADARG; }
    const int mc = (int)std::min<int64_t>(m, 64);
    const int cls = column_class(mc);
    const int di = dtype == H2_BF16 ? 1 : 0;
    const Tune keep = A->tune[di][cls];
    const int keep_flow = A->use_flow;
    const int keep_up = A->up_target, keep_down = A->down_target;
    A->use_flow = -1;  // the candidates set the path themselves
    double* buf = nullptr;
    H2_CUDA_TRY(cudaMallocAsync((void**)&buf, 2 * (size_t)A->n * m * sizeof(double), st));
    H2_CUDA_TRY(cudaMemsetAsync(buf, 0, 2 * (size_t)A->n * m * sizeof(double), st));
    double* Xb = buf;
    double* Yb = buf + (size_t)A->n * m;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    h2_tune_result r{};
    r.dtype = dtype;
    r.m = (int32_t)m;
    int rc = 0;
    double best = -1.0;
    Tune best_t = keep;
    int best_up = keep_up, best_down = keep_down;
    auto trial = [&](Tune t, int up, int down) {
        if (rc || r.n_candidates >= 16) return;
        A->tune[di][cls] = t;
        if ((rc = set_transfer_targets(A, up, down, st))) return;
        double ms = -1.0;
        if ((rc = time_variant(A, m, dtype, st, Xb, Yb, e0, e1, &ms))) return;
        const int i = r.n_candidates++;
        r.ms[i] = ms;
        r.cand_path[i] = t.path;
        r.cand_stages[i] = t.stages;
        r.cand_up[i] = up;
        r.cand_down[i] = down;
        if (best < 0.0 || ms < best) { best = ms; best_t = t; best_up = up; best_down = down; }
    };
    // 1. the product path
    const bool tc = dtype == H2_BF16 || A->tc.has_tf32;
    if (tc) trial(Tune{kPathTcOwn, 0}, keep_up, keep_down);
    if (dtype == H2_F32 && A->tc.flow) {
        trial(Tune{kPathTcFlow, 0}, keep_up, keep_down);
        trial(Tune{kPathTcFused, 0}, keep_up, keep_down);
    }
    if (dtype == H2_F32) trial(Tune{kPathSimt, 0}, keep_up, keep_down);
    // 2. the stage count of the tensor-core kernels on the best path
    if (!rc && best_t.path != kPathSimt)
        for (int sc : {4, 5}) trial(Tune{best_t.path, (int8_t)sc}, best_up, best_down);
    // 3. the cut of the CUDA-core subtree passes, upward then downward
    const bool subtree = A->f32.Et && A->k % 8 == 0 && A->k <= 64 && mc % 4 == 0 && A->T.leaf_size <= 64;
    if (!rc && best_t.path == kPathTcOwn && subtree) {
        const int up0 = best_up;
        for (int u : {kUpTasks / 2, kUpTasks * 2}) trial(best_t, u, best_down);
        (void)up0;
        for (int d : {kDownTasks / 2, kDownTasks * 2}) trial(best_t, best_up, d);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, st);
    cudaStreamSynchronize(st);
    A->use_flow = keep_flow;
    if (rc) {
        A->tune[di][cls] = keep;
        set_transfer_targets(A, keep_up, keep_down, st);
        return rc;
    }
    A->tune[di][cls] = best_t;
    if ((rc = set_transfer_targets(A, best_up, best_down, st))) return rc;
    r.path = best_t.path;
    r.stages = best_t.stages;
    r.up_target = best_up;
    r.down_target = best_down;
    r.ms_best = best;
    if (out) *out = r;
    return 0;
}

int h2_autotune(h2_matrix* A, int64_t m, void* stream, double* ms) {
    h2_tune_result r{};
    const int rc = h2_autotune_ex(A, m, H2_F32, stream, &r);
    if (rc) return rc;
    if (ms) {
        ms[0] = ms[1] = -1.0;
        for (int i = 0; i < r.n_candidates; ++i) {
            if (r.cand_path[i] == kPathSimt) ms[1] = r.ms[i];
            else if (ms[0] < 0.0 || r.ms[i] < ms[0]) ms[0] = r.ms[i];
        }
    }
    return 0;
}

}  // extern "C"
