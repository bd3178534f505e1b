// Batches of independent systems: products captured into one CUDA graph with
// one branch per system, and the autotuner that picks the FP32 product path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <functional>
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

// The two multi-system launches of an FP32 product of the systems `sys` (with
// their buffers fb): the upward pass with the coupling phase and the downward
// pass with the leaf phase, each one work list over the items of all systems,
// merged by dependency key (system index in bits 18.. of np), with the systems'
// argument tables.  Lists and tables go to *mem (grown to *bytes as needed);
// p1 and p2 receive the launch arguments.
int flow_tables(h2_batch* b, const std::vector<int>& sys, const std::vector<FlowBufs>& fb, void** mem, size_t* bytes,
                TcGemmParams* p1, TcGemmParams* p2, cudaStream_t st) {
    const int ns = (int)sys.size();
    int Rmax = 16;
    std::vector<int32_t> k1, k2;
    std::vector<TcItem> i1, i2;
    std::vector<TcSys> t1(ns), t2(ns);
    for (int j = 0; j < ns; ++j) {
        h2_matrix* A = b->mats[sys[j]];
        const TcData& D = A->tc;
        const int32_t tag = (int32_t)((uint32_t)j << 18);
        for (size_t e = 0; e < D.f1_host.size(); ++e) {
            TcItem it = D.f1_host[e];
            it.np |= tag;
            k1.push_back(D.f1_keys[e]);
            i1.push_back(it);
        }
        for (size_t e = 0; e < D.f2_host.size(); ++e) {
            TcItem it = D.f2_host[e];
            it.np |= tag;
            k2.push_back(D.f2_keys[e]);
            i2.push_back(it);
        }
        const FlowBufs& f = fb[j];
        Rmax = std::max(Rmax, f.R);
        t1[j] = TcSys{D.f1_terms, f.xcm, f.Xcm, nullptr, D.mat32, f.xcm, f.ycp, f.fflag, f.Xp,
                      A->d_leaves, A->d_cl_off, A->d_cl_size, f.R, f.mc, A->k, D.KP, f.mc, 0};
        t2[j] = TcSys{D.f2_terms, f.ycm, f.ycp, f.Xcm, D.mat32, f.ycm, nullptr, f.fflag + A->nc, f.Xp,
                      A->d_leaves, A->d_cl_off, A->d_cl_size, f.R, f.mc, A->k, D.KP, f.mc, 0};
    }
    std::vector<TcItem> m1, m2;
    merge_by_key(k1, i1, m1);
    merge_by_key(k2, i2, m2);
    const size_t o1 = 0, o2 = o1 + m1.size() * sizeof(TcItem), o3 = o2 + m2.size() * sizeof(TcItem),
                 o4 = o3 + ns * sizeof(TcSys), need = o4 + ns * sizeof(TcSys);
    if (*bytes < need) {
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        if (*mem) cudaFree(*mem);
        *mem = nullptr;
        *bytes = 0;
        H2_CUDA_TRY(cudaMalloc(mem, need));
        *bytes = need;
    }
    char* dm = (char*)*mem;
    H2_CUDA_TRY(cudaMemcpyAsync(dm + o1, m1.data(), m1.size() * sizeof(TcItem), cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaMemcpyAsync(dm + o2, m2.data(), m2.size() * sizeof(TcItem), cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaMemcpyAsync(dm + o3, t1.data(), ns * sizeof(TcSys), cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaMemcpyAsync(dm + o4, t2.data(), ns * sizeof(TcSys), cudaMemcpyHostToDevice, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    *p1 = TcGemmParams{};
    p1->n_items = (int)m1.size();
    p1->items = (const TcItem*)(dm + o1);
    p1->sys = (const TcSys*)(dm + o3);
    p1->R = Rmax;
    p1->epoch = 1;
    p1->err = b->mats[sys[0]]->err_dev;
    *p2 = *p1;
    p2->n_items = (int)m2.size();
    p2->items = (const TcItem*)(dm + o2);
    p2->sys = (const TcSys*)(dm + o4);
    return 0;
}

// Capture into *exec: pre(j) on every system's branch, the two launches, then
// post(j) on every system's branch, all forked from and joined into b->origin.
int flow_capture(h2_batch* b, const std::vector<int>& sys, const TcGemmParams& p1, const TcGemmParams& p2,
                 const std::function<int(int, cudaStream_t)>& pre, const std::function<int(int, cudaStream_t)>& post,
                 cudaGraphExec_t* exec) {
    *exec = nullptr;
    const int ns = (int)sys.size();
    H2_CUDA_TRY(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    cudaError_t e = cudaEventRecord(b->fork, b->origin);
    for (int j = 0; j < ns && !rc && e == cudaSuccess; ++j) {
        const int i = sys[j];
        if ((e = cudaStreamWaitEvent(b->streams[i], b->fork, 0)) != cudaSuccess) break;
        if ((rc = pre(j, b->streams[i]))) break;
        if ((e = cudaEventRecord(b->join[i], b->streams[i])) != cudaSuccess) break;
        e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
    }
    if (!rc && e == cudaSuccess) rc = launch_tc_gemm(3, 1, p1, std::min(p1.n_items, kTcGrid), b->origin);
    if (!rc && e == cudaSuccess) rc = launch_tc_gemm(3, 1, p2, std::min(p2.n_items, kTcGrid), b->origin);
    if (!rc && e == cudaSuccess) e = cudaEventRecord(b->fork, b->origin);
    for (int j = 0; j < ns && !rc && e == cudaSuccess; ++j) {
        const int i = sys[j];
        if ((e = cudaStreamWaitEvent(b->streams[i], b->fork, 0)) != cudaSuccess) break;
        if ((rc = post(j, b->streams[i]))) break;
        if ((e = cudaEventRecord(b->join[i], b->streams[i])) != cudaSuccess) break;
        e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->origin, &graph);
    if (rc || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (!rc) {
            set_error(std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ee));
            rc = H2_E_CUDA;
        }
        return rc;
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        set_error(std::string("batch graph instantiate: ") + cudaGetErrorString(e));
        return H2_E_CUDA;
    }
    return 0;
}

bool flow_batch_ok(h2_batch* b, const std::vector<int>& sys, const int64_t* m, int32_t dtype) {
    bool multi = dtype == H2_F32 && b->multi_launch;
    for (int i : sys) multi = multi && flow_batchable(b->mats[i], m[i]) && b->mats[i]->use_flow != 0;
    return multi;
}

namespace {

// One FP32 product of every system with the two multi-system launches, captured
// into one graph with the systems' gathers and scatters as branches.
int batch_flow_matmul(h2_batch* b, double alpha, const double* const* X, const int64_t* ldx, double* const* Y,
                      const int64_t* ldy, const int64_t* m, const std::vector<int>& sys) {
    const int ns = (int)sys.size();
    std::vector<FlowBufs> fb(ns);
    int rc = 0;
    for (int j = 0; j < ns && !rc; ++j) rc = flow_prepare(b->mats[sys[j]], (int)m[sys[j]], b->origin, &fb[j]);
    if (rc) return rc;
    std::vector<int64_t> key;
    int64_t abits;
    memcpy(&abits, &alpha, sizeof(abits));
    key.push_back(abits);
    for (int j = 0; j < ns; ++j) {
        const int i = sys[j];
        key.insert(key.end(), {i, (int64_t)(uintptr_t)X[i], ldx[i], (int64_t)(uintptr_t)Y[i], ldy[i], m[i],
                               (int64_t)(uintptr_t)fb[j].Xp});
    }
    if (!b->flow_exec || key != b->flow_key) {
        if (b->flow_exec) { cudaGraphExecDestroy(b->flow_exec); b->flow_exec = nullptr; }
        TcGemmParams p1, p2;
        if ((rc = flow_tables(b, sys, fb, &b->flow_mem, &b->flow_bytes, &p1, &p2, b->origin))) return rc;
        auto pre = [&](int j, cudaStream_t s) { const int i = sys[j]; return flow_pre(b->mats[i], X[i], ldx[i], fb[j], s); };
        auto post = [&](int j, cudaStream_t s) {
            const int i = sys[j];
            return flow_post(b->mats[i], alpha, X[i], ldx[i], Y[i], ldy[i], fb[j], false, s);
        };
        if ((rc = flow_capture(b, sys, p1, p2, pre, post, &b->flow_exec))) return rc;
        b->flow_key = key;
    }
    H2_CUDA_TRY(cudaGraphLaunch(b->flow_exec, b->origin));
    return 0;
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
        if (int rc = refuse_complex(mats[i], "h2_batch_create")) { delete b; return rc; }
        b->mats.push_back(mats[i]);
    }
    const char* mv = getenv("H2_BATCH_MULTI");
    b->multi_launch = !(mv && mv[0] == '0');
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
    if (b->flow_exec) cudaGraphExecDestroy(b->flow_exec);
    if (b->flow_mem) cudaFree(b->flow_mem);
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
    // FP32 with the tensor-core transfer passes on every system: multi-system launches
    if (flow_batch_ok(b, sys, m, dtype)) {
        H2_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
        int rc = batch_flow_matmul(b, alpha, X, ldx, Y, ldy, m, sys);
        if (rc) return rc;
        H2_CUDA_TRY(cudaEventRecord(b->ev_out, b->origin));
        H2_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_out, 0));
        return 0;
    }
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
    if (int rc = refuse_complex(A, "h2_autotune_ex")) return rc;
    if (dtype == H2_F32 && !A->f32.built) { set_error("FP32 copy not built"); return H2_E_UNSUPPORTED; }
    if (dtype == H2_BF16 && !A->tc.has_bf16) { set_error("BF16 copy not built"); return H2_E_UNSUPPORTED; }
    cudaStream_t st = (cudaStream_t)stream;
    if (stream_capture_active(st)) { set_error("h2_autotune_ex: not inside a stream capture"); return H2_E_BADARG; }
    const int mc = (int)std::min<int64_t>(m, 64);
    const int cls = column_class(mc);
    const int di = dtype == H2_BF16 ? 1 : 0;
    const Tune keep = A->tune[di][cls];
    const int keep_flow = A->use_flow, keep_hybrid = A->use_hybrid;
    const int keep_up = A->up_target, keep_down = A->down_target;
    A->use_flow = -1;  // the candidates set the path themselves
    A->use_hybrid = -1;
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
    if (dtype == H2_F32 ? A->tc.hybrid : A->tc.hybrid_bf16) trial(Tune{kPathTcHybrid, 0}, keep_up, keep_down);
    if (dtype == H2_F32) trial(Tune{kPathSimt, 0}, keep_up, keep_down);
    // 2. the stage count of the tensor-core kernels on the best path
    if (!rc && best_t.path != kPathSimt)
        for (int sc : {4, 5}) trial(Tune{best_t.path, (int8_t)sc}, best_up, best_down);
    // 3. the cut of the CUDA-core subtree passes, upward then downward
    const bool subtree = A->f32.Et && A->k % 8 == 0 && A->k <= 64 && mc % 4 == 0 && A->T.leaf_size <= 64;
    if (!rc && (best_t.path == kPathTcOwn || best_t.path == kPathTcHybrid) && subtree) {
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
    A->use_hybrid = keep_hybrid;
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
