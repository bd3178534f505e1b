// Block CG (Sec. 5.1, Alg. "block CG") on the device, FP64 vector
// arithmetic, and the mixed-precision iterative refinement around it.
//
// Per iteration, after the block product a = A p:
//   k_cg_dots    β_i = <p_i, a_i>, α_i = <p_i, r_i>/β_i            (reduction over rows)
//   k_cg_update  x_i += α_i p_i, r_i -= α_i a_i, then γ_i = <a_i, r_i>/β_i
//                and |r_i| (reduction over rows)
//   k_cg_dir     p_i = r_i - γ_i p_i
// Reductions are two-stage and deterministic: every CTA writes its partial
// sums, the last CTA to finish (ticket counter) adds them in CTA order and
// derives the per-column scalars.  Converged columns are frozen (α_i = 0).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <vector>

#include "h2_internal.cuh"

namespace h2 {

namespace {

constexpr int kRowBlocks = 304;  // CTAs along the rows: 2 per SM on a 152-SM part
constexpr int kColsPerCta = 32;

// Row loops: this thread visits rows i = blockIdx.x·8 + threadIdx.y + k·S with
// S = 8·gridDim.x; f4(i, S) takes rows i, i+S, i+2S, i+3S at once (independent
// loads in flight), f1(i) the tail.
template <typename F4, typename F1>
__device__ __forceinline__ void rows4(int64_t n, F4 f4, F1 f1) {
    const int64_t S = (int64_t)gridDim.x * 8;
    int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.y;
    for (; i + 3 * S < n; i += 4 * S) f4(i, S);
    for (; i < n; i += S) f1(i);
}

// Reduce the block's (32 columns × 8 row lanes) partial sums over the row lanes.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double (*sm)[8][kColsPerCta]) {
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[q][ty][tx] = v[q];
    __syncthreads();
    if (ty == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int y = 0; y < 8; ++y) s += sm[q][y][tx];
            v[q] = s;
        }
    }
}

// Returns true in every thread of the CTA that finished last for this column group.
__device__ __forceinline__ bool last_cta(unsigned* ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned t = atomicAdd(&ticket[blockIdx.y], 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Sum the per-CTA partials of `col` (two components) over the nb CTAs in the
// last CTA: each of the 8 row lanes takes every 8th CTA, then the lanes are
// added in fixed order.  Called by every thread; the result is in ty == 0.
__device__ __forceinline__ void tail_sum2(const double* part, int m, int col, unsigned nb,
                                          double (*sm)[8][kColsPerCta], double& s0, double& s1) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    double a0 = 0.0, a1 = 0.0;
    if (col < m) {
#pragma unroll 4
        for (unsigned b = ty; b < nb; b += 8) {
            a0 += __ldcg(&part[((size_t)b * m + col) * 2 + 0]);
            a1 += __ldcg(&part[((size_t)b * m + col) * 2 + 1]);
        }
    }
    __syncthreads();
    sm[0][ty][tx] = a0;
    sm[1][ty][tx] = a1;
    __syncthreads();
    s0 = s1 = 0.0;
    if (ty == 0)
        for (int y = 0; y < 8; ++y) {
            s0 += sm[0][y][tx];
            s1 += sm[1][y][tx];
        }
}

// Column norms |B_i|, |R_i| and the initial activity flags (two-stage, fixed order).
__global__ void __launch_bounds__(256) k_cg_init(const double* __restrict__ B, int64_t ldb,
                                                 const double* __restrict__ R, int64_t ldr, int64_t n, int m,
                                                 double tol, CgDev d) {
    __shared__ double sm[2][8][kColsPerCta];
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (col < m)
        rows4(n, [&](int64_t i_, int64_t S_) {
            double b[4], r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { b[u] = B[(i_ + u * S_) * ldb + col]; r[u] = R[(i_ + u * S_) * ldr + col]; }
#pragma unroll
            for (int u = 0; u < 4; ++u) { v[0] = fma(b[u], b[u], v[0]); v[1] = fma(r[u], r[u], v[1]); } }, [&](int64_t i_) {
            const double b = B[i_ * ldb + col], r = R[i_ * ldr + col];
            v[0] = fma(b, b, v[0]); v[1] = fma(r, r, v[1]); });
    block_reduce<2>(v, sm);
    if (threadIdx.y == 0 && col < m) {
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 0] = v[0];
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 1] = v[1];
    }
    if (!last_cta(d.ticket)) return;
    double bb, rr;
    tail_sum2(d.partial, m, col, gridDim.x, sm, bb, rr);
    if (threadIdx.y == 0 && col < m) {
        const double bn = bb > 0.0 ? sqrt(bb) : 1.0;
        d.bnorm[col] = bn;
        d.rnorm[col] = sqrt(rr);
        const int act = !(sqrt(rr) / bn <= tol);
        d.active[col] = act;
        d.conv_iter[col] = 0;
        d.alpha[col] = d.beta[col] = d.gamma[col] = 0.0;
        if (act) atomicAdd(&d.summary[0], 1);
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) d.ticket[blockIdx.y] = 0;
}

__global__ void __launch_bounds__(256) k_cg_dots(const double* __restrict__ P, const double* __restrict__ AP,
                                                 const double* __restrict__ R, int64_t ld, int64_t n, int m,
                                                 CgDev d) {
    __shared__ double sm[2][8][kColsPerCta];
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (col < m && d.active[col])
        rows4(n, [&](int64_t i_, int64_t S_) {
            double p[4], a[4], r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = (i_ + u * S_) * ld + col;
                p[u] = P[e]; a[u] = AP[e]; r[u] = R[e];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) { v[0] = fma(p[u], a[u], v[0]); v[1] = fma(p[u], r[u], v[1]); } }, [&](int64_t i_) {
            const double p = P[i_ * ld + col];
            v[0] = fma(p, AP[i_ * ld + col], v[0]);
            v[1] = fma(p, R[i_ * ld + col], v[1]); });
    block_reduce<2>(v, sm);
    if (threadIdx.y == 0 && col < m) {
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 0] = v[0];
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 1] = v[1];
    }
    if (!last_cta(d.ticket)) return;
    double pa, pr;
    tail_sum2(d.partial, m, col, gridDim.x, sm, pa, pr);
    if (threadIdx.y == 0 && col < m) {
        double alpha = 0.0;
        if (d.active[col]) {
            if (!(pa > 0.0) || !isfinite(pa) || !isfinite(pr)) {
                atomicOr(&d.summary[1], 1);
            } else {
                alpha = pr / pa;
            }
        }
        d.beta[col] = pa;
        d.alpha[col] = alpha;
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) d.ticket[blockIdx.y] = 0;
}

__global__ void __launch_bounds__(256) k_cg_update(double* __restrict__ X, int64_t ldx, const double* __restrict__ P,
                                                   const double* __restrict__ AP, double* __restrict__ R,
                                                   int64_t ld, int64_t n, int m, double tol, int iter, CgDev d) {
    __shared__ double sm[2][8][kColsPerCta];
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (col < m && d.active[col]) {
        const double a = d.alpha[col];
        rows4(n, [&](int64_t i_, int64_t S_) {
            double p[4], ap[4], r[4], x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = (i_ + u * S_) * ld + col;
                p[u] = P[e]; ap[u] = AP[e]; r[u] = R[e]; x[u] = X[(i_ + u * S_) * ldx + col];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                X[(i_ + u * S_) * ldx + col] = fma(a, p[u], x[u]);
                r[u] = fma(-a, ap[u], r[u]);
                R[(i_ + u * S_) * ld + col] = r[u];
                v[0] = fma(ap[u], r[u], v[0]);
                v[1] = fma(r[u], r[u], v[1]);
            } }, [&](int64_t i_) {
            const double p = P[i_ * ld + col], ap = AP[i_ * ld + col];
            X[i_ * ldx + col] = fma(a, p, X[i_ * ldx + col]);
            const double r = fma(-a, ap, R[i_ * ld + col]);
            R[i_ * ld + col] = r;
            v[0] = fma(ap, r, v[0]);
            v[1] = fma(r, r, v[1]); });
    }
    block_reduce<2>(v, sm);
    if (threadIdx.y == 0 && col < m) {
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 0] = v[0];
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 1] = v[1];
    }
    if (!last_cta(d.ticket)) return;
    double ar, rr;
    tail_sum2(d.partial, m, col, gridDim.x, sm, ar, rr);
    if (threadIdx.y == 0 && col < m && d.active[col]) {
        const double gamma = ar / d.beta[col];
        d.gamma[col] = gamma;
        const double rn = sqrt(rr);
        d.rnorm[col] = rn;
        if (!isfinite(gamma) || !isfinite(rn)) atomicOr(&d.summary[1], 1);
        d.conv_iter[col] += 1;  // iterations while active (graph-replay safe, no baked counter)
        if (rn / d.bnorm[col] <= tol) {
            d.active[col] = 0;
            atomicSub(&d.summary[0], 1);
        }
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) d.ticket[blockIdx.y] = 0;
}

// p_i = r_i - γ_i p_i for columns that are still active.
__global__ void k_cg_dir(double* __restrict__ P, const double* __restrict__ R, int64_t ld, int64_t n, int m,
                         CgDev d) {
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    if (col >= m || !d.active[col]) return;
    const double g = d.gamma[col];
    rows4(n, [&](int64_t i_, int64_t S_) {
        double p[4], r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { p[u] = P[(i_ + u * S_) * ld + col]; r[u] = R[(i_ + u * S_) * ld + col]; }
#pragma unroll
        for (int u = 0; u < 4; ++u) P[(i_ + u * S_) * ld + col] = fma(-g, p[u], r[u]); }, [&](int64_t i_) {
        P[i_ * ld + col] = fma(-g, P[i_ * ld + col], R[i_ * ld + col]); });
}

// Reliable update of mixed-precision CG: the recurrence residual of every
// column is replaced by the true FP64 residual Rt = B - A X; a column whose
// true residual meets the tolerance is frozen, one that the recurrence had
// frozen but whose true residual does not is restarted with p = r.  One CTA
// column group per 32 columns; the norms are reduced in fixed order.
__global__ void __launch_bounds__(256) k_cg_reliable(const double* __restrict__ Rt, double* __restrict__ R,
                                                     double* __restrict__ P, int64_t ld, int64_t n, int m,
                                                     double tol, double* __restrict__ rupd, CgDev d) {
    __shared__ double sm[2][8][kColsPerCta];
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    double v[1] = {0.0};
    if (col < m)
        for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < n; i += (int64_t)gridDim.x * 8) {
            const double r = Rt[i * ld + col];
            v[0] = fma(r, r, v[0]);
        }
    block_reduce<1>(v, sm);
    if (threadIdx.y == 0 && col < m) {
        d.partial[((size_t)blockIdx.x * m + col) * 2] = v[0];
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 1] = 0.0;
    }
    if (!last_cta(d.ticket)) return;
    double rr, unused;
    tail_sum2(d.partial, m, col, gridDim.x, sm, rr, unused);
    if (threadIdx.y == 0 && col < m) {
        const double rn = sqrt(rr);
        d.rnorm[col] = rn;
        rupd[col] = rn;
        const int now = !(rn / d.bnorm[col] <= tol);
        const int was = d.active[col];
        // reactivated columns restart their direction (flag 2 = copy r into p)
        d.active[col] = now ? (was ? 1 : 2) : 0;
        if (now) atomicAdd(&d.summary[0], 1);
        if (!isfinite(rn)) atomicOr(&d.summary[1], 1);
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) d.ticket[blockIdx.y] = 0;
}

// R = Rt for every column; P = R for restarted columns (active flag 2 -> 1).
__global__ void k_cg_reliable_copy(const double* __restrict__ Rt, double* __restrict__ R, double* __restrict__ P,
                                   int64_t ld, int64_t n, int m, CgDev d) {
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    if (col >= m) return;
    const bool restart = d.active[col] == 2;
    for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < n; i += (int64_t)gridDim.x * 8) {
        const double r = Rt[i * ld + col];
        R[i * ld + col] = r;
        if (restart) P[i * ld + col] = r;
    }
}

// P = Z for restarted columns (active flag 2), preconditioned restart.
__global__ void k_cg_restart_from(const double* __restrict__ Z, double* __restrict__ P, int64_t ld, int64_t n, int m,
                                  CgDev d) {
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    if (col >= m || d.active[col] != 2) return;
    for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < n; i += (int64_t)gridDim.x * 8) P[i * ld + col] = Z[i * ld + col];
}

__global__ void k_cg_reliable_flags(int m, CgDev d) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col < m && d.active[col] == 2) d.active[col] = 1;
}

// Y[:, :] = X (2-D copy with leading dimensions), also used to zero-fill when X == nullptr.
__global__ void k_copy2d(const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy, int64_t n,
                         int m) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m;
        const int c = (int)(e % m);
        Y[i * ldy + c] = X ? X[i * ldx + c] : 0.0;
    }
}

// X += D
__global__ void k_axpy2d(const double* __restrict__ D, int64_t ldd, double* __restrict__ X, int64_t ldx, int64_t n,
                         int m) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m;
        const int c = (int)(e % m);
        X[i * ldx + c] += D[i * ldd + c];
    }
}

// Relative residual per column |R_i| / |B_i| (|B_i| = 0 read as 1), two-stage.
__global__ void __launch_bounds__(256) k_col_relnorm(const double* __restrict__ R, int64_t ldr,
                                                     const double* __restrict__ B, int64_t ldb, int64_t n, int m,
                                                     double* __restrict__ out, CgDev d) {
    __shared__ double sm[2][8][kColsPerCta];
    const int col = blockIdx.y * kColsPerCta + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (col < m)
        rows4(n, [&](int64_t i_, int64_t S_) {
            double b[4], r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { b[u] = B[(i_ + u * S_) * ldb + col]; r[u] = R[(i_ + u * S_) * ldr + col]; }
#pragma unroll
            for (int u = 0; u < 4; ++u) { v[0] = fma(r[u], r[u], v[0]); v[1] = fma(b[u], b[u], v[1]); } }, [&](int64_t i_) {
            const double b = B[i_ * ldb + col], r = R[i_ * ldr + col];
            v[0] = fma(r, r, v[0]); v[1] = fma(b, b, v[1]); });
    block_reduce<2>(v, sm);
    if (threadIdx.y == 0 && col < m) {
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 0] = v[0];
        d.partial[((size_t)blockIdx.x * m + col) * 2 + 1] = v[1];
    }
    if (!last_cta(d.ticket)) return;
    double rr, bb;
    tail_sum2(d.partial, m, col, gridDim.x, sm, rr, bb);
    if (threadIdx.y == 0 && col < m) {
        out[col] = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) d.ticket[blockIdx.y] = 0;
}

struct Solver {
    h2_matrix* A;
    cudaStream_t st;
    int64_t n;
    int m;
    bool trans = false;  // products with Aᵀ (adjoint solve)
    bool gram = false;   // variant H2_CG_GRAM (m <= 64)
    bool pcg = false;    // block-Jacobi preconditioned block CG (Alg. "pcg block")
    double* Z = nullptr; // [n×m] M⁻¹ R when pcg
    bool pc_low = false; // M⁻¹ in FP32 (the low-precision iterations of a mixed solve)
    CgDev d{};
    GramDev g{};
    double *R = nullptr, *P = nullptr, *AP = nullptr;
    int* h_summary = nullptr;  // pinned
    void* mem = nullptr;
    int h2mm_calls = 0;

    int init() {
        const size_t nm = (size_t)n * m;
        const int groups = (m + kColsPerCta - 1) / kColsPerCta;
        // carve one allocation into 256-byte aligned pieces; offsets first, then the total
        size_t off = 0;
        auto piece = [&](size_t b) { const size_t o = off; off += (b + 255) & ~(size_t)255; return o; };
        const size_t oR = piece(nm * sizeof(double)), oP = piece(nm * sizeof(double)),
                     oAP = piece(nm * sizeof(double));
        const size_t oBn = piece(m * sizeof(double)), oAl = piece(m * sizeof(double)),
                     oBe = piece(m * sizeof(double)), oGa = piece(m * sizeof(double)),
                     oRn = piece(m * sizeof(double));
        const size_t oAct = piece(m * sizeof(int)), oCi = piece(m * sizeof(int)), oSum = piece(4 * sizeof(int));
        const size_t oPart = piece((size_t)kRowBlocks * m * 2 * sizeof(double));
        const size_t oTk = piece(groups * sizeof(unsigned));
        if (gram && m > kGramMaxCols) {
            set_error("the Gram-matrix block CG takes at most 64 columns");
            return H2_E_UNSUPPORTED;
        }
        const size_t oGram = gram ? piece(gram_scratch_bytes(m)) : 0;
        const size_t oZ = pcg ? piece(nm * sizeof(double)) : 0;
        if (pcg) {
            int rc = bj_prepare(A, st);
            if (rc) return rc;
        }
        if (gram) {
            int rc = gram_prepare();
            if (rc) return rc;
        }
        H2_CUDA_TRY(cudaMallocAsync(&mem, off, st));
        char* p = (char*)mem;
        R = (double*)(p + oR);
        P = (double*)(p + oP);
        AP = (double*)(p + oAP);
        d.bnorm = (double*)(p + oBn);
        d.alpha = (double*)(p + oAl);
        d.beta = (double*)(p + oBe);
        d.gamma = (double*)(p + oGa);
        d.rnorm = (double*)(p + oRn);
        d.active = (int*)(p + oAct);
        d.conv_iter = (int*)(p + oCi);
        d.summary = (int*)(p + oSum);
        d.partial = (double*)(p + oPart);
        d.ticket = (unsigned*)(p + oTk);
        if (gram) gram_carve(&g, p + oGram, m);
        if (pcg) Z = (double*)(p + oZ);
        H2_CUDA_TRY(cudaMemsetAsync(d.ticket, 0, groups * sizeof(unsigned), st));
        H2_CUDA_TRY(cudaHostAlloc(&h_summary, 4 * sizeof(int), cudaHostAllocDefault));
        return 0;
    }
    ~Solver() {
        if (mem) cudaFreeAsync(mem, st);
        if (h_summary) cudaFreeHost(h_summary);
    }

    dim3 grid2d() const { return dim3(kRowBlocks, (m + kColsPerCta - 1) / kColsPerCta); }
    unsigned copy_grid() const { return (unsigned)std::min<int64_t>(((int64_t)n * m + 255) / 256, 152 * 16); }

    // R = B - A X (product in dtype, FP64 by default)
    int residual(const double* B, int64_t ldb, const double* X, int64_t ldx, int32_t dtype = H2_F64) {
        k_copy2d<<<copy_grid(), 256, 0, st>>>(B, ldb, R, m, n, m);
        H2_LAUNCH_CHECK();
        ++h2mm_calls;
        return matmul_device(A, -1.0, X, ldx, R, m, m, dtype, st, trans, false);
    }

    // rel[i] = |R_i| / |b_i| on the host (R as the last residual() left it)
    int true_rel(const double* B, int64_t ldb, double* rel) {
        double* d_rel = nullptr;
        H2_CUDA_TRY(cudaMallocAsync(&d_rel, m * sizeof(double), st));
        k_col_relnorm<<<grid2d(), dim3(kColsPerCta, 8), 0, st>>>(R, m, B, ldb, n, m, d_rel, d);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(rel, d_rel, m * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(d_rel, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("true residual: ") + cudaGetErrorString(e));
            return H2_E_CUDA;
        }
        return 0;
    }

    // Mixed-precision block CG with reliable updates: products in dtype, FP64
    // vectors; the recurrence residuals are replaced by the true FP64
    // residual B - A X whenever the largest active one has fallen by a factor
    // delta since the last replacement, or when every column looks converged.
    // Convergence is decided on the true residual.  R must hold B - A X.
    int cg_reliable(int32_t dtype, const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int max_iter,
                    int check_every, double delta, double* Rt, double* rupd, int* iters, int* updates) {
        if (gram) return cg_gram(dtype, B, ldb, X, ldx, tol, max_iter, check_every, delta, Rt, rupd, iters, updates);
        if (pcg) return cg_pcg(dtype, B, ldb, X, ldx, tol, max_iter, check_every, delta, Rt, rupd, iters, updates);
        const dim3 blk(kColsPerCta, 8);
        const dim3 grid(kRowBlocks, (m + kColsPerCta - 1) / kColsPerCta);
        H2_CUDA_TRY(cudaMemsetAsync(d.summary, 0, 4 * sizeof(int), st));
        k_cg_init<<<grid2d(), dim3(kColsPerCta, 8), 0, st>>>(B, ldb, R, m, n, m, tol, d);
        H2_LAUNCH_CHECK();
        k_copy2d<<<copy_grid(), 256, 0, st>>>(R, m, P, m, n, m);
        H2_LAUNCH_CHECK();
        H2_CUDA_TRY(cudaMemcpyAsync(rupd, d.rnorm, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<double> rn(m), ru(m);
        std::vector<int> act(m);
        int it = 0, status = 0, restarts = 0;
        const int max_restarts = std::max(10, max_iter / 50);
        *updates = 0;
        if (h_summary[0] > 0) {
            for (it = 1; it <= max_iter; ++it) {
                ++h2mm_calls;
                int rc = matmul_device(A, 1.0, P, m, AP, m, m, dtype, st, trans, true);
                if (rc) return rc;
                k_cg_dots<<<grid, blk, 0, st>>>(P, AP, R, m, n, m, d);
                H2_LAUNCH_CHECK();
                k_cg_update<<<grid, blk, 0, st>>>(X, ldx, P, AP, R, m, n, m, tol, it, d);
                H2_LAUNCH_CHECK();
                k_cg_dir<<<grid, blk, 0, st>>>(P, R, m, n, m, d);
                H2_LAUNCH_CHECK();
                if (it % check_every != 0 && it != max_iter) continue;
                H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaMemcpyAsync(rn.data(), d.rnorm, m * sizeof(double), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaMemcpyAsync(ru.data(), rupd, m * sizeof(double), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaMemcpyAsync(act.data(), d.active, m * sizeof(int), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaStreamSynchronize(st));
                if (h_summary[1]) {
                    if (++restarts > max_restarts) { status = H2_E_BREAKDOWN; break; }
                    ++*updates;
                    if ((rc = restart_all(B, ldb, X, ldx, tol, Rt, rupd))) return rc;
                    H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaStreamSynchronize(st));
                    if (h_summary[0] == 0) break;
                    continue;
                }
                bool update = h_summary[0] == 0;
                for (int i = 0; i < m && !update; ++i) update = act[i] && rn[i] < delta * ru[i];
                if (!update) continue;
                // true residual in FP64, then replace
                k_copy2d<<<copy_grid(), 256, 0, st>>>(B, ldb, Rt, m, n, m);
                H2_LAUNCH_CHECK();
                ++h2mm_calls;
                ++*updates;
                if ((rc = matmul_device(A, -1.0, X, ldx, Rt, m, m, H2_F64, st, trans, false))) return rc;
                H2_CUDA_TRY(cudaMemsetAsync(d.summary, 0, sizeof(int), st));
                k_cg_reliable<<<grid, blk, 0, st>>>(Rt, R, P, m, n, m, tol, rupd, d);
                H2_LAUNCH_CHECK();
                k_cg_reliable_copy<<<grid, blk, 0, st>>>(Rt, R, P, m, n, m, d);
                H2_LAUNCH_CHECK();
                k_cg_reliable_flags<<<(m + 63) / 64, 64, 0, st>>>(m, d);
                H2_LAUNCH_CHECK();
                H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaStreamSynchronize(st));
                if (h_summary[1]) { status = H2_E_BREAKDOWN; break; }
                if (h_summary[0] == 0) break;
            }
            if (it > max_iter) { it = max_iter; status = H2_E_NOCONVERGE; }
        }
        *iters = it;
        return status;
    }

    // Column-wise block CG on A_dtype X = B with R already holding B - A X.
    // Returns 0 / H2_E_BREAKDOWN / H2_E_NOCONVERGE; *iters = iterations run.
    int cg(int32_t dtype, const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int max_iter,
           int check_every, int* iters) {
        if (gram || pcg) {
            int upd = 0;
            if (gram) return cg_gram(dtype, B, ldb, X, ldx, tol, max_iter, check_every, 0.0, nullptr, nullptr, iters, &upd);
            return cg_pcg(dtype, B, ldb, X, ldx, tol, max_iter, check_every, 0.0, nullptr, nullptr, iters, &upd);
        }
        const dim3 blk(kColsPerCta, 8);
        const dim3 grid(kRowBlocks, (m + kColsPerCta - 1) / kColsPerCta);
        H2_CUDA_TRY(cudaMemsetAsync(d.summary, 0, 4 * sizeof(int), st));
        k_cg_init<<<grid2d(), dim3(kColsPerCta, 8), 0, st>>>(B, ldb, R, m, n, m, tol, d);
        H2_LAUNCH_CHECK();
        k_copy2d<<<copy_grid(), 256, 0, st>>>(R, m, P, m, n, m);
        H2_LAUNCH_CHECK();
        H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        int it = 0;
        int status = 0;
        // H2_CG_TRACE=k prints the largest relative recurrence residual every k checks
        const char* tr = getenv("H2_CG_TRACE");
        const int trace = tr ? atoi(tr) : 0;
        if (h_summary[0] > 0) {
            for (it = 1; it <= max_iter; ++it) {
                ++h2mm_calls;
                int rc = matmul_device(A, 1.0, P, m, AP, m, m, dtype, st, trans, true);
                if (rc) return rc;
                k_cg_dots<<<grid, blk, 0, st>>>(P, AP, R, m, n, m, d);
                H2_LAUNCH_CHECK();
                k_cg_update<<<grid, blk, 0, st>>>(X, ldx, P, AP, R, m, n, m, tol, it, d);
                H2_LAUNCH_CHECK();
                k_cg_dir<<<grid, blk, 0, st>>>(P, R, m, n, m, d);
                H2_LAUNCH_CHECK();
                if (it % check_every == 0 || it == max_iter) {
                    H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaStreamSynchronize(st));
                    if (trace && (it % trace == 0 || it <= 3)) {
                        std::vector<double> rn(m), bn(m);
                        double a0 = 0, b0 = 0, g0 = 0;
                        cudaMemcpy(rn.data(), d.rnorm, m * sizeof(double), cudaMemcpyDeviceToHost);
                        cudaMemcpy(bn.data(), d.bnorm, m * sizeof(double), cudaMemcpyDeviceToHost);
                        cudaMemcpy(&a0, d.alpha, sizeof(double), cudaMemcpyDeviceToHost);
                        cudaMemcpy(&b0, d.beta, sizeof(double), cudaMemcpyDeviceToHost);
                        cudaMemcpy(&g0, d.gamma, sizeof(double), cudaMemcpyDeviceToHost);
                        double mx = 0.0;
                        for (int i = 0; i < m; ++i) mx = std::max(mx, rn[i] / bn[i]);
                        fprintf(stderr, "[h2 cg] dtype %d iter %d active %d max |r|/|b| %.3e  col0 alpha %.3e beta %.3e gamma %.3e |r| %.3e |b| %.3e\n", dtype, it,
                                h_summary[0], mx, a0, b0, g0, rn[0], bn[0]);
                    }
                    if (h_summary[1]) { status = H2_E_BREAKDOWN; break; }
                    if (h_summary[0] == 0) break;
                }
            }
            if (it > max_iter) { it = max_iter; status = H2_E_NOCONVERGE; }
        }
        // iterations actually needed: the largest convergence iteration
        std::vector<int> ci(m);
        H2_CUDA_TRY(cudaMemcpyAsync(ci.data(), d.conv_iter, m * sizeof(int), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        int mx = 0;
        for (int v : ci) mx = std::max(mx, v);
        *iters = status == 0 ? mx : it;
        return status;
    }

    // Replace the recurrence residuals by the true FP64 residual Rt = B - A X
    // (reliable update, see cg_reliable); the Gram variant also clears the
    // directions of columns that left the active set.
    int reliable_update(const double* B, int64_t ldb, const double* X, int64_t ldx, double tol, double* Rt,
                        double* rupd) {
        const dim3 blk(kColsPerCta, 8);
        const dim3 grid(kRowBlocks, (m + kColsPerCta - 1) / kColsPerCta);
        k_copy2d<<<copy_grid(), 256, 0, st>>>(B, ldb, Rt, m, n, m);
        H2_LAUNCH_CHECK();
        ++h2mm_calls;
        int rc = matmul_device(A, -1.0, X, ldx, Rt, m, m, H2_F64, st, trans, false);
        if (rc) return rc;
        H2_CUDA_TRY(cudaMemsetAsync(d.summary, 0, sizeof(int), st));
        k_cg_reliable<<<grid, blk, 0, st>>>(Rt, R, P, m, n, m, tol, rupd, d);
        H2_LAUNCH_CHECK();
        k_cg_reliable_copy<<<grid, blk, 0, st>>>(Rt, R, P, m, n, m, d);
        H2_LAUNCH_CHECK();
        if (pcg) {
            // restarted columns take the preconditioned residual as direction
            if ((rc = bj_apply(A, R, Z, n, m, nullptr, d, st, pc_low))) return rc;
            k_cg_restart_from<<<grid, blk, 0, st>>>(Z, P, m, n, m, d);
            H2_LAUNCH_CHECK();
        }
        k_cg_reliable_flags<<<(m + 63) / 64, 64, 0, st>>>(m, d);
        H2_LAUNCH_CHECK();
        if (gram && (rc = gram_mask(P, n, m, d, st))) return rc;
        return 0;
    }

    // After a low-precision step lost positive curvature (<p, A_dtype p> <= 0:
    // the product's error exceeds the smallest eigenvalue on p), replace the
    // residual by the FP64 one and restart every direction from it (M⁻¹r with
    // a preconditioner).  X is untouched by the failed step (α = 0 there).
    int restart_all(const double* B, int64_t ldb, const double* X, int64_t ldx, double tol, double* Rt,
                    double* rupd) {
        H2_CUDA_TRY(cudaMemsetAsync(d.summary + 1, 0, sizeof(int), st));
        int rc = reliable_update(B, ldb, X, ldx, tol, Rt, rupd);
        if (rc) return rc;
        const double* src = R;
        if (pcg) {
            if ((rc = bj_apply(A, R, Z, n, m, nullptr, d, st, pc_low))) return rc;
            src = Z;
        }
        if (gram) return gram_start(P, src, n, m, g, d, st);
        k_copy2d<<<copy_grid(), 256, 0, st>>>(src, m, P, m, n, m);
        H2_LAUNCH_CHECK();
        return 0;
    }

    // Preconditioned block CG (Alg. "pcg block") with the block-Jacobi M:
    // per iteration a = A p; β = <p, a>, α = <p, r>/β; x += αp, r -= αa;
    // z = M⁻¹ r; γ = <a, z>/β; p = z - γp (the paper's form with q = M⁻¹r).
    // R holds B - A X on entry; Rt != nullptr adds reliable updates.
    int cg_pcg(int32_t dtype, const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int max_iter,
               int check_every, double delta, double* Rt, double* rupd, int* iters, int* updates) {
        const dim3 blk(kColsPerCta, 8);
        const dim3 grid(kRowBlocks, (m + kColsPerCta - 1) / kColsPerCta);
        H2_CUDA_TRY(cudaMemsetAsync(d.summary, 0, 4 * sizeof(int), st));
        k_cg_init<<<grid2d(), dim3(kColsPerCta, 8), 0, st>>>(B, ldb, R, m, n, m, tol, d);
        H2_LAUNCH_CHECK();
        int rc = bj_apply(A, R, Z, n, m, nullptr, d, st, pc_low);
        if (rc) return rc;
        k_copy2d<<<copy_grid(), 256, 0, st>>>(Z, m, P, m, n, m);
        H2_LAUNCH_CHECK();
        if (Rt) H2_CUDA_TRY(cudaMemcpyAsync(rupd, d.rnorm, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<double> rn(m), ru(m);
        std::vector<int> act(m);
        int it = 0, status = 0, restarts = 0;
        const int max_restarts = std::max(10, max_iter / 50);
        *updates = 0;
        if (h_summary[0] > 0) {
            for (it = 1; it <= max_iter; ++it) {
                ++h2mm_calls;
                if ((rc = matmul_device(A, 1.0, P, m, AP, m, m, dtype, st, trans, true))) return rc;
                k_cg_dots<<<grid, blk, 0, st>>>(P, AP, R, m, n, m, d);
                H2_LAUNCH_CHECK();
                k_cg_update<<<grid, blk, 0, st>>>(X, ldx, P, AP, R, m, n, m, tol, it, d);
                H2_LAUNCH_CHECK();
                if ((rc = bj_apply(A, R, Z, n, m, AP, d, st, pc_low))) return rc;
                k_cg_dir<<<grid, blk, 0, st>>>(P, Z, m, n, m, d);
                H2_LAUNCH_CHECK();
                if (it % check_every != 0 && it != max_iter) continue;
                H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                if (Rt) {
                    H2_CUDA_TRY(cudaMemcpyAsync(rn.data(), d.rnorm, m * sizeof(double), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaMemcpyAsync(ru.data(), rupd, m * sizeof(double), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaMemcpyAsync(act.data(), d.active, m * sizeof(int), cudaMemcpyDeviceToHost, st));
                }
                H2_CUDA_TRY(cudaStreamSynchronize(st));
                if (h_summary[1]) {
                    if (!Rt || ++restarts > max_restarts) { status = H2_E_BREAKDOWN; break; }
                    ++*updates;
                    if ((rc = restart_all(B, ldb, X, ldx, tol, Rt, rupd))) return rc;
                    H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaStreamSynchronize(st));
                    if (h_summary[0] == 0) break;
                    continue;
                }
                if (!Rt) {
                    if (h_summary[0] == 0) break;
                    continue;
                }
                bool update = h_summary[0] == 0;
                for (int i = 0; i < m && !update; ++i) update = act[i] && rn[i] < delta * ru[i];
                if (!update) continue;
                ++*updates;
                if ((rc = reliable_update(B, ldb, X, ldx, tol, Rt, rupd))) return rc;
                H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaStreamSynchronize(st));
                if (h_summary[1]) { status = H2_E_BREAKDOWN; break; }
                if (h_summary[0] == 0) break;
            }
            if (it > max_iter) { it = max_iter; status = H2_E_NOCONVERGE; }
        }
        std::vector<int> ci(m);
        H2_CUDA_TRY(cudaMemcpyAsync(ci.data(), d.conv_iter, m * sizeof(int), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        int mx = 0;
        for (int v : ci) mx = std::max(mx, v);
        *iters = (status == 0 && !Rt) ? mx : it;
        return status;
    }

    // Gram-matrix block CG (variant H2_CG_GRAM, h2_gram.cu) on A_dtype X = B
    // with R holding B - A X.  With Rt != nullptr the recurrence residuals are
    // replaced by the FP64 residual as in cg_reliable (convergence is then
    // decided on the true residual).
    int cg_gram(int32_t dtype, const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int max_iter,
                int check_every, double delta, double* Rt, double* rupd, int* iters, int* updates) {
        H2_CUDA_TRY(cudaMemsetAsync(d.summary, 0, 4 * sizeof(int), st));
        k_cg_init<<<grid2d(), dim3(kColsPerCta, 8), 0, st>>>(B, ldb, R, m, n, m, tol, d);
        H2_LAUNCH_CHECK();
        int rc = 0;
        if (pcg && (rc = bj_apply(A, R, Z, n, m, nullptr, d, st, pc_low))) return rc;
        if ((rc = gram_start(P, pcg ? Z : R, n, m, g, d, st))) return rc;
        if (Rt) H2_CUDA_TRY(cudaMemcpyAsync(rupd, d.rnorm, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<double> rn(m), ru(m);
        std::vector<int> act(m);
        int it = 0, status = 0, restarts = 0;
        const int max_restarts = std::max(10, max_iter / 50);
        *updates = 0;
        if (h_summary[0] > 0) {
            for (it = 1; it <= max_iter; ++it) {
                ++h2mm_calls;
                if ((rc = matmul_device(A, 1.0, P, m, AP, m, m, dtype, st, trans, true))) return rc;
                if ((rc = gram_alpha(P, AP, R, n, m, g, d, st))) return rc;
                if (pcg) {
                    if ((rc = gram_update(X, ldx, P, AP, R, n, m, g, st))) return rc;
                    if ((rc = bj_apply(A, R, Z, n, m, nullptr, d, st, pc_low))) return rc;
                    if ((rc = gram_gamma_dir_from(P, AP, Z, n, m, tol, g, d, st))) return rc;
                } else if ((rc = gram_update_dir(X, ldx, P, AP, R, n, m, tol, g, d, st))) {
                    return rc;
                }
                if (it % check_every != 0 && it != max_iter) continue;
                H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                if (Rt) {
                    H2_CUDA_TRY(cudaMemcpyAsync(rn.data(), d.rnorm, m * sizeof(double), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaMemcpyAsync(ru.data(), rupd, m * sizeof(double), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaMemcpyAsync(act.data(), d.active, m * sizeof(int), cudaMemcpyDeviceToHost, st));
                }
                H2_CUDA_TRY(cudaStreamSynchronize(st));
                if (h_summary[1]) {
                    if (!Rt || ++restarts > max_restarts) { status = H2_E_BREAKDOWN; break; }
                    ++*updates;
                    if ((rc = restart_all(B, ldb, X, ldx, tol, Rt, rupd))) return rc;
                    H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                    H2_CUDA_TRY(cudaStreamSynchronize(st));
                    if (h_summary[0] == 0) break;
                    continue;
                }
                if (!Rt) {
                    if (h_summary[0] == 0) break;
                    continue;
                }
                bool update = h_summary[0] == 0;
                for (int i = 0; i < m && !update; ++i) update = act[i] && rn[i] < delta * ru[i];
                if (!update) continue;
                ++*updates;
                if ((rc = reliable_update(B, ldb, X, ldx, tol, Rt, rupd))) return rc;
                H2_CUDA_TRY(cudaMemcpyAsync(h_summary, d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaStreamSynchronize(st));
                if (h_summary[1]) { status = H2_E_BREAKDOWN; break; }
                if (h_summary[0] == 0) break;
            }
            if (it > max_iter) { it = max_iter; status = H2_E_NOCONVERGE; }
        }
        std::vector<int> ci(m);
        H2_CUDA_TRY(cudaMemcpyAsync(ci.data(), d.conv_iter, m * sizeof(int), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        int mx = 0;
        for (int v : ci) mx = std::max(mx, v);
        *iters = (status == 0 && !Rt) ? mx : it;
        return status;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Batched block CG over independent systems: every iteration of all unconverged
// systems (product + the three column-wise kernels) is one CUDA graph launch.
// ---------------------------------------------------------------------------
namespace {

struct BatchSys {
    Solver* S = nullptr;
    const double* B = nullptr;
    int64_t ldb = 0;
    double* X = nullptr;
    int64_t ldx = 0;
    double* Rt = nullptr;  // true residual buffer [n×m] followed by rupd [m]
    double* rupd = nullptr;
    bool done = false;
    int status = 0, iters = 0, updates = 0;
};

struct BatchIterCtx {
    std::vector<BatchSys>* sys;
    int32_t dtype;
    double tol;
};

// The iteration's vector work after AP = A·P (Gram or column-wise).
int batch_iter_after_product(BatchIterCtx* c, int i, cudaStream_t st) {
    Solver& S = *(*c->sys)[i].S;
    if (S.gram) {
        int rc = gram_alpha(S.P, S.AP, S.R, S.n, S.m, S.g, S.d, st);
        if (rc) return rc;
        return gram_update_dir((*c->sys)[i].X, (*c->sys)[i].ldx, S.P, S.AP, S.R, S.n, S.m, c->tol, S.g, S.d, st);
    }
    const dim3 blk(kColsPerCta, 8);
    const dim3 grid(kRowBlocks, (S.m + kColsPerCta - 1) / kColsPerCta);
    k_cg_dots<<<grid, blk, 0, st>>>(S.P, S.AP, S.R, S.m, S.n, S.m, S.d);
    H2_LAUNCH_CHECK();
    k_cg_update<<<grid, blk, 0, st>>>((*c->sys)[i].X, (*c->sys)[i].ldx, S.P, S.AP, S.R, S.m, S.n, S.m, c->tol, 0,
                                      S.d);
    H2_LAUNCH_CHECK();
    k_cg_dir<<<grid, blk, 0, st>>>(S.P, S.R, S.m, S.n, S.m, S.d);
    H2_LAUNCH_CHECK();
    return 0;
}

int batch_iter_body(void* ctx, int i, cudaStream_t st) {
    BatchIterCtx* c = (BatchIterCtx*)ctx;
    Solver& S = *(*c->sys)[i].S;
    int rc = matmul_device(S.A, 1.0, S.P, S.m, S.AP, S.m, S.m, c->dtype, st, false, true);
    if (rc) return rc;
    return batch_iter_after_product(c, i, st);
}

}  // namespace

int batch_block_cg(h2_batch* b, const double* const* B, const int64_t* ldb, double* const* X, const int64_t* ldx,
                   const int64_t* m, const h2_cg_params* p, h2_cg_result* res) {
    if (!b || !B || !ldb || !X || !ldx || !m || !p || !res) { set_error("null argument"); return H2_E_BADARG; }
    if (!(p->tol >= 0.0) || p->max_iter < 0 || p->check_every < 1) { set_error("bad solver parameters"); return H2_E_BADARG; }
    const int32_t dtype = p->dtype;
    if (dtype != H2_F64 && dtype != H2_F32 && dtype != H2_BF16) { set_error("bad dtype"); return H2_E_BADARG; }
    if (p->transposed) { set_error("batched solves take A, not Aᵀ"); return H2_E_UNSUPPORTED; }
    if (p->variant != H2_CG_COLUMNWISE && p->variant != H2_CG_GRAM) { set_error("unsupported CG variant"); return H2_E_UNSUPPORTED; }
    const bool gram = p->variant == H2_CG_GRAM;
    if (p->precond != H2_PRECOND_NONE) { set_error("batched solves take no preconditioner"); return H2_E_UNSUPPORTED; }
    const int count = (int)b->mats.size();
    // graphs are captured on and launched from the batch's own stream, after the caller's work
    H2_CUDA_TRY(cudaEventRecord(b->ev_in, (cudaStream_t)p->stream));
    H2_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
    cudaStream_t st = b->origin;
    for (auto si : b->streams) H2_CUDA_TRY(cudaStreamWaitEvent(si, b->ev_in, 0));
    auto t0 = std::chrono::steady_clock::now();
    std::vector<BatchSys> sys(count);
    std::vector<std::unique_ptr<Solver>> solvers;
    for (int i = 0; i < count; ++i) {
        res[i].status = 0;
        res[i].iterations = res[i].outer_steps = res[i].h2mm_calls = 0;
        res[i].seconds = 0.0;
        if (m[i] < 0 || ldb[i] < m[i] || ldx[i] < m[i]) { set_error("bad m / leading dimension"); return H2_E_BADARG; }
        if (m[i] == 0) { sys[i].done = true; continue; }
        if (!is_device_pointer(B[i]) || !is_device_pointer(X[i])) {
            set_error("batched solves take device B and X");
            return H2_E_BADARG;
        }
        if (b->mats[i]->timing.on) { set_error("disable timing on batched matrices"); return H2_E_UNSUPPORTED; }
        if (gram && m[i] > kGramMaxCols) {
            set_error("the Gram-matrix block CG (H2_CG_GRAM) takes at most 64 columns per system");
            return H2_E_UNSUPPORTED;
        }
    }
    const double delta = p->inner_tol > 0.0 && p->inner_tol < 1.0 ? p->inner_tol : 0.1;
    const bool reliable = dtype != H2_F64;
    // set-up on each system's own stream: residual, CG state, product resources
    for (int i = 0; i < count; ++i) {
        if (sys[i].done) continue;
        h2_matrix* A = b->mats[i];
        cudaStream_t si = b->streams[i];
        solvers.emplace_back(new Solver{A, si, A->n, (int)m[i]});
        Solver& S = *solvers.back();
        S.gram = gram;
        sys[i].S = &S;
        sys[i].B = B[i];
        sys[i].ldb = ldb[i];
        sys[i].X = X[i];
        sys[i].ldx = ldx[i];
        int rc = S.init();
        if (rc) return rc;
        H2_CUDA_TRY(cudaMallocAsync((void**)&sys[i].Rt, ((size_t)A->n * m[i] + m[i]) * sizeof(double), si));
        sys[i].rupd = sys[i].Rt + (size_t)A->n * m[i];
        if ((rc = product_prepare(A, m[i], H2_F64, si))) return rc;
        if (dtype != H2_F64 && (rc = product_prepare(A, m[i], dtype, si))) return rc;
        if ((rc = S.residual(B[i], ldb[i], X[i], ldx[i]))) return rc;
        H2_CUDA_TRY(cudaMemsetAsync(S.d.summary, 0, 4 * sizeof(int), si));
        k_cg_init<<<S.grid2d(), dim3(kColsPerCta, 8), 0, si>>>(B[i], ldb[i], S.R, m[i], A->n, (int)m[i], p->tol, S.d);
        H2_LAUNCH_CHECK();
        if (gram) {
            if ((rc = gram_start(S.P, S.R, A->n, (int)m[i], S.g, S.d, si))) return rc;
        } else {
            k_copy2d<<<S.copy_grid(), 256, 0, si>>>(S.R, m[i], S.P, m[i], A->n, (int)m[i]);
            H2_LAUNCH_CHECK();
        }
        H2_CUDA_TRY(cudaMemcpyAsync(sys[i].rupd, S.d.rnorm, m[i] * sizeof(double), cudaMemcpyDeviceToDevice, si));
        H2_CUDA_TRY(cudaMemcpyAsync(S.h_summary, S.d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, si));
    }
    for (int i = 0; i < count; ++i) {
        if (sys[i].done) continue;
        H2_CUDA_TRY(cudaStreamSynchronize(b->streams[i]));
        if (sys[i].S->h_summary[0] == 0) sys[i].done = true;
    }
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    BatchIterCtx ctx{&sys, dtype, p->tol};
    cudaGraphExec_t exec = nullptr;
    std::vector<int> in_graph;
    int status = 0, it = 0;
    // FP32 products of every system in two multi-system launches per iteration
    // (the upward pass with the coupling phase, the downward pass with the leaf
    // phase), when every system can take them; their buffers are sized once here
    std::vector<int> all_active;
    for (int i = 0; i < count; ++i) if (!sys[i].done) all_active.push_back(i);
    const bool multi = !all_active.empty() && flow_batch_ok(b, all_active, m, dtype);
    std::vector<FlowBufs> fbs(count);
    void* fmem = nullptr;
    size_t fbytes = 0;
    if (multi)
        for (int i : all_active) {
            int rc = flow_prepare(b->mats[i], (int)m[i], b->streams[i], &fbs[i]);
            if (rc) return rc;
        }
    auto rebuild = [&]() -> int {
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        in_graph.clear();
        for (int i = 0; i < count; ++i) if (!sys[i].done) in_graph.push_back(i);
        if (in_graph.empty()) return 0;
        if (!multi) return batch_capture(b, st, in_graph, batch_iter_body, &ctx, &exec);
        std::vector<FlowBufs> fb;
        for (int i : in_graph) fb.push_back(fbs[i]);
        TcGemmParams p1, p2;
        int rc = flow_tables(b, in_graph, fb, &fmem, &fbytes, &p1, &p2, st);
        if (rc) return rc;
        auto pre = [&](int j, cudaStream_t s) {
            const int i = in_graph[j];
            Solver& S = *sys[i].S;
            return flow_pre(S.A, S.P, S.m, fbs[i], s);
        };
        auto post = [&](int j, cudaStream_t s) {
            const int i = in_graph[j];
            Solver& S = *sys[i].S;
            int rc2 = flow_post(S.A, 1.0, S.P, S.m, S.AP, S.m, fbs[i], true, s);
            if (rc2) return rc2;
            return batch_iter_after_product(&ctx, i, s);
        };
        return flow_capture(b, in_graph, p1, p2, pre, post, &exec);
    };
    int rc = rebuild();
    if (rc) return rc;
    int done_since_build = 0;
    for (it = 1; it <= p->max_iter && !in_graph.empty(); ++it) {
        H2_CUDA_TRY(cudaGraphLaunch(exec, st));
        for (int i : in_graph) if (!sys[i].done) sys[i].iters = it;
        if (it % p->check_every != 0 && it != p->max_iter) continue;
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        bool all = true;
        for (int i : in_graph) {
            BatchSys& y = sys[i];
            if (y.done) continue;
            Solver& S = *y.S;
            cudaStream_t si = b->streams[i];
            const int mi = S.m;
            std::vector<double> rn(mi), ru(mi);
            std::vector<int> act(mi);
            H2_CUDA_TRY(cudaMemcpyAsync(S.h_summary, S.d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, si));
            H2_CUDA_TRY(cudaMemcpyAsync(rn.data(), S.d.rnorm, mi * sizeof(double), cudaMemcpyDeviceToHost, si));
            H2_CUDA_TRY(cudaMemcpyAsync(ru.data(), y.rupd, mi * sizeof(double), cudaMemcpyDeviceToHost, si));
            H2_CUDA_TRY(cudaMemcpyAsync(act.data(), S.d.active, mi * sizeof(int), cudaMemcpyDeviceToHost, si));
            H2_CUDA_TRY(cudaStreamSynchronize(si));
            if (S.h_summary[1]) { y.status = H2_E_BREAKDOWN; y.done = true; ++done_since_build; continue; }
            bool update = S.h_summary[0] == 0;
            if (reliable)
                for (int c = 0; c < mi && !update; ++c) update = act[c] && rn[c] < delta * ru[c];
            if (!update) { all = false; continue; }
            if (!reliable) { y.done = true; ++done_since_build; continue; }
            // true FP64 residual replaces the recurrence residual (eager, off the graph)
            ++y.updates;
            if ((rc = S.reliable_update(y.B, y.ldb, y.X, y.ldx, p->tol, y.Rt, y.rupd))) return rc;
            H2_CUDA_TRY(cudaMemcpyAsync(S.h_summary, S.d.summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, si));
            H2_CUDA_TRY(cudaStreamSynchronize(si));
            if (S.h_summary[1]) { y.status = H2_E_BREAKDOWN; y.done = true; ++done_since_build; continue; }
            if (S.h_summary[0] == 0) { y.done = true; ++done_since_build; continue; }
            all = false;
        }
        if (all) break;
        // systems that left: rebuild the graph once a quarter of it has converged
        if (done_since_build > 0 && done_since_build * 4 >= (int)in_graph.size()) {
            if ((rc = rebuild())) return rc;
            done_since_build = 0;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    if (fmem) cudaFree(fmem);
    // report: true FP64 residual per column
    for (int i = 0; i < count; ++i) {
        BatchSys& y = sys[i];
        if (!y.S) continue;
        Solver& S = *y.S;
        cudaStream_t si = b->streams[i];
        const int mi = S.m;
        if (!y.done && y.status == 0) y.status = H2_E_NOCONVERGE;
        if ((rc = S.residual(y.B, y.ldb, y.X, y.ldx))) return rc;
        k_col_relnorm<<<S.grid2d(), dim3(kColsPerCta, 8), 0, si>>>(S.R, mi, y.B, y.ldb, S.n, mi, y.rupd, S.d);
        H2_LAUNCH_CHECK();
        std::vector<double> rel(mi);
        std::vector<int> ci(mi);
        H2_CUDA_TRY(cudaMemcpyAsync(rel.data(), y.rupd, mi * sizeof(double), cudaMemcpyDeviceToHost, si));
        H2_CUDA_TRY(cudaMemcpyAsync(ci.data(), S.d.conv_iter, mi * sizeof(int), cudaMemcpyDeviceToHost, si));
        cudaFreeAsync(y.Rt, si);
        H2_CUDA_TRY(cudaStreamSynchronize(si));
        if (res[i].rel_residual) for (int c = 0; c < mi; ++c) res[i].rel_residual[c] = rel[c];
        if (res[i].col_iterations) for (int c = 0; c < mi; ++c) res[i].col_iterations[c] = ci[c];
        res[i].status = y.status;
        res[i].iterations = y.iters;
        res[i].outer_steps = y.updates;
        res[i].h2mm_calls = S.h2mm_calls + y.iters;
        if (y.status && !status) status = y.status;
    }
    solvers.clear();
    for (auto s2 : b->streams) cudaStreamSynchronize(s2);
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < count; ++i) res[i].seconds = secs;
    if (status) set_error("some systems did not converge (see the per-system status)");
    return status;
}

int block_cg(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
             const h2_cg_params* p, h2_cg_result* res) {
    if (!A || !p || !res) { set_error("null argument"); return H2_E_BADARG; }
    if (m < 0 || (m > 0 && (!B || !X)) || ldb < m || ldx < m) { set_error("bad m / leading dimension"); return H2_E_BADARG; }
    if (!(p->tol >= 0.0) || p->max_iter < 0 || p->check_every < 1) { set_error("bad solver parameters"); return H2_E_BADARG; }
    if (p->variant != H2_CG_COLUMNWISE && p->variant != H2_CG_GRAM) { set_error("unsupported CG variant"); return H2_E_UNSUPPORTED; }
    if (p->precond != H2_PRECOND_NONE && p->precond != H2_PRECOND_BLOCK_JACOBI) { set_error("unknown preconditioner"); return H2_E_BADARG; }
    if (p->precond == H2_PRECOND_BLOCK_JACOBI && p->transposed) {
        set_error("the block-Jacobi preconditioner is available for solves with A");
        return H2_E_UNSUPPORTED;
    }
    if (p->variant == H2_CG_GRAM && m > kGramMaxCols) {
        set_error("the Gram-matrix block CG (H2_CG_GRAM) takes at most 64 columns");
        return H2_E_UNSUPPORTED;
    }
    const int32_t inner = p->dtype;
    if (inner != H2_F64 && inner != H2_F32 && inner != H2_BF16) { set_error("bad dtype"); return H2_E_BADARG; }
    const bool refine = inner != H2_F64 && p->refine != 0;
    res->status = 0;
    res->iterations = res->outer_steps = res->h2mm_calls = 0;
    res->seconds = 0.0;
    if (m == 0) return 0;
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)p->stream;
    const int64_t n = A->n;

    // device copies of host blocks
    const bool db = is_device_pointer(B), dxp = is_device_pointer(X);
    double *Bd = (double*)B, *Xd = X;
    int64_t ldbd = ldb, ldxd = ldx;
    void* stage = nullptr;
    if (!db || !dxp) {
        H2_CUDA_TRY(cudaMallocAsync(&stage, 2 * (size_t)n * m * sizeof(double), st));
        if (!db) {
            Bd = (double*)stage;
            ldbd = m;
            H2_CUDA_TRY(cudaMemcpy2DAsync(Bd, m * sizeof(double), B, ldb * sizeof(double), m * sizeof(double), n,
                                          cudaMemcpyHostToDevice, st));
        }
        if (!dxp) {
            Xd = (double*)stage + (size_t)n * m;
            ldxd = m;
            H2_CUDA_TRY(cudaMemcpy2DAsync(Xd, m * sizeof(double), X, ldx * sizeof(double), m * sizeof(double), n,
                                          cudaMemcpyHostToDevice, st));
        }
    }
    int status = 0;
    {
        Solver S{A, st, n, (int)m};
        S.trans = p->transposed != 0;
        S.gram = p->variant == H2_CG_GRAM;
        S.pcg = p->precond == H2_PRECOND_BLOCK_JACOBI;
        S.pc_low = p->dtype != H2_F64;
        int rc = S.init();
        if (rc) return rc;
        int total_iters = 0;
        bool restarted = false;
        std::vector<double> rel_chk(m);
        if (refine && p->refine == 2) {
            // reliable updates: one CG run, FP64 true residual substituted periodically
            double* Rt = nullptr;
            H2_CUDA_TRY(cudaMallocAsync(&Rt, ((size_t)n * m + m) * sizeof(double), st));
            double* rupd = Rt + (size_t)n * m;
            if ((rc = S.residual(Bd, ldbd, Xd, ldxd))) return rc;
            int it = 0, upd = 0;
            const double delta = p->inner_tol > 0.0 && p->inner_tol < 1.0 ? p->inner_tol : 0.1;
            status = S.cg_reliable(inner, Bd, ldbd, Xd, ldxd, p->tol, p->max_iter, p->check_every, delta, Rt, rupd,
                                   &it, &upd);
            cudaFreeAsync(Rt, st);
            if (status < 0 && status != H2_E_BREAKDOWN && status != H2_E_NOCONVERGE) return status;
            total_iters = it;
            res->outer_steps = upd;
        } else if (!refine) {
            if ((rc = S.residual(Bd, ldbd, Xd, ldxd, inner))) return rc;
            int it = 0;
            status = S.cg(inner, Bd, ldbd, Xd, ldxd, p->tol, p->max_iter, p->check_every, &it);
            if (status < 0 && status != H2_E_BREAKDOWN && status != H2_E_NOCONVERGE) return status;
            total_iters = it;
            // FP64: convergence is confirmed on the true residual B - A X.  A column
            // whose recurrence residual met tol but whose true residual does not
            // continues from the true residual (p = r, a restart), at most a few times.
            for (int check = 0; inner == H2_F64 && status == 0 && check < 4; ++check) {
                if ((rc = S.residual(Bd, ldbd, Xd, ldxd))) return rc;
                if ((rc = S.true_rel(Bd, ldbd, rel_chk.data()))) return rc;
                bool all = true;
                for (double v : rel_chk) all = all && (v <= p->tol);
                if (all) break;
                restarted = true;
                it = 0;
                status = S.cg(inner, Bd, ldbd, Xd, ldxd, p->tol, p->max_iter - total_iters, p->check_every, &it);
                if (status < 0 && status != H2_E_BREAKDOWN && status != H2_E_NOCONVERGE) return status;
                total_iters += it;
                if (status == 0 && check == 3) status = H2_E_NOCONVERGE;
            }
        } else {
            // Iterative refinement: FP64 residual outside, low-precision block CG inside.
            double* D = nullptr;
            double* Rk = nullptr;
            H2_CUDA_TRY(cudaMallocAsync(&D, 2 * (size_t)n * m * sizeof(double), st));
            Rk = D + (size_t)n * m;
            std::vector<double> rel(m);
            double* d_rel = nullptr;
            H2_CUDA_TRY(cudaMallocAsync(&d_rel, m * sizeof(double), st));
            status = H2_E_NOCONVERGE;
            const int max_outer = p->max_outer > 0 ? p->max_outer : 20;
            for (int outer = 0; outer <= max_outer; ++outer) {
                if ((rc = S.residual(Bd, ldbd, Xd, ldxd))) return rc;
                k_col_relnorm<<<S.grid2d(), dim3(kColsPerCta, 8), 0, st>>>(S.R, m, Bd, ldbd, n, (int)m, d_rel, S.d);
                H2_LAUNCH_CHECK();
                H2_CUDA_TRY(cudaMemcpyAsync(rel.data(), d_rel, m * sizeof(double), cudaMemcpyDeviceToHost, st));
                H2_CUDA_TRY(cudaStreamSynchronize(st));
                bool all = true;
                for (double v : rel) all = all && (v <= p->tol);
                if (all) { status = 0; break; }
                if (outer == max_outer || total_iters >= p->max_iter) break;
                res->outer_steps = outer + 1;
                // inner solve A D = R to a relative reduction inner_tol; D0 = 0
                k_copy2d<<<S.copy_grid(), 256, 0, st>>>(S.R, m, Rk, m, n, (int)m);
                H2_LAUNCH_CHECK();
                k_copy2d<<<S.copy_grid(), 256, 0, st>>>(nullptr, 0, D, m, n, (int)m);
                H2_LAUNCH_CHECK();
                int it = 0;
                const double itol = p->inner_tol > 0.0 ? p->inner_tol : 1e-4;
                int st_in = S.cg(inner, Rk, m, D, m, itol, p->max_iter - total_iters, p->check_every, &it);
                total_iters += it;
                if (st_in == H2_E_BREAKDOWN) { status = H2_E_BREAKDOWN; break; }
                if (st_in < 0 && st_in != H2_E_NOCONVERGE) return st_in;
                k_axpy2d<<<S.copy_grid(), 256, 0, st>>>(D, m, Xd, ldxd, n, (int)m);
                H2_LAUNCH_CHECK();
            }
            cudaFreeAsync(D, st);
            cudaFreeAsync(d_rel, st);
        }
        res->iterations = total_iters;
        // true FP64 residual per column
        if ((rc = S.residual(Bd, ldbd, Xd, ldxd))) return rc;
        double* d_rel = nullptr;
        H2_CUDA_TRY(cudaMallocAsync(&d_rel, m * sizeof(double), st));
        k_col_relnorm<<<S.grid2d(), dim3(kColsPerCta, 8), 0, st>>>(S.R, m, Bd, ldbd, n, (int)m, d_rel, S.d);
        H2_LAUNCH_CHECK();
        std::vector<double> rel(m);
        std::vector<int> ci(m);
        H2_CUDA_TRY(cudaMemcpyAsync(rel.data(), d_rel, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaMemcpyAsync(ci.data(), S.d.conv_iter, m * sizeof(int), cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(d_rel, st);
        if (!dxp)
            H2_CUDA_TRY(cudaMemcpy2DAsync(X, ldx * sizeof(double), Xd, m * sizeof(double), m * sizeof(double), n,
                                          cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        if (res->rel_residual) for (int64_t i = 0; i < m; ++i) res->rel_residual[i] = rel[i];
        if (res->col_iterations)
            for (int64_t i = 0; i < m; ++i) res->col_iterations[i] = (refine || restarted) ? total_iters : ci[i];
        res->h2mm_calls = S.h2mm_calls;
    }
    if (stage) cudaFreeAsync(stage, st);
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    res->status = status;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (status == H2_E_BREAKDOWN) set_error("block CG breakdown: <p, Ap> <= 0 or a non-finite scalar");
    if (status == H2_E_NOCONVERGE) set_error("block CG did not converge within the iteration caps");
    return status;
}

}  // namespace h2
