// Block GMRES (Sec. 5.2, Alg. "pgmres block") on the device: every column i
// runs restarted, left-preconditioned GMRES(ℓ) on its own Krylov space; the
// only shared operation is the block product a = M⁻¹ A q_k.
//
// One cycle:  r = M⁻¹(b − A x) in FP64 (the product in FP64: the restart is
// also the refinement step of a mixed-precision solve), β_i = |r_i|,
// q_0 = r/β, r̂ = β e_1; then per step k
//   a = M⁻¹ A q_k                              (product in the chosen precision)
//   k_gm_dots     h_{j,k} = <q_j, a>, j <= k    (all at once: classical Gram–Schmidt, as printed)
//   k_gm_orth     a -= Σ_j q_j h_{j,k}, |a|²; the last CTA finishes the column of H:
//                 earlier Givens rotations, the new rotation, r̂, convergence
//   k_gm_next     q_{k+1} = a / h_{k+1,k}
// and at the end of the cycle  R y = r̂ (back substitution, one thread per
// column) and  x += Σ_j q_j y_j.  A column whose Givens residual reaches
// tol·|M⁻¹b| stops extending its basis (frozen).  Reductions are two-stage and
// in fixed order (per-CTA partials, last CTA by ticket).  All vector work is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "h2_internal.cuh"

namespace h2 {

namespace {

constexpr int kRows = 304;       // CTAs along the rows (2 per SM)
constexpr int kCols = 32;        // columns per CTA (one per lane)
constexpr int kMaxRestart = 64;  // ℓ
constexpr int kJ = 8;            // inner products per pass

struct GmDev {
    double* V;       // [(ℓ+1)][n][m] basis q_0..q_ℓ
    double* H;       // [m][ℓ+1][ℓ] Hessenberg columns (rotated in place)
    double* cs;      // [m][ℓ]
    double* sn;      // [m][ℓ]
    double* rh;      // [m][ℓ+1] rotated residual r̂
    double* y;       // [m][ℓ]
    double* bnorm;   // [m] |M⁻¹ b_i| (1 when 0)
    double* rel;     // [m] relative residual of the last check
    double* part;    // [kRows][m][kJ] partial sums
    int* active;     // [m]
    int* steps;      // [m] basis size of the current cycle
    int* col_it;     // [m] steps while active, over all cycles
    int* summary;    // [0] active columns
    unsigned* ticket;// [ceil(m/32)]
    int64_t n;
    int m, ell;
};

__device__ __forceinline__ bool gm_last_cta(unsigned* ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) last = atomicAdd(&ticket[blockIdx.y], 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Sum over the row lanes of the CTA (fixed order); result valid in ty == 0.
__device__ __forceinline__ double lane_sum(double v, double (*sm)[kCols]) {
    __syncthreads();
    sm[threadIdx.y][threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.y == 0)
        for (int y = 0; y < 8; ++y) s += sm[y][threadIdx.x];
    return s;
}

// Column norms of R (FP64 true or preconditioned residual), the first basis
// vector q_0 = R/β, r̂ = β e_1, relative residuals and the active set.  Also
// |M⁻¹B| when `init` (R then holds M⁻¹B).  Two passes share one kernel: the
// norms reduce first (all CTAs), then the last CTA updates the column state;
// q_0 is written by k_gm_scale.
__global__ void __launch_bounds__(256) k_gm_norms(const double* __restrict__ R, GmDev g, double tol, int init) {
    __shared__ double sm[8][kCols];
    const int col = blockIdx.y * kCols + threadIdx.x;
    double v = 0.0;
    if (col < g.m)
        for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < g.n; i += (int64_t)gridDim.x * 8) {
            const double r = R[i * g.m + col];
            v = fma(r, r, v);
        }
    v = lane_sum(v, sm);
    if (threadIdx.y == 0 && col < g.m) g.part[((size_t)blockIdx.x * g.m + col) * kJ] = v;
    if (!gm_last_cta(g.ticket)) return;
    if (threadIdx.y == 0 && col < g.m) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&g.part[((size_t)b * g.m + col) * kJ]);
        const double nrm = sqrt(s);
        if (init) {
            g.bnorm[col] = nrm > 0.0 ? nrm : 1.0;
        } else {
            const double rel = nrm / g.bnorm[col];
            g.rel[col] = rel;
            const int act = !(rel <= tol) && nrm > 0.0;
            g.active[col] = act;
            if (act) atomicAdd(&g.summary[0], 1);
            g.steps[col] = 0;
            double* rh = g.rh + (size_t)col * (g.ell + 1);
            for (int j = 0; j <= g.ell; ++j) rh[j] = 0.0;
            rh[0] = nrm;
        }
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) g.ticket[blockIdx.y] = 0;
}

// q_0 = R / β on active columns, 0 elsewhere.
__global__ void k_gm_scale(const double* __restrict__ R, GmDev g) {
    const int col = blockIdx.y * kCols + threadIdx.x;
    if (col >= g.m) return;
    const bool act = g.active[col] != 0;
    const double inv = act ? 1.0 / g.rh[(size_t)col * (g.ell + 1)] : 0.0;
    for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < g.n; i += (int64_t)gridDim.x * 8)
        g.V[i * g.m + col] = act ? R[i * g.m + col] * inv : 0.0;
}

// h_{j,k} = <q_j, a> for j in [j0, j0 + kJ) ∩ [0, k], active columns; the last
// CTA writes H[col][j][k].
__global__ void __launch_bounds__(256) k_gm_dots(const double* __restrict__ a, GmDev g, int k, int j0) {
    __shared__ double sm[8][kCols];
    const int col = blockIdx.y * kCols + threadIdx.x;
    const int nj = min(kJ, k + 1 - j0);
    double v[kJ];
#pragma unroll
    for (int u = 0; u < kJ; ++u) v[u] = 0.0;
    const size_t nm = (size_t)g.n * g.m;
    if (col < g.m && g.active[col])
        for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < g.n; i += (int64_t)gridDim.x * 8) {
            const double ai = a[i * g.m + col];
#pragma unroll
            for (int u = 0; u < kJ; ++u)
                if (u < nj) v[u] = fma(g.V[(size_t)(j0 + u) * nm + i * g.m + col], ai, v[u]);
        }
#pragma unroll
    for (int u = 0; u < kJ; ++u) {
        const double s = lane_sum(v[u], sm);
        if (threadIdx.y == 0 && col < g.m && u < nj) g.part[((size_t)blockIdx.x * g.m + col) * kJ + u] = s;
    }
    if (!gm_last_cta(g.ticket)) return;
    if (threadIdx.y == 0 && col < g.m && g.active[col]) {
        for (int u = 0; u < nj; ++u) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&g.part[((size_t)b * g.m + col) * kJ + u]);
            g.H[((size_t)col * (g.ell + 1) + j0 + u) * g.ell + k] = s;
        }
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) g.ticket[blockIdx.y] = 0;
}

// a -= Σ_{j<=k} q_j h_{j,k} and |a|² on active columns; the last CTA completes
// column k of H: h_{k+1,k} = |a|, earlier rotations, the new rotation, r̂, and
// the convergence test |r̂_{k+1}| <= tol·|M⁻¹b| (or h_{k+1,k} = 0).
__global__ void __launch_bounds__(256) k_gm_orth(double* __restrict__ a, GmDev g, int k, double tol) {
    __shared__ double sm[8][kCols];
    __shared__ double sh[kMaxRestart + 1][kCols];
    const int col = blockIdx.y * kCols + threadIdx.x;
    const bool act = col < g.m && g.active[col];
    for (int j = threadIdx.y; j <= k; j += 8)
        sh[j][threadIdx.x] = act ? g.H[((size_t)col * (g.ell + 1) + j) * g.ell + k] : 0.0;
    __syncthreads();
    const size_t nm = (size_t)g.n * g.m;
    double v = 0.0;
    if (act)
        for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < g.n; i += (int64_t)gridDim.x * 8) {
            double s = a[i * g.m + col];
            for (int j = 0; j <= k; ++j) s = fma(-g.V[(size_t)j * nm + i * g.m + col], sh[j][threadIdx.x], s);
            a[i * g.m + col] = s;
            v = fma(s, s, v);
        }
    v = lane_sum(v, sm);
    if (threadIdx.y == 0 && col < g.m) g.part[((size_t)blockIdx.x * g.m + col) * kJ] = v;
    if (!gm_last_cta(g.ticket)) return;
    if (threadIdx.y == 0 && act) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&g.part[((size_t)b * g.m + col) * kJ]);
        const double hn = sqrt(s);
        const int L = g.ell;
        double* Hc = g.H + (size_t)col * (L + 1) * L;
        double* cs = g.cs + (size_t)col * L;
        double* sn = g.sn + (size_t)col * L;
        double* rh = g.rh + (size_t)col * (L + 1);
        Hc[(size_t)(k + 1) * L + k] = hn;
        for (int j = 0; j < k; ++j) {  // earlier rotations on the new column
            const double h0 = Hc[(size_t)j * L + k], h1 = Hc[(size_t)(j + 1) * L + k];
            Hc[(size_t)j * L + k] = cs[j] * h0 + sn[j] * h1;
            Hc[(size_t)(j + 1) * L + k] = -sn[j] * h0 + cs[j] * h1;
        }
        const double h0 = Hc[(size_t)k * L + k];
        double c = 1.0, sg = 0.0;
        if (hn != 0.0) {
            const double r = hypot(h0, hn);
            c = h0 / r;
            sg = hn / r;
        }
        cs[k] = c;
        sn[k] = sg;
        Hc[(size_t)k * L + k] = c * h0 + sg * hn;
        Hc[(size_t)(k + 1) * L + k] = 0.0;
        rh[k + 1] = -sg * rh[k];
        rh[k] = c * rh[k];
        g.steps[col] = k + 1;
        g.col_it[col] += 1;
        const double rel = fabs(rh[k + 1]) / g.bnorm[col];
        g.rel[col] = rel;
        if (rel <= tol || hn == 0.0 || !isfinite(rel)) {
            g.active[col] = 0;
            atomicSub(&g.summary[0], 1);
        }
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) g.ticket[blockIdx.y] = 0;
}

// q_{k+1} = a / h_{k+1,k} for the columns that are still extending their basis.
__global__ void k_gm_next(const double* __restrict__ a, GmDev g, int k) {
    const int col = blockIdx.y * kCols + threadIdx.x;
    if (col >= g.m || !g.active[col]) return;
    // h_{k+1,k} is kept in H before the rotation zeroed it: recompute from |a|
    // via the rotation: h_{k+1,k} = sn_k · r where r = H[k][k] after rotation
    const int L = g.ell;
    const double hn = g.sn[(size_t)col * L + k] * g.H[((size_t)col * (L + 1) + k) * L + k];
    const double inv = hn != 0.0 ? 1.0 / hn : 0.0;
    const size_t nm = (size_t)g.n * g.m;
    for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < g.n; i += (int64_t)gridDim.x * 8)
        g.V[(size_t)(k + 1) * nm + i * g.m + col] = a[i * g.m + col] * inv;
}

// y = R⁻¹ r̂ per column (one thread per column, k = steps[col]).
__global__ void k_gm_backsolve(GmDev g) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= g.m) return;
    const int L = g.ell, kk = g.steps[col];
    const double* Hc = g.H + (size_t)col * (L + 1) * L;
    const double* rh = g.rh + (size_t)col * (L + 1);
    double* y = g.y + (size_t)col * L;
    for (int j = kk - 1; j >= 0; --j) {
        double s = rh[j];
        for (int l = j + 1; l < kk; ++l) s -= Hc[(size_t)j * L + l] * y[l];
        y[j] = s / Hc[(size_t)j * L + j];
    }
}

// x += Σ_{j < steps} q_j y_j.
__global__ void k_gm_update(double* __restrict__ X, int64_t ldx, GmDev g) {
    const int col = blockIdx.y * kCols + threadIdx.x;
    if (col >= g.m) return;
    const int kk = g.steps[col];
    if (kk == 0) return;
    const double* y = g.y + (size_t)col * g.ell;
    const size_t nm = (size_t)g.n * g.m;
    for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < g.n; i += (int64_t)gridDim.x * 8) {
        double s = X[i * ldx + col];
        for (int j = 0; j < kk; ++j) s = fma(g.V[(size_t)j * nm + i * g.m + col], y[j], s);
        X[i * ldx + col] = s;
    }
}

__global__ void k_gm_copy(const double* __restrict__ B, int64_t ldb, double* __restrict__ R, int64_t n, int m) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        R[e] = B[(e / m) * ldb + e % m];
}

__global__ void k_gm_relnorm(const double* __restrict__ R, const double* __restrict__ B, int64_t ldb, GmDev g,
                             double* __restrict__ out) {
    __shared__ double sm[8][kCols];
    __shared__ double sm2[8][kCols];
    const int col = blockIdx.y * kCols + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (col < g.m)
        for (int64_t i = blockIdx.x * 8 + threadIdx.y; i < g.n; i += (int64_t)gridDim.x * 8) {
            const double r = R[i * g.m + col], b = B[i * ldb + col];
            rr = fma(r, r, rr);
            bb = fma(b, b, bb);
        }
    rr = lane_sum(rr, sm);
    bb = lane_sum(bb, sm2);
    if (threadIdx.y == 0 && col < g.m) {
        g.part[((size_t)blockIdx.x * g.m + col) * kJ + 0] = rr;
        g.part[((size_t)blockIdx.x * g.m + col) * kJ + 1] = bb;
    }
    if (!gm_last_cta(g.ticket)) return;
    if (threadIdx.y == 0 && col < g.m) {
        double r = 0.0, b = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) {
            r += __ldcg(&g.part[((size_t)k * g.m + col) * kJ + 0]);
            b += __ldcg(&g.part[((size_t)k * g.m + col) * kJ + 1]);
        }
        out[col] = sqrt(r) / (b > 0.0 ? sqrt(b) : 1.0);
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) g.ticket[blockIdx.y] = 0;
}

}  // namespace

int block_gmres(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
                const h2_gmres_params* p, h2_cg_result* res) {
    if (!A || !p || !res) { set_error("null argument"); return H2_E_BADARG; }
    if (m < 0 || (m > 0 && (!B || !X)) || ldb < m || ldx < m) { set_error("bad m / leading dimension"); return H2_E_BADARG; }
    if (!(p->tol >= 0.0) || p->max_iter < 0 || p->restart < 1 || p->restart > kMaxRestart) {
        set_error("bad GMRES parameters (1 <= restart <= 64)");
        return H2_E_BADARG;
    }
    if (p->dtype != H2_F64 && p->dtype != H2_F32 && p->dtype != H2_BF16) { set_error("bad dtype"); return H2_E_BADARG; }
    if (p->precond != H2_PRECOND_NONE && p->precond != H2_PRECOND_BLOCK_JACOBI) { set_error("unknown preconditioner"); return H2_E_BADARG; }
    if (p->transposed && p->dtype == H2_BF16) { set_error("the BF16 product supports A·X only"); return H2_E_UNSUPPORTED; }
    res->status = 0;
    res->iterations = res->outer_steps = res->h2mm_calls = 0;
    res->seconds = 0.0;
    if (m == 0) return 0;
    if (!is_device_pointer(B) || !is_device_pointer(X)) {
        set_error("h2_block_gmres takes device B and X");
        return H2_E_BADARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)p->stream;
    const int64_t n = A->n;
    const int L = p->restart;
    const bool pc = p->precond == H2_PRECOND_BLOCK_JACOBI;
    const bool tr = p->transposed != 0;
    int rc = 0;
    if (pc && (rc = bj_prepare(A, st))) return rc;

    // one allocation, 256-byte aligned pieces
    const size_t nm = (size_t)n * m;
    size_t off = 0;
    auto piece = [&](size_t b) { const size_t o = off; off += (b + 255) & ~(size_t)255; return o; };
    const size_t oV = piece((size_t)(L + 1) * nm * sizeof(double)), oA = piece(nm * sizeof(double)),
                 oZ = piece(nm * sizeof(double)), oH = piece((size_t)m * (L + 1) * L * sizeof(double)),
                 oCs = piece((size_t)m * L * sizeof(double)), oSn = piece((size_t)m * L * sizeof(double)),
                 oRh = piece((size_t)m * (L + 1) * sizeof(double)), oY = piece((size_t)m * L * sizeof(double)),
                 oBn = piece(m * sizeof(double)), oRel = piece(m * sizeof(double)),
                 oPart = piece((size_t)kRows * m * kJ * sizeof(double)), oAct = piece(m * sizeof(int)),
                 oSteps = piece(m * sizeof(int)), oIt = piece(m * sizeof(int)), oSum = piece(4 * sizeof(int)),
                 oTk = piece(((m + kCols - 1) / kCols) * sizeof(unsigned));
    void* mem = nullptr;
    H2_CUDA_TRY(cudaMallocAsync(&mem, off, st));
    char* base = (char*)mem;
    GmDev g{};
    g.V = (double*)(base + oV);
    double* a = (double*)(base + oA);
    double* Z = (double*)(base + oZ);
    g.H = (double*)(base + oH);
    g.cs = (double*)(base + oCs);
    g.sn = (double*)(base + oSn);
    g.rh = (double*)(base + oRh);
    g.y = (double*)(base + oY);
    g.bnorm = (double*)(base + oBn);
    g.rel = (double*)(base + oRel);
    g.part = (double*)(base + oPart);
    g.active = (int*)(base + oAct);
    g.steps = (int*)(base + oSteps);
    g.col_it = (int*)(base + oIt);
    g.summary = (int*)(base + oSum);
    g.ticket = (unsigned*)(base + oTk);
    g.n = n;
    g.m = (int)m;
    g.ell = L;
    const dim3 blk(kCols, 8), grid(kRows, (unsigned)((m + kCols - 1) / kCols));
    const unsigned cg = (unsigned)std::min<int64_t>(((int64_t)nm + 255) / 256, 152 * 16);
    CgDev dummy{};  // the block-Jacobi apply without the <Ap, z> reduction touches no CG state
    int status = 0;
    int h2mm = 0, total = 0, cycles = 0;
    std::vector<int> hsum(1);
    auto cleanup = [&]() { cudaFreeAsync(mem, st); };
    auto fail = [&](int r) { cleanup(); cudaStreamSynchronize(st); return r; };

    cudaError_t ce = cudaMemsetAsync(g.ticket, 0, ((m + kCols - 1) / kCols) * sizeof(unsigned), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g.col_it, 0, m * sizeof(int), st);
    if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); return fail(H2_E_CUDA); }
    // |M⁻¹ B|
    const double* Bsrc = B;
    if (pc) {
        k_gm_copy<<<cg, 256, 0, st>>>(B, ldb, a, n, (int)m);
        if ((rc = bj_apply(A, a, Z, n, (int)m, nullptr, dummy, st))) return fail(rc);
        Bsrc = Z;
    } else {
        k_gm_copy<<<cg, 256, 0, st>>>(B, ldb, Z, n, (int)m);
        Bsrc = Z;
    }
    k_gm_norms<<<grid, blk, 0, st>>>(Bsrc, g, p->tol, 1);
    if ((ce = cudaGetLastError()) != cudaSuccess) { set_error(cudaGetErrorString(ce)); return fail(H2_E_CUDA); }

    while (true) {
        // r = M⁻¹(B − A X) with the FP64 product
        k_gm_copy<<<cg, 256, 0, st>>>(B, ldb, a, n, (int)m);
        ++h2mm;
        if ((rc = matmul_device(A, -1.0, X, ldx, a, m, m, H2_F64, st, tr, false))) return fail(rc);
        double* R = a;
        if (pc) {
            if ((rc = bj_apply(A, a, Z, n, (int)m, nullptr, dummy, st))) return fail(rc);
            R = Z;
        }
        ce = cudaMemsetAsync(g.summary, 0, 4 * sizeof(int), st);
        if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); return fail(H2_E_CUDA); }
        k_gm_norms<<<grid, blk, 0, st>>>(R, g, p->tol, 0);
        k_gm_scale<<<grid, blk, 0, st>>>(R, g);
        if ((ce = cudaMemcpyAsync(hsum.data(), g.summary, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (ce = cudaStreamSynchronize(st)) != cudaSuccess) {
            set_error(cudaGetErrorString(ce));
            return fail(H2_E_CUDA);
        }
        if (hsum[0] == 0) break;
        if (total >= p->max_iter) { status = H2_E_NOCONVERGE; break; }
        ++cycles;
        for (int k = 0; k < L && total < p->max_iter; ++k) {
            // a = M⁻¹ A q_k
            ++h2mm;
            ++total;
            const size_t vk = (size_t)k * nm;
            if ((rc = matmul_device(A, 1.0, g.V + vk, m, a, m, m, p->dtype, st, tr, true))) return fail(rc);
            double* av = a;
            if (pc) {
                if ((rc = bj_apply(A, a, Z, n, (int)m, nullptr, dummy, st))) return fail(rc);
                av = Z;
            }
            for (int j0 = 0; j0 <= k; j0 += kJ) k_gm_dots<<<grid, blk, 0, st>>>(av, g, k, j0);
            k_gm_orth<<<grid, blk, 0, st>>>(av, g, k, p->tol);
            k_gm_next<<<grid, blk, 0, st>>>(av, g, k);
            if ((ce = cudaGetLastError()) != cudaSuccess) { set_error(cudaGetErrorString(ce)); return fail(H2_E_CUDA); }
            if ((ce = cudaMemcpyAsync(hsum.data(), g.summary, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (ce = cudaStreamSynchronize(st)) != cudaSuccess) {
                set_error(cudaGetErrorString(ce));
                return fail(H2_E_CUDA);
            }
            if (hsum[0] == 0) break;
        }
        k_gm_backsolve<<<(unsigned)((m + 63) / 64), 64, 0, st>>>(g);
        k_gm_update<<<grid, blk, 0, st>>>(X, ldx, g);
        if ((ce = cudaGetLastError()) != cudaSuccess) { set_error(cudaGetErrorString(ce)); return fail(H2_E_CUDA); }
    }
    // true FP64 residual per column
    k_gm_copy<<<cg, 256, 0, st>>>(B, ldb, a, n, (int)m);
    ++h2mm;
    if ((rc = matmul_device(A, -1.0, X, ldx, a, m, m, H2_F64, st, tr, false))) return fail(rc);
    k_gm_relnorm<<<grid, blk, 0, st>>>(a, B, ldb, g, g.rel);
    std::vector<double> rel(m);
    std::vector<int> it(m);
    ce = cudaMemcpyAsync(rel.data(), g.rel, m * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(it.data(), g.col_it, m * sizeof(int), cudaMemcpyDeviceToHost, st);
    cleanup();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); return H2_E_CUDA; }
    if (res->rel_residual) for (int64_t i = 0; i < m; ++i) res->rel_residual[i] = rel[i];
    if (res->col_iterations) for (int64_t i = 0; i < m; ++i) res->col_iterations[i] = it[i];
    int mx = 0;
    for (int v : it) mx = std::max(mx, v);
    res->iterations = mx;
    res->outer_steps = cycles;
    res->h2mm_calls = h2mm;
    res->status = status;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (status == H2_E_NOCONVERGE) set_error("block GMRES did not converge within max_iter");
    return status;
}

}  // namespace h2
