// Block CG with m×m Gram matrices (variant H2_CG_GRAM): O'Leary's block CG
// written in the conjugacy form of Sec. 5.1, Alg. "CG", with the per-column
// scalars replaced by m×m matrices,
//
//   G = Pᵀ(AP),  W = PᵀR,  α = G⁻¹W,  X += Pα,  R -= (AP)α,
//   Γ = G⁻¹(AP)ᵀR,  P = R - PΓ.
//
// G⁻¹ is applied through a Cholesky factor of G computed with deflation: in
// index order, direction j is kept when its Schur pivot exceeds kDeflate times
// its diagonal (it is not A-dependent on the kept directions before it) and
// dropped for this step otherwise; a diagonal <p_j, A p_j> <= 0 on an active
// column is a breakdown.  Columns that reach the tolerance are frozen: their
// columns of α and Γ are zero and their direction is zero.
//
// Everything runs in FP64 on the device.  Per iteration, after the product:
//   k_gram_partial      per-CTA partial sums of [G | W] over row tiles
//   k_gram_reduce<0>    fixed-order sum of the partials: G, W
//   k_gram_solve<0>     deflating Cholesky of G and α = G⁻¹W, 4 columns per CTA
//   k_gram_update       X += Pα, R -= (AP)α, partial sums of (AP)ᵀR and |r_j|²
//   k_gram_reduce<1>    fixed-order sum: (AP)ᵀR, |r_j|²
//   k_gram_solve<1>     active set and Γ = G⁻¹(AP)ᵀR, 4 columns per CTA
//   k_gram_dir          P = R - PΓ (zero on inactive columns)
// The row passes are FP64-FMA bound (2m² flops per row and Gram product).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "h2_internal.cuh"

namespace h2 {

namespace {

constexpr int kGramCtas = 152;   // one CTA per SM for the row passes
constexpr int kTRg = 16;         // rows per tile in the Gram pass
constexpr int kTRu = 8;          // rows per tile in the update and direction passes
constexpr double kDeflate = 1e-10;
constexpr int kSolveLd = kGramMaxCols + 1;

__host__ __device__ __forceinline__ int pstride(int m) { return 2 * m * m + m; }

// part[cta][0:m²] = Uᵀ V0, part[cta][m²:2m²] = Uᵀ V1 over the CTA's row tiles
// (U, V0, V1: n×m, ld m).  MP is m rounded up to 16, 32 or 64; thread (tx, ty)
// owns entries (ty + 16a, tx + 16b).
template <int MP, int NT>
__global__ void __launch_bounds__(256) k_gram_partial(const double* __restrict__ U, const double* __restrict__ V0,
                                                      const double* __restrict__ V1, int64_t n, int m,
                                                      double* __restrict__ part) {
    constexpr int T = MP / 16;
    __shared__ double su[kTRg][MP], s0[kTRg][MP], s1[kTRg][MP];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double a0[T][T], a1[T][T];
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) a0[i][j] = a1[i][j] = 0.0;
    const int64_t tiles = (n + kTRg - 1) / kTRg;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * kTRg;
        for (int e = threadIdx.x; e < kTRg * MP; e += 256) {
            const int r = e / MP, c = e % MP;
            const int64_t row = r0 + r;
            const bool ok = row < n && c < m;
            su[r][c] = ok ? U[row * m + c] : 0.0;
            s0[r][c] = ok ? V0[row * m + c] : 0.0;
            if (NT == 2) s1[r][c] = ok ? V1[row * m + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kTRg; ++r) {
            double u[T], v0[T], v1[T];
#pragma unroll
            for (int i = 0; i < T; ++i) {
                u[i] = su[r][ty + 16 * i];
                v0[i] = s0[r][tx + 16 * i];
                v1[i] = NT == 2 ? s1[r][tx + 16 * i] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j) {
                    a0[i][j] = fma(u[i], v0[j], a0[i][j]);
                    if (NT == 2) a1[i][j] = fma(u[i], v1[j], a1[i][j]);
                }
        }
        __syncthreads();
    }
    double* out = part + (size_t)blockIdx.x * pstride(m);
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int r = ty + 16 * i, c = tx + 16 * j;
            if (r < m && c < m) {
                out[r * m + c] = a0[i][j];
                if (NT == 2) out[m * m + r * m + c] = a1[i][j];
            }
        }
}

// Fixed-order sum of the per-CTA partials: PHASE 0 gives G = Pᵀ(AP) and
// W = PᵀR, PHASE 1 gives C = (AP)ᵀR and |r_j|².
template <int PHASE>
__global__ void __launch_bounds__(256) k_gram_reduce(int nct, int m, GramDev g) {
    const int ps = pstride(m);
    const int nterm = PHASE == 0 ? 2 * m * m : m * m + m;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nterm) return;
    // four interleaved partial sums keep loads in flight; fixed order
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    int c = 0;
    for (; c + 3 < nct; c += 4)
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[u] += __ldcg(&g.part[(size_t)(c + u) * ps + e]);
    for (; c < nct; ++c) s4[0] += __ldcg(&g.part[(size_t)c * ps + e]);
    const double s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    if (e < m * m) (PHASE == 0 ? g.G : g.W)[e] = s;
    else if (PHASE == 0) g.W[e - m * m] = s;
    else g.rr[e - m * m] = s;
}

constexpr int kSolveCols = 4;     // right-hand-side columns of the m×m solve per CTA
constexpr int kSolveThreads = 128;

// The m×m step, kSolveCols columns per CTA.
// PHASE 0: every CTA factors G (deflating Cholesky, identical in all CTAs) and
//   solves α[:, c] = G_KK⁻¹ W[K, c] for its active columns c; CTA 0 keeps L and
//   the kept set for PHASE 1.
// PHASE 1: each CTA updates the active set of its columns from |r_c| and solves
//   Γ[:, c] = G_KK⁻¹ C[K, c] for those still active.
template <int PHASE>
__global__ void __launch_bounds__(kSolveThreads) k_gram_solve(int m, double tol, GramDev g, CgDev d) {
    __shared__ double sA[kGramMaxCols][kSolveLd];
    __shared__ double sB[kGramMaxCols][kSolveCols];
    __shared__ double sdg[kGramMaxCols];
    __shared__ int sk[kGramMaxCols], sa[kGramMaxCols], sown[kSolveCols];
    __shared__ int sbrk;
    const int t = threadIdx.x;
    const int c0 = blockIdx.x * kSolveCols;
    const int nc = min(kSolveCols, m - c0);
    if (t == 0) sbrk = 0;
    if (PHASE == 0) {
        for (int x = t; x < m * m; x += blockDim.x) sA[x / m][x % m] = __ldcg(&g.G[x]);
        for (int j = t; j < m; j += blockDim.x) {
            sa[j] = d.active[j] != 0;
            sdg[j] = __ldcg(&g.G[j * m + j]);
        }
        __syncthreads();
        // right-looking Cholesky with deflation
        for (int j = 0; j < m; ++j) {
            if (t == 0) {
                int keep = 0;
                if (sa[j]) {
                    const double gjj = sdg[j];
                    if (!(gjj > 0.0) || !isfinite(gjj)) {
                        sbrk = 1;
                    } else {
                        const double dj = sA[j][j];
                        if (dj > kDeflate * gjj) {
                            keep = 1;
                            sA[j][j] = sqrt(dj);
                        }
                    }
                }
                sk[j] = keep;
            }
            __syncthreads();
            if (sk[j]) {
                const double piv = sA[j][j];
                for (int i = j + 1 + t; i < m; i += blockDim.x) sA[i][j] /= piv;
                __syncthreads();
                const int w = m - j - 1;
                for (int x = t; x < w * w; x += blockDim.x) {
                    const int i = j + 1 + x / w, k = j + 1 + x % w;
                    if (k <= i) sA[i][k] -= sA[i][j] * sA[k][j];
                }
            }
            __syncthreads();
        }
        for (int c = t; c < nc; c += blockDim.x) sown[c] = sa[c0 + c];
        for (int x = t; x < m * nc; x += blockDim.x) sB[x / nc][x % nc] = __ldcg(&g.W[(x / nc) * m + c0 + x % nc]);
        if (blockIdx.x == 0) {
            for (int x = t; x < m * m; x += blockDim.x) g.L[x] = sA[x / m][x % m];
            for (int j = t; j < m; j += blockDim.x) g.kept[j] = sk[j];
        }
    } else {
        for (int x = t; x < m * m; x += blockDim.x) sA[x / m][x % m] = __ldcg(&g.L[x]);
        for (int j = t; j < m; j += blockDim.x) sk[j] = __ldcg(&g.kept[j]);
        for (int c = t; c < nc; c += blockDim.x) {
            const int col = c0 + c;
            int act = d.active[col] != 0;
            if (act) {
                const double rn = sqrt(__ldcg(&g.rr[col]));
                d.rnorm[col] = rn;
                d.conv_iter[col] += 1;  // iterations while active
                if (!isfinite(rn)) atomicOr(&d.summary[1], 1);
                if (rn / d.bnorm[col] <= tol) {
                    act = 0;
                    d.active[col] = 0;
                    atomicSub(&d.summary[0], 1);
                }
            }
            sown[c] = act;
        }
        for (int x = t; x < m * nc; x += blockDim.x) sB[x / nc][x % nc] = __ldcg(&g.W[(x / nc) * m + c0 + x % nc]);
    }
    __syncthreads();
    // sB[:, c] = G_KK⁻¹ sB[K, c]: L z = b, then Lᵀ y = z; rows outside K are 0
    for (int j = 0; j < m; ++j) {
        if (sk[j]) {
            const double piv = sA[j][j];
            if (t < nc) sB[j][t] /= piv;
            __syncthreads();
            const int w = m - j - 1;
            for (int x = t; x < w * nc; x += blockDim.x) {
                const int i = j + 1 + x / nc, c = x % nc;
                sB[i][c] -= sA[i][j] * sB[j][c];
            }
        } else if (t < nc) {
            sB[j][t] = 0.0;
        }
        __syncthreads();
    }
    for (int j = m - 1; j >= 0; --j) {
        if (sk[j]) {
            const double piv = sA[j][j];
            if (t < nc) sB[j][t] /= piv;
            __syncthreads();
            for (int x = t; x < j * nc; x += blockDim.x) {
                const int i = x / nc, c = x % nc;
                if (sk[i]) sB[i][c] -= sA[j][i] * sB[j][c];
            }
        }
        __syncthreads();
    }
    double* out = PHASE == 0 ? g.alpha : g.gamma;
    for (int x = t; x < m * nc; x += blockDim.x) {
        const int i = x / nc, c = x % nc;
        const double v = sB[i][c];
        const bool ok = sown[c] && isfinite(v);
        if (sown[c] && !isfinite(v)) sbrk = 1;
        out[i * m + c0 + c] = (ok && !(PHASE == 0 && sbrk)) ? v : 0.0;
    }
    __syncthreads();
    if (t == 0 && sbrk) atomicOr(&d.summary[1], 1);
}

// X += Pα, R -= Qα (Q = AP) over the CTA's row tiles, then the partial sums of
// QᵀR_new and |r_j|² for k_gram_reduce<1>.
template <int MP, bool WITH_C>
__global__ void __launch_bounds__(256) k_gram_update(double* __restrict__ X, int64_t ldx, const double* __restrict__ P,
                                                     const double* __restrict__ Q, double* __restrict__ R, int64_t n,
                                                     int m, const double* __restrict__ alpha,
                                                     double* __restrict__ part) {
    constexpr int T = MP / 16;
    __shared__ double sal[MP][MP];
    __shared__ double sp[kTRu][MP], sq[kTRu][MP], sr[kTRu][MP];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    for (int x = t; x < MP * MP; x += 256) {
        const int i = x / MP, j = x % MP;
        sal[i][j] = (i < m && j < m) ? alpha[i * m + j] : 0.0;
    }
    double acc[T][T];
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = 0.0;
    double rr = 0.0;
    const int64_t tiles = (n + kTRu - 1) / kTRu;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * kTRu;
        __syncthreads();  // sal written (first tile); previous tile's reads done
        for (int e = t; e < kTRu * MP; e += 256) {
            const int r = e / MP, c = e % MP;
            const int64_t row = r0 + r;
            const bool ok = row < n && c < m;
            sp[r][c] = ok ? P[row * m + c] : 0.0;
            sq[r][c] = ok ? Q[row * m + c] : 0.0;
            sr[r][c] = ok ? R[row * m + c] : 0.0;
        }
        __syncthreads();
        for (int o = t; o < kTRu * MP; o += 256) {
            const int r = o / MP, j = o % MP;
            double xs = 0.0, rs = 0.0;
#pragma unroll 16
            for (int i = 0; i < MP; ++i) {
                xs = fma(sp[r][i], sal[i][j], xs);
                rs = fma(sq[r][i], sal[i][j], rs);
            }
            const int64_t row = r0 + r;
            if (row < n && j < m) {
                const double rn = sr[r][j] - rs;
                X[row * ldx + j] += xs;
                R[row * m + j] = rn;
                sr[r][j] = rn;
            }
        }
        __syncthreads();
        if (WITH_C)
#pragma unroll
        for (int r = 0; r < kTRu; ++r) {
            double u[T], v[T];
#pragma unroll
            for (int i = 0; i < T; ++i) {
                u[i] = sq[r][ty + 16 * i];
                v[i] = sr[r][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j) acc[i][j] = fma(u[i], v[j], acc[i][j]);
        }
        if (t < MP)
#pragma unroll
            for (int r = 0; r < kTRu; ++r) rr = fma(sr[r][t], sr[r][t], rr);
    }
    double* out = part + (size_t)blockIdx.x * pstride(m);
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int r = ty + 16 * i, c = tx + 16 * j;
            if (r < m && c < m) out[r * m + c] = WITH_C ? acc[i][j] : 0.0;
        }
    if (t < m) out[m * m + t] = rr;
}

// P = R - PΓ on active columns, 0 on the others (in place, row tile by tile).
template <int MP>
__global__ void __launch_bounds__(256) k_gram_dir(double* __restrict__ P, const double* __restrict__ R, int64_t n,
                                                  int m, const double* __restrict__ gamma,
                                                  const int* __restrict__ active) {
    __shared__ double sg[MP][MP];
    __shared__ double sp[kTRu][MP];
    __shared__ int sa[MP];
    const int t = threadIdx.x;
    for (int x = t; x < MP * MP; x += 256) {
        const int i = x / MP, j = x % MP;
        sg[i][j] = (i < m && j < m) ? gamma[i * m + j] : 0.0;
    }
    for (int j = t; j < MP; j += 256) sa[j] = j < m ? active[j] != 0 : 0;
    const int64_t tiles = (n + kTRu - 1) / kTRu;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * kTRu;
        __syncthreads();
        for (int e = t; e < kTRu * MP; e += 256) {
            const int r = e / MP, c = e % MP;
            const int64_t row = r0 + r;
            sp[r][c] = (row < n && c < m) ? P[row * m + c] : 0.0;
        }
        __syncthreads();
        for (int o = t; o < kTRu * MP; o += 256) {
            const int r = o / MP, j = o % MP;
            const int64_t row = r0 + r;
            if (row >= n || j >= m) continue;
            double v = 0.0;
            if (sa[j]) {
                double s = 0.0;
#pragma unroll 16
                for (int i = 0; i < MP; ++i) s = fma(sp[r][i], sg[i][j], s);
                v = R[row * m + j] - s;
            }
            P[row * m + j] = v;
        }
    }
}

__global__ void k_gram_mask(double* __restrict__ P, int64_t n, int m, const int* __restrict__ active) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        if (!active[e % m]) P[e] = 0.0;
}

unsigned row_grid(int64_t n, int rows) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + rows - 1) / rows, kGramCtas)); }

template <int MP>
int launch_alpha(const double* P, const double* AP, const double* R, int64_t n, int m, const GramDev& g,
                 const CgDev& d, cudaStream_t st) {
    const unsigned gp = row_grid(n, kTRg);
    k_gram_partial<MP, 2><<<gp, 256, 0, st>>>(P, AP, R, n, m, g.part);
    H2_LAUNCH_CHECK();
    const unsigned gr = (unsigned)((2 * m * m + 255) / 256);
    k_gram_reduce<0><<<gr, 256, 0, st>>>((int)gp, m, g);
    H2_LAUNCH_CHECK();
    k_gram_solve<0><<<(unsigned)((m + kSolveCols - 1) / kSolveCols), kSolveThreads, 0, st>>>(m, 0.0, g, d);
    H2_LAUNCH_CHECK();
    return 0;
}

template <int MP>
int launch_update(double* X, int64_t ldx, const double* P, const double* AP, double* R, int64_t n, int m,
                  bool with_c, const GramDev& g, cudaStream_t st) {
    const unsigned gu = row_grid(n, kTRu);
    if (with_c) k_gram_update<MP, true><<<gu, 256, 0, st>>>(X, ldx, P, AP, R, n, m, g.alpha, g.part);
    else k_gram_update<MP, false><<<gu, 256, 0, st>>>(X, ldx, P, AP, R, n, m, g.alpha, g.part);
    H2_LAUNCH_CHECK();
    return 0;
}

template <int MP>
int launch_c_partial(const double* AP, const double* Z, int64_t n, int m, const GramDev& g, cudaStream_t st) {
    // the partials of the update pass hold zeros in the C slots of its CTAs;
    // this pass (no more CTAs than the update pass) overwrites them
    k_gram_partial<MP, 1><<<row_grid(n, kTRg), 256, 0, st>>>(AP, Z, nullptr, n, m, g.part);
    H2_LAUNCH_CHECK();
    return 0;
}

template <int MP>
int launch_gamma_dir(double* P, const double* D, int64_t n, int m, double tol, const GramDev& g, const CgDev& d,
                     cudaStream_t st) {
    const unsigned gu = row_grid(n, kTRu);
    const unsigned gr = (unsigned)((m * m + m + 255) / 256);
    k_gram_reduce<1><<<gr, 256, 0, st>>>((int)gu, m, g);
    H2_LAUNCH_CHECK();
    k_gram_solve<1><<<(unsigned)((m + kSolveCols - 1) / kSolveCols), kSolveThreads, 0, st>>>(m, tol, g, d);
    H2_LAUNCH_CHECK();
    k_gram_dir<MP><<<gu, 256, 0, st>>>(P, D, n, m, g.gamma, d.active);
    H2_LAUNCH_CHECK();
    return 0;
}

size_t carve_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t gram_scratch_bytes(int m) {
    const size_t mm = (size_t)m * m * sizeof(double);
    return carve_up((size_t)kGramCtas * pstride(m) * sizeof(double)) + 5 * carve_up(mm) +
           carve_up(m * sizeof(double)) + carve_up(m * sizeof(int)) + carve_up(sizeof(unsigned));
}

void gram_carve(GramDev* g, void* base, int m) {
    char* p = (char*)base;
    const size_t mm = carve_up((size_t)m * m * sizeof(double));
    g->part = (double*)p;
    p += carve_up((size_t)kGramCtas * pstride(m) * sizeof(double));
    g->G = (double*)p;
    p += mm;
    g->W = (double*)p;
    p += mm;
    g->L = (double*)p;
    p += mm;
    g->alpha = (double*)p;
    p += mm;
    g->gamma = (double*)p;
    p += mm;
    g->rr = (double*)p;
    p += carve_up(m * sizeof(double));
    g->kept = (int*)p;
    p += carve_up(m * sizeof(int));
    g->ticket = (unsigned*)p;
}

namespace {
int g_gram_attr_device = -1;
}

int gram_prepare() {
    int dev = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    if (dev == g_gram_attr_device) return 0;
    g_gram_attr_device = dev;
    return 0;
}

int gram_start(double* P, const double* R, int64_t n, int m, const GramDev& g, const CgDev& d, cudaStream_t st) {
    if (m < 1 || m > kGramMaxCols) { set_error("the Gram-matrix block CG takes 1 <= m <= 64 columns"); return H2_E_UNSUPPORTED; }
    H2_CUDA_TRY(cudaMemsetAsync(g.ticket, 0, sizeof(unsigned), st));
    H2_CUDA_TRY(cudaMemsetAsync(P, 0, (size_t)n * m * sizeof(double), st));
    H2_CUDA_TRY(cudaMemsetAsync(g.gamma, 0, (size_t)m * m * sizeof(double), st));
    const unsigned gu = row_grid(n, kTRu);
    if (m <= 16) k_gram_dir<16><<<gu, 256, 0, st>>>(P, R, n, m, g.gamma, d.active);
    else if (m <= 32) k_gram_dir<32><<<gu, 256, 0, st>>>(P, R, n, m, g.gamma, d.active);
    else k_gram_dir<64><<<gu, 256, 0, st>>>(P, R, n, m, g.gamma, d.active);
    H2_LAUNCH_CHECK();
    return 0;
}

int gram_alpha(const double* P, const double* AP, const double* R, int64_t n, int m, const GramDev& g,
               const CgDev& d, cudaStream_t st) {
    if (m <= 16) return launch_alpha<16>(P, AP, R, n, m, g, d, st);
    if (m <= 32) return launch_alpha<32>(P, AP, R, n, m, g, d, st);
    return launch_alpha<64>(P, AP, R, n, m, g, d, st);
}

#define H2_GRAM_DISPATCH(call) (m <= 16 ? call<16> : m <= 32 ? call<32> : call<64>)

int gram_update_dir(double* X, int64_t ldx, double* P, const double* AP, double* R, int64_t n, int m, double tol,
                    const GramDev& g, const CgDev& d, cudaStream_t st) {
    int rc = H2_GRAM_DISPATCH(launch_update)(X, ldx, P, AP, R, n, m, true, g, st);
    if (rc) return rc;
    return H2_GRAM_DISPATCH(launch_gamma_dir)(P, R, n, m, tol, g, d, st);
}

int gram_update(double* X, int64_t ldx, const double* P, const double* AP, double* R, int64_t n, int m,
                const GramDev& g, cudaStream_t st) {
    return H2_GRAM_DISPATCH(launch_update)(X, ldx, P, AP, R, n, m, false, g, st);
}

int gram_gamma_dir_from(double* P, const double* AP, const double* Z, int64_t n, int m, double tol,
                        const GramDev& g, const CgDev& d, cudaStream_t st) {
    int rc = H2_GRAM_DISPATCH(launch_c_partial)(AP, Z, n, m, g, st);
    if (rc) return rc;
    return H2_GRAM_DISPATCH(launch_gamma_dir)(P, Z, n, m, tol, g, d, st);
}

int gram_mask(double* P, int64_t n, int m, const CgDev& d, cudaStream_t st) {
    const unsigned g = (unsigned)std::min<int64_t>((n * m + 255) / 256, 152 * 16);
    k_gram_mask<<<g, 256, 0, st>>>(P, n, m, d.active);
    H2_LAUNCH_CHECK();
    return 0;
}

}  // namespace h2
