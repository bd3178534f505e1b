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
//   k_gram_reduce<0>    fixed-order sum of the partials; the last CTA factors
//                       G and solves α
//   k_gram_update       X += Pα, R -= (AP)α, partial sums of (AP)ᵀR and |r_j|²
//   k_gram_reduce<1>    fixed-order sum; the last CTA updates the active set
//                       and solves Γ
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
constexpr int kSolveSmem = 2 * kGramMaxCols * kSolveLd * (int)sizeof(double);

__device__ __forceinline__ bool gram_last_cta(unsigned* ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__host__ __device__ __forceinline__ int pstride(int m) { return 2 * m * m + m; }

// part[cta][0:m²] = Uᵀ V0, part[cta][m²:2m²] = Uᵀ V1 over the CTA's row tiles
// (U, V0, V1: n×m, ld m).  MP is m rounded up to 16, 32 or 64; thread (tx, ty)
// owns entries (ty + 16a, tx + 16b).
template <int MP>
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
            s1[r][c] = ok ? V1[row * m + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kTRg; ++r) {
            double u[T], v0[T], v1[T];
#pragma unroll
            for (int i = 0; i < T; ++i) {
                u[i] = su[r][ty + 16 * i];
                v0[i] = s0[r][tx + 16 * i];
                v1[i] = s1[r][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j) {
                    a0[i][j] = fma(u[i], v0[j], a0[i][j]);
                    a1[i][j] = fma(u[i], v1[j], a1[i][j]);
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
                out[m * m + r * m + c] = a1[i][j];
            }
        }
}

// B[:, c] = G_KK⁻¹ B[K, c] for every column c < m, with L (lower, on K) from a
// deflating Cholesky; rows outside K become 0.  All threads of the CTA call it.
__device__ void tri_solve(double (*sA)[kSolveLd], double (*sB)[kSolveLd], const int* sk, int m) {
    const int t = threadIdx.x;
    for (int j = 0; j < m; ++j) {  // L z = b
        if (sk[j]) {
            const double piv = sA[j][j];
            for (int c = t; c < m; c += blockDim.x) sB[j][c] /= piv;
            __syncthreads();
            const int w = m - j - 1;
            for (int x = t; x < w * m; x += blockDim.x) {
                const int i = j + 1 + x / m, c = x % m;
                sB[i][c] -= sA[i][j] * sB[j][c];
            }
        } else {
            for (int c = t; c < m; c += blockDim.x) sB[j][c] = 0.0;
        }
        __syncthreads();
    }
    for (int j = m - 1; j >= 0; --j) {  // Lᵀ y = z
        if (sk[j]) {
            const double piv = sA[j][j];
            for (int c = t; c < m; c += blockDim.x) sB[j][c] /= piv;
            __syncthreads();
            for (int x = t; x < j * m; x += blockDim.x) {
                const int i = x / m, c = x % m;
                if (sk[i]) sB[i][c] -= sA[j][i] * sB[j][c];
            }
        }
        __syncthreads();
    }
}

// Fixed-order sum of the per-CTA partials, then (last CTA) the m×m step:
// PHASE 0: G, W -> deflating Cholesky of G, α = G⁻¹W on active columns;
// PHASE 1: C = (AP)ᵀR, |r_j|² -> active set, Γ = G⁻¹C on still-active columns.
template <int PHASE>
__global__ void __launch_bounds__(256) k_gram_reduce(int nct, int m, double tol, GramDev g, CgDev d) {
    extern __shared__ double dsm[];
    __shared__ int sk[kGramMaxCols], sa[kGramMaxCols];
    __shared__ double sdg[kGramMaxCols];
    __shared__ int sbrk;
    const int ps = pstride(m);
    const int nterm = PHASE == 0 ? 2 * m * m : m * m + m;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nterm) {
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
    if (!gram_last_cta(g.ticket)) return;
    double(*sA)[kSolveLd] = (double(*)[kSolveLd])dsm;
    double(*sB)[kSolveLd] = (double(*)[kSolveLd])(dsm + kGramMaxCols * kSolveLd);
    const int t = threadIdx.x;
    if (t == 0) sbrk = 0;
    if (PHASE == 0) {
        for (int x = t; x < m * m; x += blockDim.x) {
            const int i = x / m, j = x % m;
            sA[i][j] = __ldcg(&g.G[x]);
            sB[i][j] = __ldcg(&g.W[x]);
        }
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
        tri_solve(sA, sB, sk, m);
        for (int x = t; x < m * m; x += blockDim.x) {
            const int i = x / m, c = x % m;
            const double a = sB[i][c];
            g.alpha[x] = (sa[c] && !sbrk && isfinite(a)) ? a : 0.0;
            g.L[x] = sA[i][c];
            if (sa[c] && !isfinite(a)) sbrk = 1;
        }
        for (int j = t; j < m; j += blockDim.x) g.kept[j] = sk[j];
        __syncthreads();
        if (t == 0 && sbrk) atomicOr(&d.summary[1], 1);
    } else {
        for (int x = t; x < m * m; x += blockDim.x) {
            const int i = x / m, j = x % m;
            sA[i][j] = __ldcg(&g.L[x]);
            sB[i][j] = __ldcg(&g.W[x]);
        }
        for (int j = t; j < m; j += blockDim.x) {
            sk[j] = __ldcg(&g.kept[j]);
            int act = d.active[j] != 0;
            if (act) {
                const double rn = sqrt(__ldcg(&g.rr[j]));
                d.rnorm[j] = rn;
                d.conv_iter[j] += 1;  // iterations while active
                if (!isfinite(rn)) atomicOr(&d.summary[1], 1);
                if (rn / d.bnorm[j] <= tol) {
                    act = 0;
                    d.active[j] = 0;
                    atomicSub(&d.summary[0], 1);
                }
            }
            sa[j] = act;
        }
        __syncthreads();
        tri_solve(sA, sB, sk, m);
        for (int x = t; x < m * m; x += blockDim.x) {
            const int c = x % m;
            const double v = sB[x / m][c];
            g.gamma[x] = (sa[c] && isfinite(v)) ? v : 0.0;
            if (sa[c] && !isfinite(v)) sbrk = 1;
        }
        __syncthreads();
        if (t == 0 && sbrk) atomicOr(&d.summary[1], 1);
    }
    if (t == 0) *g.ticket = 0;
}

// X += Pα, R -= Qα (Q = AP) over the CTA's row tiles, then the partial sums of
// QᵀR_new and |r_j|² for k_gram_reduce<1>.
template <int MP>
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
            if (r < m && c < m) out[r * m + c] = acc[i][j];
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
    k_gram_partial<MP><<<gp, 256, 0, st>>>(P, AP, R, n, m, g.part);
    H2_LAUNCH_CHECK();
    const unsigned gr = (unsigned)((2 * m * m + 255) / 256);
    k_gram_reduce<0><<<gr, 256, kSolveSmem, st>>>((int)gp, m, 0.0, g, d);
    H2_LAUNCH_CHECK();
    return 0;
}

template <int MP>
int launch_update_dir(double* X, int64_t ldx, double* P, const double* AP, double* R, int64_t n, int m, double tol,
                      const GramDev& g, const CgDev& d, cudaStream_t st) {
    const unsigned gu = row_grid(n, kTRu);
    k_gram_update<MP><<<gu, 256, 0, st>>>(X, ldx, P, AP, R, n, m, g.alpha, g.part);
    H2_LAUNCH_CHECK();
    const unsigned gr = (unsigned)((m * m + m + 255) / 256);
    k_gram_reduce<1><<<gr, 256, kSolveSmem, st>>>((int)gu, m, tol, g, d);
    H2_LAUNCH_CHECK();
    k_gram_dir<MP><<<gu, 256, 0, st>>>(P, R, n, m, g.gamma, d.active);
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
    H2_CUDA_TRY(cudaFuncSetAttribute(k_gram_reduce<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_gram_reduce<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem));
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

int gram_update_dir(double* X, int64_t ldx, double* P, const double* AP, double* R, int64_t n, int m, double tol,
                    const GramDev& g, const CgDev& d, cudaStream_t st) {
    if (m <= 16) return launch_update_dir<16>(X, ldx, P, AP, R, n, m, tol, g, d, st);
    if (m <= 32) return launch_update_dir<32>(X, ldx, P, AP, R, n, m, tol, g, d, st);
    return launch_update_dir<64>(X, ldx, P, AP, R, n, m, tol, g, d, st);
}

int gram_mask(double* P, int64_t n, int m, const CgDev& d, cudaStream_t st) {
    const unsigned g = (unsigned)std::min<int64_t>((n * m + 255) / 256, 152 * 16);
    k_gram_mask<<<g, 256, 0, st>>>(P, n, m, d.active);
    H2_LAUNCH_CHECK();
    return 0;
}

}  // namespace h2
