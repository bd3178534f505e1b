// Block-Jacobi preconditioner for the preconditioned block CG (Sec. 5.1,
// Alg. "pcg block"): M = blockdiag over the leaves t of D_t = G_(t,t) + σI,
// the diagonal inadmissible blocks with the shift (always present: a leaf is
// never admissible with itself, dist = 0).  D_t is a kernel matrix of the
// exponential kernel plus σI, symmetric positive definite; n_t <= 64.
//
// Setup (k_bj_invert, once per matrix and σ): one CTA per leaf factors
// D_t = L Lᵀ in shared memory and forms D_t⁻¹ = L⁻ᵀ L⁻¹ in FP64.
// Apply (k_bj_apply, every iteration): Z|_t̂ = D_t⁻¹ R|_t̂ per leaf, rows
// gathered from and scattered to the caller's point order, 2 n_t² m flops per
// leaf; optionally the per-column dots <AP_i, Z_i> for γ_i of the paper's
// recurrence, reduced in fixed order by the last CTA.  In FP64, or, inside the
// low-precision iterations of a mixed solve, in FP32 with the inverses rounded
// to FP32 (R and Z stay FP64 in memory, the dots accumulate in FP64): the
// apply is then as cheap next to the FP32 product as the FP64 apply is next
// to the FP64 one, and its rounding stays below the FP32 product's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "h2_internal.cuh"

namespace h2 {

namespace {

constexpr int kLd = 65;           // padded row length of the 64×64 shared tiles
constexpr int kBjCtas = 456;      // CTAs of the apply pass (three per SM)
constexpr int kBjSmem = 2 * 64 * kLd * (int)sizeof(double);

__device__ __forceinline__ bool bj_last_cta(unsigned* ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__global__ void __launch_bounds__(256) k_bj_invert(const int32_t* __restrict__ leaves, int NL,
                                                   const int32_t* __restrict__ cl_size,
                                                   const int64_t* __restrict__ diag_off,
                                                   const double* __restrict__ near, double sigma,
                                                   const int64_t* __restrict__ bj_off, double* __restrict__ inv,
                                                   int* __restrict__ err) {
    extern __shared__ double sm[];
    double(*sA)[kLd] = (double(*)[kLd])sm;
    double(*sB)[kLd] = (double(*)[kLd])(sm + 64 * kLd);
    __shared__ int bad;
    const int t = threadIdx.x;
    for (int lp = blockIdx.x; lp < NL; lp += gridDim.x) {
        const int l = cl_size[leaves[lp]];
        const double* g = near + diag_off[lp];
        if (t == 0) bad = 0;
        for (int x = t; x < l * l; x += blockDim.x) {
            const int i = x / l, j = x % l;
            sA[i][j] = g[x] + (i == j ? sigma : 0.0);
            sB[i][j] = i == j ? 1.0 : 0.0;
        }
        __syncthreads();
        // right-looking Cholesky D = L Lᵀ (lower triangle of sA)
        for (int j = 0; j < l; ++j) {
            if (t == 0) {
                const double d = sA[j][j];
                if (!(d > 0.0) || !isfinite(d)) {
                    bad = 1;
                    sA[j][j] = 1.0;
                } else {
                    sA[j][j] = sqrt(d);
                }
            }
            __syncthreads();
            const double piv = sA[j][j];
            for (int i = j + 1 + t; i < l; i += blockDim.x) sA[i][j] /= piv;
            __syncthreads();
            const int w = l - j - 1;
            for (int x = t; x < w * w; x += blockDim.x) {
                const int i = j + 1 + x / w, k = j + 1 + x % w;
                if (k <= i) sA[i][k] -= sA[i][j] * sA[k][j];
            }
            __syncthreads();
        }
        // D⁻¹ = L⁻ᵀ (L⁻¹ I): forward then backward substitution on all l columns
        for (int j = 0; j < l; ++j) {
            const double piv = sA[j][j];
            for (int c = t; c < l; c += blockDim.x) sB[j][c] /= piv;
            __syncthreads();
            const int w = l - j - 1;
            for (int x = t; x < w * l; x += blockDim.x) {
                const int i = j + 1 + x / l, c = x % l;
                sB[i][c] -= sA[i][j] * sB[j][c];
            }
            __syncthreads();
        }
        for (int j = l - 1; j >= 0; --j) {
            const double piv = sA[j][j];
            for (int c = t; c < l; c += blockDim.x) sB[j][c] /= piv;
            __syncthreads();
            for (int x = t; x < j * l; x += blockDim.x) {
                const int i = x / l, c = x % l;
                sB[i][c] -= sA[j][i] * sB[j][c];
            }
            __syncthreads();
        }
        double* out = inv + bj_off[lp];
        for (int x = t; x < l * l; x += blockDim.x) out[x] = sB[x / l][x % l];
        if (t == 0 && bad) atomicExch(err, 1);
        __syncthreads();
    }
}

// Z|_t̂ = D_t⁻¹ R|_t̂ for the CTA's leaves, in column chunks of 64; with AP the
// per-column partial sums of <AP, Z> go to d.partial[cta·m + c] and the last
// CTA forms γ_c = <AP_c, Z_c> / β_c on active columns.  Thread t owns column
// t mod cw of the chunk (cw = chunk width rounded up to 32 or 64) and every
// (256/cw)-th row of the leaf.  Three CTAs fit on an SM (66.5 KB of tiles each).
template <typename T>
__global__ void __launch_bounds__(256) k_bj_apply(const double* __restrict__ R, double* __restrict__ Z, int m,
                                                  const int32_t* __restrict__ perm,
                                                  const int32_t* __restrict__ leaves, int NL,
                                                  const int32_t* __restrict__ cl_off,
                                                  const int32_t* __restrict__ cl_size,
                                                  const int64_t* __restrict__ bj_off,
                                                  const T* __restrict__ inv, const double* __restrict__ AP,
                                                  CgDev d) {
    extern __shared__ double sm_raw[];
    T* sm = reinterpret_cast<T*>(sm_raw);
    T(*sD)[kLd] = (T(*)[kLd])sm;
    T(*sR)[kLd] = (T(*)[kLd])(sm + 64 * kLd);
    __shared__ double red[8][64];
    __shared__ int srow[64];
    const int t = threadIdx.x;
    for (int c0 = 0; c0 < m; c0 += 64) {
        const int mc = min(64, m - c0);
        const int cw = mc <= 32 ? 32 : 64;
        const int tc = t % cw, tr = t / cw, nr = 256 / cw;
        double aq = 0.0;
        for (int lp = blockIdx.x; lp < NL; lp += gridDim.x) {
            const int cl = leaves[lp];
            const int off = cl_off[cl], l = cl_size[cl];
            const T* Dt = inv + bj_off[lp];
            // The leaf's loads are issued together, each thread's into registers
            // (l² ≤ 4096 and l·mc ≤ 4096 entries: at most 16 per thread), so a leaf
            // waits for two rounds of global latency (D_t⁻¹ and the point indices,
            // then the rows of R) instead of one per loop trip.
            constexpr int kPer = 64 * 64 / 256;
            T dv[kPer];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int x = t + 256 * i;
                dv[i] = x < l * l ? Dt[x] : (T)0;
            }
            __syncthreads();  // previous leaf's tiles are consumed
            if (t < l) srow[t] = perm[off + t];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int x = t + 256 * i;
                if (x < l * l) sD[x / l][x % l] = dv[i];
            }
            __syncthreads();
            double rv[kPer];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int x = t + 256 * i;
                rv[i] = x < l * mc ? R[(int64_t)srow[x / mc] * m + c0 + x % mc] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int x = t + 256 * i;
                if (x < l * mc) sR[x / mc][x % mc] = (T)rv[i];
            }
            __syncthreads();
            if (tc < mc)
                for (int a = tr; a < l; a += nr) {
                    T z = 0;
                    for (int b = 0; b < l; ++b) z = fma(sD[a][b], sR[b][tc], z);
                    const int64_t e = (int64_t)srow[a] * m + c0 + tc;
                    Z[e] = (double)z;
                    if (AP) aq = fma(AP[e], (double)z, aq);
                }
        }
        if (AP) {
            red[tr][tc] = aq;
            __syncthreads();
            if (t < mc) {
                double sum = 0.0;
                for (int y = 0; y < nr; ++y) sum += red[y][t];
                d.partial[(size_t)blockIdx.x * m + c0 + t] = sum;
            }
            __syncthreads();
        }
    }
    if (!AP || !bj_last_cta(d.ticket)) return;
    for (int c = t; c < m; c += blockDim.x) {
        if (!d.active[c]) continue;
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        unsigned b = 0;
        for (; b + 3 < gridDim.x; b += 4)
#pragma unroll
            for (unsigned u = 0; u < 4; ++u) s4[u] += __ldcg(&d.partial[(size_t)(b + u) * m + c]);
        for (; b < gridDim.x; ++b) s4[0] += __ldcg(&d.partial[(size_t)b * m + c]);
        const double gmm = ((s4[0] + s4[1]) + (s4[2] + s4[3])) / d.beta[c];
        d.gamma[c] = gmm;
        if (!isfinite(gmm)) atomicOr(&d.summary[1], 1);
    }
    if (t == 0) d.ticket[0] = 0;
}

__global__ void k_bj_round_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

int g_bj_attr_device = -1;

int bj_attr() {
    int dev = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    if (dev == g_bj_attr_device) return 0;
    H2_CUDA_TRY(cudaFuncSetAttribute(k_bj_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, kBjSmem));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_bj_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBjSmem));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_bj_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBjSmem));
    g_bj_attr_device = dev;
    return 0;
}

}  // namespace

int bj_prepare(h2_matrix* A, cudaStream_t st) {
    int rc = bj_attr();
    if (rc) return rc;
    if (A->bj_valid && A->bj_sigma == A->sigma) return 0;
    const int NL = (int)A->leaves.size();
    if (!A->bj_inv) {
        std::vector<int64_t> off(NL);
        int64_t acc = 0;
        for (int lp = 0; lp < NL; ++lp) {
            off[lp] = acc;
            const int64_t l = A->T.size[A->leaves[lp]];
            if (l > 64) { set_error("block-Jacobi preconditioner: leaf larger than 64 points"); return H2_E_UNSUPPORTED; }
            acc += l * l;
        }
        if ((rc = device_alloc(A, (void**)&A->bj_off, NL * sizeof(int64_t)))) return rc;
        if ((rc = device_alloc(A, (void**)&A->bj_inv, std::max<int64_t>(acc, 1) * sizeof(double)))) return rc;
        if ((rc = device_alloc(A, (void**)&A->bj_inv32, std::max<int64_t>(acc, 1) * sizeof(float)))) return rc;
        A->bj_count = acc;
        H2_CUDA_TRY(cudaMemcpyAsync(A->bj_off, off.data(), NL * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));  // `off` is pageable host memory
    }
    int* d_err = nullptr;
    H2_CUDA_TRY(cudaMallocAsync((void**)&d_err, sizeof(int), st));
    H2_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    const unsigned g = (unsigned)std::min(NL, 152 * 4);
    k_bj_invert<<<g, 256, kBjSmem, st>>>(A->d_leaves, NL, A->d_cl_size, A->d_near_diag, (const double*)A->f64.Near,
                                         A->sigma, A->bj_off, A->bj_inv, d_err);
    H2_LAUNCH_CHECK();
    int h_err = 0;
    H2_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(d_err, st);
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) {
        set_error("block-Jacobi preconditioner: a diagonal block G_(t,t) + σI is not positive definite");
        return H2_E_BREAKDOWN;
    }
    if (A->bj_count > 0) {
        k_bj_round_f32<<<(unsigned)std::min<int64_t>((A->bj_count + 255) / 256, 152 * 8), 256, 0, st>>>(
            A->bj_inv, A->bj_inv32, A->bj_count);
        H2_LAUNCH_CHECK();
    }
    A->bj_valid = true;
    A->bj_sigma = A->sigma;
    return 0;
}

int bj_apply(h2_matrix* A, const double* R, double* Z, int64_t n, int m, const double* AP, const CgDev& d,
             cudaStream_t st, bool low) {
    (void)n;
    const int NL = (int)A->leaves.size();
    const unsigned g = (unsigned)std::min(NL, kBjCtas);
    if (low)
        k_bj_apply<float><<<g, 256, kBjSmem, st>>>(R, Z, m, A->d_perm, A->d_leaves, NL, A->d_cl_off, A->d_cl_size,
                                                   A->bj_off, A->bj_inv32, AP, d);
    else
        k_bj_apply<double><<<g, 256, kBjSmem, st>>>(R, Z, m, A->d_perm, A->d_leaves, NL, A->d_cl_off, A->d_cl_size,
                                                    A->bj_off, A->bj_inv, AP, d);
    H2_LAUNCH_CHECK();
    return 0;
}

}  // namespace h2
