// Parameters of A (coupling matrices S_b, shift σ) and the gradients of a loss
// through X = A⁻¹B with respect to them.
//
// With Λ = A⁻ᵀ ∂L/∂X, ∂L/∂A = −Λ Xᵀ.  An admissible block of A is
// V_t S_b V_sᵀ (Eq. (h2_admissible), W = V), so
//   ∂L/∂S_b = V_tᵀ (−Λ Xᵀ)|_{t̂×ŝ} V_s = −(V_tᵀ Λ|_t̂)(V_sᵀ X|_ŝ)ᵀ = −λ̂_t x̂_sᵀ,
// where λ̂, x̂ are the forward transformations of Λ and X (Alg.
// "forward/backward", left part: nested bases make V_tᵀ Λ|_t̂ of every cluster
// one upward pass).  The shift enters as σI, so ∂L/∂σ = −<Λ, X>_F.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "h2_internal.cuh"

namespace h2 {

namespace {

// dS_j = −λ̂_t x̂_sᵀ for admissible blocks j = (t, s): a k×k result from two
// k×m FP64 blocks, one CTA per block, 4×4 outputs per thread.
__global__ void __launch_bounds__(256) k_grad_coupling(const int32_t* __restrict__ adm_row,
                                                       const int32_t* __restrict__ adm_col, int64_t n_adm,
                                                       const double* __restrict__ lhat,
                                                       const double* __restrict__ xhat, int k, int m,
                                                       double* __restrict__ dS) {
    __shared__ double sl[64][33], sx[64][33];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int64_t j = blockIdx.x; j < n_adm; j += gridDim.x) {
        const double* L = lhat + (int64_t)adm_row[j] * k * m;
        const double* Xh = xhat + (int64_t)adm_col[j] * k * m;
        for (int r0 = 0; r0 < k; r0 += 64)
            for (int q0 = 0; q0 < k; q0 += 64) {
                double acc[4][4] = {};
                for (int c0 = 0; c0 < m; c0 += 32) {
                    __syncthreads();
                    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
                        const int rr = e / 32, cc = e % 32;
                        const bool okc = c0 + cc < m;
                        sl[rr][cc] = (r0 + rr < k && okc) ? L[(int64_t)(r0 + rr) * m + c0 + cc] : 0.0;
                        sx[rr][cc] = (q0 + rr < k && okc) ? Xh[(int64_t)(q0 + rr) * m + c0 + cc] : 0.0;
                    }
                    __syncthreads();
                    for (int cc = 0; cc < 32; ++cc) {
                        double a[4], b[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) a[i] = sl[ty + 16 * i][cc];
#pragma unroll
                        for (int i = 0; i < 4; ++i) b[i] = sx[tx + 16 * i][cc];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int l = 0; l < 4; ++l) acc[i][l] = fma(a[i], b[l], acc[i][l]);
                    }
                }
                double* out = dS + j * k * k;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        const int nu = r0 + ty + 16 * i, mu = q0 + tx + 16 * l;
                        if (nu < k && mu < k) out[(int64_t)nu * k + mu] = -acc[i][l];
                    }
            }
    }
}

// Partial sums of Σ L∘X per CTA (fixed order), then a fixed-order final sum.
__global__ void k_dot_partial(const double* __restrict__ L, int64_t ldl, const double* __restrict__ X, int64_t ldx,
                              int64_t n, int m, double* __restrict__ part) {
    __shared__ double sm[256];
    double v = 0.0;
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m;
        const int c = (int)(e % m);
        v = fma(L[i * ldl + c], X[i * ldx + c], v);
    }
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_dot_final(const double* __restrict__ part, int count, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < count; ++i) s += part[i];
        *out = s;
    }
}

}  // namespace

}  // namespace h2

using namespace h2;

extern "C" {

int h2_coupling_get(h2_matrix* A, double* S, void* stream) {
    if (!A || (!S && A->n_adm > 0)) { set_error("null argument"); return H2_E_BADARG; }
    if (int rc = refuse_complex(A, "h2_coupling_get")) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)A->n_adm * A->k * A->k * sizeof(double);
    if (bytes) H2_CUDA_TRY(cudaMemcpyAsync(S, A->f64.S, bytes, cudaMemcpyDefault, st));
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int h2_coupling_set(h2_matrix* A, const double* S, void* stream) {
    if (!A || (!S && A->n_adm > 0)) { set_error("null argument"); return H2_E_BADARG; }
    if (int rc = refuse_complex(A, "h2_coupling_set")) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t count = A->n_adm * A->k * A->k;
    if (count == 0) return 0;
    H2_CUDA_TRY(cudaMemcpyAsync(A->f64.S, S, (size_t)count * sizeof(double), cudaMemcpyDefault, st));
    A->s_replaced = true;  // the matrix-free product (H2_F32_MF) no longer applies
    int rc = 0;
    if (A->f32.built && A->f32.S) {
        if ((rc = cast_f32((const double*)A->f64.S, (float*)A->f32.S, count, st))) return rc;
    }
    const TcData& D = A->tc;
    if (D.d_tiles && D.n_s_tiles > 0) {
        if (D.has_bf16 && (rc = launch_pack_tiles(D.d_tiles, D.n_s_tiles, (const double*)A->f64.S, D.mat, 2, st)))
            return rc;
        if (D.has_tf32 && (rc = launch_pack_tiles(D.d_tiles, D.n_s_tiles, (const double*)A->f64.S, D.mat32, 4, st)))
            return rc;
    }
    if (D.t_built) {  // the S_bᵀ tiles of the product with Aᵀ come first in its descriptor list
        if (D.matT && (rc = launch_pack_tiles(D.d_tilesT, D.n_s_tiles, (const double*)A->f64.S, D.matT, 2, st)))
            return rc;
        if (D.matT32 && (rc = launch_pack_tiles(D.d_tilesT, D.n_s_tiles, (const double*)A->f64.S, D.matT32, 4, st)))
            return rc;
    }
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int h2_shift_set(h2_matrix* A, double sigma) {
    if (!A || !std::isfinite(sigma)) { set_error("bad argument"); return H2_E_BADARG; }
    A->sigma = sigma;
    return 0;
}

int h2_adjoint_grads(h2_matrix* A, const double* L, int64_t ldl, const double* X, int64_t ldx, int64_t m,
                     double* dS, double* dsigma, void* stream) {
    if (int rc = refuse_complex(A, "h2_adjoint_grads")) return rc;
    if (!A || (m > 0 && (!L || !X)) || m < 0 || ldl < m || ldx < m) {
        set_error("bad argument");
        return H2_E_BADARG;
    }
    if (m > 0 && (!is_device_pointer(L) || !is_device_pointer(X) || (dS && !is_device_pointer(dS)))) {
        set_error("h2_adjoint_grads: L, X and dS must be device memory");
        return H2_E_BADARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int k = A->k;
    if (m == 0) {
        if (dS && A->n_adm) H2_CUDA_TRY(cudaMemsetAsync(dS, 0, (size_t)A->n_adm * k * k * sizeof(double), st));
        if (dsigma) *dsigma = 0.0;
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        return 0;
    }
    int rc = 0;
    if (dS && A->n_adm > 0) {
        const size_t bXp = (size_t)A->n * m, bC = (size_t)A->nc * k * m;
        double* buf = nullptr;
        H2_CUDA_TRY(cudaMallocAsync((void**)&buf, (bXp + 2 * bC) * sizeof(double), st));
        double* lhat = buf + bXp;
        double* xhat = lhat + bC;
        if ((rc = forward_transform_f64(A, L, ldl, m, buf, lhat, st))) return rc;
        if ((rc = forward_transform_f64(A, X, ldx, m, buf, xhat, st))) return rc;
        const unsigned g = (unsigned)std::min<int64_t>(A->n_adm, 152 * 16);
        k_grad_coupling<<<g, 256, 0, st>>>(A->d_adm_row, A->d_adm_col, A->n_adm, lhat, xhat, k, (int)m, dS);
        H2_LAUNCH_CHECK();
        cudaFreeAsync(buf, st);
    }
    if (dsigma) {
        const int blocks = 304;
        double* part = nullptr;
        H2_CUDA_TRY(cudaMallocAsync((void**)&part, (blocks + 1) * sizeof(double), st));
        k_dot_partial<<<blocks, 256, 0, st>>>(L, ldl, X, ldx, A->n, (int)m, part);
        H2_LAUNCH_CHECK();
        k_dot_final<<<1, 32, 0, st>>>(part, blocks, part + blocks);
        H2_LAUNCH_CHECK();
        double dot = 0.0;
        H2_CUDA_TRY(cudaMemcpyAsync(&dot, part + blocks, sizeof(double), cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(part, st);
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        *dsigma = -dot;
    }
    H2_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

}  // extern "C"
