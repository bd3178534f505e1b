// H² matrix × dense block, SIMT kernels for FP64 and FP32 (Sec. 3 Alg.
// "H2_mvm" with the k×m coefficient blocks of Sec. 4).
//
// The product Y += α·A·X runs as a stream-ordered chain:
//   gather      Xp = X[perm]                       (cluster order, compute type)
//   leaf_fwd    x̂_t = V_tᵀ Xp|_t̂                  (forward transformation, leaves)
//   up(l)       x̂_t = Σ_{t'∈sons(t)} E_{t'}ᵀ x̂_{t'}  levels deepest-1 .. 0
//   coupling    ŷ_t = Σ_{b=(t,s)∈L+} S_b x̂_s      (multiplication phase, admissible part;
//                                                  one owner per row cluster, Alg. "list_addeval")
//   down(l)     ŷ_{t'} += E_{t'} ŷ_t                levels 1 .. deepest
//   leaf_bwd    Y|_t̂ += α (V_t ŷ_t + Σ_{b=(t,s)∈L-} G_b Xp|_ŝ + σ Xp|_t̂)   scattered through perm
// Every output tile has exactly one owning CTA, so no atomics are needed: the
// race the paper resolves by sequential sums (Sec. 3, after Alg.
// "forward/backward") is resolved here by ownership.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "h2_async.cuh"
#include "h2_internal.cuh"

namespace h2 {

namespace {

constexpr int kThreads = 256;  // 16 × 16 thread grid per CTA
constexpr int kKC = 32;        // K chunk staged in shared memory

// Per-thread register tile: rows RM·ty + r (r < RM), columns CN·tx + c (c < CN),
// ty = thread / 16, tx = thread % 16; the RM rows and the CN columns of one
// thread are contiguous in shared memory, so one vector load fetches each.
template <typename T, int RM, int CN>
struct Acc {
    T v[RM][CN];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
            for (int c = 0; c < CN; ++c) v[r][c] = T(0);
    }
};

template <typename T, int RM, int CN>
struct Smem {
    alignas(16) T a[kKC][16 * RM + 4];  // [k][row]; +4 keeps rows 16-byte aligned
    alignas(16) T b[kKC][16 * CN];      // [k][column]
};

// Vector loads of n consecutive values from 16-byte-aligned shared memory.
template <int N>
__device__ __forceinline__ void lds_vec(const float* p, float (&v)[N]) {
    if constexpr (N == 4) {
        const float4 x = *(const float4*)p;
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if constexpr (N == 2) {
        const float2 x = *(const float2*)p;
        v[0] = x.x; v[1] = x.y;
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = p[i];
    }
}
template <int N>
__device__ __forceinline__ void lds_vec(const double* p, double (&v)[N]) {
    if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const double2 x = *(const double2*)(p + i);
            v[i] = x.x; v[i + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = p[i];
    }
}

// acc += op(A)[row0 : row0+16RM, 0:K] · B[0:K, col0 : col0+16CN]
// op(A) = A (A is M×K row-major, leading dimension lda) or, with TA, Aᵀ
// (A stored K×M row-major).  Rows >= M, k >= K and columns >= ncol read as 0.
// CGB: read B through L2 only (ld.global.cg), for data another CTA of the same
// launch wrote.  IB: B holds interleaved complex columns (real part 2j,
// imaginary part 2j+1) and i·B is staged instead: column 2j gets -B[:, 2j+1]
// and column 2j+1 gets B[:, 2j] (ncol even).
template <typename T, int RM, int CN, bool TA, bool CGB = false, bool IB = false>
__device__ __forceinline__ void mac(Acc<T, RM, CN>& acc, Smem<T, RM, CN>& sm, const T* __restrict__ A,
                                    int64_t lda, int M, int K, int row0, const T* B,
                                    int64_t ldb, int ncol, int col0) {
    constexpr int MT = 16 * RM, NT = 16 * CN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int k0 = 0; k0 < K; k0 += kKC) {
        const int kc = min(kKC, K - k0);
        __syncthreads();
        if (TA) {
            for (int e = tid; e < MT * kKC; e += kThreads) {
                const int r = e % MT, kk = e / MT;
                const int gr = row0 + r;
                sm.a[kk][r] = (gr < M && kk < kc) ? A[(int64_t)(k0 + kk) * lda + gr] : T(0);
            }
        } else {
            for (int e = tid; e < MT * kKC; e += kThreads) {
                const int kk = e % kKC, r = e / kKC;
                const int gr = row0 + r;
                sm.a[kk][r] = (gr < M && kk < kc) ? A[(int64_t)gr * lda + k0 + kk] : T(0);
            }
        }
        for (int e = tid; e < NT * kKC; e += kThreads) {
            const int c = e % NT, kk = e / NT;
            const int gc = col0 + c;
            if (IB) {
                const T v = (gc < ncol && kk < kc) ? B[(int64_t)(k0 + kk) * ldb + (gc ^ 1)] : T(0);
                sm.b[kk][c] = (gc & 1) ? v : -v;
            } else if (CGB) sm.b[kk][c] = (gc < ncol && kk < kc) ? __ldcg(B + (int64_t)(k0 + kk) * ldb + gc) : T(0);
            else sm.b[kk][c] = (gc < ncol && kk < kc) ? B[(int64_t)(k0 + kk) * ldb + gc] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kc; ++kk) {
            T a[RM], b[CN];
            lds_vec<RM>(&sm.a[kk][RM * ty], a);
            lds_vec<CN>(&sm.b[kk][CN * tx], b);
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < CN; ++c) acc.v[r][c] = fma(a[r], b[c], acc.v[r][c]);
        }
    }
}

template <typename T, int RM, int CN, bool ACCUM>
__device__ __forceinline__ void store_tile(const Acc<T, RM, CN>& acc, T* __restrict__ C, int64_t ldc, int M,
                                           int ncol, int row0, int col0) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        const int gr = row0 + RM * ty + r;
        if (gr >= M) continue;
#pragma unroll
        for (int c = 0; c < CN; ++c) {
            const int gc = col0 + CN * tx + c;
            if (gc >= ncol) continue;
            T* p = C + (int64_t)gr * ldc + gc;
            if (ACCUM) *p += acc.v[r][c]; else *p = acc.v[r][c];
        }
    }
}

// acc += E·B (TR: Eᵀ·B) for q = 4, with E = F_z ⊗ F_y ⊗ F_x (4×4 factors at f,
// F_a[μ][ν] row-major: F_x, F_y, F_z; ν = ν_x + 4ν_y + 16ν_z) and B the 64 rows ×
// columns col0.. of a block (leading dimension ldb; columns >= ncol read as 0,
// read through L2 as in mac<CGB>): three 4×4 mode products in place in the
// CTA's shared memory (the Smem struct as one flat buffer), instead of a 64×64
// product.  Thread (tx, ty) owns rows 4ty.. (an x-fiber: μ_y = ty & 3, μ_z =
// ty >> 2) and columns CN·tx.., as in mac with RM = 4.
template <typename T, int CN, bool TR>
__device__ __forceinline__ void kron_tile(Acc<T, 4, CN>& acc, Smem<T, 4, CN>& sm, const T* __restrict__ f,
                                          const T* B, int64_t ldb, int ncol, int col0) {
    constexpr int NT = 16 * CN;
    static_assert(sizeof(Smem<T, 4, CN>) >= sizeof(T) * (64 * NT + 48), "kron_tile needs 64 rows and the factors");
    T* X = reinterpret_cast<T*>(&sm);  // [64][NT]
    T* Fs = X + 64 * NT;               // [48]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    __syncthreads();  // earlier readers of the shared memory are done
    for (int e = tid; e < 64 * NT; e += kThreads) {
        const int r = e / NT, c = e % NT, gc = col0 + c;
        X[e] = gc < ncol ? __ldcg(B + (int64_t)r * ldb + gc) : T(0);
    }
    if (tid < 48) Fs[tid] = f[tid];
    __syncthreads();
    auto F = [&](int a, int mu, int nu) { return TR ? Fs[16 * a + 4 * nu + mu] : Fs[16 * a + 4 * mu + nu]; };
    const int my = ty & 3, mz = ty >> 2;
    T t[4][CN];
    // x: the thread's own fiber
#pragma unroll
    for (int j = 0; j < CN; ++j) {
        T x[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) x[v] = X[(4 * ty + v) * NT + CN * tx + j];
#pragma unroll
        for (int mx = 0; mx < 4; ++mx) {
            T a = T(0);
#pragma unroll
            for (int v = 0; v < 4; ++v) a = fma(F(0, mx, v), x[v], a);
            t[mx][j] = a;
        }
    }
    __syncthreads();
#pragma unroll
    for (int mx = 0; mx < 4; ++mx)
#pragma unroll
        for (int j = 0; j < CN; ++j) X[(4 * ty + mx) * NT + CN * tx + j] = t[mx][j];
    __syncthreads();
    // y: rows μ_x + 4ν_y + 16μ_z
#pragma unroll
    for (int mx = 0; mx < 4; ++mx)
#pragma unroll
        for (int j = 0; j < CN; ++j) {
            T a = T(0);
#pragma unroll
            for (int v = 0; v < 4; ++v) a = fma(F(1, my, v), X[(mx + 4 * v + 16 * mz) * NT + CN * tx + j], a);
            t[mx][j] = a;
        }
    __syncthreads();
#pragma unroll
    for (int mx = 0; mx < 4; ++mx)
#pragma unroll
        for (int j = 0; j < CN; ++j) X[(4 * ty + mx) * NT + CN * tx + j] = t[mx][j];
    __syncthreads();
    // z: rows μ_x + 4μ_y + 16ν_z
#pragma unroll
    for (int mx = 0; mx < 4; ++mx)
#pragma unroll
        for (int j = 0; j < CN; ++j) {
            T a = T(0);
#pragma unroll
            for (int v = 0; v < 4; ++v) a = fma(F(2, mz, v), X[(mx + 4 * my + 16 * v) * NT + CN * tx + j], a);
            acc.v[mx][j] += a;
        }
}

// Lanes per row for m columns: the power of two ≥ m, at most 32, so a warp
// covers 32 / P rows per step, each with one perm lookup and contiguous columns
// (no per-element division).
__device__ __forceinline__ int row_lanes(int m) {
    int P = 1;
    while (P < m && P < 32) P <<= 1;
    return P;
}

// ---- gather: Xp[i, :] = X[perm[i], :] in the compute type ----
template <typename T>
// With z1/z2/z3 it also zeroes the counters and flags the passes after it use,
// and with zid the k×zmc blocks of ŷ (rows of zld) of the clusters zid[0..nzc)
// (in place of separate memsets and launches on the stream).
__global__ void k_gather(const double* __restrict__ X, int64_t ldx, const int32_t* __restrict__ perm, int64_t n,
                         int m, T* __restrict__ Xp, unsigned* __restrict__ z1 = nullptr, int n1 = 0,
                         unsigned* __restrict__ z2 = nullptr, int n2 = 0, int* __restrict__ z3 = nullptr, int n3 = 0,
                         const int32_t* __restrict__ zid = nullptr, int nzc = 0, float* __restrict__ zy = nullptr,
                         int zk = 0, int zld = 0, int zmc = 0) {
    {
        const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = t; i < n1; i += nt) z1[i] = 0u;
        for (int64_t i = t; i < n2; i += nt) z2[i] = 0u;
        for (int64_t i = t; i < n3; i += nt) z3[i] = 0;
        const int64_t blk = (int64_t)zk * zmc;
        for (int64_t e = t; e < nzc * blk; e += nt) {
            const int64_t c = e / blk, r = e % blk;
            zy[((int64_t)zid[c] * zk + r / zmc) * zld + r % zmc] = 0.f;
        }
    }
    const int P = row_lanes(m), R = 32 / P;
    const int lane = threadIdx.x & 31, sub = lane / P, cl = lane % P;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * R + sub; i < n; i += nw * R) {
        const double* x = X + (int64_t)perm[i] * ldx;
        T* o = Xp + i * m;
        for (int c = cl; c < m; c += P) o[c] = (T)x[c];
    }
}

// ---- scatter of the tensor-core leaf result: Y[perm[i], :] (+)= α (Z[i, :] + σ X[perm[i], :]) ----
__global__ void k_scatter_y(const float* __restrict__ Z, int ldz, const int32_t* __restrict__ perm, int64_t n, int m,
                            const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy,
                            double alpha, double sigma, int overwrite) {
    const int P = row_lanes(m), R = 32 / P;
    const int lane = threadIdx.x & 31, sub = lane / P, cl = lane % P;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * R + sub; i < n; i += nw * R) {
        const int64_t g = perm[i];
        const float* z = Z + i * ldz;
        const double* x = X + g * ldx;
        double* y = Y + g * ldy;
        for (int c = cl; c < m; c += P) {
            const double v = alpha * ((double)z[c] + sigma * x[c]);
            if (overwrite) y[c] = v; else y[c] += v;
        }
    }
}

// ---- the same over C: interleaved (real, imaginary) columns, m2 = 2·m_c, and
// Y[perm[i], :] (+)= α (Z[i, :] + σ X[perm[i], :]) with α = alpha_re + i·alpha_im ----
__global__ void k_scatter_yc(const float* __restrict__ Z, int ldz, const int32_t* __restrict__ perm, int64_t n,
                             int m2, const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy,
                             double alpha_re, double alpha_im, double sigma, int overwrite) {
    const int mc = m2 >> 1;
    const int P = row_lanes(mc), R = 32 / P;
    const int lane = threadIdx.x & 31, sub = lane / P, cl = lane % P;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * R + sub; i < n; i += nw * R) {
        const int64_t g = perm[i];
        const float* z = Z + i * ldz;
        const double* x = X + g * ldx;
        double* y = Y + g * ldy;
        for (int c = cl; c < mc; c += P) {
            const double zr = (double)z[2 * c] + sigma * x[2 * c], zi = (double)z[2 * c + 1] + sigma * x[2 * c + 1];
            const double vr = alpha_re * zr - alpha_im * zi, vi = alpha_re * zi + alpha_im * zr;
            if (overwrite) {
                y[2 * c] = vr;
                y[2 * c + 1] = vi;
            } else {
                y[2 * c] += vr;
                y[2 * c + 1] += vi;
            }
        }
    }
}

// ---- forward transformation at the leaves: x̂_t = V_tᵀ Xp|_t̂ ----
template <typename T, int RM, int CN>
__global__ void __launch_bounds__(kThreads) k_leaf_fwd(const int32_t* __restrict__ leaves,
                                                       const int32_t* __restrict__ cl_off,
                                                       const int32_t* __restrict__ cl_size,
                                                       const T* __restrict__ V, const T* __restrict__ Xp,
                                                       T* __restrict__ xhat, int k, int m) {
    __shared__ Smem<T, RM, CN> sm;
    const int t = leaves[blockIdx.x];
    const int col0 = blockIdx.y * 16 * CN, row0 = blockIdx.z * 16 * RM;
    Acc<T, RM, CN> acc;
    acc.zero();
    const int off = cl_off[t];
    mac<T, RM, CN, true>(acc, sm, V + (int64_t)off * k, k, k, cl_size[t], row0, Xp + (int64_t)off * m, m, m,
                         col0);
    store_tile<T, RM, CN, false>(acc, xhat + (int64_t)t * k * m, m, k, m, row0, col0);
}

// ---- upward pass on one level: x̂_t = Σ_{t'} E_{t'}ᵀ x̂_{t'} ----
template <typename T, int RM, int CN>
__global__ void __launch_bounds__(kThreads) k_up(const int32_t* __restrict__ list, const int32_t* __restrict__ son0,
                                                 const int32_t* __restrict__ son1, const T* __restrict__ E,
                                                 T* __restrict__ xhat, int k, int m) {
    __shared__ Smem<T, RM, CN> sm;
    const int t = list[blockIdx.x];
    const int col0 = blockIdx.y * 16 * CN, row0 = blockIdx.z * 16 * RM;
    Acc<T, RM, CN> acc;
    acc.zero();
    const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
    const int s0 = son0[t], s1 = son1[t];
    mac<T, RM, CN, true>(acc, sm, E + s0 * kk, k, k, k, row0, xhat + s0 * km, m, m, col0);
    mac<T, RM, CN, true>(acc, sm, E + s1 * kk, k, k, k, row0, xhat + s1 * km, m, m, col0);
    store_tile<T, RM, CN, false>(acc, xhat + (int64_t)t * km, m, k, m, row0, col0);
}

// ---- forward transformation in one launch (leaves and all levels) ----
// One CTA per (leaf, column tile) computes x̂_leaf = V_tᵀ X|_t̂, then climbs:
// the second son to finish (arrival counter of the parent) computes the
// parent x̂_t = Σ_{t'} E_{t'}ᵀ x̂_{t'} and continues; the first one stops.  No
// CTA ever waits.  Counters are reset by their second arrival.
template <typename T, int RM, int CN>
__global__ void __launch_bounds__(kThreads) k_up_fused(const int32_t* __restrict__ leaves,
                                                       const int32_t* __restrict__ cl_off,
                                                       const int32_t* __restrict__ cl_size,
                                                       const int32_t* __restrict__ parent,
                                                       const int32_t* __restrict__ son0,
                                                       const int32_t* __restrict__ son1, const T* __restrict__ V,
                                                       const T* __restrict__ E, const T* __restrict__ Xp, T* xhat,
                                                       unsigned* __restrict__ cnt, int k, int m,
                                                       const T* __restrict__ kron) {
    __shared__ Smem<T, RM, CN> sm;
    __shared__ int s_go;
    const int tile = blockIdx.y, gy = gridDim.y;
    const int col0 = tile * 16 * CN;
    const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
    int c = leaves[blockIdx.x];
    Acc<T, RM, CN> acc;
    acc.zero();
    const int off = cl_off[c];
    mac<T, RM, CN, true>(acc, sm, V + (int64_t)off * k, k, k, cl_size[c], 0, Xp + (int64_t)off * m, m, m, col0);
    store_tile<T, RM, CN, false>(acc, xhat + (int64_t)c * km, m, k, m, 0, col0);
    while (true) {
        const int par = parent[c];
        if (par < 0) break;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned old = atomicAdd(&cnt[(int64_t)par * gy + tile], 1u);
            s_go = old == 1u;
            if (old == 1u) cnt[(int64_t)par * gy + tile] = 0u;
        }
        __syncthreads();
        if (!s_go) break;
        __threadfence();
        c = par;
        const int s0 = son0[c], s1 = son1[c];
        acc.zero();
        if constexpr (RM == 4) {
            if (kron) {  // q = 4: E_sᵀ as Kronecker products
                kron_tile<T, CN, true>(acc, sm, kron + (int64_t)s0 * 48, xhat + s0 * km, m, m, col0);
                kron_tile<T, CN, true>(acc, sm, kron + (int64_t)s1 * 48, xhat + s1 * km, m, m, col0);
                store_tile<T, RM, CN, false>(acc, xhat + (int64_t)c * km, m, k, m, 0, col0);
                continue;
            }
        }
        mac<T, RM, CN, true, true>(acc, sm, E + s0 * kk, k, k, k, 0, xhat + s0 * km, m, m, col0);
        mac<T, RM, CN, true, true>(acc, sm, E + s1 * kk, k, k, k, 0, xhat + s1 * km, m, m, col0);
        store_tile<T, RM, CN, false>(acc, xhat + (int64_t)c * km, m, k, m, 0, col0);
    }
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- backward transfer pass in one launch ----
// Items are the non-root clusters in top-down level order.  A CTA claims the
// next item (atomic ticket), waits until its parent's ŷ is final (the parent
// has a smaller ticket, so a running CTA holds it; the wait is bounded and
// reports a timeout through err), adds E_{t'} ŷ_parent and publishes its own
// ready flag (set to `epoch`; the flags are cleared before each launch).
template <typename T, int RM, int CN>
__global__ void __launch_bounds__(kThreads) k_down_fused(const int32_t* __restrict__ order, int n_items,
                                                         const int32_t* __restrict__ parent, const T* __restrict__ E,
                                                         T* yhat, unsigned* __restrict__ claim, int* flag, int epoch,
                                                         int* __restrict__ err, int k, int m, long long spin_limit,
                                                         const T* __restrict__ kron) {
    __shared__ Smem<T, RM, CN> sm;
    __shared__ int s_item, s_ok;
    const int tile = blockIdx.y, gy = gridDim.y;
    const int col0 = tile * 16 * CN;
    const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&claim[tile], 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int c = order[item];
        const int par = parent[c];
        if (threadIdx.x == 0) {
            int ok = 1;
            if (parent[par] >= 0) {  // the root's ŷ is final after the coupling phase
                const int* f = flag + (int64_t)par * gy + tile;
                // spin_limit < 0: give up without looking at the flag (the timeout
                // path's test setting, h2_set_wait_limit)
                long long spins = 0;
                while (spin_limit < 0 || ld_acquire(f) != epoch) {
                    if (spin_limit < 0 || ++spins > spin_limit) { ok = 0; break; }
                    __nanosleep(32);
                }
            }
            s_ok = ok;
            if (!ok) atomicExch(err, 8);
        }
        __syncthreads();
        if (!s_ok) break;
        Acc<T, RM, CN> acc;
        acc.zero();
        bool done = false;
        if constexpr (RM == 4) {
            if (kron) {  // q = 4: E_c as a Kronecker product
                kron_tile<T, CN, false>(acc, sm, kron + (int64_t)c * 48, yhat + (int64_t)par * km, m, m, col0);
                done = true;
            }
        }
        if (!done)
            mac<T, RM, CN, false, true>(acc, sm, E + (int64_t)c * kk, k, k, k, 0, yhat + (int64_t)par * km, m, m, col0);
        store_tile<T, RM, CN, true>(acc, yhat + (int64_t)c * km, m, k, m, 0, col0);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(flag + (int64_t)c * gy + tile, epoch);
    }
}

// ---- multiplication phase, admissible part: ŷ_t = Σ_{b∈C_t} S_b x̂_s ----
// TRANS: the list is by column cluster and S_bᵀ is applied (product with Aᵀ).
template <typename T, int RM, int CN, bool TRANS>
__global__ void __launch_bounds__(kThreads) k_coupling(const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ other,
                                                       const int32_t* __restrict__ blk, const T* __restrict__ S,
                                                       const T* __restrict__ xhat, T* __restrict__ yhat, int k,
                                                       int m) {
    __shared__ Smem<T, RM, CN> sm;
    const int t = blockIdx.x;
    const int col0 = blockIdx.y * 16 * CN, row0 = blockIdx.z * 16 * RM;
    Acc<T, RM, CN> acc;
    acc.zero();
    const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
    for (int e = rowptr[t]; e < rowptr[t + 1]; ++e) {
        const int s = other[e];
        const int64_t j = TRANS ? blk[e] : e;
        mac<T, RM, CN, TRANS>(acc, sm, S + j * kk, k, k, k, row0, xhat + s * km, m, m, col0);
    }
    store_tile<T, RM, CN, false>(acc, yhat + (int64_t)t * km, m, k, m, row0, col0);
}

// ---- downward pass on one level: ŷ_{t'} += E_{t'} ŷ_{parent(t')} ----
template <typename T, int RM, int CN>
__global__ void __launch_bounds__(kThreads) k_down(const int32_t* __restrict__ list,
                                                   const int32_t* __restrict__ parent, const T* __restrict__ E,
                                                   T* __restrict__ yhat, int k, int m) {
    __shared__ Smem<T, RM, CN> sm;
    const int c = list[blockIdx.x];
    const int col0 = blockIdx.y * 16 * CN, row0 = blockIdx.z * 16 * RM;
    Acc<T, RM, CN> acc;
    acc.zero();
    const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
    mac<T, RM, CN, false>(acc, sm, E + c * kk, k, k, k, row0, yhat + (int64_t)parent[c] * km, m, m, col0);
    store_tile<T, RM, CN, true>(acc, yhat + (int64_t)c * km, m, k, m, row0, col0);
}

// ---- backward transformation at the leaves + inadmissible part + shift ----
// Y[perm[off_t + i], :] += α (V_t ŷ_t + Σ_b G_b Xp|_ŝ + σ Xp|_t̂)[i, :]
template <typename T, int RM, int CN, bool TRANS>
__global__ void __launch_bounds__(kThreads) k_leaf_bwd_near(
    const int32_t* __restrict__ leaves, const int32_t* __restrict__ cl_off, const int32_t* __restrict__ cl_size,
    const int32_t* __restrict__ perm, const T* __restrict__ V, const T* __restrict__ yhat,
    const int32_t* __restrict__ nptr, const int32_t* __restrict__ nother, const int32_t* __restrict__ nblk,
    const int64_t* __restrict__ near_off, const T* __restrict__ G, const T* __restrict__ Xp, double* __restrict__ Y,
    int64_t ldy, double alpha, double sigma, int k, int m, int overwrite) {
    __shared__ Smem<T, RM, CN> sm;
    const int lp = blockIdx.x;
    const int t = leaves[lp];
    const int col0 = blockIdx.y * 16 * CN, row0 = blockIdx.z * 16 * RM;
    const int off = cl_off[t], nt = cl_size[t];
    Acc<T, RM, CN> acc;
    acc.zero();
    mac<T, RM, CN, false>(acc, sm, V + (int64_t)off * k, k, nt, k, row0, yhat + (int64_t)t * k * m, m, m, col0);
    for (int e = nptr[lp]; e < nptr[lp + 1]; ++e) {
        const int s = nother[e];
        const int64_t j = TRANS ? nblk[e] : e;
        const int os = cl_off[s], ns = cl_size[s];
        // G_j is |row leaf| × |column leaf| row-major; for Aᵀ the row leaf is s.
        mac<T, RM, CN, TRANS>(acc, sm, G + near_off[j], TRANS ? nt : ns, nt, ns, row0, Xp + (int64_t)os * m, m, m,
                              col0);
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        const int i = row0 + RM * ty + r;
        if (i >= nt) continue;
        double* yrow = Y + (int64_t)perm[off + i] * ldy;
        const T* xrow = Xp + (int64_t)(off + i) * m;
#pragma unroll
        for (int c = 0; c < CN; ++c) {
            const int gc = col0 + CN * tx + c;
            if (gc >= m) continue;
            const double z = (double)acc.v[r][c] + sigma * (double)xrow[gc];
            if (overwrite) yrow[gc] = alpha * z; else yrow[gc] += alpha * z;
        }
    }
}

// ---- the complex product (K = C, Sec. 2): real bases, complex S_b and G_b ----
// Coefficient blocks and X are interleaved complex columns (2m real columns), so
// the transfer passes are the real kernels above; only the phases that apply
// S_b and G_b differ.  With S = S_re + i·S_im (two planes im_off elements apart),
// S·x̂ = S_re·x̂ + S_im·(i·x̂), two real products into one accumulator.
template <typename T, int RM, int CN>
__global__ void __launch_bounds__(kThreads) k_coupling_c(const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ other,
                                                         const T* __restrict__ S, int64_t im_off,
                                                         const T* __restrict__ xhat, T* __restrict__ yhat, int k,
                                                         int m2) {
    __shared__ Smem<T, RM, CN> sm;
    const int t = blockIdx.x;
    const int col0 = blockIdx.y * 16 * CN, row0 = blockIdx.z * 16 * RM;
    Acc<T, RM, CN> acc;
    acc.zero();
    const int64_t kk = (int64_t)k * k, km = (int64_t)k * m2;
    for (int e = rowptr[t]; e < rowptr[t + 1]; ++e) {
        const T* xs = xhat + (int64_t)other[e] * km;
        mac<T, RM, CN, false>(acc, sm, S + e * kk, k, k, k, row0, xs, m2, m2, col0);
        mac<T, RM, CN, false, false, true>(acc, sm, S + im_off + e * kk, k, k, k, row0, xs, m2, m2, col0);
    }
    store_tile<T, RM, CN, false>(acc, yhat + (int64_t)t * km, m2, k, m2, row0, col0);
}

// Y[perm[off_t + i], :] (+)= α (V_t ŷ_t + Σ_b G_b Xp|_ŝ + σ Xp|_t̂)[i, :] over C:
// G_b = G_re + i·G_im (planes im_off elements apart), α = alpha_re + i·alpha_im.
// CN is even, so a thread holds both parts of each complex column.
template <typename T, int RM, int CN>
__global__ void __launch_bounds__(kThreads) k_leaf_bwd_near_c(
    const int32_t* __restrict__ leaves, const int32_t* __restrict__ cl_off, const int32_t* __restrict__ cl_size,
    const int32_t* __restrict__ perm, const T* __restrict__ V, const T* __restrict__ yhat,
    const int32_t* __restrict__ nptr, const int32_t* __restrict__ nother, const int64_t* __restrict__ near_off,
    const T* __restrict__ G, int64_t im_off, const T* __restrict__ Xp, double* __restrict__ Y, int64_t ldy,
    double alpha_re, double alpha_im, double sigma, int k, int m2, int overwrite) {
    static_assert(CN % 2 == 0, "complex columns are pairs within a thread");
    __shared__ Smem<T, RM, CN> sm;
    const int lp = blockIdx.x;
    const int t = leaves[lp];
    const int col0 = blockIdx.y * 16 * CN, row0 = blockIdx.z * 16 * RM;
    const int off = cl_off[t], nt = cl_size[t];
    Acc<T, RM, CN> acc;
    acc.zero();
    mac<T, RM, CN, false>(acc, sm, V + (int64_t)off * k, k, nt, k, row0, yhat + (int64_t)t * k * m2, m2, m2, col0);
    for (int e = nptr[lp]; e < nptr[lp + 1]; ++e) {
        const int s = nother[e];
        const int os = cl_off[s], ns = cl_size[s];
        const T* xs = Xp + (int64_t)os * m2;
        mac<T, RM, CN, false>(acc, sm, G + near_off[e], ns, nt, ns, row0, xs, m2, m2, col0);
        mac<T, RM, CN, false, false, true>(acc, sm, G + im_off + near_off[e], ns, nt, ns, row0, xs, m2, m2, col0);
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        const int i = row0 + RM * ty + r;
        if (i >= nt) continue;
        double* yrow = Y + (int64_t)perm[off + i] * ldy;
        const T* xrow = Xp + (int64_t)(off + i) * m2;
#pragma unroll
        for (int c = 0; c < CN; c += 2) {
            const int gc = col0 + CN * tx + c;  // even: the real part of a complex column
            if (gc >= m2) continue;
            const double zr = (double)acc.v[r][c] + sigma * (double)xrow[gc];
            const double zi = (double)acc.v[r][c + 1] + sigma * (double)xrow[gc + 1];
            const double vr = alpha_re * zr - alpha_im * zi, vi = alpha_re * zi + alpha_im * zr;
            if (overwrite) {
                yrow[gc] = vr;
                yrow[gc + 1] = vi;
            } else {
                yrow[gc] += vr;
                yrow[gc + 1] += vi;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 transfer passes for k % 4 == 0, k <= 64, m % 4 == 0, leaves of at most
// 64 points.  The tree is cut at one level; each task (a cut cluster) is owned
// by one CTA, which evaluates its subtree with every intermediate x̂ or ŷ kept
// in shared memory.  Static operands (V_t, X|_t̂, the transfer matrices, the
// coupling results) arrive by bulk copies one step ahead.  Only the clusters
// above the cut in the upward pass are shared between CTAs (last arriver of
// two brothers computes the father).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16_cg(void* s, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit_wait() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// acc[4][4] += a[0:K][rows 4ty..4ty+3] contracted with b[0:K][cols 4tx..4tx+3],
// row strides lda and ldb floats (multiples of 4).  The operand rows of eight
// contraction steps are loaded before their 128 FMAs, walking two pointers
// (a 64×64×32 contraction on four warps: about 2450 cycles, against about 3900
// for a per-step indexed loop with runtime strides).  Rows and columns past the
// valid ones read neighbouring data and give outputs nobody stores.
__device__ __forceinline__ void contract44(float (&acc)[4][4], const float* a, int lda, const float* b, int ldb, int K,
                                           int tx, int ty) {
    const float* pa = a + 4 * ty;
    const float* pb = b + 4 * tx;
    auto step = [&](const float4 x, const float4 y) {
        const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(xv[r], yv[c], acc[r][c]);
    };
    int kk = 0;
    for (; kk + 8 <= K; kk += 8) {
        float4 x[8], y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            x[u] = *(const float4*)(pa + u * lda);
            y[u] = *(const float4*)(pb + u * ldb);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) step(x[u], y[u]);
        pa += 8 * lda;
        pb += 8 * ldb;
    }
    for (; kk < K; ++kk) {
        step(*(const float4*)pa, *(const float4*)pb);
        pa += lda;
        pb += ldb;
    }
}

// Split activation tiles written by the transfer passes for the tensor-core
// phases (the layout k_pack_act writes): act holds one R×KP tile per cluster
// (x̂ in the upward pass, leaf ŷ in the downward pass), leafX one R×kp tile per
// leaf (kp = xkoff[l+1] - xkoff[l]) of the leaf's X rows.
struct PackOut {
    uint8_t* act;
    uint8_t* leafX;
    const int64_t* xkoff;
    int KP, R, es;
};

// The thread's 4×4 block of a k×m result (rows 4ty.., columns 4tx..) into a
// cluster's tile, zeros in the padding rows (columns i >= m) and columns
// (κ >= k).
__device__ __forceinline__ void pack_rows(const PackOut& pk, uint8_t* tile, const float (&acc)[4][4], int tx, int ty,
                                          int k, int m) {
    if (4 * ty >= pk.KP) return;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int i = 4 * tx + c;
        if (2 * i >= pk.R) continue;
        float v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = (i < m && 4 * ty + r < k) ? acc[r][c] : 0.f;
        put_act4(tile, pk.KP, pk.es, i, 4 * ty, v);
    }
}

// A leaf's X rows (nt points × m columns in shared memory, row stride m) into
// its tile of kp contraction columns (the points), zero padded.
__device__ __forceinline__ void pack_points(const PackOut& pk, uint8_t* tile, int kp, const float* x, int nt, int m) {
    const int half = pk.R >> 1;
    for (int it = threadIdx.x; it < (kp >> 2) * half; it += blockDim.x) {
        const int q0 = 4 * (it / half), i = it % half;
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (i < m && q0 + u < nt) ? x[(q0 + u) * m + i] : 0.f;
        put_act4(tile, kp, pk.es, i, q0, v);
    }
}

// acc (rows 4ty.., columns 4tx.. of a 64-row block) += E_cᵀ x for q = 4, E_c =
// F_z ⊗ F_y ⊗ F_x with the factors at f (global memory, F_a[μ][ν] row-major) and x
// in shared memory (row stride ldx): the x mode product in the thread (its rows
// are one x-fiber), the y and z mode products through `scratch` (64 rows of ld
// floats, ld >= 4·(tx + 1), of shared memory free for the call).  Columns past
// the block's read neighbouring data and give outputs nobody stores.  Every
// thread of the CTA calls it.
__device__ __forceinline__ void kron_own_t(float (&acc)[4][4], const float* x, int ldx, float* scratch, int ld,
                                           const float* __restrict__ f, int tx, int ty) {
    float F[48];
#pragma unroll
    for (int i = 0; i < 48; ++i) F[i] = __ldg(f + i);
    // transposed factors: Fᵀ_a[μ][ν] = F_a[ν][μ]
    auto Ft = [&](int a, int mu, int nu) { return F[16 * a + 4 * nu + mu]; };
    const int my = ty & 3, mz = ty >> 2;
    float t[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = x[(4 * ty + r) * ldx + 4 * tx + j];
#pragma unroll
        for (int mx = 0; mx < 4; ++mx) {
            float a = 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) a = fmaf(Ft(0, mx, r), v[r], a);
            t[mx][j] = a;
        }
    }
    __syncthreads();  // earlier users of the scratch are done
#pragma unroll
    for (int mx = 0; mx < 4; ++mx)
        *(float4*)(scratch + (4 * ty + mx) * ld + 4 * tx) = make_float4(t[mx][0], t[mx][1], t[mx][2], t[mx][3]);
    __syncthreads();
#pragma unroll
    for (int mx = 0; mx < 4; ++mx) {
        float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 w = *(const float4*)(scratch + (mx + 4 * v + 16 * mz) * ld + 4 * tx);
            const float c = Ft(1, my, v);
            a[0] = fmaf(c, w.x, a[0]); a[1] = fmaf(c, w.y, a[1]); a[2] = fmaf(c, w.z, a[2]); a[3] = fmaf(c, w.w, a[3]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) t[mx][j] = a[j];
    }
    __syncthreads();
#pragma unroll
    for (int mx = 0; mx < 4; ++mx)
        *(float4*)(scratch + (4 * ty + mx) * ld + 4 * tx) = make_float4(t[mx][0], t[mx][1], t[mx][2], t[mx][3]);
    __syncthreads();
#pragma unroll
    for (int mx = 0; mx < 4; ++mx)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 w = *(const float4*)(scratch + (mx + 4 * my + 16 * v) * ld + 4 * tx);
            const float c = Ft(2, mz, v);
            acc[mx][0] = fmaf(c, w.x, acc[mx][0]);
            acc[mx][1] = fmaf(c, w.y, acc[mx][1]);
            acc[mx][2] = fmaf(c, w.z, acc[mx][2]);
            acc[mx][3] = fmaf(c, w.w, acc[mx][3]);
        }
}

// Upward pass with subtree ownership (schedule: up_schedule, h2_build.cu), the
// forward transformation of Alg. "fast_addeval" (Sec. 3): x̂_t = V_tᵀ X|_t̂ at
// the leaves and x̂_t = E_s0ᵀ x̂_s0 + E_s1ᵀ x̂_s1 above.  A CTA claims a task and
// evaluates its subtree in post-order; the static operands of step s + 1 (V_c
// and X|_ĉ, or E_s0 and E_s1) arrive by bulk copies while step s computes, the
// sons' x̂ come from the shared-memory stack.  Above the cut the last of two
// brothers to finish computes their father (an atomic counter per cluster,
// reset by the last arriver), adding the two brothers' contributions E_sᵀ x̂_s,
// which each brother computes and publishes before the atomic.  One IEEE
// addition of two contributions does not depend on their order, so the result
// does not depend on which brother arrives last.  With climb = 0 a CTA stops
// at its task's root: the clusters above the cut are then items of the
// coupling launch (k_tc_gemm<4, 1>).  64·CN threads, thread (tx, ty) owns rows
// 4ty.. and columns 4tx.. of the k×m result.
template <int CN>
__global__ void __launch_bounds__(64 * CN) k_up_own(const int32_t* __restrict__ task_ptr, int ntasks,
                                                    const UpStep* __restrict__ steps,
                                                    const int32_t* __restrict__ cl_off,
                                                    const int32_t* __restrict__ cl_size,
                                                    const int32_t* __restrict__ parent,
                                                    const int32_t* __restrict__ son0,
                                                    const int32_t* __restrict__ son1, const float* __restrict__ V,
                                                    const float* __restrict__ E, const float* __restrict__ Xp,
                                                    float* xhat, float* part, unsigned* __restrict__ cnt,
                                                    unsigned* __restrict__ claim, int* __restrict__ err, int nent, int k,
                                                    int m, PackOut pk, int climb, const float* __restrict__ kron) {
    constexpr int NT = 16 * CN;
    extern __shared__ __align__(16) float fsm[];
    float* sbuf = fsm;                 // [2 slots][2][64·64]  V_c and X|_ĉ, or E_s0 and E_s1
    float* stk = sbuf + 4 * 64 * 64;   // [entries][64·NT]     x̂ waiting for the father
    __shared__ int s_task, s_go;
    __shared__ UpStep s_steps[kUpMaxSteps];
    __shared__ int s_off[kUpMaxSteps], s_nt[kUpMaxSteps];
    __shared__ __align__(8) uint64_t bar[2];
    const int tx = threadIdx.x % (4 * CN), ty = threadIdx.x / (4 * CN);
    const bool colv = 4 * tx < m;
    const int64_t kk = (int64_t)k * k, km = (int64_t)k * m;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;
    bool failed = false;
    auto slot = [&](int b, int h) { return sbuf + (2 * b + h) * 64 * 64; };
    auto ent = [&](int e) { return stk + e * 64 * NT; };
    // acc → stack entry e, x̂_c in global memory and its split tile for the coupling phase
    // (the tensor-core phases read only the split tiles, so x̂ is not stored in FP32)
    auto put = [&](const float (&acc)[4][4], int e, int c) {
        pack_rows(pk, pk.act + (int64_t)c * pk.KP * pk.R * pk.es, acc, tx, ty, k, m);
        if (!colv) return;
        float* out = ent(e);
#pragma unroll
        for (int r = 0; r < 4; ++r)
            *(float4*)(out + (4 * ty + r) * m + 4 * tx) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    };
    auto wait_slot = [&](int b) {
        const bool ok = mbar_wait(&bar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        return ok;
    };
    while (!failed) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = (int)atomicAdd(claim, 1u);
        __syncthreads();
        const int task = s_task;
        if (task >= ntasks) break;
        const int s0 = task_ptr[task], s1 = min(task_ptr[task + 1], s0 + kUpMaxSteps);
        for (int i = threadIdx.x; i < s1 - s0; i += blockDim.x) {
            const UpStep u = steps[s0 + i];
            s_steps[i] = u;
            s_off[i] = cl_off[u.c];
            s_nt[i] = cl_size[u.c];
        }
        __syncthreads();
        auto issue = [&](int s, int b) {
            if (threadIdx.x != 0) return;
            const UpStep u = s_steps[s - s0];
            if (u.rd0 < 0) {
                const int off = s_off[s - s0], nt = s_nt[s - s0];
                const uint32_t vb = (uint32_t)nt * k * 4, xb = (uint32_t)nt * m * 4;
                mbar_expect_tx(&bar[b], vb + xb);
                bulk_g2s(slot(b, 0), V + (int64_t)off * k, vb, &bar[b]);
                bulk_g2s(slot(b, 1), Xp + (int64_t)off * m, xb, &bar[b]);
            } else if (kron) {
                mbar_arrive(&bar[b]);  // Kronecker factors: nothing to copy, the phase completes now
            } else {
                mbar_expect_tx(&bar[b], (uint32_t)(2 * kk * 4));
                bulk_g2s(slot(b, 0), E + (int64_t)son0[u.c] * kk, (uint32_t)(kk * 4), &bar[b]);
                bulk_g2s(slot(b, 1), E + (int64_t)son1[u.c] * kk, (uint32_t)(kk * 4), &bar[b]);
            }
        };
        issue(s0, 0);
        int cur = -1;
        for (int s = s0; s < s1; ++s) {
            const int b = (s - s0) & 1;
            if (s + 1 < s1) issue(s + 1, b ^ 1);
            const bool ok = wait_slot(b);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicExch(err, 10);
                    mbar_wait(&bar[b], ((phase >> b) & 1u) ^ 1u);
                    if (s + 1 < s1) mbar_wait(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u);
                }
                failed = true;
                break;
            }
            const UpStep u = s_steps[s - s0];
            float acc[4][4] = {};
            if (u.rd0 < 0) {
                const int nt = s_nt[s - s0];
                contract44(acc, slot(b, 0), k, slot(b, 1), m, nt, tx, ty);
                // X|_ĉ (in shared memory) as the leaf's split tile for the nearfield phase
                const int64_t x0 = pk.xkoff[u.rd1];
                pack_points(pk, pk.leafX + x0 * pk.R * pk.es, (int)(pk.xkoff[u.rd1 + 1] - x0), slot(b, 1), nt, m);
            } else if (kron) {
                // q = 4: E_sᵀ as Kronecker products, slot b (no E copied) as scratch
                kron_own_t(acc, ent(u.rd0), m, slot(b, 0), NT, kron + (int64_t)son0[u.c] * 48, tx, ty);
                kron_own_t(acc, ent(u.rd1), m, slot(b, 0), NT, kron + (int64_t)son1[u.c] * 48, tx, ty);
                __syncthreads();  // x̂ of the father goes into its first son's entry
            } else {
                contract44(acc, slot(b, 0), k, ent(u.rd0), m, k, tx, ty);
                contract44(acc, slot(b, 1), k, ent(u.rd1), m, k, tx, ty);
                __syncthreads();  // x̂ of the father goes into its first son's entry
            }
            put(acc, u.wr, u.c);
            cur = u.wr;
            __syncthreads();
        }
        if (failed || cur < 0) break;
        if (!climb) continue;
        // ---- climb above the cut ----
        // Every CTA publishes its cluster's contribution P_c = E_cᵀ x̂_c to the father
        // (in `part`, the ŷ buffer, unused until the coupling phase) before the
        // atomic, so the last of two brothers only adds P_s0 + P_s1: one
        // contraction per level on the critical path.
        int c = s_steps[s1 - 1 - s0].c;
        // E_c of the next contribution is copied one level ahead (slot 0 is free
        // after the task's last step)
        auto fetch_e = [&](int cl) {
            if (threadIdx.x == 0) {
                if (kron) {
                    mbar_arrive(&bar[0]);  // nothing to copy
                } else {
                    mbar_expect_tx(&bar[0], (uint32_t)(kk * 4));
                    bulk_g2s(slot(0, 0), E + (int64_t)cl * kk, (uint32_t)(kk * 4), &bar[0]);
                }
            }
        };
        if (parent[c] >= 0) fetch_e(c);
        while (true) {
            const int par = parent[c];
            if (par < 0) break;
            const bool ok = wait_slot(0);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicExch(err, 10);
                failed = true;
                break;
            }
            float pc[4][4] = {};
            if (kron) kron_own_t(pc, ent(cur), m, slot(0, 1), NT, kron + (int64_t)c * 48, tx, ty);
            else contract44(pc, slot(0, 0), k, ent(cur), m, k, tx, ty);
            if (colv) {
                float* g = part + (int64_t)c * km;
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (4 * ty + r < k) *(float4*)(g + (4 * ty + r) * m + 4 * tx) = make_float4(pc[r][0], pc[r][1], pc[r][2], pc[r][3]);
            }
            __syncthreads();  // every store of P_c is done
            if (threadIdx.x == 0) {
                __threadfence();
                const unsigned old = atomicAdd(&cnt[par], 1u);
                s_go = old == 1u;
                if (old == 1u) {
                    cnt[par] = 0u;
                    __threadfence();
                }
            }
            __syncthreads();
            if (!s_go) break;
            if (parent[par] >= 0) fetch_e(par);  // every thread has finished reading slot 0
            // the brother's contribution (written by another CTA) through the generic proxy
            const int bro = son0[par] == c ? son1[par] : son0[par];
            const int eb = (cur + 1) % 3, er = (cur + 2) % 3;
            const float* gsrc = part + (int64_t)bro * km;
            for (int e = threadIdx.x; e < (int)(km / 4); e += blockDim.x) cp16_cg(ent(eb) + 4 * e, gsrc + 4 * e);
            cp_commit_wait();
            __syncthreads();
            const float* pb = ent(eb);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 v = *(const float4*)(pb + (4 * ty + r) * m + 4 * tx);
                pc[r][0] += v.x;
                pc[r][1] += v.y;
                pc[r][2] += v.z;
                pc[r][3] += v.w;
            }
            put(pc, er, par);
            cur = er;
            c = par;
        }
    }
}

// ---- 3xTF32 warp MMAs (mma.sync m16n8k8) for the transfer passes ----
// A 16×8 TF32 A fragment and 8×8 B fragment per thread (g = lane / 4,
// t = lane % 4): a0 = A[g][t], a1 = A[g+8][t], a2 = A[g][t+4], a3 = A[g+8][t+4];
// b0 = B[t][g], b1 = B[t+4][g]; D: d0 = D[g][2t], d1 = D[g][2t+1], d2 = D[g+8][2t],
// d3 = D[g+8][2t+1].  An FP32 operand x is split into hi = tf32(x) (rounded)
// and lo = x - hi; D += A_lo·B_hi + A_hi·B_lo + A_hi·B_hi keeps FP32 accuracy.
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = h;
    lo = __float_as_uint(x - __uint_as_float(h));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// d[nt] (N-tile nt: columns 8nt..8nt+7) += A·B over K = kdim (a multiple of 8)
// for the warp's 16 rows m0..m0+15, with A[i][j] = a[j·lda + i] (a transposed
// K-major block) and B[j][n] = b[j·ldb + n]; lda, ldb ≡ 8 (mod 32) keep the
// fragment loads free of bank conflicts.
template <int NTILES>
__device__ __forceinline__ void mma_contract(float (&d)[NTILES][4], const float* a, int lda, const float* b, int ldb,
                                             int kdim, int m0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < kdim; k0 += 8) {
        const float* ar = a + (k0 + t) * lda + m0 + g;
        uint32_t ah[4], al[4];
        tf32_split(ar[0], ah[0], al[0]);
        tf32_split(ar[8], ah[1], al[1]);
        tf32_split(ar[4 * lda], ah[2], al[2]);
        tf32_split(ar[4 * lda + 8], ah[3], al[3]);
        const float* br = b + (k0 + t) * ldb + g;
#pragma unroll
        for (int nt = 0; nt < NTILES; ++nt) {
            uint32_t bh0, bl0, bh1, bl1;
            tf32_split(br[8 * nt], bh0, bl0);
            tf32_split(br[4 * ldb + 8 * nt], bh1, bl1);
            mma_tf32(d[nt], al, bh0, bh1);
            mma_tf32(d[nt], ah, bl0, bl1);
            mma_tf32(d[nt], ah, bh0, bh1);
        }
    }
}

// Downward pass with subtree ownership (schedule: down_schedule, h2_build.cu).
// A CTA claims tasks in the stored order; a task is a list of steps, each
// ŷ_c += E_c ŷ_father (Sec. 3, the downward transformation of
// Alg. "fast_addeval"), with ŷ_father in a shared-memory stack entry written by
// an earlier step of the same task, so no step waits for another CTA.
// Four warps, warp w computing rows 16w..16w+15 of the k×m result with 3xTF32
// warp MMAs (mma_contract).  Eᵀ_c of step s + 1 (stored with rows of kEtLd
// floats) arrives by one bulk copy while step s computes; the coupling result
// ŷ_c of step s + 1 is loaded into the fragment registers meanwhile.  Stack
// rows have stride NT + 8; the root's ŷ of a task's first step is copied into
// its entry row by row (warp 0's lanes).
template <int CN>
__global__ void __launch_bounds__(128) k_down_own(const int32_t* __restrict__ task_ptr, int ntasks,
                                                  const DownStep* __restrict__ steps,
                                                  const float* __restrict__ Et, float* yhat,
                                                  unsigned* __restrict__ claim, int* __restrict__ err, int k, int m,
                                                  PackOut pk) {
    constexpr int NT = 16 * CN, NTILES = 2 * CN, LDA = kEtLd, LDY = NT + 8;
    extern __shared__ __align__(16) float fsm[];
    float* ebuf = fsm;                 // [2][64 rows j][LDA]   Eᵀ_c
    float* stk = ebuf + 2 * 64 * LDA;  // [entries][64][LDY]    final ŷ along the current path
    __shared__ int s_task;
    __shared__ DownStep s_steps[kDownMaxSteps];  // the task's steps: no global load between two steps
    __shared__ __align__(8) uint64_t bar[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = 16 * warp;
    const int64_t ke = (int64_t)k * LDA, km = (int64_t)k * m;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;  // bit b: parity of the next completion of bar[b]
    bool failed = false;
    // the thread's fragment positions of a k×m block: rows m0+g, m0+g+8; columns 8nt+2t, +1
    auto load_frag = [&](float (&v)[NTILES][4], const float* src) {
#pragma unroll
        for (int nt = 0; nt < NTILES; ++nt) {
            const int c = 8 * nt + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + g + 8 * h;
                float2 x = make_float2(0.f, 0.f);
                if (r < k && c < m) x = __ldcg((const float2*)(src + (int64_t)r * m + c));
                v[nt][2 * h] = x.x;
                v[nt][2 * h + 1] = x.y;
            }
        }
    };
    while (!failed) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = (int)atomicAdd(claim, 1u);
        __syncthreads();
        const int task = s_task;
        if (task >= ntasks) break;
        const int s0 = task_ptr[task], s1 = min(task_ptr[task + 1], s0 + kDownMaxSteps);
        for (int i = threadIdx.x; i < s1 - s0; i += blockDim.x) s_steps[i] = steps[s0 + i];
        __syncthreads();
        // warp 0 arms the buffer's barrier and starts the step's copies: one of
        // Eᵀ_c, or the root's rows into the stack entry (lane l: rows l, l + 32)
        auto issue = [&](int s, int b) {
            if (warp != 0) return;
            const DownStep d = s_steps[s - s0];
            if (d.flags & kDownLoad) {
                const uint32_t rowb = (uint32_t)m * 4;
                if (lane == 0) mbar_expect_tx(&bar[b], rowb * (uint32_t)k);
                __syncwarp();
                for (int r = lane; r < k; r += 32)
                    bulk_g2s(stk + (d.wr * 64 + r) * LDY, yhat + (int64_t)d.c * km + (int64_t)r * m, rowb, &bar[b]);
            } else if (lane == 0) {
                mbar_expect_tx(&bar[b], (uint32_t)(ke * 4));
                bulk_g2s(ebuf + b * 64 * LDA, Et + (int64_t)d.c * ke, (uint32_t)(ke * 4), &bar[b]);
            }
        };
        float ccur[NTILES][4], cnext[NTILES][4];
        issue(s0, 0);
        for (int s = s0; s < s1; ++s) {
            const int b = (s - s0) & 1;
            if (s + 1 < s1) {
                issue(s + 1, b ^ 1);
                const DownStep dn = s_steps[s + 1 - s0];
                if (!(dn.flags & kDownLoad)) load_frag(cnext, yhat + (int64_t)dn.c * km);
            }
            const bool ok = mbar_wait(&bar[b], (phase >> b) & 1u);
            phase ^= 1u << b;
            if (__syncthreads_or(!ok)) {
                // a copy did not land in time: report, let the copies in flight
                // finish (bounded), stop
                if (threadIdx.x == 0) {
                    atomicExch(err, 9);
                    mbar_wait(&bar[b], ((phase >> b) & 1u) ^ 1u);
                    if (s + 1 < s1) mbar_wait(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u);
                }
                failed = true;
                break;
            }
            const DownStep d = s_steps[s - s0];
            if (!(d.flags & kDownLoad)) {
                mma_contract<NTILES>(ccur, ebuf + b * 64 * LDA, LDA, stk + d.rd * 64 * LDY, LDY, k, m0);
                float* out = stk + d.wr * 64 * LDY;
#pragma unroll
                for (int nt = 0; nt < NTILES; ++nt)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        *(float2*)(out + (m0 + g + 8 * h) * LDY + 8 * nt + 2 * t) =
                            make_float2(ccur[nt][2 * h], ccur[nt][2 * h + 1]);
                if (d.flags & kDownStore) {
                    // a leaf: ŷ_c into its split tile (what the leaf phase reads), read back
                    // from the stack entry in 4×4 blocks
                    __syncthreads();
                    uint8_t* tile = pk.act + (int64_t)d.c * pk.KP * pk.R * pk.es;
                    for (int blk = threadIdx.x; blk < 16 * (NT / 4); blk += blockDim.x) {
                        const int ty = blk / (NT / 4), tx = blk % (NT / 4);
                        float acc[4][4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const float4 v = *(const float4*)(out + (4 * ty + r) * LDY + 4 * tx);
                            acc[r][0] = v.x; acc[r][1] = v.y; acc[r][2] = v.z; acc[r][3] = v.w;
                        }
                        pack_rows(pk, tile, acc, tx, ty, k, m);
                    }
                }
            }
            if (s + 1 < s1) {
#pragma unroll
                for (int nt = 0; nt < NTILES; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) ccur[nt][e] = cnext[nt][e];
            }
            __syncthreads();
        }
    }
}

// ---- transfer matrices as Kronecker products (q = 4) ----
// With tensor Chebyshev interpolation E_c[μ, ν] = L_{ν_x}(ξ_{μ_x}) L_{ν_y}(ξ_{μ_y})
// L_{ν_z}(ξ_{μ_z}) (1-D Lagrange polynomials of the father's nodes at the son's
// nodes, per axis), so E_c = F_z ⊗ F_y ⊗ F_x with 4×4 factors (ν = ν_x + 4ν_y +
// 16ν_z): E_c y costs three 4×4 mode products (48 multiply-adds per column and
// slab) instead of a 64×64 product, and E_c is 48 numbers.  kron[c] holds F_x,
// F_y, F_z row-major (F_a[μ][ν]).
//
// The thread layout of kron_step: lane quad (4 consecutive lanes) g = 0..3 holds
// the z-slab ν_z = g of one column; the x and y mode products stay in the
// thread, the z mode product sums the quad's four slabs through shuffles.
//   f:   F_x and F_y (32 values); fz: the thread's row g of F_z (TR: its column g)
//   in:  x[ν_y][ν_x] = block rows 16g + 4ν_y + ν_x, one column
//   out: y[μ_y][μ_x] = rows 16g + 4μ_y + μ_x of (F_z ⊗ F_y ⊗ F_x) x (TR: of the
//        transposed product, (F_z ⊗ F_y ⊗ F_x)ᵀ = F_zᵀ ⊗ F_yᵀ ⊗ F_xᵀ)
template <bool TR>
__device__ __forceinline__ void kron_step(const float (&f)[32], const float (&fz)[4], const float (&x)[16],
                                          float (&y)[16]) {
    auto F = [&](int a, int mu, int nu) { return TR ? f[16 * a + 4 * nu + mu] : f[16 * a + 4 * mu + nu]; };
    float t[16];
#pragma unroll
    for (int vy = 0; vy < 4; ++vy)
#pragma unroll
        for (int mx = 0; mx < 4; ++mx) {
            float a = 0.f;
#pragma unroll
            for (int vx = 0; vx < 4; ++vx) a = fmaf(F(0, mx, vx), x[4 * vy + vx], a);
            t[4 * vy + mx] = a;
        }
    float u[16];
#pragma unroll
    for (int my = 0; my < 4; ++my)
#pragma unroll
        for (int mx = 0; mx < 4; ++mx) {
            float a = 0.f;
#pragma unroll
            for (int vy = 0; vy < 4; ++vy) a = fmaf(F(1, my, vy), t[4 * vy + mx], a);
            u[4 * my + mx] = a;
        }
    const int base = (threadIdx.x & 31) & ~3;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        float a = 0.f;
#pragma unroll
        for (int vz = 0; vz < 4; ++vz) a = fmaf(fz[vz], __shfl_sync(0xffffffffu, u[e], base | vz), a);
        y[e] = a;
    }
}

// Downward pass with subtree ownership for q = 4 (the schedule of k_down_own):
// each step ŷ_c = ŷ_c + E_c ŷ_father as the Kronecker product above, on the
// CUDA cores.  The father's ŷ comes from a shared-memory stack entry written by
// an earlier step of the same task; the factors of the next step and its
// coupling result load into registers while the current step computes.  The
// first step of a task copies the root's ŷ into its entry (bulk copies); a
// leaf's ŷ goes to global memory and into its split tile, as in k_down_own.
// 128 threads: quad (column c, slab g), c = threadIdx.x / 4 + 32j for j < NT/32.
template <int CN>
__global__ void __launch_bounds__(128) k_down_kron(const int32_t* __restrict__ task_ptr, int ntasks,
                                                   const DownStep* __restrict__ steps,
                                                   const float* __restrict__ kron, float* yhat,
                                                   unsigned* __restrict__ claim, int* __restrict__ err, int m,
                                                   PackOut pk) {
    constexpr int NT = 16 * CN, LDY = NT + 8, NJ = NT >= 32 ? NT / 32 : 1;
    constexpr int k = 64;
    extern __shared__ __align__(16) float fsm[];
    float* stk = fsm;  // [entries][64][LDY]   final ŷ along the current path
    __shared__ int s_task;
    __shared__ DownStep s_steps[kDownMaxSteps];
    __shared__ __align__(8) uint64_t bar;
    const int g = threadIdx.x & 3, cq = threadIdx.x >> 2;
    const int64_t km = (int64_t)k * m;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    bool failed = false;
    // factors (F_x, F_y and row g of F_z) and coupling rows of one step (this
    // thread's slab, columns c_j)
    auto load_step = [&](int c, float (&f)[32], float (&fz)[4], float (&cp)[NJ][16]) {
        if (c < 0) return;
#pragma unroll
        for (int i = 0; i < 32; ++i) f[i] = __ldg(kron + (int64_t)c * 48 + i);
#pragma unroll
        for (int i = 0; i < 4; ++i) fz[i] = __ldg(kron + (int64_t)c * 48 + 32 + 4 * g + i);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int col = cq + 32 * j;
#pragma unroll
            for (int e = 0; e < 16; ++e)
                cp[j][e] = (col < m) ? __ldcg(yhat + (int64_t)c * km + (int64_t)(16 * g + e) * m + col) : 0.f;
        }
    };
    while (!failed) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = (int)atomicAdd(claim, 1u);
        __syncthreads();
        const int task = s_task;
        if (task >= ntasks) break;
        const int s0 = task_ptr[task], s1 = min(task_ptr[task + 1], s0 + kDownMaxSteps);
        for (int i = threadIdx.x; i < s1 - s0; i += blockDim.x) s_steps[i] = steps[s0 + i];
        __syncthreads();
        float fcur[32], fnext[32], zcur[4], znext[4], ccur[NJ][16], cnext[NJ][16];
        {
            int f0 = -1;
            for (int t = s0; t < s1; ++t)
                if (!(s_steps[t - s0].flags & kDownLoad)) { f0 = t; break; }
            if (f0 >= 0) load_step(s_steps[f0 - s0].c, fcur, zcur, ccur);
        }
        for (int s = s0; s < s1; ++s) {
            const DownStep d = s_steps[s - s0];
            if (d.flags & kDownLoad) {
                // the root's ŷ (its coupling result) into entry wr, one bulk copy per row
                const uint32_t rowb = (uint32_t)m * 4;
                if (threadIdx.x < 32) {
                    if (threadIdx.x == 0) mbar_expect_tx(&bar, rowb * (uint32_t)k);
                    __syncwarp();
                    for (int r = threadIdx.x; r < k; r += 32)
                        bulk_g2s(stk + (d.wr * 64 + r) * LDY, yhat + (int64_t)d.c * km + (int64_t)r * m, rowb, &bar);
                }
                const bool ok = mbar_wait(&bar, phase);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) {
                    if (threadIdx.x == 0) {
                        atomicExch(err, 9);
                        mbar_wait(&bar, phase);  // the copies land before the CTA leaves (bounded)
                    }
                    failed = true;
                    break;
                }
                continue;
            }
            // the next step's factors and coupling rows load while this one computes
            int nx = -1;
            for (int t = s + 1; t < s1; ++t)
                if (!(s_steps[t - s0].flags & kDownLoad)) { nx = t; break; }
            load_step(nx >= 0 ? s_steps[nx - s0].c : -1, fnext, znext, cnext);
            const float* in = stk + d.rd * 64 * LDY;
            float* out = stk + d.wr * 64 * LDY;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int col = cq + 32 * j;
                if (cq < NT) {  // whole quads: the shuffles stay within active lanes
                    float x[16], y[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) x[e] = in[(16 * g + e) * LDY + col];
                    kron_step<false>(fcur, zcur, x, y);
#pragma unroll
                    for (int e = 0; e < 16; ++e) out[(16 * g + e) * LDY + col] = y[e] + ccur[j][e];
                }
            }
            __syncthreads();  // entry wr complete
            if (d.flags & kDownStore) {
                // a leaf: ŷ_c into its split tile (what the leaf phase reads), read back in 4×4 blocks
                uint8_t* tile = pk.act + (int64_t)d.c * pk.KP * pk.R * pk.es;
                for (int blk = threadIdx.x; blk < 16 * (NT / 4); blk += blockDim.x) {
                    const int ty = blk / (NT / 4), tx = blk % (NT / 4);
                    float acc[4][4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float4 v = *(const float4*)(out + (4 * ty + r) * LDY + 4 * tx);
                        acc[r][0] = v.x; acc[r][1] = v.y; acc[r][2] = v.z; acc[r][3] = v.w;
                    }
                    pack_rows(pk, tile, acc, tx, ty, k, m);
                }
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) fcur[i] = fnext[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) zcur[i] = znext[i];
#pragma unroll
            for (int j = 0; j < NJ; ++j)
#pragma unroll
                for (int e = 0; e < 16; ++e) ccur[j][e] = cnext[j][e];
        }
    }
}

// k_up_own: two slots of two 64×64 blocks plus the stack
int up_own_smem_bytes(int cn, int entries) { return (4 * 64 * 64 + entries * 64 * 16 * cn) * (int)sizeof(float); }
// k_down_own: two Eᵀ buffers (rows of 72) plus the stack (rows of 16·cn + 8, at most 8 entries)
int down_own_smem_bytes(int cn, int entries) { return (2 * 64 * 72 + entries * 64 * (16 * cn + 8)) * (int)sizeof(float); }
// k_down_kron: the stack only (rows of 16·cn + 8)
int down_kron_smem_bytes(int cn, int entries) { return entries * 64 * (16 * cn + 8) * (int)sizeof(float); }

int g_fast_attr_device = -1;

int fast_prepare() {
    int dev = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    if (dev == g_fast_attr_device) return 0;
    H2_CUDA_TRY(cudaFuncSetAttribute(k_up_own<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, up_own_smem_bytes(1, kUpMaxEntries)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_up_own<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, up_own_smem_bytes(2, kUpMaxEntries)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_up_own<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, up_own_smem_bytes(4, kUpMaxEntries)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_down_own<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_own_smem_bytes(1, 8)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_down_own<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_own_smem_bytes(2, 8)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_down_own<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_own_smem_bytes(4, 8)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_down_kron<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_kron_smem_bytes(1, 8)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_down_kron<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_kron_smem_bytes(2, 8)));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_down_kron<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_kron_smem_bytes(4, 8)));
    g_fast_attr_device = dev;
    return 0;
}

struct PhaseMarks {
    h2_matrix* A;
    cudaStream_t st;
    TimingRecord rec;
    bool failed = false;
    PhaseMarks(h2_matrix* a, cudaStream_t s) : A(a), st(s) {}
    cudaEvent_t record() {
        if (!A || !A->timing.on || failed) return nullptr;
        cudaEvent_t e;
        if (!A->timing.free_events.empty()) {
            e = A->timing.free_events.back();
            A->timing.free_events.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            failed = true;
            return nullptr;
        }
        if (cudaEventRecord(e, st) != cudaSuccess) failed = true;
        return e;
    }
    void mark() {
        cudaEvent_t e = record();
        if (e) rec.ev.push_back(e);
    }
    // events around the coupling kernel alone (phase slot 6)
    void kernel_begin() { if (!rec.k0) rec.k0 = record(); }
    void kernel_end() { if (rec.k0 && !rec.k1) rec.k1 = record(); }
    int commit() {
        if (!A || !A->timing.on) return 0;
        if (failed) {
            for (auto e : rec.ev) A->timing.free_events.push_back(e);
            if (rec.k0) A->timing.free_events.push_back(rec.k0);
            if (rec.k1) A->timing.free_events.push_back(rec.k1);
            set_error("timing event record failed");
            return H2_E_CUDA;
        }
        A->timing.pending.push_back(rec);
        rec = TimingRecord();
        return 0;
    }
};

// Forward transformation: leaves + upward pass (one launch when k <= 64, per
// level otherwise).  Records the leaf-forward and upward phase marks.
template <typename T, int RM, int CN>
int forward_pass(h2_matrix* A, const T* V, const T* E, const T* Xp, T* xhat, int m, unsigned gy, unsigned gzk,
                 cudaStream_t st, const SyncBufs& sb, PhaseMarks& marks, const T* kron = nullptr) {
    const int k = A->k;
    const unsigned NL = (unsigned)A->leaves.size();
    if (gzk == 1) {
        k_up_fused<T, RM, CN><<<dim3(NL, gy), kThreads, 0, st>>>(A->d_leaves, A->d_cl_off, A->d_cl_size,
                                                                A->d_parent, A->d_son0, A->d_son1, V, E, Xp, xhat,
                                                                sb.cnt, k, m, kron);
        H2_LAUNCH_CHECK();
        marks.mark();
        marks.mark();
        return 0;
    }
    k_leaf_fwd<T, RM, CN><<<dim3(NL, gy, gzk), kThreads, 0, st>>>(A->d_leaves, A->d_cl_off, A->d_cl_size, V, Xp,
                                                                  xhat, k, m);
    H2_LAUNCH_CHECK();
    marks.mark();
    for (int l = A->depth - 1; l >= 0; --l) {
        const int64_t b = A->up_ptr[l], e = A->up_ptr[l + 1];
        if (e == b) continue;
        k_up<T, RM, CN><<<dim3((unsigned)(e - b), gy, gzk), kThreads, 0, st>>>(A->d_up_list + b, A->d_son0,
                                                                              A->d_son1, E, xhat, k, m);
        H2_LAUNCH_CHECK();
    }
    marks.mark();
    return 0;
}

// Backward transfer pass ŷ_{t'} += E_{t'} ŷ_t (one launch when k <= 64).
template <typename T, int RM, int CN>
int backward_pass(h2_matrix* A, const T* E, T* yhat, int m, unsigned gy, unsigned gzk, cudaStream_t st,
                  const SyncBufs& sb, const T* kron = nullptr) {
    const int k = A->k;
    const int n_items = (int)A->down_ptr[A->depth + 1];
    if (n_items == 0) return 0;
    if (gzk == 1) {
        // ready flags and claim tickets start at zero for every product (graph-replay safe)
        H2_CUDA_TRY(cudaMemsetAsync(sb.flag, 0, (size_t)A->nc * gy * sizeof(int), st));
        H2_CUDA_TRY(cudaMemsetAsync(sb.claim, 0, gy * sizeof(unsigned), st));
        const unsigned g = (unsigned)std::min(n_items, 152 * 6);
        k_down_fused<T, RM, CN><<<dim3(g, gy), kThreads, 0, st>>>(A->d_down_list, n_items, A->d_parent, E, yhat,
                                                                 sb.claim, sb.flag, sb.epoch, sb.err, k, m,
                                                                 wait_limit(), kron);
        H2_LAUNCH_CHECK();
        return 0;
    }
    for (int l = 1; l <= A->depth; ++l) {
        const int64_t b = A->down_ptr[l], e = A->down_ptr[l + 1];
        if (e == b) continue;
        k_down<T, RM, CN><<<dim3((unsigned)(e - b), gy, gzk), kThreads, 0, st>>>(A->d_down_list + b, A->d_parent, E,
                                                                                yhat, k, m);
        H2_LAUNCH_CHECK();
    }
    return 0;
}

// alpha_im: the complex product (m counts the 2·m_c real columns of the interleaved
// complex blocks; CN is even); the transfer passes are the real ones.
template <typename T, int RM, int CN>
int run_chain(h2_matrix* A, const MatData& D, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
              int m, cudaStream_t st, bool transposed, bool overwrite, T* Xp, T* xhat, T* yhat, const SyncBufs& sb,
              const double* alpha_im = nullptr) {
    constexpr int MT = 16 * RM, NT = 16 * CN;
    const int k = A->k;
    const unsigned gy = (unsigned)((m + NT - 1) / NT);
    const unsigned gzk = (unsigned)((k + MT - 1) / MT);
    const unsigned gzl = (unsigned)((A->T.leaf_size + MT - 1) / MT);
    const T* V = (const T*)D.V;
    const T* E = (const T*)D.E;
    const T* S = (const T*)D.S;
    const T* G = (const T*)D.Near;
    // q = 4: the transfer passes apply E_c as a Kronecker product of its 1-D factors
    const T* kron = (k == 64 && RM == 4 && A->use_kron) ? (const T*)D.kron : nullptr;
    PhaseMarks marks(A, st);
    int rc = 0;
    marks.mark();
    {
        const int64_t total = A->n * m;
        const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
        k_gather<T><<<g, 256, 0, st>>>(X, ldx, A->d_perm, A->n, m, Xp);
        H2_LAUNCH_CHECK();
    }
    marks.mark();
    const unsigned NL = (unsigned)A->leaves.size();
    if ((rc = forward_pass<T, RM, CN>(A, V, E, Xp, xhat, m, gy, gzk, st, sb, marks, kron))) return rc;
    marks.kernel_begin();
    if (alpha_im) {
        if constexpr (CN % 2 == 0) {
            k_coupling_c<T, RM, CN><<<dim3((unsigned)A->nc, gy, gzk), kThreads, 0, st>>>(
                A->d_adm_rowptr, A->d_adm_col, S, A->n_adm * (int64_t)k * k, xhat, yhat, k, m);
        } else {
            set_error("complex product: column tiles must hold whole complex columns");
            return H2_E_UNSUPPORTED;
        }
    } else if (transposed)
        k_coupling<T, RM, CN, true><<<dim3((unsigned)A->nc, gy, gzk), kThreads, 0, st>>>(
            A->d_admT_rowptr, A->d_admT_row, A->d_admT_blk, S, xhat, yhat, k, m);
    else
        k_coupling<T, RM, CN, false><<<dim3((unsigned)A->nc, gy, gzk), kThreads, 0, st>>>(
            A->d_adm_rowptr, A->d_adm_col, nullptr, S, xhat, yhat, k, m);
    H2_LAUNCH_CHECK();
    marks.kernel_end();
    marks.mark();
    if ((rc = backward_pass<T, RM, CN>(A, E, yhat, m, gy, gzk, st, sb, kron))) return rc;
    marks.mark();
    if ((rc = wait_y_staged(A->ws, st))) return rc;
    if (alpha_im) {
        if constexpr (CN % 2 == 0) {
            k_leaf_bwd_near_c<T, RM, CN><<<dim3(NL, gy, gzl), kThreads, 0, st>>>(
                A->d_leaves, A->d_cl_off, A->d_cl_size, A->d_perm, V, yhat, A->d_near_ptr, A->d_near_col,
                A->d_near_off, G, A->nnz_near, Xp, Y, ldy, alpha, *alpha_im, A->sigma, k, m, overwrite ? 1 : 0);
        } else {
            set_error("complex product: column tiles must hold whole complex columns");
            return H2_E_UNSUPPORTED;
        }
    } else if (transposed)
        k_leaf_bwd_near<T, RM, CN, true><<<dim3(NL, gy, gzl), kThreads, 0, st>>>(
            A->d_leaves, A->d_cl_off, A->d_cl_size, A->d_perm, V, yhat, A->d_nearT_ptr, A->d_nearT_row,
            A->d_nearT_blk, A->d_near_off, G, Xp, Y, ldy, alpha, A->sigma, k, m, overwrite ? 1 : 0);
    else
        k_leaf_bwd_near<T, RM, CN, false><<<dim3(NL, gy, gzl), kThreads, 0, st>>>(
            A->d_leaves, A->d_cl_off, A->d_cl_size, A->d_perm, V, yhat, A->d_near_ptr, A->d_near_col, nullptr,
            A->d_near_off, G, Xp, Y, ldy, alpha, A->sigma, k, m, overwrite ? 1 : 0);
    H2_LAUNCH_CHECK();
    marks.mark();
    return marks.commit();
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }



int ensure_workspace(h2_matrix* A, size_t bytes, cudaStream_t st) {
    if (A->ws.bytes >= bytes) return 0;
    if (A->ws.base) {
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        H2_CUDA_TRY(cudaFree(A->ws.base));
        A->ws.base = nullptr;
        A->ws.bytes = 0;
    }
    H2_CUDA_TRY(cudaMalloc(&A->ws.base, bytes));
    A->ws.bytes = bytes;
    return 0;
}


// Tensor-core product (KIND 0: BF16; KIND 1: FP32 on split TF32): the
// coupling and the leaf phase (nearfield + backward transformation + shift)
// run on the tensor cores (h2_tc.cu); the gather, the forward transformation
// and the transfer passes run in FP32 on the CUDA cores with the FP32 copies of
// V and E.  Columns are processed in chunks of at most 64 (128 MMA rows: the
// high and low parts of each column).
template <int CN>
int run_chain_tc(h2_matrix* A, int kind, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy, int m,
                 cudaStream_t st, bool overwrite, const SyncBufs& sb, bool trans, const double* alpha_im) {
    // alpha_im: the complex product (m counts the 2·m_c interleaved real columns; the
    // term lists carry the S_im and G_im terms, the transfer passes are the real ones)
    const bool cx = alpha_im != nullptr;
    // kind 2: the TF32 product with the matrix-free coupling (tensor-core kernel mode 2)
    const bool mf = kind == 2;
    if (mf) kind = 1;
    const int es = kind == 0 ? 2 : 4;
    constexpr int RM = 4, MT = 16 * RM, NT = 16 * CN;
    const TcData& D = A->tc;
    const int k = A->k, KP = D.KP;
    const int64_t n = A->n, nc = A->nc;
    const int NL = (int)A->leaves.size();
    const float* V = (const float*)A->f32.V;
    const float* E = (const float*)A->f32.E;

    const int grid_cap = kTcGrid;
    SyncBufs sbc = sb;
    for (int c0 = 0; c0 < m; c0 += 64) {
        const int mc = std::min(64, m - c0);
        const int R = round16(2 * mc);
        const size_t bXp = align_up((size_t)n * mc * 4), bC = align_up((size_t)nc * k * mc * 4);
        const size_t bXcm = align_up((size_t)R * D.xk_total * es), bAct = align_up((size_t)nc * R * KP * es);
        // The variant of this column chunk: the autotuner's choice, else the built-in
        // rule (the tensor-core transfer passes where the CUDA-core subtree passes do
        // not apply).  The tensor-core transfer passes are FP32 only, and not used
        // inside a stream capture, whose concurrent branches could keep some of their
        // CTAs from being resident.
        const Tune tn = A->tune[kind == 0 ? 1 : 0][column_class(mc)];
        const int stg = tn.stages;
        const bool fast = A->f32.Et && k % 8 == 0 && k <= 64 && mc % 4 == 0 && A->T.leaf_size <= 64;
        bool want_flow = !fast;
        if (tn.path == kPathTcOwn || tn.path == kPathTcHybrid) want_flow = false;
        if (tn.path == kPathTcFlow || tn.path == kPathTcFused) want_flow = true;
        if (A->use_flow >= 0) want_flow = A->use_flow == 1;
        const bool capturing = stream_capture_active(st);
        const bool flow = kind == 1 && D.flow && want_flow && !capturing && !cx;
        // hybrid: the subtree passes stop at the upward cut, and the clusters above it
        // are transfer items of the coupling launch (k_tc_gemm<4, KIND>), which waits
        // for them only where a coupling reads them
        bool want_hybrid = tn.path == kPathTcHybrid || (tn.path == kPathDefault && D.h_default);
        if (A->use_hybrid >= 0) want_hybrid = A->use_hybrid == 1;
        const bool lists = kind == 1 ? D.hybrid : D.hybrid_bf16;
        const bool hybrid = fast && !flow && !trans && !mf && !cx && lists && want_hybrid && !capturing;
        int rc = ensure_workspace(A, bXp + 2 * bC + bXcm + 3 * bAct, st);
        if (rc) return rc;
        char* base = (char*)A->ws.base;
        float* Xp = (float*)base;
        float* xhat = (float*)(base + bXp);
        float* yhat = (float*)(base + bXp + bC);
        uint8_t* Xcm = (uint8_t*)(base + bXp + 2 * bC);
        uint8_t* xcm = Xcm + bXcm;
        uint8_t* ycm = xcm + bAct;
        uint8_t* ycp = ycm + bAct;  // flow: the coupling results as split tiles
        const unsigned gy = (unsigned)((mc + NT - 1) / NT), gzk = (unsigned)((k + MT - 1) / MT);
        PhaseMarks marks(A, st);
        marks.mark();
        // the subtree passes' arrival counters and task counters, and the hybrid
        // launch's ready flags, are zeroed by the gather
        const bool reset_in_gather = fast && !flow && sbc.claim2;
        {
            const int64_t total = n * mc;
            const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
            // claim2 follows the claim counters in the same allocation: zero them all
            // with the hybrid pass (no climb, so nothing writes ŷ before the coupling
            // launch) also ŷ of the clusters without couplings
            if (reset_in_gather)
                k_gather<float><<<g, 256, 0, st>>>(X + c0, ldx, A->d_perm, n, mc, Xp, sbc.cnt, (int)nc, sbc.claim,
                                                   (int)(sbc.claim2 - sbc.claim) + 1, hybrid ? sbc.fflag : nullptr,
                                                   hybrid ? (int)nc : 0, hybrid ? D.c_zero : nullptr,
                                                   hybrid ? D.c_nzero : 0, yhat, k, mc, mc);
            else
                k_gather<float><<<g, 256, 0, st>>>(X + c0, ldx, A->d_perm, n, mc, Xp);
            H2_LAUNCH_CHECK();
        }
        // (fast: the subtree-owning CUDA-core transfer passes apply, rows of 16-byte
        // multiples; they also write the split tiles of X (leaves), x̂ and leaf ŷ)
        if ((!fast || flow) &&
            (rc = launch_pack_act(Xp, mc, NL, nullptr, D.leaf_base, D.leaf_kdim, 0, D.xkoff, 0, mc, R, Xcm, es, st)))
            return rc;
        marks.mark();
        const int fcn = mc <= 16 ? 1 : (mc <= 32 ? 2 : 4);
        if (flow) {
            // Both transfer passes on the tensor cores.  With A (and the stored
            // couplings) the upward pass shares one launch with the coupling phase
            // and the downward pass one with the leaf phase; with Aᵀ, or the
            // matrix-free coupling, the four phases are launched one by one.
            H2_CUDA_TRY(cudaMemsetAsync(sbc.fflag, 0, 2 * (size_t)nc * sizeof(int), st));
            if ((rc = launch_zero_tiles(trans ? D.ct_zero : D.c_zero, trans ? D.ct_nzero : D.c_nzero, ycp,
                                        (int64_t)KP * R * es, st)))
                return rc;
            TcGemmParams fp{};
            fp.bmat = D.mat32;
            fp.R = R;
            fp.mc = mc;
            fp.k = k;
            fp.ldc = mc;
            fp.err = A->err_dev;
            fp.KP = KP;
            fp.epoch = 1;
            fp.leaves = A->d_leaves;
            fp.cl_off = A->d_cl_off;
            fp.cl_size = A->d_cl_size;
            TcGemmParams f1 = fp, f2 = fp;
            // upward items: act0 the x̂ tiles of the launch, act1 the X tiles; coupling items
            // write the ŷ tiles of the coupling results (ycp)
            f1.act0 = xcm;
            f1.act1 = Xcm;
            f1.out_act = xcm;
            f1.out_act2 = ycp;
            f1.flag = sbc.fflag;
            // downward items: act0 the ŷ tiles of the launch, act1 the coupling results; leaf
            // items: act2 the X tiles, output the rows of Z (over the gathered X)
            f2.act0 = ycm;
            f2.act1 = ycp;
            f2.act2 = Xcm;
            f2.out_act = ycm;
            f2.flag = sbc.fflag + nc;
            f2.zp = Xp;
            const bool fused = !trans && !mf && tn.path != kPathTcFlow;
            if (fused) {
                f1.n_items = D.f1_nitems;
                f1.items = D.f1_items;
                f1.terms = D.f1_terms;
                f2.n_items = D.f2_nitems;
                f2.items = D.f2_items;
                f2.terms = D.f2_terms;
                marks.kernel_begin();
                if ((rc = launch_tc_gemm(3, 1, f1, std::min(f1.n_items, grid_cap), st, stg))) return rc;
                marks.kernel_end();
                marks.mark();
                marks.mark();
                marks.mark();
                if ((rc = launch_tc_gemm(3, 1, f2, std::min(f2.n_items, grid_cap), st, stg))) return rc;
                marks.mark();
            } else {
                f1.n_items = D.up_nitems;
                f1.items = D.up_items;
                f1.terms = D.up_terms;
                if ((rc = launch_tc_gemm(3, 1, f1, std::min(f1.n_items, grid_cap), st, stg))) return rc;
                marks.mark();
                marks.mark();
                TcGemmParams cp{};
                cp.n_items = trans ? D.ct_nitems : D.c_nitems;
                cp.items = trans ? D.ct_items : D.c_items;
                cp.terms = trans ? D.ct_terms : D.c_terms;
                cp.act0 = xcm;
                cp.act1 = xcm;
                cp.bmat = trans ? D.matT32 : D.mat32;
                cp.R = R;
                cp.mc = mc;
                cp.yhat = yhat;
                cp.k = k;
                cp.ldc = mc;
                cp.err = A->err_dev;
                cp.nodes = D.nodes4;
                cp.inv_len = (float)(1.0 / A->length);
                cp.KP = KP;
                cp.out_act = ycp;  // split tiles for the downward pass's identity terms
                marks.kernel_begin();
                if (cp.n_items > 0 && (rc = launch_tc_gemm(mf ? 2 : 0, 1, cp, std::min(cp.n_items, grid_cap), st, stg)))
                    return rc;
                marks.kernel_end();
                marks.mark();
                f2.n_items = D.dn_nitems;
                f2.items = D.dn_items;
                f2.terms = D.dn_terms;
                if ((rc = launch_tc_gemm(3, 1, f2, std::min(f2.n_items, grid_cap), st, stg))) return rc;
                marks.mark();
                TcGemmParams lp{};
                lp.n_items = trans ? D.lt_nitems : D.l_nitems;
                lp.items = trans ? D.lt_items : D.l_items;
                lp.terms = trans ? D.lt_terms : D.l_terms;
                lp.act0 = Xcm;
                lp.act1 = ycm;
                lp.bmat = trans ? D.matT32 : D.mat32;
                lp.R = R;
                lp.mc = mc;
                lp.leaves = A->d_leaves;
                lp.cl_off = A->d_cl_off;
                lp.cl_size = A->d_cl_size;
                lp.err = A->err_dev;
                lp.zp = Xp;
                lp.ldc = mc;
                if ((rc = launch_tc_gemm(1, 1, lp, std::min(lp.n_items, grid_cap), st, stg))) return rc;
            }
            const int64_t total = n * mc;
            const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
            if ((rc = wait_y_staged(A->ws, st))) return rc;
            k_scatter_y<<<g, 256, 0, st>>>(Xp, mc, A->d_perm, n, mc, X + c0, ldx, Y + c0, ldy, alpha, A->sigma,
                                           overwrite ? 1 : 0);
            H2_LAUNCH_CHECK();
            marks.mark();
            if ((rc = marks.commit())) return rc;
            continue;
        }
        if (fast) {
            if ((rc = fast_prepare())) return rc;
            const PackOut pk{xcm, Xcm, D.xkoff, KP, R, es};
            const int usm = up_own_smem_bytes(fcn, A->up_entries);
            const unsigned g = (unsigned)std::min(A->up_ntasks, 152 * std::max(1, (227 * 1024) / (usm + 2048)));
            if (!reset_in_gather) {
                H2_CUDA_TRY(cudaMemsetAsync(sbc.cnt, 0, (size_t)nc * sizeof(unsigned), st));
                H2_CUDA_TRY(cudaMemsetAsync(sbc.claim, 0, sizeof(unsigned), st));
            }
            const int climb = hybrid ? 0 : 1;
            // q = 4: the inner steps and the climb apply E_sᵀ as Kronecker products
            const float* ukron = (k == 64 && A->use_kron) ? (const float*)A->f32.kron : nullptr;
            if (fcn == 1) k_up_own<1><<<g, 64, usm, st>>>(A->d_up_task_ptr, A->up_ntasks, A->d_up_steps, A->d_cl_off, A->d_cl_size, A->d_parent, A->d_son0, A->d_son1, V, E, Xp, xhat, yhat, sbc.cnt, sbc.claim, sbc.err, A->up_entries, k, mc, pk, climb, ukron);
            else if (fcn == 2) k_up_own<2><<<g, 128, usm, st>>>(A->d_up_task_ptr, A->up_ntasks, A->d_up_steps, A->d_cl_off, A->d_cl_size, A->d_parent, A->d_son0, A->d_son1, V, E, Xp, xhat, yhat, sbc.cnt, sbc.claim, sbc.err, A->up_entries, k, mc, pk, climb, ukron);
            else k_up_own<4><<<g, 256, usm, st>>>(A->d_up_task_ptr, A->up_ntasks, A->d_up_steps, A->d_cl_off, A->d_cl_size, A->d_parent, A->d_son0, A->d_son1, V, E, Xp, xhat, yhat, sbc.cnt, sbc.claim, sbc.err, A->up_entries, k, mc, pk, climb, ukron);
            H2_LAUNCH_CHECK();
            marks.mark();
            marks.mark();
        } else if ((rc = forward_pass<float, RM, CN>(A, V, E, Xp, xhat, mc, gy, gzk, st, sbc, marks))) {
            return rc;
        }
        if (!fast &&
            (rc = launch_pack_act(xhat, mc, (int)nc, nullptr, nullptr, nullptr, k, nullptr, KP, mc, R, xcm, es, st)))
            return rc;
        // Aᵀ: the coupling runs over column clusters with S_bᵀ, the leaf phase over
        // column leaves with G_bᵀ (tiles and lists of build_tc_transposed)
        const uint8_t* bmat = trans ? (kind == 0 ? D.matT : D.matT32) : (kind == 0 ? D.mat : D.mat32);
        if (!(reset_in_gather && hybrid) &&
            (rc = launch_zero_clusters(trans ? D.ct_zero : D.c_zero, trans ? D.ct_nzero : D.c_nzero, yhat, k, mc, mc,
                                       st)))
            return rc;
        TcGemmParams cp{};
        cp.n_items = trans ? D.ct_nitems : D.c_nitems;
        cp.items = trans ? D.ct_items : D.c_items;
        cp.terms = trans ? D.ct_terms : D.c_terms;
        cp.act0 = xcm;
        cp.act1 = xcm;
        cp.bmat = bmat;
        cp.R = R;
        cp.mc = mc;
        cp.yhat = yhat;
        cp.k = k;
        cp.ldc = mc;
        cp.err = A->err_dev;
        cp.nodes = D.nodes4;
        cp.inv_len = (float)(1.0 / A->length);
        cp.KP = KP;
        cp.cplx = cx ? 1 : 0;
        if (hybrid) {
            cp.n_items = kind == 1 ? D.h_nitems : D.hb_nitems;
            cp.items = kind == 1 ? D.h_items : D.hb_items;
            cp.terms = kind == 1 ? D.h_terms : D.hb_terms;
            cp.out_act = xcm;  // the transfer items' split tiles
            cp.flag = sbc.fflag;
            cp.epoch = 1;
            if (!reset_in_gather) H2_CUDA_TRY(cudaMemsetAsync(sbc.fflag, 0, (size_t)nc * sizeof(int), st));
        }
        marks.kernel_begin();
        if (cp.n_items > 0 &&
            (rc = launch_tc_gemm(hybrid ? 4 : (mf ? 2 : 0), kind, cp, std::min(cp.n_items, grid_cap), st, stg)))
            return rc;
        marks.kernel_end();
        marks.mark();
        bool leaf_y_packed = false;
        if (fast) {
            const int n_items = (int)A->down_ptr[A->depth + 1];
            if (n_items > 0) {
                const PackOut pk{ycm, nullptr, nullptr, KP, R, es};
                leaf_y_packed = true;
                // the task counter of this pass: claim2, zeroed by the gather (else claim again)
                unsigned* dclaim = reset_in_gather ? sbc.claim2 : sbc.claim;
                if (!reset_in_gather) H2_CUDA_TRY(cudaMemsetAsync(sbc.claim, 0, sizeof(unsigned), st));
                const float* Et = (const float*)A->f32.Et;
                const int smem = down_own_smem_bytes(fcn, A->dn_entries);
                const unsigned g = (unsigned)std::min(A->dn_ntasks, 152 * std::max(1, (227 * 1024) / (smem + 4096)));
                const float* kron = (const float*)A->f32.kron;
                if (kron && k == 64 && A->use_kron && fcn >= 2) {
                    // q = 4: each step as three 4×4 mode products (E_c = F_z ⊗ F_y ⊗ F_x); with
                    // 16 columns or fewer half its threads would idle, and the dense pass is faster
                    const int ksm = down_kron_smem_bytes(fcn, A->dn_entries);
                    const unsigned gk =
                        (unsigned)std::min(A->dn_ntasks, 152 * std::max(1, (227 * 1024) / (ksm + 4096)));
                    if (fcn == 1) k_down_kron<1><<<gk, 128, ksm, st>>>(A->d_dn_task_ptr, A->dn_ntasks, A->d_dn_steps, kron, yhat, dclaim, sbc.err, mc, pk);
                    else if (fcn == 2) k_down_kron<2><<<gk, 128, ksm, st>>>(A->d_dn_task_ptr, A->dn_ntasks, A->d_dn_steps, kron, yhat, dclaim, sbc.err, mc, pk);
                    else k_down_kron<4><<<gk, 128, ksm, st>>>(A->d_dn_task_ptr, A->dn_ntasks, A->d_dn_steps, kron, yhat, dclaim, sbc.err, mc, pk);
                } else if (fcn == 1) k_down_own<1><<<g, 128, smem, st>>>(A->d_dn_task_ptr, A->dn_ntasks, A->d_dn_steps, Et, yhat, dclaim, sbc.err, k, mc, pk);
                else if (fcn == 2) k_down_own<2><<<g, 128, smem, st>>>(A->d_dn_task_ptr, A->dn_ntasks, A->d_dn_steps, Et, yhat, dclaim, sbc.err, k, mc, pk);
                else k_down_own<4><<<g, 128, smem, st>>>(A->d_dn_task_ptr, A->dn_ntasks, A->d_dn_steps, Et, yhat, dclaim, sbc.err, k, mc, pk);
                H2_LAUNCH_CHECK();
            }
        } else if ((rc = backward_pass<float, RM, CN>(A, E, yhat, mc, gy, gzk, st, sbc))) {
            return rc;
        }
        if (!leaf_y_packed &&
            (rc = launch_pack_act(yhat, mc, NL, A->d_leaves, nullptr, nullptr, k, nullptr, KP, mc, R, ycm, es, st)))
            return rc;
        marks.mark();
        TcGemmParams lp{};
        lp.n_items = trans ? D.lt_nitems : D.l_nitems;
        lp.items = trans ? D.lt_items : D.l_items;
        lp.terms = trans ? D.lt_terms : D.l_terms;
        lp.act0 = Xcm;
        lp.act1 = ycm;
        lp.bmat = bmat;
        lp.R = R;
        lp.mc = mc;
        lp.leaves = A->d_leaves;
        lp.cl_off = A->d_cl_off;
        lp.cl_size = A->d_cl_size;
        lp.err = A->err_dev;
        lp.zp = Xp;  // the gathered FP32 X is no longer read after the forward pass and its packing
        lp.ldc = mc;
        lp.cplx = cx ? 1 : 0;
        if ((rc = launch_tc_gemm(1, kind, lp, std::min(lp.n_items, grid_cap), st, stg))) return rc;
        {
            const int64_t total = n * mc;
            const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
            if ((rc = wait_y_staged(A->ws, st))) return rc;
            if (cx)
                k_scatter_yc<<<g, 256, 0, st>>>(Xp, mc, A->d_perm, n, mc, X + c0, ldx, Y + c0, ldy, alpha, *alpha_im,
                                                A->sigma, overwrite ? 1 : 0);
            else
                k_scatter_y<<<g, 256, 0, st>>>(Xp, mc, A->d_perm, n, mc, X + c0, ldx, Y + c0, ldy, alpha, A->sigma,
                                               overwrite ? 1 : 0);
            H2_LAUNCH_CHECK();
        }
        marks.mark();
        if ((rc = marks.commit())) return rc;
    }
    return 0;
}

int dispatch_tc(h2_matrix* A, int kind, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
                int64_t m, cudaStream_t st, bool overwrite, const SyncBufs& sb, bool trans = false,
                const double* alpha_im = nullptr) {
    if (trans) {
        int rc = build_tc_transposed(A, st);
        if (rc) return rc;
    }
    if (m <= 16) return run_chain_tc<1>(A, kind, alpha, X, ldx, Y, ldy, (int)m, st, overwrite, sb, trans, alpha_im);
    if (m <= 32) return run_chain_tc<2>(A, kind, alpha, X, ldx, Y, ldy, (int)m, st, overwrite, sb, trans, alpha_im);
    return run_chain_tc<4>(A, kind, alpha, X, ldx, Y, ldy, (int)m, st, overwrite, sb, trans, alpha_im);
}

template <typename T>
int dispatch_cn(h2_matrix* A, const MatData& D, double alpha, const double* X, int64_t ldx, double* Y,
                int64_t ldy, int m, cudaStream_t st, bool transposed, bool overwrite, T* Xp, T* xhat, T* yhat,
                const SyncBufs& sb, const double* alpha_im = nullptr) {
    if (alpha_im) {  // complex: column tiles of an even width (2 or 4 per thread)
        if (m <= 32)
            return run_chain<T, 4, 2>(A, D, alpha, X, ldx, Y, ldy, m, st, false, overwrite, Xp, xhat, yhat, sb,
                                      alpha_im);
        return run_chain<T, 4, 4>(A, D, alpha, X, ldx, Y, ldy, m, st, false, overwrite, Xp, xhat, yhat, sb,
                                  alpha_im);
    }
    if (m <= 16) return run_chain<T, 4, 1>(A, D, alpha, X, ldx, Y, ldy, m, st, transposed, overwrite, Xp, xhat, yhat, sb);
    if (m <= 32) return run_chain<T, 4, 2>(A, D, alpha, X, ldx, Y, ldy, m, st, transposed, overwrite, Xp, xhat, yhat, sb);
    return run_chain<T, 4, 4>(A, D, alpha, X, ldx, Y, ldy, m, st, transposed, overwrite, Xp, xhat, yhat, sb);
}

// Column tiles of the SIMT chain (and of the tensor-core chain, whose chunks of
// at most 64 columns are one tile): the bookkeeping is sized per tile.
int64_t sync_tiles_for(int64_t m) { return m <= 32 ? 1 : (m + 63) / 64; }

int ensure_sync(h2_matrix* A, int64_t tiles, cudaStream_t st, SyncBufs* sb) {
    if (A->sync_tiles < tiles) {
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        if (A->sync_cnt) cudaFree(A->sync_cnt);
        A->sync_cnt = nullptr;
        A->sync_tiles = 0;
        const size_t per = (size_t)A->nc * tiles;
        // claim: `tiles` counters and one more (the tensor-core chain's downward pass)
        const size_t bytes = per * (sizeof(unsigned) + sizeof(int)) + (tiles + 1) * sizeof(unsigned) +
                             2 * (size_t)A->nc * sizeof(int);
        H2_CUDA_TRY(cudaMalloc(&A->sync_cnt, bytes));
        H2_CUDA_TRY(cudaMemsetAsync(A->sync_cnt, 0, bytes, st));
        A->sync_flag = (int*)(A->sync_cnt + per);
        A->sync_claim = (unsigned*)(A->sync_flag + per);
        A->sync_fflag = (int*)(A->sync_claim + tiles + 1);
        A->sync_tiles = tiles;
    }
    sb->cnt = A->sync_cnt;
    sb->flag = A->sync_flag;
    sb->claim = A->sync_claim;
    sb->claim2 = A->sync_claim + A->sync_tiles;
    sb->fflag = A->sync_fflag;
    sb->epoch = 1;  // flags are cleared before every downward pass
    sb->err = A->err_dev;
    return 0;
}

int check_device_error(h2_matrix* A) {
    if (A->err_host && *A->err_host) {
        *A->err_host = 0;
        set_error("a previous product hit a bounded device-side wait (its result is invalid)");
        return H2_E_TIMEOUT;
    }
    return 0;
}

}  // namespace

int refuse_complex(const h2_matrix* A, const char* what) {
    if (A && A->cplx) {
        set_error(std::string(what) + ": the matrix has a complex kernel; use h2_matmul_complex");
        return H2_E_UNSUPPORTED;
    }
    return 0;
}

int matmul_device(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                  int32_t dtype, cudaStream_t st, bool transposed, bool overwrite, const double* alpha_im) {
    if (!alpha_im) {
        const int rc = refuse_complex(A, "real product");
        if (rc) return rc;
    } else {
        if (!A->cplx) { set_error("h2_matmul_complex: the matrix has a real kernel"); return H2_E_UNSUPPORTED; }
        if (transposed || (dtype != H2_F64 && dtype != H2_F32) || (m & 1)) {
            set_error("complex product: A·X in H2_F64 or H2_F32 only");
            return H2_E_UNSUPPORTED;
        }
    }
    if (m == 0) return 0;
    const size_t elt = dtype == H2_F64 ? sizeof(double) : sizeof(float);
    const size_t bXp = align_up((size_t)A->n * m * elt);
    const size_t bC = align_up((size_t)A->nc * A->k * m * elt);
    int rc = check_device_error(A);
    if (rc) return rc;
    rc = dtype == H2_BF16 ? 0 : ensure_workspace(A, bXp + 2 * bC, st);
    if (rc) return rc;
    SyncBufs sb;
    if ((rc = ensure_sync(A, sync_tiles_for(m), st, &sb))) return rc;
    char* base = (char*)A->ws.base;
    if (dtype == H2_F64) {
        if (!A->f64.built) { set_error("FP64 data not built"); return H2_E_UNSUPPORTED; }
        return dispatch_cn<double>(A, A->f64, alpha, X, ldx, Y, ldy, (int)m, st, transposed, overwrite,
                                   (double*)base, (double*)(base + bXp), (double*)(base + bXp + bC), sb, alpha_im);
    }
    if (dtype == H2_F32) {
        if (!A->f32.built) { set_error("FP32 copy not built (add 1<<H2_F32 to params->precisions)"); return H2_E_UNSUPPORTED; }
        if (alpha_im) {
            // the complex product: split-TF32 tensor cores where their tiles were built
            if (A->tc.has_tf32 && !A->force_simt)
                return dispatch_tc(A, 1, alpha, X, ldx, Y, ldy, m, st, overwrite, sb, false, alpha_im);
            return dispatch_cn<float>(A, A->f32, alpha, X, ldx, Y, ldy, (int)m, st, false, overwrite, (float*)base,
                                      (float*)(base + bXp), (float*)(base + bXp + bC), sb, alpha_im);
        }
        const Tune& tn = A->tune[0][column_class((int)std::min<int64_t>(m, 64))];
        if (A->tc.has_tf32 && !A->force_simt && tn.path != kPathSimt)
            return dispatch_tc(A, 1, alpha, X, ldx, Y, ldy, m, st, overwrite, sb, transposed);
        return dispatch_cn<float>(A, A->f32, alpha, X, ldx, Y, ldy, (int)m, st, transposed, overwrite,
                                  (float*)base, (float*)(base + bXp), (float*)(base + bXp + bC), sb);
    }
    if (dtype == H2_F32_MF) {
        if (!A->tc.has_tf32 || !A->tc.nodes4 || A->force_simt) {
            set_error("matrix-free product: TF32 tiles not built (add 1<<H2_F32 to params->precisions)");
            return H2_E_UNSUPPORTED;
        }
        if (transposed) { set_error("the matrix-free product supports A·X only"); return H2_E_UNSUPPORTED; }
        if (A->s_replaced) {
            set_error("matrix-free product: the coupling matrices were replaced (h2_coupling_set), they are no longer g's values");
            return H2_E_UNSUPPORTED;
        }
        return dispatch_tc(A, 2, alpha, X, ldx, Y, ldy, m, st, overwrite, sb);
    }
    if (dtype == H2_BF16) {
        if (!A->tc.has_bf16) { set_error("BF16 copy not built (add 1<<H2_BF16 to params->precisions)"); return H2_E_UNSUPPORTED; }
        return dispatch_tc(A, 0, alpha, X, ldx, Y, ldy, m, st, overwrite, sb, transposed);
    }
    set_error("unsupported dtype for the product");
    return H2_E_UNSUPPORTED;
}

int product_prepare(h2_matrix* A, int64_t m, int32_t dtype, cudaStream_t st) {
    if (m <= 0) return 0;
    int rc = 0;
    const int64_t n = A->n, nc = A->nc;
    const int k = A->k;
    size_t need = 0;
    const bool tc = (dtype == H2_BF16) || ((dtype == H2_F32 || dtype == H2_F32_MF) && A->tc.has_tf32 && !A->force_simt &&
                                           A->tune[0][column_class((int)std::min<int64_t>(m, 64))].path != kPathSimt);
    if (tc) {
        const TcData& D = A->tc;
        const int es = dtype == H2_BF16 ? 2 : 4;
        const int mc = (int)std::min<int64_t>(64, m);
        const int R = round16(2 * mc);
        need = align_up((size_t)n * mc * 4) + 2 * align_up((size_t)nc * k * mc * 4) +
               align_up((size_t)R * D.xk_total * es) + 3 * align_up((size_t)nc * R * D.KP * es);
        if ((rc = tc_prepare())) return rc;
    } else {
        const size_t elt = dtype == H2_F64 ? sizeof(double) : sizeof(float);
        need = align_up((size_t)n * m * elt) + 2 * align_up((size_t)nc * k * m * elt);
    }
    if ((rc = ensure_workspace(A, need, st))) return rc;
    SyncBufs sb;
    return ensure_sync(A, sync_tiles_for(m), st, &sb);
}

bool flow_batchable(const h2_matrix* A, int64_t m) {
    return m >= 1 && m <= 64 && A->f32.built && A->tc.has_tf32 && A->tc.flow && !A->force_simt;
}

// The workspace layout of run_chain_tc for one chunk of m <= 64 columns (FP32).
int flow_prepare(h2_matrix* A, int m, cudaStream_t st, FlowBufs* fb) {
    const TcData& D = A->tc;
    const int k = A->k, KP = D.KP, es = 4;
    const int64_t n = A->n, nc = A->nc;
    const int R = round16(2 * m);
    const size_t bXp = align_up((size_t)n * m * 4), bC = align_up((size_t)nc * k * m * 4);
    const size_t bXcm = align_up((size_t)R * D.xk_total * es), bAct = align_up((size_t)nc * R * KP * es);
    int rc = ensure_workspace(A, bXp + 2 * bC + bXcm + 3 * bAct, st);
    if (rc) return rc;
    SyncBufs sb;
    if ((rc = ensure_sync(A, 1, st, &sb))) return rc;
    if ((rc = tc_prepare())) return rc;
    char* base = (char*)A->ws.base;
    fb->Xp = (float*)base;
    fb->Xcm = (uint8_t*)(base + bXp + 2 * bC);
    fb->xcm = fb->Xcm + bXcm;
    fb->ycm = fb->xcm + bAct;
    fb->ycp = fb->ycm + bAct;
    fb->fflag = sb.fflag;
    fb->R = R;
    fb->mc = m;
    return 0;
}

// Before the multi-system launches: X into cluster order and its leaf tiles, the
// ready flags cleared, zero coupling tiles for clusters without couplings.
int flow_pre(h2_matrix* A, const double* X, int64_t ldx, const FlowBufs& fb, cudaStream_t st) {
    const TcData& D = A->tc;
    const int64_t n = A->n, nc = A->nc;
    const int mc = fb.mc, NL = (int)A->leaves.size();
    const int64_t total = n * mc;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_gather<float><<<g, 256, 0, st>>>(X, ldx, A->d_perm, n, mc, fb.Xp);
    H2_LAUNCH_CHECK();
    int rc = launch_pack_act(fb.Xp, mc, NL, nullptr, D.leaf_base, D.leaf_kdim, 0, D.xkoff, 0, mc, fb.R, fb.Xcm, 4, st);
    if (rc) return rc;
    H2_CUDA_TRY(cudaMemsetAsync(fb.fflag, 0, 2 * (size_t)nc * sizeof(int), st));
    return launch_zero_tiles(D.c_zero, D.c_nzero, fb.ycp, (int64_t)D.KP * fb.R * 4, st);
}

// After them: Y += α(Z + σX) in the caller's order (Y = α(Z + σX) with overwrite).
int flow_post(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy, const FlowBufs& fb,
              bool overwrite, cudaStream_t st) {
    const int64_t n = A->n;
    const int mc = fb.mc;
    const int64_t total = n * mc;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_scatter_y<<<g, 256, 0, st>>>(fb.Xp, mc, A->d_perm, n, mc, X, ldx, Y, ldy, alpha, A->sigma, overwrite ? 1 : 0);
    H2_LAUNCH_CHECK();
    return 0;
}

int forward_transform_f64(h2_matrix* A, const double* X, int64_t ldx, int64_t m, double* Xp, double* xhat,
                          cudaStream_t st) {
    if (m <= 0) return 0;
    SyncBufs sb;
    int rc = ensure_sync(A, sync_tiles_for(m), st, &sb);
    if (rc) return rc;
    const int64_t total = A->n * m;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_gather<double><<<g, 256, 0, st>>>(X, ldx, A->d_perm, A->n, (int)m, Xp);
    H2_LAUNCH_CHECK();
    PhaseMarks none(nullptr, st);
    const double* V = (const double*)A->f64.V;
    const double* E = (const double*)A->f64.E;
    const unsigned gzk = (unsigned)((A->k + 63) / 64);
    if (m <= 16) return forward_pass<double, 4, 1>(A, V, E, Xp, xhat, (int)m, (unsigned)((m + 15) / 16), gzk, st, sb, none);
    if (m <= 32) return forward_pass<double, 4, 2>(A, V, E, Xp, xhat, (int)m, (unsigned)((m + 31) / 32), gzk, st, sb, none);
    return forward_pass<double, 4, 4>(A, V, E, Xp, xhat, (int)m, (unsigned)((m + 63) / 64), gzk, st, sb, none);
}

size_t product_scratch_bytes(const h2_matrix* A, int64_t m, int32_t dtype) {
    const size_t elt = dtype == H2_F64 ? sizeof(double) : sizeof(float);
    const int64_t tiles = sync_tiles_for(m);
    return align_up((size_t)A->n * m * elt) + 2 * align_up((size_t)A->nc * A->k * m * elt) +
           align_up((size_t)A->nc * tiles * (sizeof(unsigned) + sizeof(int)) + tiles * sizeof(unsigned));
}

int matmul_in_scratch(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                      int32_t dtype, cudaStream_t st, void* scratch) {
    int rc = check_device_error(A);
    if (rc) return rc;
    const size_t elt = dtype == H2_F64 ? sizeof(double) : sizeof(float);
    const size_t bXp = align_up((size_t)A->n * m * elt);
    const size_t bC = align_up((size_t)A->nc * A->k * m * elt);
    char* base = (char*)scratch;
    // transfer-pass bookkeeping lives in the scratch too; it must start at zero
    const int64_t tiles = sync_tiles_for(m);
    const size_t per = (size_t)A->nc * tiles;
    SyncBufs sb;
    sb.cnt = (unsigned*)(base + bXp + 2 * bC);
    sb.flag = (int*)(sb.cnt + per);
    sb.claim = (unsigned*)(sb.flag + per);
    sb.epoch = 1;
    sb.err = A->err_dev;
    H2_CUDA_TRY(cudaMemsetAsync(sb.cnt, 0, per * (sizeof(unsigned) + sizeof(int)) + tiles * sizeof(unsigned), st));
    if (dtype == H2_F64)
        return dispatch_cn<double>(A, A->f64, alpha, X, ldx, Y, ldy, (int)m, st, false, false, (double*)base,
                                   (double*)(base + bXp), (double*)(base + bXp + bC), sb);
    return dispatch_cn<float>(A, A->f32, alpha, X, ldx, Y, ldy, (int)m, st, false, false, (float*)base,
                              (float*)(base + bXp), (float*)(base + bXp + bC), sb);
}

int matmul(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
           int32_t dtype, cudaStream_t st, bool transposed, const double* alpha_im) {
    if (!A || (!X && m > 0) || (!Y && m > 0)) { set_error("null argument"); return H2_E_BADARG; }
    if (m < 0 || ldx < m || ldy < m || m > (int64_t)1 << 20) { set_error("bad m / leading dimension"); return H2_E_BADARG; }
    if (dtype != H2_F64 && dtype != H2_F32 && dtype != H2_BF16 && dtype != H2_F32_MF) {
        set_error("bad dtype");
        return H2_E_BADARG;
    }
    if (!alpha_im) {
        const int rc = refuse_complex(A, transposed ? "h2_matmul_transposed" : "h2_matmul");
        if (rc) return rc;
    } else if (!A->cplx) {
        set_error("h2_matmul_complex: the matrix has a real kernel");
        return H2_E_UNSUPPORTED;
    }
    if (m == 0) return 0;
    const bool dx = is_device_pointer(X), dy = is_device_pointer(Y);
    if (dx && dy) return matmul_device(A, alpha, X, ldx, Y, ldy, m, dtype, st, transposed, false, alpha_im);
    // Host blocks go through device staging buffers by the copy engines: X in on the
    // call's stream before the product, Y in on a side stream while the product
    // computes (its final pass waits for that copy), Y back out after it.  The call
    // returns when Y is complete on the host.
    // host blocks: stage through device buffers (packed, ld = m)
    const size_t bytes = (size_t)A->n * m * sizeof(double);
    if (A->ws.stage_bytes < bytes) {
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        if (A->ws.stage_x) cudaFree(A->ws.stage_x);
        if (A->ws.stage_y) cudaFree(A->ws.stage_y);
        A->ws.stage_x = A->ws.stage_y = nullptr;
        A->ws.stage_bytes = 0;
        H2_CUDA_TRY(cudaMalloc(&A->ws.stage_x, bytes));
        H2_CUDA_TRY(cudaMalloc(&A->ws.stage_y, bytes));
        A->ws.stage_bytes = bytes;
    }
    Workspace& W = A->ws;
    if (!W.side) {
        H2_CUDA_TRY(cudaStreamCreateWithFlags(&W.side, cudaStreamNonBlocking));
        H2_CUDA_TRY(cudaEventCreateWithFlags(&W.y_in, cudaEventDisableTiming));
        H2_CUDA_TRY(cudaEventCreateWithFlags(&W.st_mark, cudaEventDisableTiming));
    }
    int rc = 0;
    const double* Xd = X;
    int64_t ldxd = ldx;
    if (!dx) {
        H2_CUDA_TRY(cudaMemcpy2DAsync(W.stage_x, m * sizeof(double), X, ldx * sizeof(double), m * sizeof(double), A->n,
                                      cudaMemcpyHostToDevice, st));
        Xd = W.stage_x;
        ldxd = m;
    }
    double* Yd = Y;
    int64_t ldyd = ldy;
    if (!dy) {
        // Y comes in on the side stream while the product computes; its final pass
        // waits for y_in.  The copy starts after the call's earlier work on st (which
        // may still read stage_y).
        H2_CUDA_TRY(cudaEventRecord(W.st_mark, st));
        H2_CUDA_TRY(cudaStreamWaitEvent(W.side, W.st_mark, 0));
        H2_CUDA_TRY(cudaMemcpy2DAsync(W.stage_y, m * sizeof(double), Y, ldy * sizeof(double), m * sizeof(double), A->n,
                                      cudaMemcpyHostToDevice, W.side));
        H2_CUDA_TRY(cudaEventRecord(W.y_in, W.side));
        W.y_wait = true;
        Yd = W.stage_y;
        ldyd = m;
    }
    rc = matmul_device(A, alpha, Xd, ldxd, Yd, ldyd, m, dtype, st, transposed, false, alpha_im);
    if (!rc) rc = wait_y_staged(W, st);  // a path that never reached its final pass
    if (rc) {
        W.y_wait = false;
        return rc;
    }
    if (!dy) {
        H2_CUDA_TRY(cudaMemcpy2DAsync(Y, ldy * sizeof(double), W.stage_y, m * sizeof(double), m * sizeof(double), A->n,
                                      cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return 0;
}

}  // namespace h2
