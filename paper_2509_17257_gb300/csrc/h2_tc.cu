// Tensor-core (tcgen05) kernels of the BF16 and FP32 products: the coupling phase
// (ŷ_t = Σ_{b∈C_t} S_b x̂_s, Sec. 3 Alg. "list_addeval" over the row-cluster
// lists of Alg. "prepare_addeval") and the leaf phase (Y|_t̂ += α(V_t ŷ_t +
// Σ_{b∈L-} G_b X|_ŝ + σ X|_t̂), Alg. "fast_addeval" inadmissible part + the
// backward transformation at the leaves), with the k×m coefficient blocks of
// Sec. 4.
//
// Formulation: every product is computed transposed, Dᵀ = Σ Aᵀ Bᵀ, so that the
// right-hand-side columns are the MMA rows (M) and the matrices (S_b, G_b, V_t)
// are the B operand in their natural row-major orientation:
//   D[r, n] = Σ_k act[r, k] · mat[n, k]
// act rows r = 2i + h hold column i of x̂ / X / ŷ split into a BF16 high part
// (h = 0) and the BF16 rounding remainder (h = 1); the two rows are added in
// the epilogue (adjacent TMEM lanes, one shuffle).  The matrices are stored in
// HBM once, in BF16, already in the tcgen05 "no swizzle, K-major" core-matrix
// order (8 rows × 16 bytes per core matrix, row groups outermost), so one bulk
// copy per tile lands it in shared memory ready for the MMA.
//
// The FP32 product (KIND 1) runs the same schedule on the TF32 units with
// split operands: the activation rows carry x and x - tf32(x), the matrix tiles
// are stored in FP32, and the splitter warps write each tile B together with
// its remainder B_lo = B - tf32(B) into TMEM, so A_hi·B + A_hi·B_lo + A_lo·B +
// A_lo·B_lo keeps FP32 accuracy ("3xTF32", the A_lo·B_lo term comes free with
// the row split).  Its MMA runs the other way round, D[n, r] = Σ_k [B; B_lo][n, k]
// · act[r, k] with M = 128 ([B; B_lo], the A operand in TMEM) and N = R: a
// tcgen05 MMA takes time in proportion to N and the same time for M = 64 as for
// M = 128, so B_lo rides along in M at no cost.
//
// Kernel roles (one persistent CTA per SM; 7 warps for KIND 0, 11 for KIND 1):
//   warp 0          bulk-copy producer (cp.async.bulk + mbarrier complete_tx)
//   warp 1          TMEM owner and MMA issuer (tcgen05.mma kind::f16 or
//                   kind::tf32, FP32 accumulate): KIND 0 all terms, KIND 1 the
//                   even terms; the converged warp runs the loop and elect.sync
//                   issues, which keeps its operands warp-uniform
//   warps 2..5      epilogue (tcgen05.ld, hi+lo combine, stores)
//   warps 6..9      KIND 1 only: the splitter, [B; B_lo] into TMEM
//   last warp       KIND 1: MMA issuer of the odd terms (warp 10); KIND 0: idle
// KIND 1: every term accumulates in its own TMEM buffer (round robin over the
// accumulators), so the epilogue's FP32 sum of earlier terms overlaps the MMAs
// of the next ones and keeps FP32 accuracy.  KIND 0 (BF16): all terms of an
// item accumulate in one buffer, read once per item.  Every wait is bounded; on a timeout the kernel raises an
// error flag, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "h2_async.cuh"
#include "h2_internal.cuh"

namespace h2 {

namespace {

constexpr int kMaxStages = 16;
constexpr int kSmemBudget = 225 * 1024;  // dynamic shared memory per CTA (one CTA per SM)
constexpr int kSplitWarps = 4;  // KIND 1: warps 6..9 write [B; B_lo] into TMEM, one lane quadrant each
constexpr int kASlots = 4;      // KIND 1: TMEM slots of the MMA's A operand (64 columns each, after the accumulators)
// warps: 0 producer, 1 and kIssuer2 MMA issuers (even and odd terms), 2..5
// epilogue, KIND 1: 6..9 splitter
template <int KIND>
__host__ __device__ constexpr int tc_issuer2() { return KIND == 1 ? 6 + kSplitWarps : 6; }
template <int KIND>
__host__ __device__ constexpr int tc_threads() { return 32 * (tc_issuer2<KIND>() + 1); }
constexpr int kAccCols = 64;                // output columns of one term (the matrix tile's rows)
constexpr int kAccBufs = 4;                 // accumulator buffers: MMAs of a term overlap the epilogue of the 3 before
constexpr int kXchBytes = 2 * 64 * 64 * 4;  // TF32 epilogue: remainder sums handed over, two items deep

// Shared-memory matrix descriptor, no swizzle, K-major: LBO = byte distance of
// core matrices adjacent along K, SBO = byte distance of adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor: FP32 accumulate, A and B K-major, BF16 (KIND 0:
// format 1 of kind::f16) or TF32 (KIND 1: format 2 of kind::tf32).
template <int KIND>
__device__ __forceinline__ uint32_t idesc_for(int M, int N) {
    const uint32_t fmt = KIND == 0 ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// One tcgen05.mma (D = A·Bᵀ, or D += A·Bᵀ when acc != 0) from a converged warp:
// elect.sync hands it to the lowest active lane, so every MMA and commit of the
// warp comes from one thread, as tcgen05.commit requires.
template <int KIND>
__device__ __forceinline__ void mma_issue_elect(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (KIND == 0)
        asm volatile(
            "{ .reg .pred p, e; setp.ne.b32 p, %4, 0; elect.sync _|e, 0xffffffff;\n"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{ .reg .pred p, e; setp.ne.b32 p, %4, 0; elect.sync _|e, 0xffffffff;\n"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
}
// The TF32 MMA with its A operand (M = 128 rows, K = 8 columns) in TMEM at
// column address a_tmem, lanes 0..127.
__device__ __forceinline__ void mma_tf32_ta_elect(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                                  uint32_t acc) {
    asm volatile(
        "{ .reg .pred p, e; setp.ne.b32 p, %4, 0; elect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p; }" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit_elect(uint64_t* bar) {
    asm volatile(
        "{ .reg .pred e; elect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0]; }" ::"r"(smem_u32(bar))
        : "memory");
}
// Named barrier over `count` threads that also ORs a predicate across them.
__device__ __forceinline__ bool bar_red_or(int id, int count, bool pred) {
    uint32_t r;
    asm volatile(
        "{ .reg .pred pi, po; setp.ne.u32 pi, %1, 0; bar.red.or.pred po, %2, %3, pi; selp.u32 %0, 1, 0, po; }"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Ready flags of the transfer passes: the writer's generic stores are made
// visible to the bulk copies (async proxy) of other CTAs by a proxy fence and a
// release store; the reader acquires the flag and fences again before copying.
__device__ __forceinline__ int flag_acquire(const int* f) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    return v;
}
__device__ __forceinline__ void flag_release(int* f, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// x - tf32(x) per component: what the TF32 MMA drops from an FP32 operand
// (it reads the top 19 bits).
__device__ __forceinline__ float4 tf32_lo(const float4 v) {
    float4 l;
    l.x = v.x - __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
    l.y = v.y - __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
    l.z = v.z - __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
    l.w = v.w - __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
    return l;
}

// 32 consecutive TMEM columns of this warp's 32 lanes, without waiting: the
// caller issues several and then one tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 64 consecutive TMEM columns of this warp's 32 lanes from registers; the
// caller waits with tmem_wait_st before signalling the MMA.
__device__ __forceinline__ void tmem_st64(uint32_t taddr, const uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,"
        "%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63,%64};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]), "r"(v[32]), "r"(v[33]), "r"(v[34]), "r"(v[35]), "r"(v[36]),
        "r"(v[37]), "r"(v[38]), "r"(v[39]), "r"(v[40]), "r"(v[41]), "r"(v[42]), "r"(v[43]), "r"(v[44]), "r"(v[45]),
        "r"(v[46]), "r"(v[47]), "r"(v[48]), "r"(v[49]), "r"(v[50]), "r"(v[51]), "r"(v[52]), "r"(v[53]), "r"(v[54]),
        "r"(v[55]), "r"(v[56]), "r"(v[57]), "r"(v[58]), "r"(v[59]), "r"(v[60]), "r"(v[61]), "r"(v[62]), "r"(v[63])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }


}  // namespace

// ---------------------------------------------------------------------------
// Packing kernels
// ---------------------------------------------------------------------------

// One tile per CTA: dst (np × kp core-matrix tile, BF16 if es = 2 else FP32)
// ← src (n × k row-major FP64, leading dimension ld), zero padding.  Tile
// offsets are given for BF16 and scaled by es/2.
__global__ void k_pack_tiles(const TcPackTile* __restrict__ tiles, int64_t count, const double* __restrict__ src,
                             uint8_t* __restrict__ dst, int es) {
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const TcPackTile d = tiles[t];
        uint8_t* base = dst + d.dst * (es / 2);
        for (int e = threadIdx.x; e < d.np * d.kp; e += blockDim.x) {
            const int r = e / d.kp, c = e % d.kp;
            double v = (r < d.n && c < d.k)
                           ? src[d.src + ((d.tr & 1) ? (int64_t)c * d.ld + r : (int64_t)r * d.ld + c)]
                           : 0.0;
            if (es == 2) {
                __nv_bfloat16 b = __double2bfloat16(v);
                if (d.tr & 2) b = __double2bfloat16(v - (double)__bfloat162float(b));
                *(__nv_bfloat16*)(base + cm_off(r, c, d.kp, 2)) = b;
            } else {
                *(float*)(base + cm_off(r, c, d.kp, 4)) = (float)v;
            }
        }
    }
}

// Activation tiles: for each id (cluster or leaf), rows r = 2i + h (i < mc)
// hold column i of the FP32 source split into a high part (h = 0) and the
// remainder (h = 1): BF16 (es = 2): bf16(x) and bf16(x - bf16(x)); TF32 (es = 4):
// x itself (the MMA reads tf32(x)) and x - tf32(x).  Columns κ < kdim(id) read
// src[(base(id) + κ) * ld + i]; zero padding to R rows and kp(id) columns;
// kp(id) = kp_fixed, or koff[id+1] - koff[id].  With idmap only the ids
// idmap[0..ids) are packed.
// Threads walk the tile in its memory order, 4 bytes each, so a warp writes one
// whole 128-byte core matrix (8 rows × 16 bytes).
__global__ void k_pack_act(const float* __restrict__ src, int64_t ld, int ids, const int32_t* __restrict__ idmap,
                           const int32_t* __restrict__ base, const int32_t* __restrict__ kdim, int kdim_fixed,
                           const int64_t* __restrict__ koff, int kp_fixed, int mc, int R, uint8_t* __restrict__ dst,
                           int es) {
    const int per = 16 / es;  // elements of one core-matrix row
    for (int j = blockIdx.x; j < ids; j += gridDim.x) {
        const int id = idmap ? idmap[j] : j;
        const int kp = koff ? (int)(koff[id + 1] - koff[id]) : kp_fixed;
        const int64_t tile = (koff ? koff[id] : (int64_t)id * kp_fixed) * (int64_t)R * es;
        const int kd = kdim ? kdim[id] : kdim_fixed;
        const int64_t b = base ? (int64_t)base[id] : (int64_t)id * kdim_fixed;
        const int cgroups = kp / per;
        const int words = R * kp * es / 4;  // 4-byte words of the tile
        uint32_t* out = (uint32_t*)(dst + tile);
        for (int w = threadIdx.x; w < words; w += blockDim.x) {
            const int cmi = w >> 5, within = (w & 31) * 4;  // core matrix, byte inside it
            const int r = (cmi / cgroups) * 8 + (within >> 4);
            const int c0 = (cmi % cgroups) * per + ((within & 15) / es);
            const int i = r >> 1;
            const bool lo = r & 1;
            if (es == 4) {
                float x = 0.f;
                if (i < mc && c0 < kd) x = src[(b + c0) * ld + i];
                const float v = lo ? x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u) : x;
                out[w] = __float_as_uint(v);
            } else {
                uint32_t pk = 0;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int c = c0 + u;
                    float x = 0.f;
                    if (i < mc && c < kd) x = src[(b + c) * ld + i];
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    const __nv_bfloat16 v = lo ? __float2bfloat16_rn(x - __bfloat162float(hi)) : hi;
                    pk |= (uint32_t)__bfloat16_as_ushort(v) << (16 * u);
                }
                out[w] = pk;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The tcgen05 segmented GEMM
// ---------------------------------------------------------------------------
// KIND 0: BF16 operands, one MMA (kind::f16) per 16-wide K step.
// KIND 1: FP32 data on the TF32 units with split operands ("3xTF32"): the
//   activation rows carry x and x - tf32(x); the matrix tile is read once as
//   tf32(S) (the MMA drops the low 13 mantissa bits) and once as the remainder
//   S - tf32(S): the splitter warps write both into TMEM as the MMA's A operand
//   [S; S - tf32(S)], so D = x·tf32(S) + x·(S - tf32(S)) with both parts of x
//   reaches FP32 accuracy.
// Stage layout: [A: R activation rows | B: 64 matrix rows], element size es = 2
// (KIND 0) or 4 (KIND 1), 64 contraction columns at most.
// MODE 0: coupling (outputs ŷ_t); MODE 1: leaf phase (outputs Z); MODE 2 (KIND 1
// only): coupling without the stored S_b, whose rows the splitter warps evaluate
// from the Chebyshev nodes (Eq. (h2_admissible)): only the activation tile is
// copied.  MODE 3 (KIND 1 only): a work list in dependency order whose items
// carry their role (item_role): transfer-pass items (Alg. "forward/backward",
// one per cluster) put their result, split, into the cluster's activation tile
// and release it with a ready flag; coupling items write split tiles; leaf items
// write rows of Z.  A term marked kTermWait waits (bounded) for the ready flag
// of the tile it reads before its copy.  MODE 4 (KIND 1 only): such a list for
// one system, whose role-0 items write rows of ŷ like MODE 0: the coupling
// launch that also computes the clusters above the upward pass's cut (their
// transfer items wait for their sons and release their own tiles).
template <int MODE, int KIND>
__global__ void __launch_bounds__(tc_threads<KIND>(), 1) k_tc_gemm(const TcGemmParams p) {
    constexpr bool MF = MODE == 2;
    constexpr bool FLOW = MODE == 3;
    constexpr bool LIST = MODE == 3 || MODE == 4;  // items carry roles, terms may wait for ready flags
    // the coupling writes its result as split tiles when the downward pass runs on
    // the tensor cores (p.out_act set)
    const bool COUP_SPLIT = (MODE == 0 || MODE == 2) && p.out_act != nullptr;
    constexpr int ES = KIND == 0 ? 2 : 4;
    constexpr int KSTEP = KIND == 0 ? 16 : 8;  // K of one MMA instruction
    constexpr int F_FIRST = 1, F_LAST = 2, F_END = 4;
    // TMEM: KIND 0 has kAccBufs accumulators of 64 columns.  KIND 1 has
    // accumulators of R columns (64 or 128: 4 or 2 of them, 256 columns) and
    // after them kASlots slots of 64 columns for the MMA's A operand [B; B_lo].
    constexpr int TMEM_COLS = KIND == 1 ? 512 : kAccBufs * kAccCols;
    constexpr int A_BASE = 256;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], split_bar[kMaxStages], empty_bar[kMaxStages];
    __shared__ __align__(8) uint64_t accf_bar[kAccBufs], acce_bar[kAccBufs], drain_bar[2], aempty_bar[kASlots];
    __shared__ int s_total;  // terms of this CTA
    __shared__ uint32_t tmem_slot;
    __shared__ int stage_kp[kMaxStages], stage_np[kMaxStages], stage_fl[kMaxStages], stage_R[kMaxStages];
    __shared__ int stage_t[kMaxStages], stage_s[kMaxStages];  // MODE 2: target and source cluster
    __shared__ int abort_shared;
    volatile int& abort_flag = abort_shared;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = p.R;
    const int M = R <= 64 ? 64 : 128;
    const int nst = p.nstages;
    const int a_bytes = p.a_stage_bytes, b_bytes = 64 * 64 * ES;
    const int stage_bytes = a_bytes + b_bytes;
    const int G = gridDim.x;
    const int acc_cols = KIND == 1 ? (R <= 64 ? 64 : 128) : kAccCols;  // TMEM columns of one accumulator
    const int nacc = KIND == 1 ? 256 / acc_cols : kAccBufs;             // accumulator buffers

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&split_bar[s], kSplitWarps);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], 4);  // one arrival per epilogue warp
        }
        mbar_init(&drain_bar[0], 1);
        mbar_init(&drain_bar[1], 1);
        for (int a = 0; a < kASlots; ++a) mbar_init(&aempty_bar[a], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        // the CTA's term count: the two issuers split the terms by parity and stop there
        int tot = 0;
        for (int w = blockIdx.x + lane * G; w < p.n_items; w += 32 * G) tot += p.items[w].e1 - p.items[w].e0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if (lane == 0) s_total = tot;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---------------- producer ----------------
        // Item and term descriptors are packed 16-byte records; the next item's
        // descriptors are loaded while the current item's copies are issued,
        // so no dependent global load sits between two stages.  Stage
        // metadata (contraction length, output width, first/last/end flags)
        // goes to the MMA thread through shared memory, published by the
        // mbarrier arrive.
        int stage = 0;
        uint32_t phase = 0;
        uint32_t pend_mask = 0, pend_par = 0;
        bool aborted = false;
        const uint64_t pol_keep = l2_policy_evict_last(), pol_stream = l2_policy_evict_first();
        // an item's system: its terms, buffers and sizes (PSYS reads a field of the
        // system table of a multi-system launch, else of the launch's own arguments)
#define PSYS(it_, f_) ((FLOW && p.sys) ? p.sys[item_sys(it_)].f_ : p.f_)
        TcItem cur = blockIdx.x < p.n_items ? p.items[blockIdx.x] : TcItem{-1, 0, 0, 0};
        TcTerm tcur{};
        if (cur.id >= 0 && lane < cur.e1 - cur.e0) tcur = PSYS(cur, terms)[cur.e0 + lane];
        for (int w = blockIdx.x; w < p.n_items && !aborted; w += G) {
            aborted = abort_flag != 0;
            const int wn = w + G;
            const TcItem nxt = wn < p.n_items ? p.items[wn] : TcItem{-1, 0, 0, 0};
            const int nterms = cur.e1 - cur.e0;
            const int Ri = PSYS(cur, R);
            for (int base = 0; base < nterms && !aborted; base += 32) {
                TcTerm t = tcur;
                if (base > 0) {
                    t = TcTerm{};
                    if (base + lane < nterms) t = PSYS(cur, terms)[cur.e0 + base + lane];
                }
                const int cnt = min(32, nterms - base);
                // Terms that read a tile of this launch wait for its ready flag.  The
                // lanes poll the flags of the batch's terms together (one round trip
                // for all), and lane 0 issues a term's copies once its bit is set.
                uint32_t ready_mask = 0xffffffffu;
                const int* my_flag = nullptr;
                if (LIST) {
                    if (lane < cnt && (t.asrc & kTermWait)) my_flag = PSYS(cur, flag) + t.akoff / PSYS(cur, KP);
                    ready_mask = __ballot_sync(0xffffffffu, !my_flag || flag_acquire(my_flag) == p.epoch);
                    __syncwarp();
                }
                const uint64_t t_batch = LIST ? global_ns() : 0;
                for (int j = 0; j < cnt; ++j) {
                    const int kpj = __shfl_sync(0xffffffffu, (int)t.kp, j);
                    const int asj = __shfl_sync(0xffffffffu, (int)t.asrc, j);
                    const int64_t bj = __shfl_sync(0xffffffffu, t.boff, j);
                    const int akj = __shfl_sync(0xffffffffu, t.akoff, j);
                    const int64_t aj = (int64_t)akj * Ri * ES;
                    bool ready = true;
                    if (LIST && !((ready_mask >> j) & 1u)) {
                        // poll again (bounded: gives up after about one second)
                        while (true) {
                            __nanosleep(32);
                            ready_mask |= __ballot_sync(0xffffffffu, my_flag && flag_acquire(my_flag) == p.epoch);
                            __syncwarp();
                            if ((ready_mask >> j) & 1u) break;
                            if (__any_sync(0xffffffffu, abort_flag || global_ns() - t_batch > 1000000000ull)) {
                                ready = false;  // warp-uniform: every lane leaves together
                                break;
                            }
                        }
                    }
                    int bad = 0;
                    if (lane == 0) {
                        // the flags acquired by the warp order the tiles' writes before this copy
                        if (LIST && (asj & kTermWait)) fence_proxy_async_global();
                        if (!ready || !mbar_wait(&empty_bar[stage], phase ^ 1)) {
                            bad = 1;
                        } else {
                            const uint32_t ab = (uint32_t)(Ri * kpj * ES);
                            const uint32_t bb = (uint32_t)(item_np(cur) * kpj * ES);
                            uint8_t* sA = smem + stage * stage_bytes;
                            uint8_t* sB = sA + a_bytes;
                            stage_kp[stage] = kpj;
                            stage_np[stage] = item_np(cur);
                            stage_R[stage] = Ri;
                            stage_fl[stage] = (base + j == 0 ? F_FIRST : 0) | (base + j == nterms - 1 ? F_LAST : 0);
                            if (MF) {
                                // the source cluster: the activation rows of cluster s start at s·KP
                                stage_t[stage] = cur.id;
                                stage_s[stage] = (int)(aj / ((int64_t)R * ES) / p.KP);
                                mbar_expect_tx(&full_bar[stage], ab);
                                bulk_g2s(sA, (asj ? p.act1 : p.act0) + aj, ab, &full_bar[stage]);
                            } else {
                                mbar_expect_tx(&full_bar[stage], ab + bb);
                                const uint8_t* asrc = (asj & 3) == 0 ? PSYS(cur, act0)
                                                                     : ((asj & 3) == 1 ? PSYS(cur, act1) : PSYS(cur, act2));
                                // the activation tiles are read by many terms, the matrix tiles once
                                bulk_g2s_hint(sA, asrc + aj, ab, &full_bar[stage], pol_keep);
                                bulk_g2s_hint(sB, PSYS(cur, bmat) + bj * (ES / 2), bb, &full_bar[stage], pol_stream);
                            }
                            pend_mask |= 1u << stage;
                            pend_par = (pend_par & ~(1u << stage)) | (phase << stage);
                        }
                    }
                    if (__shfl_sync(0xffffffffu, bad, 0)) {
                        if (lane == 0) atomicExch(p.err, 1);
                        abort_flag = 1;
                        aborted = true;
                        break;
                    }
                    if (++stage == nst) { stage = 0; phase ^= 1; }
                }
            }
            tcur = TcTerm{};
            if (nxt.id >= 0 && lane < nxt.e1 - nxt.e0) tcur = PSYS(nxt, terms)[nxt.e0 + lane];
            cur = nxt;
        }
        if (lane == 0) {
            // end marker for the MMA thread (and the splitters): a stage without data
            if (mbar_wait(&empty_bar[stage], phase ^ 1)) {
                // the stage is free, so its earlier copy has landed and been consumed;
                // the marker moves its barrier on, so it leaves the drain set
                pend_mask &= ~(1u << stage);
                stage_fl[stage] = F_END;
                mbar_arrive(&full_bar[stage]);
            } else {
                atomicExch(p.err, 1);
                abort_flag = 1;
            }
            // every copy issued by this CTA lands before the CTA exits
            for (int s2 = 0; s2 < nst; ++s2)
                if ((pend_mask >> s2) & 1u)
                    if (!mbar_wait(&full_bar[s2], (pend_par >> s2) & 1u)) atomicExch(p.err, 2);
        }
#undef PSYS
    } else if (warp == 1 || warp == tc_issuer2<KIND>()) {
        // ---------------- MMA issuers: driven by the stage metadata ----------------
        // Two warps take the terms by parity (term t uses stage t mod nst,
        // accumulator t mod nacc and A slot t mod kASlots), so one warp's waits
        // overlap the other's MMAs.  Each reuse of a stage, slot or accumulator
        // waits for the consumer of its previous use, so every barrier's
        // arrivals come in order whichever issuer commits them.  Each converged warp runs its loop (waits and descriptors are
        // warp-uniform); elect.sync hands each MMA and commit to one lane.
        const int j = warp == 1 ? 0 : 1;
        const int T = s_total;
        bool issued = false;
        if (KIND == 0 && j == 0) {
            // BF16: one issuer takes every term in order and accumulates all terms of
            // an item in one TMEM accumulator (an item's first term starts it from
            // zero); the epilogue reads each accumulator once per item.  The FP32
            // accumulation of the tensor cores is far finer than the BF16 operands.
            int item_idx = 0, acc = 0;
            for (int it = 0; it < T; ++it) {
                const int stage = it % nst;
                const uint32_t phase = (uint32_t)(it / nst) & 1u;
                if (!__any_sync(0xffffffffu, mbar_wait(&full_bar[stage], phase))) {
                    abort_flag = 1;
                    if (lane == 0) atomicExch(p.err, 4);
                    break;
                }
                const int fl = stage_fl[stage];
                if (fl & F_FIRST) {
                    acc = item_idx % kAccBufs;
                    if (!__any_sync(0xffffffffu, mbar_wait(&acce_bar[acc], ((item_idx / kAccBufs) & 1) ^ 1))) {
                        abort_flag = 1;
                        if (lane == 0) atomicExch(p.err, 3);
                        break;
                    }
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * acc_cols);
                const int kp = stage_kp[stage];
                const uint32_t sA = smem_u32(smem + stage * stage_bytes);
                const uint32_t sB = sA + a_bytes;
                const uint32_t sbo = (uint32_t)(kp * ES / 16) * 128;
                const uint32_t idesc = idesc_for<KIND>(M, stage_np[stage]);
                const uint64_t ad0 = smem_desc(sA, 128, sbo);
                const uint64_t bd0 = smem_desc(sB, 128, sbo);
                const int nk = kp / KSTEP;
#pragma unroll
                for (int kk = 0; kk < 64 / KSTEP; ++kk) {
                    if (kk >= nk) break;
                    const uint64_t off = (uint64_t)(kk * 16);
                    mma_issue_elect<KIND>(d, ad0 + off, bd0 + off, idesc, (kk == 0 && (fl & F_FIRST)) ? 0u : 1u);
                }
                issued = true;
                mma_commit_elect(&empty_bar[stage]);
                if (fl & F_LAST) {
                    mma_commit_elect(&accf_bar[acc]);
                    ++item_idx;
                }
            }
            if (issued) {
                mma_commit_elect(&drain_bar[0]);
                if (!__any_sync(0xffffffffu, mbar_wait(&drain_bar[0], 0)) && lane == 0) atomicExch(p.err, 5);
                issued = false;  // drained
            }
        }
        for (int it = j; it < T && KIND == 1; it += 2) {
            const int stage = it % nst;
            const uint32_t phase = (uint32_t)(it / nst) & 1u;
            if (!__any_sync(0xffffffffu, mbar_wait(KIND == 1 ? &split_bar[stage] : &full_bar[stage], phase))) {
                abort_flag = 1;
                if (lane == 0) atomicExch(p.err, 4);
                break;
            }
            // every term accumulates from zero in its own TMEM buffer; the epilogue
            // adds the terms of an item in FP32 registers (round to nearest), so
            // the tensor-core accumulator never sums more than one term's K steps
            const int acc = it % nacc;
            if (!__any_sync(0xffffffffu, mbar_wait(&acce_bar[acc], ((it / nacc) & 1) ^ 1))) {
                abort_flag = 1;
                if (lane == 0) atomicExch(p.err, 3);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(acc * acc_cols);
            const int kp = stage_kp[stage];
            const uint32_t sA = smem_u32(smem + stage * stage_bytes);
            const uint32_t sB = sA + a_bytes;
            const uint32_t sbo = (uint32_t)(kp * ES / 16) * 128;
            // KIND 0: D[r, n] = act · matᵀ (M = activation rows, N = the tile's rows),
            // both operands in shared memory.
            // KIND 1: D[n, r] = [mat; mat_lo] · actᵀ: M = 128, the tile (rows 0..63)
            // and its TF32 remainder (rows 64..127), which the splitter warps have
            // put into TMEM slot `as`; N = R activation rows from shared memory.
            // The MMA time grows with N, not with M up to 128, so the remainder
            // costs no extra instructions.  Rows np..63 of either part hold stale
            // data whose TMEM lanes the epilogue ignores.
            const uint32_t idesc = KIND == 1 ? idesc_for<KIND>(128, stage_R[stage]) : idesc_for<KIND>(M, stage_np[stage]);
            // descriptors of K step kk: the start address field moves by 256 bytes
            // (two core matrices along K), i.e. 16 in its 16-byte units; a TMEM
            // operand moves by KSTEP columns
            const uint64_t ad0 = smem_desc(sA, 128, sbo);
            const uint64_t bd0 = smem_desc(sB, 128, sbo);
            const int as = it % kASlots;
            const uint32_t a_tmem = tmem + (uint32_t)(A_BASE + 64 * as);
            const int nk = kp / KSTEP;
#pragma unroll
            for (int kk = 0; kk < 64 / KSTEP; ++kk) {
                if (kk >= nk) break;
                const uint64_t off = (uint64_t)(kk * 16);
                if (KIND == 1) mma_tf32_ta_elect(d, a_tmem + (uint32_t)(kk * KSTEP), ad0 + off, idesc, kk == 0 ? 0u : 1u);
                else mma_issue_elect<KIND>(d, ad0 + off, bd0 + off, idesc, kk == 0 ? 0u : 1u);
            }
            issued = true;
            mma_commit_elect(&empty_bar[stage]);
            if (KIND == 1) mma_commit_elect(&aempty_bar[as]);
            mma_commit_elect(&accf_bar[acc]);
        }
        if (issued) {
            mma_commit_elect(&drain_bar[j]);
            if (!__any_sync(0xffffffffu, mbar_wait(&drain_bar[j], 0)) && lane == 0) atomicExch(p.err, 5);
        }
    } else if (warp < 6 && KIND == 1) {
        // ---------------- epilogue, KIND 1 (warps 2..5, TMEM lane quadrant warp % 4) ----------------
        // TMEM lane 32q + lane holds row n = 32(q & 1) + lane of the tile (q = 0, 1)
        // or of its remainder (q = 2, 3); column r = 2i + h of that lane is the
        // product with the high (h = 0) or low (h = 1) part of right-hand-side
        // column i.  Each thread adds its two columns per i over the item's terms;
        // at the item's end the remainder warps hand their sums to the tile warps
        // through shared memory (double buffered by item parity, one barrier per
        // item), which add them and store row n.
        const int q = warp & 3;
        const int n = 32 * (q & 1) + lane;
        const bool lo_part = q >= 2;
        float* xch = reinterpret_cast<float*>(smem + nst * stage_bytes);  // [2][64 i][64 n]
        int it = 0, par = 0;
        // rows of Z: the leaf phase, and the leaf items of a transfer-pass launch
        auto leaf_rows = [&](const TcItem& t) { return MODE == 1 || (LIST && item_role(t) == kRoleLeaf); };
        TcItem cur = blockIdx.x < p.n_items ? p.items[blockIdx.x] : TcItem{-1, 0, 0, 0};
        // an item's system: its sizes and buffers (SYSF reads a field of the system
        // table of a multi-system launch, else of the launch's own arguments)
#define SYSF(it_, f_) ((FLOW && p.sys) ? p.sys[item_sys(it_)].f_ : p.f_)
        int cur_off = 0, cur_nt = 0;
        if (cur.id >= 0 && leaf_rows(cur)) {
            const int t = SYSF(cur, leaves)[cur.id];
            cur_off = SYSF(cur, cl_off)[t];
            cur_nt = SYSF(cur, cl_size)[t];
        }
        for (int w = blockIdx.x; w < p.n_items; w += G) {
            const TcItem nxt = w + G < p.n_items ? p.items[w + G] : TcItem{-1, 0, 0, 0};
            int nxt_off = 0, nxt_nt = 0;
            if (nxt.id >= 0 && leaf_rows(nxt)) {
                const int t = SYSF(nxt, leaves)[nxt.id];
                nxt_off = SYSF(nxt, cl_off)[t];
                nxt_nt = SYSF(nxt, cl_size)[t];
            }
            const int id = cur.id, np = item_np(cur), nterms = cur.e1 - cur.e0;
            const int Ri = SYSF(cur, R), mci = SYSF(cur, mc), ki = SYSF(cur, k), KPi = SYSF(cur, KP),
                      ldci = SYSF(cur, ldc);
            const bool wide = Ri > 64;
            const bool vec4 = (mci & 3) == 0 && (ldci & 3) == 0;
            const int role = LIST ? item_role(cur) : 0;
            // role 0 (MODE 4's coupling items): rows of ŷ, as in MODE 0
            const bool split_out = COUP_SPLIT || (LIST && role != kRoleLeaf && role != 0);
            float sum[kAccCols];
#pragma unroll
            for (int j = 0; j < kAccCols; ++j) sum[j] = 0.f;
            bool failed = false;
            uint32_t imask = 0;  // complex product: bit t of the batch of 32 terms applies i·act
            for (int term = 0; term < nterms; ++term, ++it) {
                if (!FLOW && p.cplx && (term & 31) == 0) {
                    const int tt = term + lane;
                    imask = __ballot_sync(0xffffffffu, tt < nterms && (p.terms[cur.e0 + tt].asrc & kTermImag));
                }
                const bool imag = (imask >> (term & 31)) & 1u;
                const int acc = it % nacc;
                if (!__any_sync(0xffffffffu, mbar_wait(&accf_bar[acc], (it / nacc) & 1))) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * acc_cols);
                if constexpr (FLOW) {
                    // 32 columns per read (16 right-hand-side columns; R > 64 takes four):
                    // one register buffer, which the multi-system bookkeeping needs room for
                    uint32_t r0[32];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        if (h >= 2 && !wide) break;
                        tmem_ld32_async(ta + 32 * h, r0);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            sum[16 * h + j] += __uint_as_float(r0[2 * j]) + __uint_as_float(r0[2 * j + 1]);
                    }
                } else {
                    // 64 columns per read (two loads in flight, one wait); R > 64 takes two
                    uint32_t r0[32], r1[32];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h == 1 && !wide) break;
                        tmem_ld32_async(ta + 64 * h, r0);
                        tmem_ld32_async(ta + 64 * h + 32, r1);
                        tmem_wait_ld();
                        if (!imag) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                sum[32 * h + j] += __uint_as_float(r0[2 * j]) + __uint_as_float(r0[2 * j + 1]);
                                sum[32 * h + 16 + j] += __uint_as_float(r1[2 * j]) + __uint_as_float(r1[2 * j + 1]);
                            }
                        } else {
                            // i·act: column 2j takes -(column 2j + 1), column 2j + 1 takes column 2j
#pragma unroll
                            for (int j = 0; j < 16; j += 2) {
                                const float a0 = __uint_as_float(r0[2 * j]) + __uint_as_float(r0[2 * j + 1]);
                                const float a1 = __uint_as_float(r0[2 * j + 2]) + __uint_as_float(r0[2 * j + 3]);
                                const float b0 = __uint_as_float(r1[2 * j]) + __uint_as_float(r1[2 * j + 1]);
                                const float b1 = __uint_as_float(r1[2 * j + 2]) + __uint_as_float(r1[2 * j + 3]);
                                sum[32 * h + j] -= a1;
                                sum[32 * h + j + 1] += a0;
                                sum[32 * h + 16 + j] -= b1;
                                sum[32 * h + 16 + j + 1] += b0;
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce_bar[acc]);
            }
            float* xb = xch + par * (64 * 64);
            if (lo_part && !failed) {
#pragma unroll
                for (int i = 0; i < kAccCols; ++i)
                    if (i < mci) xb[i * 64 + n] = sum[i];
            }
            // every epilogue warp reaches this barrier once per item, failed or not,
            // and all of them learn whether any failed
            if (bar_red_or(1, 128, failed)) {
                if (lane == 0) atomicExch(p.err, 6);
                abort_flag = 1;
                break;
            }
            if (!lo_part && split_out) {
#pragma unroll
                for (int i = 0; i < kAccCols; ++i)
                    if (i < mci) sum[i] += xb[i * 64 + n];
                // The result goes, split as the activations are (rows 2i: x; 2i + 1: x -
                // tf32(x); zero past the columns and past column k), into the cluster's
                // tile: staged in this item's exchange buffer (free once both tile warps
                // have read it) and stored by one bulk copy per 64 rows.
                asm volatile("bar.sync 4, 64;" ::: "memory");
                uint8_t* gtile = (role == kRoleCoupling ? SYSF(cur, out_act2) : SYSF(cur, out_act)) + (int64_t)id * KPi * Ri * 4;
                const bool nv = n < ki;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int h0 = 64 * hh;
                    if (h0 >= Ri) break;
                    const int rows = min(64, Ri - h0);
                    if (h0 > 0) asm volatile("bar.sync 4, 64;" ::: "memory");  // the last store read the buffer
                    if (n < KPi) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            if (2 * i >= rows) break;
                            const int ii = 32 * hh + i;
                            const float v = (nv && ii < mci) ? sum[ii] : 0.f;
                            const float lo = v - __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
                            *(float*)((uint8_t*)xb + cm_off(2 * i, n, KPi, 4)) = v;
                            *(float*)((uint8_t*)xb + cm_off(2 * i + 1, n, KPi, 4)) = lo;
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("bar.sync 4, 64;" ::: "memory");
                    if (q == 0 && lane == 0) {
                        const uint32_t bytes = (uint32_t)(rows * KPi * 4);
                        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                                         gtile + (int64_t)h0 * KPi * 4),
                                     "r"(smem_u32(xb)), "r"(bytes)
                                     : "memory");
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
                    }
                }
                // the tile is in global memory: release it to the CTAs that wait for it
                if (LIST && role == kRoleTransfer && q == 0 && lane == 0) {
                    fence_proxy_async_global();
                    flag_release(SYSF(cur, flag) + id, p.epoch);
                }
            } else if (!lo_part) {
#pragma unroll
                for (int i = 0; i < kAccCols; ++i)
                    if (i < mci) sum[i] += xb[i * 64 + n];
                float* out = nullptr;
                if (!leaf_rows(cur)) {
                    if (n < np && n < ki) out = p.yhat + ((int64_t)id * ki + n) * ldci;
                } else {
                    // Z in cluster order; the scatter into Y (with α, σX) is a separate
                    // coalesced pass, so the epilogue only stores
                    if (n < cur_nt) out = SYSF(cur, zp) + ((int64_t)cur_off + n) * ldci;
                }
                if (out) {
                    if (vec4) {
#pragma unroll
                        for (int i = 0; i < kAccCols; i += 4)
                            if (i < mci)
                                *reinterpret_cast<float4*>(out + i) = make_float4(sum[i], sum[i + 1], sum[i + 2], sum[i + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < kAccCols; ++i)
                            if (i < mci) out[i] = sum[i];
                    }
                }
            }
            par ^= 1;
            cur = nxt;
            cur_off = nxt_off;
            cur_nt = nxt_nt;
        }
#undef SYSF
    } else if (warp < 6) {
        // ---------------- epilogue, KIND 0 (warps 2..5, TMEM lane quadrant warp % 4) ----------------
        const int q = warp & 3;
        int row;
        if (M == 128) row = 32 * q + lane;
        else row = lane < 16 ? 16 * q + lane : -1;
        const int i = row >> 1;
        const bool writer = row >= 0 && !(row & 1) && i < p.mc;
        int it = 0;
        TcItem cur = blockIdx.x < p.n_items ? p.items[blockIdx.x] : TcItem{-1, 0, 0, 0};
        int cur_off = 0, cur_nt = 0;
        if (MODE == 1 && cur.id >= 0) {
            const int t = p.leaves[cur.id];
            cur_off = p.cl_off[t];
            cur_nt = p.cl_size[t];
        }
        for (int w = blockIdx.x; w < p.n_items; w += G) {
            // the next item's descriptor (and leaf extent) load while this one waits
            const TcItem nxt = w + G < p.n_items ? p.items[w + G] : TcItem{-1, 0, 0, 0};
            int nxt_off = 0, nxt_nt = 0;
            if (MODE == 1 && nxt.id >= 0) {
                const int t = p.leaves[nxt.id];
                nxt_off = p.cl_off[t];
                nxt_nt = p.cl_size[t];
            }
            const int id = cur.id, np = item_np(cur);
            float sum[kAccCols];
#pragma unroll
            for (int j = 0; j < kAccCols; ++j) sum[j] = 0.f;
            bool failed = false;
            {
                // the item's terms accumulate in one accumulator (`it` counts items)
                const int acc = it % kAccBufs;
                // warp-uniform wait: a completed phase stays completed, so any lane's
                // success is the warp's success
                const bool ok = __any_sync(0xffffffffu, mbar_wait(&accf_bar[acc], (it / kAccBufs) & 1));
                ++it;
                if (!ok) {
                    failed = true;
                }
            }
            if (!failed) {
                const int acc = (it - 1) % kAccBufs;
                tc_fence_after();
                // both halves of the accumulator in flight, one wait; the row pair
                // (2i, 2i + 1) is adjacent lanes, added by one shuffle
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * acc_cols);
                uint32_t r0[32], r1[32];
                tmem_ld32_async(ta, r0);
                if (np > 32) tmem_ld32_async(ta + 32, r1);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float v = __uint_as_float(r0[j]);
                    sum[j] += v + __shfl_xor_sync(0xffffffffu, v, 1);
                }
                if (np > 32) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float v = __uint_as_float(r1[j]);
                        sum[32 + j] += v + __shfl_xor_sync(0xffffffffu, v, 1);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce_bar[acc]);
            }
            if (LIST && item_role(cur) == kRoleTransfer) {
                // A transfer item of the hybrid upward pass: x̂ of the cluster as a
                // split BF16 tile (row 2i: bf16(v), row 2i + 1: bf16(v - bf16(v)); zero
                // for columns i >= mc and past row k), stored by the even-row threads, ordered for the bulk copies of other
                // CTAs by a proxy fence, and released by the ready flag once all four
                // warps have stored.  Every epilogue warp meets the barrier once per
                // transfer item, failed or not, and all of them learn of a failure.
                if (bar_red_or(1, 128, failed)) {
                    if (lane == 0) atomicExch(p.err, 6);
                    abort_flag = 1;
                    break;
                }
                if (row >= 0 && !(row & 1) && i < R / 2) {
                    uint8_t* gt = p.out_act + (int64_t)id * p.KP * R * 2;
                    const bool live = i < p.mc;
#pragma unroll
                    for (int u = 0; u < kAccCols / 8; ++u) {
                        if (8 * u >= p.KP) break;
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float v0 = live && 8 * u + 2 * e < p.k ? sum[8 * u + 2 * e] : 0.f;
                            const float v1 = live && 8 * u + 2 * e + 1 < p.k ? sum[8 * u + 2 * e + 1] : 0.f;
                            const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
                            const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
                            const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
                            hw[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                            lw[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                        }
                        *(uint4*)(gt + cm_off(2 * i, 8 * u, p.KP, 2)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *(uint4*)(gt + cm_off(2 * i + 1, 8 * u, p.KP, 2)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                    fence_proxy_async_global();
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (warp == 2 && lane == 0) {
                    __threadfence();
                    flag_release(p.flag + id, p.epoch);
                }
            } else if (failed) {
                if (lane == 0) atomicExch(p.err, 6);
                abort_flag = 1;
                break;
            } else if (writer) {
                if (MODE != 1) {
                    float* out = p.yhat + (int64_t)id * p.k * p.ldc;
#pragma unroll
                    for (int j = 0; j < kAccCols; ++j)
                        if (j < np && j < p.k) out[(int64_t)j * p.ldc + i] = sum[j];
                } else {
                    // Z in cluster order; the scatter into Y (with α, σX) is a separate
                    // coalesced pass, so the epilogue only stores
                    float* z = p.zp + (int64_t)cur_off * p.ldc + i;
#pragma unroll
                    for (int j = 0; j < kAccCols; ++j)
                        if (j < cur_nt) z[(int64_t)j * p.ldc] = sum[j];
                }
            }
            cur = nxt;
            cur_off = nxt_off;
            cur_nt = nxt_nt;
        }
    } else if (KIND == 1 && warp < 6 + kSplitWarps) {
        // ---------------- splitter (warps 6..9): [B; B_lo] into TMEM ----------------
        // Warp w owns TMEM lanes 32q..32q+31 (q = w mod 4): row n = 32(q & 1) + lane
        // of the tile B (q = 0, 1) or of its remainder B_lo = B - tf32(B) (q = 2, 3).
        // Each thread reads its row (kp values, 16 bytes per core matrix) from the
        // stage and writes it to TMEM slot `as` of the MMA's A operand.
        const int q = warp & 3;
        const int n = 32 * (q & 1) + lane;
        const bool lo_part = q >= 2;
        // The splitter is the one serial stage of the pipeline, so it tests the next
        // term's barriers while it works on the current one: a phase seen complete
        // then costs no wait at the top of the next iteration.
        int stage = 0, sit = 0;
        uint32_t phase = 0;
        bool pre = false;  // the next iteration's stage and A-slot phases were seen complete
        while (true) {
            bool ok = pre || __any_sync(0xffffffffu, mbar_wait(&full_bar[stage], phase));
            const int fl = ok ? stage_fl[stage] : 0;
            const bool end = ok && (fl & F_END);
            const int as = sit % kASlots;
            // the slot is free once the MMAs of term sit - kASlots have completed
            if (ok && !end && !pre) ok = __any_sync(0xffffffffu, mbar_wait(&aempty_bar[as], ((sit / kASlots) & 1) ^ 1));
            pre = false;
            if (ok && !end) tc_fence_after();
            const int kp = ok ? stage_kp[stage] : 0;
            float* xbuf = (float*)(smem + stage * stage_bytes + a_bytes);  // MODE 2: [64 μ][64 rows]
            if (MF) {
                // row n of S_b: g(ξ_{t,n}, ξ_{s,μ}) = exp(-|ξ_{t,n} - ξ_{s,μ}| / length) for
                // n, μ < k, zero in the padding.  The tile warp (q < 2) and the remainder
                // warp (q + 2) of the same rows each evaluate half of the columns and
                // swap halves through the stage's (unused) matrix region.  The exponential
                // is 2^(-r·log2(e)/length) with r = d²·rsqrt(d²) (hardware approximations,
                // relative error below 1e-6).
                if (ok && !end) {
                    const bool rv = n < p.k;
                    const float4 xt = p.nodes[(int64_t)stage_t[stage] * p.KP + (rv ? n : 0)];
                    const int mu0 = lo_part ? 32 : 0;
                    // the warp's 32 source nodes: one coalesced load (lane l holds node
                    // mu0 + l), handed to every lane by shuffles
                    const float4 ys = mu0 + lane < p.KP ? p.nodes[(int64_t)stage_s[stage] * p.KP + mu0 + lane]
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float sc = -p.inv_len * 1.4426950408889634f;
#pragma unroll 8
                    for (int j = 0; j < 32; ++j) {
                        const int mu = mu0 + j;
                        const float y0 = __shfl_sync(0xffffffffu, ys.x, j), y1 = __shfl_sync(0xffffffffu, ys.y, j),
                                    y2 = __shfl_sync(0xffffffffu, ys.z, j);
                        float g = 0.f;
                        if (rv && mu < p.k) {
                            const float d0 = xt.x - y0, d1 = xt.y - y1, d2 = xt.z - y2;
                            const float r2 = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
                            const float e = r2 * rsqrtf(r2) * sc;
                            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(e));
                        }
                        xbuf[mu * 64 + n] = g;
                    }
                }
                // the pair (quadrants q and q ^ 2, named barrier 2 or 3) meets once per
                // stage, end marker and failures included, and both learn whether to stop
                if (bar_red_or(2 + (q & 1), 64, !ok)) {
                    if (lane == 0) atomicExch(p.err, 8);
                    abort_flag = 1;
                    break;
                }
            } else if (!ok) {
                if (lane == 0) atomicExch(p.err, 7);
                abort_flag = 1;
                break;
            }
            if (!end) {
                const int nstage = stage + 1 == nst ? 0 : stage + 1;
                const uint32_t nphase = stage + 1 == nst ? phase ^ 1u : phase;
                const bool pf = mbar_test(&full_bar[nstage], nphase);
                const bool pa = mbar_test(&aempty_bar[(sit + 1) % kASlots], (((sit + 1) / kASlots) & 1) ^ 1);
                uint32_t v[64];
                if (MF) {
#pragma unroll
                    for (int mu = 0; mu < 64; ++mu) {
                        float g = mu < kp ? xbuf[mu * 64 + n] : 0.f;
                        if (lo_part) g -= __uint_as_float(__float_as_uint(g) & 0xFFFFE000u);
                        v[mu] = __float_as_uint(g);
                    }
                } else {
                    const uint8_t* row =
                        smem + stage * stage_bytes + a_bytes + (n >> 3) * (kp >> 2) * 128 + (n & 7) * 16;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (4 * c < kp) x = *(const float4*)(row + c * 128);
                        if (lo_part) x = tf32_lo(x);
                        v[4 * c] = __float_as_uint(x.x);
                        v[4 * c + 1] = __float_as_uint(x.y);
                        v[4 * c + 2] = __float_as_uint(x.z);
                        v[4 * c + 3] = __float_as_uint(x.w);
                    }
                }
                tmem_st64(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(A_BASE + 64 * as), v);
                tmem_wait_st();
                tc_fence_before();
                ++sit;
                pre = __all_sync(0xffffffffu, pf && pa);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&split_bar[stage]);
            if (fl & F_END) break;
            if (++stage == nst) { stage = 0; phase ^= 1; }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Zero ŷ of clusters whose coupling list is empty.
__global__ void k_zero_clusters(const int32_t* __restrict__ ids, int count, float* __restrict__ yhat, int k, int ldc,
                                int mc) {
    for (int c = blockIdx.x; c < count; c += gridDim.x) {
        float* y = yhat + (int64_t)ids[c] * k * ldc;
        for (int e = threadIdx.x; e < k * mc; e += blockDim.x) y[(int64_t)(e / mc) * ldc + e % mc] = 0.f;
    }
}

// Zero the activation tiles (bytes each, a multiple of 16) of the clusters ids[0..count).
__global__ void k_zero_tiles(const int32_t* __restrict__ ids, int count, uint8_t* __restrict__ buf, int64_t bytes) {
    for (int c = blockIdx.x; c < count; c += gridDim.x) {
        uint4* t = reinterpret_cast<uint4*>(buf + (int64_t)ids[c] * bytes);
        for (int64_t e = threadIdx.x; e < bytes / 16; e += blockDim.x) t[e] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Stage geometry for R activation rows and element size es: A holds R rows,
// B 64 rows, both with up to 64 contraction columns.  The TF32 kernel keeps
// its epilogue exchange tile (kXchBytes) after the stages (its B_lo lives in
// TMEM).
void tc_stage_geometry(int R, int es, int* a_bytes, int* stage_bytes, int* nstages) {
    const int rows = R <= 64 ? 64 : 128;  // the BF16 MMA reads M = 64 or 128 activation rows
    *a_bytes = rows * 64 * es;
    *stage_bytes = *a_bytes + 64 * 64 * es;
    *nstages = std::min(kMaxStages, (kSmemBudget - 1024 - (es == 4 ? kXchBytes : 0)) / *stage_bytes);
}

template <int MODE, int KIND>
int launch_one(const TcGemmParams& p, int grid, int smem, cudaStream_t st) {
    k_tc_gemm<MODE, KIND><<<grid, tc_threads<KIND>(), smem, st>>>(p);
    H2_LAUNCH_CHECK();
    return 0;
}

// Set the shared-memory attribute of every tensor-core kernel instance up
// front (needed before a product is captured into a CUDA graph).
namespace {
int g_tc_attr_device = -1;  // device whose kernel attributes are set
}

int tc_prepare() {
    int dev = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    if (dev == g_tc_attr_device) return 0;
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    H2_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    g_tc_attr_device = dev;
    return 0;
}

int launch_tc_gemm(int mode, int kind, TcGemmParams p, int grid, cudaStream_t st, int stages) {
    int a_bytes, stage_bytes, nstages;
    tc_stage_geometry(p.R, kind == 0 ? 2 : 4, &a_bytes, &stage_bytes, &nstages);
    // a tuned stage count (h2_autotune) below the number that fits
    if (stages >= 2 && stages < nstages) nstages = stages;
    // A parity wait is exact only while its waiter cannot get two uses of a stage
    // ahead (the protocol model in tests/test_pipeline_protocol.py checks this).
    // The FP32 issuers wait on the in-order splitter, which keeps them in step;
    // the BF16 kernel has one issuer, which waits on every stage in order.
    if (nstages < 2) { set_error("tensor-core stage does not fit in shared memory"); return H2_E_UNSUPPORTED; }
    p.a_stage_bytes = a_bytes;
    p.nstages = nstages;
    int rc = tc_prepare();
    if (rc) return rc;
    const int smem = nstages * stage_bytes + (kind == 1 ? kXchBytes : 0) + 1024;
    if (mode == 2) {
        if (kind != 1) { set_error("matrix-free coupling runs on the TF32 path only"); return H2_E_UNSUPPORTED; }
        return launch_one<2, 1>(p, grid, smem, st);
    }
    if (mode == 3) {
        if (kind != 1) { set_error("the tensor-core transfer passes run on the TF32 path only"); return H2_E_UNSUPPORTED; }
        // its CTAs wait on each other's ready flags: one CTA per SM, at most one per SM
        // of the device, so that every CTA is resident (the waits are bounded in any case)
        return launch_one<3, 1>(p, grid, smem, st);
    }
    // waits on flags too: one CTA per SM, every CTA resident
    if (mode == 4) return kind == 1 ? launch_one<4, 1>(p, grid, smem, st) : launch_one<4, 0>(p, grid, smem, st);
    if (mode == 0 && kind == 0) return launch_one<0, 0>(p, grid, smem, st);
    if (mode == 1 && kind == 0) return launch_one<1, 0>(p, grid, smem, st);
    if (mode == 0 && kind == 1) return launch_one<0, 1>(p, grid, smem, st);
    return launch_one<1, 1>(p, grid, smem, st);
}

int launch_pack_tiles(const TcPackTile* tiles, int64_t count, const double* src, uint8_t* dst, int es,
                      cudaStream_t st) {
    if (count <= 0) return 0;
    const unsigned g = (unsigned)std::min<int64_t>(count, 152 * 16);
    k_pack_tiles<<<g, 256, 0, st>>>(tiles, count, src, dst, es);
    H2_LAUNCH_CHECK();
    return 0;
}

int launch_pack_act(const float* src, int64_t ld, int ids, const int32_t* idmap, const int32_t* base,
                    const int32_t* kdim, int kdim_fixed, const int64_t* koff, int kp_fixed, int mc, int R,
                    uint8_t* dst, int es, cudaStream_t st) {
    if (ids <= 0) return 0;
    const unsigned g = (unsigned)std::min(ids, 152 * 8);
    k_pack_act<<<g, 256, 0, st>>>(src, ld, ids, idmap, base, kdim, kdim_fixed, koff, kp_fixed, mc, R, dst, es);
    H2_LAUNCH_CHECK();
    return 0;
}

int launch_zero_tiles(const int32_t* ids, int count, uint8_t* buf, int64_t tile_bytes, cudaStream_t st) {
    if (count <= 0) return 0;
    k_zero_tiles<<<(unsigned)std::min(count, 152 * 8), 256, 0, st>>>(ids, count, buf, tile_bytes);
    H2_LAUNCH_CHECK();
    return 0;
}

int launch_zero_clusters(const int32_t* ids, int count, float* yhat, int k, int ldc, int mc, cudaStream_t st) {
    if (count <= 0) return 0;
    k_zero_clusters<<<(unsigned)std::min(count, 152 * 8), 256, 0, st>>>(ids, count, yhat, k, ldc, mc);
    H2_LAUNCH_CHECK();
    return 0;
}

}  // namespace h2
