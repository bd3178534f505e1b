/*
 * h2.h — C ABI of the GB300 H²-matrix block-Krylov library (libh2.so).
 *
 * The library computes, for an H² matrix A built from a point cloud, the
 * product of A with a dense block of m columns and solves A X = B for m
 * right-hand sides by block CG (arXiv 2509.17257: the problem statement
 * A x^(i) = b^(i), i = 1..m, of Sec. 1, Eq. (matrix_system); the product
 * y <- y + alpha G x of Sec. 3 Alg. "H2_mvm" and its block form of Sec. 4;
 * the block CG of Sec. 5.1 Alg. "block CG").
 *
 * Conventions for every entry point:
 *  - Return 0 (H2_OK) on success, a negative H2_E_* code otherwise.  No call
 *    aborts or traps; h2_last_error_string() describes the last failure of
 *    the calling thread.
 *  - Dense blocks are row-major n×m arrays of double with a leading
 *    dimension (ld >= m, in elements); row i belongs to point i in the
 *    caller's original order.  A pointer may be device memory or host
 *    memory (pageable or pinned).  A product given host blocks copies them
 *    through device buffers owned by the matrix: X in on the call's stream
 *    before the product, Y in on a stream of the matrix's own while the
 *    product computes (the pass that updates Y waits for it), Y back out
 *    after it; the call returns after the result is complete on the host.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls on
 *    device pointers are asynchronous with respect to the host unless stated.
 *  - The library owns every h2_matrix / h2_tree it returns; free them with
 *    h2_free / h2_tree_free.  The caller owns X, Y, B and the result arrays.
 *  - A matrix handle may be used by one thread/stream at a time (its
 *    internal workspace is shared by the calls on it).
 */
#ifndef H2_H_
#define H2_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define H2_OK 0
#define H2_E_BADARG (-1)      /* invalid argument (null pointer, bad size, NaN point, ...) */
#define H2_E_CUDA (-2)        /* a CUDA runtime call failed */
#define H2_E_NOCONVERGE (-3)  /* block CG hit max_iter / max_outer before every column converged */
#define H2_E_BREAKDOWN (-4)   /* block CG breakdown: <p, A p> <= 0 or a non-finite scalar */
#define H2_E_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define H2_E_OOM (-6)         /* device or host allocation failed */
#define H2_E_UNSUPPORTED (-7) /* precision copy not built, or parameter outside the supported range */

/* ---- compute precision of the H² product ------------------------------- */
typedef enum h2_dtype {
    H2_F64 = 0,  /* all arithmetic in FP64 */
    H2_F32 = 1,  /* FP32 matrices and coefficients, FP32 accumulation */
    H2_BF16 = 2, /* BF16 matrices on the tensor cores, FP32 accumulation */
    H2_F32_MF = 3 /* as H2_F32 on the tensor cores, but the coupling matrices are not read:
                     the coupling kernel evaluates S_b[ν, μ] = g(ξ_{t,ν}, ξ_{s,μ}) (Eq. (h2_admissible))
                     in FP32 from the Chebyshev nodes.  A·X only; H2_E_UNSUPPORTED without the
                     TF32 tiles or after h2_coupling_set (the couplings are then no longer g's) */
} h2_dtype;

/* ---- construction ------------------------------------------------------ */
/* Parameters of the interpolation-based H² matrix
 *   A = Â + sigma·I,  Â ≈ [g(x_i, x_j)],  g(x, y) = exp(-|x - y|_2 / length).
 * Cluster tree: bisection of the tight bounding box at the midpoint of its
 * longest side while a cluster has more than leaf_size points (Sec. 2, Def.
 * "Cluster tree").  Block tree: sons rule of Sec. 2 Def. "Block tree", a
 * block is a leaf iff admissible (Eq. (admiss): max diam <= eta·dist, dist >
 * 0) or leaf × leaf.  Cluster bases: tensor Chebyshev interpolation of order
 * q per axis, rank k = q³, nested through transfer matrices (Def. "Cluster
 * basis"); coupling matrices S_b = [g(ξ_t,ν, ξ_s,μ)] (Eq. (h2_admissible));
 * inadmissible leaves stored densely.
 *
 * kernel selects g.  H2_KERNEL_EXP (0, the default of a zeroed struct) is the
 * real kernel above.  H2_KERNEL_HELMHOLTZ (1) is the complex Helmholtz kernel
 * of Sec. 2 (K = C, g_κ(x, y) = exp(iκr)/(4πr), r = |x - y|_2), regularised
 * at r = 0 as
 *   g(x, y) = exp(i·kappa·r) / (4π·sqrt(r² + delta²)),   delta > 0,
 * with sigma still a real shift.  The bases V and E stay real (interpolation
 * of real nodes); S_b and the nearfield blocks are complex, stored as a plane
 * of real parts followed by a plane of imaginary parts.  A complex matrix is
 * multiplied with h2_matmul_complex only (H2_F64, or H2_F32 with the FP32
 * copy, both on the CUDA cores); every other entry point that computes with
 * A returns H2_E_UNSUPPORTED for it, and precisions may not ask for BF16. */
typedef enum h2_kernel {
    H2_KERNEL_EXP = 0,       /* exp(-r / length), real                              */
    H2_KERNEL_HELMHOLTZ = 1  /* exp(i·kappa·r) / (4π·sqrt(r² + delta²)), complex     */
} h2_kernel;
typedef struct h2_build_params {
    int32_t q;           /* interpolation order per axis, 1 <= q <= 5 (k = q³)   */
    int32_t leaf_size;   /* maximum points per leaf cluster, 1 <= leaf_size <= 64 */
    double eta;          /* admissibility parameter, > 0                          */
    double length;       /* kernel length scale, > 0                              */
    double sigma;        /* diagonal shift                                        */
    uint32_t precisions; /* bit mask of extra copies to build: (1u<<H2_F32) | (1u<<H2_BF16);
                            the FP64 copy is always built                         */
    void* stream;        /* cudaStream_t used for the device part of the build    */
    int32_t kernel;      /* h2_kernel                                              */
    double kappa;        /* H2_KERNEL_HELMHOLTZ: wave number, finite               */
    double delta;        /* H2_KERNEL_HELMHOLTZ: regularisation length, > 0        */
} h2_build_params;

typedef struct h2_matrix h2_matrix;

/* Sizes of a built matrix. */
typedef struct h2_info_t {
    int64_t n;            /* points                                   */
    int64_t k;            /* rank q³                                   */
    int64_t n_clusters;   /* |T_I|                                     */
    int64_t n_leaves;     /* |L_I|                                     */
    int64_t n_adm;        /* |L+|  (admissible leaf blocks)            */
    int64_t n_near;       /* |L-|  (inadmissible leaf blocks)          */
    int64_t nnz_near;     /* sum over L- of |t̂|·|ŝ|                    */
    int32_t depth;        /* deepest cluster level (root = 0)          */
    int32_t q;
    int64_t bytes_f64;    /* device bytes of the FP64 matrix data      */
    int64_t bytes_f32;    /* device bytes of the FP32 copy (0 if none) */
    int64_t bytes_bf16;   /* device bytes of the BF16 copy (0 if none) */
    double flops_per_col; /* algorithmic flops of one product per column of X */
    int32_t launches;     /* kernel launches of one product on the CUDA cores (FP64, Aᵀ) */
    int32_t launches_tc;  /* kernel launches of one tensor-core product (FP32, BF16) of at
                             most 64 columns, a multiple of 4 of them; with k % 4 == 0 and
                             k <= 64 the transfer passes pack the tensor-core operands
                             themselves, otherwise three packing launches are counted  */
    int32_t kernel;       /* h2_kernel of the build                                     */
    int32_t hybrid;       /* 1: the FP32 and BF16 tensor-core products take, by default,
                             the hybrid upward pass (the CUDA-core subtree pass stops at its
                             cut, the clusters above it are transfer items of the coupling
                             launch)                                                      */
    int64_t n_above_cut;  /* clusters above that cut (transfer items of that launch)      */
} h2_info_t;

/* Environment variables read by the library (none is needed; each forces one
 * choice of the built-in rules or of h2_autotune_ex, for comparisons and tests):
 *   read by h2_build for that matrix:
 *     H2_FORCE_SIMT=1        FP32 products on the CUDA cores only
 *     H2_TC_TRANSFER=0|1     FP32 transfer passes on the CUDA cores / the tensor cores
 *     H2_TC_HYBRID=0|1       the hybrid upward pass off / on
 *     H2_KRON=0              q = 4 transfer passes on the dense transfer matrices
 *     H2_HYBRID_ROUND_TERMS  coupling terms per CTA between two heights of the hybrid
 *                            pass's transfer items (1..64, default 16)
 *   read by h2_batch_create for that batch:
 *     H2_BATCH_MULTI=0       batched FP32 products as per-system graph branches
 *   read by each solve:
 *     H2_CG_TRACE=k          block CG prints its largest residual every k checks */

/* Build A from n points (pts: n×3 row-major doubles, host or device).  On
 * success *out owns all device memory of the matrix.  The call synchronises
 * params->stream before returning.  Errors: H2_E_BADARG (n < 1, bad params,
 * non-finite coordinate), H2_E_OOM, H2_E_CUDA. */
int h2_build(const h2_build_params* params, const double* pts, int64_t n, h2_matrix** out);

/* Release a matrix (NULL is allowed). */
int h2_free(h2_matrix* A);

/* Report sizes. */
int h2_info(const h2_matrix* A, h2_info_t* info);

/* Y <- Y + alpha·A·X  (Sec. 3 Alg. "H2_mvm": forward transformation, the
 * multiplication phase over the row-cluster lists of Alg. "prepare_addeval"
 * / "list_addeval", backward transformation; Sec. 4 for m columns).
 * X: n×m (ldx >= m), Y: n×m (ldy >= m), doubles, host or device; X and Y must
 * not overlap.  dtype selects the compute precision; H2_F32 / H2_BF16 need
 * that copy in params->precisions at build time (else H2_E_UNSUPPORTED).
 * m = 0 is a no-op.  Not re-entrant on the same A. */
int h2_matmul(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
              int64_t m, int32_t dtype, void* stream);

/* Y <- Y + alpha·A·X over K = C for a matrix built with H2_KERNEL_HELMHOLTZ
 * (Sec. 2 "unless stated otherwise, K = C"; the product of Sec. 3–4 with
 * complex coupling and nearfield blocks).  X and Y are n×m complex blocks,
 * row-major, each element two doubles (real part, imaginary part): the
 * layout of C99 double _Complex, std::complex<double> and complex128 arrays.
 * ldx, ldy count complex elements (>= m); m <= 2^19.  alpha = alpha_re +
 * i·alpha_im.  Host or device, like h2_matmul.  The forward and backward
 * transformations run the real kernels on the 2m real columns; the coupling
 * and nearfield kernels apply S_b = S_re + i·S_im as S_re·x̂ + S_im·(i·x̂).
 * dtype H2_F64 or H2_F32 (the FP32 copy of the build; FP64 in and out).
 * A real matrix gives H2_E_UNSUPPORTED.  A complex symmetric kernel gives
 * Aᵀ = A, so no transposed complex product is provided. */
int h2_matmul_complex(h2_matrix* A, double alpha_re, double alpha_im, const double* X, int64_t ldx,
                      double* Y, int64_t ldy, int64_t m, int32_t dtype, void* stream);

/* Y <- Y + alpha·Aᵀ·X: the same traversal with the roles of row and column
 * clusters swapped (S_bᵀ on admissible blocks, G_bᵀ on inadmissible ones). */
int h2_matmul_transposed(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y,
                         int64_t ldy, int64_t m, int32_t dtype, void* stream);

/* ---- product without allocation ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers of
 * the library that cannot allocate device memory when they call the product:
 * processes whose device memory is handed out by their own allocator under a
 * fixed budget (another framework's caching allocator owns the GPU), and hot
 * paths that cannot afford cudaMalloc's implicit device synchronisation.
 * h2_matmul may call cudaMalloc to grow the matrix's workspace; this variant
 * never calls cudaMalloc, cudaFree or any allocating routine.
 *
 * Same operation and arguments as h2_matmul (Y <- Y + alpha·A·X), except:
 *  - X and Y must be device memory (no host staging); dtype H2_F64 or H2_F32;
 *    m <= 2^20 (H2_E_BADARG beyond).
 *  - Both precisions run the product on the CUDA cores (the FP32 product of
 *    h2_matmul runs split-TF32 tensor cores where they are built, whose
 *    operand tiles need more scratch): the result equals h2_matmul's to the
 *    precision's tolerance (1e-12 relative for FP64, 1e-5 for FP32), not bit
 *    for bit, and the FP32 product is slower than h2_matmul's.
 *  - Its scratch (X gathered into cluster order, x̂ and ŷ of every cluster) is a
 *    fixed array of H2_NOALLOC_SCRATCH_BYTES (32 MiB) compiled into the
 *    library, reserved on every GPU that loads it until the process exits.
 *    A product that needs more scratch, about elt·(n·m + 2·n_clusters·k·m)
 *    bytes (elt = 8 for H2_F64, 4 for H2_F32) plus 8·n_clusters bytes per
 *    64 columns of counters, is rejected with
 *    H2_E_UNSUPPORTED and a message giving the size; call h2_matmul or pass
 *    fewer columns per call.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it; make that first call before any
 *    stream capture.  The cache remembers the context it was filled in; after
 *    cudaDeviceReset the next call looks the address up again (matrices
 *    built before the reset are invalid anyway: their memory went with the
 *    old context).
 *  - All calls share the one array, which keeps the last call's contents.
 *    Each call first clears the small region of counters and flags its
 *    transfer passes start from (a stream-ordered memset, not an allocation)
 *    and writes every other byte before reading it.  Calls whose work
 *    overlaps on the GPU (different streams, or different matrices at the
 *    same time) race on the array: serialise them.
 *  - Rejected while h2_timing_enable is on for A (timing records events). */
#define H2_NOALLOC_SCRATCH_BYTES (32ull << 20)
int h2_matmul_noalloc(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
                      int64_t m, int32_t dtype, void* stream);

/* ---- per-phase device timing ---------------------------------------------
 * Phases of one product: 0 gather of X into cluster order, 1 leaf forward
 * transformation, 2 upward transfer pass, 3 coupling (admissible part of the
 * multiplication phase), 4 downward transfer pass, 5 leaf backward
 * transformation + nearfield + shift (scatter into Y).  When enabled, every
 * product records CUDA events on its stream between the phases; the times are
 * resolved when queried.  Slot 6 is the coupling kernel launch alone (phase 3
 * without the packing of x̂ for the tensor cores); slot 7 is reserved (0).
 * In the tensor-core chain the upward pass is fused into the leaf forward
 * transformation (phase 1, phase 2 ≈ 0) and the packing of x̂ is in phase 3. */
#define H2_NPHASE 8
/* enable != 0 turns recording on, 0 turns it off; pending records are kept. */
int h2_timing_enable(h2_matrix* A, int32_t enable);
/* ms[H2_NPHASE] receives the accumulated milliseconds per phase and *calls the
 * number of recorded products since the last reset; reset != 0 clears them.
 * Synchronises with the recorded events. */
int h2_timing_query(h2_matrix* A, double* ms, int64_t* calls, int32_t reset);

/* ---- block CG (Sec. 5.1, Alg. "block CG") ------------------------------- */
typedef enum h2_cg_variant {
    H2_CG_COLUMNWISE = 0, /* the paper's block CG: per-column α_i, β_i, γ_i                           */
    H2_CG_GRAM = 1        /* O'Leary's block CG (not in the paper): the same recurrences with m×m Gram
                             matrices, G = Pᵀ(AP), α = G⁻¹ PᵀR, X += Pα, R -= (AP)α, Γ = G⁻¹ (AP)ᵀR,
                             P = R - PΓ; G⁻¹ through a Cholesky factor of G that drops a direction whose
                             pivot is below 1e-10 of its diagonal (deflation).  All Gram matrices, the
                             Cholesky factor and the step solves are FP64 on the device.  Every column
                             searches the whole block Krylov space, so it needs fewer iterations than
                             COLUMNWISE.  1 <= m <= 64 (H2_E_UNSUPPORTED otherwise).                 */
} h2_cg_variant;

typedef enum h2_precond {
    H2_PRECOND_NONE = 0,
    H2_PRECOND_BLOCK_JACOBI = 1 /* M = blockdiag over the leaves t of G_(t,t) + σI (the diagonal nearfield
                                   blocks with the shift), factored once per matrix and σ by FP64 Cholesky;
                                   z = M⁻¹ r costs 2·n_t²·m flops per leaf                                  */
} h2_precond;

typedef struct h2_cg_params {
    double tol;          /* per-column relative residual target |r_i|/|b_i| (|b_i| = 0 read as 1) */
    int32_t max_iter;    /* cap on CG iterations (inner iterations summed for refinement)        */
    int32_t variant;     /* h2_cg_variant                                                          */
    int32_t dtype;       /* precision of the product inside block CG (vectors are always FP64)    */
    int32_t refine;      /* dtype != H2_F64 only: 1 = iterative refinement (FP64 residual B - A X
                            outside, block CG with the dtype product inside, X += D); 2 = one block
                            CG with the dtype product whose recurrence residuals are replaced by the
                            FP64 residual B - A X ("reliable updates") whenever the largest active
                            one fell by the factor inner_tol (default 0.1); a step whose low-
                            precision <p, Ap> is not positive restarts every direction from the
                            FP64 residual (at most max(10, max_iter/50) times, then
                            H2_E_BREAKDOWN); 0 = plain block CG with the dtype product (converges
                            to the dtype operator's solution)                                       */
    double inner_tol;    /* refine 1: relative reduction asked of each inner solve;
                            refine 2: residual reduction between reliable updates                  */
    int32_t max_outer;   /* cap on refinement steps                                                  */
    int32_t check_every; /* convergence test every this many iterations (>= 1)                      */
    int32_t transposed;  /* != 0: solve Aᵀ X = B (the adjoint system), products with Aᵀ                  */
    int32_t precond;     /* h2_precond: H2_PRECOND_BLOCK_JACOBI gives the preconditioned block CG of
                            Sec. 5.1, Alg. "pcg block" (column-wise variant, A only)                  */
    void* stream;        /* cudaStream_t                                                            */
} h2_cg_params;

typedef struct h2_cg_result {
    int32_t status;         /* H2_OK, H2_E_NOCONVERGE or H2_E_BREAKDOWN (also the return value)    */
    int32_t iterations;     /* CG iterations performed (max over columns; summed over refinement)   */
    int32_t outer_steps;    /* refinement steps (refine 1) or reliable updates (refine 2)          */
    int32_t h2mm_calls;     /* H² products performed                                                */
    int32_t* col_iterations;/* optional, caller-owned [m]: iteration at which column i converged    */
    double* rel_residual;   /* optional, caller-owned [m]: |b_i - A x_i|/|b_i| recomputed in FP64     */
    double seconds;         /* wall time of the solve                                                */
} h2_cg_result;

/* Solve A X = B for m columns.  B: n×m (ldb >= m), X: n×m (ldx >= m), host
 * or device doubles; X holds the initial guess on entry and the solution on
 * exit.  Blocks until the solve ends.  Returns H2_OK when every column
 * reached tol, H2_E_NOCONVERGE / H2_E_BREAKDOWN otherwise (X then holds the
 * last iterate and `res` is filled). */
int h2_block_cg(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
                const h2_cg_params* params, h2_cg_result* res);

/* ---- block GMRES (Sec. 5.2, Alg. "pgmres block") -------------------------
 * Every column runs restarted, left-preconditioned GMRES(restart) on its own
 * Krylov space; one block product a = M⁻¹ A q per step (in `dtype`); the
 * Arnoldi step orthogonalises with all inner products first (classical
 * Gram–Schmidt, as the algorithm prints it) and eliminates the new subdiagonal
 * entry with a Givens rotation.  Every restart recomputes r = M⁻¹(b − A x)
 * with the FP64 product, so a low-precision `dtype` gives a mixed-precision
 * solve refined in FP64.  Column i stops extending its basis once its Givens
 * residual |r̂| ≤ tol·|M⁻¹ b_i|; the solve ends when every column's FP64
 * preconditioned residual at a restart meets that bound.  For any A (no
 * symmetry needed). */
typedef struct h2_gmres_params {
    double tol;          /* per-column relative (preconditioned) residual target                 */
    int32_t max_iter;    /* cap on Arnoldi steps (block products), summed over restarts          */
    int32_t restart;     /* ℓ: basis size of one cycle, 1..64                                     */
    int32_t dtype;       /* precision of the product inside a cycle                              */
    int32_t precond;     /* h2_precond (H2_PRECOND_BLOCK_JACOBI: left preconditioning)             */
    int32_t transposed;  /* != 0: solve Aᵀ X = B (products with Aᵀ; M is symmetric)                  */
    void* stream;        /* cudaStream_t                                                          */
} h2_gmres_params;

/* Solve A X = B (device B and X, n×m, ldb/ldx >= m; X holds the initial guess
 * and receives the solution).  res: iterations = Arnoldi steps of the slowest
 * column, outer_steps = restart cycles, rel_residual = |b − A x|/|b| in FP64
 * at exit.  Returns H2_OK or H2_E_NOCONVERGE (res filled either way).  Device
 * memory: (restart + 3)·n·m doubles plus O(m·restart²). */
int h2_block_gmres(h2_matrix* A, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t m,
                   const h2_gmres_params* params, h2_cg_result* res);

/* ---- parameters of A and the adjoint -------------------------------------
 * The method's data that a caller may differentiate: the coupling matrices
 * S_b (Eq. (h2_admissible)), in admissible-list order (the row-cluster lists
 * of Alg. "prepare_addeval", see h2_tree_view.adm_*), each k×k row-major
 * S_b[ν][μ], and the diagonal shift σ. */

/* Copy the FP64 coupling matrices out (S: n_adm·k·k doubles, host or device). */
int h2_coupling_get(h2_matrix* A, double* S, void* stream);
/* Replace the coupling matrices (FP64 in, host or device); the FP32 / BF16
 * copies are rebuilt from them.  Synchronises the stream. */
int h2_coupling_set(h2_matrix* A, const double* S, void* stream);
/* Replace the diagonal shift σ. */
int h2_shift_set(h2_matrix* A, double sigma);

/* Gradients of a loss L through X = A⁻¹B, given Λ = A⁻ᵀ ∂L/∂X (from
 * h2_block_cg with transposed = 1) and X (both n×m device FP64):
 *   dS_b = ∂L/∂S_b = −λ̂_t x̂_sᵀ for every admissible block b = (t, s), where
 *          λ̂ and x̂ are the forward transformations (Alg. "forward/backward",
 *          left part) of Λ and X: since A|_{t̂×ŝ} = V_t S_b V_sᵀ + ..., the
 *          chain rule with ∂L/∂A = −Λ Xᵀ gives V_tᵀ(−Λ Xᵀ)|_{t̂×ŝ} V_s;
 *   dsigma = ∂L/∂σ = −<Λ, X>_F.
 * dS (n_adm·k·k doubles, device) and dsigma (one double, host) may each be
 * NULL.  Computed in FP64; synchronises the stream. */
int h2_adjoint_grads(h2_matrix* A, const double* L, int64_t ldl, const double* X, int64_t ldx, int64_t m,
                     double* dS, double* dsigma, void* stream);

/* ---- many independent systems ---------------------------------------------
 * The paper solves one matrix with many right-hand sides; independent
 * systems (Sec. 5: "the m linear systems" are independent) of different
 * sizes can also share the GPU.  A batch groups existing matrices (it does not
 * own them).  Its products and solver iterations run as one CUDA graph launch
 * covering every system: each system's kernels form an independent branch of
 * the graph, so small systems fill the GPU together.  The graph is captured on
 * first use for a given set of pointers and column counts and replayed
 * afterwards; everything it needs is allocated before the capture. */
typedef struct h2_batch h2_batch;

int h2_batch_create(h2_matrix* const* mats, int32_t count, h2_batch** out);
int h2_batch_free(h2_batch* batch);

/* Y_i <- Y_i + alpha·A_i·X_i for every system i (device pointers; m[i] columns,
 * leading dimensions ldx[i] >= m[i], ldy[i] >= m[i]; m[i] = 0 skips system i).
 * One graph launch on `stream`. */
int h2_batch_matmul(h2_batch* batch, double alpha, const double* const* X, const int64_t* ldx, double* const* Y,
                    const int64_t* ldy, const int64_t* m, int32_t dtype, void* stream);

/* Block CG for every system (device B_i, X_i; X_i holds the initial guess).
 * dtype H2_F64: plain FP64 block CG.  H2_F32 / H2_BF16: block CG with that
 * product and FP64 vectors, recurrence residuals replaced by the FP64 residual
 * B_i - A_i X_i whenever they fell by params->inner_tol (reliable updates, as
 * h2_cg_params.refine = 2).  Every iteration of all unconverged systems is one
 * graph launch; converged systems leave the graph.  res[i] reports system i;
 * its col_iterations / rel_residual pointers may each be NULL or point to
 * m[i] entries.  Returns H2_OK if every system converged. */
int h2_batch_block_cg(h2_batch* batch, const double* const* B, const int64_t* ldb, double* const* X,
                      const int64_t* ldx, const int64_t* m, const h2_cg_params* params, h2_cg_result* res);

/* Autotuning of the product for this matrix and m columns (not in the paper;
 * the product's kernels have shapes and schedules that the fastest choice
 * depends on).  h2_autotune_ex times, for the precision dtype (H2_F32 or
 * H2_BF16), with 2 warm-up and 5 timed products each on zero blocks:
 *   1. the product path: tensor cores with the CUDA-core transfer passes
 *      (path 1), tensor cores with the tensor-core transfer passes (Alg.
 *      "forward/backward" as work lists in dependency order: one launch per
 *      phase, path 2, or sharing the coupling's and the leaf phase's launches,
 *      path 3; FP32 only), CUDA cores only (path 4; FP32 only), and tensor
 *      cores with the CUDA-core subtree passes stopping at the upward cut,
 *      whose clusters above the cut become transfer items of the coupling
 *      launch (path 5; FP32 and BF16);
 *   2. on the best path, the pipeline stage count of the tensor-core kernels
 *      (4 and 5 against as many as fit);
 *   3. on paths 1 and 5, the cut targets of the CUDA-core subtree passes (the task
 *      counts that the upward and the downward schedules aim at: half and
 *      twice the default, upward first).
 * The fastest variant is kept for later products of this precision whose
 * column chunks fall in the same class (at most 8, 16, 32 or 64 columns per
 * 64-column chunk); the cut targets are per matrix.  Synchronises the stream;
 * allocates two n×m blocks for the duration; not inside a stream capture
 * (H2_E_BADARG).  out (optional) receives the candidates and the choice. */
typedef struct h2_tune_result {
    int32_t dtype, m;
    int32_t path;          /* chosen path (1..5, as above)                          */
    int32_t stages;        /* chosen stage count (0: as many as fit)                */
    int32_t up_target;     /* chosen cut targets of the CUDA-core transfer passes   */
    int32_t down_target;
    int32_t n_candidates;  /* candidates timed, in the order above (at most 16)     */
    double ms_best;        /* time per product of the choice, milliseconds           */
    double ms[16];
    int32_t cand_path[16], cand_stages[16], cand_up[16], cand_down[16];
} h2_tune_result;
int h2_autotune_ex(h2_matrix* A, int64_t m, int32_t dtype, void* stream, h2_tune_result* out);

/* h2_autotune_ex for H2_F32; ms[0], ms[1] (optional) receive the fastest
 * tensor-core time and the CUDA-core time per product in milliseconds (ms[0] <
 * 0 when the tensor-core copy was not built). */
int h2_autotune(h2_matrix* A, int64_t m, void* stream, double* ms);

/* ---- host-only topology (Sec. 2 trees; Alg. "prepare_addeval" lists) ---- */
typedef struct h2_tree h2_tree;

typedef struct h2_tree_view {
    int64_t n, n_clusters, n_adm, n_near;
    int32_t depth;
    const int64_t* perm;       /* [n]   point index at each position of the cluster order       */
    const int64_t* cl_offset;  /* [n_clusters] first position of t̂ (clusters in pre-order)       */
    const int64_t* cl_size;    /* [n_clusters]                                                   */
    const int32_t* cl_level;   /* [n_clusters] root = 0                                          */
    const int32_t* cl_parent;  /* [n_clusters] -1 for the root                                   */
    const int32_t* cl_son0;    /* [n_clusters] -1 for a leaf                                     */
    const int32_t* cl_son1;    /* [n_clusters] -1 for a leaf                                     */
    const double* cl_box;      /* [n_clusters×6] lo x,y,z then hi x,y,z                          */
    const int64_t* adm_rowptr; /* [n_clusters+1] admissible blocks of row cluster t: [rowptr[t], rowptr[t+1]) */
    const int32_t* adm_col;    /* [n_adm] column cluster s of each admissible block              */
    const int64_t* near_rowptr;/* [n_clusters+1] inadmissible blocks of row cluster t            */
    const int32_t* near_col;   /* [n_near] column cluster of each inadmissible block             */
} h2_tree_view;

/* Build only the host topology (no GPU needed).  pts: host n×3 doubles.
 * Only q, leaf_size and eta of params are read. */
int h2_tree_build(const h2_build_params* params, const double* pts, int64_t n, h2_tree** out);
/* Pointers stay valid until h2_tree_free. */
int h2_tree_view_get(const h2_tree* T, h2_tree_view* view);
int h2_tree_free(h2_tree* T);
/* The schedules of the FP32/BF16 transfer passes for this tree (each CTA owns
 * the subtrees of cut clusters; the same builder serves h2_build), for
 * inspection and tests.  which = 0: downward pass, steps (c, rd, wr, flags)
 * with flags 1 = load the root's ŷ into entry wr, 2 = store ŷ_c (a leaf);
 * which = 1: upward pass, steps (c, rd0, rd1, wr), a leaf having rd0 = -1 and
 * rd1 = its position among the leaves.  Entries index a per-task stack of
 * *entries k×m blocks.  Call with task_ptr = steps = NULL for *ntasks,
 * *nsteps and *entries; then task_ptr holds ntasks + 1 int32 (task t runs
 * steps task_ptr[t] .. task_ptr[t+1]-1) and steps 4·nsteps int32.
 * Errors: H2_E_BADARG (null T or counts, which not 0 or 1). */
int h2_tree_schedule(const h2_tree* T, int32_t which, int32_t* ntasks, int32_t* nsteps, int32_t* entries,
                     int32_t* task_ptr, int32_t* steps);

/* ---- limits (process-wide; for callers that budget device memory, and for
 * tests of the failure paths) ------------------------------------------------
 * h2_set_alloc_limit: cap on the device bytes that all live matrices of the
 * process hold for their stored data (what h2_build allocates, and the
 * block-Jacobi factors a preconditioned solve adds); 0 (the default) removes
 * the cap.  An allocation past the cap fails as an out-of-memory cudaMalloc
 * would: the call returns H2_E_OOM, and a failed h2_build releases everything
 * it had allocated.  Workspace grown by products and solves is not counted.
 * h2_alloc_bytes: the bytes currently held that way (the count the cap is
 * checked against).
 * h2_set_wait_limit: poll limit of the bounded device-side waits on another
 * CTA's ready flag (the FP64 downward transfer pass, Alg. "forward/backward"
 * in one launch); each poll sleeps about 32 ns.  0 restores the default (2^24
 * polls); a negative value makes every such wait give up at once without
 * looking at the flag, so that a test can exercise the timeout path: the
 * product's kernel then returns early and the next call on that matrix
 * returns H2_E_TIMEOUT (its result is invalid).  Errors: H2_E_BADARG
 * (negative bytes, null pointer). */
int h2_set_alloc_limit(int64_t bytes);
int h2_alloc_bytes(int64_t* bytes);
int h2_set_wait_limit(int64_t polls);

/* Description of the last error on the calling thread ("" if none). */
const char* h2_last_error_string(void);

/* Library version string. */
const char* h2_version(void);

#ifdef __cplusplus
}
#endif
#endif /* H2_H_ */
