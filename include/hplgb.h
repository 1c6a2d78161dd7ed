/*
 * hplgb — dense LU solve of HPL and HPL-MxP on one GB300 GPU (sm_103a).
 *
 * C ABI. Every pointer argument is a DEVICE pointer owned by the caller unless
 * stated otherwise; the library never frees caller memory and never calls
 * cudaMalloc on the compute path (scratch comes from the caller's workspace,
 * sized by the matching *_workspace_size query). Matrices are column-major
 * with a leading dimension ld >= rows. Pivot vectors are 0-based int32 with
 * LAPACK semantics: in order k = 0, 1, ..., row k was interchanged with row
 * ipiv[k] >= k.
 *
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Calls are asynchronous on that stream unless a function says otherwise.
 * The return value reports argument and launch errors at once (nothing is
 * launched when it is not HPL_OK). Conditions found on the device (a zero
 * pivot, a timed-out wait, non-convergence) are written to the caller's
 * hpl_info, which lives in device memory and is valid after the stream
 * synchronizes.
 *
 * Paper: arXiv 2604.09517, "Sustaining Exascale Performance: Lessons from HPL
 * and HPL-MxP on Aurora". Sec. III-A.1 defines the HPL problem (Ax=b, dense
 * random FP64 A, LU with partial pivoting then triangular solves, 2/3 N^3 +
 * O(N^2) flops) and the per-panel phases PFACT, SWAP, DTRSM, DGEMM with
 * look-ahead. Sec. III-A.2 defines HPL-MxP (factor and trailing update in low
 * precision without pivoting, residual and corrections in FP64). Sec. II-B
 * names GMRES-based refinement and a scalable matrix generator.
 */
#ifndef HPLGB_H
#define HPLGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes returned by every call and stored in hpl_info.status. */
enum {
    HPL_OK = 0,
    HPL_ERR_INVALID = 1,        /* bad size, leading dimension, pointer or workspace */
    HPL_ERR_SINGULAR = 2,       /* exact zero pivot; hpl_info.info = its 1-based index */
    HPL_ERR_NONFINITE = 3,      /* NaN or Inf met where a finite value is required */
    HPL_ERR_NOT_CONVERGED = 4,  /* refinement hit max_iter above the tolerance */
    HPL_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    HPL_ERR_NOMEM = 6,          /* workspace too small */
    HPL_ERR_CUDA = 7            /* a CUDA runtime call failed */
};

/* Generator kinds (hpl_generate). */
enum {
    HPL_GEN_GENERAL = 0,        /* i.i.d. uniform[-0.5, 0.5) */
    HPL_GEN_DIAG_DOMINANT = 1   /* same, diagonal replaced by the row sum of |a_ij| */
};

/* Low-precision operand formats of the mixed-precision factorization. */
enum { HPL_PREC_BF16 = 0, HPL_PREC_FP8_E4M3 = 1, HPL_PREC_FP16 = 2, HPL_PREC_TF32 = 3 };

/* Refinement methods of the mixed-precision solve. */
enum { HPL_REFINE_IR = 0, HPL_REFINE_GMRES = 1 };

/* Options. A NULL hpl_opts* means the defaults listed here. Host memory. */
typedef struct {
    int64_t nb;          /* panel width NB; 0 = default (256 FP64, 3072 mixed, 32 batched) */
    int32_t lookahead;   /* 0 = none, 1 = depth-1 look-ahead on a second stream (default 1) */
    int32_t prec;        /* HPL_PREC_* for the mixed-precision factor (default BF16) */
    int32_t refine;      /* HPL_REFINE_* (default GMRES) */
    int32_t max_iter;    /* outer refinement iterations (default 50) */
    int32_t gmres_m;     /* Arnoldi steps per GMRES cycle (default 30) */
    int32_t ns_iters;    /* Newton-Schulz steps of each diagonal-block inverse, mixed precision (default 2, <= 8) */
    double tol;          /* scaled-residual target (default 16) */
    int64_t timeout_ns;  /* limit for any device-side wait (default 20 s) */
    int32_t fp64_emulation; /* lu_factor: 0 = DFMA trailing update (default); 1 = the same update on the BF16
                               tensor cores with FP64 accuracy (sliced products, see lu_factor) */
    int32_t pfact;       /* lu_factor panel leaves: 0 = auto (default: a leaf whose rows fit in the shared
                            memory of one thread-block cluster runs on that cluster, others on a
                            grid-cooperative launch); 1 = grid-cooperative leaves only. Same pivots and
                            factors either way. */
    int32_t storage;     /* mxp_solve / lu_solve_backward: HPL_STORAGE_FP32 (default) or HPL_STORAGE_BF16, the
                            element type of the working matrix / factor (BF16: with HPL_PREC_BF16 only) */
    int32_t inner;       /* mxp_solve with GMRES refinement: HPL_INNER_FP64 (default) computes the matrix-vector
                            products inside GMRES with the FP64 A; HPL_INNER_FP32 with an FP32 copy of A that
                            the factorization's conversion pass also writes (4 n^2 more workspace bytes). The
                            residual of every refinement step and the acceptance test stay FP64. Ignored by
                            classic refinement and by lu_solve_backward. */
} hpl_opts;

/* Precision of GMRES's inner matrix-vector products (opts.inner). */
enum { HPL_INNER_FP64 = 0, HPL_INNER_FP32 = 1 };

/* Working-matrix storage of the mixed-precision factorization. */
enum { HPL_STORAGE_FP32 = 0, HPL_STORAGE_BF16 = 1 };

/* Result record, written on the device. Caller-allocated in device memory. */
typedef struct {
    int32_t status;          /* HPL_* code of the device-side outcome */
    int32_t iters;           /* refinement corrections applied (mixed precision) */
    int64_t info;            /* first exact zero pivot, 1-based; 0 if none */
    double scaled_residual;  /* last scaled residual computed (mixed precision) */
    int32_t inner_iters;     /* preconditioner applications inside GMRES */
    int32_t reserved;
} hpl_info;

/* Fill the opts struct with the defaults above. Host pointer. */
void hpl_default_opts(hpl_opts* opts);

/* Name of a status code (static string). */
const char* hpl_status_string(int status);

/*
 * hpl_generate — the seeded input generator (Sec. III-A.1: "random entries";
 * Sec. II-B: HPL-MxP's scalable generator; the exact definition is this
 * library's): entry (i,j) of the m x ncols matrix is draw number j*m + i of
 * stream `stream_id`, i.e. SplitMix64 output j*m+i+1 from the state
 * mix(seed + (stream_id+1)*GAMMA), mapped by its top 53 bits to
 * uniform[-0.5, 0.5) exactly. With kind = HPL_GEN_DIAG_DOMINANT (m == ncols)
 * the diagonal of each row becomes the sum of |a_ij| over the row, summed
 * exactly in integers and rounded once (nearest even).
 * Stream tags used by this library: A = 0, b/B = 1.
 * A: device, m x ncols, ld lda >= m. Returns HPL_ERR_INVALID on bad sizes.
 */
int hpl_generate(uint64_t seed, uint64_t stream_id, int64_t m, int64_t ncols, int kind,
                 double* A, int64_t lda, void* stream);

/*
 * lu_factor — HPL's LU with partial pivoting (Sec. III-A.1, phases PFACT,
 * SWAP, DTRSM, DGEMM per panel of width NB, look-ahead depth 1 as in the
 * paper's Table I). In place: A (n x n, lda) is overwritten by L (unit lower,
 * below the diagonal) and U; ipiv (device, n entries) receives the pivots.
 * The pivot of each column is the first row attaining the largest magnitude.
 * A zero pivot sets info->info to its 1-based index, leaves that column
 * unscaled and sets info->status = HPL_ERR_SINGULAR; the factorization goes on.
 * ws (device) must hold lu_factor_workspace_size(n, opts) bytes.
 * With look-ahead the call forks work onto a second, higher-priority stream
 * and joins it back into `stream` before returning; ordering with respect to
 * `stream` is as for a single kernel launch.
 * opts->fp64_emulation = 1 (not in the paper) computes the trailing update on
 * the BF16 tensor cores with FP64 accuracy: each row of L21 and column of U12
 * is cut into 11 integer slices of 6 bits (exact in BF16), the slice products
 * are summed exactly by the tensor cores in 11 groups and combined in 64-bit
 * integers, and the result is rounded to FP64; the panel, swaps and TRSM stay
 * FP64. It needs NB <= 256 (HPL_ERR_INVALID otherwise) and a larger
 * workspace, about 44 n (min(n, 8192) + NB) bytes more (lu_factor_workspace_size
 * depends on n then: 12 GB at n = 32768).
 */
size_t lu_factor_workspace_size(int64_t n, const hpl_opts* opts);
int lu_factor(int64_t n, double* A, int64_t lda, int32_t* ipiv, const hpl_opts* opts,
              void* ws, size_t ws_bytes, hpl_info* info, void* stream);

/*
 * lu_factor_noalloc — lu_factor without a workspace argument, for callers
 * that cannot allocate device memory where they factor (code running under
 * an allocator it does not own, or with a device-memory budget fixed at
 * start-up). The paper has no counterpart; this is a convenience of this
 * library. Same arguments, results and errors as lu_factor, except that the
 * scratch lu_factor needs comes from one fixed device array inside the
 * library (lu_factor_noalloc_max_scratch() bytes, 320 KiB, enough for any
 * NB <= 512), held by every GPU that loads the library until the process
 * exits. opts.fp64_emulation is not available here (its scratch grows with
 * n): it returns HPL_ERR_INVALID with a message naming the option. Options
 * lu_factor refuses return HPL_ERR_INVALID before any size test;
 * HPL_ERR_NOMEM is kept for valid options whose scratch would exceed the
 * array (none with NB <= 512 today). Messages are in hplgb_last_error. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and caches it: make that
 * first call before any stream capture. The array is shared by all calls on a
 * device and cleared by each call on its stream; calls whose GPU work
 * overlaps race on it. It calls no cudaMalloc, cudaFree or other
 * memory-allocating routine (like lu_factor, its first call on a device also
 * creates the library's look-ahead stream and events, once).
 */
size_t lu_factor_noalloc_max_scratch(void);
int lu_factor_noalloc(int64_t n, double* A, int64_t lda, int32_t* ipiv, const hpl_opts* opts,
                      hpl_info* info, void* stream);

/*
 * lu_solve — the triangular solves that follow the factorization
 * (Sec. III-A.1). trans = 0 solves A X = B: the interchanges are applied to B,
 * then L (unit lower) forward and U backward substitution. trans = 1 solves
 * A^T X = B (U^T, then L^T, then the interchanges in reverse order).
 * B (n x nrhs, ldb) holds b on entry and x on exit. ws (256-byte aligned)
 * must hold lu_solve_workspace_size(n, nrhs) bytes. One right-hand side
 * without transpose runs both triangles in one persistent launch, 64-row
 * diagonal blocks applied through their inverses (the same solution as
 * substitution up to rounding). A zero on the diagonal of U sets
 * info->status = HPL_ERR_SINGULAR (the solve still runs; x has Inf/NaN); a
 * device-side wait that expires sets HPL_ERR_TIMEOUT.
 */
size_t lu_solve_workspace_size(int64_t n, int64_t nrhs);
int lu_solve(int64_t n, int64_t nrhs, const double* LU, int64_t lda, const int32_t* ipiv, int trans,
             double* B, int64_t ldb, void* ws, size_t ws_bytes, hpl_info* info, void* stream);

/*
 * hpl_scaled_residual — the HPL acceptance quantity (not printed in the paper;
 * the standard HPL check): ||A x - b||_inf / (eps (||A||_inf ||x||_inf +
 * ||b||_inf) n), eps = 2^-53, all in FP64. A (n x n, lda) is the ORIGINAL
 * matrix; with A == NULL it is regenerated from (seed, stream 0, kind) as
 * hpl_generate defines it. x, b: device vectors of n. out: one device double.
 * ws must hold hpl_residual_workspace_size(n) bytes.
 */
size_t hpl_residual_workspace_size(int64_t n);
int hpl_scaled_residual(int64_t n, const double* A, int64_t lda, uint64_t seed, int kind,
                        const double* x, const double* b, double* out, void* ws, size_t ws_bytes,
                        void* stream);

/*
 * mxp_solve — the HPL-MxP solve (Sec. III-A.2: factorization and trailing
 * updates in low precision without pivoting, residual and corrections in
 * FP64; Sec. II-B: non-stationary refinement based on GMRES). A (n x n, lda,
 * FP64, read only) should be diagonally dominant (the HPL-MxP matrix class,
 * hpl_generate with HPL_GEN_DIAG_DOMINANT). The factorization is the block LU
 * without pivoting of an FP32 copy of A with panel width opts->nb (default
 * 3072): per step, the inverse of the diagonal block by Newton-Schulz
 * iterations with split-BF16 tensor-core products, then L21 = A21 D^-1 and
 * A22 -= L21 A12 with BF16 operands and FP32 accumulation. Each of the nrhs
 * columns of B (ldb) is then solved into X (ldx) by FP64 refinement (opts->
 * refine: classic iterative refinement or GMRES(opts->gmres_m) with the
 * factor as right preconditioner) until the HPL scaled residual is below
 * opts->tol (default 16) or opts->max_iter corrections were made.
 * On return info (device) holds the status (HPL_OK, HPL_ERR_NOT_CONVERGED with
 * the best x so far, HPL_ERR_NONFINITE), the largest correction count and
 * scaled residual over the right-hand sides, and the preconditioner
 * applications. The call blocks the host until the solve is done (the
 * refinement reads one scalar per step). ws (device, mxp_workspace_size
 * bytes) keeps the factor afterwards: F (n x n, ld n) at byte offset 0
 * (L21 blocks below the diagonal, U blocks above, D_k on it; FP32, or BF16
 * with opts->storage = HPL_STORAGE_BF16) and FP32 D_k^-1 (n x nb, ld n,
 * block k in rows k*nb..) at offset align256(4 n^2), or align256(2 n^2) for
 * BF16 storage. BF16 storage (the Aurora runs' choice for a larger N) halves
 * the working matrix: the copy of A is rounded once to BF16 and every value
 * the factorization writes back (L21, the updated trailing matrix) is
 * rounded to BF16 after its FP32 computation; the refinement then restores
 * FP64 accuracy as before (typically with more inner iterations). opts->prec = HPL_PREC_FP8_E4M3 runs the trailing update
 * with FP8 E4M3 operands instead (one power-of-two scale per row of L21 and
 * per column of A12 over the panel width, applied in the GEMM epilogue; the
 * panel product L21 = A21 D^-1 keeps BF16). opts->prec = HPL_PREC_FP16 uses
 * IEEE FP16 operands, scaled the same way (bound 65504), in both the panel
 * product and the trailing update: about 8x less factorization error than
 * BF16 at the same tensor-core rate. opts->prec = HPL_PREC_TF32 uses TF32
 * operands (FP32's exponent range, 10 fraction bits, round to nearest even,
 * no scales) in both products: FP16's accuracy at half the tensor-core rate.
 * FP8, FP16 and TF32 operands need FP32 storage.
 * With nrhs > 1 and opts->refine == HPL_REFINE_IR (and A stored) the columns
 * are refined together: each step forms R = B - A X for all of them as one
 * FP64 product and applies the factor to all of them at once (FP32 block
 * triangular solves); the workspace then also holds these block buffers, so
 * mxp_workspace_size depends on nrhs and opts->refine.
 * A == NULL (lda ignored) solves with the HPL-MxP matrix of `seed` (stream 0,
 * HPL_GEN_DIAG_DOMINANT, as hpl_generate defines it) without storing it: the
 * FP32 working copy is generated directly and every FP64 residual regenerates
 * the entries (the diagonal is kept in ws), so the 8 n^2 bytes of an FP64 A
 * are never needed. seed is ignored when A != NULL.
 */
size_t mxp_workspace_size(int64_t n, int64_t nrhs, const hpl_opts* opts);
int mxp_solve(int64_t n, int64_t nrhs, const double* A, int64_t lda, uint64_t seed, const double* B, int64_t ldb,
              double* X, int64_t ldx, const hpl_opts* opts, void* ws, size_t ws_bytes, hpl_info* info,
              void* stream);

/*
 * lu_solve_backward — the adjoint of X = A^-1 B (not in the paper; the
 * differentiable form of the mixed-precision solve): grad_B = A^-T G and, if
 * gradA != NULL, grad_A = -grad_B X^T. ws must be the workspace of an
 * mxp_solve of the same A with the same n and opts: its saved block factor is
 * reused (transposed: M^-T = L^-T U^-T as preconditioner) and each column of
 * G (n x nrhs, ldg) is refined in FP64 against A^T to the scaled-residual
 * tolerance, into gradB (ldgb); with nrhs > 1 and opts->refine ==
 * HPL_REFINE_IR the columns are refined together as in mxp_solve (ws must
 * then hold mxp_workspace_size(n, nrhs, opts) bytes for this nrhs). X (ldx)
 * is the forward solution; gradA
 * (n x n, ldga) is written, not accumulated. info as for mxp_solve (residuals
 * of the transposed system). Blocks the host like mxp_solve.
 */
int lu_solve_backward(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X, int64_t ldx,
                      const double* G, int64_t ldg, double* gradB, int64_t ldgb, double* gradA, int64_t ldga,
                      const hpl_opts* opts, void* ws, size_t ws_bytes, hpl_info* info, void* stream);

/*
 * Batched solve — many independent small systems (32 <= n <= 512) in one
 * persistent launch, each system solved by one CTA taken from an atomic work
 * queue ordered longest first. kind[s] = 0: HPL's FP64 LU with partial
 * pivoting (Sec. III-A.1) then the triangular solves, pivots into ipiv[s];
 * kind[s] = 1: a diagonally dominant system solved the HPL-MxP way
 * (Sec. III-A.2): the BF16 block-LU factor of mxp_solve (panel width 32,
 * BF16-rounded operands, FP32 accumulation) then FP64 iterative refinement to
 * opts->tol within opts->max_iter corrections. A[s] (device, n[s] x n[s],
 * lda[s]; overwritten by L\U for kind 0, read only for kind 1) and B[s]
 * (device, n[s]: b in, x out) are per-system pointers given in HOST arrays, as
 * are n, lda, ipiv and kind. infos: device array of count hpl_info, one per
 * system in the caller's order.
 * variant[s] (host array, NULL = all 0) picks the system's tile shape: panel
 * width 32 (0) or 16 (1); the package's autotuner measures both per kind and
 * size bucket and stores the choice in a table the Python binding applies.
 * solve_batched_plan writes the work table into ws (synchronous host-to-device
 * copy; ws must hold solve_batched_workspace_size bytes) and launches nothing.
 * solve_batched_run (re)launches the planned work on `stream`: a queue reset
 * and one kernel, no host synchronisation, so it can be captured into a CUDA
 * graph and replayed; max_ctas <= 0 means one CTA per SM. solve_batched is
 * plan + run. hpl_batch_sizes draws the sizes of the batched workload,
 * n_s = 32 + (draw s of generator stream 2 mod 481), into a host array.
 */
int hpl_batch_sizes(uint64_t seed, int64_t count, int64_t* n_out);
/*
 * hpl_batch_shard — host only, no GPU needed: splits the systems of a batch
 * over `world` ranks, one GPU each (the systems are independent, so no data
 * is exchanged between ranks). Longest estimated time first, each system to
 * the rank with the least estimated work so far, lowest rank on ties;
 * deterministic, so every rank computes the same split. n, kind: host arrays
 * of count entries; owner: host array of count int32 receiving each system's
 * rank. HPL_ERR_INVALID for count < 0, world < 1, n < 1 or kind > 1.
 */
int hpl_batch_shard(int64_t count, const int64_t* n, const uint8_t* kind, int32_t world, int32_t* owner);
size_t solve_batched_workspace_size(int64_t count, const int64_t* n, const uint8_t* kind);
int solve_batched_plan(int64_t count, const int64_t* n, double* const* A, const int64_t* lda, double* const* B,
                       int32_t* const* ipiv, const uint8_t* kind, const uint8_t* variant, const hpl_opts* opts,
                       void* ws, size_t ws_bytes);
int solve_batched_run(void* ws, hpl_info* infos, int max_ctas, void* stream);
int solve_batched(int64_t count, const int64_t* n, double* const* A, const int64_t* lda, double* const* B,
                  int32_t* const* ipiv, const uint8_t* kind, const uint8_t* variant, const hpl_opts* opts, void* ws,
                  size_t ws_bytes, hpl_info* infos, void* stream);

/*
 * hpl_upload — copy an FP64 column-major m x n matrix from host memory the
 * device can address (src, leading dimension lds: page-locked memory from
 * cudaHostAlloc / cudaHostRegister or a torch pinned tensor, or any host
 * memory on platforms that give the GPU access to pageable memory, such as
 * Grace) into device memory (dst, ldd), asynchronously on
 * `stream`, by a kernel that reads the host buffer through its mapped device
 * address rather than by the copy engine (on GB300 the copy engine's large
 * host-to-device copies were measured to stall for hundreds of ms after the
 * GPU had been busy or idle; the kernel copy ran at the link's 210 GB/s every
 * time). Not in the paper: the data staging of a solve whose inputs start on
 * the host. HPL_ERR_INVALID for bad sizes or a host buffer the device cannot
 * address (message in hplgb_last_error); nothing is launched then.
 */
int hpl_upload(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd, void* stream);

/*
 * hpl_download — the reverse copy: an FP64 column-major m x n matrix from
 * device memory (src, lds) into host memory the device can address (dst,
 * ldd; as for hpl_upload), asynchronously on `stream`, by a kernel that writes
 * the host buffer through its mapped device address (the result read-back of
 * a solve without the copy engine). The host sees the values once the stream
 * has been synchronized. Not in the paper. Errors as hpl_upload.
 */
int hpl_download(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd, void* stream);

/*
 * hplgb_gemm_bf16 — the tensor-core product of the mixed-precision path
 * (Sec. III-A.2: the factorization and trailing updates run in low precision;
 * Table I: BF16 + FP32 + FP64): C = C - A B^T (sub = 1) or C = A B^T (sub = 0),
 * BF16 operands, FP32 accumulation in tensor memory (tcgen05), FP32 result.
 * A: M x K, B: N x K, BF16 (raw 16-bit words), K contiguous with row strides
 * lda, ldb (multiples of 8, base addresses 16-byte aligned). C: FP32
 * column-major, ldc >= M. err: device int32 the caller zeroes; a bounded
 * device-side wait that expires stores HPL_ERR_TIMEOUT there. Returns
 * HPL_ERR_INVALID for bad sizes, strides or alignment.
 */
int hplgb_gemm_bf16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                    int64_t ldb, float* C, int64_t ldc, int sub, int32_t* err, void* stream);

/*
 * hplgb_gemm_fp8 — the FP8 variant of the update product (configs only; the
 * paper names FP32, FP16 and BF16): C = C - (A B^T) .* (sa sb^T) (sub = 1) or
 * C = (A B^T) .* (sa sb^T), A: M x K and B: N x K FP8 E4M3 bytes, K contiguous,
 * row strides lda, ldb multiples of 16 bytes, 16-byte aligned bases; sa (M)
 * and sb (N) device FP32 scales (NULL = 1); FP32 accumulation in tensor
 * memory (tcgen05 kind::f8f6f4). C, err as hplgb_gemm_bf16.
 */
int hplgb_gemm_fp8(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda, const uint8_t* B, int64_t ldb,
                   const float* sa, const float* sb, float* C, int64_t ldc, int sub, int32_t* err, void* stream);

/*
 * hplgb_gemm_f16 — the FP16 variant (Sec. III-A.2 names FP16 among the low
 * precisions): as hplgb_gemm_fp8 with IEEE binary16 operands (raw 16-bit
 * words, K contiguous, row strides multiples of 8 elements, 16-byte aligned
 * bases) and tcgen05 kind::f16 with F16 inputs; sa, sb optional scales.
 */
int hplgb_gemm_f16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                   const float* sa, const float* sb, float* C, int64_t ldc, int sub, int32_t* err, void* stream);

/*
 * hplgb_gemm_tf32 — the TF32 variant (tcgen05 kind::tf32): A (M x K) and B
 * (N x K) are FP32 words with K contiguous (row strides lda, ldb multiples of
 * 4 elements, 16-byte aligned), already rounded to TF32 (the MMA reads only
 * the sign, exponent and top 10 fraction bits); no scales. C, err as
 * hplgb_gemm_bf16.
 */
int hplgb_gemm_tf32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                    float* C, int64_t ldc, int sub, int32_t* err, void* stream);

/*
 * hplgb_gemm_config — tuning switches of the tensor-core product, for
 * measurement (not in the paper). what = 0: epilogue (value 0, the default:
 * an FP32 C that is 16-byte aligned with a leading dimension divisible by 4
 * is updated by bulk tensor reductions from shared memory, C += -(A B^T), so
 * the SMs never read C; 1: every C read and written by the epilogue threads).
 * what = 1: rows-of-tiles per band of the tile walk (0 = the default per
 * operand kind). what = 2: largest M x N given to the two-SM pair kernel
 * (0 = the default, negative = never). what = 3: 128-byte swizzle atoms of K
 * per pipeline stage of the pair kernel (1:
 * 32 KB stages, four MMAs per barrier round trip; 2, the default: 64 KB
 * stages, eight; the same MMAs in the same order). Process-wide, not thread-safe; results
 * are bit-identical for every setting except where FP32 subnormals occur (the
 * bulk reduction flushes them to zero). Returns HPL_ERR_INVALID for an unknown
 * switch or value.
 */
int hplgb_gemm_config(int what, long long value);

/*
 * hplgb_lu_config — measurement switches of the FP64 LU and its solve (not
 * in the paper).
 * what = 0: the TRSM of the block row, U12 = L11^-1 A12, as one kernel
 * (value 0) or blocked by 64 (value 1, the default: each 64 x 64 diagonal
 * block solved in shared memory, the rows below it updated by the DFMA
 * product kernel). Both apply the same fused multiply-adds to every entry in
 * the same order, so the factors are bit-identical.
 * what = 1: lu_solve of one right-hand side (trans = 0) as one persistent
 * launch for both triangles (value 1, the default) or as per-block
 * launches (value 0). The two sum in different orders (the same solution to
 * rounding).
 * what = 2: CTAs of that persistent launch, 0 (default) = one per SM, else
 * at most value (1 .. 4096); the result is the same bits for every value.
 * Process-wide, not thread-safe; HPL_ERR_INVALID for an unknown switch or
 * value.
 */
int hplgb_lu_config(int what, long long value);

/*
 * hplgb_batched_config — residency switch of the batched solver, for
 * measurement (not in the paper). what = 0: value 0 (default) runs a plan
 * whose systems all use 16-wide panels with two CTAs per SM (its shared
 * memory fits twice), value 1 always one CTA per SM. Same results either way.
 * Process-wide; HPL_ERR_INVALID for an unknown switch or value.
 */
int hplgb_batched_config(int what, long long value);

/*
 * Diagnostics.
 * hplgb_launch_count: kernels launched by the library so far (process-wide).
 * Phase timers, after the paper's per-panel performance model (Sec. III-A.1,
 * "Performance Model": each step costs the slowest of DGEMM, PFACT + BCAST and
 * SWAP; Sec. VI-A, Fig. 4 breaks a run down by phase): while on, lu_factor
 * brackets each phase with CUDA events on the stream that runs it.
 * hplgb_phase_times synchronizes those events and returns, per phase
 * (0 PFACT or the mixed-precision diagonal inverse + L21, 1 SWAP, 2 DTRSM,
 * 3 trailing update, 4 preconditioner / outer product, 5 FP64 -> FP32 copy,
 * 6 FP64 residuals and matrix-vector products, 7 whole refinement, which
 * contains 4 and 6, 8 low-precision operand copies of the mixed-precision
 * products), the summed milliseconds, the algorithmic work (flops; bytes
 * moved for 1, 5, 6 and 8) and the number of timed intervals, then clears
 * the record. ms, work, count: host arrays of 9, any may be NULL. Returns
 * HPL_ERR_CUDA if an event query fails.
 * hplgb_phase_records returns the same intervals one by one, in the order
 * they were opened, without clearing them (call it before hplgb_phase_times):
 * phase id, factorization step k (lu_factor; -1 elsewhere), start relative to
 * the first interval and duration in ms, algorithmic work. Host arrays of cap
 * entries, any may be NULL; *count receives the number of intervals (which
 * may exceed cap). This is the per-step breakdown the paper's performance
 * model is written in.
 * hplgb_last_error: text of the last CUDA error the library met.
 */
long long hplgb_launch_count(void);
void hplgb_set_phase_timing(int on);
int hplgb_phase_times(double* ms, double* work, long long* count);
int hplgb_phase_records(int32_t* phase, int32_t* step, double* start_ms, double* ms, double* work, long long cap,
                        long long* count);
const char* hplgb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HPLGB_H */
