/*
 * CPU oracle for the dense LU solve of HPL and HPL-MxP.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the GPU library computes. Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it. The product
 * path (the CUDA library and its Python binding) never calls into it, and the
 * two share no code: no headers, helpers, tables or constants.
 *
 * Everything is FP64 unless the method fixes a lower precision (the HPL-MxP
 * emulation below). Matrices are column-major with a leading dimension, pivot
 * vectors are 0-based int32 with LAPACK semantics (row k was swapped with row
 * ipiv[k] >= k, in order k = 0, 1, ...).
 *
 * Paper references (arXiv 2604.09517, "Sustaining Exascale Performance:
 * Lessons from HPL and HPL-MxP on Aurora"):
 *   Sec. III-A.1 (HPL): solve Ax=b, A dense random FP64, by LU with partial
 *     pivoting followed by triangular solves; flop count 2/3 N^3 + O(N^2).
 *   Sec. III-A.2 (HPL-MxP): the same structure with factorization and trailing
 *     updates in low precision, no pivoting, residual and corrections in FP64.
 *   Sec. II-B: HPL-MxP refines with a non-stationary (GMRES-based) method and
 *     uses a scalable generator for its input matrix.
 * Where the paper is silent the readings are listed at each function.
 *
 * Parity status of each function (what pins it, in tests/):
 *   orc_sm64_next / orc_uniform / orc_generate : published SplitMix64 outputs,
 *       exact-rational diagonal sums, distribution moments.
 *   orc_getrf / orc_getrs : exact rational elimination (n <= 6), Cramer's rule,
 *       LAPACK getrf via scipy, closed forms, ||PA-LU|| invariant.
 *   orc_scaled_residual(_gen) : closed forms and a hand-computed case; NaN for
 *       a NaN or infinite x.
 *   orc_mxp_refine(_plain) iteration counts : the same GMRES-IR around scipy's
 *       GMRES with the preconditioner restated in numpy (equal corrections,
 *       GMRES steps within one per cycle), every operand precision.
 *   orc_round_bf16 / orc_round_e4m3 : PyTorch's RNE casts (library routine),
 *       normals, ties, FP32 subnormals and the overflow threshold.
 *   orc_round_fp16 : NumPy's float16 cast (library routine).
 *   orc_round_tf32 : brute-force nearest search over exact rationals, ties,
 *       subnormals and the overflow threshold.
 *   orc_mxp_factor : FP32 mode equals unpivoted LU; BF16 mode error bound.
 *   orc_mxp_lu_plain : a hand-worked 4 x 4 case in exact rationals for every
 *       operand precision (tests/golden/mxp_2step_by_hand.txt); FP32 mode
 *       against exact rational unpivoted elimination within FP32's bound and
 *       against LAPACK's LU (no interchanges on dominant matrices); the
 *       factor's independence of the panel width in FP32 mode.
 *   orc_mxp_solve : converged x equals the FP64 LU solution; iteration
 *       behaviour with an exact preconditioner (one step).
 *   orc_adjoint : central finite differences and torch.linalg.solve autograd.
 *   FP8 and FP16 operand encodings (prec = 1, 2): element rounding pinned;
 *       the per-row / per-column scale choice is a reading (the paper fixes
 *       none), pinned by a brute-force check of its defining property;
 *       their iteration counts as for every precision (above).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

/* ------------------------------------------------------------------------ */
/* Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used as a counter-based generator.
 * The paper only says the entries are random (Sec. III-A.1) and that HPL-MxP
 * has a scalable generator (Sec. II-B); this definition is the build's own. */

/* The SplitMix64 output function (the variant-13 mixer of the paper above). */
static uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* c-th output (c >= 1) of a SplitMix64 generator whose state starts at s:
 * the state advances by GAMMA before each output. */
uint64_t orc_sm64_next(uint64_t s, uint64_t c) { return orc_mix64(s + c * ORC_GAMMA); }

/* Key of stream `stream` under `seed`: output number stream+1 of the
 * generator seeded with `seed`. Stream tags: A = 0, b/B = 1, batch sizes = 2,
 * batched system s: A = 16 + 2s, b = 17 + 2s. */
uint64_t orc_stream_key(uint64_t seed, uint64_t stream) { return orc_sm64_next(seed, stream + 1); }

/* Raw 64-bit draw number idx (0-based) of a stream. */
uint64_t orc_raw(uint64_t key, uint64_t idx) { return orc_sm64_next(key, idx + 1); }

/* Entry draw: top 53 bits scaled to [0,1), shifted to [-0.5, 0.5). Exact. */
double orc_uniform(uint64_t key, uint64_t idx) {
    uint64_t h = orc_raw(key, idx);
    return (double)(h >> 11) * 0x1p-53 - 0.5;
}

/* |entry| as an integer multiple of 2^-53 (exact): |(h>>11) - 2^52|. */
static uint64_t orc_abs_units(uint64_t key, uint64_t idx) {
    uint64_t m = orc_raw(key, idx) >> 11;
    const uint64_t half = 1ULL << 52;
    return m >= half ? m - half : half - m;
}

/* Fill the m x ncols column-major matrix A (leading dimension lda) with the
 * i.i.d. uniform[-0.5,0.5) entries of stream `stream`; entry (i,j) is draw
 * number j*m + i. With dominant != 0 (square only), the diagonal entry of each
 * row is replaced by the sum over that row of |a_ij| (the original |a_ii|
 * included), summed exactly in 128-bit integers and rounded once to double
 * (round to nearest even). This is the diagonally dominant HPL-MxP input. */
void orc_generate(uint64_t seed, uint64_t stream, int64_t m, int64_t ncols, int dominant,
                  double* A, int64_t lda) {
    uint64_t key = orc_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < ncols; j++)
        for (int64_t i = 0; i < m; i++)
            A[j * lda + i] = orc_uniform(key, (uint64_t)(j * m + i));
    if (dominant && m == ncols) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; i++) {
            unsigned __int128 s = 0;
            for (int64_t j = 0; j < ncols; j++) s += orc_abs_units(key, (uint64_t)(j * m + i));
            A[i * lda + i] = (double)s * 0x1p-53; /* one rounding: int128 -> double */
        }
    }
}

/* Sampled entries (rows[t], cols[t]) of the m-row matrix of a stream, for
 * checks at sizes whose matrix is not kept on the host. With dominant != 0
 * (square, m x m) a diagonal entry is the exact row sum. */
static double orc_row_diag_stream(uint64_t key, int64_t n, int64_t i);
void orc_generate_at(uint64_t seed, uint64_t stream, int64_t m, int dominant, int64_t count,
                     const int64_t* rows, const int64_t* cols, double* out) {
    uint64_t key = orc_stream_key(seed, stream);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < count; t++) {
        int64_t i = rows[t], j = cols[t];
        out[t] = (dominant && i == j) ? orc_row_diag_stream(key, m, i)
                                      : orc_uniform(key, (uint64_t)(j * m + i));
    }
}

/* Entry (i,j) of the generated n x n matrix without storing the matrix. For a
 * dominant matrix the caller supplies the row's diagonal value. */
static double orc_entry(uint64_t key, int64_t n, int64_t i, int64_t j) {
    return orc_uniform(key, (uint64_t)(j * n + i));
}

static double orc_row_diag(uint64_t key, int64_t n, int64_t i) {
    unsigned __int128 s = 0;
    for (int64_t j = 0; j < n; j++) s += orc_abs_units(key, (uint64_t)(j * n + i));
    return (double)s * 0x1p-53;
}

static double orc_row_diag_stream(uint64_t key, int64_t n, int64_t i) { return orc_row_diag(key, n, i); }

/* ------------------------------------------------------------------------ */
/* HPL: LU with partial pivoting (Sec. III-A.1), unblocked, LAPACK dgetf2
 * semantics. Readings: the pivot is the first index attaining the largest
 * |a_ik| (as BLAS idamax); full rows are swapped (factored L columns too);
 * multipliers use true division by the pivot; a zero pivot records
 * info = k+1 (first occurrence, 1-based) and the column is left unscaled.
 * min_gap (optional) receives min over k of (max - second max)/max of the
 * candidate magnitudes, which flags near-ties that rounding order can flip. */
int64_t orc_getrf(int64_t n, double* A, int64_t lda, int32_t* ipiv, double* min_gap) {
    int64_t info = 0;
    double gap_min = INFINITY;
    for (int64_t k = 0; k < n; k++) {
        double* colk = A + k * lda;
        int64_t p = k;
        double vmax = fabs(colk[k]);
        for (int64_t i = k + 1; i < n; i++) {
            double v = fabs(colk[i]);
            if (v > vmax) { vmax = v; p = i; }
        }
        if (min_gap && vmax > 0.0 && n - k > 1) {
            double second = 0.0;
            for (int64_t i = k; i < n; i++)
                if (i != p && fabs(colk[i]) > second) second = fabs(colk[i]);
            double g = (vmax - second) / vmax;
            if (g < gap_min) gap_min = g;
        }
        ipiv[k] = (int32_t)p;
        if (p != k) {
            for (int64_t j = 0; j < n; j++) {
                double t = A[j * lda + k];
                A[j * lda + k] = A[j * lda + p];
                A[j * lda + p] = t;
            }
        }
        double piv = colk[k];
        if (piv != 0.0) {
            for (int64_t i = k + 1; i < n; i++) colk[i] = colk[i] / piv;
        } else if (info == 0) {
            info = k + 1;
        }
        if (piv != 0.0) {
#pragma omp parallel for schedule(static) if (n - k > 256)
            for (int64_t j = k + 1; j < n; j++) {
                double* colj = A + j * lda;
                double ukj = colj[k];
                for (int64_t i = k + 1; i < n; i++) colj[i] -= colk[i] * ukj;
            }
        }
    }
    if (min_gap) *min_gap = gap_min;
    return info;
}

/* Triangular solves after getrf (Sec. III-A.1 "followed by triangular
 * solves"). trans = 0 solves A X = B: apply the interchanges to B in order,
 * then L (unit lower) forward and U backward. trans = 1 solves A^T X = B:
 * U^T forward, L^T backward, then the interchanges in reverse order. */
void orc_getrs(int64_t n, int64_t nrhs, const double* LU, int64_t lda, const int32_t* ipiv,
               int trans, double* B, int64_t ldb) {
#pragma omp parallel for schedule(dynamic) if (nrhs > 1)
    for (int64_t c = 0; c < nrhs; c++) {
        double* b = B + c * ldb;
        if (!trans) {
            for (int64_t k = 0; k < n; k++) {
                int64_t p = ipiv[k];
                if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
            }
            for (int64_t i = 0; i < n; i++) {
                double s = b[i];
                for (int64_t j = 0; j < i; j++) s -= LU[j * lda + i] * b[j];
                b[i] = s;
            }
            for (int64_t i = n - 1; i >= 0; i--) {
                double s = b[i];
                for (int64_t j = i + 1; j < n; j++) s -= LU[j * lda + i] * b[j];
                b[i] = s / LU[i * lda + i];
            }
        } else {
            /* U^T z = b: U^T is lower, (U^T)_ij = U_ji = LU[i*lda + j]. */
            for (int64_t i = 0; i < n; i++) {
                double s = b[i];
                for (int64_t j = 0; j < i; j++) s -= LU[i * lda + j] * b[j];
                b[i] = s / LU[i * lda + i];
            }
            /* L^T w = z: unit upper, (L^T)_ij = L_ji = LU[i*lda + j], j > i. */
            for (int64_t i = n - 1; i >= 0; i--) {
                double s = b[i];
                for (int64_t j = i + 1; j < n; j++) s -= LU[i * lda + j] * b[j];
                b[i] = s;
            }
            for (int64_t k = n - 1; k >= 0; k--) {
                int64_t p = ipiv[k];
                if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* HPL scaled residual (the acceptance test; the paper prints no formula, this
 * is the standard HPL check): ||Ax-b||_inf / (eps (||A||_inf ||x||_inf +
 * ||b||_inf) n) with eps = 2^-53. Each r_i = sum_j a_ij x_j - b_i in FP64. */
/* max |v_i|; NaN if any entry is NaN (a comparison would skip it) */
static double orc_norm_inf_vec(int64_t n, const double* v) {
    double m = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double a = fabs(v[i]);
        if (a != a) return a;
        if (a > m) m = a;
    }
    return m;
}

/* The HPL acceptance quantity. A NaN residual entry makes the result NaN
 * (it is no pass), as does a NaN in x or b. */
double orc_scaled_residual(int64_t n, const double* A, int64_t lda, const double* x, const double* b) {
    double rmax = 0.0, amax = 0.0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(max : rmax, amax) reduction(| : bad)
    for (int64_t i = 0; i < n; i++) {
        double r = 0.0, s = 0.0;
        for (int64_t j = 0; j < n; j++) {
            double a = A[j * lda + i];
            r += a * x[j];
            s += fabs(a);
        }
        r -= b[i];
        if (r != r) bad = 1;
        if (fabs(r) > rmax) rmax = fabs(r);
        if (s > amax) amax = s;
    }
    if (bad) return NAN;
    double eps = 0x1p-53;
    return rmax / (eps * (amax * orc_norm_inf_vec(n, x) + orc_norm_inf_vec(n, b)) * (double)n);
}

/* The same residual with A regenerated from (seed, stream 0) row by row, for
 * sizes whose matrix is not kept. */
double orc_scaled_residual_gen(uint64_t seed, int64_t n, int dominant, const double* x, const double* b) {
    uint64_t key = orc_stream_key(seed, 0);
    double rmax = 0.0, amax = 0.0;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : rmax, amax) reduction(| : bad)
    for (int64_t i = 0; i < n; i++) {
        double r = 0.0, s = 0.0;
        double dii = dominant ? orc_row_diag(key, n, i) : 0.0;
        for (int64_t j = 0; j < n; j++) {
            double a = (dominant && j == i) ? dii : orc_entry(key, n, i, j);
            r += a * x[j];
            s += fabs(a);
        }
        r -= b[i];
        if (r != r) bad = 1;
        if (fabs(r) > rmax) rmax = fabs(r);
        if (s > amax) amax = s;
    }
    if (bad) return NAN;
    double eps = 0x1p-53;
    return rmax / (eps * (amax * orc_norm_inf_vec(n, x) + orc_norm_inf_vec(n, b)) * (double)n);
}

/* Sampled factorization check for sizes the oracle cannot factor: for each
 * sample (i,j) returns (PA)_ij - (LU)_ij with A regenerated, P from ipiv and
 * L, U read from the factored matrix. rowmap[i] must give the original row of
 * A that sits in position i after the interchanges (computed by the caller
 * from ipiv, see orc_perm_from_ipiv). */
void orc_perm_from_ipiv(int64_t n, const int32_t* ipiv, int64_t* rowmap) {
    for (int64_t i = 0; i < n; i++) rowmap[i] = i;
    for (int64_t k = 0; k < n; k++) {
        int64_t p = ipiv[k];
        if (p != k) { int64_t t = rowmap[k]; rowmap[k] = rowmap[p]; rowmap[p] = t; }
    }
}

void orc_lu_sample_diff(uint64_t seed, int64_t n, int dominant, const double* LU, int64_t lda,
                        const int64_t* rowmap, int64_t count, const int64_t* si, const int64_t* sj,
                        double* diff) {
    uint64_t key = orc_stream_key(seed, 0);
#pragma omp parallel for schedule(dynamic)
    for (int64_t t = 0; t < count; t++) {
        int64_t i = si[t], j = sj[t];
        int64_t r = rowmap[i];
        double a = (dominant && r == j) ? orc_row_diag(key, n, r) : orc_entry(key, n, r, j);
        int64_t kmax = i < j ? i : j;
        double s = 0.0;
        for (int64_t k = 0; k < kmax; k++) s += LU[k * lda + i] * LU[j * lda + k];
        s += (i <= j) ? LU[j * lda + i] : LU[j * lda + i] * LU[j * lda + j];
        diff[t] = a - s;
    }
}

/* ------------------------------------------------------------------------ */
/* HPL-MxP emulation (Sec. III-A.2: low-precision factor and update, no
 * pivoting, FP64 residual and corrections; Sec. II-B: GMRES-based refinement).
 * Readings, none of which the paper fixes:
 *   - working storage FP32 (FP64 -> FP32 round to nearest);
 *   - the factorization is the block LU without pivoting (Demmel, Higham &
 *     Schreiber, "Stability of block LU factorization", Numer. Linear Algebra
 *     Appl. 2, 1995): A = L U with L block unit lower and U block upper whose
 *     diagonal blocks D_k are the Schur-complemented diagonal blocks. Per step
 *     of width nb: D = current diagonal block; Dinv = D^-1 by Newton-Schulz
 *     (Schulz 1933: X <- X (2I - D X)) from X = diag(D)^-1, ns_iters steps;
 *     L21 = A21 Dinv; A22 -= L21 A12 (A12 is the block row of U as it stands);
 *   - products take their operands rounded to the low precision and
 *     accumulate in FP32 in increasing k. The Newton-Schulz products are kept
 *     near FP32 accuracy by splitting each operand x into hi = bf16(x) and
 *     lo = bf16(x - hi) and summing hi*hi, then hi*lo, then lo*hi (three BF16
 *     products, FP32 accumulation);
 *   - low precision prec = 0: BF16, round to nearest even;
 *     prec = 1: FP8 E4M3 (finite, max 448), round to nearest even, with one
 *     power-of-two scale per operand row (A operand) or column (B operand)
 *     over the whole contraction index, the smallest one that keeps
 *     amax/scale <= 448; FP8 applies to the trailing update, the panel
 *     product L21 = A21 D^-1 keeps BF16 operands;
 *     prec = 2: FP16 (IEEE binary16), round to nearest even, scaled like FP8
 *     with the bound 65504 (the entries of L21 are about 1/n and would sit in
 *     FP16's subnormal range unscaled), in the panel product L21 = A21 D^-1
 *     as well as in the trailing update (its 3 extra fraction bits over BF16
 *     are lost if L21 is formed from BF16 operands);
 *     prec = 3: no rounding (FP32 operands, FP32 Newton-Schulz), a reference
 *     mode;
 *     prec = 4: TF32 (FP32 exponent range, 10 fraction bits), round to nearest
 *     even, no scales (the range is FP32's), in the panel product and the
 *     trailing update like FP16.                                             */

/* BF16 round-to-nearest-even, written from the format definition (1 sign,
 * 8 exponent, 7 stored fraction bits; the exponent range is FP32's). Normal
 * values keep 8 significant bits. Below 2^-126 (BF16's smallest normal) the
 * grid is the fixed subnormal spacing 2^-133, so fewer bits survive there.
 * Results above the largest finite BF16 (0x1.FEp127) overflow to infinity.
 * Applied to a double, this is one rounding (no intermediate FP32 rounding). */
static double orc_bf16_rne(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    double r;
    if (fabs(x) < 0x1p-126) {
        r = ldexp(nearbyint(ldexp(x, 133)), -133);  /* multiples of 2^-133, RNE */
    } else {
        int e;
        double f = frexp(x, &e);                    /* x = f * 2^e, 0.5 <= |f| < 1 */
        r = ldexp(nearbyint(ldexp(f, 8)), e - 8);   /* 8 significant bits, RNE */
    }
    if (fabs(r) > 0x1.FEp127) r = copysign(INFINITY, r);
    return r;
}

float orc_round_bf16(float x) { return (float)orc_bf16_rne((double)x); }

/* The same rounding applied once to a double (the working copy of a
 * BF16-stored factorization is taken from FP64 A). */
float orc_round_bf16_d(double x) { return (float)orc_bf16_rne(x); }

/* BF16 working copy of an FP64 matrix (values stored as float). */
void orc_to_bf16_storage(int64_t m, int64_t n, const double* A, int64_t lda, float* F, int64_t ldf) {
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++) F[j * ldf + i] = orc_round_bf16_d(A[j * lda + i]);
}

/* FP8 E4M3 (OCP "fn" variant) round-to-nearest-even with saturation to
 * +-448: normals 2^-6 .. 448 with 3 fraction bits, subnormals k * 2^-9. */
float orc_round_e4m3(float x) {
    if (x == 0.0f) return x;
    double a = fabs((double)x);
    double spacing;
    if (a < 0x1p-6) spacing = 0x1p-9;
    else {
        int e;
        frexp(a, &e);                           /* a in [2^(e-1), 2^e) */
        spacing = ldexp(1.0, e - 1 - 3);
    }
    double q = nearbyint(a / spacing) * spacing;
    if (q > 448.0) q = 448.0;
    return (float)copysign(q, (double)x);
}

/* IEEE binary16 round-to-nearest-even: normals 2^-14 .. 65504 with 10
 * fraction bits, subnormals k * 2^-24, overflow to infinity (from 65520 up,
 * the midpoint between 65504 and 2^16). Written from the format definition. */
float orc_round_fp16(float x) {
    if (x == 0.0f || !isfinite(x)) return x;
    double a = fabs((double)x);
    double spacing;
    if (a < 0x1p-14) spacing = 0x1p-24;
    else {
        int e;
        frexp(a, &e);                           /* a in [2^(e-1), 2^e) */
        spacing = ldexp(1.0, e - 1 - 10);
    }
    double q = nearbyint(a / spacing) * spacing;
    if (q > 65504.0) q = INFINITY;
    return (float)copysign(q, (double)x);
}

/* TF32 (the tensor cores' 19-bit format: FP32's sign and 8-bit exponent, 10
 * stored fraction bits) round-to-nearest-even of a float, written from the
 * format definition: normal values keep 11 significant bits; below 2^-126 the
 * grid is the fixed spacing 2^-136; results beyond the largest finite TF32
 * value (2 - 2^-10) 2^127 overflow to infinity. The result is an FP32 value
 * whose 13 low fraction bits are zero. */
float orc_round_tf32(float x) {
    if (x == 0.0f || !isfinite(x)) return x;
    double a = (double)x, r;
    if (fabs(a) < 0x1p-126) {
        r = ldexp(nearbyint(ldexp(a, 136)), -136);
    } else {
        int e;
        double f = frexp(a, &e);                       /* a = f 2^e, 0.5 <= |f| < 1 */
        r = ldexp(nearbyint(ldexp(f, 11)), e - 11);    /* 11 significant bits, RNE */
    }
    if (fabs(r) > 0x1.FFCp127) r = copysign(INFINITY, r);
    return (float)r;
}

/* Scale exponent for a block with max magnitude amax: smallest e with
 * amax * 2^-e <= bound (448 for E4M3, 65504 for FP16). Returns 0 for an
 * all-zero block. */
static int orc_block_exp(double amax, double bound) {
    if (amax == 0.0) return 0;
    int e = (int)ceil(log2(amax / bound));
    while (ldexp(amax, -e) > bound) e++;
    while (e > -127 && ldexp(amax, -(e - 1)) <= bound) e--;
    return e;
}

/* Round an operand to the low precision. X is r x c column-major (ld);
 * kdim_is_rows says whether the contraction index runs along rows (the B
 * operand, k x ncols) or along columns (the A operand, mrows x k). The result
 * is the dequantised value, stored as float. */
static void orc_round_operand(int prec, float* X, int64_t r, int64_t c, int64_t ld, int kdim_is_rows) {
    if (prec == 3) return;
    if (prec == 0 || prec == 4) {
        float (*rnd)(float) = prec == 0 ? orc_round_bf16 : orc_round_tf32;
        for (int64_t j = 0; j < c; j++)
            for (int64_t i = 0; i < r; i++) X[j * ld + i] = rnd(X[j * ld + i]);
        return;
    }
    /* FP8 or FP16 with one scale per operand row (A) or column (B), i.e. per
     * 1 x K tile along the whole contraction index. */
    const double bound = prec == 1 ? 448.0 : 65504.0;
    float (*rnd)(float) = prec == 1 ? orc_round_e4m3 : orc_round_fp16;
    if (kdim_is_rows) {
        for (int64_t j = 0; j < c; j++) {
            double amax = 0.0;
            for (int64_t i = 0; i < r; i++) if (fabs(X[j * ld + i]) > amax) amax = fabs(X[j * ld + i]);
            int e = orc_block_exp(amax, bound);
            for (int64_t i = 0; i < r; i++)
                X[j * ld + i] = (float)ldexp(rnd((float)ldexp(X[j * ld + i], -e)), e);
        }
    } else {
        for (int64_t i = 0; i < r; i++) {
            double amax = 0.0;
            for (int64_t j = 0; j < c; j++) if (fabs(X[j * ld + i]) > amax) amax = fabs(X[j * ld + i]);
            int e = orc_block_exp(amax, bound);
            for (int64_t j = 0; j < c; j++)
                X[j * ld + i] = (float)ldexp(rnd((float)ldexp(X[j * ld + i], -e)), e);
        }
    }
}

/* Exported for the tests: the operand rounding above, in place. */
void orc_round_operand_ext(int prec, float* X, int64_t r, int64_t c, int64_t ld, int kdim_is_rows) {
    orc_round_operand(prec, X, r, c, ld, kdim_is_rows);
}

/* C (m x n, ldc) = sub ? C - A*B : A*B, with A (m x k, lda) and B (k x n, ldb)
 * float, products accumulated in FP32 in increasing k. */
static void orc_gemm32(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda,
                       const float* B, int64_t ldb, float* C, int64_t ldc, int sub) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++) {
            float acc = 0.0f;
            for (int64_t p = 0; p < k; p++) acc += A[p * lda + i] * B[j * ldb + p];
            C[j * ldc + i] = sub ? C[j * ldc + i] - acc : acc;
        }
}

/* C (m x n) += A * B for split operands: A ~ Ah + Al, B ~ Bh + Bl (BF16
 * parts), accumulating hi*hi, then hi*lo, then lo*hi in FP32 per entry (the
 * order of one product over a contraction index of length 3k). */
static void orc_gemm32_split(int64_t m, int64_t n, int64_t k, const float* Ah, const float* Al, int64_t lda,
                             const float* Bh, const float* Bl, int64_t ldb, float* C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++) {
            float acc = 0.0f;
            for (int64_t p = 0; p < k; p++) acc += Ah[p * lda + i] * Bh[j * ldb + p];
            for (int64_t p = 0; p < k; p++) acc += Ah[p * lda + i] * Bl[j * ldb + p];
            for (int64_t p = 0; p < k; p++) acc += Al[p * lda + i] * Bh[j * ldb + p];
            C[j * ldc + i] = acc;
        }
}

/* hi = bf16(x), lo = bf16(x - hi) for an r x c block (x - hi is exact in FP32). */
static void orc_split_bf16(const float* X, int64_t r, int64_t c, int64_t ld, float* hi, float* lo) {
    for (int64_t j = 0; j < c; j++)
        for (int64_t i = 0; i < r; i++) {
            float x = X[j * ld + i];
            float h = orc_round_bf16(x);
            hi[j * r + i] = h;
            lo[j * r + i] = orc_round_bf16(x - h);
        }
}

/* Newton-Schulz inverse of the kb x kb FP32 block D (ld ldd) into X (ld kb):
 * X = diag(D)^-1, then ns_iters times R = D X, T = 2I - R, X = X T. The
 * first step starts from a diagonal X, so its two products are scalings,
 * X_ij = x_i (2 delta_ij - D_ij x_j) with x_i = 1 / D_ii, computed directly in
 * FP32 (a multiply, a subtraction, a multiply, each rounded once). Later steps
 * use split BF16 operands in their products when split != 0, else plain FP32. */
static void orc_newton_schulz(int64_t kb, const float* D, int64_t ldd, int ns_iters, int split, float* X) {
    size_t sz = sizeof(float) * kb * kb;
    float *R = (float*)malloc(sz), *Dh = (float*)malloc(sz), *Dl = (float*)malloc(sz);
    float *Xh = (float*)malloc(sz), *Xl = (float*)malloc(sz), *Th = (float*)malloc(sz), *Tl = (float*)malloc(sz);
    float* Dc = (float*)malloc(sz);
    for (int64_t j = 0; j < kb; j++)
        for (int64_t i = 0; i < kb; i++) {
            Dc[j * kb + i] = D[j * ldd + i];
            X[j * kb + i] = (i == j) ? 1.0f / D[j * ldd + j] : 0.0f;
        }
    if (split) orc_split_bf16(Dc, kb, kb, kb, Dh, Dl);
    for (int it = 0; it < ns_iters; it++) {
        if (it == 0) {                                   /* X is diag(D)^-1: scalings */
            for (int64_t j = 0; j < kb; j++)
                for (int64_t i = 0; i < kb; i++) {
                    float xi = 1.0f / Dc[i * kb + i], xj = 1.0f / Dc[j * kb + j];
                    float r = Dc[j * kb + i] * xj;
                    float t = ((i == j) ? 2.0f : 0.0f) - r;
                    X[j * kb + i] = xi * t;
                }
            continue;
        }
        if (split) {
            orc_split_bf16(X, kb, kb, kb, Xh, Xl);
            orc_gemm32_split(kb, kb, kb, Dh, Dl, kb, Xh, Xl, kb, R, kb);          /* R = D X */
        } else {
            orc_gemm32(kb, kb, kb, Dc, kb, X, kb, R, kb, 0);
        }
        for (int64_t j = 0; j < kb; j++)                                         /* T = 2I - R (in R) */
            for (int64_t i = 0; i < kb; i++) R[j * kb + i] = ((i == j) ? 2.0f : 0.0f) - R[j * kb + i];
        if (split) {
            orc_split_bf16(R, kb, kb, kb, Th, Tl);
            orc_gemm32_split(kb, kb, kb, Xh, Xl, kb, Th, Tl, kb, X, kb);                     /* X = X T */
        } else {
            memcpy(Th, X, sz);
            orc_gemm32(kb, kb, kb, Th, kb, R, kb, X, kb, 0);
        }
    }
    free(R); free(Dh); free(Dl); free(Xh); free(Xl); free(Th); free(Tl); free(Dc);
}

/* Storage rounding of a block (BF16 storage keeps every stored value in BF16). */
static void orc_round_block_bf16(float* X, int64_t r, int64_t c, int64_t ld) {
    for (int64_t j = 0; j < c; j++)
        for (int64_t i = 0; i < r; i++) X[j * ld + i] = orc_round_bf16(X[j * ld + i]);
}

/* Block LU without pivoting of the FP32 matrix A (n x n, lda), in place:
 * below the diagonal the blocks L21 of every step, above it the block rows
 * A12 as they stood at their step, on it the Schur-complemented diagonal
 * blocks D_k. Dinv (n x nb, ld n) receives D_k^-1 in rows k0..k0+kb.
 * Returns info = 1-based index of the first exactly zero diagonal entry of a
 * D_k (Newton-Schulz cannot start there), else 0.
 * storage = 1 keeps the working matrix in BF16 (Sec. III-A.2 / the Aurora runs
 * stored the trailing matrix in BF16 to fit a larger N): A holds BF16 values
 * on entry, and every value written back (L21, the updated A22) is rounded to
 * BF16 once, after its FP32 computation; storage = 0 keeps FP32. */
int64_t orc_mxp_factor(int64_t n, int64_t nb, int prec, int ns_iters, int storage, float* A, int64_t lda,
                       float* Dinv) {
    int64_t info = 0;
    float* X = (float*)malloc(sizeof(float) * nb * nb);
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        int64_t kb = n - k0 < nb ? n - k0 : nb;
        float* D = A + k0 * lda + k0;
        for (int64_t c = 0; c < kb; c++)
            if (D[c * lda + c] == 0.0f && !info) info = k0 + c + 1;
        /* 1. D^-1 by Newton-Schulz */
        orc_newton_schulz(kb, D, lda, ns_iters, prec != 3, X);
        for (int64_t j = 0; j < kb; j++)
            for (int64_t i = 0; i < kb; i++) Dinv[j * n + k0 + i] = X[j * kb + i];
        int64_t m = n - k0 - kb;
        if (m == 0) break;
        float* A12 = A + (k0 + kb) * lda + k0;            /* kb x m */
        float* A21 = A + k0 * lda + k0 + kb;              /* m x kb */
        float* A22 = A + (k0 + kb) * lda + k0 + kb;       /* m x m  */
        float* t12 = (float*)malloc(sizeof(float) * kb * m);
        float* t21 = (float*)malloc(sizeof(float) * m * kb);
        float* Xq = (float*)malloc(sizeof(float) * kb * kb);
        /* 2. L21 = A21 Dinv with low-precision operands */
        memcpy(Xq, X, sizeof(float) * kb * kb);
        for (int64_t j = 0; j < kb; j++) memcpy(t21 + j * m, A21 + j * lda, sizeof(float) * m);
        const int pprec = prec == 1 ? 0 : prec;          /* FP8: the panel product stays BF16 */
        orc_round_operand(pprec, t21, m, kb, m, 0);      /* A operand: k along columns */
        orc_round_operand(pprec, Xq, kb, kb, kb, 1);     /* B operand: k along rows    */
        orc_gemm32(m, kb, kb, t21, m, Xq, kb, A21, lda, 0);
        if (storage == 1) orc_round_block_bf16(A21, m, kb, lda);
        /* 3. trailing update A22 -= L21 A12 */
        for (int64_t j = 0; j < m; j++) memcpy(t12 + j * kb, A12 + j * lda, sizeof(float) * kb);
        for (int64_t j = 0; j < kb; j++) memcpy(t21 + j * m, A21 + j * lda, sizeof(float) * m);
        orc_round_operand(prec, t21, m, kb, m, 0);
        orc_round_operand(prec, t12, kb, m, kb, 1);
        orc_gemm32(m, m, kb, t21, m, t12, kb, A22, lda, 1);
        if (storage == 1) orc_round_block_bf16(A22, m, m, lda);
        free(t12); free(t21); free(Xq);
    }
    free(X);
    return info;
}

/* HPL-MxP factor as a plain right-looking LU without pivoting, in the order
 * the paper states it (Sec. III-A.2: factorization and trailing updates in
 * low precision, no pivoting; Table I: BF16 + FP32 on Aurora). This is the
 * independent reference for the GPU's block factor: it shares nothing with
 * that design (no block inverse, no Newton-Schulz). Per step k0 of width kb:
 *   1. panel: FP32 unpivoted elimination of columns k0..k0+kb over rows
 *      k0..n-1 (true division by the pivot, rank-1 updates inside the panel);
 *   2. U12 = L11^-1 A12 by FP32 forward substitution with the unit lower L11;
 *   3. A22 -= L21 U12 with L21 and U12 rounded to the low precision as
 *      operands (prec as in orc_round_operand: 0 BF16, 1 FP8 E4M3 and 2 FP16
 *      with their power-of-two row / column scales, 3 none), products summed
 *      in FP32 in increasing k, the sum subtracted from the FP32 A22.
 * A (n x n, FP32 working copy) is overwritten by L (unit lower, strictly
 * below the diagonal) and U (on and above it); U12 is stored as computed in
 * FP32 (only the update's operands are rounded). A zero pivot records
 * info = its 1-based index (first occurrence); its column is left unscaled. */
int64_t orc_mxp_lu_plain(int64_t n, int64_t nb, int prec, float* A, int64_t lda) {
    int64_t info = 0;
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        int64_t kb = n - k0 < nb ? n - k0 : nb;
        int64_t k1 = k0 + kb;
        /* 1. panel */
        for (int64_t c = k0; c < k1; c++) {
            float* colc = A + c * lda;
            float piv = colc[c];
            if (piv == 0.0f) {
                if (!info) info = c + 1;
                continue;
            }
            for (int64_t i = c + 1; i < n; i++) colc[i] = colc[i] / piv;
            for (int64_t j = c + 1; j < k1; j++) {
                float* colj = A + j * lda;
                float ucj = colj[c];
                for (int64_t i = c + 1; i < n; i++) colj[i] = colj[i] - colc[i] * ucj;
            }
        }
        int64_t m = n - k1;
        if (m == 0) break;
        /* 2. U12 = L11^-1 A12 */
#pragma omp parallel for schedule(static) if (m > 256)
        for (int64_t j = k1; j < n; j++) {
            float* colj = A + j * lda;
            for (int64_t c = k0; c < k1; c++) {
                float ucj = colj[c];
                for (int64_t i = c + 1; i < k1; i++) colj[i] = colj[i] - A[c * lda + i] * ucj;
            }
        }
        /* 3. A22 -= round(L21) round(U12) */
        float* t21 = (float*)malloc(sizeof(float) * m * kb);
        float* t12 = (float*)malloc(sizeof(float) * kb * m);
        for (int64_t j = 0; j < kb; j++) memcpy(t21 + j * m, A + (k0 + j) * lda + k1, sizeof(float) * m);
        for (int64_t j = 0; j < m; j++) memcpy(t12 + j * kb, A + (k1 + j) * lda + k0, sizeof(float) * kb);
        orc_round_operand(prec, t21, m, kb, m, 0);      /* A operand: k along columns */
        orc_round_operand(prec, t12, kb, m, kb, 1);     /* B operand: k along rows    */
        orc_gemm32(m, m, kb, t21, m, t12, kb, A + k1 * lda + k1, lda, 1);
        free(t21);
        free(t12);
    }
    return info;
}

/* Preconditioner M^-1 v with M = L U the plain factor above, in FP32:
 * y = fl32(v); forward substitution by columns with the unit lower L (for
 * j = 0, 1, ...: y_i -= L_ij y_j for i > j), backward substitution by columns
 * with U (for j = n-1 down to 0: y_j /= U_jj, then y_i -= U_ij y_j for i < j).
 * Widened to FP64. */
static void orc_precond_plain(int64_t n, const float* F, int64_t ldf, const double* v, double* out, float* y) {
    for (int64_t i = 0; i < n; i++) y[i] = (float)v[i];
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = j + 1; i < n; i++) y[i] = y[i] - F[j * ldf + i] * y[j];
    for (int64_t j = n - 1; j >= 0; j--) {
        y[j] = y[j] / F[j * ldf + j];
        for (int64_t i = 0; i < j; i++) y[i] = y[i] - F[j * ldf + i] * y[j];
    }
    for (int64_t i = 0; i < n; i++) out[i] = (double)y[i];
}

/* Preconditioner M^-1 v with M = L U the block factor, in FP32: y = fl32(v);
 * forward with the block unit lower L (y_i -= sum_j L_ij y_j over each block
 * column, in order); backward over the block rows from the last: x_k =
 * Dinv_k y_k, then y_i -= sum_j U_ij x_j for the rows above. Widened to FP64. */
static void orc_precond(int64_t n, int64_t nb, const float* F, int64_t ldf, const float* Dinv, const double* v,
                        double* out, float* y) {
    float* t = y + n;
    for (int64_t i = 0; i < n; i++) y[i] = (float)v[i];
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        int64_t kb = n - k0 < nb ? n - k0 : nb;
        for (int64_t i = k0 + kb; i < n; i++) {
            float s = 0.0f;
            for (int64_t j = k0; j < k0 + kb; j++) s += F[j * ldf + i] * y[j];
            y[i] -= s;
        }
    }
    int64_t last = ((n - 1) / nb) * nb;
    for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
        int64_t kb = n - k0 < nb ? n - k0 : nb;
        for (int64_t i = 0; i < kb; i++) {
            float s = 0.0f;
            for (int64_t j = 0; j < kb; j++) s += Dinv[j * n + k0 + i] * y[k0 + j];
            t[i] = s;
        }
        for (int64_t i = 0; i < kb; i++) y[k0 + i] = t[i];
        for (int64_t i = 0; i < k0; i++) {
            float s = 0.0f;
            for (int64_t j = k0; j < k0 + kb; j++) s += F[j * ldf + i] * y[j];
            y[i] -= s;
        }
    }
    for (int64_t i = 0; i < n; i++) out[i] = (double)y[i];
}

static void orc_matvec(int64_t n, const double* A, int64_t lda, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < n; j++) s += A[j * lda + i] * x[j];
        y[i] = s;
    }
}

/* GMRES's inner product in FP32 data (inner = 1): y = fl32(A) fl32(x), the
 * products of two FP32 values exact in FP64 and summed in FP64 in increasing
 * j, so the only error is the FP32 rounding of A and x. */
static void orc_matvec_f32data(int64_t n, const double* A, int64_t lda, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < n; j++) s += (double)(float)A[j * lda + i] * (double)(float)x[j];
        y[i] = s;
    }
}

static double orc_dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Refinement to FP64 accuracy with the low-precision block factor (F, Dinv) (Sec. III-A.2,
 * Sec. II-B). x0 = M^-1 b. Each outer iteration computes r = b - A x in FP64
 * and the scaled residual; it stops once that is below tol. Otherwise the
 * correction d solves A d = r either by one preconditioner application
 * (refine = 0, classic iterative refinement) or by GMRES with at most gmres_m
 * Arnoldi steps, right-preconditioned by M^-1, modified Gram-Schmidt and
 * Givens rotations in FP64, stopping early once the estimated residual is
 * below 1e-10 of ||r||_2 (refine = 1, GMRES-IR after Carson & Higham, SIAM J.
 * Sci. Comput. 2018, with the preconditioner on the right). inner_f32 = 1
 * computes GMRES's inner matrix-vector products from the FP32 rounding of A
 * and of the vector (the lower "matrix-vector precision" of the
 * five-precision GMRES-IR analysis of Amestoy, Buttari, Higham, L'Excellent,
 * Mary & Vieuble, 2024); the residual of every outer step stays FP64. Then x += d.
 * Returns 0 when converged, 4 when max_iter corrections did not get there.
 * iters = corrections applied, inner = preconditioner applications inside
 * GMRES (equal to iters for refine = 0). hist (optional, max_iter+1) receives
 * the scaled residual before each correction. */
/* The preconditioner in use: the block factor (Dinv != NULL) or the plain one. */
typedef struct {
    int64_t n, nb;
    const float* F;
    int64_t ldf;
    const float* Dinv;
} orc_prec_t;

static void orc_apply_prec(const orc_prec_t* P, const double* v, double* out, float* tmp) {
    if (P->Dinv) orc_precond(P->n, P->nb, P->F, P->ldf, P->Dinv, v, out, tmp);
    else orc_precond_plain(P->n, P->F, P->ldf, v, out, tmp);
}

static int orc_refine_impl(int64_t n, const double* A, int64_t lda, const orc_prec_t* P,
                           const double* b, double* x, int refine, int max_iter, int gmres_m, int inner_f32,
                           double tol, int* iters, int* inner, double* final_sr, double* hist);

int orc_mxp_refine(int64_t n, const double* A, int64_t lda, int64_t nb, const float* F, int64_t ldf,
                   const float* Dinv,
                   const double* b, double* x, int refine, int max_iter, int gmres_m, int inner_f32, double tol,
                   int* iters, int* inner, double* final_sr, double* hist) {
    orc_prec_t P = {n, nb, F, ldf, Dinv};
    return orc_refine_impl(n, A, lda, &P, b, x, refine, max_iter, gmres_m, inner_f32, tol, iters, inner, final_sr,
                           hist);
}

/* The same refinement with the plain factor of orc_mxp_lu_plain as M. */
int orc_mxp_refine_plain(int64_t n, const double* A, int64_t lda, const float* F, int64_t ldf,
                         const double* b, double* x, int refine, int max_iter, int gmres_m, int inner_f32,
                         double tol, int* iters, int* inner, double* final_sr, double* hist) {
    orc_prec_t P = {n, n, F, ldf, NULL};
    return orc_refine_impl(n, A, lda, &P, b, x, refine, max_iter, gmres_m, inner_f32, tol, iters, inner, final_sr,
                           hist);
}

static int orc_refine_impl(int64_t n, const double* A, int64_t lda, const orc_prec_t* P,
                           const double* b, double* x, int refine, int max_iter, int gmres_m, int inner_f32,
                           double tol, int* iters, int* inner, double* final_sr, double* hist) {
    double eps = 0x1p-53;
    double anorm = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < n; j++) s += fabs(A[j * lda + i]);
        if (s > anorm) anorm = s;
    }
    double bnorm = orc_norm_inf_vec(n, b);
    float* tmp = (float*)malloc(sizeof(float) * 2 * n);
    double* r = (double*)malloc(sizeof(double) * n);
    double* d = (double*)malloc(sizeof(double) * n);
    int m = gmres_m > 0 ? gmres_m : 1;
    double* V = (double*)malloc(sizeof(double) * n * (m + 1));
    double* Z = (double*)malloc(sizeof(double) * n * m);
    double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * m);
    double* sn = (double*)malloc(sizeof(double) * m);
    double* g = (double*)malloc(sizeof(double) * (m + 1));
    double* y = (double*)malloc(sizeof(double) * m);
    orc_apply_prec(P, b, x, tmp);
    int it = 0, inn = 0, status = 4;
    double sr = INFINITY;
    for (;;) {
        orc_matvec(n, A, lda, x, r);
        for (int64_t i = 0; i < n; i++) r[i] = b[i] - r[i];
        sr = orc_norm_inf_vec(n, r) / (eps * (anorm * orc_norm_inf_vec(n, x) + bnorm) * (double)n);
        if (hist) hist[it] = sr;
        if (!isfinite(sr)) { status = 3; break; }   /* NaN or Inf: no pass, no further correction */
        if (sr < tol) { status = 0; break; }
        if (it >= max_iter) break;
        if (refine == 0) {
            orc_apply_prec(P, r, d, tmp);
            inn++;
        } else {
            double beta = sqrt(orc_dot(n, r, r));
            for (int64_t i = 0; i < n; i++) V[i] = r[i] / beta;
            for (int i = 0; i <= m; i++) g[i] = 0.0;
            g[0] = beta;
            int j, kk = 0;
            for (j = 0; j < m; j++) {
                double* vj = V + (int64_t)j * n;
                double* zj = Z + (int64_t)j * n;
                double* w = V + (int64_t)(j + 1) * n;
                orc_apply_prec(P, vj, zj, tmp);
                inn++;
                if (inner_f32) orc_matvec_f32data(n, A, lda, zj, w);
                else orc_matvec(n, A, lda, zj, w);
                for (int i = 0; i <= j; i++) {
                    double h = orc_dot(n, w, V + (int64_t)i * n);
                    H[j * (m + 1) + i] = h;
                    for (int64_t q = 0; q < n; q++) w[q] -= h * V[(int64_t)i * n + q];
                }
                double hn = sqrt(orc_dot(n, w, w));
                H[j * (m + 1) + j + 1] = hn;
                if (hn != 0.0) for (int64_t q = 0; q < n; q++) w[q] /= hn;
                for (int i = 0; i < j; i++) {          /* previous rotations */
                    double a = H[j * (m + 1) + i], c = H[j * (m + 1) + i + 1];
                    H[j * (m + 1) + i] = cs[i] * a + sn[i] * c;
                    H[j * (m + 1) + i + 1] = -sn[i] * a + cs[i] * c;
                }
                double a = H[j * (m + 1) + j], c = H[j * (m + 1) + j + 1];
                double rho = hypot(a, c);
                cs[j] = a / rho;
                sn[j] = c / rho;
                H[j * (m + 1) + j] = rho;
                H[j * (m + 1) + j + 1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                kk = j + 1;
                if (fabs(g[j + 1]) <= 1e-10 * beta || hn == 0.0) break;
            }
            for (int i = kk - 1; i >= 0; i--) {       /* back substitution H y = g */
                double s = g[i];
                for (int q = i + 1; q < kk; q++) s -= H[q * (m + 1) + i] * y[q];
                y[i] = s / H[i * (m + 1) + i];
            }
            for (int64_t q = 0; q < n; q++) d[q] = 0.0;
            for (int i = 0; i < kk; i++)
                for (int64_t q = 0; q < n; q++) d[q] += y[i] * Z[(int64_t)i * n + q];
        }
        for (int64_t i = 0; i < n; i++) x[i] += d[i];
        it++;
    }
    if (iters) *iters = it;
    if (inner) *inner = inn;
    if (final_sr) *final_sr = sr;
    free(tmp); free(r); free(d); free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of x = A^-1 b (not in the paper; the differentiable form of the
 * solve): grad_B = A^-T G and grad_A = -grad_B X^T, with the FP64 LU of A. */
int64_t orc_adjoint(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X, int64_t ldx,
                    const double* G, int64_t ldg, double* gradB, int64_t ldgb, double* gradA, int64_t ldga) {
    double* LU = (double*)malloc(sizeof(double) * n * n);
    int32_t* ipiv = (int32_t*)malloc(sizeof(int32_t) * n);
    for (int64_t j = 0; j < n; j++) memcpy(LU + j * n, A + j * lda, sizeof(double) * n);
    int64_t info = orc_getrf(n, LU, n, ipiv, NULL);
    for (int64_t c = 0; c < nrhs; c++) memcpy(gradB + c * ldgb, G + c * ldg, sizeof(double) * n);
    orc_getrs(n, nrhs, LU, n, ipiv, 1, gradB, ldgb);
    if (gradA) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = 0; i < n; i++) {
                double s = 0.0;
                for (int64_t c = 0; c < nrhs; c++) s += gradB[c * ldgb + i] * X[c * ldx + j];
                gradA[j * ldga + i] = -s;
            }
    }
    free(LU); free(ipiv);
    return info;
}

/* Batched workload sizes: n_s = 32 + (draw s of stream 2 mod 481), i.e.
 * uniform on [32, 512] up to a modulo bias below 1e-16. */
void orc_batch_sizes(uint64_t seed, int64_t count, int64_t* nout) {
    uint64_t key = orc_stream_key(seed, 2);
    for (int64_t s = 0; s < count; s++) nout[s] = 32 + (int64_t)(orc_raw(key, (uint64_t)s) % 481ULL);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
