// solve_batched: many independent small systems in one persistent launch.
//
// Each CTA takes the next system from one of two atomic work lists (general
// systems and dominant ones, each ordered by decreasing estimated cost,
// longest first; the two CTAs that share an SM prefer different lists) and
// solves it alone, its matrix in global memory (L2-resident) with one panel
// of NB columns staged in shared memory:
//   kind 0 (general): HPL's LU with partial pivoting in FP64 (Sec. III-A.1):
//     blocked right-looking, panel factored in SMEM (block argmax with the
//     first-index tie rule, row swaps, true division, rank-1), interchanges
//     applied to the other columns, TRSM of the block row, DFMA update of the
//     trailing matrix in 64 x 64 register-tiled blocks; then P b, forward and
//     backward substitution.
//   kind 1 (diagonally dominant): the HPL-MxP reading (Sec. III-A.2) used by
//     mxp_solve, per system: block LU without pivoting of an FP32 copy with
//     panel width NB, D^-1 by Newton-Schulz with split-BF16 products,
//     L21 = A21 D^-1 and A22 -= L21 A12 with BF16-rounded operands and FP32
//     accumulation (here on the CUDA cores: a product of two BF16 values is
//     exact in FP32, as in the tensor cores), then FP64 iterative refinement
//     (r = b - A x in FP64, x += M^-1 r) to the scaled-residual tolerance.
// The run launch (queue reset + kernel) holds no host synchronisation, so it
// can be captured in a CUDA graph and replayed.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <numeric>
#include <utility>
#include <vector>

#include "common.cuh"

namespace hplgb {
namespace bt {

constexpr int NBMAX = 32;          // widest panel (storage); variants use 32 or 16
constexpr int NMAX = 512;          // largest system handled
constexpr int THREADS = 256;
// SMEM panel row stride (doubles) of a panel NB wide: NB + 1, so that the
// rows of one column fall in different banks.
template <int NB>
constexpr int panel_stride() { return NB + 1; }

struct Sys {
    long long n, lda;
    double* A;        // FP64 matrix (kind 0: factored in place; kind 1: read only)
    double* b;        // right-hand side in, solution out
    int32_t* ipiv;    // kind 0
    float* W;         // kind 1: FP32 block factor (n x n, ld n)
    float* Dinv;      // kind 1: D_k^-1 (n x NBMAX, ld n)
    double* r;        // kind 1: FP64 residual / correction scratch (2n)
    float* y32;       // kind 1: FP32 scratch (2n)
    int kind;
    int pad;
    int variant;      // panel width: 0 -> 32, 1 -> 16 (chosen by the autotuner's table)
    int pad2;
};

// Two work lists, each ordered longest first: general systems (FP64-bound)
// at table[0, count0), dominant ones (mostly FP32 work) at table[count0,
// count). Each CTA prefers one list and takes from the other once its own is
// empty; the two CTAs that share an SM prefer different lists (the first to
// start on an SM takes the general list), so an FP64-bound system and a
// mostly-FP32 one run side by side. The counters are cleared by every run.
constexpr int kMaxSmSlots = 512;
struct Header {
    unsigned int counter[2];    // next index in list 0 / list 1
    int count0;                 // systems in list 0
    int count;
    int max_iter;
    int nb_max;                 // widest panel of the plan (16 or 32)
    double tol;
    unsigned int sm_slot[kMaxSmSlots];   // CTAs started per SM (role by arrival)
};

// ---- block-wide reductions -------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; w++) s += red[w];
    return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; w++) s = fmax(s, red[w]);
    return s;
}

// ---- kind 0: FP64 LU with partial pivoting -----------------------------------

// Update C (rows r0.., cols c0..; m x nn) -= L (m x kb, in the SMEM panel at
// panel row offset prow) * U (kb x nn, global rows k0.., cols c0..).
template <int NB>
__device__ void upd64(double* A, long long lda, const double* P, int prow, int m, int nn, int kb, long long r0,
                      long long c0, long long k0, double* Us) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int tj = 0; tj < nn; tj += 64) {
        __syncthreads();
        for (int e = threadIdx.x; e < NB * 64; e += THREADS) {
            int kq = e / 64, c = e % 64;
            Us[kq * 65 + c] = (kq < kb && tj + c < nn) ? A[(c0 + tj + c) * lda + k0 + kq] : 0.0;
        }
        __syncthreads();
        for (int ti = 0; ti < m; ti += 64) {
            double acc[4][4];
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    int r = ti + tx + 16 * i, c = tj + ty + 16 * j;
                    acc[i][j] = (r < m && c < nn) ? A[(c0 + c) * lda + r0 + r] : 0.0;
                }
            // 16-row / 16-column groups entirely outside the matrix are skipped
            // (CTA-uniform bounds): FP64 issue slots are the scarce resource
            const int ni = min(4, (m - ti + 15) / 16), nj = min(4, (nn - tj + 15) / 16);
            for (int kq = 0; kq < kb; kq++) {
                double a[4], bb[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    int r = ti + tx + 16 * i;
                    a[i] = r < m ? P[(prow + r) * panel_stride<NB>() + kq] : 0.0;
                }
#pragma unroll
                for (int j = 0; j < 4; j++) bb[j] = Us[kq * 65 + ty + 16 * j];
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (j < nj) {
#pragma unroll
                        for (int i = 0; i < 4; i++)
                            if (i < ni) acc[i][j] = fma(-a[i], bb[j], acc[i][j]);
                    }
            }
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    int r = ti + tx + 16 * i, c = tj + ty + 16 * j;
                    if (r < m && c < nn) A[(c0 + c) * lda + r0 + r] = acc[i][j];
                }
        }
    }
}

template <int NB>
__device__ void lu64(const Sys& S, double* P, double* Us, long long* redk, long long* redi, hpl_info* info) {
    __shared__ int s_np, s_dst[2 * NBMAX], s_src[2 * NBMAX], s_pos[2 * NBMAX], s_con[2 * NBMAX];
    const int n = (int)S.n;
    const long long lda = S.lda;
    double* A = S.A;
    int first_zero = 0;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = min(NB, n - k0), pm = n - k0;
        __syncthreads();
        for (int e = threadIdx.x; e < pm * kb; e += THREADS) {
            int c = e / pm, r = e % pm;
            P[r * panel_stride<NB>() + c] = A[(long long)(k0 + c) * lda + k0 + r];
        }
        __syncthreads();
        for (int j = 0; j < kb; j++) {
            // argmax of |P(j.., j)|, first index on ties, on integer keys
            // (mag_key: no FP64 compares, which issue at the FP64 rate)
            long long bk = -1, br = 0x7fffffffffffffffLL;
            for (int r = j + threadIdx.x; r < pm; r += THREADS) {
                const long long k = mag_key(P[r * panel_stride<NB>() + j]);
                if (key_better(k, r, bk, br)) { bk = k; br = r; }
            }
            warp_best(bk, br);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            __syncthreads();
            if (lane == 0) { redk[warp] = bk; redi[warp] = br; }
            __syncthreads();
            if (warp == 0) {
                long long k = lane < THREADS / 32 ? redk[lane] : -1;
                long long r = lane < THREADS / 32 ? redi[lane] : 0x7fffffffffffffffLL;
                warp_best(k, r);
                if (lane == 0) redi[THREADS / 32] = r == 0x7fffffffffffffffLL ? j : r;   // only NaN: keep row j
            }
            __syncthreads();
            const int p = (int)redi[THREADS / 32];
            if (threadIdx.x == 0) S.ipiv[k0 + j] = k0 + p;
            if (p != j)
                for (int c = threadIdx.x; c < kb; c += THREADS) {
                    double t = P[j * panel_stride<NB>() + c];
                    P[j * panel_stride<NB>() + c] = P[p * panel_stride<NB>() + c];
                    P[p * panel_stride<NB>() + c] = t;
                }
            __syncthreads();
            const double piv = P[j * panel_stride<NB>() + j];
            if (piv == 0.0) {
                if (!first_zero) first_zero = k0 + j + 1;
                continue;
            }
            for (int r = j + 1 + threadIdx.x; r < pm; r += THREADS) {
                double l = P[r * panel_stride<NB>() + j] / piv;
                P[r * panel_stride<NB>() + j] = l;
                for (int c = j + 1; c < kb; c++) P[r * panel_stride<NB>() + c] = fma(-l, P[j * panel_stride<NB>() + c], P[r * panel_stride<NB>() + c]);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < pm * kb; e += THREADS) {
            int c = e / pm, r = e % pm;
            A[(long long)(k0 + c) * lda + k0 + r] = P[r * panel_stride<NB>() + c];
        }
        __syncthreads();
        // interchanges on the other columns. Panels of 16: warp 0 replays the kb
        // swaps on the list of touched rows and emits the gather pairs
        // new[dst] = old[src]; then one thread per column reads all sources
        // before it writes (one round of independent loads instead of kb
        // dependent swaps through L2). Panels of 32 (the pairs would not fit a
        // thread's registers): the swaps in order, one thread per column.
        if constexpr (NB > 16) {
            for (int c = threadIdx.x; c < n; c += THREADS) {
                if (c >= k0 && c < k0 + kb) continue;
                double* col = A + (long long)c * lda;
                for (int j = 0; j < kb; j++) {
                    int p = S.ipiv[k0 + j];
                    if (p != k0 + j) {
                        double t = col[k0 + j];
                        col[k0 + j] = col[p];
                        col[p] = t;
                    }
                }
            }
        } else {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            for (int i = lane; i < kb; i += 32) s_pos[i] = s_con[i] = k0 + i;
            __syncwarp();
            int L = kb;
            for (int j = 0; j < kb; j++) {
                const int p = S.ipiv[k0 + j];
                if (p == k0 + j) continue;
                int q;
                if (p < k0 + kb) {
                    q = p - k0;
                } else {
                    q = -1;
                    for (int base = kb; base < L && q < 0; base += 32) {
                        const int e = base + lane;
                        const unsigned bal = __ballot_sync(0xffffffffu, e < L && s_pos[e] == p);
                        if (bal) q = base + __ffs(bal) - 1;
                    }
                    if (q < 0) {
                        q = L;
                        if (lane == 0) s_pos[L] = s_con[L] = p;
                        L++;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    const int t = s_con[j];
                    s_con[j] = s_con[q];
                    s_con[q] = t;
                }
                __syncwarp();
            }
            int cnt = 0;
            for (int b = 0; b < L; b += 32) {
                const int e = b + lane;
                const bool mv = e < L && s_pos[e] != s_con[e];
                const unsigned bal = __ballot_sync(0xffffffffu, mv);
                if (mv) {
                    const int o = cnt + __popc(bal & ((1u << lane) - 1));
                    s_dst[o] = s_pos[e];
                    s_src[o] = s_con[e];
                }
                cnt += __popc(bal);
            }
            if (lane == 0) s_np = cnt;
        }
        __syncthreads();
        {
            const int np = s_np;
            for (int c = threadIdx.x; c < n; c += THREADS) {
                if (c >= k0 && c < k0 + kb) continue;
                double* col = A + (long long)c * lda;
                double v[2 * NB];
#pragma unroll
                for (int t = 0; t < 2 * NB; t++)
                    if (t < np) v[t] = col[s_src[t]];
#pragma unroll
                for (int t = 0; t < 2 * NB; t++)
                    if (t < np) col[s_dst[t]] = v[t];
            }
        }
        }
        __syncthreads();
        const int c1 = k0 + kb, m = n - c1;
        if (m > 0) {
            // U12 = L11^-1 A12, one thread per column; panels of 16 keep the
            // column's kb entries in registers (same FMAs in the same order)
            if constexpr (NB > 16) {
                for (int c = c1 + threadIdx.x; c < n; c += THREADS) {
                    double* col = A + (long long)c * lda + k0;
                    for (int i = 1; i < kb; i++) {
                        double s = col[i];
                        for (int q = 0; q < i; q++) s = fma(-P[i * panel_stride<NB>() + q], col[q], s);
                        col[i] = s;
                    }
                }
            } else
            for (int c = c1 + threadIdx.x; c < n; c += THREADS) {
                double* col = A + (long long)c * lda + k0;
                double x[NB];
#pragma unroll
                for (int i = 0; i < NB; i++) x[i] = i < kb ? col[i] : 0.0;
#pragma unroll
                for (int i = 1; i < NB; i++) {
                    if (i < kb) {
                        double s = x[i];
#pragma unroll
                        for (int q = 0; q < i; q++) s = fma(-P[i * panel_stride<NB>() + q], x[q], s);
                        x[i] = s;
                    }
                }
#pragma unroll
                for (int i = 1; i < NB; i++)
                    if (i < kb) col[i] = x[i];
            }
            __syncthreads();
            upd64<NB>(A, lda, P, kb, m, m, kb, c1, c1, k0, Us);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && first_zero) info->info = first_zero;
    // solve: P b, then L forward and U backward in blocks of 32 rows: warp 0
    // solves the diagonal block with shuffles, then every thread updates its
    // rows outside the block. Each b_i sees the same FMAs in the same order as
    // column-by-column substitution, with two block barriers per 32 columns.
    double* b = S.b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        for (int k = 0; k < n; k++) {
            int p = S.ipiv[k];
            if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
        }
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int jb = min(32, n - j0);
        if (warp == 0) {
            // lane holds row j0 + lane of the diagonal block in registers, so
            // the dependent chain per column is one shuffle and one FMA
            double t[32];
#pragma unroll
            for (int j = 0; j < 32; j++) t[j] = (j < jb && lane < jb) ? A[(long long)(j0 + j) * lda + j0 + lane] : 0.0;
            double v = lane < jb ? b[j0 + lane] : 0.0;
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const double xj = __shfl_sync(0xffffffffu, v, j);
                if (lane > j && lane < jb) v = fma(-t[j], xj, v);
            }
            if (lane < jb) b[j0 + lane] = v;
        }
        __syncthreads();
        for (int i = j0 + jb + threadIdx.x; i < n; i += THREADS) {
            double acc = b[i];
            for (int j = 0; j < jb; j++) acc = fma(-A[(long long)(j0 + j) * lda + i], b[j0 + j], acc);
            b[i] = acc;
        }
        __syncthreads();
    }
    for (int j1 = n; j1 > 0; j1 -= 32) {
        const int j0 = max(0, j1 - 32), jb = j1 - j0;
        if (warp == 0) {
            // as above, with the reciprocals of the diagonal taken once per
            // block, all lanes at once (an FP64 division is a chain of FP64
            // instructions; in the substitution it would be on the critical path)
            double t[32];
#pragma unroll
            for (int j = 0; j < 32; j++) t[j] = (j < jb && lane < jb) ? A[(long long)(j0 + j) * lda + j0 + lane] : 0.0;
            const double rinv = lane < jb ? 1.0 / A[(long long)(j0 + lane) * lda + j0 + lane] : 0.0;
            double v = lane < jb ? b[j0 + lane] : 0.0;
#pragma unroll
            for (int j = 31; j >= 0; j--) {
                if (j < jb) {
                    if (lane == j) v = v * rinv;
                    const double xj = __shfl_sync(0xffffffffu, v, j);
                    if (lane < j) v = fma(-t[j], xj, v);
                }
            }
            if (lane < jb) b[j0 + lane] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < j0; i += THREADS) {
            double acc = b[i];
            for (int j = jb - 1; j >= 0; j--) acc = fma(-A[(long long)(j0 + j) * lda + i], b[j0 + j], acc);
            b[i] = acc;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) info->status = first_zero ? HPL_ERR_SINGULAR : HPL_OK;
}

// ---- kind 1: BF16 block LU + FP64 refinement ----------------------------------

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C (m x nn, FP32, ldc) (= or -=) rnd(A) (m x kb, lda) * rnd(B) (kb x nn, ldb),
// FP32 accumulation; operands rounded to BF16 (split = 0) or split into
// hi + lo with hi*hi, hi*lo, lo*hi accumulated in that order (split = 1).
__device__ void gemm32(int m, int nn, int kb, const float* A, long long lda, const float* B, long long ldb, float* C,
                       long long ldc, int sub, int split) {
    for (int e = threadIdx.x; e < m * nn; e += THREADS) {
        int j = e / m, i = e % m;
        float acc = 0.0f;
        if (!split) {
            for (int q = 0; q < kb; q++) acc = fmaf(bfr(A[(long long)q * lda + i]), bfr(B[(long long)j * ldb + q]), acc);
        } else {
            for (int q = 0; q < kb; q++) acc = fmaf(bfr(A[(long long)q * lda + i]), bfr(B[(long long)j * ldb + q]), acc);
            for (int q = 0; q < kb; q++) {
                float bv = B[(long long)j * ldb + q];
                acc = fmaf(bfr(A[(long long)q * lda + i]), bfr(bv - bfr(bv)), acc);
            }
            for (int q = 0; q < kb; q++) {
                float av = A[(long long)q * lda + i];
                acc = fmaf(bfr(av - bfr(av)), bfr(B[(long long)j * ldb + q]), acc);
            }
        }
        C[(long long)j * ldc + i] = sub ? C[(long long)j * ldc + i] - acc : acc;
    }
}

// Block LU without pivoting of W (FP32 copy of A); D^-1 in Dinv. X, R: SMEM
// NB x NB FP32 scratch.
// A22 (m x m, ld ld) -= bf16(L21) (m x kb) bf16(A12) (kb x m), FP32
// accumulation in increasing k, then one subtraction (the order of gemm32):
// the operands are rounded once into shared memory (scratch: 2 m kb floats),
// then 64 x 64 output tiles with a 4 x 4 register tile per thread.
__device__ void upd32(int m, int kb, const float* L21, const float* A12, float* A22, long long ld, float* scratch) {
    float* Lr = scratch;              // Lr[q * m + i] = bf16(L21(i, q))
    float* Ur = scratch + m * kb;     // Ur[j * kb + q] = bf16(A12(q, j))
    for (int e = threadIdx.x; e < m * kb; e += THREADS) {
        const int q = e / m, i = e - q * m;
        Lr[e] = bfr(L21[(long long)q * ld + i]);
    }
    for (int e = threadIdx.x; e < m * kb; e += THREADS) {
        const int j = e / kb, q = e - j * kb;
        Ur[e] = bfr(A12[(long long)j * ld + q]);
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int tj = 0; tj < m; tj += 64)
        for (int ti = 0; ti < m; ti += 64) {
            float acc[4][4] = {};
            int r[4], c[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                r[i] = min(ti + tx + 16 * i, m - 1);
                c[i] = min(tj + ty + 16 * i, m - 1);
            }
            for (int q = 0; q < kb; q++) {
                float a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = Lr[q * m + r[i]];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = Ur[c[j] * kb + q];
#pragma unroll
                for (int j = 0; j < 4; j++)
#pragma unroll
                    for (int i = 0; i < 4; i++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int rr = ti + tx + 16 * i, cc = tj + ty + 16 * j;
                    if (rr < m && cc < m) A22[(long long)cc * ld + rr] -= acc[i][j];
                }
        }
}

template <int NB>
__device__ void blocklu32(const Sys& S, float* X, float* R, float* T, float* scratch, hpl_info* info) {
    const int n = (int)S.n;
    float* W = S.W;
    for (int e = threadIdx.x; e < n * n; e += THREADS) {
        int j = e / n, i = e % n;
        W[(long long)j * n + i] = f64_to_f32_rn(S.A[(long long)j * S.lda + i]);   // integer pipe, not FP64
    }
    __syncthreads();
    int first_zero = 0;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = min(NB, n - k0), m = n - k0 - kb;
        float* D = W + (long long)k0 * n + k0;
        for (int e = threadIdx.x; e < kb * kb; e += THREADS) {
            int j = e / kb, i = e % kb;
            X[j * NB + i] = (i == j) ? 1.0f / D[(long long)j * n + j] : 0.0f;
        }
        if (threadIdx.x == 0)
            for (int i = 0; i < kb; i++)
                if (D[(long long)i * n + i] == 0.0f && !first_zero) first_zero = k0 + i + 1;
        float* Ds = scratch;                  // D staged in shared memory for the products
        for (int e = threadIdx.x; e < kb * kb; e += THREADS) Ds[e] = D[(long long)(e / kb) * n + e % kb];
        __syncthreads();
        // first step from X0 = diag(D)^-1: diagonal scalings, each operation rounded once
        for (int e = threadIdx.x; e < kb * kb; e += THREADS) {
            const int j = e / kb, i = e % kb;
            const float xi = 1.0f / Ds[i * kb + i], xj = 1.0f / Ds[j * kb + j];
            X[j * NB + i] = __fmul_rn(xi, __fsub_rn(i == j ? 2.0f : 0.0f, __fmul_rn(Ds[j * kb + i], xj)));
        }
        __syncthreads();
        for (int it = 1; it < 3; it++) {     // 3 steps: systems this small are only weakly dominant
            gemm32(kb, kb, kb, Ds, kb, X, NB, R, NB, 0, 1);             // R = D X
            __syncthreads();
            for (int e = threadIdx.x; e < kb * kb; e += THREADS) {
                int j = e / kb, i = e % kb;
                R[j * NB + i] = ((i == j) ? 2.0f : 0.0f) - R[j * NB + i];
            }
            __syncthreads();
            gemm32(kb, kb, kb, X, NB, R, NB, T, NB, 0, 1);              // T = X (2I - R)
            __syncthreads();
            for (int e = threadIdx.x; e < kb * kb; e += THREADS) X[(e / kb) * NB + e % kb] = T[(e / kb) * NB + e % kb];
            __syncthreads();
        }
        for (int e = threadIdx.x; e < kb * kb; e += THREADS) {
            int j = e / kb, i = e % kb;
            S.Dinv[(long long)j * n + k0 + i] = X[j * NB + i];
        }
        if (m > 0) {
            float* A21 = W + (long long)k0 * n + k0 + kb;
            float* A12 = W + (long long)(k0 + kb) * n + k0;
            float* A22 = W + (long long)(k0 + kb) * n + k0 + kb;
            // L21 = bf16(A21) bf16(D^-1), FP32 accumulation in increasing k (the
            // order of gemm32): both operands rounded once into shared memory,
            // then every entry from there (A21 is read entirely before it is
            // overwritten, and no product waits on an L2 load)
            {
                float* Ar = scratch;              // Ar[q * m + i] = bf16(A21(i, q))
                float* Xr = scratch + m * kb;     // Xr[j * kb + q] = bf16(D^-1(q, j))
                for (int e = threadIdx.x; e < m * kb; e += THREADS) {
                    const int q = e / m, i = e - q * m;
                    Ar[e] = bfr(A21[(long long)q * n + i]);
                }
                for (int e = threadIdx.x; e < kb * kb; e += THREADS) {
                    const int j = e / kb, q = e - j * kb;
                    Xr[e] = bfr(X[j * NB + q]);
                }
                __syncthreads();
                for (int e = threadIdx.x; e < m * kb; e += THREADS) {
                    const int j = e / m, i = e - j * m;
                    float acc = 0.0f;
                    for (int q = 0; q < kb; q++) acc = fmaf(Ar[q * m + i], Xr[j * kb + q], acc);
                    A21[(long long)j * n + i] = acc;
                }
                __syncthreads();
            }
            upd32(m, kb, A21, A12, A22, n, scratch);                   // A22 -= L21 A12
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && first_zero) info->info = first_zero;
    __syncthreads();
}

// out = M^-1 v (FP64 in and out), M the block factor, FP32 inside.
template <int NB>
__device__ void precond32(const Sys& S, const double* v, double* out) {
    const int n = (int)S.n;
    float* y = S.y32;
    float* t = S.y32 + n;
    for (int i = threadIdx.x; i < n; i += THREADS) y[i] = (float)v[i];
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = min(NB, n - k0);
        for (int i = k0 + kb + threadIdx.x; i < n; i += THREADS) {
            float s = 0.0f;
            for (int j = k0; j < k0 + kb; j++) s = fmaf(S.W[(long long)j * n + i], y[j], s);
            y[i] -= s;
        }
        __syncthreads();
    }
    const int last = ((n - 1) / NB) * NB;
    for (int k0 = last; k0 >= 0; k0 -= NB) {
        const int kb = min(NB, n - k0);
        for (int i = threadIdx.x; i < kb; i += THREADS) {
            float s = 0.0f;
            for (int j = 0; j < kb; j++) s = fmaf(S.Dinv[(long long)j * n + k0 + i], y[k0 + j], s);
            t[i] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kb; i += THREADS) y[k0 + i] = t[i];
        __syncthreads();
        for (int i = threadIdx.x; i < k0; i += THREADS) {
            float s = 0.0f;
            for (int j = k0; j < k0 + kb; j++) s = fmaf(S.W[(long long)j * n + i], y[j], s);
            y[i] -= s;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += THREADS) out[i] = (double)y[i];
    __syncthreads();
}

// r = b - A x (FP64), returns the HPL scaled residual. ||A||_inf is summed on
// the first call (*anorm < 0) and reused after (FP64 instructions are scarce).
__device__ double resid64(const Sys& S, const double* x, const double* b, double* r, double* red, double* anorm) {
    const int n = (int)S.n;
    const bool sum_norm = *anorm < 0.0;
    double rmax = 0.0, amax = 0.0, xmax = 0.0, bmax = 0.0;
    for (int i = threadIdx.x; i < n; i += THREADS) {
        double s = 0.0, a = 0.0;
        if (sum_norm) {
            // row sums of |a_ij| in FP32 from the truncated magnitudes (integer
            // operations; the stopping test's norm, as in the large solve)
            float af = 0.0f;
            for (int j = 0; j < n; j++) {
                double v = S.A[(long long)j * S.lda + i];
                s = fma(v, x[j], s);
                const unsigned long long u = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
                const int ex = (int)(u >> 52) - 1023 + 127;
                af += ex <= 0 ? 0.0f : ex >= 255 ? __int_as_float(0x7f800000) :
                      __int_as_float((ex << 23) | (int)((u >> 29) & 0x7fffff));
            }
            a = (double)af;
        } else {
            for (int j = 0; j < n; j++) s = fma(S.A[(long long)j * S.lda + i], x[j], s);
        }
        r[i] = b[i] - s;
        rmax = fmax(rmax, fabs(r[i]) != fabs(r[i]) ? INFINITY : fabs(r[i]));
        amax = fmax(amax, a);
        xmax = fmax(xmax, fabs(x[i]));
        bmax = fmax(bmax, fabs(b[i]));
    }
    rmax = block_max(rmax, red);
    if (sum_norm) *anorm = block_max(amax, red);
    amax = *anorm;
    xmax = block_max(xmax, red);
    bmax = block_max(bmax, red);
    return rmax / (0x1p-53 * (amax * xmax + bmax) * (double)n);
}

template <int NB>
__device__ void mxp_one(const Sys& S, const Header* H, float* X, float* R, float* T, float* scratch, double* red,
                        hpl_info* info) {
    const int n = (int)S.n;
    blocklu32<NB>(S, X, R, T, scratch, info);
    double* bx = S.b;             // b in, x out
    double* r = S.r;
    double* b0 = S.r + n;         // keep b
    for (int i = threadIdx.x; i < n; i += THREADS) b0[i] = bx[i];
    __syncthreads();
    precond32<NB>(S, b0, bx);
    int it = 0;
    double sr = INFINITY, anorm = -1.0;
    int status = HPL_ERR_NOT_CONVERGED;
    for (;;) {
        sr = resid64(S, bx, b0, r, red, &anorm);
        if (!(sr == sr) || sr == INFINITY) { status = HPL_ERR_NONFINITE; break; }
        if (sr < H->tol) { status = HPL_OK; break; }
        if (it >= H->max_iter) break;
        precond32<NB>(S, r, r);
        for (int i = threadIdx.x; i < n; i += THREADS) bx[i] += r[i];
        __syncthreads();
        it++;
    }
    if (threadIdx.x == 0) {
        info->status = status;
        info->iters = it;
        info->inner_iters = it;
        info->scaled_residual = sr;
    }
}

// Dynamic shared memory of a run whose widest panel is NBR: the FP64 panel
// (NMAX x (NBR + 1)), the U block (NBR x 65), three NBR x NBR FP32 blocks.
template <int NBR>
constexpr size_t smem_bytes() {
    return sizeof(double) * (NMAX * panel_stride<NBR>() + NBR * 65) + sizeof(float) * 3 * NBR * NBR;
}

}  // namespace bt

// Workspace: header, system table, then per dominant system W (n x n FP32),
// Dinv (n x NBMAX FP32), r (2n FP64), y32 (2n FP32).
static size_t batched_ws_layout(int64_t count, const int64_t* n, const uint8_t* kind, std::vector<size_t>* offs) {
    size_t off = align_up(sizeof(bt::Header), 256);
    off = align_up(off + sizeof(bt::Sys) * (size_t)count, 256);
    if (offs) offs->assign((size_t)count, 0);
    for (int64_t s = 0; s < count; s++) {
        if (kind[s] != 1) continue;
        if (offs) (*offs)[s] = off;
        int64_t m = n[s];
        off = align_up(off + sizeof(float) * m * m, 256);
        off = align_up(off + sizeof(float) * m * bt::NBMAX, 256);
        off = align_up(off + sizeof(double) * 2 * m, 256);
        off = align_up(off + sizeof(float) * 2 * m, 256);
    }
    return off;
}

}  // namespace hplgb

using namespace hplgb;

// Estimated time of one system: FP64 work costs ~64x FP32 work on this part;
// a dominant system adds a few FP64 refinement passes over its matrix.
static double system_cost(int64_t n, uint8_t kind) {
    const double m = (double)n;
    return kind == 0 ? 64.0 * m * m * m / 3.0 : m * m * m / 3.0 + 3.0 * 64.0 * m * m;
}

// Split the systems over `world` ranks (one GPU each): longest first, each to
// the rank with the least estimated work so far (lowest rank on ties). Host
// only; every rank computes the same split, so no exchange is needed.
extern "C" int hpl_batch_shard(int64_t count, const int64_t* n, const uint8_t* kind, int32_t world, int32_t* owner) {
    if (count < 0 || world < 1 || (count > 0 && (!n || !kind || !owner))) return HPL_ERR_INVALID;
    std::vector<double> cost((size_t)count);
    for (int64_t s = 0; s < count; s++) {
        if (n[s] < 1 || kind[s] > 1) return HPL_ERR_INVALID;
        cost[s] = system_cost(n[s], kind[s]);
    }
    std::vector<int64_t> order((size_t)count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
    std::vector<double> load((size_t)world, 0.0);
    for (int64_t s : order) {
        int32_t best = 0;
        for (int32_t r = 1; r < world; r++)
            if (load[r] < load[best]) best = r;
        owner[s] = best;
        load[best] += cost[s];
    }
    return HPL_OK;
}

namespace hplgb {
namespace bt {
void remember_plan(const void* ws, int nb_max);
}  // namespace bt
}  // namespace hplgb

extern "C" size_t solve_batched_workspace_size(int64_t count, const int64_t* n, const uint8_t* kind) {
    if (count <= 0 || !n || !kind) return 256;
    return batched_ws_layout(count, n, kind, nullptr);
}

extern "C" int solve_batched_plan(int64_t count, const int64_t* n, double* const* A, const int64_t* lda,
                                  double* const* B, int32_t* const* ipiv, const uint8_t* kind, const uint8_t* variant,
                                  const hpl_opts* opts, void* ws, size_t ws_bytes) {
    if (count <= 0 || count > 0x7fffffff || !n || !A || !lda || !B || !kind || !ws) return HPL_ERR_INVALID;
    for (int64_t s = 0; s < count; s++) {
        if (n[s] < 1 || n[s] > bt::NMAX || lda[s] < n[s] || !A[s] || !B[s] || kind[s] > 1) return HPL_ERR_INVALID;
        if (kind[s] == 0 && (!ipiv || !ipiv[s])) return HPL_ERR_INVALID;
        if (variant && variant[s] > 1) return HPL_ERR_INVALID;
    }
    std::vector<size_t> offs;
    size_t need = batched_ws_layout(count, n, kind, &offs);
    if (ws_bytes < need) return HPL_ERR_NOMEM;
    if ((uintptr_t)ws & 255) return HPL_ERR_INVALID;
    Opts o = resolve_opts(opts, bt::NBMAX);
    // longest first
    // general systems first, then dominant ones, each list longest first
    std::vector<double> cost((size_t)count);
    for (int64_t s = 0; s < count; s++) cost[s] = system_cost(n[s], kind[s]);
    std::vector<int64_t> order((size_t)count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        if (kind[a] != kind[b]) return kind[a] < kind[b];
        return cost[a] > cost[b];
    });
    int64_t count0 = 0;
    for (int64_t s = 0; s < count; s++) count0 += kind[s] == 0;
    std::vector<bt::Sys> table((size_t)count);
    char* base = (char*)ws;
    for (int64_t q = 0; q < count; q++) {
        int64_t s = order[q];
        bt::Sys& S = table[q];
        memset(&S, 0, sizeof(S));
        S.n = n[s];
        S.lda = lda[s];
        S.A = A[s];
        S.b = B[s];
        S.ipiv = kind[s] == 0 ? ipiv[s] : nullptr;
        S.kind = kind[s];
        S.pad = (int)s;                     // original index: infos are written in the caller's order
        S.variant = variant ? variant[s] : 0;
        if (kind[s] == 1) {
            int64_t m = n[s];
            size_t off = offs[s];
            S.W = (float*)(base + off);
            off = align_up(off + sizeof(float) * m * m, 256);
            S.Dinv = (float*)(base + off);
            off = align_up(off + sizeof(float) * m * bt::NBMAX, 256);
            S.r = (double*)(base + off);
            off = align_up(off + sizeof(double) * 2 * m, 256);
            S.y32 = (float*)(base + off);
        }
    }
    bt::Header h;
    memset(&h, 0, sizeof(h));
    h.count = (int)count;
    h.count0 = (int)count0;
    h.max_iter = o.max_iter;
    h.tol = o.tol;
    h.nb_max = 16;
    for (int64_t s = 0; s < count; s++)
        if (!variant || variant[s] == 0) h.nb_max = bt::NBMAX;
    bt::remember_plan(ws, h.nb_max);
    HPL_CUDA_TRY(cudaMemcpy(base, &h, sizeof(h), cudaMemcpyHostToDevice));
    HPL_CUDA_TRY(cudaMemcpy(base + align_up(sizeof(bt::Header), 256), table.data(), sizeof(bt::Sys) * count,
                            cudaMemcpyHostToDevice));
    return HPL_OK;
}

namespace hplgb {
namespace bt {
// Table entries carry the caller's index in `pad`; the kernel writes infos there.
// NBR is the widest panel the launch handles; MINB CTAs share an SM.
template <int NBR, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_batched_run(const Sys* __restrict__ table, Header* H,
                                                               hpl_info* infos);

// The widest panel of each planned workspace (host side), so that the run
// launch picks its kernel without reading the device: a plan whose systems all
// use 16-wide panels runs two CTAs per SM (79 KB of shared memory each),
// otherwise one (the 32-wide panel takes 164 KB). A workspace that was not
// planned in this process gets the one-per-SM kernel, which handles both.
std::mutex g_plan_mu;
std::vector<std::pair<const void*, int>> g_plan_nb;
int g_residency_mode = 0;           // hplgb_batched_config: 0 auto, 1 always one CTA per SM

void remember_plan(const void* ws, int nb_max) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto& e : g_plan_nb)
        if (e.first == ws) { e.second = nb_max; return; }
    if (g_plan_nb.size() >= 64) g_plan_nb.erase(g_plan_nb.begin());
    g_plan_nb.emplace_back(ws, nb_max);
}
int planned_nb(const void* ws) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto& e : g_plan_nb)
        if (e.first == ws) return e.second;
    return NBMAX;
}
}  // namespace bt
}  // namespace hplgb

extern "C" int solve_batched_run(void* ws, hpl_info* infos, int max_ctas, void* stream) {
    if (!ws || !infos) return HPL_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    bt::Header* H = (bt::Header*)base;
    const bt::Sys* table = (const bt::Sys*)(base + align_up(sizeof(bt::Header), 256));
    static std::atomic<bool> attr[kMaxDevices];
    const int dv = device_slot();
    if (dv < 0) return HPL_ERR_CUDA;
    if (!attr[dv].load()) {
        HPL_CUDA_TRY(cudaFuncSetAttribute((const void*)bt::k_batched_run<bt::NBMAX, 1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)bt::smem_bytes<bt::NBMAX>()));
        HPL_CUDA_TRY(cudaFuncSetAttribute((const void*)bt::k_batched_run<16, 2>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt::smem_bytes<16>()));
        attr[dv].store(true);
    }
    int dev = 0, sms = kNumSMsGB300;
    HPL_CUDA_TRY(cudaGetDevice(&dev));
    HPL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool narrow = bt::planned_nb(ws) == 16 && bt::g_residency_mode == 0;
    const int per_sm = narrow ? 2 : 1;
    int grid = max_ctas > 0 ? std::min(max_ctas, per_sm * sms) : per_sm * sms;
    HPL_CUDA_TRY(cudaMemsetAsync(H->counter, 0, sizeof(H->counter), s));
    HPL_CUDA_TRY(cudaMemsetAsync(H->sm_slot, 0, sizeof(H->sm_slot), s));
    if (narrow)
        bt::k_batched_run<16, 2><<<grid, bt::THREADS, bt::smem_bytes<16>(), s>>>(table, H, infos);
    else
        bt::k_batched_run<bt::NBMAX, 1><<<grid, bt::THREADS, bt::smem_bytes<bt::NBMAX>(), s>>>(table, H, infos);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

extern "C" int solve_batched(int64_t count, const int64_t* n, double* const* A, const int64_t* lda,
                             double* const* B, int32_t* const* ipiv, const uint8_t* kind, const uint8_t* variant,
                             const hpl_opts* opts, void* ws, size_t ws_bytes, hpl_info* infos, void* stream) {
    int st = solve_batched_plan(count, n, A, lda, B, ipiv, kind, variant, opts, ws, ws_bytes);
    if (st) return st;
    return solve_batched_run(ws, infos, 0, stream);
}

namespace hplgb {
namespace bt {
template <int NBR, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_batched_run(const Sys* __restrict__ table, Header* H,
                                                               hpl_info* infos) {
    extern __shared__ double bsm[];
    __shared__ double red[THREADS / 32 + 1];
    __shared__ long long redk[THREADS / 32 + 1];
    __shared__ long long redi[THREADS / 32 + 1];
    __shared__ int s_idx;
    double* P = bsm;
    double* Us = bsm + NMAX * panel_stride<NBR>();
    float* X = (float*)(Us + NBR * 65);
    float* R = X + NBR * NBR;
    float* T = R + NBR * NBR;
    __shared__ int s_pref;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        s_pref = (int)(atomicAdd(&H->sm_slot[smid % kMaxSmSlots], 1u) & 1u);
    }
    __syncthreads();
    const int pref = s_pref;
    const int lo[2] = {0, H->count0}, sz[2] = {H->count0, H->count - H->count0};
    for (;;) {
        if (threadIdx.x == 0) {
            int idx = -1;
            for (int q = 0; q < 2 && idx < 0; q++) {
                const int l = pref ^ q;
                if (sz[l] > 0 && (int)*(volatile unsigned int*)&H->counter[l] < sz[l]) {
                    const int t = (int)atomicAdd(&H->counter[l], 1u);
                    if (t < sz[l]) idx = lo[l] + t;
                }
            }
            s_idx = idx;
        }
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx < 0) break;
        const Sys S = table[idx];
        hpl_info* info = infos + S.pad;
        if (threadIdx.x == 0) {
            info->status = 0;
            info->iters = 0;
            info->info = 0;
            info->scaled_residual = 0.0;
            info->inner_iters = 0;
        }
        __syncthreads();
        if (S.kind == 0) {
            if constexpr (NBR == 16) {
                lu64<16>(S, P, Us, redk, redi, info);
            } else {
                if (S.variant) lu64<16>(S, P, Us, redk, redi, info);
                else lu64<32>(S, P, Us, redk, redi, info);
            }
        } else {
            // the FP64 panel area is free in this path: bf16 operand copies
            if constexpr (NBR == 16) {
                mxp_one<16>(S, H, X, R, T, (float*)P, red, info);
            } else {
                if (S.variant) mxp_one<16>(S, H, X, R, T, (float*)P, red, info);
                else mxp_one<32>(S, H, X, R, T, (float*)P, red, info);
            }
        }
        __syncthreads();
    }
}
template __global__ void k_batched_run<NBMAX, 1>(const Sys* __restrict__, Header*, hpl_info*);
template __global__ void k_batched_run<16, 2>(const Sys* __restrict__, Header*, hpl_info*);
}  // namespace bt
}  // namespace hplgb

extern "C" int hplgb_batched_config(int what, long long value) {
    if (what != 0 || value < 0 || value > 1) return HPL_ERR_INVALID;
    hplgb::bt::g_residency_mode = (int)value;
    return HPL_OK;
}
