// lu_solve: the triangular solves that follow the factorization (paper
// Sec. III-A.1), FP64.
//
// Interchanges: the pivot vector is cut into blocks of 256; one warp per block
// turns its sequential swaps into (dst, src) pairs (done in parallel for all
// blocks), then one CTA per right-hand side applies the blocks in order
// (reverse order, inverse pairs, for the transposed solve).
// Triangles, one right-hand side without transpose: both in one persistent
// launch (k_trsv_wave, below). Otherwise blocked substitution with 64-row
// diagonal blocks: a diagonal block is solved by one warp per right-hand side
// with shuffles; the rows below (forward) or above (backward) are then
// updated by a GEMV/GEMM kernel.
#include <algorithm>

#include "common.cuh"

namespace hplgb {

constexpr int kPivBlock = 256;
constexpr int kTB = 64;   // diagonal block of the substitution

// Defined in lu64.cu.
__global__ void k_perm_pairs(const int32_t* __restrict__ ipiv, int64_t k0_base, int pb, int64_t n_end,
                             int64_t n_total, int* __restrict__ cnt, int* __restrict__ dst, int* __restrict__ src);

__global__ void __launch_bounds__(512) k_apply_perm(int64_t n, int nblk, const int* __restrict__ cnt,
                                                    const int* __restrict__ dst, const int* __restrict__ src,
                                                    int reverse, double* __restrict__ B, int64_t ldb) {
    double* b = B + (int64_t)blockIdx.x * ldb;
    for (int q = 0; q < nblk; q++) {
        const int blk = reverse ? nblk - 1 - q : q;
        const int np = cnt[blk];
        const int* d = dst + (int64_t)blk * 2 * kPivBlock;
        const int* s = src + (int64_t)blk * 2 * kPivBlock;
        double v = 0.0;
        const int t = threadIdx.x;
        if (t < np) v = b[reverse ? d[t] : s[t]];
        __syncthreads();
        if (t < np) b[reverse ? s[t] : d[t]] = v;
        __syncthreads();
    }
}

// T(i, j) of the triangle being solved: trans = 0 reads LU(i, j), trans = 1
// reads LU(j, i).
__device__ __forceinline__ double tri_at(const double* LU, int64_t lda, int64_t i, int64_t j, int trans) {
    return trans ? LU[i * lda + j] : LU[j * lda + i];
}

// Diagonal block [b0, b0+bs) (bs <= 64): lower = forward substitution, else
// backward; unit = implicit ones on the diagonal. One warp per RHS column;
// lane l holds rows l and l+32 of the block.
__global__ void __launch_bounds__(256) k_trsv_diag(const double* __restrict__ LU, int64_t lda, int64_t b0, int bs,
                                                   int lower, int unit, int trans, double* __restrict__ B,
                                                   int64_t ldb, int64_t nrhs) {
    __shared__ double Ts[kTB][kTB + 1];
    for (int idx = threadIdx.x; idx < bs * bs; idx += blockDim.x) {
        int a = idx / bs, c = idx - a * bs;
        int i = trans ? a : c, j = trans ? c : a;        // coalesced along the contiguous index
        Ts[i][j] = tri_at(LU, lda, b0 + i, b0 + j, trans);
    }
    // reciprocals of the diagonal, all at once: the substitution then multiplies
    // (one FP64 division is a chain of FP64 instructions, scarce on this part)
    __shared__ double Tinv[kTB];
    __syncthreads();
    if (!unit && threadIdx.x < bs) Tinv[threadIdx.x] = 1.0 / Ts[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = warp; c < nrhs; c += blockDim.x / 32) {
        double* b = B + c * ldb + b0;
        double y[2];
        y[0] = lane < bs ? b[lane] : 0.0;
        y[1] = lane + 32 < bs ? b[lane + 32] : 0.0;
        if (lower) {
            for (int j = 0; j < bs; j++) {
                const int hj = j >> 5, lj = j & 31;
                if (!unit && lane == lj) y[hj] = y[hj] * Tinv[j];
                const double xj = __shfl_sync(0xffffffffu, y[hj], lj);
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    int i = lane + 32 * h;
                    if (i > j && i < bs) y[h] = fma(-Ts[i][j], xj, y[h]);
                }
            }
        } else {
            for (int j = bs - 1; j >= 0; j--) {
                const int hj = j >> 5, lj = j & 31;
                if (!unit && lane == lj) y[hj] = y[hj] * Tinv[j];
                const double xj = __shfl_sync(0xffffffffu, y[hj], lj);
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    int i = lane + 32 * h;
                    if (i < j) y[h] = fma(-Ts[i][j], xj, y[h]);
                }
            }
        }
        if (lane < bs) b[lane] = y[0];
        if (lane + 32 < bs) b[lane + 32] = y[1];
    }
}

// Rows [r_beg, r_end) -= T(rows, b0:b0+bs) * X(b0:b0+bs, :). One CTA per 64
// rows; the T tile and the block of X are staged in shared memory.
__global__ void __launch_bounds__(256) k_trsv_update(const double* __restrict__ LU, int64_t lda, int64_t b0, int bs,
                                                     int trans, int64_t r_beg, int64_t r_end, double* __restrict__ B,
                                                     int64_t ldb, int64_t nrhs) {
    __shared__ double Ts[kTB][kTB + 1];
    __shared__ double Xs[kTB][kTB + 1];
    const int64_t r0 = r_beg + (int64_t)blockIdx.x * kTB;
    const int rows = (int)std::min<int64_t>(kTB, r_end - r0);
    for (int idx = threadIdx.x; idx < rows * bs; idx += blockDim.x) {
        int a, c;
        if (trans) { a = idx / bs; c = idx - a * bs; }   // a = row, c = column: contiguous c
        else { c = idx / rows; a = idx - c * rows; }     // contiguous rows
        Ts[a][c] = tri_at(LU, lda, r0 + a, b0 + c, trans);
    }
    for (int64_t c0 = 0; c0 < nrhs; c0 += kTB) {
        const int nc = (int)std::min<int64_t>(kTB, nrhs - c0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < bs * nc; idx += blockDim.x) {
            int c = idx / bs, j = idx - c * bs;
            Xs[j][c] = B[(c0 + c) * ldb + b0 + j];
        }
        __syncthreads();
        const int r = threadIdx.x & 63;
        for (int c = threadIdx.x >> 6; c < nc; c += 4) {
            if (r < rows) {
                double s = 0.0;
                for (int j = 0; j < bs; j++) s = fma(Ts[r][j], Xs[j][c], s);
                double* p = B + (c0 + c) * ldb + r0 + r;
                *p = *p - s;
            }
        }
    }
}

__global__ void k_check_udiag(int64_t n, const double* __restrict__ LU, int64_t lda, hpl_info* info) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (LU[i * lda + i] == 0.0) info->status = HPL_ERR_SINGULAR;
}

// Workspace: the interchange pairs, then for the one-launch solve of a single
// right-hand side its published blocks (y, then x: 64 values per row block
// each) and its abort word.
struct SolveWs {
    int* cnt;
    int* dst;
    int* src;
    double* pub;
    int* abort_flag;
};
static size_t solve_ws_layout(int64_t n, SolveWs* w, char* base) {
    const int64_t nblk = (n + kPivBlock - 1) / kPivBlock;
    const int64_t tblk = (n + kTB - 1) / kTB;
    size_t off = 0;
    size_t o_cnt = off; off = align_up(off + sizeof(int) * nblk, 256);
    size_t o_dst = off; off = align_up(off + sizeof(int) * nblk * 2 * kPivBlock, 256);
    size_t o_src = off; off = align_up(off + sizeof(int) * nblk * 2 * kPivBlock, 256);
    size_t o_y = off; off = align_up(off + sizeof(double) * 2 * tblk * kTB, 256);
    size_t o_f = off; off = align_up(off + sizeof(int), 256);
    if (base) {
        w->cnt = (int*)(base + o_cnt);
        w->dst = (int*)(base + o_dst);
        w->src = (int*)(base + o_src);
        w->pub = (double*)(base + o_y);
        w->abort_flag = (int*)(base + o_f);
    }
    return std::max<size_t>(off, 256);
}

// ---------------------------------------------------------------------------
// Both triangles for one right-hand side (no transpose, P b applied) in one
// persistent launch: the dependent chain of 2 * nblk diagonal blocks no longer
// pays a kernel launch per block, and every SM's FP64 pipe works on the
// off-diagonal products (on this part the FP64 rate, not HBM, bounds them).
//
// Row blocks of 64 are dealt round-robin to the G co-resident CTAs (CTA c owns
// blocks q_k = c + k G). Forward sweep: column blocks j = 0, 1, ... in order;
// a CTA multiplies y_j into every owned block below j (per-thread partial sums
// in shared memory, 16 columns of the tile each), and as soon as column q - 1
// has reached its next block q it finishes that block first: r = b_q - sum,
// y_q = inv(L_qq) r, published before the remaining products of column j. The
// backward sweep runs the same way from the last block with inv(U_qq). The
// inverses of the owned diagonal blocks are formed in shared memory in the
// CTA's slack (the first at the start), so a step of the chain is two 64 x 64
// products spread over all warps instead of a 64-deep serial substitution.
// Every partial sum runs over the columns in the same order whatever G is, so
// the result does not depend on the grid size.
//
// Publication without flags: the buffers of published blocks (y, then x) are
// filled with the all-ones bit pattern (a NaN no arithmetic result has, since
// a published value with that pattern is replaced by the canonical NaN) before
// the launch; a solved value is one 8-byte store, and a reader takes its 16
// values of a column once none of them holds the pattern (relaxed loads, each
// value written once). Each thread reads its values of the next column ahead
// of need, so a CTA that runs behind the front never waits on memory latency.
// Waits are bounded: after timeout_ns a waiting thread raises the shared abort
// word (and info->status = HPL_ERR_TIMEOUT); every other waiter sees it, and
// the CTA returns at its next barrier.
constexpr int kWaveThreads = 256;
constexpr int kWaveUEarly = 12;        // CTAs from here on invert their last U block before the forward
                                       // sweep (about 3 us per block reaches CTA c after c blocks; an
                                       // inverse takes about 33 us)
constexpr int kInvLd = kTB + 1;
constexpr unsigned long long kWaveEmpty = ~0ull;   // bit pattern of a block not yet published

int g_solve_wave = 1;                  // single right-hand side: 1 wavefront kernel, 0 per-block launches
int g_solve_wave_grid = 0;             // CTAs of the wavefront kernel (0: one per SM)

__device__ __forceinline__ void ld_relaxed_v2(const double* p, double& a, double& b) {
    asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool wave_empty(double v) {
    return (unsigned long long)__double_as_longlong(v) == kWaveEmpty;
}
// a published value never carries the empty pattern
__device__ __forceinline__ double wave_canon(double v) {
    return wave_empty(v) ? __longlong_as_double(0x7ff8000000000000LL) : v;
}

// This thread's 16 values of a published block (p 16-byte aligned): keeps
// re-reading until none holds the empty pattern. v may hold values read
// earlier. Returns false on timeout or abort.
__device__ bool wave_fetch(const double* p, double (&v)[16], int* abort_flag, uint64_t deadline, hpl_info* info) {
    for (uint32_t it = 0;; it++) {
        bool full = true;
#pragma unroll
        for (int c = 0; c < 16; c++) full = full && !wave_empty(v[c]);
        if (full) return true;
        if ((it & 63) == 63) {
            if (ld_relaxed_s32(abort_flag)) return false;
            if (globaltimer_ns() > deadline) {
                atomicExch(abort_flag, 1);
                if (info) info->status = HPL_ERR_TIMEOUT;
                return false;
            }
        }
#pragma unroll
        for (int c = 0; c < 8; c++) ld_relaxed_v2(p + 2 * c, v[2 * c], v[2 * c + 1]);
    }
}

// Inverse of the 64 x 64 diagonal block of LU at (b0, b0), rows and columns
// >= bs taken as the identity: lower = the unit lower factor (its stored
// diagonal belongs to U), else the upper factor U. Column sweep in place in
// X = inv[64][kInvLd], one step (and one barrier) per pivot k, the step's
// whole rectangle of updates dealt over all threads (lanes run along a row:
// on this part a warp-wide DFMA costs the same however few lanes are active).
//   lower, k = 0 .. 62:  X(i, e) -= L(i, k) X(k, e), i > k, e <= k
//   upper, k = 63 .. 1:  X(i, e) -= U(i, k) X(k, e), i < k, e >= k, and row
//                        k - 1, final after this step, is scaled by 1 / U(k-1, k-1)
// X(k, k) is 1 (lower) or 1 / U(k, k) (upper) and X(i, k) starts from zero;
// column k of the factor, overwritten by its own step, is saved a step ahead
// (colbuf, double buffered).
__device__ void wave_block_inverse(const double* __restrict__ LU, int64_t lda, int64_t b0, int bs, bool lower,
                                   double* X, double* colbuf, double* rinv) {
    const int t = threadIdx.x;
    for (int idx = t; idx < kTB * kTB; idx += kWaveThreads) {
        const int e = idx >> 6, i = idx & 63;       // coalesced along the column
        double v = (i < bs && e < bs) ? LU[(b0 + e) * lda + b0 + i] : (i == e ? 1.0 : 0.0);
        if (lower ? e > i : e < i) v = 0.0;
        else if (lower && e == i) v = 1.0;
        X[i * kInvLd + e] = v;
    }
    __syncthreads();
    if (!lower) {
        if (t < kTB) rinv[t] = 1.0 / X[t * kInvLd + t];
        __syncthreads();
        if (t < kTB - 1) colbuf[t] = X[t * kInvLd + kTB - 1];
        if (t == kTB - 1) X[t * kInvLd + t] = rinv[t];
    } else {
        if (t > 0 && t < kTB) colbuf[t] = X[t * kInvLd];
    }
    __syncthreads();
    for (int st = 0; st < kTB - 1; st++) {
        const int k = lower ? st : kTB - 1 - st;
        const double* cb = colbuf + (st & 1) * kTB;
        double* cbn = colbuf + ((st + 1) & 1) * kTB;
        const int C = lower ? k + 1 : kTB - k;          // columns of the rectangle
        const int cnt = (lower ? kTB - 1 - k : k) * C;
        const double* xk = X + k * kInvLd;
        const double rs = lower ? 1.0 : rinv[k - 1];
        for (int idx = t; idx < cnt; idx += kWaveThreads) {
            const int r = idx / C, cc = idx - r * C;
            const int i = lower ? k + 1 + r : r;
            const int e = lower ? cc : k + cc;
            double v = e == k ? 0.0 : X[i * kInvLd + e];
            v = fma(-cb[i], xk[e], v);
            if (!lower && i == k - 1) v *= rs;
            X[i * kInvLd + e] = v;
        }
        // the next step's column (its entries are untouched by this step) and,
        // upper, the next diagonal entry
        if (lower) {
            if (t > k + 1 && t < kTB) cbn[t] = X[t * kInvLd + k + 1];
        } else {
            if (t < k - 1) cbn[t] = X[t * kInvLd + k - 1];
            else if (t == k - 1) X[t * kInvLd + t] = rs;
        }
        __syncthreads();
    }
}

// out[t] (t < 64) = inv * rvec: thread (i, g) sums 16 columns, the four
// partial sums are added in a fixed order.
__device__ __forceinline__ double wave_apply_inverse(const double* inv, const double* rvec, double* part) {
    const int t = threadIdx.x, i = t & 63, g = t >> 6;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 16; c++) s = fma(inv[i * kInvLd + 16 * g + c], rvec[16 * g + c], s);
    part[g * kTB + i] = s;
    __syncthreads();
    return t < kTB ? (part[t] + part[kTB + t]) + (part[2 * kTB + t] + part[3 * kTB + t]) : 0.0;
}

__device__ __forceinline__ void wave_cp8(double* smem, const double* gmem, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void wave_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wave_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kWaveTile = kTB * kTB;   // doubles of one staged tile

// Shared memory of k_trsv_wave: two inverses, small vectors, S staged tiles,
// and per owned block 256 partial sums and 64 values of b / y.
__host__ __device__ constexpr size_t wave_smem_doubles(int R, int S) {
    return (size_t)2 * kTB * kInvLd + kTB + 4 * kTB + 2 * kTB + kTB + (size_t)S * kWaveTile +
           (size_t)R * (kWaveThreads + kTB);
}

// S - 1 tiles in flight: tile (q, j) of a task is copied S - 1 tasks ahead by
// cp.async, each thread its own 16 elements (the ones it multiplies), so no
// barrier guards the ring.
template <int S>
__global__ void __launch_bounds__(kWaveThreads, 1)
k_trsv_wave(int64_t n, const double* __restrict__ LU, int64_t lda, double* __restrict__ b,
            double* __restrict__ ybuf, double* __restrict__ xbuf, int* __restrict__ abort_flag, hpl_info* info,
            int64_t timeout_ns) {
    extern __shared__ __align__(16) double wsm[];
    const int t = threadIdx.x, i = t & 63, g = t >> 6;
    const int G = (int)gridDim.x, c = (int)blockIdx.x;
    const int nblk = (int)((n + kTB - 1) / kTB);
    const int R = c < nblk ? (nblk - 1 - c) / G + 1 : 0;
    if (R == 0) return;
    double* inv_l = wsm;
    double* inv_u = inv_l + kTB * kInvLd;
    double* rvec = inv_u + kTB * kInvLd;
    double* part = rvec + kTB;
    double* colbuf = part + 4 * kTB;
    double* rinv = colbuf + 2 * kTB;
    double* ring = rinv + kTB;               // [S][16][256]: element cc of thread t at cc * 256 + t
    double* accp = ring + S * kWaveTile;     // [R][256] per-thread partial sums
    double* yown = accp + R * kWaveThreads;  // [R][64] b, then the forward results, of the owned blocks
    const uint64_t deadline = globaltimer_ns() + (uint64_t)timeout_ns;
    bool dead = false;                       // a wait of this thread gave up
    auto q_of = [&](int k) { return c + k * G; };
    auto bs_of = [&](int q) { return (int)std::min<int64_t>(kTB, n - (int64_t)q * kTB); };
    // first owned block below column block j / last owned block above it
    auto first_f = [&](int j) { return j < c ? 0 : (j - c) / G + 1; };
    auto last_b = [&](int j) { return j > c ? std::min(R - 1, (j - c - 1) / G) : -1; };
    // tile (q, j) into a ring slot: rows q*64 + i, columns j*64 + 16 g + cc (zero outside n)
    auto issue_tile = [&](int slot, int q, int j) {
        const int64_t row = (int64_t)q * kTB + i;
        const int64_t col = (int64_t)j * kTB + 16 * g;
        double* dst = ring + slot * kWaveTile + t;
#pragma unroll
        for (int cc = 0; cc < 16; cc++) {
            const bool ok = row < n && col + cc < n;
            wave_cp8(dst + cc * kWaveThreads, ok ? LU + (col + cc) * lda + row : LU, ok);
        }
    };

    wave_block_inverse(LU, lda, (int64_t)q_of(0) * kTB, bs_of(q_of(0)), true, inv_l, colbuf, rinv);
    const bool u_early = c >= kWaveUEarly || q_of(R - 1) == nblk - 1;
    if (u_early)
        wave_block_inverse(LU, lda, (int64_t)q_of(R - 1) * kTB, bs_of(q_of(R - 1)), false, inv_u, colbuf, rinv);
    for (int k = 0; k < R; k++) {
        accp[k * kWaveThreads + t] = 0.0;
        if (t < kTB) {                       // b of the owned blocks, off the chain of dependent steps
            const int64_t row = (int64_t)q_of(k) * kTB + t;
            yown[k * kTB + t] = row < n ? b[row] : 0.0;
        }
    }

    // forward block k: y = inv(L_qq) (b_q - sum), published; then the
    // inverses this CTA needs next. False: a wait in this CTA gave up.
    auto solve_fwd = [&](int k) -> bool {
        const int q = q_of(k);
        if (__syncthreads_or(dead)) return false;
        if (t < kTB) {
            const double* a = accp + k * kWaveThreads;
            rvec[t] = yown[k * kTB + t] - ((a[t] + a[kTB + t]) + (a[2 * kTB + t] + a[3 * kTB + t]));
        }
        __syncthreads();
        const double y = wave_apply_inverse(inv_l, rvec, part);
        if (t < kTB) {
            yown[k * kTB + t] = y;
            st_relaxed_f64(ybuf + (int64_t)q * kTB + t, wave_canon(y));
        }
        if (k == 0 && !u_early)
            wave_block_inverse(LU, lda, (int64_t)q_of(R - 1) * kTB, bs_of(q_of(R - 1)), false, inv_u, colbuf, rinv);
        if (k + 1 < R)
            wave_block_inverse(LU, lda, (int64_t)q_of(k + 1) * kTB, bs_of(q_of(k + 1)), true, inv_l, colbuf, rinv);
        return true;
    };
    // backward block k: x = inv(U_qq) (y_q - sum), published and written into b
    auto solve_bwd = [&](int k) -> bool {
        const int q = q_of(k);
        if (__syncthreads_or(dead)) return false;
        if (t < kTB) {
            const double* a = accp + k * kWaveThreads;
            rvec[t] = yown[k * kTB + t] - ((a[t] + a[kTB + t]) + (a[2 * kTB + t] + a[3 * kTB + t]));
        }
        __syncthreads();
        const double x = wave_apply_inverse(inv_u, rvec, part);
        if (t < kTB) {
            st_relaxed_f64(xbuf + (int64_t)q * kTB + t, wave_canon(x));
            if ((int64_t)q * kTB + t < n) b[(int64_t)q * kTB + t] = x;
        }
        if (k > 0)
            wave_block_inverse(LU, lda, (int64_t)q_of(k - 1) * kTB, bs_of(q_of(k - 1)), false, inv_u, colbuf, rinv);
        return true;
    };

    double yv[16], yn[16];
    // this thread's 16 values of published block j of buf, read ahead into yn
    auto read_ahead = [&](const double* buf, int j) {
        const double* p = buf + (int64_t)j * kTB + 16 * g;
#pragma unroll
        for (int cc = 0; cc < 8; cc++) ld_relaxed_v2(p + 2 * cc, yn[2 * cc], yn[2 * cc + 1]);
    };

    // ---- forward: L y = b ----
    if (q_of(0) == 0 && !solve_fwd(0)) return;
    {
        int k = first_f(0), j = 0;           // task multiplied next
        int pk = k, pj = j, issued = 0;      // task copied next
        auto step_f = [&](int& kk, int& jj) {
            if (++kk >= R) kk = first_f(++jj);
        };
        for (int s2 = 0; s2 < S - 1; s2++, issued++) {
            if (pk < R) {
                issue_tile(issued % S, q_of(pk), pj);
                step_f(pk, pj);
            }
            wave_cp_commit();
        }
        if (k < R) read_ahead(ybuf, j);
        for (int done = 0; k < R; done++, issued++) {
            if (pk < R) {
                issue_tile(issued % S, q_of(pk), pj);
                step_f(pk, pj);
            }
            wave_cp_commit();
            const bool first = k == first_f(j);
            if (first) {
#pragma unroll
                for (int cc = 0; cc < 16; cc++) yv[cc] = yn[cc];
                if (!dead && !wave_fetch(ybuf + (int64_t)j * kTB + 16 * g, yv, abort_flag, deadline, info))
                    dead = true;
                if (first_f(j + 1) < R) read_ahead(ybuf, j + 1);
            }
            wave_cp_wait<S - 1>();
            const double* tile = ring + (done % S) * kWaveTile + t;
            double p = accp[k * kWaveThreads + t];
#pragma unroll
            for (int cc = 0; cc < 16; cc++) p = fma(tile[cc * kWaveThreads], yv[cc], p);
            accp[k * kWaveThreads + t] = p;
            if (first && q_of(k) == j + 1 && !solve_fwd(k)) {
                wave_cp_wait<0>();           // no copy outlives the CTA
                return;
            }
            step_f(k, j);
        }
        wave_cp_wait<0>();
    }
    if (__syncthreads_or(dead)) return;

    // ---- backward: U x = y ----
    for (int k = 0; k < R; k++) accp[k * kWaveThreads + t] = 0.0;
    if (q_of(R - 1) == nblk - 1 && !solve_bwd(R - 1)) return;
    {
        int k = last_b(nblk - 1), j = nblk - 1;
        int pk = k, pj = j, issued = 0;
        auto step_b = [&](int& kk, int& jj) {
            if (--kk < 0) kk = last_b(--jj);
        };
        for (int s2 = 0; s2 < S - 1; s2++, issued++) {
            if (pk >= 0) {
                issue_tile(issued % S, q_of(pk), pj);
                step_b(pk, pj);
            }
            wave_cp_commit();
        }
        if (k >= 0) read_ahead(xbuf, j);
        for (int done = 0; k >= 0; done++, issued++) {
            if (pk >= 0) {
                issue_tile(issued % S, q_of(pk), pj);
                step_b(pk, pj);
            }
            wave_cp_commit();
            const bool first = k == last_b(j);
            if (first) {
#pragma unroll
                for (int cc = 0; cc < 16; cc++) yv[cc] = yn[cc];
                if (!dead && !wave_fetch(xbuf + (int64_t)j * kTB + 16 * g, yv, abort_flag, deadline, info))
                    dead = true;
                // columns beyond n (the last block's padding) take no part
                const int64_t col = (int64_t)j * kTB + 16 * g;
#pragma unroll
                for (int cc = 0; cc < 16; cc++)
                    if (col + cc >= n) yv[cc] = 0.0;
                if (last_b(j - 1) >= 0) read_ahead(xbuf, j - 1);
            }
            wave_cp_wait<S - 1>();
            const double* tile = ring + (done % S) * kWaveTile + t;
            double p = accp[k * kWaveThreads + t];
#pragma unroll
            for (int cc = 0; cc < 16; cc++) p = fma(tile[cc * kWaveThreads], yv[cc], p);
            accp[k * kWaveThreads + t] = p;
            if (first && q_of(k) == j - 1 && !solve_bwd(k)) {
                wave_cp_wait<0>();
                return;
            }
            step_b(k, j);
        }
        wave_cp_wait<0>();
    }
}

// Opt-in shared memory per CTA of the current device (0 on error).
static size_t wave_smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (size_t)v;
}

// Ring depth for R owned blocks: 4 when it fits, else 3, else 2 (0: the
// kernel does not fit).
static int wave_stages(int64_t R, size_t limit) {
    for (int S : {4, 3, 2})
        if (wave_smem_doubles((int)R, S) * sizeof(double) <= limit) return S;
    return 0;
}

template <int S>
static const void* wave_fn() {
    return (const void*)k_trsv_wave<S>;
}

// Co-resident CTAs of k_trsv_wave (one per SM; 0 = unavailable), cached per
// device; raises every variant's shared-memory limit to the device's.
static int wave_max_ctas(size_t limit) {
    static std::atomic<int> cache[kMaxDevices];      // CTAs + 1; 0: not yet known
    const int dv = device_slot();
    if (dv < 0) return 0;
    if (const int v = cache[dv].load()) return v - 1;
    int best = 0, dev = 0, sms = 0;
    bool ok = limit > 0 && cudaGetDevice(&dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    for (const void* f : {wave_fn<4>(), wave_fn<3>(), wave_fn<2>()}) {
        int per = 0;
        ok = ok && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) == cudaSuccess &&
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, kWaveThreads, limit) == cudaSuccess && per >= 1;
    }
    if (ok) best = sms;                               // one CTA per SM
    cudaGetLastError();
    cache[dv].store(best + 1);
    return best;
}

// One launch for both triangles of one right-hand side; returns -1 (nothing
// launched) when the kernel is unavailable or the matrix has too many blocks.
static int solve_wave(int64_t n, const double* LU, int64_t lda, double* b, double* pub, int* abort_flag,
                      hpl_info* info, cudaStream_t s) {
    const size_t limit = wave_smem_limit();
    const int cmax = wave_max_ctas(limit);
    const int64_t nblk = (n + kTB - 1) / kTB;
    if (cmax < 1) return -1;
    int G = (int)std::min<int64_t>(nblk, cmax);
    if (g_solve_wave_grid > 0) G = std::min(G, g_solve_wave_grid);
    const int64_t R = (nblk + G - 1) / G;
    const int S = wave_stages(R, limit);
    if (S < 2) return -1;
    HPL_CUDA_TRY(cudaMemsetAsync(pub, 0xff, sizeof(double) * (size_t)(2 * nblk * kTB), s));   // kWaveEmpty
    HPL_CUDA_TRY(cudaMemsetAsync(abort_flag, 0, sizeof(int), s));
    const size_t smem = wave_smem_doubles((int)R, S) * sizeof(double);
    double* ybuf = pub;
    double* xbuf = pub + nblk * kTB;
    int64_t timeout_ns = kDefaultTimeoutNs;
    void* args[] = {&n, &LU, &lda, &b, &ybuf, &xbuf, &abort_flag, &info, &timeout_ns};
    const void* f = S == 4 ? wave_fn<4>() : S == 3 ? wave_fn<3>() : wave_fn<2>();
    HPL_CUDA_TRY(cudaLaunchCooperativeKernel(f, dim3((unsigned)G), dim3(kWaveThreads), args, smem, s));
    count_launch();
    return HPL_OK;
}

// One triangle: forward (lower) or backward (upper) blocked substitution.
static int tri_solve(int64_t n, const double* LU, int64_t lda, int lower, int unit, int trans, double* B, int64_t ldb,
                     int64_t nrhs, cudaStream_t s) {
    const int64_t nbk = (n + kTB - 1) / kTB;
    for (int64_t q = 0; q < nbk; q++) {
        const int64_t blk = lower ? q : nbk - 1 - q;
        const int64_t b0 = blk * kTB;
        const int bs = (int)std::min<int64_t>(kTB, n - b0);
        k_trsv_diag<<<1, 256, 0, s>>>(LU, lda, b0, bs, lower, unit, trans, B, ldb, nrhs);
        HPL_LAUNCH_CHECK();
        int64_t rb = lower ? b0 + bs : 0, re = lower ? n : b0;
        if (re > rb) {
            unsigned g = (unsigned)((re - rb + kTB - 1) / kTB);
            k_trsv_update<<<g, 256, 0, s>>>(LU, lda, b0, bs, trans, rb, re, B, ldb, nrhs);
            HPL_LAUNCH_CHECK();
        }
    }
    return HPL_OK;
}

}  // namespace hplgb

using namespace hplgb;

extern "C" size_t lu_solve_workspace_size(int64_t n, int64_t nrhs) {
    (void)nrhs;
    return solve_ws_layout(n > 0 ? n : 1, nullptr, nullptr);
}

extern "C" int lu_solve(int64_t n, int64_t nrhs, const double* LU, int64_t lda, const int32_t* ipiv, int trans,
                        double* B, int64_t ldb, void* ws, size_t ws_bytes, hpl_info* info, void* stream) {
    if (n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return HPL_ERR_INVALID;
    if (trans != 0 && trans != 1) return HPL_ERR_INVALID;
    if (n > 0 && nrhs > 0 && (!LU || !ipiv || !B)) return HPL_ERR_INVALID;
    if (nrhs > 65535) return HPL_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (info) HPL_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(hpl_info), s));
    if (n == 0 || nrhs == 0) return HPL_OK;
    size_t need = solve_ws_layout(n, nullptr, nullptr);
    if (!ws || ws_bytes < need) return HPL_ERR_NOMEM;
    if ((uintptr_t)ws & 255) return HPL_ERR_INVALID;
    SolveWs w;
    solve_ws_layout(n, &w, (char*)ws);
    int *cnt = w.cnt, *dst = w.dst, *src = w.src;
    const int nblk = (int)((n + kPivBlock - 1) / kPivBlock);
    k_perm_pairs<<<nblk, 32, perm_pairs_smem(kPivBlock), s>>>(ipiv, 0, kPivBlock, n, n, cnt, dst, src);
    HPL_LAUNCH_CHECK();
    if (info) {
        k_check_udiag<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(n, LU, lda, info);
        HPL_LAUNCH_CHECK();
    }
    if (!trans) {
        k_apply_perm<<<(unsigned)nrhs, 512, 0, s>>>(n, nblk, cnt, dst, src, 0, B, ldb);
        HPL_LAUNCH_CHECK();
        if (nrhs == 1 && g_solve_wave) {
            int st = solve_wave(n, LU, lda, B, w.pub, w.abort_flag, info, s);
            if (st != -1) return st;
        }
        int st = tri_solve(n, LU, lda, 1, 1, 0, B, ldb, nrhs, s);
        if (st) return st;
        st = tri_solve(n, LU, lda, 0, 0, 0, B, ldb, nrhs, s);
        if (st) return st;
    } else {
        int st = tri_solve(n, LU, lda, 1, 0, 1, B, ldb, nrhs, s);   // U^T z = b
        if (st) return st;
        st = tri_solve(n, LU, lda, 0, 1, 1, B, ldb, nrhs, s);       // L^T w = z
        if (st) return st;
        k_apply_perm<<<(unsigned)nrhs, 512, 0, s>>>(n, nblk, cnt, dst, src, 1, B, ldb);
        HPL_LAUNCH_CHECK();
    }
    return HPL_OK;
}
