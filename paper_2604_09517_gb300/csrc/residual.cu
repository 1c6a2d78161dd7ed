// hpl_scaled_residual: ||Ax - b||_inf / (eps (||A||_inf ||x||_inf + ||b||_inf) n),
// eps = 2^-53, FP64 (the standard HPL acceptance test; the paper prints no
// formula). A is read, or regenerated from the seed (hpl_generate's
// definition) so that very large systems need not keep a copy of A.
//
// Pass 1: grid (row blocks of 256, column chunks); each thread owns one row
// and sums a_ij x_j and |a_ij| over its chunk (deterministic per-chunk
// partials). Pass 2: per row, the chunks are summed in order, b_i is
// subtracted and the maxima are combined with an integer atomicMax on the bit
// patterns of non-negative doubles (order-independent). Pass 3: the quotient.
#include <algorithm>

#include "common.cuh"

namespace hplgb {

constexpr int kResChunks = 16;
#ifndef HPLGB_REGEN_I2F
#define HPLGB_REGEN_I2F 1
#endif

__host__ __device__ __forceinline__ uint64_t res_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double res_u128_to_double(uint64_t hi, uint64_t lo) {
    if (hi == 0) return __ull2double_rn(lo);
    int sh = 64 - __clzll((long long)hi);
    uint64_t top = (sh == 64) ? hi : ((hi << (64 - sh)) | (lo >> sh));
    uint64_t dropped = (sh == 64) ? lo : (lo & ((1ull << sh) - 1));
    top |= (dropped != 0);
    return ldexp(__ull2double_rn(top), sh);
}

struct ResWs {
    double* part_r;      // [chunks][n]
    double* part_a;      // [chunks][n]
    uint64_t* part_lo;   // [chunks][n] (regenerated dominant matrices)
    uint64_t* part_hi;   // [chunks][n]
    unsigned long long* maxima;   // [4]: |r|, row sum, |x|, |b|
};

static size_t res_ws_layout(int64_t n, ResWs* w, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return base ? (void*)(base + o) : (void*)nullptr;
    };
    void* a = take(sizeof(double) * kResChunks * n);
    void* b = take(sizeof(double) * kResChunks * n);
    void* c = take(sizeof(uint64_t) * kResChunks * n);
    void* d = take(sizeof(uint64_t) * kResChunks * n);
    void* e = take(sizeof(unsigned long long) * 4);
    if (w) {
        w->part_r = (double*)a;
        w->part_a = (double*)b;
        w->part_lo = (uint64_t*)c;
        w->part_hi = (uint64_t*)d;
        w->maxima = (unsigned long long*)e;
    }
    return off;
}

// |a| as a float with the mantissa truncated to 23 bits, by integer
// operations only: on this part FP64 arithmetic (2 FMA/clk/SM) bounds an n^2
// FP64 matrix-vector product, so the norm's row sums stay off the FP64 pipe
// (relative error below 2^-23 per term; entries below the FP32 range count 0).
__device__ __forceinline__ float abs_as_float(double a) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
    const int e = (int)(u >> 52) - 1023 + 127;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __int_as_float(0x7f800000);
    return __int_as_float((e << 23) | (int)((u >> 29) & 0x7fffff));
}

// want_norm: 0 skips the row sums of |a_ij| (plain matrix-vector product),
// 1 sums them in FP32 from abs_as_float (the refinement's stopping test),
// 2 sums them in FP64 (the HPL acceptance check).
// A == NULL regenerates the entries from key (hpl_generate's definition); for
// the dominant matrix the diagonal is skipped here and added per row later,
// either from the exact row sums accumulated here (diag == NULL) or from diag.
__global__ void __launch_bounds__(256) k_res_partial(int64_t n, const double* __restrict__ A, int64_t lda,
                                                     uint64_t key, int dominant, const double* __restrict__ diag,
                                                     const double* __restrict__ x, ResWs w, int want_norm) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int chunk = blockIdx.y;
    const int64_t cw = (n + kResChunks - 1) / kResChunks;
    const int64_t j0 = chunk * cw, j1 = std::min<int64_t>(n, j0 + cw);
    if (i >= n) return;
    double r = 0.0, s = 0.0;
    uint64_t lo = 0, hi = 0;
    if (A) {
        float sf = 0.0f;
        if (want_norm == 2) {
#pragma unroll 8
            for (int64_t j = j0; j < j1; j++) {
                double a = A[j * lda + i];
                r = fma(a, x[j], r);
                s += fabs(a);
            }
        } else {
            // two interleaved FP64 accumulators shorten the dependent FMA chain
            double r1 = 0.0;
            int64_t j = j0;
            if (want_norm == 1) {
#pragma unroll 4
                for (; j + 1 < j1; j += 2) {
                    double a0 = A[j * lda + i], a1 = A[(j + 1) * lda + i];
                    r = fma(a0, x[j], r);
                    r1 = fma(a1, x[j + 1], r1);
                    sf += abs_as_float(a0) + abs_as_float(a1);
                }
                if (j < j1) {
                    double a0 = A[j * lda + i];
                    r = fma(a0, x[j], r);
                    sf += abs_as_float(a0);
                }
                s = (double)sf;
            } else {
#pragma unroll 4
                for (; j + 1 < j1; j += 2) {
                    r = fma(A[j * lda + i], x[j], r);
                    r1 = fma(A[(j + 1) * lda + i], x[j + 1], r1);
                }
                if (j < j1) r = fma(A[j * lda + i], x[j], r);
            }
            r += r1;
        }
    } else if (dominant && diag && want_norm == 0 && HPLGB_REGEN_I2F) {
        // the plain product with the integer t = a * 2^53 converted by the
        // hardware (exact, |t| <= 2^52): sum t_ij x_j, then one exact scaling by
        // 2^-53 per row; every intermediate is the a_ij version times 2^53, so
        // the rounding is the same
        const uint64_t step = (uint64_t)n * 0x9E3779B97F4A7C15ull;
        uint64_t z = key + ((uint64_t)j0 * (uint64_t)n + (uint64_t)i + 1) * 0x9E3779B97F4A7C15ull;
        double r1 = 0.0;
        int64_t j = j0;
        for (; j + 1 < j1; j += 2, z += 2 * step) {
            const long long t0 = (long long)(res_mix(z) >> 11) - (1LL << 52);
            const long long t1 = (long long)(res_mix(z + step) >> 11) - (1LL << 52);
            r = fma(j == i ? 0.0 : (double)t0, x[j], r);
            r1 = fma(j + 1 == i ? 0.0 : (double)t1, x[j + 1], r1);
        }
        if (j < j1) {
            const long long t0 = (long long)(res_mix(z) >> 11) - (1LL << 52);
            r = fma(j == i ? 0.0 : (double)t0, x[j], r);
        }
        r = (r + r1) * 0x1p-53;
    } else if (dominant && diag && want_norm != 2) {
        // diagonal known: plain regenerated product over the off-diagonal
        // entries, one FP64 instruction (the FMA) per entry
        const uint64_t step = (uint64_t)n * 0x9E3779B97F4A7C15ull;
        uint64_t z = key + ((uint64_t)j0 * (uint64_t)n + (uint64_t)i + 1) * 0x9E3779B97F4A7C15ull;
        double r1 = 0.0;
        float sf = 0.0f;
        int64_t j = j0;
        for (; j + 1 < j1; j += 2, z += 2 * step) {
            const double a0 = j == i ? 0.0 : gen_value(res_mix(z));
            const double a1 = j + 1 == i ? 0.0 : gen_value(res_mix(z + step));
            r = fma(a0, x[j], r);
            r1 = fma(a1, x[j + 1], r1);
            if (want_norm == 1) sf += abs_as_float(a0) + abs_as_float(a1);
        }
        if (j < j1) {
            const double a0 = j == i ? 0.0 : gen_value(res_mix(z));
            r = fma(a0, x[j], r);
            if (want_norm == 1) sf += abs_as_float(a0);
        }
        r += r1;
        if (want_norm == 1) s = (double)sf;
    } else {
        const uint64_t step = (uint64_t)n * 0x9E3779B97F4A7C15ull;
        uint64_t z = key + ((uint64_t)j0 * (uint64_t)n + (uint64_t)i + 1) * 0x9E3779B97F4A7C15ull;
        for (int64_t j = j0; j < j1; j++, z += step) {
            uint64_t h = res_mix(z);
            double a = gen_value(h);
            if (dominant) {
                uint64_t m = h >> 11, u = m >= (1ull << 52) ? m - (1ull << 52) : (1ull << 52) - m;
                uint64_t nl = lo + u;
                hi += (nl < lo);
                lo = nl;
                if (j == i) continue;     // the diagonal is added once the row sum is known
            }
            r = fma(a, x[j], r);
            s += fabs(a);
        }
    }
    w.part_r[chunk * n + i] = r;
    w.part_a[chunk * n + i] = s;
    w.part_lo[chunk * n + i] = lo;
    w.part_hi[chunk * n + i] = hi;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// regen_dominant: the diagonal was skipped by k_res_partial; it is diag[i] if
// diag is given, else the row's exact sum of |a_ij| rounded once. anorm: a
// known ||A||_inf (the row sums were not formed), else NULL.
__global__ void __launch_bounds__(256) k_res_rows(int64_t n, int regen_dominant, const double* __restrict__ diag,
                                                  const double* __restrict__ anorm, const double* __restrict__ x,
                                                  const double* __restrict__ b, ResWs w) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double mr = 0.0, ma = 0.0, mx = 0.0, mb = 0.0;
    if (i < n) {
        double r = 0.0, s = 0.0;
        uint64_t lo = 0, hi = 0;
        for (int c = 0; c < kResChunks; c++) {
            r += w.part_r[c * n + i];
            s += w.part_a[c * n + i];
            uint64_t nl = lo + w.part_lo[c * n + i];
            hi += w.part_hi[c * n + i] + (nl < lo);
            lo = nl;
        }
        if (regen_dominant) {
            double d = diag ? diag[i] : res_u128_to_double(hi, lo) * 0x1p-53;
            r = fma(d, x[i], r);
            s += d;
        }
        r -= b[i];
        mr = fabs(r);
        ma = anorm ? *anorm : s;
        mx = fabs(x[i]);
        mb = fabs(b[i]);
    }
    // NaN compares false everywhere; flag it through the |r| slot as +Inf bits
    if (mr != mr) mr = __longlong_as_double(0x7ff0000000000000LL);
    for (int off = 16; off > 0; off >>= 1) {
        mr = fmax(mr, __shfl_down_sync(0xffffffffu, mr, off));
        ma = fmax(ma, __shfl_down_sync(0xffffffffu, ma, off));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
        mb = fmax(mb, __shfl_down_sync(0xffffffffu, mb, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&w.maxima[0], mr);
        atomic_max_nonneg(&w.maxima[1], ma);
        atomic_max_nonneg(&w.maxima[2], mx);
        atomic_max_nonneg(&w.maxima[3], mb);
    }
}

__global__ void k_res_final(int64_t n, const unsigned long long* maxima, double* out) {
    double mr = __longlong_as_double((long long)maxima[0]);
    double ma = __longlong_as_double((long long)maxima[1]);
    double mx = __longlong_as_double((long long)maxima[2]);
    double mb = __longlong_as_double((long long)maxima[3]);
    *out = mr / (0x1p-53 * (ma * mx + mb) * (double)n);
}

// Residual vector and matrix-vector product for the refinement loop: after
// k_res_partial, r_i = b_i - sum of the row's partials (b != NULL) or
// r_i = sum of the partials (b == NULL, i.e. r = A x); diag != NULL adds the
// diagonal term diag_i x_i that a regenerating k_res_partial skipped.
__global__ void __launch_bounds__(256) k_res_vec(int64_t n, const double* __restrict__ diag,
                                                 const double* __restrict__ x, const double* __restrict__ b, ResWs w,
                                                 double* __restrict__ r) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < kResChunks; c++) s += w.part_r[c * n + i];
    if (diag) s = fma(diag[i], x[i], s);
    r[i] = b ? b[i] - s : s;
}

// Transposed residual for the adjoint solve: one warp per column j of A,
// r_j = b_j - sum_i a_ij x_i (b != NULL) or r_j = sum_i a_ij x_i (b == NULL),
// and the column sums of |a_ij| (the row sums of A^T) into part_a[0..n).
__global__ void __launch_bounds__(256) k_res_cols_t(int64_t n, const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ x, const double* __restrict__ b,
                                                    double* __restrict__ r, double* __restrict__ csum,
                                                    int want_norm) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    const double* col = A + j * lda;
    double s = 0.0;
    float a = 0.0f;
    if (want_norm) {
#pragma unroll 4
        for (int64_t i = lane; i < n; i += 32) {
            double v = col[i];
            s = fma(v, x[i], s);
            a += abs_as_float(v);
        }
    } else {
#pragma unroll 4
        for (int64_t i = lane; i < n; i += 32) s = fma(col[i], x[i], s);
    }
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, off);
        a += __shfl_down_sync(0xffffffffu, a, off);
    }
    if (lane == 0) {
        r[j] = b ? b[j] - s : s;
        csum[j] = a;
    }
}

// anorm_in: a known ||A^T||_inf (csum not formed), else NULL; anorm_out: if
// given (and zeroed), receives max_i csum[i] for later calls.
__global__ void __launch_bounds__(256) k_res_max_t(int64_t n, const double* __restrict__ r,
                                                   const double* __restrict__ csum,
                                                   const double* __restrict__ anorm_in,
                                                   unsigned long long* anorm_out, const double* __restrict__ x,
                                                   const double* __restrict__ b, unsigned long long* maxima) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double mr = 0.0, ma = 0.0, mx = 0.0, mb = 0.0;
    if (i < n) {
        mr = fabs(r[i]);
        ma = anorm_in ? *anorm_in : csum[i];
        mx = fabs(x[i]);
        mb = fabs(b[i]);
    }
    if (mr != mr) mr = __longlong_as_double(0x7ff0000000000000LL);
    for (int off = 16; off > 0; off >>= 1) {
        mr = fmax(mr, __shfl_down_sync(0xffffffffu, mr, off));
        ma = fmax(ma, __shfl_down_sync(0xffffffffu, ma, off));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
        mb = fmax(mb, __shfl_down_sync(0xffffffffu, mb, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&maxima[0], mr);
        atomic_max_nonneg(&maxima[1], ma);
        atomic_max_nonneg(&maxima[2], mx);
        atomic_max_nonneg(&maxima[3], mb);
        if (anorm_out) atomic_max_nonneg(anorm_out, ma);
    }
}

// r = b - A^T x (or A^T x when b == NULL), with the scaled residual of the
// transposed system (||A^T||_inf = max column sum of |A|) into sr if given.
// anorm (device double) caches that norm across calls: norm_mode 0 ignores
// it, 1 computes the norm and stores it there, 2 uses the stored value.
int launch_residual_vec_t(int64_t n, const double* A, int64_t lda, double* anorm, int norm_mode, const double* x,
                          const double* b, double* r, double* sr, void* ws, cudaStream_t s) {
    ResWs w;
    res_ws_layout(n, &w, (char*)ws);
    const bool use = norm_mode == 2 && anorm, store = norm_mode == 1 && anorm;
    k_res_cols_t<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(n, A, lda, x, b, r, w.part_a, sr && b && !use);
    HPL_LAUNCH_CHECK();
    if (sr && b) {
        HPL_CUDA_TRY(cudaMemsetAsync(w.maxima, 0, sizeof(unsigned long long) * 4, s));
        if (store) HPL_CUDA_TRY(cudaMemsetAsync(anorm, 0, sizeof(double), s));
        k_res_max_t<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, r, w.part_a, use ? anorm : nullptr,
                                                                store ? (unsigned long long*)anorm : nullptr, x, b,
                                                                w.maxima);
        HPL_LAUNCH_CHECK();
        k_res_final<<<1, 1, 0, s>>>(n, w.maxima, sr);
        HPL_LAUNCH_CHECK();
    }
    return HPL_OK;
}

size_t residual_ws_bytes(int64_t n) { return res_ws_layout(n > 0 ? n : 1, nullptr, nullptr); }

// r = b - A x (b != NULL) or r = A x (b == NULL), A stored column-major (FP64),
// or, with A == NULL, the dominant generated matrix of key (the generator's
// stream key) regenerated entry by entry with its diagonal taken from diag.
// With sr != NULL (and b != NULL) also the scaled residual of x, with
// ||A||_inf read from anorm (device) if given, else summed here in FP32.
int launch_residual_vec(int64_t n, const double* A, int64_t lda, uint64_t key, const double* diag,
                        const double* anorm, const double* x, const double* b, double* r, double* sr, void* ws,
                        cudaStream_t s) {
    if (!A && !diag) return HPL_ERR_INVALID;
    ResWs w;
    res_ws_layout(n, &w, (char*)ws);
    const double* dg = A ? nullptr : diag;
    dim3 g1((unsigned)((n + 255) / 256), kResChunks);
    k_res_partial<<<g1, 256, 0, s>>>(n, A, lda, key, A ? 0 : 1, dg, x, w, (sr && !anorm) ? 1 : 0);
    HPL_LAUNCH_CHECK();
    k_res_vec<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, dg, x, b, w, r);
    HPL_LAUNCH_CHECK();
    if (sr && b) {
        HPL_CUDA_TRY(cudaMemsetAsync(w.maxima, 0, sizeof(unsigned long long) * 4, s));
        k_res_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, dg != nullptr, dg, anorm, x, b, w);
        HPL_LAUNCH_CHECK();
        k_res_final<<<1, 1, 0, s>>>(n, w.maxima, sr);
        HPL_LAUNCH_CHECK();
    }
    return HPL_OK;
}

// Shared by the mixed-precision solver: computes the scaled residual into out.
int launch_scaled_residual(int64_t n, const double* A, int64_t lda, uint64_t seed, int kind, const double* x,
                           const double* b, double* out, void* ws, cudaStream_t s) {
    ResWs w;
    res_ws_layout(n, &w, (char*)ws);
    HPL_CUDA_TRY(cudaMemsetAsync(w.maxima, 0, sizeof(unsigned long long) * 4, s));
    uint64_t key = res_mix(seed + 1ull * 0x9E3779B97F4A7C15ull);    // stream 0 of the generator
    dim3 g1((unsigned)((n + 255) / 256), kResChunks);
    k_res_partial<<<g1, 256, 0, s>>>(n, A, lda, key, kind == HPL_GEN_DIAG_DOMINANT, nullptr, x, w, 2);
    HPL_LAUNCH_CHECK();
    k_res_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, !A && kind == HPL_GEN_DIAG_DOMINANT, nullptr, nullptr,
                                                           x, b, w);
    HPL_LAUNCH_CHECK();
    k_res_final<<<1, 1, 0, s>>>(n, w.maxima, out);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

}  // namespace hplgb

using namespace hplgb;

extern "C" size_t hpl_residual_workspace_size(int64_t n) { return residual_ws_bytes(n); }

extern "C" int hpl_scaled_residual(int64_t n, const double* A, int64_t lda, uint64_t seed, int kind, const double* x,
                                   const double* b, double* out, void* ws, size_t ws_bytes, void* stream) {
    if (n <= 0 || !x || !b || !out) return HPL_ERR_INVALID;
    if (A && lda < n) return HPL_ERR_INVALID;
    if (kind != HPL_GEN_GENERAL && kind != HPL_GEN_DIAG_DOMINANT) return HPL_ERR_INVALID;
    if (!ws || ws_bytes < residual_ws_bytes(n)) return HPL_ERR_NOMEM;
    if ((uintptr_t)ws & 255) return HPL_ERR_INVALID;
    return launch_scaled_residual(n, A, lda, seed, kind, x, b, out, ws, (cudaStream_t)stream);
}
