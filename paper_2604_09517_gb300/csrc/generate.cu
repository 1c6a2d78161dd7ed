// hpl_generate: seeded counter-based matrix generator.
//
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a counter-based
// generator: output c >= 1 of a generator whose state starts at s is
// mix(s + c * GAMMA). Stream key = output (stream_id + 1) under the seed;
// entry (i, j) of an m-row matrix = output (j*m + i + 1) under the key, its top
// 53 bits scaled to [0,1) and shifted by -0.5 (exact). The paper says only
// that the HPL matrix is random (Sec. III-A.1) and that HPL-MxP has a scalable
// generator (Sec. II-B); this definition is the library's own.
#include <algorithm>

#include <type_traits>

#include "common.cuh"

namespace hplgb {

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm64_host_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_generate(uint64_t key, int64_t m, int64_t ncols, double* __restrict__ A, int64_t lda) {
    const int64_t total = m * ncols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = t / m, i = t - j * m;
        uint64_t h = sm64_mix(key + (uint64_t)(t + 1) * kGamma);
        A[j * lda + i] = gen_value(h);
    }
}

// Round a 128-bit unsigned integer (hi:lo) to the nearest double, ties to
// even: the top 64 significant bits carry a sticky bit for what is shifted
// out, then one correctly rounded 64-bit conversion.
__device__ __forceinline__ double u128_to_double_rn(uint64_t hi, uint64_t lo) {
    if (hi == 0) return __ull2double_rn(lo);
    int sh = 64 - __clzll((long long)hi);          // bits of hi, 1..64
    uint64_t top = (sh == 64) ? hi : ((hi << (64 - sh)) | (lo >> sh));
    uint64_t dropped = (sh == 64) ? lo : (lo & ((1ull << sh) - 1));
    top |= (dropped != 0);
    return ldexp(__ull2double_rn(top), sh);
}

// Diagonal dominance: block of 32 rows (lane = row), 8 warps split the
// columns; each lane sums |a_ij| / 2^-53 exactly in 128 bits; the warps'
// partial sums are combined exactly; the diagonal is rounded once.
__global__ void __launch_bounds__(256) k_dominant_diag(int64_t n, double* __restrict__ A, int64_t lda) {
    __shared__ uint64_t s_lo[8][32], s_hi[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    uint64_t lo = 0, hi = 0;
    if (i < n) {
        for (int64_t j = warp; j < n; j += 8) {
            // |a| / 2^-53, exact: |a| = k * 2^-53 with k <= 2^52; taken from the bits
            // (integer operations) as (2^52 + fraction) >> (1022 - biased exponent)
            const unsigned long long bits = (unsigned long long)__double_as_longlong(A[j * lda + i]);
            const int e = (int)((bits >> 52) & 0x7ff);
            const int sh = 1022 - e;
            uint64_t u = (e == 0 || sh >= 64) ? 0 : (((bits & ((1ull << 52) - 1)) | (1ull << 52)) >> sh);
            uint64_t nl = lo + u;
            hi += (nl < lo);
            lo = nl;
        }
    }
    s_lo[warp][lane] = lo;
    s_hi[warp][lane] = hi;
    __syncthreads();
    if (warp == 0 && i < n) {
        for (int w = 1; w < 8; w++) {
            uint64_t nl = lo + s_lo[w][lane];
            hi += s_hi[w][lane] + (nl < lo);
            lo = nl;
        }
        A[i * lda + i] = u128_to_double_rn(hi, lo) * 0x1p-53;
    }
}

// ---------------------------------------------------------------------------
// The dominant matrix straight into an FP32 (or BF16) working copy, for a
// mixed-precision solve that keeps no FP64 copy of A (its residuals
// regenerate the entries). Every entry is the FP64 generated value rounded
// once to nearest, exactly what converting a stored FP64 matrix gives.
//
// One pass over the entries: rows in blocks of 256 (blockIdx.x), `chunks`
// column chunks (blockIdx.y). Per (row, chunk) the kernel writes the FP32
// entries, the exact sum of |a_ij| / 2^-53 = |(h >> 11) - 2^52| over the
// chunk in 128 bits (the diagonal's dominance, all j), and the FP32 sum of
// |fl32(a_ij)| over the chunk's off-diagonal entries (||A||_inf for the
// refinement's stopping test).
__device__ __forceinline__ float gen_store(float* p, uint64_t h) {
    // t = (h >> 11) - 2^52 converted by the hardware (one rounding to nearest
    // even of the integer), then the exact scaling by 2^-53: the FP32 rounding
    // of the FP64 value (t 2^-53) in one step
    const long long t = (long long)(h >> 11) - (1LL << 52);
    const float v = __ll2float_rn(t) * 0x1p-53f;
    *p = v;
    return v;
}
__device__ __forceinline__ float gen_store(__nv_bfloat16* p, uint64_t h) {
    const __nv_bfloat16 v = f64_to_bf16_rn(gen_value(h));
    *p = v;
    return __bfloat162float(v);
}

// A32 (optional, n x n, ld n) receives the FP32 rounding of each entry as
// well (GMRES's inner products in FP32 data).
template <typename FT>
__global__ void __launch_bounds__(256) k_generate_f32(uint64_t key, int64_t n, FT* __restrict__ F, int64_t ldf,
                                                      int chunks, uint64_t* __restrict__ plo,
                                                      uint64_t* __restrict__ phi, float* __restrict__ pf,
                                                      float* __restrict__ A32) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int64_t cw = (n + chunks - 1) / chunks;
    const int64_t j0 = (int64_t)blockIdx.y * cw, j1 = std::min<int64_t>(n, j0 + cw);
    const uint64_t step = (uint64_t)n * kGamma;
    uint64_t z = key + ((uint64_t)j0 * (uint64_t)n + (uint64_t)i + 1) * kGamma;
    uint64_t lo = 0, hi = 0;
    float sf = 0.0f;
    for (int64_t j = j0; j < j1; j++, z += step) {
        const uint64_t h = sm64_mix(z);
        const float v = gen_store(F + j * ldf + i, h);
        if (A32) {
            if constexpr (std::is_same<FT, float>::value) {
                A32[j * n + i] = v;
            } else {
                A32[j * n + i] = __ll2float_rn((long long)(h >> 11) - (1LL << 52)) * 0x1p-53f;
            }
        }
        const uint64_t m = h >> 11, u = m >= (1ull << 52) ? m - (1ull << 52) : (1ull << 52) - m;
        const uint64_t nl = lo + u;
        hi += (nl < lo);
        lo = nl;
        sf += j == i ? 0.0f : fabsf(v);
    }
    plo[(int64_t)blockIdx.y * n + i] = lo;
    phi[(int64_t)blockIdx.y * n + i] = hi;
    pf[(int64_t)blockIdx.y * n + i] = sf;
}

// Per row: the exact row sum over the chunks, rounded once, is the FP64
// diagonal (into diag); its FP32 rounding goes onto F's diagonal and into the
// row's norm partial of the chunk that holds column i.
template <typename FT>
__global__ void __launch_bounds__(256) k_dominant_diag_fin(int64_t n, int chunks, const uint64_t* __restrict__ plo,
                                                           const uint64_t* __restrict__ phi, double* __restrict__ diag,
                                                           FT* __restrict__ F, int64_t ldf, float* __restrict__ pf,
                                                           float* __restrict__ A32) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    uint64_t lo = 0, hi = 0;
    for (int c = 0; c < chunks; c++) {
        const uint64_t nl = lo + plo[(int64_t)c * n + i];
        hi += phi[(int64_t)c * n + i] + (nl < lo);
        lo = nl;
    }
    const double d = u128_to_double_rn(hi, lo) * 0x1p-53;
    diag[i] = d;
    const float f = st_f64(F + i * ldf + i, d);
    if (A32) A32[i * n + i] = f64_to_f32_rn(d);
    const int64_t cw = (n + chunks - 1) / chunks;
    pf[(i / cw) * n + i] += fabsf(f);
}

// Stream 0 (the matrix) of seed, kind HPL_GEN_DIAG_DOMINANT, n x n, as FP32
// (bf16 = 0) or BF16 (bf16 = 1) into F (ldf >= n) with the FP64 diagonal into
// diag (n doubles); returns the stream key the residual kernels regenerate
// from in *key_out. plo, phi (chunks x n each) are scratch; pf (chunks x n)
// receives the row sums of |F| split by column chunk.
int launch_generate_dominant_f32(uint64_t seed, int64_t n, void* F, int64_t ldf, int bf16, double* diag,
                                 uint64_t* key_out, int chunks, uint64_t* plo, uint64_t* phi, float* pf,
                                 float* A32, cudaStream_t s) {
    const uint64_t key = sm64_host_mix(seed + 1 * kGamma);
    if (key_out) *key_out = key;
    if (n <= 0) return HPL_OK;
    const dim3 g1((unsigned)((n + 255) / 256), (unsigned)chunks), g2((unsigned)((n + 255) / 256));
    if (bf16) {
        __nv_bfloat16* Fb = (__nv_bfloat16*)F;
        k_generate_f32<<<g1, 256, 0, s>>>(key, n, Fb, ldf, chunks, plo, phi, pf, A32);
        HPL_LAUNCH_CHECK();
        k_dominant_diag_fin<<<g2, 256, 0, s>>>(n, chunks, plo, phi, diag, Fb, ldf, pf, A32);
    } else {
        float* Ff = (float*)F;
        k_generate_f32<<<g1, 256, 0, s>>>(key, n, Ff, ldf, chunks, plo, phi, pf, A32);
        HPL_LAUNCH_CHECK();
        k_dominant_diag_fin<<<g2, 256, 0, s>>>(n, chunks, plo, phi, diag, Ff, ldf, pf, A32);
    }
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

}  // namespace hplgb

using namespace hplgb;

// Sizes of the batched workload: n_s = 32 + (draw s of stream 2 mod 481),
// uniform on [32, 512] up to a modulo bias below 1e-16. Host memory out.
extern "C" int hpl_batch_sizes(uint64_t seed, int64_t count, int64_t* n_out) {
    if (count < 0 || (count > 0 && !n_out)) return HPL_ERR_INVALID;
    const uint64_t key = sm64_host_mix(seed + 3 * kGamma);
    for (int64_t s = 0; s < count; s++) n_out[s] = 32 + (int64_t)(sm64_host_mix(key + (uint64_t)(s + 1) * kGamma) % 481);
    return HPL_OK;
}

extern "C" int hpl_generate(uint64_t seed, uint64_t stream_id, int64_t m, int64_t ncols, int kind, double* A,
                            int64_t lda, void* stream) {
    if (m < 0 || ncols < 0 || (m > 0 && ncols > 0 && !A) || lda < (m > 1 ? m : 1)) return HPL_ERR_INVALID;
    if (kind != HPL_GEN_GENERAL && kind != HPL_GEN_DIAG_DOMINANT) return HPL_ERR_INVALID;
    if (kind == HPL_GEN_DIAG_DOMINANT && m != ncols) return HPL_ERR_INVALID;
    if (m == 0 || ncols == 0) return HPL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t key = sm64_host_mix(seed + (stream_id + 1) * kGamma);
    int64_t total = m * ncols;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_generate<<<(unsigned)blocks, 256, 0, s>>>(key, m, ncols, A, lda);
    HPL_LAUNCH_CHECK();
    if (kind == HPL_GEN_DIAG_DOMINANT) {
        k_dominant_diag<<<(unsigned)((m + 31) / 32), 256, 0, s>>>(m, A, lda);
        HPL_LAUNCH_CHECK();
    }
    return HPL_OK;
}
