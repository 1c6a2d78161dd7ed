// mxp_solve: the HPL-MxP solve (paper Sec. III-A.2; Sec. II-B for GMRES-based
// refinement) on one GB300.
//
// Factorization: block LU without pivoting (Demmel, Higham & Schreiber 1995)
// of an FP32 working copy F of A, panel width NB. Per step k:
//   D   = diagonal block of F (kb x kb, the Schur complement so far)
//   D^-1 by Newton-Schulz, X <- X (2I - D X) from X = diag(D)^-1, with each
//        product on the tcgen05 tensor cores in split BF16 (operands hi + lo,
//        products hi*hi + hi*lo + lo*hi over a contraction of length 3kb)
//   L21 = A21 D^-1         (BF16 operands, FP32 accumulate, written into F)
//   A22 = A22 - L21 A12    (BF16 operands, FP32 accumulate in TMEM, FP32 C)
// Every O(n^2 NB) and O(n^3) product runs on the tensor cores; the FP32 work
// outside them is elementwise.
// Refinement (FP64): x0 = M^-1 b with M = L U applied in FP32 by block
// forward / backward substitution (GEMV kernels over the factor's panels and
// the stored D_k^-1); then r = b - A x in FP64 with the scaled residual; stop
// below tol; correction by classic iterative refinement (d = M^-1 r) or by
// GMRES right-preconditioned with M^-1 (modified Gram-Schmidt and Givens
// rotations in FP64; the Hessenberg least-squares problem is solved on the
// host), x += d. The host reads one scalar per GMRES step and per outer
// iteration, so mxp_solve returns only when the solve is done.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace hplgb {

int launch_gemm_bf16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                     float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns, int max_ctas, cudaStream_t s);
bool gemm_bf16_copy_ok(const float* C, int64_t ldc, const uint16_t* C16, int64_t N, int64_t ld16);
int launch_gemm_bf16_copy(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                          int64_t ldb, float* C, int64_t ldc, uint16_t* C16, int64_t ld16, int* err, int64_t timeout_ns,
                          cudaStream_t s);
int launch_gemm_f16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                    const float* sa, const float* sb, float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns,
                    int max_ctas, cudaStream_t s);
int launch_gemm_bf16_c16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                         int64_t ldb, uint16_t* C, int64_t ldc, int sub, int* err, int64_t timeout_ns, int max_ctas,
                         cudaStream_t s);
int launch_gemm_fp8(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda, const uint8_t* B, int64_t ldb,
                    const float* sa, const float* sb, float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns,
                    int max_ctas, cudaStream_t s);
int launch_gemm_tf32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                     float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns, int max_ctas, cudaStream_t s);
size_t residual_ws_bytes(int64_t n);
int launch_residual_vec(int64_t n, const double* A, int64_t lda, uint64_t key, const double* diag,
                        const double* anorm, const double* x, const double* b, double* r, double* sr, void* ws,
                        cudaStream_t s);
int launch_generate_dominant_f32(uint64_t seed, int64_t n, void* F, int64_t ldf, int bf16, double* diag,
                                 uint64_t* key_out, int chunks, uint64_t* plo, uint64_t* phi, float* pf,
                                 float* A32, cudaStream_t s);
int launch_residual_vec_t(int64_t n, const double* A, int64_t lda, double* anorm, int norm_mode, const double* x,
                          const double* b, double* r, double* sr, void* ws, cudaStream_t s);

constexpr int kDotBlocks = 304;
constexpr int kGemvSplitMax = 16;
// Default panel width: with an FP32 trailing matrix each update step moves 8
// bytes of C per 2 NB flops, so NB must be large for the update to stay
// compute-bound (BF16 needs NB >~ 1250 at the measured HBM bandwidth, FP8
// twice that); 3072 measured fastest for both at n = 98304.
constexpr int64_t kMxpDefaultNb = 3072;

static inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// ---------------------------------------------------------------------------
// Operand conversion. X is FP32 column-major (rows x cols, ldx). The BF16
// operand has K contiguous with row stride ldo and starts at column seg_off:
//   trans = 1: operand row r (< rows) holds X(r, 0..cols): the M x K operand
//              of X itself (K = cols);
//   trans = 0: operand row c (< cols) holds X(0..rows, c): the N x K operand
//              for a product with X on the right (K = rows).
// part 0 = round to nearest even, 1 = hi = bf16(x), 2 = lo = bf16(x - hi).
// nseg segments are written at column offsets seg_off + q * seg_stride, with
// the part of segment q in bits 2q..2q+1 of `parts` (the split operands of
// the Newton-Schulz products are [hi | hi | lo] or [hi | lo | hi]). With
// eye2 the converted value is 2 delta_ij - X(i, j) (the 2I - R step).
// K positions in [K extent, kpad) of each segment are written as zeros.
__device__ __forceinline__ float bf16_part(float x, int part) {
    float h = __bfloat162float(__float2bfloat16_rn(x));
    return part == 2 ? __bfloat162float(__float2bfloat16_rn(x - h)) : h;
}

struct Seg {
    int nseg, parts, eye2;
    int64_t seg_off, seg_stride, kpad;
};

__device__ __forceinline__ float eye2_of(float v, int64_t r, int64_t c) { return (r == c ? 2.0f : 0.0f) - v; }

// trans = 1: a transpose through a 32 (K) x 128 (operand rows) shared tile, one
// per CTA. Each warp reads 512 contiguous bytes of one column of X per
// instruction (four FP32 values per lane when aligned) and writes 64
// contiguous bytes (32 BF16 values) of each of two operand rows per
// instruction. (Measured on GB300 at 94208 x 4096, X column-major with
// ld 98304: 5986 GB/s of reads + writes, against 4774 GB/s for a 64 x 64 tile
// that reads only 256 bytes of each column.)
template <typename XT>
__global__ void __launch_bounds__(256) k_to_bf16_t(const XT* __restrict__ X, int64_t ldx, int64_t rows,
                                                   int64_t cols, __nv_bfloat16* __restrict__ out, int64_t ldo,
                                                   Seg g, int vec4) {
    __shared__ float tile[32][129];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 128;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int cc = warp + 8 * j;
        const int64_t c = c0 + cc, r = r0 + 4 * lane;
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (c < cols) {
            const XT* xc = X + c * ldx;
            if constexpr (std::is_same<XT, float>::value) {
                if (vec4 && r + 3 < rows) {
                    const float4 t = *reinterpret_cast<const float4*>(xc + r);
                    v[0] = t.x;
                    v[1] = t.y;
                    v[2] = t.z;
                    v[3] = t.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++)
                        if (r + e < rows) v[e] = xc[r + e];
                }
            } else if (vec4 && r + 3 < rows) {          // BF16 source: four values in one 8-byte load
                const uint2 t = *reinterpret_cast<const uint2*>(xc + r);
                v[0] = __uint_as_float(t.x << 16);
                v[1] = __uint_as_float(t.x & 0xffff0000u);
                v[2] = __uint_as_float(t.y << 16);
                v[3] = __uint_as_float(t.y & 0xffff0000u);
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (r + e < rows) v[e] = ld_f(xc + r + e);
            }
            if (g.eye2) {
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (r + e < rows) v[e] = eye2_of(v[e], r + e, c);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; e++) tile[cc][4 * lane + e] = v[e];
    }
    __syncthreads();
    // lanes 0-15 write row rr, lanes 16-31 row rr + 1, two values each
    const int sub = lane >> 4, l = lane & 15;
    const int64_t c = c0 + 2 * l;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int rr = warp * 16 + 2 * i + sub;
        const int64_t r = r0 + rr;
        if (r >= rows) continue;
        const float v0 = tile[2 * l][rr], v1 = tile[2 * l + 1][rr];
        for (int q = 0; q < g.nseg; q++) {
            const int part = (g.parts >> (2 * q)) & 3;
            __nv_bfloat16* o = out + r * ldo + g.seg_off + q * g.seg_stride + c;
            if (c + 1 < g.kpad) {
                __nv_bfloat162 h;
                h.x = __float2bfloat16_rn(bf16_part(v0, part));
                h.y = __float2bfloat16_rn(bf16_part(v1, part));
                *reinterpret_cast<__nv_bfloat162*>(o) = h;
            } else if (c < g.kpad) {
                *o = __float2bfloat16_rn(bf16_part(v0, part));
            }
        }
    }
}

// trans = 0: a straight conversion along the contraction index; each thread
// converts 8 consecutive values (two 16-byte loads, one 16-byte store when
// aligned), a grid-stride loop over (operand row, group of 8).
template <typename XT>
__global__ void __launch_bounds__(256) k_to_bf16_n(const XT* __restrict__ X, int64_t ldx, int64_t rows,
                                                   int64_t cols, __nv_bfloat16* __restrict__ out, int64_t ldo,
                                                   Seg g, int vec) {
    const int64_t groups = (g.kpad + 7) / 8;
    const int64_t total = groups * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / groups;
        const int64_t r = (t - c * groups) * 8;
        float v[8];
        const XT* xc = X + c * ldx;
        if (vec && r + 7 < rows) {
            if constexpr (std::is_same<XT, float>::value) {
                const float4 a = *reinterpret_cast<const float4*>(xc + r);
                const float4 b = *reinterpret_cast<const float4*>(xc + r + 4);
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
            } else {                                   // BF16 source: eight values in one 16-byte load
                const uint4 t = *reinterpret_cast<const uint4*>(xc + r);
                const uint32_t w4[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    v[2 * e] = __uint_as_float(w4[e] << 16);
                    v[2 * e + 1] = __uint_as_float(w4[e] & 0xffff0000u);
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; e++) v[e] = r + e < rows ? ld_f(xc + r + e) : 0.0f;
        }
        if (g.eye2) {
#pragma unroll
            for (int e = 0; e < 8; e++)
                if (r + e < rows) v[e] = eye2_of(v[e], r + e, c);
        }
        for (int q = 0; q < g.nseg; q++) {
            const int part = (g.parts >> (2 * q)) & 3;
            __nv_bfloat16* o = out + c * ldo + g.seg_off + q * g.seg_stride + r;
            if (vec && r + 7 < g.kpad) {
                __align__(16) __nv_bfloat16 h[8];
#pragma unroll
                for (int e = 0; e < 8; e++) h[e] = __float2bfloat16_rn(bf16_part(v[e], part));
                *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(h);
            } else {
                for (int e = 0; e < 8 && r + e < g.kpad; e++) o[e] = __float2bfloat16_rn(bf16_part(v[e], part));
            }
        }
    }
}

template <typename XT>
static int to_bf16_seg(const XT* X, int64_t ldx, int64_t rows, int64_t cols, int trans, uint16_t* out, int64_t ldo,
                       Seg g, cudaStream_t s) {
    if (trans) {
        // BF16 pairs are stored 4-byte aligned: even strides and offsets
        if ((ldo | g.seg_off | g.seg_stride) & 1 || ((uintptr_t)out & 3)) return HPL_ERR_INVALID;
        // one 32 x 128 tile per CTA (a grid-stride loop over tiles measured slower)
        if ((g.kpad + 31) / 32 > 0x7fffffff || (rows + 127) / 128 > 65535) return HPL_ERR_INVALID;
        dim3 grid((unsigned)((g.kpad + 31) / 32), (unsigned)((rows + 127) / 128));
        // four-value loads: 16-byte aligned FP32 or 8-byte aligned BF16 columns
        const int vec4 = ((uintptr_t)X & (4 * sizeof(XT) - 1)) == 0 && ldx % 4 == 0;
        k_to_bf16_t<<<grid, 256, 0, s>>>(X, ldx, rows, cols, (__nv_bfloat16*)out, ldo, g, vec4);
        HPL_LAUNCH_CHECK();
        return HPL_OK;
    }
    // 16-byte accesses: X column starts and out row starts / segment offsets aligned
    // (a BF16 X: eight values per 16-byte load, so columns starting on 16 bytes: ldx % 8 == 0)
    const int vec = ((uintptr_t)X & 15) == 0 && ldx % (16 / sizeof(XT)) == 0 && ((uintptr_t)out & 15) == 0 &&
                    ldo % 8 == 0 && g.seg_off % 8 == 0 && g.seg_stride % 8 == 0;
    const int64_t items = ((g.kpad + 7) / 8) * cols;
    const int64_t blocks = std::min<int64_t>((items + 255) / 256, 152 * 32);
    k_to_bf16_n<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(X, ldx, rows, cols, (__nv_bfloat16*)out, ldo, g,
                                                                       vec);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

// ---------------------------------------------------------------------------
// TF32 operands: FP32 words rounded to TF32 (round to nearest even at
// fraction bit 13, on the bit pattern: the carry moves into the exponent and
// past the largest finite value to infinity; subnormals on their fixed grid;
// NaN and infinity unchanged), so the 13 bits the MMA ignores are zero.
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        u += 0x0FFFu + ((u >> 13) & 1u);
        u &= 0xFFFFE000u;
    }
    return __uint_as_float(u);
}

// trans = 1 (operand row r holds X(r, 0..cols)): 64 x 32 shared tiles, two
// values (8 bytes) per lane and store, 256 contiguous bytes per warp.
__global__ void __launch_bounds__(256) k_to_tf32_t(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                                   int64_t cols, float* __restrict__ out, int64_t ldo, int64_t kpad,
                                                   int vec4) {
    // a 32 (K) x 128 (operand rows) tile per CTA: 512-byte reads of each
    // column of X, 128-byte writes of each operand row (as k_to_bf16_t)
    __shared__ float tile[32][129];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 128;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int cc = warp + 8 * j;
        const int64_t c = c0 + cc, r = r0 + 4 * lane;
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (c < cols) {
            const float* xc = X + c * ldx;
            if (vec4 && r + 3 < rows) {
                const float4 t = *reinterpret_cast<const float4*>(xc + r);
                v[0] = t.x;
                v[1] = t.y;
                v[2] = t.z;
                v[3] = t.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (r + e < rows) v[e] = xc[r + e];
            }
        }
#pragma unroll
        for (int e = 0; e < 4; e++) tile[cc][4 * lane + e] = v[e];
    }
    __syncthreads();
    const int sub = lane >> 4, l = lane & 15;
    const int64_t c = c0 + 2 * l;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int rr = warp * 16 + 2 * i + sub;
        const int64_t r = r0 + rr;
        if (r >= rows) continue;
        float* o = out + r * ldo + c;
        if (c + 1 < kpad)
            *reinterpret_cast<float2*>(o) = make_float2(round_tf32(tile[2 * l][rr]), round_tf32(tile[2 * l + 1][rr]));
        else if (c < kpad)
            *o = round_tf32(tile[2 * l][rr]);
    }
}

// trans = 0 (operand row c holds X(0..rows, c)): 8 values per thread, 16-byte
// loads and stores when aligned, a grid-stride loop.
__global__ void __launch_bounds__(256) k_to_tf32_n(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                                   int64_t cols, float* __restrict__ out, int64_t ldo, int64_t kpad,
                                                   int vec) {
    const int64_t groups = (kpad + 7) / 8;
    const int64_t total = groups * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / groups;
        const int64_t r = (t - c * groups) * 8;
        const float* xc = X + c * ldx;
        float* o = out + c * ldo + r;
        if (vec && r + 7 < rows && r + 7 < kpad) {
            const float4 a = *reinterpret_cast<const float4*>(xc + r);
            const float4 b = *reinterpret_cast<const float4*>(xc + r + 4);
            *reinterpret_cast<float4*>(o) = make_float4(round_tf32(a.x), round_tf32(a.y), round_tf32(a.z), round_tf32(a.w));
            *reinterpret_cast<float4*>(o + 4) =
                make_float4(round_tf32(b.x), round_tf32(b.y), round_tf32(b.z), round_tf32(b.w));
        } else {
            for (int e = 0; e < 8 && r + e < kpad; e++) o[e] = r + e < rows ? round_tf32(xc[r + e]) : 0.0f;
        }
    }
}

static int to_tf32(const float* X, int64_t ldx, int64_t rows, int64_t cols, int trans, float* out, int64_t ldo,
                   int64_t kpad, cudaStream_t s) {
    if (trans) {
        if ((ldo & 1) || ((uintptr_t)out & 7)) return HPL_ERR_INVALID;
        if ((kpad + 31) / 32 > 0x7fffffff || (rows + 127) / 128 > 65535) return HPL_ERR_INVALID;
        dim3 grid((unsigned)((kpad + 31) / 32), (unsigned)((rows + 127) / 128));
        const int vec4 = ((uintptr_t)X & 15) == 0 && ldx % 4 == 0;
        k_to_tf32_t<<<grid, 256, 0, s>>>(X, ldx, rows, cols, out, ldo, kpad, vec4);
        HPL_LAUNCH_CHECK();
        return HPL_OK;
    }
    const int vec = ((uintptr_t)X & 15) == 0 && ldx % 4 == 0 && ((uintptr_t)out & 15) == 0 && ldo % 4 == 0;
    const int64_t items = ((kpad + 7) / 8) * cols;
    const int64_t blocks = std::min<int64_t>((items + 255) / 256, 152 * 32);
    k_to_tf32_n<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(X, ldx, rows, cols, out, ldo, kpad, vec);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

// One segment, one part (the plain operand conversions).
template <typename XT>
static int to_bf16(const XT* X, int64_t ldx, int64_t rows, int64_t cols, int trans, int part, uint16_t* out,
                   int64_t ldo, int64_t seg_off, int64_t kpad, cudaStream_t s) {
    Seg g{1, part, 0, seg_off, 0, kpad};
    return to_bf16_seg(X, ldx, rows, cols, trans, out, ldo, g, s);
}

// Split operand [p0 | p1 | p2] of three segments of width kb8 (optionally of 2I - X).
static int to_bf16_split3(const float* X, int64_t ldx, int64_t kb, int trans, int p0, int p1, int p2, int eye2,
                          uint16_t* out, int64_t kb8, cudaStream_t s) {
    Seg g{3, p0 | (p1 << 2) | (p2 << 4), eye2, 0, kb8, kb8};
    return to_bf16_seg(X, ldx, kb, kb, trans, out, 3 * kb8, g, s);
}

// ---------------------------------------------------------------------------
// FP8 E4M3 operands of the trailing update, one power-of-two scale per operand
// row (A) or column (B) over the whole contraction index: the smallest e with
// amax * 2^-e <= 448 (amax = f 2^E with 0.5 <= f < 1: e = E - 9 when
// f <= 448/512, else E - 8); values x * 2^-e rounded to nearest even with
// saturation; the scale 2^e is returned for the GEMM epilogue.
__device__ __forceinline__ int e4m3_scale_exp(float amax) {
    if (!(amax > 0.0f) || !isfinite(amax)) return 0;
    int E;
    float f = frexpf(amax, &E);
    return f <= 0.875f ? E - 9 : E - 8;
}

__device__ __forceinline__ unsigned char to_e4m3(float x) {
    return (unsigned char)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// Scaled low-precision operands (FMT 1 = FP8 E4M3, 2 = FP16): one
// power-of-two scale per operand row (A) or column (B), the smallest 2^e with
// max|x| 2^-e within the format's largest finite value (448 for E4M3,
// 65504 = (1 - 2^-11) 2^16 for FP16).
__device__ __forceinline__ int f16_scale_exp(float amax) {
    if (!(amax > 0.0f) || !isfinite(amax)) return 0;
    int E;
    float f = frexpf(amax, &E);
    return f <= 0.99951171875f ? E - 16 : E - 15;
}
template <int FMT>
struct LowFmt;
template <>
struct LowFmt<1> {
    using T = unsigned char;
    static __device__ __forceinline__ int scale_exp(float amax) { return e4m3_scale_exp(amax); }
    static __device__ __forceinline__ T cvt(float x) { return to_e4m3(x); }
};
template <>
struct LowFmt<2> {
    using T = uint16_t;
    static __device__ __forceinline__ int scale_exp(float amax) { return f16_scale_exp(amax); }
    static __device__ __forceinline__ T cvt(float x) { return __half_as_ushort(__float2half_rn(x)); }
};

// Float4 loads along a column-major matrix's columns: 16-byte aligned columns.
static inline int vec4_ok(const float* X, int64_t ldx) { return ((uintptr_t)X & 15) == 0 && ldx % 4 == 0; }

// Four consecutive low-precision values in one store (the callers keep the
// address aligned to four values: operand rows of kpad values, kpad a multiple
// of 16 for FP8 and of 8 for FP16, and column offsets that are multiples of 4).
__device__ __forceinline__ void store4(unsigned char* o, const unsigned char (&q)[4]) {
    *reinterpret_cast<uint32_t*>(o) = (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16) |
                                      ((uint32_t)q[3] << 24);
}
__device__ __forceinline__ void store4(uint16_t* o, const uint16_t (&q)[4]) {
    *reinterpret_cast<uint2*>(o) = make_uint2((uint32_t)q[0] | ((uint32_t)q[1] << 16),
                                              (uint32_t)q[2] | ((uint32_t)q[3] << 16));
}

// A operand: X (rows x cols, column-major) -> out row r = X(r, :) (K = cols),
// sa[r] = 2^e. 128 rows per CTA. Pass 1 takes each row's largest |x|, every
// warp reading 512 contiguous bytes of a column per instruction; pass 2 moves
// 32-column tiles through shared memory and writes 32 consecutive values of
// each row (the first version, 32 rows per CTA, read 128 bytes per column and
// instruction and ran at under half the HBM bandwidth).
template <int FMT>
__global__ void __launch_bounds__(256) k_quant_rows(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                                    int64_t cols, typename LowFmt<FMT>::T* __restrict__ out,
                                                    int64_t ldo, int64_t kpad, float* __restrict__ sa, int vec4) {
    using T = typename LowFmt<FMT>::T;
    __shared__ float part[8][129];
    __shared__ float inv[128];
    __shared__ float tile[32][129];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * 128;
    const int64_t r = r0 + 4 * lane;
    auto load4 = [&](int64_t c, float (&v)[4]) {
        v[0] = v[1] = v[2] = v[3] = 0.0f;
        if (c >= cols) return;
        const float* xc = X + c * ldx;
        if (vec4 && r + 3 < rows) {
            const float4 t = *reinterpret_cast<const float4*>(xc + r);
            v[0] = t.x;
            v[1] = t.y;
            v[2] = t.z;
            v[3] = t.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (r + e < rows) v[e] = xc[r + e];
        }
    };
    // four column loads in flight per warp (a CTA stays resident for the
    // whole row block, so the loads in flight per SM set the bandwidth)
    float am[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int64_t c1 = warp;
    for (; c1 + 24 < cols; c1 += 32) {
        float v0[4], v1[4], v2[4], v3[4];
        load4(c1, v0);
        load4(c1 + 8, v1);
        load4(c1 + 16, v2);
        load4(c1 + 24, v3);
#pragma unroll
        for (int e = 0; e < 4; e++)
            am[e] = fmaxf(am[e], fmaxf(fmaxf(fabsf(v0[e]), fabsf(v1[e])), fmaxf(fabsf(v2[e]), fabsf(v3[e]))));
    }
    for (; c1 < cols; c1 += 8) {
        float v[4];
        load4(c1, v);
#pragma unroll
        for (int e = 0; e < 4; e++) am[e] = fmaxf(am[e], fabsf(v[e]));
    }
#pragma unroll
    for (int e = 0; e < 4; e++) part[warp][4 * lane + e] = am[e];
    __syncthreads();
    if (threadIdx.x < 128) {
        float m = 0.0f;
        for (int w = 0; w < 8; w++) m = fmaxf(m, part[w][threadIdx.x]);
        const int e = LowFmt<FMT>::scale_exp(m);
        inv[threadIdx.x] = ldexpf(1.0f, -e);
        if (r0 + threadIdx.x < rows) sa[r0 + threadIdx.x] = ldexpf(1.0f, e);
    }
    __syncthreads();
    // 8 lanes per row, four values each; four rows per warp instruction. The
    // next tile's columns are loaded into registers while this one is written.
    const int sub = lane >> 3, l = lane & 7;
    float nv[4][4];
#pragma unroll
    for (int j = 0; j < 4; j++) load4(warp + 8 * j, nv[j]);
    for (int64_t c0 = 0; c0 < kpad; c0 += 32) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int cc = warp + 8 * j;
#pragma unroll
            for (int e = 0; e < 4; e++) tile[cc][4 * lane + e] = nv[j][e];
        }
        __syncthreads();
        if (c0 + 32 < kpad) {
#pragma unroll
            for (int j = 0; j < 4; j++) load4(c0 + 32 + warp + 8 * j, nv[j]);
        }
        const int64_t c = c0 + 4 * l;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int rr = warp * 16 + 4 * i + sub;
            const int64_t row = r0 + rr;
            if (row >= rows || c >= kpad) continue;
            const float sc = inv[rr];
            T* o = out + row * ldo + c;
            T q[4];
#pragma unroll
            for (int e = 0; e < 4; e++) q[e] = LowFmt<FMT>::cvt(tile[4 * l + e][rr] * sc);
            if (c + 3 < kpad) {
                store4(o, q);
            } else {
                for (int e = 0; e < 4 && c + e < kpad; e++) o[e] = q[e];
            }
        }
        __syncthreads();
    }
}

// B operand, K <= 4096: one CTA per column, read once into registers (16
// values per thread), the column's largest |x| reduced in the CTA, then the
// scaled values converted and written.
template <int FMT>
__global__ void __launch_bounds__(256) k_quant_col_cta(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                                       typename LowFmt<FMT>::T* __restrict__ out, int64_t ldo,
                                                       int64_t kpad, float* __restrict__ sb) {
    using T = typename LowFmt<FMT>::T;
    __shared__ float red[8];
    const int64_t c = blockIdx.x;
    const float* col = X + c * ldx;
    const int t = threadIdx.x;
    float v[16];
    float am = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int64_t r = 1024 * k + 4 * t;
        if (r + 3 < rows) {
            const float4 q = *reinterpret_cast<const float4*>(col + r);
            v[4 * k] = q.x;
            v[4 * k + 1] = q.y;
            v[4 * k + 2] = q.z;
            v[4 * k + 3] = q.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++) v[4 * k + e] = r + e < rows ? col[r + e] : 0.0f;
        }
#pragma unroll
        for (int e = 0; e < 4; e++) am = fmaxf(am, fabsf(v[4 * k + e]));
    }
    for (int off = 16; off > 0; off >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, off));
    if ((t & 31) == 0) red[t >> 5] = am;
    __syncthreads();
    float m = red[0];
#pragma unroll
    for (int w = 1; w < 8; w++) m = fmaxf(m, red[w]);
    const int e = LowFmt<FMT>::scale_exp(m);
    const float inv = ldexpf(1.0f, -e);
    if (t == 0) sb[c] = ldexpf(1.0f, e);
    T* o = out + c * ldo;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int64_t r = 1024 * k + 4 * t;
        if (r >= kpad) continue;
        T q[4];
#pragma unroll
        for (int e2 = 0; e2 < 4; e2++) q[e2] = LowFmt<FMT>::cvt(v[4 * k + e2] * inv);
        if (r + 3 < kpad) {
            store4(o + r, q);
        } else {
            for (int e2 = 0; e2 < 4 && r + e2 < kpad; e2++) o[r + e2] = q[e2];
        }
    }
}

// B operand: X (K rows x cols, column-major) -> out row c = X(:, c), sb[c] = 2^e.
// One warp per column.
template <int FMT>
__global__ void __launch_bounds__(256) k_quant_cols(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                                    int64_t cols, typename LowFmt<FMT>::T* __restrict__ out,
                                                    int64_t ldo, int64_t kpad, float* __restrict__ sb, int vec) {
    using T = typename LowFmt<FMT>::T;
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= cols) return;
    const float* col = X + c * ldx;
    float amax = 0.0f;
    if (vec) {      // four values per lane and load: 512 contiguous bytes per warp instruction
        int64_t r = 4 * lane;
        for (; r + 3 < rows; r += 128) {
            const float4 v = *reinterpret_cast<const float4*>(col + r);
            amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        for (; r < rows; r++) amax = fmaxf(amax, fabsf(col[r]));
    } else {
        for (int64_t r = lane; r < rows; r += 32) amax = fmaxf(amax, fabsf(col[r]));
    }
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    const int e = LowFmt<FMT>::scale_exp(amax);
    const float inv = ldexpf(1.0f, -e);
    if (lane == 0) sb[c] = ldexpf(1.0f, e);
    T* o = out + c * ldo;
    if (vec) {
        for (int64_t r = 4 * lane; r < kpad; r += 128) {
            T q[4];
            if (r + 3 < rows) {
                const float4 v = *reinterpret_cast<const float4*>(col + r);
                q[0] = LowFmt<FMT>::cvt(v.x * inv);
                q[1] = LowFmt<FMT>::cvt(v.y * inv);
                q[2] = LowFmt<FMT>::cvt(v.z * inv);
                q[3] = LowFmt<FMT>::cvt(v.w * inv);
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) q[k] = LowFmt<FMT>::cvt(r + k < rows ? col[r + k] * inv : 0.0f);
            }
            if (r + 3 < kpad) store4(o + r, q);
            else
                for (int k = 0; k < 4 && r + k < kpad; k++) o[r + k] = q[k];
        }
    } else {
        for (int64_t r = lane; r < kpad; r += 32) o[r] = LowFmt<FMT>::cvt(r < rows ? col[r] * inv : 0.0f);
    }
}

// Host side of the scaled operand copies.
template <int FMT>
static int quant_rows(const float* X, int64_t ldx, int64_t rows, int64_t cols, typename LowFmt<FMT>::T* out,
                      int64_t ldo, int64_t kpad, float* sa, cudaStream_t s) {
    if (rows <= 0) return HPL_OK;
    k_quant_rows<FMT><<<(unsigned)((rows + 127) / 128), 256, 0, s>>>(X, ldx, rows, cols, out, ldo, kpad, sa,
                                                                     vec4_ok(X, ldx));
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

template <int FMT>
static int quant_cols(const float* X, int64_t ldx, int64_t rows, int64_t cols, typename LowFmt<FMT>::T* out,
                      int64_t ldo, int64_t kpad, float* sb, cudaStream_t s) {
    if (cols <= 0) return HPL_OK;
    const int vec = vec4_ok(X, ldx);
    if (vec && kpad <= 4096 && cols <= 0x7fffffff) {
        k_quant_col_cta<FMT><<<(unsigned)cols, 256, 0, s>>>(X, ldx, rows, out, ldo, kpad, sb);
    } else {
        k_quant_cols<FMT><<<(unsigned)((cols + 7) / 8), 256, 0, s>>>(X, ldx, rows, cols, out, ldo, kpad, sb, vec);
    }
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

// ---------------------------------------------------------------------------
// Small dense kernels.
// ||A||_inf for the refinement's stopping test, taken once per solve from the
// FP32 working copy before it is factored (each |a_ij| within 2^-24 of the FP64
// value): the conversion (stored A) or the generator (regenerated A) leaves
// row sums of |F| per column chunk; the largest row is taken here.
__global__ void __launch_bounds__(256) k_abs_rowsum_max(int64_t n, int chunks, const float* __restrict__ part,
                                                        unsigned long long* out) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double v = 0.0;
    if (i < n)
        for (int c = 0; c < chunks; c++) v += (double)part[(int64_t)c * n + i];
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// FP32 working copy F of A; on the way, the row sums of |F| over `stripes`
// column stripes into part[stripe][row] (the refinement's ||A||_inf, reduced
// by k_abs_rowsum_max), so the norm costs no extra pass over the matrix.
// A32 (optional, n x n, ld n): the FP32 rounding of A as well, for GMRES's
// inner matrix-vector products.
__device__ __forceinline__ void st_a32(float* A32, int64_t idx, double d, float stored, bool fp32_stored) {
    if (A32) A32[idx] = fp32_stored ? stored : f64_to_f32_rn(d);
}

template <typename FT>
__global__ void __launch_bounds__(256) k_f64_to_f32_mat(int64_t n, const double* __restrict__ A, int64_t lda,
                                                        FT* __restrict__ F, int64_t ldf, int stripes,
                                                        float* __restrict__ part, float* __restrict__ A32) {
    constexpr bool kF32 = std::is_same<FT, float>::value;
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int64_t cw = (n + stripes - 1) / stripes;
    const int64_t j0 = (int64_t)blockIdx.y * cw, j1 = std::min<int64_t>(n, j0 + cw);
    float s0 = 0.0f, s1 = 0.0f;
    int64_t j = j0;
#pragma unroll 4
    for (; j + 1 < j1; j += 2) {
        const double d0 = A[j * lda + i], d1 = A[(j + 1) * lda + i];
        const float v0 = st_f64(F + j * ldf + i, d0), v1 = st_f64(F + (j + 1) * ldf + i, d1);
        st_a32(A32, j * n + i, d0, v0, kF32);
        st_a32(A32, (j + 1) * n + i, d1, v1, kF32);
        s0 += fabsf(v0);
        s1 += fabsf(v1);
    }
    if (j < j1) {
        const double d0 = A[j * lda + i];
        const float v0 = st_f64(F + j * ldf + i, d0);
        st_a32(A32, j * n + i, d0, v0, kF32);
        s0 += fabsf(v0);
    }
    part[(int64_t)blockIdx.y * n + i] = s0 + s1;
}

// BF16 working copy, two adjacent rows per thread so that a warp stores 128
// contiguous bytes per column (whole cache lines; 32 rows of 2-byte values
// would leave every line half written by each warp). n and ldf even.
__global__ void __launch_bounds__(256) k_f64_to_bf16_mat2(int64_t n, const double* __restrict__ A, int64_t lda,
                                                          __nv_bfloat16* __restrict__ F, int64_t ldf, int stripes,
                                                          float* __restrict__ part, float* __restrict__ A32) {
    const int64_t i = 2 * ((int64_t)blockIdx.x * 256 + threadIdx.x);
    if (i >= n) return;
    const int64_t cw = (n + stripes - 1) / stripes;
    const int64_t j0 = (int64_t)blockIdx.y * cw, j1 = std::min<int64_t>(n, j0 + cw);
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll 4
    for (int64_t j = j0; j < j1; j++) {
        const double2 a = *reinterpret_cast<const double2*>(A + j * lda + i);
        __nv_bfloat162 v;
        v.x = f64_to_bf16_rn(a.x);
        v.y = f64_to_bf16_rn(a.y);
        *reinterpret_cast<__nv_bfloat162*>(F + j * ldf + i) = v;
        if (A32) *reinterpret_cast<float2*>(A32 + j * n + i) = make_float2(f64_to_f32_rn(a.x), f64_to_f32_rn(a.y));
        s0 += fabsf(__bfloat162float(v.x));
        s1 += fabsf(__bfloat162float(v.y));
    }
    part[(int64_t)blockIdx.y * n + i] = s0;
    part[(int64_t)blockIdx.y * n + i + 1] = s1;
}

// Column-split GEMV for the preconditioner: part[s][r] = sum over the column
// chunk s of P(r, c) x[c]. P is FP32 column-major (rows x cols, ldp); each
// CTA takes 128 rows (4 per lane, float4 loads when aligned) and one column
// chunk, its 8 warps split the chunk's columns; k_gemv_combine then adds the
// chunks in order, so the result does not depend on scheduling.
__device__ __forceinline__ float4 ld_f4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld_f4(const __nv_bfloat16* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
}

template <typename PT>
__global__ void __launch_bounds__(256) k_gemv_part(int64_t rows, int64_t cols, const PT* __restrict__ P,
                                                   int64_t ldp, const float* __restrict__ x, int64_t chunk,
                                                   float* __restrict__ part, int64_t ldpart, int vec) {
    __shared__ float red[8][129];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 128 + 4 * lane;
    const int64_t c0 = (int64_t)blockIdx.y * chunk, c1 = min(cols, c0 + chunk);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (vec && r + 3 < rows) {
#pragma unroll 8
        for (int64_t c = c0 + warp; c < c1; c += 8) {
            const float4 v = ld_f4(P + c * ldp + r);
            const float xc = __ldg(x + c);
            a0 = fmaf(v.x, xc, a0);
            a1 = fmaf(v.y, xc, a1);
            a2 = fmaf(v.z, xc, a2);
            a3 = fmaf(v.w, xc, a3);
        }
    } else {
        for (int64_t c = c0 + warp; c < c1; c += 8) {
            const float xc = __ldg(x + c);
            const PT* pc = P + c * ldp;
            if (r < rows) a0 = fmaf(ld_f(pc + r), xc, a0);
            if (r + 1 < rows) a1 = fmaf(ld_f(pc + r + 1), xc, a1);
            if (r + 2 < rows) a2 = fmaf(ld_f(pc + r + 2), xc, a2);
            if (r + 3 < rows) a3 = fmaf(ld_f(pc + r + 3), xc, a3);
        }
    }
    red[warp][4 * lane] = a0;
    red[warp][4 * lane + 1] = a1;
    red[warp][4 * lane + 2] = a2;
    red[warp][4 * lane + 3] = a3;
    __syncthreads();
    if (threadIdx.x < 128) {
        const int64_t rr = (int64_t)blockIdx.x * 128 + threadIdx.x;
        float s = 0.f;
        for (int w = 0; w < 8; w++) s += red[w][threadIdx.x];
        if (rr < rows) part[blockIdx.y * ldpart + rr] = s;
    }
}

__global__ void k_gemv_combine(int64_t rows, int nsplit, const float* __restrict__ part, int64_t ldpart,
                               float* __restrict__ y, int sub) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < nsplit; q++) s += part[q * ldpart + r];
        y[r] = sub ? y[r] - s : s;
    }
}

// GMRES's inner product w = A32 z in FP32 data (opts.inner = FP32): A32 is
// the FP32 copy of A (n x n, ld lda), z the FP32 rounding of the vector. Each
// CTA takes 128 rows (4 per lane, float4 loads when aligned) and one column
// chunk, its 8 warps split the chunk's columns; every thread sums blocks of 32
// of its products in FP32 and adds each block into FP64 accumulators, so the
// result carries about the FP32 rounding of A and z and little of the summation.
// part[s][r] holds chunk s's FP64 sum; k_matvec32_combine adds the chunks in
// order (the result does not depend on scheduling).
__global__ void __launch_bounds__(256) k_matvec32_part(int64_t n, const float* __restrict__ A, int64_t lda,
                                                       const float* __restrict__ z, int64_t chunk,
                                                       double* __restrict__ part, int vec) {
    __shared__ double red[8][129];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 128 + 4 * lane;
    const int64_t c0 = (int64_t)blockIdx.y * chunk, c1 = min(n, c0 + chunk);
    const bool v4 = vec && r + 3 < n;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    int64_t c = c0 + warp;
    // blocks of 32 of the warp's columns (a fixed trip count, so the loads
    // pipeline): FP32 sums, then one FP64 add per row
    for (; c + 8 * 31 < c1; c += 8 * 32) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (v4) {
#pragma unroll 8
            for (int q = 0; q < 32; q++) {
                const float4 v = *reinterpret_cast<const float4*>(A + (c + 8 * q) * lda + r);
                const float zc = __ldg(z + c + 8 * q);
                a0 = fmaf(v.x, zc, a0);
                a1 = fmaf(v.y, zc, a1);
                a2 = fmaf(v.z, zc, a2);
                a3 = fmaf(v.w, zc, a3);
            }
        } else {
#pragma unroll 4
            for (int q = 0; q < 32; q++) {
                const float zc = __ldg(z + c + 8 * q);
                const float* pc = A + (c + 8 * q) * lda;
                if (r < n) a0 = fmaf(pc[r], zc, a0);
                if (r + 1 < n) a1 = fmaf(pc[r + 1], zc, a1);
                if (r + 2 < n) a2 = fmaf(pc[r + 2], zc, a2);
                if (r + 3 < n) a3 = fmaf(pc[r + 3], zc, a3);
            }
        }
        d0 += a0;
        d1 += a1;
        d2 += a2;
        d3 += a3;
    }
    {   // the rest: fewer than 32 of the warp's columns
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (; c < c1; c += 8) {
            const float zc = __ldg(z + c);
            const float* pc = A + c * lda;
            if (v4) {
                const float4 v = *reinterpret_cast<const float4*>(pc + r);
                a0 = fmaf(v.x, zc, a0);
                a1 = fmaf(v.y, zc, a1);
                a2 = fmaf(v.z, zc, a2);
                a3 = fmaf(v.w, zc, a3);
            } else {
                if (r < n) a0 = fmaf(pc[r], zc, a0);
                if (r + 1 < n) a1 = fmaf(pc[r + 1], zc, a1);
                if (r + 2 < n) a2 = fmaf(pc[r + 2], zc, a2);
                if (r + 3 < n) a3 = fmaf(pc[r + 3], zc, a3);
            }
        }
        d0 += a0;
        d1 += a1;
        d2 += a2;
        d3 += a3;
    }
    red[warp][4 * lane] = d0;
    red[warp][4 * lane + 1] = d1;
    red[warp][4 * lane + 2] = d2;
    red[warp][4 * lane + 3] = d3;
    __syncthreads();
    if (threadIdx.x < 128) {
        const int64_t rr = (int64_t)blockIdx.x * 128 + threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w][threadIdx.x];
        if (rr < n) part[blockIdx.y * n + rr] = t;
    }
}

__global__ void k_matvec32_combine(int64_t n, int nsplit, const double* __restrict__ part, double* __restrict__ w) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < nsplit; q++) t += part[q * n + r];
        w[r] = t;
    }
}

// The first Newton-Schulz step from X0 = diag(D)^-1: its products are
// diagonal scalings, X1_ij = x_i (2 delta_ij - D_ij x_j), x_i = 1 / D_ii, each
// operation rounded once in FP32 (explicit _rn operations: no contraction).
__global__ void k_ns_first(const float* __restrict__ D, int64_t ldd, int kb, float* __restrict__ X) {
    const int64_t total = (int64_t)kb * kb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / kb, i = t - j * kb;
        const float xi = 1.0f / D[i * ldd + i], xj = 1.0f / D[j * ldd + j];
        const float r = __fmul_rn(D[j * ldd + i], xj);
        X[t] = __fmul_rn(xi, __fsub_rn(i == j ? 2.0f : 0.0f, r));
    }
}

template <typename ST>
__global__ void k_copy_block32(const ST* __restrict__ src, int64_t lds, int64_t rows, int64_t cols,
                               float* __restrict__ dst, int64_t ldd) {
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = t / rows, i = t - j * rows;
        dst[j * ldd + i] = ld_f(src + j * lds + i);
    }
}

__global__ void k_zero_diag_flag(const float* __restrict__ D, int64_t ldd, int kb, int64_t k0, hpl_info* info) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kb; i += gridDim.x * blockDim.x)
        if (D[(int64_t)i * ldd + i] == 0.0f)
            atomicCAS((unsigned long long*)&info->info, 0ull, (unsigned long long)(k0 + i + 1));
}

// y (= or -=) P^T x: one warp per column c of P (rows x cols, FP32 column-
// major), lanes over the rows, shuffle reduction.
template <typename PT>
__global__ void __launch_bounds__(256) k_gemvT32(int64_t rows, int64_t cols, const PT* __restrict__ P,
                                                 int64_t ldp, const float* __restrict__ x, float* __restrict__ y,
                                                 int sub) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= cols) return;
    const PT* col = P + c * ldp;
    float acc = 0.0f;
#pragma unroll 4
    for (int64_t r = lane; r < rows; r += 32) acc = fmaf(ld_f(col + r), x[r], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) y[c] = sub ? y[c] - acc : acc;
}

// ---------------------------------------------------------------------------
// Several right-hand sides at once: classic refinement on the whole block,
// with the FP64 residual R = B - op(A) X as one DFMA product split over K and
// the preconditioner as FP32 block triangular solves with the factor's panels.
constexpr int kBlkSplit = 4;     // K slices of the block residual

// part[z] (m x nn, ld m) = op(A)(rows, K slice z) X(K slice z, cols), op(A) =
// A (TA = false, A m x kk column-major) or A^T (TA = true, A kk x m).
template <bool TA>
__global__ void __launch_bounds__(256) k_dgemm_part(int64_t m, int64_t nn, int64_t kk, int64_t kchunk,
                                                    const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ X, int64_t ldx,
                                                    double* __restrict__ part) {
    __shared__ double As[16][65], Xs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * 64, col0 = (int64_t)blockIdx.y * 64;
    const int64_t kb0 = (int64_t)blockIdx.z * kchunk, kb1 = min(kk, kb0 + kchunk);
    double acc[4][4] = {};
    for (int64_t k0 = kb0; k0 < kb1; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            int kq, r;
            if (TA) { r = e >> 4; kq = e & 15; }        // A^T: contiguous along K
            else { kq = e >> 6; r = e & 63; }
            const bool ok = k0 + kq < kb1 && row0 + r < m;
            As[kq][r] = ok ? (TA ? A[(row0 + r) * lda + k0 + kq] : A[(k0 + kq) * lda + row0 + r]) : 0.0;
        }
        for (int e = tid; e < 16 * 64; e += 256) {
            const int c = e >> 4, kq = e & 15;
            const bool ok = k0 + kq < kb1 && col0 + c < nn;
            Xs[kq][c] = ok ? X[(col0 + c) * ldx + k0 + kq] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kq = 0; kq < 16; kq++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kq][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Xs[kq][ty + 16 * j];
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* P = part + (int64_t)blockIdx.z * nn * m;
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t r = row0 + tx + 16 * i, c = col0 + ty + 16 * j;
            if (r < m && c < nn) P[c * m + r] = acc[i][j];
        }
}

// R = B - (sum of the K slices, in slice order); per column the largest |R|,
// |X| and |B| (bit patterns of non-negative doubles, atomicMax) into cmax.
__global__ void __launch_bounds__(256) k_resid_blk_finish(int64_t m, int64_t nn, int split,
                                                          const double* __restrict__ part,
                                                          const double* __restrict__ B, int64_t ldb,
                                                          double* __restrict__ R, int64_t ldr,
                                                          const double* __restrict__ X, int64_t ldx,
                                                          unsigned long long* cmax) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x, c = blockIdx.y;
    double ar = 0.0, ax = 0.0, ab = 0.0;
    if (i < m) {
        double acc = 0.0;
        for (int q = 0; q < split; q++) acc += part[((int64_t)q * nn + c) * m + i];
        const double b = B[c * ldb + i], r = b - acc;
        R[c * ldr + i] = r;
        ar = fabs(r);
        if (ar != ar) ar = __longlong_as_double(0x7ff0000000000000LL);
        ax = fabs(X[c * ldx + i]);
        ab = fabs(b);
    }
    for (int off = 16; off > 0; off >>= 1) {
        ar = fmax(ar, __shfl_down_sync(0xffffffffu, ar, off));
        ax = fmax(ax, __shfl_down_sync(0xffffffffu, ax, off));
        ab = fmax(ab, __shfl_down_sync(0xffffffffu, ab, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&cmax[3 * c], (unsigned long long)__double_as_longlong(ar));
        atomicMax(&cmax[3 * c + 1], (unsigned long long)__double_as_longlong(ax));
        atomicMax(&cmax[3 * c + 2], (unsigned long long)__double_as_longlong(ab));
    }
}

// C (m x nn, FP32) = or -= op(A) (m x kk) B (kk x nn), FP32 accumulation;
// op(A)(i, q) = A[q * lda + i] (TA = false) or A[i * lda + q] (TA = true).
// With P (split K): block z of the grid's z dimension takes the K slice
// [z kslice, (z + 1) kslice) and stores its partial product in P (slice z at
// P + z nn m, ld m) instead of touching C; k_sgemm_reduce adds the slices.
template <bool TA, typename AT>
__global__ void __launch_bounds__(256) k_sgemm(int64_t m, int64_t nn, int64_t kk, const AT* __restrict__ A,
                                               int64_t lda, const float* __restrict__ B, int64_t ldb,
                                               float* __restrict__ C, int64_t ldc, int sub, int64_t kslice,
                                               float* __restrict__ P) {
    __shared__ float As[16][65], Bs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * 64, col0 = (int64_t)blockIdx.y * 64;
    const int64_t kb0 = (int64_t)blockIdx.z * kslice, kb1 = min(kk, kb0 + kslice);
    float acc[4][4] = {};
    for (int64_t k0 = kb0; k0 < kb1; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            int kq, r;
            if (TA) { r = e >> 4; kq = e & 15; }
            else { kq = e >> 6; r = e & 63; }
            const bool ok = k0 + kq < kb1 && row0 + r < m;
            As[kq][r] = ok ? ld_f(TA ? A + (row0 + r) * lda + k0 + kq : A + (k0 + kq) * lda + row0 + r) : 0.0f;
        }
        for (int e = tid; e < 16 * 64; e += 256) {
            const int c = e >> 4, kq = e & 15;
            const bool ok = k0 + kq < kb1 && col0 + c < nn;
            Bs[kq][c] = ok ? B[(col0 + c) * ldb + k0 + kq] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kq = 0; kq < 16; kq++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kq][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kq][ty + 16 * j];
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* Pz = P ? P + (int64_t)blockIdx.z * nn * m : nullptr;
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t r = row0 + tx + 16 * i, c = col0 + ty + 16 * j;
            if (r < m && c < nn) {
                if (Pz) Pz[c * m + r] = acc[i][j];
                else C[c * ldc + r] = sub ? C[c * ldc + r] - acc[i][j] : acc[i][j];
            }
        }
}

// C (m x nn) = or -= the sum of the S K-slice partial products in P, added in
// slice order (the same bits on every run).
__global__ void __launch_bounds__(256) k_sgemm_reduce(int64_t m, int64_t nn, int S, const float* __restrict__ P,
                                                      float* __restrict__ C, int64_t ldc, int sub) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x, c = blockIdx.y;
    if (i >= m) return;
    float v = 0.0f;
    for (int z = 0; z < S; z++) v += P[((int64_t)z * nn + c) * m + i];
    C[c * ldc + i] = sub ? C[c * ldc + i] - v : v;
}

// Y (FP32, ld ldy) = X (FP64, ld ldx), m x nn; and back (add: Y += X).
__global__ void k_f64_to_f32_blk(int64_t m, int64_t nn, const double* __restrict__ X, int64_t ldx,
                                 float* __restrict__ Y, int64_t ldy) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x, c = blockIdx.y;
    if (i < m) Y[c * ldy + i] = (float)X[c * ldx + i];
}
__global__ void k_f32_to_f64_blk(int64_t m, int64_t nn, const float* __restrict__ Y, int64_t ldy,
                                 double* __restrict__ X, int64_t ldx, int add) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x, c = blockIdx.y;
    if (i < m) X[c * ldx + i] = add ? X[c * ldx + i] + (double)Y[c * ldy + i] : (double)Y[c * ldy + i];
}
__global__ void k_copy32_blk(int64_t m, int64_t nn, const float* __restrict__ S, int64_t lds, float* __restrict__ D,
                             int64_t ldd) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x, c = blockIdx.y;
    if (i < m) D[c * ldd + i] = S[c * lds + i];
}

// grad_A = -G X^T for G, X n x k (FP64, column-major): 64 x 64 output tiles,
// k staged 16 at a time in shared memory, 4 x 4 DFMA register tiles.
__global__ void __launch_bounds__(256) k_outer_neg(int64_t n, int64_t k, const double* __restrict__ G, int64_t ldg,
                                                   const double* __restrict__ X, int64_t ldx, double* __restrict__ C,
                                                   int64_t ldc) {
    __shared__ double Gs[16][65], Xs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * 64, col0 = (int64_t)blockIdx.y * 64;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < k; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            int kq = e >> 6, r = e & 63;
            bool okk = k0 + kq < k;
            Gs[kq][r] = (okk && row0 + r < n) ? G[(k0 + kq) * ldg + row0 + r] : 0.0;
            Xs[kq][r] = (okk && col0 + r < n) ? X[(k0 + kq) * ldx + col0 + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kq = 0; kq < 16; kq++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = Gs[kq][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Xs[kq][ty + 16 * j];
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int64_t r = row0 + tx + 16 * i, c = col0 + ty + 16 * j;
            if (r < n && c < n) C[c * ldc + r] = -acc[i][j];
        }
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ v, float* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)v[i];
}
__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ y, double* __restrict__ v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (double)y[i];
}
__global__ void k_copy32(int64_t n, const float* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// --- FP64 vector kernels of the refinement (deterministic reductions) ---
__global__ void __launch_bounds__(256) k_dot_partial(int64_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, double* __restrict__ part) {
    __shared__ double sm[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) s = fma(a[i], b[i], s);
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void __launch_bounds__(256) k_dot_final(int nparts, const double* __restrict__ part, double* out,
                                                   int take_sqrt) {
    __shared__ double sm[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 256) s += part[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = take_sqrt ? sqrt(sm[0]) : sm[0];
}
// y += sign * (*alpha) * x
__global__ void k_axpy_dev(int64_t n, const double* __restrict__ alpha, double sign, const double* __restrict__ x,
                           double* __restrict__ y) {
    const double a = sign * *alpha;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}
// y = x / (*s) (0 when *s == 0)
__global__ void k_scale_inv_dev(int64_t n, const double* __restrict__ sc, const double* __restrict__ x,
                                double* __restrict__ y) {
    const double d = *sc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = d != 0.0 ? x[i] / d : 0.0;
}
__global__ void k_add64(int64_t n, const double* __restrict__ d, double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}
// d = sum_t y[t] * Z[:, t]
__global__ void k_combine(int64_t n, int k, const double* __restrict__ Z, int64_t ldz, const double* __restrict__ y,
                          double* __restrict__ d) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < k; t++) s = fma(y[t], Z[t * ldz + i], s);
        d[i] = s;
    }
}

// ---------------------------------------------------------------------------
// Workspace.
struct MxpWs {
    void* F;           // n x n working matrix / factor (ld = n), FP32 or BF16
    float* Dinv;       // n x nb, D_k^-1 in rows k0..k0+kb (ld = n)
    uint16_t* opA;     // BF16 operand (n x nb8)
    uint16_t* opB;     // BF16 operand (n x nb8)
    uint16_t* nsD;     // split D as A operand (nb x 3 nb8)
    uint16_t* nsX;     // split X as A operand
    uint16_t* nsB;     // split X or T as B operand
    float* R;          // nb x nb
    float* X;          // nb x nb
    void* resws;       // residual partial sums
    double* r;         // n
    double* d;         // n
    double* V;         // n x (m+1)
    double* Z;         // n x m
    double* h;         // (m+1) x m Hessenberg on the device
    double* y;         // m coefficients
    double* part;      // dot partials
    double* scal;      // 4 device scalars (sr, beta, ...)
    float* y32;        // 2n FP32 scratch
    int* err;          // device error word of the GEMM kernels
    float* sa;         // n: FP8 / FP16 row scales of a scaled product's A operand
    float* sb;         // n: FP8 / FP16 column scales of its B operand
    float* gpart;      // kGemvSplitMax x n: column-split GEMV partial sums
    uint64_t* glo;     // kGemvSplitMax x n: exact row-sum partials of a regenerated matrix (low words)
    uint64_t* ghi;     // kGemvSplitMax x n: (high words)
    double* gdiag;     // n: FP64 diagonal of a regenerated matrix (A == NULL)
    // block refinement of nrhs_blk right-hand sides (absent when 0)
    float* Yb;         // n x nrhs_blk FP32
    float* Tb;         // nb x nrhs_blk FP32
    double* Rb;        // n x nrhs_blk FP64 residuals / corrections
    double* partb;     // kBlkSplit x n x nrhs_blk FP64 K slices of the residual
    unsigned long long* cmax;   // 3 x nrhs_blk column maxima
    // GMRES's inner products in FP32 data (opts.inner = FP32; absent otherwise)
    float* A32;        // n x n FP32 copy of A
    double* mvpart;    // kGemvSplitMax x n FP64 chunk sums of A32 z
};

static size_t mxp_ws_layout(int64_t n, int64_t nb, int m, MxpWs* w, char* base, int64_t nrhs_blk = 0,
                            int fbytes = 4, int a32 = 0, int opbytes = 2) {
    const int64_t nb8 = round8(nb);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return base ? (void*)(base + o) : (void*)nullptr;
    };
    MxpWs t;
    t.F = take((size_t)fbytes * n * n);
    t.Dinv = (float*)take(sizeof(float) * n * nb);
    t.opA = (uint16_t*)take((size_t)opbytes * n * nb8);      // BF16 / FP16 / FP8, or TF32 words
    t.opB = (uint16_t*)take((size_t)opbytes * n * nb8);
    t.nsD = (uint16_t*)take(2 * nb * 3 * nb8);
    t.nsX = (uint16_t*)take(2 * nb * 3 * nb8);
    t.nsB = (uint16_t*)take(2 * nb * 3 * nb8);
    t.R = (float*)take(sizeof(float) * nb * nb);
    t.X = (float*)take(sizeof(float) * nb * nb);
    t.resws = take(residual_ws_bytes(n));
    t.r = (double*)take(sizeof(double) * n);
    t.d = (double*)take(sizeof(double) * n);
    t.V = (double*)take(sizeof(double) * n * (m + 1));
    t.Z = (double*)take(sizeof(double) * n * m);
    t.h = (double*)take(sizeof(double) * (m + 1) * m);
    t.y = (double*)take(sizeof(double) * (m + 1));
    t.part = (double*)take(sizeof(double) * kDotBlocks);
    t.scal = (double*)take(sizeof(double) * 8);
    t.y32 = (float*)take(sizeof(float) * 2 * n);
    t.err = (int*)take(sizeof(int) * 4);
    t.sa = (float*)take(sizeof(float) * n);
    t.sb = (float*)take(sizeof(float) * n);
    t.gpart = (float*)take(sizeof(float) * kGemvSplitMax * n);
    t.glo = (uint64_t*)take(sizeof(uint64_t) * kGemvSplitMax * n);
    t.ghi = (uint64_t*)take(sizeof(uint64_t) * kGemvSplitMax * n);
    t.gdiag = (double*)take(sizeof(double) * n);
    t.Yb = (float*)take(sizeof(float) * n * nrhs_blk);
    t.Tb = (float*)take(sizeof(float) * nb * nrhs_blk);
    t.Rb = (double*)take(sizeof(double) * n * nrhs_blk);
    t.partb = (double*)take(sizeof(double) * kBlkSplit * n * nrhs_blk);
    t.cmax = (unsigned long long*)take(sizeof(unsigned long long) * 3 * nrhs_blk);
    // last, so that every offset above (the factor's included) is the same with or without it
    t.A32 = a32 ? (float*)take(sizeof(float) * n * n) : nullptr;
    t.mvpart = a32 ? (double*)take(sizeof(double) * kGemvSplitMax * n) : nullptr;
    if (w) *w = t;
    return off;
}

static unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

template <typename FT>
struct Mxp {
    int64_t n, nb;
    int m;
    Opts o;
    MxpWs w;
    cudaStream_t s;
    const double* A;        // FP64 matrix, or NULL: regenerated from seed
    int64_t lda;
    uint64_t seed = 0;
    uint64_t key = 0;       // generator stream key of the regenerated matrix
    bool trans = false;     // solve A^T x = b with the same factor (the adjoint)
    bool tnorm_ready = false;   // ||A^T||_inf cached in w.scal[7]
    static constexpr bool kBf16 = std::is_same<FT, __nv_bfloat16>::value;

    FT* F() const { return (FT*)w.F; }

    // the factor's product into the working matrix: C (FT) = or -= A B^T
    int gemm_c(int64_t M, int64_t N, int64_t K, const uint16_t* Aop, int64_t lda_, const uint16_t* Bop, int64_t ldb_,
               FT* C, int64_t ldc, int sub) {
        if constexpr (kBf16)
            return launch_gemm_bf16_c16(M, N, K, Aop, lda_, Bop, ldb_, (uint16_t*)C, ldc, sub, w.err, o.timeout_ns, 0,
                                        s);
        else
            return launch_gemm_bf16(M, N, K, Aop, lda_, Bop, ldb_, C, ldc, sub, w.err, o.timeout_ns, 0, s);
    }

    // r = b - op(A) x (b != NULL, scaled residual into sr if given) or r = op(A) x
    int resid(const double* x, const double* b, double* r, double* sr) {
        int slot = phase_begin(s);
        // ||A||_inf (w.scal[6]) comes from the factorization; ||A^T||_inf
        // (w.scal[7]) from the first transposed residual that needs it
        int st = trans ? launch_residual_vec_t(n, A, lda, w.scal + 7, sr ? (tnorm_ready ? 2 : 1) : 0, x, b, r, sr,
                                               w.resws, s)
                       : launch_residual_vec(n, A, lda, key, w.gdiag, w.scal + 6, x, b, r, sr, w.resws, s);
        if (trans && sr && b) tnorm_ready = true;
        phase_end(slot, s, PH_RESID, 8.0 * n * n);
        return st;
    }

    // y (= or -=) P x for an FP32 or BF16 column-major panel (rows x cols, ldp)
    template <typename PT>
    int gemv(int64_t rows, int64_t cols, const PT* P, int64_t ldp, const float* x, float* y, int sub) {
        if (rows <= 0) return HPL_OK;
        const int64_t rb = (rows + 127) / 128;
        int64_t nsplit = std::min<int64_t>(kGemvSplitMax, std::max<int64_t>(1, (1216 + rb - 1) / rb));
        nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, cols / 64));
        const int64_t chunk = (cols + nsplit - 1) / nsplit;
        nsplit = (cols + chunk - 1) / chunk;
        const int vec = (ldp % 4 == 0) && (((uintptr_t)P & (4 * sizeof(PT) - 1)) == 0);
        k_gemv_part<<<dim3((unsigned)rb, (unsigned)nsplit), 256, 0, s>>>(rows, cols, P, ldp, x, chunk, w.gpart, n, vec);
        HPL_LAUNCH_CHECK();
        k_gemv_combine<<<grid_for(rows), 256, 0, s>>>(rows, (int)nsplit, w.gpart, n, y, sub);
        HPL_LAUNCH_CHECK();
        return HPL_OK;
    }

    int dot(const double* a, const double* b, double* out, int take_sqrt) {
        k_dot_partial<<<kDotBlocks, 256, 0, s>>>(n, a, b, w.part);
        HPL_LAUNCH_CHECK();
        k_dot_final<<<1, 256, 0, s>>>(kDotBlocks, w.part, out, take_sqrt);
        HPL_LAUNCH_CHECK();
        return HPL_OK;
    }

    // ---- factorization ----
    int factor(hpl_info* info) {
        const int64_t ldf = n;
        HPL_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 4, s));
        int cslot = phase_begin(s);
        if (A) {
            bool paired = false;
            if constexpr (kBf16) {
                paired = n % 2 == 0 && lda % 2 == 0 && ((uintptr_t)A & 15) == 0;
                if (paired)
                    k_f64_to_bf16_mat2<<<dim3((unsigned)((n + 511) / 512), kGemvSplitMax), 256, 0, s>>>(
                        n, A, lda, F(), ldf, kGemvSplitMax, w.gpart, w.A32);
            }
            if (!paired)
                k_f64_to_f32_mat<<<dim3((unsigned)((n + 255) / 256), kGemvSplitMax), 256, 0, s>>>(
                    n, A, lda, F(), ldf, kGemvSplitMax, w.gpart, w.A32);
            HPL_LAUNCH_CHECK();
        } else {
            // one pass: the FP32 entries, the exact diagonal and the norm's row sums
            int st = launch_generate_dominant_f32(seed, n, F(), ldf, kBf16 ? 1 : 0, w.gdiag, &key, kGemvSplitMax,
                                                  w.glo, w.ghi, w.gpart, w.A32, s);
            if (st) return st;
        }
        HPL_CUDA_TRY(cudaMemsetAsync(w.scal + 6, 0, sizeof(double), s));
        k_abs_rowsum_max<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, kGemvSplitMax, w.gpart,
                                                                     (unsigned long long*)(w.scal + 6));
        HPL_LAUNCH_CHECK();
        phase_end(cslot, s, PH_CONVERT, (A ? 12.0 * n * n : 8.0 * n * n) + (w.A32 ? 4.0 * n * n : 0.0));
        for (int64_t k0 = 0; k0 < n; k0 += nb) {
            const int64_t kb = std::min(nb, n - k0), m2 = n - k0 - kb, kb8 = round8(kb), K3 = 3 * kb8;
            int slot = phase_begin(s);
            // the diagonal block as FP32: in place, or (BF16 storage) widened into
            // R, which the first Newton-Schulz product overwrites only after D
            // has been split into its operand
            const float* D;
            int64_t ldd;
            if constexpr (kBf16) {
                k_copy_block32<<<grid_for(kb * kb), 256, 0, s>>>(F() + k0 * ldf + k0, ldf, kb, kb, w.R, kb);
                HPL_LAUNCH_CHECK();
                D = w.R;
                ldd = kb;
            } else {
                D = F() + k0 * ldf + k0;
                ldd = ldf;
            }
            k_zero_diag_flag<<<1, 256, 0, s>>>(D, ldd, (int)kb, k0, info);
            HPL_LAUNCH_CHECK();
            int st;
            // split D as the A operand of the later steps' products: [hi | hi | lo]
            // (before k_ns_first: with BF16 storage D lives in R, which those products overwrite)
            if (o.ns_iters > 1 && (st = to_bf16_split3(D, ldd, kb, 1, 1, 1, 2, 0, w.nsD, kb8, s))) return st;
            k_ns_first<<<grid_for(kb * kb), 256, 0, s>>>(D, ldd, (int)kb, w.X);
            HPL_LAUNCH_CHECK();
            for (int it = 1; it < o.ns_iters; it++) {
                // R = D X: B operand from X, [hi | lo | hi]
                if ((st = to_bf16_split3(w.X, kb, kb, 0, 1, 2, 1, 0, w.nsB, kb8, s))) return st;
                if ((st = launch_gemm_bf16(kb, kb, K3, w.nsD, K3, w.nsB, K3, w.R, kb, 0, w.err, o.timeout_ns, 0, s)))
                    return st;
                // X = X (2I - R): A operand from X [hi | hi | lo], B operand from 2I - R [hi | lo | hi]
                if ((st = to_bf16_split3(w.X, kb, kb, 1, 1, 1, 2, 0, w.nsX, kb8, s))) return st;
                if ((st = to_bf16_split3(w.R, kb, kb, 0, 1, 2, 1, 1, w.nsB, kb8, s))) return st;
                if ((st = launch_gemm_bf16(kb, kb, K3, w.nsX, K3, w.nsB, K3, w.X, kb, 0, w.err, o.timeout_ns, 0, s)))
                    return st;
            }
            k_copy_block32<<<grid_for(kb * kb), 256, 0, s>>>(w.X, kb, kb, kb, w.Dinv + k0, n);
            HPL_LAUNCH_CHECK();
            if (kb < nb)   // a short last block: the rest of its slot holds zeros, not stale memory
                HPL_CUDA_TRY(cudaMemset2DAsync(w.Dinv + kb * n + k0, sizeof(float) * n, 0,
                                               sizeof(float) * (size_t)(n - k0), (size_t)(nb - kb), s));
            if (m2 > 0) {
                FT* A21 = F() + k0 * ldf + k0 + kb;
                FT* A12 = F() + (k0 + kb) * ldf + k0;
                FT* A22 = F() + (k0 + kb) * ldf + k0 + kb;
                // L21 = A21 D^-1 (FP16 operands with scales for FP16, else BF16;
                // a BF16-stored working matrix is always BF16)
                bool done = false;
                if constexpr (!kBf16) {
                    if (o.prec == HPL_PREC_FP16) {
                        if ((st = quant_rows<2>(A21, ldf, m2, kb, w.opA, kb8, kb8, w.sa, s))) return st;
                        if ((st = quant_cols<2>(w.X, kb, kb, kb, w.opB, kb8, kb8, w.sb, s))) return st;
                        if ((st = launch_gemm_f16(m2, kb, kb, w.opA, kb8, w.opB, kb8, w.sa, w.sb, A21, ldf, 0, w.err,
                                                  o.timeout_ns, 0, s)))
                            return st;
                        done = true;
                    } else if (o.prec == HPL_PREC_TF32) {
                        float* ta = (float*)w.opA;
                        float* tb = (float*)w.opB;
                        const int cv = phase_begin(s);
                        if ((st = to_tf32((const float*)A21, ldf, m2, kb, 1, ta, kb8, kb8, s))) return st;
                        if ((st = to_tf32(w.X, kb, kb, kb, 0, tb, kb8, kb8, s))) return st;
                        phase_end(cv, s, PH_OPCONV, (double)(m2 + kb) * kb * 8.0);
                        if ((st = launch_gemm_tf32(m2, kb, kb, ta, kb8, tb, kb8, (float*)A21, ldf, 0, w.err, o.timeout_ns,
                                                   0, s)))
                            return st;
                        done = true;
                    }
                }
                bool l21_copied = false;     // the BF16 operand copy of L21 is in opB already
                if (!done) {
                    // D^-1's copy in nsX (free after the Newton-Schulz steps), so that
                    // the product can write L21's BF16 copy for the update into opB
                    // as it stores L21 (FP32 working matrix, bulk-tensor epilogue)
                    const bool fuse = !kBf16 && o.prec == HPL_PREC_BF16 &&
                                      gemm_bf16_copy_ok((const float*)A21, ldf, w.opB, kb, kb8);
                    uint16_t* dcopy = fuse ? w.nsX : w.opB;
                    const int cv = phase_begin(s);
                    if ((st = to_bf16(A21, ldf, m2, kb, 1, 0, w.opA, kb8, 0, kb8, s))) return st;
                    if ((st = to_bf16(w.X, kb, kb, kb, 0, 0, dcopy, kb8, 0, kb8, s))) return st;
                    phase_end(cv, s, PH_OPCONV, (double)(m2 + kb) * kb * (sizeof(FT) + 2));
                    if (fuse) {
                        if ((st = launch_gemm_bf16_copy(m2, kb, kb, w.opA, kb8, dcopy, kb8, (float*)A21, ldf, w.opB,
                                                        kb8, w.err, o.timeout_ns, s)))
                            return st;
                        l21_copied = true;
                    } else if ((st = gemm_c(m2, kb, kb, w.opA, kb8, dcopy, kb8, A21, ldf, 0))) {
                        return st;
                    }
                }
                phase_end(slot, s, PH_PANEL, 2.0 * (o.ns_iters - 1) * 2.0 * 3.0 * kb * kb * kb + 2.0 * m2 * kb * kb);
                // A22 -= L21 A12 (the operand copies timed as PH_OPCONV, the product as PH_UPDATE)
                done = false;
                if constexpr (!kBf16) {
                if (o.prec == HPL_PREC_FP8_E4M3) {
                    const int64_t kb16 = (kb + 15) / 16 * 16;
                    uint8_t* qa = (uint8_t*)w.opA;
                    uint8_t* qb = (uint8_t*)w.opB;
                    const int cv = phase_begin(s);
                    if ((st = quant_rows<1>(A21, ldf, m2, kb, qa, kb16, kb16, w.sa, s))) return st;
                    if ((st = quant_cols<1>(A12, ldf, kb, m2, qb, kb16, kb16, w.sb, s))) return st;
                    phase_end(cv, s, PH_OPCONV, 2.0 * m2 * kb * (4 + 1));
                    const int ug = phase_begin(s);
                    if ((st = launch_gemm_fp8(m2, m2, kb, qa, kb16, qb, kb16, w.sa, w.sb, A22, ldf, 1, w.err,
                                              o.timeout_ns, 0, s)))
                        return st;
                    phase_end(ug, s, PH_UPDATE, 2.0 * m2 * m2 * kb);
                } else if (o.prec == HPL_PREC_FP16) {
                    const int cv = phase_begin(s);
                    if ((st = quant_rows<2>(A21, ldf, m2, kb, w.opA, kb8, kb8, w.sa, s))) return st;
                    if ((st = quant_cols<2>(A12, ldf, kb, m2, w.opB, kb8, kb8, w.sb, s))) return st;
                    phase_end(cv, s, PH_OPCONV, 2.0 * m2 * kb * (4 + 2));
                    const int ug = phase_begin(s);
                    if ((st = launch_gemm_f16(m2, m2, kb, w.opA, kb8, w.opB, kb8, w.sa, w.sb, A22, ldf, 1, w.err,
                                              o.timeout_ns, 0, s)))
                        return st;
                    phase_end(ug, s, PH_UPDATE, 2.0 * m2 * m2 * kb);
                } else if (o.prec == HPL_PREC_TF32) {
                    float* ta = (float*)w.opA;
                    float* tb = (float*)w.opB;
                    const int cv = phase_begin(s);
                    if ((st = to_tf32((const float*)A21, ldf, m2, kb, 1, ta, kb8, kb8, s))) return st;
                    if ((st = to_tf32((const float*)A12, ldf, kb, m2, 0, tb, kb8, kb8, s))) return st;
                    phase_end(cv, s, PH_OPCONV, 2.0 * m2 * kb * 8.0);
                    const int ug = phase_begin(s);
                    if ((st = launch_gemm_tf32(m2, m2, kb, ta, kb8, tb, kb8, (float*)A22, ldf, 1, w.err, o.timeout_ns, 0,
                                               s)))
                        return st;
                    phase_end(ug, s, PH_UPDATE, 2.0 * m2 * m2 * kb);
                }
                done = o.prec == HPL_PREC_FP8_E4M3 || o.prec == HPL_PREC_FP16 || o.prec == HPL_PREC_TF32;
                }
                if (!done && l21_copied) {
                    // L21's copy came with the product: only A12's, into opA
                    const int cv = phase_begin(s);
                    if ((st = to_bf16(A12, ldf, kb, m2, 0, 0, w.opA, kb8, 0, kb8, s))) return st;
                    phase_end(cv, s, PH_OPCONV, (double)m2 * kb * (sizeof(FT) + 2));
                    const int ug = phase_begin(s);
                    if ((st = gemm_c(m2, m2, kb, w.opB, kb8, w.opA, kb8, A22, ldf, 1))) return st;
                    phase_end(ug, s, PH_UPDATE, 2.0 * m2 * m2 * kb);
                } else if (!done) {
                    const int cv = phase_begin(s);
                    if ((st = to_bf16(A21, ldf, m2, kb, 1, 0, w.opA, kb8, 0, kb8, s))) return st;
                    if ((st = to_bf16(A12, ldf, kb, m2, 0, 0, w.opB, kb8, 0, kb8, s))) return st;
                    phase_end(cv, s, PH_OPCONV, 2.0 * m2 * kb * (sizeof(FT) + 2));
                    const int ug = phase_begin(s);
                    if ((st = gemm_c(m2, m2, kb, w.opA, kb8, w.opB, kb8, A22, ldf, 1))) return st;
                    phase_end(ug, s, PH_UPDATE, 2.0 * m2 * m2 * kb);
                }
            } else {
                phase_end(slot, s, PH_PANEL, 2.0 * (o.ns_iters - 1) * 2.0 * 3.0 * kb * kb * kb);
            }
        }
        return HPL_OK;
    }

    // ---- transposed preconditioner: out = M^-T v, M^T = U^T L^T ----
    // U^T is block lower with diagonal blocks D_k^T: forward, z_k = D_k^-T y_k,
    // then the later entries lose (U row panel of block k)^T z_k. L^T is block
    // unit upper: backward, y_k -= (L column panel below block k)^T y_below.
    int precondT(const double* v, double* out) {
        const int64_t ldf = n;
        float* y = w.y32;
        float* t = w.y32 + n;
        int slot = phase_begin(s);
        k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(n, v, y);
        HPL_LAUNCH_CHECK();
        for (int64_t k0 = 0; k0 < n; k0 += nb) {
            const int64_t kb = std::min(nb, n - k0), m2 = n - k0 - kb;
            k_gemvT32<<<(unsigned)((kb + 7) / 8), 256, 0, s>>>(kb, kb, w.Dinv + k0, n, y + k0, t, 0);
            HPL_LAUNCH_CHECK();
            k_copy32<<<grid_for(kb), 256, 0, s>>>(kb, t, y + k0);
            HPL_LAUNCH_CHECK();
            if (m2 > 0) {
                k_gemvT32<<<(unsigned)((m2 + 7) / 8), 256, 0, s>>>(kb, m2, F() + (k0 + kb) * ldf + k0, ldf, y + k0,
                                                                  y + k0 + kb, 1);
                HPL_LAUNCH_CHECK();
            }
        }
        const int64_t last = ((n - 1) / nb) * nb;
        for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
            const int64_t kb = std::min(nb, n - k0), m2 = n - k0 - kb;
            if (m2 > 0) {
                k_gemvT32<<<(unsigned)((kb + 7) / 8), 256, 0, s>>>(m2, kb, F() + k0 * ldf + k0 + kb, ldf, y + k0 + kb,
                                                                  y + k0, 1);
                HPL_LAUNCH_CHECK();
            }
        }
        k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(n, y, out);
        HPL_LAUNCH_CHECK();
        phase_end(slot, s, PH_OTHER, 4.0 * n * n + 4.0 * n * nb);
        return HPL_OK;
    }

    // ---- preconditioner: out = M^-1 v (FP64 in and out, FP32 inside) ----
    int precond(const double* v, double* out) {
        if (trans) return precondT(v, out);
        const int64_t ldf = n;
        float* y = w.y32;
        float* t = w.y32 + n;
        int slot = phase_begin(s);
        k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(n, v, y);
        HPL_LAUNCH_CHECK();
        for (int64_t k0 = 0; k0 < n; k0 += nb) {
            const int64_t kb = std::min(nb, n - k0), m2 = n - k0 - kb;
            if (m2 > 0) {
                int st = gemv(m2, kb, F() + k0 * ldf + k0 + kb, ldf, y + k0, y + k0 + kb, 1);
                if (st) return st;
            }
        }
        const int64_t last = ((n - 1) / nb) * nb;
        for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
            const int64_t kb = std::min(nb, n - k0);
            int st = gemv(kb, kb, w.Dinv + k0, n, y + k0, t, 0);
            if (st) return st;
            k_copy32<<<grid_for(kb), 256, 0, s>>>(kb, t, y + k0);
            HPL_LAUNCH_CHECK();
            if (k0 > 0) {
                st = gemv(k0, kb, F() + k0 * ldf, ldf, y + k0, y, 1);
                if (st) return st;
            }
        }
        k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(n, y, out);
        HPL_LAUNCH_CHECK();
        phase_end(slot, s, PH_OTHER, 4.0 * n * n + 4.0 * n * nb);
        return HPL_OK;
    }

    int read_scalar(const double* dev, double* host) {
        HPL_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        HPL_CUDA_TRY(cudaStreamSynchronize(s));
        return HPL_OK;
    }

    int check_err(int* status) {
        int e = 0;
        HPL_CUDA_TRY(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, s));
        HPL_CUDA_TRY(cudaStreamSynchronize(s));
        if (e) *status = e;
        return HPL_OK;
    }

    // out = A32 fl32(z) (FP64 out): GMRES's inner product in FP32 data.
    int matvec32(const double* z, double* out) {
        int slot = phase_begin(s);
        float* z32 = w.y32;
        k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(n, z, z32);
        HPL_LAUNCH_CHECK();
        const int64_t rb = (n + 127) / 128;
        int64_t nsplit = std::min<int64_t>(kGemvSplitMax, std::max<int64_t>(1, (1216 + rb - 1) / rb));
        nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, n / 64));
        const int64_t chunk = (n + nsplit - 1) / nsplit;
        nsplit = (n + chunk - 1) / chunk;
        const int vec = n % 4 == 0;
        k_matvec32_part<<<dim3((unsigned)rb, (unsigned)nsplit), 256, 0, s>>>(n, w.A32, n, z32, chunk, w.mvpart, vec);
        HPL_LAUNCH_CHECK();
        k_matvec32_combine<<<grid_for(n), 256, 0, s>>>(n, (int)nsplit, w.mvpart, out);
        HPL_LAUNCH_CHECK();
        phase_end(slot, s, PH_RESID, 4.0 * n * n);
        return HPL_OK;
    }

    // GMRES correction: d solves A d = r approximately (right preconditioning).
    int gmres(const double* r, double* d, int* inner) {
        const int64_t ldv = n;
        double beta = 0.0;
        int st;
        if ((st = dot(r, r, w.scal + 1, 1))) return st;
        if ((st = read_scalar(w.scal + 1, &beta))) return st;
        if (!(beta > 0.0) || !std::isfinite(beta)) {
            HPL_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(double) * n, s));
            return HPL_OK;
        }
        k_scale_inv_dev<<<grid_for(n), 256, 0, s>>>(n, w.scal + 1, r, w.V);
        HPL_LAUNCH_CHECK();
        std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0), y(m), col(m + 1);
        g[0] = beta;
        int kk = 0;
        for (int j = 0; j < m; j++) {
            double* vj = w.V + (int64_t)j * ldv;
            double* zj = w.Z + (int64_t)j * ldv;
            double* wv = w.V + (int64_t)(j + 1) * ldv;
            if ((st = precond(vj, zj))) return st;
            (*inner)++;
            if ((st = (w.A32 && !trans) ? matvec32(zj, wv) : resid(zj, nullptr, wv, nullptr))) return st;
            for (int i = 0; i <= j; i++) {
                double* hij = w.h + (int64_t)j * (m + 1) + i;
                if ((st = dot(wv, w.V + (int64_t)i * ldv, hij, 0))) return st;
                k_axpy_dev<<<grid_for(n), 256, 0, s>>>(n, hij, -1.0, w.V + (int64_t)i * ldv, wv);
                HPL_LAUNCH_CHECK();
            }
            double* hn = w.h + (int64_t)j * (m + 1) + j + 1;
            if ((st = dot(wv, wv, hn, 1))) return st;
            k_scale_inv_dev<<<grid_for(n), 256, 0, s>>>(n, hn, wv, wv);
            HPL_LAUNCH_CHECK();
            HPL_CUDA_TRY(cudaMemcpyAsync(col.data(), w.h + (int64_t)j * (m + 1), sizeof(double) * (j + 2),
                                         cudaMemcpyDeviceToHost, s));
            HPL_CUDA_TRY(cudaStreamSynchronize(s));
            for (int i = 0; i < j; i++) {                    // previous rotations
                double a = col[i], c = col[i + 1];
                col[i] = cs[i] * a + sn[i] * c;
                col[i + 1] = -sn[i] * a + cs[i] * c;
            }
            double a = col[j], c = col[j + 1];
            double rho = std::hypot(a, c);
            cs[j] = rho != 0.0 ? a / rho : 1.0;
            sn[j] = rho != 0.0 ? c / rho : 0.0;
            col[j] = rho;
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; i++) H[(size_t)j * (m + 1) + i] = col[i];
            kk = j + 1;
            if (std::fabs(g[j + 1]) <= 1e-10 * beta || rho == 0.0) break;
        }
        for (int i = kk - 1; i >= 0; i--) {
            double sacc = g[i];
            for (int q = i + 1; q < kk; q++) sacc -= H[(size_t)q * (m + 1) + i] * y[q];
            y[i] = sacc / H[(size_t)i * (m + 1) + i];
        }
        HPL_CUDA_TRY(cudaMemcpyAsync(w.y, y.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, s));
        k_combine<<<grid_for(n), 256, 0, s>>>(n, kk, w.Z, ldv, w.y, d);
        HPL_LAUNCH_CHECK();
        HPL_CUDA_TRY(cudaStreamSynchronize(s));    // y lives on the host stack
        return HPL_OK;
    }

    // Refine one right-hand side. Returns the HPL_* outcome.
    int refine(const double* b, double* x, int* iters, int* inner, double* sr_out, int* status) {
        int rslot = phase_begin(s);
        int st = refine_body(b, x, iters, inner, sr_out, status);
        phase_end(rslot, s, PH_REFINE, 0.0);
        return st;
    }

    int refine_body(const double* b, double* x, int* iters, int* inner, double* sr_out, int* status) {
        int st;
        if ((st = precond(b, x))) return st;
        int it = 0;
        double sr = INFINITY;
        *status = HPL_ERR_NOT_CONVERGED;
        for (;;) {
            if ((st = resid(x, b, w.r, w.scal))) return st;
            if ((st = read_scalar(w.scal, &sr))) return st;
            if (!std::isfinite(sr)) { *status = HPL_ERR_NONFINITE; break; }
            if (sr < o.tol) { *status = HPL_OK; break; }
            if (it >= o.max_iter) break;
            if (o.refine == HPL_REFINE_IR) {
                if ((st = precond(w.r, w.d))) return st;
                (*inner)++;
            } else {
                if ((st = gmres(w.r, w.d, inner))) return st;
            }
            k_add64<<<grid_for(n), 256, 0, s>>>(n, w.d, x);
            HPL_LAUNCH_CHECK();
            it++;
        }
        *iters = it;
        *sr_out = sr;
        return check_err(status);
    }

    // ---- several right-hand sides: classic refinement on the block ----
    int64_t nblk = 0;       // right-hand sides of the block buffers in w

    dim3 grid_blk(int64_t rows, int64_t cols) const { return dim3((unsigned)((rows + 255) / 256), (unsigned)cols); }

    // C (rows x k) -= or = op(P) (rows x kk) Y (kk x k), FP32. A product with
    // fewer 64 x 64 tiles than SMs and a long K is split along K into up to 8
    // slices (partial products in the residual's scratch, free while the
    // preconditioner runs), then the slices are added in order.
    template <typename PT>
    int sgemm(bool ta, int64_t rows, int64_t kk, const PT* P, int64_t ldp, const float* Y, int64_t ldy, float* C,
              int64_t ldc, int64_t k, int sub) {
        if (rows <= 0 || kk <= 0 || k <= 0) return HPL_OK;
        dim3 g((unsigned)((rows + 63) / 64), (unsigned)((k + 63) / 64));
        const int64_t tiles = (int64_t)g.x * g.y;
        int S = 1;
        if (tiles < kNumSMsGB300 && kk >= 512)
            S = (int)std::min<int64_t>({8, (kNumSMsGB300 + tiles - 1) / tiles, kk / 256});
        int64_t kslice = kk;
        float* part = nullptr;
        const int64_t cap = (int64_t)(2 * kBlkSplit) * n * nblk;      // floats in w.partb
        if (S > 1 && w.partb && (int64_t)S * rows * k <= cap) {
            kslice = ((kk + S - 1) / S + 15) / 16 * 16;
            S = (int)((kk + kslice - 1) / kslice);
            g.z = (unsigned)S;
            part = (float*)w.partb;
        }
        if (ta) k_sgemm<true, PT><<<g, 256, 0, s>>>(rows, k, kk, P, ldp, Y, ldy, C, ldc, sub, kslice, part);
        else k_sgemm<false, PT><<<g, 256, 0, s>>>(rows, k, kk, P, ldp, Y, ldy, C, ldc, sub, kslice, part);
        HPL_LAUNCH_CHECK();
        if (part) {
            k_sgemm_reduce<<<grid_blk(rows, k), 256, 0, s>>>(rows, k, S, part, C, ldc, sub);
            HPL_LAUNCH_CHECK();
        }
        return HPL_OK;
    }

    // Z (FP64, n x k, ldz) = M^-1 R or M^-T R (trans), R = w.Rb; add: Z += ...
    int precond_blk(int64_t k, double* Z, int64_t ldz, int add) {
        const int64_t ldf = n;
        float* Y = w.Yb;
        float* T = w.Tb;
        int slot = phase_begin(s), st;
        k_f64_to_f32_blk<<<grid_blk(n, k), 256, 0, s>>>(n, k, w.Rb, n, Y, n);
        HPL_LAUNCH_CHECK();
        const int64_t last = ((n - 1) / nb) * nb;
        if (!trans) {
            for (int64_t k0 = 0; k0 < n; k0 += nb) {
                const int64_t kb = std::min(nb, n - k0), m2 = n - k0 - kb;
                if ((st = sgemm(false, m2, kb, F() + k0 * ldf + k0 + kb, ldf, Y + k0, n, Y + k0 + kb, n, k, 1)))
                    return st;
            }
            for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
                const int64_t kb = std::min(nb, n - k0);
                if ((st = sgemm(false, kb, kb, w.Dinv + k0, n, Y + k0, n, T, nb, k, 0))) return st;
                k_copy32_blk<<<grid_blk(kb, k), 256, 0, s>>>(kb, k, T, nb, Y + k0, n);
                HPL_LAUNCH_CHECK();
                if ((st = sgemm(false, k0, kb, F() + k0 * ldf, ldf, Y + k0, n, Y, n, k, 1))) return st;
            }
        } else {
            for (int64_t k0 = 0; k0 < n; k0 += nb) {
                const int64_t kb = std::min(nb, n - k0), m2 = n - k0 - kb;
                if ((st = sgemm(true, kb, kb, w.Dinv + k0, n, Y + k0, n, T, nb, k, 0))) return st;
                k_copy32_blk<<<grid_blk(kb, k), 256, 0, s>>>(kb, k, T, nb, Y + k0, n);
                HPL_LAUNCH_CHECK();
                if ((st = sgemm(true, m2, kb, F() + (k0 + kb) * ldf + k0, ldf, Y + k0, n, Y + k0 + kb, n, k, 1)))
                    return st;
            }
            for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
                const int64_t kb = std::min(nb, n - k0), m2 = n - k0 - kb;
                if ((st = sgemm(true, kb, m2, F() + k0 * ldf + k0 + kb, ldf, Y + k0 + kb, n, Y + k0, n, k, 1)))
                    return st;
            }
        }
        k_f32_to_f64_blk<<<grid_blk(n, k), 256, 0, s>>>(n, k, Y, n, Z, ldz, add);
        HPL_LAUNCH_CHECK();
        phase_end(slot, s, PH_OTHER, (4.0 * n * n + 4.0 * n * nb) * (double)k);
        return HPL_OK;
    }

    // w.Rb = B - op(A) X for k columns, with each column's largest |r|, |x|,
    // |b| in w.cmax
    int resid_blk(int64_t k, const double* B, int64_t ldb, const double* X, int64_t ldx) {
        int slot = phase_begin(s);
        const int64_t kchunk = ((n + kBlkSplit - 1) / kBlkSplit + 15) / 16 * 16;
        dim3 g((unsigned)((n + 63) / 64), (unsigned)((k + 63) / 64), (unsigned)kBlkSplit);
        if (trans) k_dgemm_part<true><<<g, 256, 0, s>>>(n, k, n, kchunk, A, lda, X, ldx, w.partb);
        else k_dgemm_part<false><<<g, 256, 0, s>>>(n, k, n, kchunk, A, lda, X, ldx, w.partb);
        HPL_LAUNCH_CHECK();
        HPL_CUDA_TRY(cudaMemsetAsync(w.cmax, 0, sizeof(unsigned long long) * 3 * k, s));
        k_resid_blk_finish<<<grid_blk(n, k), 256, 0, s>>>(n, k, kBlkSplit, w.partb, B, ldb, w.Rb, n, X, ldx,
                                                          w.cmax);
        HPL_LAUNCH_CHECK();
        phase_end(slot, s, PH_RESID, 8.0 * n * n + 2.0 * n * n * (double)k);
        return HPL_OK;
    }

    // Refine k right-hand sides together: X = M^-1 B, then X += M^-1 (B - A X)
    // until every column's scaled residual is below tol.
    int refine_block(int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx, int* iters, double* sr_out,
                     int* status) {
        int rslot = phase_begin(s), st;
        double anorm = 0.0;
        if (trans && !tnorm_ready) {        // ||A^T||_inf once, through one transposed residual
            if ((st = resid(B, B, w.r, w.scal))) return st;
        }
        if ((st = read_scalar(w.scal + (trans ? 7 : 6), &anorm))) return st;
        for (int64_t c = 0; c < k; c++)
            HPL_CUDA_TRY(cudaMemcpyAsync(w.Rb + c * n, B + c * ldb, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        if ((st = precond_blk(k, X, ldx, 0))) return st;
        std::vector<unsigned long long> cm((size_t)(3 * k));
        int it = 0;
        double worst = INFINITY;
        *status = HPL_ERR_NOT_CONVERGED;
        for (;;) {
            if ((st = resid_blk(k, B, ldb, X, ldx))) return st;
            HPL_CUDA_TRY(cudaMemcpyAsync(cm.data(), w.cmax, sizeof(unsigned long long) * 3 * k,
                                         cudaMemcpyDeviceToHost, s));
            HPL_CUDA_TRY(cudaStreamSynchronize(s));
            worst = 0.0;
            bool finite = true;
            for (int64_t c = 0; c < k; c++) {
                double r, xm, bm;
                memcpy(&r, &cm[3 * c], 8);
                memcpy(&xm, &cm[3 * c + 1], 8);
                memcpy(&bm, &cm[3 * c + 2], 8);
                const double den = 0x1p-53 * (anorm * xm + bm) * (double)n;
                const double sr = den > 0.0 ? r / den : (r > 0.0 ? INFINITY : 0.0);
                if (!std::isfinite(sr)) finite = false;
                worst = std::max(worst, sr);
            }
            if (!finite) { *status = HPL_ERR_NONFINITE; break; }
            if (worst < o.tol) { *status = HPL_OK; break; }
            if (it >= o.max_iter) break;
            if ((st = precond_blk(k, X, ldx, 1))) return st;
            it++;
        }
        *iters = it;
        *sr_out = worst;
        phase_end(rslot, s, PH_REFINE, 0.0);
        return check_err(status);
    }
};

}  // namespace hplgb

using namespace hplgb;

// Right-hand sides refined as one block: several, with classic refinement.
static int64_t block_rhs(int64_t nrhs, const Opts& o) { return (nrhs > 1 && o.refine == HPL_REFINE_IR) ? nrhs : 0; }

static int fbytes_of(const Opts& o) { return o.storage == HPL_STORAGE_BF16 ? 2 : 4; }

// The FP32 copy of A for GMRES's inner products (opts.inner = FP32, GMRES only).
static int a32_of(const Opts& o) { return o.inner == HPL_INNER_FP32 && o.refine == HPL_REFINE_GMRES ? 1 : 0; }

// Bytes per element of the low-precision operand copies (TF32 keeps FP32 words).
static int opbytes_of(const Opts& o) { return o.prec == HPL_PREC_TF32 ? 4 : 2; }

// Option checks shared by the solve and its adjoint: the precision, and BF16
// storage only with BF16 operands.
static bool mxp_opts_ok(const Opts& o) {
    if (o.nb < 8 || (o.prec != HPL_PREC_BF16 && o.prec != HPL_PREC_FP8_E4M3 && o.prec != HPL_PREC_FP16 &&
                     o.prec != HPL_PREC_TF32))
        return false;
    if (o.storage != HPL_STORAGE_FP32 && o.storage != HPL_STORAGE_BF16) return false;
    if (o.storage == HPL_STORAGE_BF16 && o.prec != HPL_PREC_BF16) return false;
    return true;
}

extern "C" size_t mxp_workspace_size(int64_t n, int64_t nrhs, const hpl_opts* opts) {
    Opts o = resolve_opts(opts, kMxpDefaultNb);
    int64_t nb = std::min<int64_t>(o.nb, std::max<int64_t>(n, 1));
    return mxp_ws_layout(std::max<int64_t>(n, 1), nb, o.gmres_m, nullptr, nullptr, block_rhs(nrhs, o), fbytes_of(o),
                         a32_of(o), opbytes_of(o));
}

template <typename FT>
static int mxp_solve_t(int64_t n, int64_t nrhs, const double* A, int64_t lda, uint64_t seed, const double* B,
                       int64_t ldb, double* X, int64_t ldx, const Opts& o, void* ws, size_t ws_bytes, hpl_info* info,
                       void* stream) {
    Mxp<FT> mx;
    mx.n = n;
    mx.nb = std::min<int64_t>(o.nb, n);
    mx.m = o.gmres_m;
    mx.o = o;
    mx.s = (cudaStream_t)stream;
    mx.A = A;
    mx.lda = lda;
    mx.seed = seed;
    mx.nblk = A ? block_rhs(nrhs, o) : 0;       // the block residual reads a stored A
    size_t need = mxp_ws_layout(n, mx.nb, mx.m, nullptr, nullptr, mx.nblk, fbytes_of(o), a32_of(o), opbytes_of(o));
    if (!ws || ws_bytes < need) return HPL_ERR_NOMEM;
    if (((uintptr_t)ws & 255) || ((uintptr_t)info & 7)) return HPL_ERR_INVALID;
    mxp_ws_layout(n, mx.nb, mx.m, &mx.w, (char*)ws, mx.nblk, fbytes_of(o), a32_of(o), opbytes_of(o));
    cudaStream_t s = mx.s;
    HPL_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(hpl_info), s));
    int st = mx.factor(info);
    if (st) return st;
    hpl_info h;
    memset(&h, 0, sizeof(h));
    h.status = HPL_OK;
    HPL_CUDA_TRY(cudaMemcpyAsync(&h.info, &info->info, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HPL_CUDA_TRY(cudaStreamSynchronize(s));
    int worst = HPL_OK;
    double worst_sr = 0.0;
    int max_it = 0, inner = 0;
    if (mx.nblk) {
        if ((st = mx.refine_block(nrhs, B, ldb, X, ldx, &max_it, &worst_sr, &worst))) return st;
        inner = max_it + 1;
    } else {
        for (int64_t c = 0; c < nrhs; c++) {
            int it = 0, status = HPL_OK;
            double sr = 0.0;
            if ((st = mx.refine(B + c * ldb, X + c * ldx, &it, &inner, &sr, &status))) return st;
            if (status != HPL_OK && worst == HPL_OK) worst = status;
            max_it = std::max(max_it, it);
            worst_sr = std::max(worst_sr, sr);
        }
    }
    h.status = worst;
    if (h.info != 0 && worst == HPL_OK) h.status = HPL_ERR_SINGULAR;
    h.iters = max_it;
    h.inner_iters = inner;
    h.scaled_residual = worst_sr;
    HPL_CUDA_TRY(cudaMemcpyAsync(info, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    HPL_CUDA_TRY(cudaStreamSynchronize(s));
    return HPL_OK;
}

extern "C" int mxp_solve(int64_t n, int64_t nrhs, const double* A, int64_t lda, uint64_t seed, const double* B,
                         int64_t ldb, double* X, int64_t ldx, const hpl_opts* opts, void* ws, size_t ws_bytes,
                         hpl_info* info, void* stream) {
    if (n <= 0 || nrhs < 0 || (A && lda < n) || !info) return HPL_ERR_INVALID;
    if (nrhs > 0 && (!B || !X || ldb < n || ldx < n)) return HPL_ERR_INVALID;
    if (n > 0x7fffffff) return HPL_ERR_INVALID;
    Opts o = resolve_opts(opts, kMxpDefaultNb);
    if (!mxp_opts_ok(o)) return HPL_ERR_INVALID;
    if (o.refine != HPL_REFINE_IR && o.refine != HPL_REFINE_GMRES) return HPL_ERR_INVALID;
    if (o.ns_iters > 8) return HPL_ERR_INVALID;
    if (o.inner != HPL_INNER_FP64 && o.inner != HPL_INNER_FP32) return HPL_ERR_INVALID;
    if (o.storage == HPL_STORAGE_BF16)
        return mxp_solve_t<__nv_bfloat16>(n, nrhs, A, lda, seed, B, ldb, X, ldx, o, ws, ws_bytes, info, stream);
    return mxp_solve_t<float>(n, nrhs, A, lda, seed, B, ldb, X, ldx, o, ws, ws_bytes, info, stream);
}

// Adjoint of X = A^-1 B: grad_B = A^-T G by the same refinement with the
// transposed system (M^-T from the saved block factor as preconditioner, FP64
// residuals with A^T), then grad_A = -grad_B X^T (FP64 outer product).
template <typename FT>
static int lu_solve_backward_t(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X, int64_t ldx,
                               const double* G, int64_t ldg, double* gradB, int64_t ldgb, double* gradA, int64_t ldga,
                               const Opts& o, void* ws, size_t ws_bytes, hpl_info* info, void* stream) {
    Mxp<FT> mx;
    mx.n = n;
    mx.nb = std::min<int64_t>(o.nb, n);
    mx.m = o.gmres_m;
    mx.o = o;
    mx.s = (cudaStream_t)stream;
    mx.A = A;
    mx.lda = lda;
    mx.trans = true;
    mx.nblk = block_rhs(nrhs, o);
    size_t need = mxp_ws_layout(n, mx.nb, mx.m, nullptr, nullptr, mx.nblk, fbytes_of(o), 0, opbytes_of(o));
    if (ws_bytes < need) return HPL_ERR_NOMEM;
    if (((uintptr_t)ws & 255) || ((uintptr_t)info & 7)) return HPL_ERR_INVALID;
    mxp_ws_layout(n, mx.nb, mx.m, &mx.w, (char*)ws, mx.nblk, fbytes_of(o), 0, opbytes_of(o));
    cudaStream_t s = mx.s;
    HPL_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(hpl_info), s));
    HPL_CUDA_TRY(cudaMemsetAsync(mx.w.err, 0, sizeof(int) * 4, s));
    int st, worst = HPL_OK, max_it = 0, inner = 0;
    double worst_sr = 0.0;
    if (mx.nblk) {
        if ((st = mx.refine_block(nrhs, G, ldg, gradB, ldgb, &max_it, &worst_sr, &worst))) return st;
        inner = max_it + 1;
    } else {
        for (int64_t c = 0; c < nrhs; c++) {
            int it = 0, status = HPL_OK;
            double sr = 0.0;
            if ((st = mx.refine(G + c * ldg, gradB + c * ldgb, &it, &inner, &sr, &status))) return st;
            if (status != HPL_OK && worst == HPL_OK) worst = status;
            max_it = std::max(max_it, it);
            worst_sr = std::max(worst_sr, sr);
        }
    }
    if (gradA && nrhs > 0) {
        dim3 g((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64));
        if (g.y > 65535) return HPL_ERR_INVALID;
        int slot = phase_begin(s);
        k_outer_neg<<<g, 256, 0, s>>>(n, nrhs, gradB, ldgb, X, ldx, gradA, ldga);
        HPL_LAUNCH_CHECK();
        phase_end(slot, s, PH_OTHER, 2.0 * n * n * nrhs);
    } else if (gradA) {
        for (int64_t j = 0; j < n; j++) HPL_CUDA_TRY(cudaMemsetAsync(gradA + j * ldga, 0, sizeof(double) * n, s));
    }
    hpl_info h;
    memset(&h, 0, sizeof(h));
    h.status = worst;
    h.iters = max_it;
    h.inner_iters = inner;
    h.scaled_residual = worst_sr;
    HPL_CUDA_TRY(cudaMemcpyAsync(info, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    HPL_CUDA_TRY(cudaStreamSynchronize(s));
    return HPL_OK;
}

extern "C" int lu_solve_backward(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X, int64_t ldx,
                                 const double* G, int64_t ldg, double* gradB, int64_t ldgb, double* gradA,
                                 int64_t ldga, const hpl_opts* opts, void* ws, size_t ws_bytes, hpl_info* info,
                                 void* stream) {
    if (n <= 0 || nrhs < 0 || !A || lda < n || !info || !ws) return HPL_ERR_INVALID;
    if (nrhs > 0 && (!G || !gradB || ldg < n || ldgb < n)) return HPL_ERR_INVALID;
    if (gradA && (!X || ldx < n || ldga < n)) return HPL_ERR_INVALID;
    if (n > 0x7fffffff) return HPL_ERR_INVALID;
    Opts o = resolve_opts(opts, kMxpDefaultNb);
    if (!mxp_opts_ok(o)) return HPL_ERR_INVALID;
    if (o.storage == HPL_STORAGE_BF16)
        return lu_solve_backward_t<__nv_bfloat16>(n, nrhs, A, lda, X, ldx, G, ldg, gradB, ldgb, gradA, ldga, o, ws,
                                                  ws_bytes, info, stream);
    return lu_solve_backward_t<float>(n, nrhs, A, lda, X, ldx, G, ldg, gradB, ldgb, gradA, ldga, o, ws, ws_bytes,
                                      info, stream);
}
