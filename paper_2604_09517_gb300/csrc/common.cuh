// Shared helpers of the GPU library (host and device). Not used by the oracle.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>

#include "../../include/hplgb.h"

#define HPL_CUDA_TRY(expr)                                                       \
    do {                                                                         \
        cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            hplgb_internal_set_error(e_, #expr, __FILE__, __LINE__);             \
            return HPL_ERR_CUDA;                                                 \
        }                                                                        \
    } while (0)

#define HPL_LAUNCH_CHECK()          \
    do {                            \
        hplgb::count_launch();      \
        HPL_CUDA_TRY(cudaGetLastError()); \
    } while (0)

extern "C" void hplgb_internal_set_error(cudaError_t e, const char* what, const char* file, int line);
extern "C" void hplgb_internal_set_message(const char* msg);

namespace hplgb {

constexpr int kNumSMsGB300 = 152;
// Per-device caches (function attributes set, occupancy results) are indexed
// by the current device: a process that drives several GPUs prepares each.
constexpr int kMaxDevices = 64;
inline int device_slot() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}
constexpr int64_t kDefaultTimeoutNs = 20LL * 1000 * 1000 * 1000;

// Resolved options (defaults filled in).
struct Opts {
    int64_t nb;
    int lookahead;
    int prec;
    int refine;
    int max_iter;
    int gmres_m;
    int ns_iters;
    double tol;
    int64_t timeout_ns;
    int fp64_emulation;
    int pfact;
    int storage;
    int inner;
};
Opts resolve_opts(const hpl_opts* o, int64_t default_nb);

// Per-device state created once: the look-ahead stream and a pool of events.
struct DeviceCtx {
    int device;
    int num_sms;
    cudaStream_t side;          // high-priority stream for the panel
    cudaEvent_t ev[4];          // fork/join and look-ahead events (reused in order)
};
int get_ctx(DeviceCtx** out);

// Kernel launches issued by the library (all devices, all threads).
void count_launch();

// Optional per-phase timers (phases of the paper's per-panel cost model).
enum Phase {
    PH_PANEL = 0,     // PFACT (FP64) / diagonal-block inverse and L21 (mixed precision)
    PH_SWAP = 1,
    PH_TRSM = 2,
    PH_UPDATE = 3,
    PH_OTHER = 4,     // preconditioner applications, outer products
    PH_CONVERT = 5,   // FP64 -> FP32 copy of the matrix (mixed precision)
    PH_RESID = 6,     // FP64 residuals and matrix-vector products (refinement)
    PH_REFINE = 7,    // the whole refinement of one right-hand side (contains 4 and 6)
    PH_OPCONV = 8,    // low-precision operand copies of the mixed-precision products (L21, U12, D^-1)
    PH_COUNT = 9
};
int phase_begin(cudaStream_t s);                                   // -1 when timing is off
void phase_end(int slot, cudaStream_t s, int phase, double work, int step = -1);  // work: flops or bytes

// k_perm_pairs (lu64.cu): size of its table of rows beyond the block (a power
// of two >= 2 pb) and its dynamic shared memory, for blocks of pb pivots.
__host__ __device__ inline int perm_pairs_table(int pb) {
    int h = 1;
    while (h < 2 * pb) h <<= 1;
    return h;
}
inline size_t perm_pairs_smem(int pb) {
    return sizeof(int) * (5 * (size_t)pb + 2 * (size_t)perm_pairs_table(pb));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory and thread-block-cluster helpers (inline PTX).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster; release/acquire orders the shared
// memory writes before it with the remote reads after it
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ double ld_cluster_f64(uint32_t caddr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(caddr) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster_f64(uint32_t caddr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(caddr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_s64(uint32_t caddr, long long v) {
    asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(caddr), "l"(v) : "memory");
}
__device__ __forceinline__ long long ld_cluster_s64(uint32_t caddr) {
    long long v;
    asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(caddr) : "memory");
    return v;
}

// The generator's entry value (h >> 11) * 2^-53 - 0.5 from a SplitMix64
// output h, built with integer operations only: FP64 conversions and
// arithmetic issue at the FP64 rate, which is scarce on this part.
// t = (h >> 11) - 2^52 is the value in units of 2^-53, |t| <= 2^52.
__device__ __forceinline__ double gen_value(uint64_t h) {
    const long long t = (long long)(h >> 11) - (1LL << 52);
    if (t == 0) return 0.0;
    const unsigned long long u = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
    const int p = 63 - __clzll((long long)u);                  // leading one, 0..52: exact in FP64
    const unsigned long long mant = (u << (52 - p)) & ((1ull << 52) - 1);
    const unsigned long long bits =
        ((unsigned long long)(t < 0) << 63) | ((unsigned long long)(p - 53 + 1023) << 52) | mant;
    return __longlong_as_double((long long)bits);
}

// Magnitude key of a double for the pivot search: for |v| not NaN the IEEE
// bit pattern orders like the value, so the comparison runs on the integer
// pipe (FP64 compares issue at the FP64 rate, which is scarce on this part).
// NaN gets -1 and is never chosen, as with a floating-point ">".
__device__ __forceinline__ long long mag_key(double v) {
    const long long b = __double_as_longlong(v) & 0x7fffffffffffffffLL;
    return b > 0x7ff0000000000000LL ? -1LL : b;
}
__device__ __forceinline__ bool key_better(long long k, long long r, long long bk, long long br) {
    return k > bk || (k == bk && r < br);
}
// butterfly max over the warp: every lane ends with the winner
__device__ __forceinline__ void warp_best(long long& k, long long& r) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        long long ok = __shfl_xor_sync(0xffffffffu, k, off);
        long long orr = __shfl_xor_sync(0xffffffffu, r, off);
        if (key_better(ok, orr, k, r)) { k = ok; r = orr; }
    }
}

// Element access for a working matrix stored in FP32 or BF16: read widened
// to FP32; a stored FP32 value is rounded to nearest even once.
__device__ __forceinline__ float ld_f(const float* p) { return *p; }
__device__ __forceinline__ float ld_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st_f(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_f(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// FP64 -> BF16, round to nearest even in one step (no intermediate FP32
// rounding), by integer operations on the bits only (an FP64 conversion
// would issue at the FP64 rate, which is scarce on this part): the 52-bit
// fraction is rounded to 7 bits (a carry moves into the exponent), then
// re-biased. NaN stays NaN, infinities and overflow give infinity; values
// below BF16's normal range flush to a signed zero (the matrices here never
// produce them).
__device__ __forceinline__ __nv_bfloat16 f64_to_bf16_rn(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(u >> 63) << 15;
    unsigned long long a = u & 0x7fffffffffffffffull;
    const bool nan = a > 0x7ff0000000000000ull;
    a += (1ull << 44) - 1 + ((a >> 45) & 1);
    const int e = (int)(a >> 52) - 1023 + 127;
    unsigned short h = (unsigned short)(sgn | ((unsigned)e << 7) | (unsigned)((a >> 45) & 0x7f));
    if (e >= 255) h = (unsigned short)(sgn | 0x7f80u);
    if (e <= 0) h = (unsigned short)sgn;
    if (nan) h = (unsigned short)(sgn | 0x7fc0u);
    return __ushort_as_bfloat16(h);
}
// FP64 -> FP32, round to nearest even, by integer operations (as
// f64_to_bf16_rn, 23 fraction bits kept); values below FP32's normal range
// flush to a signed zero.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(u >> 63) << 31;
    unsigned long long a = u & 0x7fffffffffffffffull;
    const bool nan = a > 0x7ff0000000000000ull;
    a += (1ull << 28) - 1 + ((a >> 29) & 1);
    const int e = (int)(a >> 52) - 1023 + 127;
    unsigned h = sgn | ((unsigned)e << 23) | (unsigned)((a >> 29) & 0x7fffff);
    if (e >= 255) h = sgn | 0x7f800000u;
    if (e <= 0) h = sgn;
    if (nan) h = sgn | 0x7fc00000u;
    return __uint_as_float(h);
}

__device__ __forceinline__ float st_f64(float* p, double a) {
    const float v = (float)a;
    *p = v;
    return v;
}
__device__ __forceinline__ float st_f64(__nv_bfloat16* p, double a) {
    const __nv_bfloat16 v = f64_to_bf16_rn(a);
    *p = v;
    return __bfloat162float(v);
}

// Align a byte offset up.
__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace hplgb
