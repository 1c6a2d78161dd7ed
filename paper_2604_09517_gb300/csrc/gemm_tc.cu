// Tensor-core GEMM for the mixed-precision factorization (paper Sec. III-A.2:
// factorization and trailing updates in low precision; the Aurora runs used
// "BF16-optimized kernels" with FP32 accumulation, Table I), BF16 or FP8 E4M3
// operands.
//
//   C (FP32, column-major, ldc) = sub ? C - A * B^T : A * B^T
//   A: M x K, K contiguous (row stride lda elements)
//   B: N x K, K contiguous (row stride ldb elements)
//
// Blackwell design: persistent, warp-specialised kernels, one CTA per SM.
//   warp 0      : TMA producer (cp.async.bulk.tensor, 128B swizzle)
//   warp 1      : TMEM allocator and single-thread tcgen05.mma issuer
//   warps 2..9  : epilogue (tcgen05.ld from TMEM, then C updated in FP32)
// With an FP32 C whose address and leading dimension suit the tensor memory
// accelerator, the epilogue stages each 32 x 32 chunk of the result in shared
// memory and hands it to a bulk tensor reduction (C += -(A B^T)) or store, so
// the SM never reads C: the read-modify-write happens in L2. Otherwise (BF16
// C, unaligned C) each thread reads and writes its row of C directly.
// The accumulator lives in TMEM, double buffered, so the epilogue of one tile
// overlaps the MMAs of the next; K advances 128 bytes per stage (one swizzle
// row). Tiles are walked in bands of row tiles so the A band stays in L2
// while B streams.
//   k_gemm_tc      : one CTA per 128 x BN tile (BN 256, or 128 for products
//                    with fewer tiles than SMs), 4 (6) stages.
//   k_gemm_tc_pair : two CTAs of a cluster per 256 x 256 tile with
//                    tcgen05.mma.cta_group::2; with the bulk-tensor epilogue
//                    3 stages of two swizzle atoms of K (64 KB per CTA), else
//                    7 stages of one; used for every product that has a
//                    256 x 256 tile for each pair of SMs.
// Every wait is bounded by a %globaltimer deadline; on expiry the CTA raises
// an error flag, drains what it has in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <type_traits>

#include "common.cuh"

namespace hplgb {
namespace tc {

constexpr int BM = 128;
constexpr int BKB = 128;                 // K bytes per stage: one 128-byte swizzle row
constexpr int A_BYTES = BM * BKB;
constexpr int THREADS = 320;
// Row tiles per band of the tile walk (measured on GB300 at M = N = 49152 and
// 95232, K = 3072: BF16 16 and FP8 32 for the single-CTA kernel).
template <int KIND>
constexpr int group_m() { return KIND == 1 ? 32 : 16; }
constexpr int GROUP_M_PAIR = 16;
// The pair kernel only for products up to this size (M x N): under the power
// cap, with FP32 C read and written every step, the single-CTA kernel is as
// fast or faster on the large trailing updates.
#ifndef HPLGB_PAIR_MAX_MN
#define HPLGB_PAIR_MAX_MN (16384LL * 16384LL)
#endif

// Tile width BN: 256 for large products; 128 when a product has fewer
// 128 x 256 tiles than the GPU has SMs (small Newton-Schulz
// products), which doubles the CTAs at work.
template <int BN_>
struct Tile {
    static constexpr int BN = BN_;
    static constexpr int B_BYTES = BN * BKB;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = BN == 256 ? 4 : 6;
    static constexpr int TMEM_COLS = 2 * BN;            // two accumulators
    static constexpr int DYN_SMEM = STAGES * STAGE_BYTES + 1024;
};
// Shared memory of the bulk-tensor epilogue: one 32 x 32 FP32 chunk per
// epilogue warp (column-major, 128 bytes per column).
constexpr int EPI_WARPS = 8;
constexpr int EPI_CHUNK_FLOATS = 32 * 32;
constexpr int EPI_SMEM = EPI_WARPS * EPI_CHUNK_FLOATS * 4;
template <int BN, bool TMA_EPI>
constexpr int dyn_smem() { return Tile<BN>::DYN_SMEM + (TMA_EPI ? EPI_SMEM : 0); }

// Operand kinds: 0 = BF16 (kind::f16, 2 bytes, 64 K per stage), 1 = FP8 E4M3
// (kind::f8f6f4, 1 byte, 128 K per stage), 2 = FP16 (kind::f16, 2 bytes),
// 3 = TF32 (kind::tf32, 4-byte FP32 words of which the MMA uses the sign,
// exponent and top 10 fraction bits; the operand copies are rounded to TF32
// beforehand, so the ignored bits are zero; 32 K per stage).
// Either way one MMA consumes 32 bytes of K (16 BF16 / FP16, 32 E4M3 or 8
// TF32 values); A and B always have the same type.
// Instruction descriptor: D = F32 (bits 4-5 = 1); A and B formats in bits
// 7-9 and 10-12 (kind::f16: F16 = 0, BF16 = 1; kind::tf32: TF32 = 2;
// kind::f8f6f4: E4M3 = 0); both K-major (bits 15, 16 = 0); N >> 3 at bits
// 17-22; M >> 4 at bits 24-28.
template <int KIND>
struct Kind;
template <>
struct Kind<0> {
    static constexpr int ELEM = 2;
    static constexpr uint32_t FORMATS = (1u << 4) | (1u << 7) | (1u << 10);
};
template <>
struct Kind<1> {
    static constexpr int ELEM = 1;
    static constexpr uint32_t FORMATS = (1u << 4);
};
template <>
struct Kind<2> {
    static constexpr int ELEM = 2;
    static constexpr uint32_t FORMATS = (1u << 4);
};
template <>
struct Kind<3> {
    static constexpr int ELEM = 4;
    static constexpr uint32_t FORMATS = (1u << 4) | (2u << 7) | (2u << 10);
};
template <int KIND, int BN>
__host__ __device__ constexpr uint32_t idesc() {
    return Kind<KIND>::FORMATS | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

struct Params {
    int M, N, K;
    void* C;               // float or __nv_bfloat16 (the kernels' CT)
    long long ldc;
    int sub;
    int* err;
    long long timeout_ns;
    const float* sa;       // optional per-row scale of the product (M)
    const float* sb;       // optional per-column scale of the product (N)
    int group_m;           // row tiles per band of the tile walk
    uint16_t* C16;         // optional BF16 copy of a stored product (sub = 0), row-major, ld16 a multiple of 8
    long long ld16;
};


__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait. Returns false (and raises the CTA's abort flag and the global
// error word) when the deadline passes or another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline, volatile int* abort,
                                          int* err) {
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (globaltimer_ns() > deadline) {
            *abort = 1;
            atomicExch(err, HPL_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Bulk tensor operations from shared memory to global memory (the epilogue):
// an element-wise add into the tensor (performed in L2), or a plain store.
// Completion is tracked per thread with bulk async-groups.
__device__ __forceinline__ void bulk_reduce_add_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     (uint64_t)map),
                 "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
                 "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the source shared memory of every committed group has been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed group has completed (its global writes are done)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the async proxy (TMA)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One 32-row x 32-column chunk of the product, held by a warp as r[j] =
// column j of the lane's row, scaled (row scale rs, optional column scales
// sb over the chunk's columns) and handed to the bulk-tensor epilogue:
// C += -value (sub) or C = value, at tensor coordinates (x = first row,
// y = first column). `stage` is the warp's 4 KB chunk of shared memory. The
// tensor map clips rows and columns outside C, so no masking is needed; only
// the scale reads are guarded. With a stored product (sub = 0) and C16, the
// lane also writes its row's 32 values rounded to BF16 to C16 (row-major,
// columns below ld16; the accumulator is zero past the product's last column,
// so the padding of each C16 row up to ld16 is written as zeros).
__device__ __forceinline__ void epi_chunk_tma(const CUtensorMap* tmC, float* stage, const uint32_t (&r)[32], float rs,
                                              const float* sb, int col0, int ncol_left, int sub, int x, int y,
                                              int lane, uint16_t* C16 = nullptr, long long ld16 = 0, int M = 0) {
    if (lane == 0) bulk_wait_read_all();      // the warp's previous chunk has left the stage
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; j++) {
        float v = __uint_as_float(r[j]) * rs;
        if (sb) v *= j < ncol_left ? sb[col0 + j] : 0.0f;
        stage[j * 32 + lane] = sub ? -v : v;
    }
    if (C16 && !sub && x + lane < M) {
        uint16_t* dst = C16 + (long long)(x + lane) * ld16 + y;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (y + 8 * q + 8 <= ld16) {
                __align__(16) __nv_bfloat16 h[8];
#pragma unroll
                for (int e = 0; e < 8; e++) h[e] = __float2bfloat16_rn(stage[(8 * q + e) * 32 + lane]);
                *reinterpret_cast<uint4*>(dst + 8 * q) = *reinterpret_cast<const uint4*>(h);
            }
        }
    }
    fence_async_smem();
    __syncwarp();
    if (lane == 0) {
        if (sub) bulk_reduce_add_2d(tmC, stage, x, y);
        else bulk_store_2d(tmC, stage, x, y);
        bulk_commit();
    }
}

// Shared-memory matrix descriptor for a K-major tile stored with the 128-byte
// swizzle (8 rows x 128 B atoms, 1024-byte aligned): start address >> 4 in
// bits 0-13, leading byte offset (unused for swizzled K-major; 1) in bits
// 16-29, stride byte offset 1024 >> 4 in bits 32-45, descriptor version 1 in
// bits 46-47, layout type 2 (128B swizzle) in bits 61-63.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

template <int KIND, int BN>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    if constexpr (KIND == 3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc<3, BN>()), "r"(accumulate)
            : "memory");
    } else if constexpr (KIND == 0 || KIND == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc<KIND, BN>()), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc<1, BN>()), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tile_coords(int t, int mt_count, int nt_count, int group, int& mt, int& nt) {
    const int per_group = group * nt_count;
    const int g = t / per_group;
    const int first = g * group;
    const int gsz = min(mt_count - first, group);
    const int r = t - g * per_group;
    mt = first + r % gsz;
    nt = r / gsz;
}

// C is FP32, or BF16 for a working matrix stored in BF16 (ld_f / st_f: read
// widened to FP32, the FP32 result rounded to nearest even when stored).
template <int KIND, int BN, typename CT, bool TMA_EPI>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmC, Params p) {
    constexpr int BK = BKB / Kind<KIND>::ELEM;     // K elements per stage
    constexpr int STAGES = Tile<BN>::STAGES, STAGE_BYTES = Tile<BN>::STAGE_BYTES, TMEM_COLS = Tile<BN>::TMEM_COLS;
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], drain_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    unsigned char* tiles = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt_count = (p.M + BM - 1) / BM, nt_count = (p.N + BN - 1) / BN;
    const int ntiles = mt_count * nt_count;
    const int nk = (p.K + BK - 1) / BK;
    const uint64_t deadline = globaltimer_ns() + (uint64_t)p.timeout_ns;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(&tfull_bar[a], 1);
            mbar_init(&tempty_bar[a], 8);
        }
        mbar_init(&drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int mt, nt;
                tile_coords(t, mt_count, nt_count, p.group_m, mt, nt);
                for (int kb = 0; kb < nk; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty_bar[s], ph ^ 1, deadline, &s_abort, p.err)) { ok = false; break; }
                    unsigned char* sa = tiles + s * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                    tma_load_2d(sa, &tmA, &full_bar[s], kb * BK, mt * BM);
                    tma_load_2d(sa + A_BYTES, &tmB, &full_bar[s], kb * BK, nt * BN);
                }
            }
            if (!ok) {
                // drain: every issued load completes before the CTA can exit
                const uint32_t first = it > STAGES ? it - STAGES : 0;
                for (uint32_t j = first; j < it; j++)
                    mbar_wait(&full_bar[j % STAGES], (j / STAGES) & 1, deadline + 1000000000ull, &s_abort, p.err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            uint32_t it = 0, tcount = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, tcount++) {
                const uint32_t acc = tcount & 1, aph = (tcount >> 1) & 1;
                if (!mbar_wait(&tempty_bar[acc], aph ^ 1, deadline, &s_abort, p.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + acc * BN;
                for (int kb = 0; kb < nk; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&full_bar[s], ph, deadline, &s_abort, p.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tiles + s * STAGE_BYTES);
                    const uint64_t ad = desc_sw128(sa), bd = desc_sw128(sa + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BKB / 32; kk++)     // 32 bytes of K per MMA: +2 in the address field
                        umma<KIND, BN>(d_tmem, ad + 2 * kk, bd + 2 * kk, (kb | kk) != 0);
                    umma_commit(&empty_bar[s]);
                }
                if (ok) umma_commit(&tfull_bar[acc]);
            }
            // all issued MMAs complete before TMEM is released
            umma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, deadline + 1000000000ull, &s_abort, p.err);
        }
    } else if constexpr (TMA_EPI) {
        // ---------------- epilogue: warps 2..9, through shared memory to a bulk tensor reduce ----------------
        // warp w reads TMEM lane quarter (w & 3) and the column half (w - 2) / 4
        // of the tile; the accumulator is released as soon as its last chunk
        // is in registers, so the next tile's MMAs start before the writes end.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        constexpr int CHUNKS = BN / 2 / 32;
        float* stage = (float*)(tiles + STAGES * STAGE_BYTES) + (warp - 2) * EPI_CHUNK_FLOATS;
        uint32_t tcount = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, tcount++) {
            int mt, nt;
            tile_coords(t, mt_count, nt_count, p.group_m, mt, nt);
            const uint32_t acc = tcount & 1, aph = (tcount >> 1) & 1;
            const int row0 = mt * BM + quarter * 32;
            const int row = row0 + lane;
            const int cbase = nt * BN + half * (BN / 2);
            const int ncol = min(BN / 2, p.N - cbase);
            const float rs = (p.sa && row < p.M) ? p.sa[row] : 1.0f;
            if (!mbar_wait(&tfull_bar[acc], aph, deadline, &s_abort, p.err)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < CHUNKS; c++) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BN + half * (BN / 2) + c * 32, r);
                tmem_wait_ld();
                if (c == CHUNKS - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty_bar[acc]);
                }
                if (c * 32 < ncol)
                    epi_chunk_tma(&tmC, stage, r, rs, p.sb, cbase + c * 32, ncol - c * 32, p.sub, row0,
                                  cbase + c * 32, lane, p.C16, p.ld16, p.M);
            }
        }
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..9 ----------------
        // warp w reads TMEM lane quarter (w & 3) and the column half (w - 2) / 4
        // of the tile. The C values of a tile's first 32-column chunk are
        // requested before its accumulator is ready (the HBM read overlaps the
        // wait for the MMAs), and those of the next chunk before the current
        // chunk is stored, so loads stay in flight.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_in_tile = quarter * 32 + lane;
        constexpr int CHUNKS = BN / 2 / 32;
        uint32_t tcount = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, tcount++) {
            int mt, nt;
            tile_coords(t, mt_count, nt_count, p.group_m, mt, nt);
            const uint32_t acc = tcount & 1, aph = (tcount >> 1) & 1;
            const int row = mt * BM + row_in_tile;
            const bool row_ok = row < p.M;
            const int cbase = nt * BN + half * (BN / 2);
            CT* cp = (CT*)p.C + (long long)cbase * p.ldc + row;
            const int ncol = min(BN / 2, p.N - cbase);      // valid columns of this half (may be <= 0)
            float cv[32];
            if (p.sub) {
#pragma unroll
                for (int j = 0; j < 32; j++) cv[j] = (row_ok && j < ncol) ? ld_f(cp + (long long)j * p.ldc) : 0.0f;
            }
            if (!mbar_wait(&tfull_bar[acc], aph, deadline, &s_abort, p.err)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < CHUNKS; c++) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BN + half * (BN / 2) + c * 32, r);
                float nv[32];
                if (p.sub && c + 1 < CHUNKS) {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const int jj = (c + 1) * 32 + j;
                        nv[j] = (row_ok && jj < ncol) ? ld_f(cp + (long long)jj * p.ldc) : 0.0f;
                    }
                }
                tmem_wait_ld();
                if (row_ok) {
                    const float rs = p.sa ? p.sa[row] : 1.0f;
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const int jj = c * 32 + j;
                        if (jj < ncol) {
                            float v = __uint_as_float(r[j]) * rs;
                            if (p.sb) v *= p.sb[cbase + jj];
                            st_f(cp + (long long)jj * p.ldc, p.sub ? cv[j] - v : v);
                        }
                    }
                }
                if (p.sub && c + 1 < CHUNKS) {
#pragma unroll
                    for (int j = 0; j < 32; j++) cv[j] = nv[j];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty_bar[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
}

// ---------------------------------------------------------------------------
// Pair kernel: the two CTAs of a cluster (two SMs) compute one 256 x 256 tile
// together with tcgen05.mma.cta_group::2. Each CTA stages only its own 128
// rows of A and its own 128 rows of B per K step (32 KB per swizzle atom of
// K), half the bytes per SM of the 128 x 256 single-CTA tile for the same MMA
// work, so the loads run further ahead (192 KB in flight per CTA).
//   leader (cluster rank 0): warp 0 TMA producer, warp 1 MMA issuer for the
//     pair (reads the A and B halves from both CTAs' shared memory, writes
//     rows 0..127 of the tile into its TMEM and rows 128..255 into the peer's)
//   peer (rank 1): warp 0 TMA producer
//   both: warps 2..9 epilogue of their own 128 rows.
// Both CTAs' loads of a stage complete on the leader's full barrier (TMA with
// .cta_group::2), which the leader arms with the bytes of both; the MMA
// commits arrive on the stage's empty barrier and on the accumulator barrier
// of both CTAs (multicast); both CTAs' epilogue warps arrive on the leader's
// tempty barrier.
constexpr int PAIR_ROWS = 128;                 // rows of A and of B staged by each CTA
// AT: 128-byte swizzle atoms of K per stage (1: 32 KB stages, 4 MMAs per
// barrier round trip; 2, the default with the bulk-tensor epilogue: 64 KB
// stages holding [A atom 0][A atom 1][B atom 0][B atom 1], 8 MMAs per round
// trip, half the stages, the same bytes in flight)
constexpr int PAIR_ATOM_BYTES = PAIR_ROWS * BKB;          // one operand half, one atom: 16 KB
template <int AT>
constexpr int pair_stage_bytes() { return 2 * AT * PAIR_ATOM_BYTES; }
template <bool TMA_EPI, int AT = 1>
constexpr int pair_stages() { return AT == 1 ? (TMA_EPI ? 6 : 7) : 3; }   // the bulk-tensor epilogue takes 32 KB
template <bool TMA_EPI, int AT = 1>
constexpr int pair_dyn_smem() {
    return pair_stages<TMA_EPI, AT>() * pair_stage_bytes<AT>() + 1024 + (TMA_EPI ? EPI_SMEM : 0);
}

template <int KIND>
__host__ __device__ constexpr uint32_t idesc_pair() {
    return Kind<KIND>::FORMATS | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on a
// barrier of either CTA of the pair (cluster address), e.g. the leader's.
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int x,
                                                 int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

template <int KIND>
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    if constexpr (KIND == 3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc_pair<3>()), "r"(accumulate)
            : "memory");
    } else if constexpr (KIND == 0 || KIND == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc_pair<KIND>()), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc_pair<1>()), "r"(accumulate)
            : "memory");
    }
}
// arrive on the barrier at this offset in both CTAs once the issued MMAs are done
__device__ __forceinline__ void umma_commit_pair_both(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}
__device__ __forceinline__ void umma_commit_pair_own(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

template <int KIND, typename CT, bool TMA_EPI, int AT = 1>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
    k_gemm_tc_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, Params p) {
    constexpr int BKA = BKB / Kind<KIND>::ELEM;     // K values per atom
    constexpr int BK = AT * BKA;                    // K values per stage
    constexpr int PAIR_STAGES = pair_stages<TMA_EPI, AT>();
    constexpr int PAIR_STAGE_BYTES = pair_stage_bytes<AT>();
    constexpr int HALF = AT * PAIR_ATOM_BYTES;      // bytes of one operand half per stage
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t full_bar[PAIR_STAGES], empty_bar[PAIR_STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], drain_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    unsigned char* tiles = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int pair = (int)cluster_id(), npairs = (int)cluster_count();
    const int mt_count = (p.M + 255) / 256, nt_count = (p.N + 255) / 256;
    const int ntiles = mt_count * nt_count;
    const int nk = (p.K + BK - 1) / BK;
    const uint64_t deadline = globaltimer_ns() + (uint64_t)p.timeout_ns;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < PAIR_STAGES; s++) {
            mbar_init(&full_bar[s], 1);      // the leader's producer arms it for both CTAs' bytes
            mbar_init(&empty_bar[s], 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(&tfull_bar[a], 1);
            mbar_init(&tempty_bar[a], 16);     // the 8 epilogue warps of each CTA
        }
        mbar_init(&drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    cluster_sync_all();      // both CTAs' barriers initialised and TMEM allocated
    tc_fence_after();
    const uint32_t tmem_base = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (each CTA: its own halves) ----------------
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
            uint32_t it = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs) {
                int mt, nt;
                tile_coords(t, mt_count, nt_count, p.group_m, mt, nt);
                for (int kb = 0; kb < nk; kb++, it++) {
                    const int s = it % PAIR_STAGES;
                    const uint32_t ph = (it / PAIR_STAGES) & 1;
                    if (!mbar_wait(&empty_bar[s], ph ^ 1, deadline, &s_abort, p.err)) { ok = false; break; }
                    unsigned char* sa = tiles + s * PAIR_STAGE_BYTES;
                    if (rank == 0) mbar_expect_tx(&full_bar[s], 2 * PAIR_STAGE_BYTES);
                    const uint32_t fb = cluster_addr(&full_bar[s], 0);
#pragma unroll
                    for (int a = 0; a < AT; a++) {
                        tma_load_2d_pair(sa + a * PAIR_ATOM_BYTES, &tmA, fb, kb * BK + a * BKA,
                                         mt * 256 + (int)rank * PAIR_ROWS);
                        tma_load_2d_pair(sa + HALF + a * PAIR_ATOM_BYTES, &tmB, fb, kb * BK + a * BKA,
                                         nt * 256 + (int)rank * PAIR_ROWS);
                    }
                }
            }
            if (!ok) {
                // the loads in flight complete on the leader's barriers, which
                // this CTA cannot watch: give them time to land before exit
                const uint64_t t0 = globaltimer_ns();
                while (globaltimer_ns() - t0 < 200000ull) __nanosleep(1000);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------- MMA issuer for the pair (leader) ----------------
            uint32_t it = 0, tcount = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs, tcount++) {
                const uint32_t acc = tcount & 1, aph = (tcount >> 1) & 1;
                if (!mbar_wait(&tempty_bar[acc], aph ^ 1, deadline, &s_abort, p.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + acc * 256;
                for (int kb = 0; kb < nk; kb++, it++) {
                    const int s = it % PAIR_STAGES;
                    const uint32_t ph = (it / PAIR_STAGES) & 1;
                    if (!mbar_wait(&full_bar[s], ph, deadline, &s_abort, p.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tiles + s * PAIR_STAGE_BYTES);
#pragma unroll
                    for (int a = 0; a < AT; a++) {
                        const uint64_t ad = desc_sw128(sa + a * PAIR_ATOM_BYTES);
                        const uint64_t bd = desc_sw128(sa + HALF + a * PAIR_ATOM_BYTES);
#pragma unroll
                        for (int kk = 0; kk < BKB / 32; kk++)
                            umma_pair<KIND>(d_tmem, ad + 2 * kk, bd + 2 * kk, (kb | a | kk) != 0);
                    }
                    umma_commit_pair_both(&empty_bar[s]);
                }
                if (ok) umma_commit_pair_both(&tfull_bar[acc]);
            }
            umma_commit_pair_own(&drain_bar);
            mbar_wait(&drain_bar, 0, deadline + 1000000000ull, &s_abort, p.err);
        }
    } else if constexpr (TMA_EPI) {
        // ---------------- epilogue: warps 2..9 of each CTA, its own 128 rows, bulk tensor reduce ----------------
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        constexpr int CHUNKS = 128 / 32;
        const uint32_t tempty_leader[2] = {cluster_addr(&tempty_bar[0], 0), cluster_addr(&tempty_bar[1], 0)};
        float* stage = (float*)(tiles + PAIR_STAGES * PAIR_STAGE_BYTES) + (warp - 2) * EPI_CHUNK_FLOATS;
        uint32_t tcount = 0;
        for (int t = pair; t < ntiles; t += npairs, tcount++) {
            int mt, nt;
            tile_coords(t, mt_count, nt_count, p.group_m, mt, nt);
            const uint32_t acc = tcount & 1, aph = (tcount >> 1) & 1;
            const int row0 = mt * 256 + (int)rank * PAIR_ROWS + quarter * 32;
            const int row = row0 + lane;
            const int cbase = nt * 256 + half * 128;
            const int ncol = min(128, p.N - cbase);
            const float rs = (p.sa && row < p.M) ? p.sa[row] : 1.0f;
            if (!mbar_wait(&tfull_bar[acc], aph, deadline, &s_abort, p.err)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < CHUNKS; c++) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * 256 + half * 128 + c * 32, r);
                tmem_wait_ld();
                if (c == CHUNKS - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_remote(tempty_leader[acc]);
                }
                if (c * 32 < ncol)
                    epi_chunk_tma(&tmC, stage, r, rs, p.sb, cbase + c * 32, ncol - c * 32, p.sub, row0,
                                  cbase + c * 32, lane, p.C16, p.ld16, p.M);
            }
        }
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..9 of each CTA, its own 128 rows ----------------
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_in_tile = (int)rank * PAIR_ROWS + quarter * 32 + lane;
        constexpr int CHUNKS = 128 / 32;
        const uint32_t tempty_leader[2] = {cluster_addr(&tempty_bar[0], 0), cluster_addr(&tempty_bar[1], 0)};
        uint32_t tcount = 0;
        for (int t = pair; t < ntiles; t += npairs, tcount++) {
            int mt, nt;
            tile_coords(t, mt_count, nt_count, p.group_m, mt, nt);
            const uint32_t acc = tcount & 1, aph = (tcount >> 1) & 1;
            const int row = mt * 256 + row_in_tile;
            const bool row_ok = row < p.M;
            const int cbase = nt * 256 + half * 128;
            CT* cp = (CT*)p.C + (long long)cbase * p.ldc + row;
            const int ncol = min(128, p.N - cbase);
            float cv[32];
            if (p.sub) {
#pragma unroll
                for (int j = 0; j < 32; j++) cv[j] = (row_ok && j < ncol) ? ld_f(cp + (long long)j * p.ldc) : 0.0f;
            }
            if (!mbar_wait(&tfull_bar[acc], aph, deadline, &s_abort, p.err)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < CHUNKS; c++) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * 256 + half * 128 + c * 32, r);
                float nv[32];
                if (p.sub && c + 1 < CHUNKS) {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const int jj = (c + 1) * 32 + j;
                        nv[j] = (row_ok && jj < ncol) ? ld_f(cp + (long long)jj * p.ldc) : 0.0f;
                    }
                }
                tmem_wait_ld();
                if (row_ok) {
                    const float rs = p.sa ? p.sa[row] : 1.0f;
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const int jj = c * 32 + j;
                        if (jj < ncol) {
                            float v = __uint_as_float(r[j]) * rs;
                            if (p.sb) v *= p.sb[cbase + jj];
                            st_f(cp + (long long)jj * p.ldc, p.sub ? cv[j] - v : v);
                        }
                    }
                }
                if (p.sub && c + 1 < CHUNKS) {
#pragma unroll
                    for (int j = 0; j < 32; j++) cv[j] = nv[j];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(tempty_leader[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();      // the leader's MMAs have drained; no CTA touches the other any more
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------
// Host side: tensor maps through the driver entry point (no libcuda link).

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

// rows x K matrix of `elem`-byte values, K contiguous, row stride ld
// elements; box of one 128-byte swizzle row (128 / elem values) x box_rows.
static int make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t K, int64_t ld, int box_rows, int elem) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return HPL_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * elem};
    cuuint32_t box[2] = {(cuuint32_t)(BKB / elem), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUresult r = enc(m, dt, 2,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HPL_OK : HPL_ERR_INVALID;
}

// C (FP32, column-major): rows x cols, leading dimension ld; box of 32 x 32
// (the epilogue's chunk), no swizzle.
static int make_map_c(CUtensorMap* m, const float* base, int64_t rows, int64_t cols, int64_t ld) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return HPL_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HPL_OK : HPL_ERR_INVALID;
}

// Tuning and diagnostics (hplgb_gemm_config): the epilogue kind (0: the
// bulk-tensor epilogue wherever C allows it, 1: always the per-thread one),
// an override of the band height of the tile walk (0: the per-kind default),
// and of the largest product (M x N) given to the pair kernel (0: default,
// < 0: never).
static int g_epilogue_mode = 0;
static int g_group_m_override = 0;
static long long g_pair_max_mn = 0;
// two atoms per stage: measured on GB300, n = 98304 MxP solve 502 -> 484 ms
// (BF16) and 343 -> 337 ms (FP8); BF16 products of 20480^2 x 4096 1391-1566
// -> 1670-1678 TF/s
static int g_pair_atoms = 2;

// The bulk-tensor epilogue: FP32 C at a 16-byte aligned address with a
// leading dimension that is a multiple of 4 (TMA strides are multiples of 16
// bytes), and rows / columns within the tensor map's 32-bit extents.
template <typename CT>
static bool tma_epilogue_ok(const CT* C, int64_t ldc) {
    if constexpr (!std::is_same<CT, float>::value) {
        return false;
    } else {
        return g_epilogue_mode == 0 && ((uintptr_t)C & 15) == 0 && ldc % 4 == 0;
    }
}

template <int KIND, int BN, typename CT, bool TMA_EPI>
static int launch_kind_epi(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mc, const Params& p,
                           int grid, cudaStream_t s) {
    static std::atomic<bool> attr_set[kMaxDevices];
    const int dv = device_slot();
    if (dv < 0) return HPL_ERR_CUDA;
    if (!attr_set[dv].load()) {
        HPL_CUDA_TRY(cudaFuncSetAttribute((const void*)k_gemm_tc<KIND, BN, CT, TMA_EPI>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem<BN, TMA_EPI>()));
        attr_set[dv].store(true);
    }
    k_gemm_tc<KIND, BN, CT, TMA_EPI><<<grid, THREADS, dyn_smem<BN, TMA_EPI>(), s>>>(ma, mb, mc, p);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

template <int KIND, int BN, typename CT = float>
static int launch_kind(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                       const float* sa, const float* sb, CT* C, int64_t ldc, int sub, int* err, int64_t timeout_ns,
                       int max_ctas, cudaStream_t s, uint16_t* C16 = nullptr, int64_t ld16 = 0) {
    constexpr int elem = Kind<KIND>::ELEM;
    if (M <= 0 || N <= 0) return HPL_OK;
    if (K <= 0) return HPL_ERR_INVALID;
    if (M > 0x7fffffff || N > 0x7fffffff || K > 0x7fffffff) return HPL_ERR_INVALID;
    // TMA: 16-byte aligned base addresses and row strides
    if (lda < K || ldb < K || ldc < M || (lda * elem) % 16 || (ldb * elem) % 16) return HPL_ERR_INVALID;
    if (((uintptr_t)A | (uintptr_t)B) & 15) return HPL_ERR_INVALID;
    CUtensorMap ma, mb, mc;
    int st = make_map(&ma, A, M, K, lda, BM, elem);
    if (st) return st;
    st = make_map(&mb, B, N, K, ldb, BN, elem);
    if (st) return st;
    const bool tma_epi = tma_epilogue_ok(C, ldc);
    memset(&mc, 0, sizeof(mc));
    if constexpr (std::is_same<CT, float>::value) {
        if (tma_epi && (st = make_map_c(&mc, C, M, N, ldc))) return st;
    }
    int dev = 0, sms = kNumSMsGB300;
    HPL_CUDA_TRY(cudaGetDevice(&dev));
    HPL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ntiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int grid = (int)std::min<int64_t>(ntiles, max_ctas > 0 ? std::min(max_ctas, sms) : sms);
    Params p;
    p.M = (int)M;
    p.N = (int)N;
    p.K = (int)K;
    p.C = C;
    p.ldc = ldc;
    p.sub = sub;
    p.err = err;
    p.timeout_ns = timeout_ns > 0 ? timeout_ns : kDefaultTimeoutNs;
    p.sa = sa;
    p.sb = sb;
    p.C16 = C16;
    p.ld16 = ld16;
    p.group_m = g_group_m_override > 0 ? g_group_m_override : group_m<KIND>();
    if (tma_epi) return launch_kind_epi<KIND, BN, CT, true>(ma, mb, mc, p, grid, s);
    return launch_kind_epi<KIND, BN, CT, false>(ma, mb, mc, p, grid, s);
}

// Clusters of the pair kernel that fit on the GPU at once (set-up once per
// instantiation; -1 on a CUDA error).
template <int KIND, typename CT, bool TMA_EPI, int AT = 1>
static int pair_capacity() {
    static std::atomic<int> cache[kMaxDevices];      // 0: not yet known
    const int dv = device_slot();
    if (dv < 0) return -1;
    int max_pairs = cache[dv].load();
    if (!max_pairs) {
        const void* f = (const void*)k_gemm_tc_pair<KIND, CT, TMA_EPI, AT>;
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, pair_dyn_smem<TMA_EPI, AT>()) !=
            cudaSuccess)
            return -1;
        int dev = 0, sms = kNumSMsGB300;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return -1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(sms & ~1));
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = pair_dyn_smem<TMA_EPI, AT>();
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, f, &cfg) != cudaSuccess) return -1;
        max_pairs = nc > 0 ? nc : sms / 2;
        cache[dv].store(max_pairs);
    }
    return max_pairs;
}

// The pair kernel: grid = 2 x min(tiles, clusters that fit at once).
template <int KIND, typename CT = float>
static int launch_pair(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                       const float* sa, const float* sb, CT* C, int64_t ldc, int sub, int* err, int64_t timeout_ns,
                       int max_ctas, cudaStream_t s, uint16_t* C16 = nullptr, int64_t ld16 = 0) {
    constexpr int elem = Kind<KIND>::ELEM;
    if (M <= 0 || N <= 0) return HPL_OK;
    if (K <= 0) return HPL_ERR_INVALID;
    if (M > 0x7fffffff || N > 0x7fffffff || K > 0x7fffffff) return HPL_ERR_INVALID;
    if (lda < K || ldb < K || ldc < M || (lda * elem) % 16 || (ldb * elem) % 16) return HPL_ERR_INVALID;
    if (((uintptr_t)A | (uintptr_t)B) & 15) return HPL_ERR_INVALID;
    CUtensorMap ma, mb, mc;
    int st = make_map(&ma, A, M, K, lda, PAIR_ROWS, elem);
    if (st) return st;
    st = make_map(&mb, B, N, K, ldb, PAIR_ROWS, elem);
    if (st) return st;
    const bool tma_epi = tma_epilogue_ok(C, ldc);
    memset(&mc, 0, sizeof(mc));
    if constexpr (std::is_same<CT, float>::value) {
        if (tma_epi && (st = make_map_c(&mc, C, M, N, ldc))) return st;
    }
    // two swizzle atoms per stage (switch 3 of hplgb_gemm_config)
    const bool two_atoms = g_pair_atoms == 2;
    const int max_pairs = two_atoms ? (tma_epi ? pair_capacity<KIND, CT, true, 2>() : pair_capacity<KIND, CT, false, 2>())
                                    : (tma_epi ? pair_capacity<KIND, CT, true>() : pair_capacity<KIND, CT, false>());
    if (max_pairs < 0) return HPL_ERR_CUDA;
    const int64_t ntiles = ((M + 255) / 256) * ((N + 255) / 256);
    int pairs = (int)std::min<int64_t>(ntiles, max_pairs);
    if (max_ctas > 0) pairs = std::max(1, std::min(pairs, max_ctas / 2));
    Params p;
    p.M = (int)M;
    p.N = (int)N;
    p.K = (int)K;
    p.C = C;
    p.ldc = ldc;
    p.sub = sub;
    p.err = err;
    p.timeout_ns = timeout_ns > 0 ? timeout_ns : kDefaultTimeoutNs;
    p.sa = sa;
    p.sb = sb;
    p.C16 = C16;
    p.ld16 = ld16;
    p.group_m = g_group_m_override > 0 ? g_group_m_override : GROUP_M_PAIR;
    if (two_atoms) {
        if (tma_epi)
            k_gemm_tc_pair<KIND, CT, true, 2><<<2 * pairs, THREADS, pair_dyn_smem<true, 2>(), s>>>(ma, mb, mc, p);
        else
            k_gemm_tc_pair<KIND, CT, false, 2><<<2 * pairs, THREADS, pair_dyn_smem<false, 2>(), s>>>(ma, mb, mc, p);
        HPL_LAUNCH_CHECK();
        return HPL_OK;
    }
    if (tma_epi)
        k_gemm_tc_pair<KIND, CT, true><<<2 * pairs, THREADS, pair_dyn_smem<true>(), s>>>(ma, mb, mc, p);
    else
        k_gemm_tc_pair<KIND, CT, false><<<2 * pairs, THREADS, pair_dyn_smem<false>(), s>>>(ma, mb, mc, p);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

// A product with a 256 x 256 tile for every SM pair goes to the pair kernel:
// any size when its epilogue is the bulk-tensor one (measured faster than the
// single-CTA kernel at every size: M = N = 20480 and 49152, K = 4096, BF16 +9
// and +4 %, FP8 +8 and +7 %), otherwise only up to HPLGB_PAIR_MAX_MN (with the
// per-thread epilogue the single-CTA kernel is as fast on large updates).
static bool pair_tiles(int64_t M, int64_t N, bool tma_epi) {
    const long long max_mn = g_pair_max_mn != 0 ? g_pair_max_mn : (tma_epi ? LLONG_MAX : HPLGB_PAIR_MAX_MN);
    return M * N <= max_mn && ((M + 255) / 256) * ((N + 255) / 256) >= kNumSMsGB300 / 2;
}

// Fewer 128 x 256 tiles than SMs: use 128 x 128 tiles.
static bool narrow_tiles(int64_t M, int64_t N) {
    return ((M + BM - 1) / BM) * ((N + 255) / 256) < kNumSMsGB300;
}

}  // namespace tc

// C = sub ? C - A B^T : A B^T (see the top of this file). max_ctas <= 0 means
// one CTA per SM. err: device int that receives HPL_ERR_TIMEOUT on a timeout.
int launch_gemm_bf16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                     float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns, int max_ctas, cudaStream_t s) {
    if (tc::pair_tiles(M, N, tc::tma_epilogue_ok(C, ldc)))
        return tc::launch_pair<0>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, sub, err, timeout_ns, max_ctas, s);
    if (tc::narrow_tiles(M, N))
        return tc::launch_kind<0, 128>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, sub, err, timeout_ns,
                                       max_ctas, s);
    return tc::launch_kind<0, 256>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, sub, err, timeout_ns, max_ctas,
                                   s);
}

// A stored BF16 product C = A B^T (FP32 C) that also writes C rounded to BF16,
// row-major, into C16 (ld16 >= N, a multiple of 8; columns N .. ld16-1 of each
// row written as zeros): the operand copy of the next product without a
// separate pass. Only where the bulk-tensor epilogue serves C
// (gemm_bf16_copy_ok); HPL_ERR_INVALID otherwise.
bool gemm_bf16_copy_ok(const float* C, int64_t ldc, const uint16_t* C16, int64_t N, int64_t ld16) {
    // columns N .. ld16-1 must lie in the last 32-column chunk that holds product columns
    return tc::tma_epilogue_ok(C, ldc) && C16 && ((uintptr_t)C16 & 15) == 0 && ld16 % 8 == 0 && ld16 >= N &&
           ld16 <= (N + 31) / 32 * 32;
}

int launch_gemm_bf16_copy(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                          int64_t ldb, float* C, int64_t ldc, uint16_t* C16, int64_t ld16, int* err, int64_t timeout_ns,
                          cudaStream_t s) {
    if (!gemm_bf16_copy_ok(C, ldc, C16, N, ld16)) return HPL_ERR_INVALID;
    if (tc::pair_tiles(M, N, true))
        return tc::launch_pair<0>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, 0, err, timeout_ns, 0, s, C16,
                                  ld16);
    if (tc::narrow_tiles(M, N))
        return tc::launch_kind<0, 128>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, 0, err, timeout_ns, 0, s,
                                       C16, ld16);
    return tc::launch_kind<0, 256>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, 0, err, timeout_ns, 0, s, C16,
                                   ld16);
}

// FP8 E4M3 operands (bytes, K contiguous); the product of row i and column j
// is multiplied by sa[i] * sb[j] before it is stored or subtracted.
int launch_gemm_fp8(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda, const uint8_t* B, int64_t ldb,
                    const float* sa, const float* sb, float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns,
                    int max_ctas, cudaStream_t s) {
    if (tc::pair_tiles(M, N, tc::tma_epilogue_ok(C, ldc)))
        return tc::launch_pair<1>(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, err, timeout_ns, max_ctas, s);
    if (tc::narrow_tiles(M, N))
        return tc::launch_kind<1, 128>(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, err, timeout_ns, max_ctas, s);
    return tc::launch_kind<1, 256>(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, err, timeout_ns, max_ctas, s);
}

// BF16 operands and a BF16 C (a working matrix stored in BF16): the FP32
// accumulator is combined with C in FP32 and rounded once when stored.
int launch_gemm_bf16_c16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                         int64_t ldb, uint16_t* C, int64_t ldc, int sub, int* err, int64_t timeout_ns, int max_ctas,
                         cudaStream_t s) {
    __nv_bfloat16* Cb = reinterpret_cast<__nv_bfloat16*>(C);
    if (tc::pair_tiles(M, N, tc::tma_epilogue_ok(Cb, ldc)))
        return tc::launch_pair<0>(M, N, K, A, lda, B, ldb, nullptr, nullptr, Cb, ldc, sub, err, timeout_ns, max_ctas, s);
    if (tc::narrow_tiles(M, N))
        return tc::launch_kind<0, 128>(M, N, K, A, lda, B, ldb, nullptr, nullptr, Cb, ldc, sub, err, timeout_ns,
                                       max_ctas, s);
    return tc::launch_kind<0, 256>(M, N, K, A, lda, B, ldb, nullptr, nullptr, Cb, ldc, sub, err, timeout_ns, max_ctas,
                                   s);
}

// FP16 operands (K contiguous) with the same per-row / per-column scales.
int launch_gemm_f16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                    const float* sa, const float* sb, float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns,
                    int max_ctas, cudaStream_t s) {
    if (tc::pair_tiles(M, N, tc::tma_epilogue_ok(C, ldc)))
        return tc::launch_pair<2>(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, err, timeout_ns, max_ctas, s);
    if (tc::narrow_tiles(M, N))
        return tc::launch_kind<2, 128>(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, err, timeout_ns, max_ctas, s);
    return tc::launch_kind<2, 256>(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, err, timeout_ns, max_ctas, s);
}

// TF32 operands (FP32 words already rounded to TF32, K contiguous), no scales.
int launch_gemm_tf32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                     float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns, int max_ctas, cudaStream_t s) {
    if (tc::pair_tiles(M, N, tc::tma_epilogue_ok(C, ldc)))
        return tc::launch_pair<3>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, sub, err, timeout_ns, max_ctas, s);
    if (tc::narrow_tiles(M, N))
        return tc::launch_kind<3, 128>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, sub, err, timeout_ns,
                                       max_ctas, s);
    return tc::launch_kind<3, 256>(M, N, K, A, lda, B, ldb, nullptr, nullptr, C, ldc, sub, err, timeout_ns, max_ctas,
                                   s);
}

}  // namespace hplgb

using namespace hplgb;

extern "C" int hplgb_gemm_tf32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                               int64_t ldb, float* C, int64_t ldc, int sub, int32_t* err, void* stream) {
    if (!err || !C || !A || !B) return HPL_ERR_INVALID;
    return launch_gemm_tf32(M, N, K, A, lda, B, ldb, C, ldc, sub, (int*)err, 0, 0, (cudaStream_t)stream);
}

extern "C" int hplgb_gemm_config(int what, long long value) {
    switch (what) {
        case 0:
            if (value < 0 || value > 1) return HPL_ERR_INVALID;
            tc::g_epilogue_mode = (int)value;
            return HPL_OK;
        case 1:
            if (value < 0 || value > 4096) return HPL_ERR_INVALID;
            tc::g_group_m_override = (int)value;
            return HPL_OK;
        case 2:
            tc::g_pair_max_mn = value;
            return HPL_OK;
        case 3:
            if (value != 1 && value != 2) return HPL_ERR_INVALID;
            tc::g_pair_atoms = (int)value;
            return HPL_OK;
        default:
            return HPL_ERR_INVALID;
    }
}

extern "C" int hplgb_gemm_bf16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                               int64_t ldb, float* C, int64_t ldc, int sub, int32_t* err, void* stream) {
    if (!err || !C || !A || !B) return HPL_ERR_INVALID;
    return launch_gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, sub, (int*)err, 0, 0, (cudaStream_t)stream);
}

extern "C" int hplgb_gemm_fp8(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda, const uint8_t* B,
                              int64_t ldb, const float* sa, const float* sb, float* C, int64_t ldc, int sub,
                              int32_t* err, void* stream) {
    if (!err || !C || !A || !B) return HPL_ERR_INVALID;
    return launch_gemm_fp8(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, (int*)err, 0, 0, (cudaStream_t)stream);
}

extern "C" int hplgb_gemm_f16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                              int64_t ldb, const float* sa, const float* sb, float* C, int64_t ldc, int sub,
                              int32_t* err, void* stream) {
    if (!err || !C || !A || !B) return HPL_ERR_INVALID;
    return launch_gemm_f16(M, N, K, A, lda, B, ldb, sa, sb, C, ldc, sub, (int*)err, 0, 0, (cudaStream_t)stream);
}
