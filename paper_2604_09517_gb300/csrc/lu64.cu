// lu_factor: HPL's blocked right-looking LU with partial pivoting in FP64.
//
// Paper Sec. III-A.1: each step k factors the panel of width NB (PFACT),
// applies its row interchanges to the rest of the matrix (SWAP), solves for
// the block row U12 = L11^-1 A12 (DTRSM) and updates the trailing matrix
// A22 -= L21 U12 (DGEMM); look-ahead overlaps the next panel with the update
// (depth 1, Table I). On one GPU the broadcast phase disappears.
//
// GB300 notes. FP64 runs at ~2 FMA/clk/SM on this part (measured: DFMA
// 1.196 TFLOP/s, mma.sync f64 1.05 TFLOP/s), so the update is a DFMA kernel
// and every FP64 phase is bound by the same FP64 pipe; keeping that pipe busy
// is what look-ahead is for. The panel runs on a second, higher-priority
// stream, so its CTAs take SMs as soon as update CTAs retire.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace hplgb {

// ---------------------------------------------------------------------------
// Workspace layout of lu_factor (device memory supplied by the caller).
struct PanelSync {
    unsigned int count;
    unsigned int gen;
    int abort;
    int pad;
};

constexpr int kLeafW = 32;          // widest leaf of the recursive panel
constexpr int kLeafStride = 33;     // SMEM row stride (doubles) of the leaf
constexpr int kLeafThreads = 256;
constexpr int kMaxLeafCluster = 16;    // CTAs of the cluster panel leaf (the non-portable maximum)
constexpr int kMaxPanelCtas = 512;
// panels up to this many rows are factored by the cluster leaf when they fit
#ifndef HPLGB_CLUSTER_LEAF_MAX_ROWS
#define HPLGB_CLUSTER_LEAF_MAX_ROWS (1LL << 40)
#endif

struct Cand {
    double absval;
    long long row;
    double vals[kLeafW];
};

// FP64 accuracy from the BF16 tensor cores (opts.fp64_emulation): see
// emu_update below.
constexpr int kEmuSlices = 11;         // 6-bit slices: 66 bits below the top bit of each row / column
constexpr int kEmuBits = 6;
constexpr int kEmuGroups = kEmuSlices; // weights 2^-6g, g = 2 .. kEmuSlices + 1
constexpr int64_t kEmuChunk = 8192;    // columns of the trailing matrix per combine pass

struct LuWs {
    PanelSync* sync;
    Cand* slots;        // [2][kMaxPanelCtas]
    double* drow;       // [2][kLeafW]
    int* perm_cnt;      // [2]
    int* perm_dst;      // [2][2*nb]
    int* perm_src;      // [2][2*nb]
    int* emu_err;       // error word of the tensor-core GEMMs of the emulated update
    size_t base_bytes;  // the part above, cleared at every factorization
    // emulated update (absent unless requested)
    uint16_t* sA;       // n x (kEmuSlices kbp) BF16 slices of L21, row-major
    uint16_t* sB;       // n x (kEmuSlices kbp) BF16 slices of U12 (one column per row), slots reversed
    int* eA;            // n row exponents of L21
    int* eB;            // n column exponents of U12
    float* cg;          // kEmuGroups x n x kEmuChunk FP32 group products
};

static int64_t emu_kbp(int64_t nb) { return (nb + 7) / 8 * 8; }

static size_t lu_ws_layout(int64_t nb, LuWs* w, char* base, int64_t n_emu = 0) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return base ? (void*)(base + o) : (void*)nullptr;
    };
    void* p0 = take(sizeof(PanelSync));
    void* p1 = take(sizeof(Cand) * 2 * kMaxPanelCtas);
    void* p2 = take(sizeof(double) * 2 * kLeafW);
    void* p3 = take(sizeof(int) * 2);
    void* p4 = take(sizeof(int) * 2 * 2 * nb);
    void* p5 = take(sizeof(int) * 2 * 2 * nb);
    void* p6 = take(sizeof(int) * 4);
    const size_t base_bytes = off;
    const int64_t kbp = emu_kbp(nb), ne = n_emu;
    void* q0 = take(sizeof(uint16_t) * ne * kEmuSlices * kbp);
    void* q1 = take(sizeof(uint16_t) * ne * kEmuSlices * kbp);
    void* q2 = take(sizeof(int) * ne);
    void* q3 = take(sizeof(int) * ne);
    void* q4 = take(sizeof(float) * kEmuGroups * ne * std::min<int64_t>(ne, kEmuChunk));
    if (w) {
        w->sync = (PanelSync*)p0;
        w->slots = (Cand*)p1;
        w->drow = (double*)p2;
        w->perm_cnt = (int*)p3;
        w->perm_dst = (int*)p4;
        w->perm_src = (int*)p5;
        w->emu_err = (int*)p6;
        w->base_bytes = base_bytes;
        w->sA = (uint16_t*)q0;
        w->sB = (uint16_t*)q1;
        w->eA = (int*)q2;
        w->eB = (int*)q3;
        w->cg = (float*)q4;
    }
    return off;
}

// ---------------------------------------------------------------------------
// Grid-wide barrier for the cooperative panel kernel. Bounded: after the
// deadline it raises `abort`, every CTA sees it and the kernel returns.
__device__ bool grid_barrier(PanelSync* s, unsigned nblocks, uint64_t deadline) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &s->gen;
        volatile int* vab = &s->abort;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(&s->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&s->count, 0u);
            __threadfence();
            atomicAdd(&s->gen, 1u);
        } else {
            while (*vgen == g) {
                if (*vab) break;
                if (globaltimer_ns() > deadline) {
                    atomicExch(&s->abort, 1);
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)&s->abort == 0;
}

// Larger magnitude wins; on equal magnitude the smaller row index wins
// (first index attaining the maximum, as BLAS idamax).
__device__ __forceinline__ bool cand_better(double v, long long r, double bv, long long br) {
    return v > bv || (v == bv && r < br);
}

// PFACT leaf: factor columns [c0, c0+w) (w <= 32) of rows [c0, n) with
// partial pivoting. Cooperative launch, P CTAs; CTA b owns rows
// [c0 + b*rows_per, ...) of the leaf, staged in shared memory (row-major,
// stride 33). Per column: every CTA finds its local argmax (warp shuffles),
// publishes it with the candidate row's values (and the owner of the diagonal
// row publishes that row), one grid barrier, then every CTA picks the same
// global pivot, swaps, scales by the pivot (true division) and applies the
// rank-1 update with one warp per row and the multiplier broadcast by shuffle.
// The interchanges are also applied to the other columns of the enclosing
// NB-wide panel [pc0, pc0+pw) (the leaf's own columns live in SMEM).
__global__ void __launch_bounds__(kLeafThreads) k_panel_leaf(
    int64_t n, double* __restrict__ A, int64_t lda, int64_t c0, int w, int rows_per, int64_t pc0,
    int64_t pw, int32_t* __restrict__ ipiv, Cand* __restrict__ slots, double* __restrict__ drow,
    PanelSync* sync, hpl_info* info, int64_t timeout_ns) {
    extern __shared__ double sm[];
    __shared__ double s_piv[kLeafW], s_diag[kLeafW];
    __shared__ double s_wv[kLeafThreads / 32];
    __shared__ long long s_wr[kLeafThreads / 32];
    __shared__ long long s_p;
    __shared__ int s_win;

    const uint64_t deadline = globaltimer_ns() + (uint64_t)timeout_ns;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned P = gridDim.x;
    const int64_t m = n - c0;
    const int64_t rbeg = (int64_t)blockIdx.x * rows_per;           // local to c0
    const int nloc = (int)max((int64_t)0, min((int64_t)rows_per, m - rbeg));
    const int S = kLeafStride;

    for (int idx = tid; idx < nloc * w; idx += kLeafThreads) {
        int c = idx / nloc, r = idx - c * nloc;
        sm[r * S + c] = A[(c0 + c) * lda + c0 + rbeg + r];
    }
    // other panel columns handled by this thread for the interchanges
    const int64_t nother = pw - w;
    const int64_t gtid = (int64_t)blockIdx.x * kLeafThreads + tid;
    __syncthreads();

    for (int j = 0; j < w; j++) {
        const int par = j & 1;
        const int64_t rowj = c0 + j;                    // global diagonal row
        // local argmax over owned rows with global index >= rowj
        double bv = -1.0;
        long long br = 0x7fffffffffffffffLL;
        int rstart = (int)max((int64_t)0, (int64_t)j - rbeg);
        for (int r = rstart + tid; r < nloc; r += kLeafThreads) {
            double v = fabs(sm[r * S + j]);
            long long gr = c0 + rbeg + r;
            if (cand_better(v, gr, bv, br)) { bv = v; br = gr; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            double ov = __shfl_down_sync(0xffffffffu, bv, off);
            long long orr = __shfl_down_sync(0xffffffffu, br, off);
            if (cand_better(ov, orr, bv, br)) { bv = ov; br = orr; }
        }
        if (lane == 0) { s_wv[warp] = bv; s_wr[warp] = br; }
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < kLeafThreads / 32; q++)
                if (cand_better(s_wv[q], s_wr[q], bv, br)) { bv = s_wv[q]; br = s_wr[q]; }
            s_p = br;
            Cand* sl = slots + par * kMaxPanelCtas + blockIdx.x;
            sl->absval = bv;
            sl->row = br;
        }
        __syncthreads();
        {
            Cand* sl = slots + par * kMaxPanelCtas + blockIdx.x;
            long long mr = s_p;
            if (tid < w && mr != 0x7fffffffffffffffLL) sl->vals[tid] = sm[(int)(mr - c0 - rbeg) * S + tid];
            int64_t rd = rowj - c0 - rbeg;               // local index of the diagonal row
            if (rd >= 0 && rd < nloc && tid < w) drow[par * kLeafW + tid] = sm[rd * S + tid];
        }
        __threadfence();
        if (!grid_barrier(sync, P, deadline)) {
            if (blockIdx.x == 0 && tid == 0) info->status = HPL_ERR_TIMEOUT;
            return;
        }
        // global pivot: warp 0 scans the P candidates
        if (warp == 0) {
            double gv = -1.0;
            long long gr = 0x7fffffffffffffffLL;
            int gw = 0;
            for (unsigned q = lane; q < P; q += 32) {
                const volatile Cand* sl = slots + par * kMaxPanelCtas + q;
                double v = sl->absval;
                long long r = sl->row;
                if (cand_better(v, r, gv, gr)) { gv = v; gr = r; gw = (int)q; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                double ov = __shfl_down_sync(0xffffffffu, gv, off);
                long long orr = __shfl_down_sync(0xffffffffu, gr, off);
                int ow = __shfl_down_sync(0xffffffffu, gw, off);
                if (cand_better(ov, orr, gv, gr)) { gv = ov; gr = orr; gw = ow; }
            }
            if (lane == 0) {
                // no comparable candidate (the column holds only NaN): keep the diagonal row
                if (gr == 0x7fffffffffffffffLL) { gr = rowj; gw = -1; }
                s_p = gr;
                s_win = gw;
            }
        }
        __syncthreads();
        const long long p = s_p;
        if (tid < w) {
            double dv = ((volatile double*)drow)[par * kLeafW + tid];
            s_diag[tid] = dv;
            s_piv[tid] = s_win >= 0 ? ((const volatile Cand*)(slots + par * kMaxPanelCtas + s_win))->vals[tid] : dv;
        }
        __syncthreads();
        const double piv = s_piv[j];
        if (blockIdx.x == 0 && tid == 0) {
            ipiv[rowj] = (int32_t)p;
            if (piv == 0.0) atomicCAS((unsigned long long*)&info->info, 0ull, (unsigned long long)(rowj + 1));
        }
        // interchange rows rowj and p inside the leaf (SMEM) ...
        if (p != rowj) {
            int64_t rp = p - c0 - rbeg, rd = rowj - c0 - rbeg;
            if (rp >= 0 && rp < nloc && tid < w) sm[rp * S + tid] = s_diag[tid];
            if (rd >= 0 && rd < nloc && tid < w) sm[rd * S + tid] = s_piv[tid];
            // ... and in the panel's other columns (global memory)
            for (int64_t o = gtid; o < nother; o += (int64_t)P * kLeafThreads) {
                int64_t col = pc0 + (o < c0 - pc0 ? o : o + w);
                double* cp = A + col * lda;
                double t = cp[rowj];
                cp[rowj] = cp[p];
                cp[p] = t;
            }
        }
        __syncthreads();
        // scale the column below the diagonal (one true division per row: FP64
        // instructions are scarce on this part, so no lane repeats another's),
        // then the rank-1 update of the leaf's remaining columns, a warp per row
        if (piv != 0.0) {
            const int rs = (int)max((int64_t)0, rowj + 1 - c0 - rbeg);
            for (int r = rs + tid; r < nloc; r += kLeafThreads) sm[r * S + j] = sm[r * S + j] / piv;
            __syncthreads();
            if (j + 1 < w) {
                const double pl = (lane < w) ? s_piv[lane] : 0.0;
                for (int r = rs + warp; r < nloc; r += kLeafThreads / 32) {
                    const double l = sm[r * S + j];
                    if (lane > j && lane < w) sm[r * S + lane] = fma(-l, pl, sm[r * S + lane]);
                }
            }
        }
        __syncthreads();
    }
    for (int idx = tid; idx < nloc * w; idx += kLeafThreads) {
        int c = idx / nloc, r = idx - c * nloc;
        A[(c0 + c) * lda + c0 + rbeg + r] = sm[r * S + c];
    }
}

// PFACT leaf on one thread-block cluster, for panels whose rows fit in the
// cluster's shared memory (the short panels of a small matrix or of the last
// steps of a large one). Same pivots and arithmetic as k_panel_leaf (first
// row of largest magnitude, true division, one rank-1 update per column),
// organised around two facts of this part: FP64 instructions are scarce
// (about 2 FMA per clock per SM, and a warp instruction costs the same
// however few of its lanes are active), and a cluster barrier with
// distributed shared memory is much cheaper than a grid barrier through
// global memory.
//  * Pivot search on integer keys (mag_key); the search for column j + 1 is
//    fused into the rank-1 update of column j, by the threads that produce
//    column j + 1's new values.
//  * The rank-1 update maps threads densely onto the active (row, column)
//    pairs, so no FP64 instruction runs for finished columns.
//  * Exchange: per column every CTA pushes its candidate (key, row, values)
//    and, its owner, the diagonal row into the shared memory of every CTA of
//    the cluster (distributed shared memory stores, the destinations split
//    over the warps); one cluster barrier; then every CTA picks the winner
//    from its own copies, with no remote read on the critical path (reading
//    the candidates and then the winning row from their publishers after the
//    barrier cost two dependent remote round trips per column). The buffers
//    alternate by column parity: a CTA writes buffer j & 1 of another CTA
//    again only after the cluster barrier of column j + 1, which that CTA
//    passes after its reads of column j.
// W: leaf width bound (32 or 64; w <= W columns are factored).
template <int W>
__global__ void __launch_bounds__(kLeafThreads) k_panel_leaf_cl(
    int64_t n, double* __restrict__ A, int64_t lda, int64_t c0, int w, int rows_per, int64_t pc0, int64_t pw,
    int32_t* __restrict__ ipiv, hpl_info* info) {
    constexpr int S = W + 1;
    constexpr int NW = kLeafThreads / 32;
    extern __shared__ double sm[];
    __shared__ double cand_vals[2][kMaxLeafCluster][W], pub_diag[2][W];
    __shared__ long long cand_key[2][kMaxLeafCluster], cand_row[2][kMaxLeafCluster];
    __shared__ long long s_wk[NW], s_wr[NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned C = gridDim.x;                        // the launch is one cluster
    const unsigned me = cluster_rank();
    const int64_t m = n - c0;
    const int64_t rbeg = (int64_t)me * rows_per;
    const int nloc = (int)max((int64_t)0, min((int64_t)rows_per, m - rbeg));
    const long long kNone = 0x7fffffffffffffffLL;
    const long long grow0 = c0 + rbeg;                   // global row of local row 0

    for (int idx = tid; idx < nloc * w; idx += kLeafThreads) {
        int c = idx / nloc, r = idx - c * nloc;
        sm[r * S + c] = A[(c0 + c) * lda + grow0 + r];
    }
    const int64_t nother = pw - w;
    const int64_t gtid = (int64_t)me * kLeafThreads + tid;
    // every CTA of the cluster runs before any pushes into its shared memory
    cluster_sync_all();
    // this thread's candidate for column 0
    long long bk = -1, br = kNone;
    for (int r = tid; r < nloc; r += kLeafThreads) {
        long long k = mag_key(sm[r * S]);
        if (key_better(k, grow0 + r, bk, br)) { bk = k; br = grow0 + r; }
    }

    for (int j = 0; j < w; j++) {
        const int par = j & 1;
        const int64_t rowj = c0 + j;
        const int64_t rd = rowj - grow0;                 // local index of the diagonal row
        warp_best(bk, br);
        if (lane == 0) { s_wk[warp] = bk; s_wr[warp] = br; }
        __syncthreads();
        {
            // every warp forms the CTA's candidate and pushes it (and, in the
            // diagonal row's owner, that row) to the CTAs q = warp, warp + NW, ...
            long long k = lane < NW ? s_wk[lane] : -1, r = lane < NW ? s_wr[lane] : kNone;
            warp_best(k, r);
            const bool have = r != kNone, diag = rd >= 0 && rd < nloc;
            const int lr = have ? (int)(r - grow0) : 0;
            for (unsigned q = warp; q < C; q += NW) {
                if (lane == 0) {
                    st_cluster_s64(cluster_addr(&cand_key[par][me], q), k);
                    st_cluster_s64(cluster_addr(&cand_row[par][me], q), r);
                }
                if (have)
                    for (int c = lane; c < w; c += 32)
                        st_cluster_f64(cluster_addr(&cand_vals[par][me][c], q), sm[lr * S + c]);
                if (diag)
                    for (int c = lane; c < w; c += 32)
                        st_cluster_f64(cluster_addr(&pub_diag[par][c], q), sm[rd * S + c]);
            }
        }
        cluster_sync_all();
        // every warp picks the winner from the local copies (no CTA barrier):
        // the pivot row and the diagonal row are read where they were pushed
        long long gk = -1, gr = kNone, gw = -1;
        for (unsigned q = lane; q < C; q += 32) {
            const long long k = cand_key[par][q], r = cand_row[par][q];
            if (key_better(k, r, gk, gr)) { gk = k; gr = r; gw = (long long)q; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            long long ok = __shfl_xor_sync(0xffffffffu, gk, off);
            long long orr = __shfl_xor_sync(0xffffffffu, gr, off);
            long long ow = __shfl_xor_sync(0xffffffffu, gw, off);
            if (key_better(ok, orr, gk, gr)) { gk = ok; gr = orr; gw = ow; }
        }
        if (gr == kNone) { gr = rowj; gw = -1; }         // only NaN in the column: keep the diagonal row
        const double* diagrow = pub_diag[par];
        const double* pivrow = gw >= 0 ? cand_vals[par][gw] : diagrow;
        const long long p = gr;
        const double piv = pivrow[j];
        if (me == 0 && tid == 0) {
            ipiv[rowj] = (int32_t)p;
            if (piv == 0.0) atomicCAS((unsigned long long*)&info->info, 0ull, (unsigned long long)(rowj + 1));
        }
        const int64_t rp = p - grow0;
        const bool swap = p != rowj;
        // interchange rows rowj and p (row p's column j is written by the scaling
        // below when there is one), scale the column below the diagonal with one
        // true division per row, interchange in the panel's other columns
        if (swap && tid < w) {
            if (rp >= 0 && rp < nloc && (tid != j || piv == 0.0)) sm[rp * S + tid] = diagrow[tid];
            if (rd >= 0 && rd < nloc) sm[rd * S + tid] = pivrow[tid];
        }
        const int rs = (int)max((int64_t)0, (int64_t)(rowj + 1 - grow0));
        if (piv != 0.0)
            for (int r = rs + tid; r < nloc; r += kLeafThreads) {
                const double v = (swap && r == rp) ? diagrow[j] : sm[r * S + j];
                sm[r * S + j] = v / piv;
            }
        if (swap)
            for (int64_t o = gtid; o < nother; o += (int64_t)C * kLeafThreads) {
                int64_t col = pc0 + (o < c0 - pc0 ? o : o + w);
                double* cp = A + col * lda;
                double t = cp[rowj];
                cp[rowj] = cp[p];
                cp[p] = t;
            }
        __syncthreads();
        // rank-1 update of columns (j, w) on rows >= rs, threads dense over the
        // active pairs; the producers of column j + 1 track its pivot candidate
        bk = -1;
        br = kNone;
        if (j + 1 < w) {
            const int ncol = w - j - 1, nr = nloc - rs;
            if (piv != 0.0) {
                int q = tid / ncol, cc = tid - q * ncol;
                const int dq = kLeafThreads / ncol, dc = kLeafThreads - dq * ncol;
                while (q < nr) {
                    const int r = rs + q, c = j + 1 + cc;
                    const double a = fma(-sm[r * S + j], pivrow[c], sm[r * S + c]);
                    sm[r * S + c] = a;
                    if (cc == 0) {
                        long long k = mag_key(a);
                        if (key_better(k, grow0 + r, bk, br)) { bk = k; br = grow0 + r; }
                    }
                    cc += dc;
                    q += dq;
                    if (cc >= ncol) { cc -= ncol; q++; }
                }
            } else {
                for (int r = rs + tid; r < nloc; r += kLeafThreads) {
                    long long k = mag_key(sm[r * S + j + 1]);
                    if (key_better(k, grow0 + r, bk, br)) { bk = k; br = grow0 + r; }
                }
            }
        }
    }
    __syncthreads();
    for (int idx = tid; idx < nloc * w; idx += kLeafThreads) {
        int c = idx / nloc, r = idx - c * nloc;
        A[(c0 + c) * lda + grow0 + r] = sm[r * S + c];
    }
    cluster_sync_all();          // no CTA leaves while another may still read its publications
}

// ---------------------------------------------------------------------------
// SWAP: the sequential interchanges ipiv[k0 .. k0+kb) as a gather. One lane
// replays them on a list of touched positions (the block's own rows first,
// then every row beyond the block that a pivot names, found through an
// open-addressing table in shared memory) and the warp emits (dst, src) pairs
// with new[dst] = old[src]; the gather kernel then moves whole rows.
// Block b of the launch handles ipiv[k0_base + b*pb, ... + pb) (clipped at
// n_end) and writes cnt[b], dst/src + b*2*pb. Shared memory:
// perm_pairs_smem(pb) bytes.
// Entries outside [k, n_total) are not interchanges and are skipped.
__global__ void k_perm_pairs(const int32_t* __restrict__ ipiv, int64_t k0_base, int pb, int64_t n_end,
                             int64_t n_total, int* __restrict__ cnt, int* __restrict__ dst, int* __restrict__ src) {
    extern __shared__ int psm[];
    __shared__ int s_len;
    const int64_t k0 = k0_base + (int64_t)blockIdx.x * pb;
    const int kb = (int)min((int64_t)pb, n_end - k0);
    cnt += blockIdx.x;
    dst += (int64_t)blockIdx.x * 2 * pb;
    src += (int64_t)blockIdx.x * 2 * pb;
    const int H = perm_pairs_table(pb);
    int* pos = psm;               // [2*pb] touched positions
    int* con = psm + 2 * pb;      // [2*pb] their contents (original row numbers)
    int* pv = psm + 4 * pb;       // [pb] the block's pivots, read once (coalesced)
    int* hkey = psm + 5 * pb;     // [H] rows beyond the block seen so far (-1: free)
    int* hslot = hkey + H;        // [H] their index in pos / con
    const int lane = threadIdx.x;
    for (int i = lane; i < kb; i += 32) {
        pos[i] = (int)(k0 + i);
        con[i] = (int)(k0 + i);
        pv[i] = ipiv[k0 + i];
    }
    for (int h = lane; h < H; h += 32) hkey[h] = -1;
    __syncwarp();
    if (lane == 0) {
        int L = kb;
        for (int i = 0; i < kb; i++) {
            const int p = pv[i];
            if (p <= k0 + i || p >= n_total) continue;
            int q;
            if (p < k0 + kb) {
                q = (int)(p - k0);
            } else {
                // at most pb rows beyond the block, H >= 2 pb: a free entry always exists
                for (int h = p & (H - 1);; h = (h + 1) & (H - 1)) {
                    const int key = hkey[h];
                    if (key == p) {
                        q = hslot[h];
                        break;
                    }
                    if (key < 0) {
                        q = L++;
                        hkey[h] = p;
                        hslot[h] = q;
                        pos[q] = p;
                        con[q] = p;
                        break;
                    }
                }
            }
            const int t = con[i];
            con[i] = con[q];
            con[q] = t;
        }
        s_len = L;
    }
    __syncwarp();
    const int L = s_len;
    // compact the pairs that move something
    int base_out = 0;
    for (int b = 0; b < L; b += 32) {
        int e = b + lane;
        bool mv = e < L && pos[e] != con[e];
        unsigned bal = __ballot_sync(0xffffffffu, mv);
        if (mv) {
            int o = base_out + __popc(bal & ((1u << lane) - 1));
            dst[o] = pos[e];
            src[o] = con[e];
        }
        base_out += __popc(bal);
    }
    if (lane == 0) *cnt = base_out;
}

// Gather rows for the columns [0, cA) and [cB, n): every CTA takes 8 columns;
// all reads of a column finish (barrier) before any write.
constexpr int kSwapCols = 8;
constexpr int kSwapPairsPerThread = 4;   // 256 threads x 4 >= 2*NB for NB <= 512

__global__ void __launch_bounds__(256) k_laswp_gather(double* __restrict__ A, int64_t lda, int64_t cA, int64_t cB,
                                                      int64_t n, const int* __restrict__ cnt,
                                                      const int* __restrict__ dst, const int* __restrict__ src) {
    const int np = *cnt;
    if (np == 0) return;
    const int64_t ncols = cA + (n - cB);
    const int64_t cbase = (int64_t)blockIdx.x * kSwapCols;
    double v[kSwapPairsPerThread][kSwapCols];
#pragma unroll
    for (int q = 0; q < kSwapPairsPerThread; q++) {
        int t = threadIdx.x + q * 256;
#pragma unroll
        for (int c = 0; c < kSwapCols; c++) {
            int64_t ci = cbase + c;
            if (t < np && ci < ncols) {
                int64_t col = ci < cA ? ci : ci - cA + cB;
                v[q][c] = A[col * lda + src[t]];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSwapPairsPerThread; q++) {
        int t = threadIdx.x + q * 256;
#pragma unroll
        for (int c = 0; c < kSwapCols; c++) {
            int64_t ci = cbase + c;
            if (t < np && ci < ncols) {
                int64_t col = ci < cA ? ci : ci - cA + cB;
                A[col * lda + dst[t]] = v[q][c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// DTRSM: B <- L^-1 B with L the kk x kk unit lower triangle at A(r0, r0) and
// B = A(r0 : r0+kk, cb : ce). Each CTA stages 16 columns of B in SMEM and
// runs forward substitution; 16 thread groups split the rows.
constexpr int kTrsmCols = 16;

// kk <= 64: L11 staged in shared memory once (the loop above re-reads a
// column of L from L2 at every step, which at this size is latency, not
// work), COLS columns of B per CTA, loads and stores coalesced along rows.
template <int COLS>
__global__ void __launch_bounds__(256) k_trsm_lunit_small(double* __restrict__ A, int64_t lda, int64_t r0, int kk,
                                                          int64_t cb, int64_t ce) {
    constexpr int G = 256 / COLS;
    __shared__ double Ls[64][65];
    __shared__ double xs[64][COLS];
    const int c = threadIdx.x % COLS, g = threadIdx.x / COLS;
    const int64_t cbase = cb + (int64_t)blockIdx.x * COLS;
    const int ncol = (int)min((int64_t)COLS, ce - cbase);
    for (int idx = threadIdx.x; idx < kk * kk; idx += 256) {
        const int j = idx / kk, i = idx - j * kk;
        if (i > j) Ls[i][j] = A[(r0 + j) * lda + r0 + i];
    }
    for (int idx = threadIdx.x; idx < kk * COLS; idx += 256) {
        const int cc = idx / kk, i = idx - cc * kk;
        xs[i][cc] = cc < ncol ? A[(cbase + cc) * lda + r0 + i] : 0.0;
    }
    for (int j = 0; j < kk - 1; j++) {
        __syncthreads();
        const double xj = xs[j][c];
        for (int i = j + 1 + g; i < kk; i += G) xs[i][c] = fma(-Ls[i][j], xj, xs[i][c]);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kk * ncol; idx += 256) {
        const int cc = idx / kk, i = idx - cc * kk;
        A[(cbase + cc) * lda + r0 + i] = xs[i][cc];
    }
}

__global__ void __launch_bounds__(256) k_trsm_lunit(double* __restrict__ A, int64_t lda, int64_t r0, int kk,
                                                    int64_t cb, int64_t ce) {
    extern __shared__ double xs[];            // [kk][16]
    const int c = threadIdx.x & 15, g = threadIdx.x >> 4;
    const int64_t col = cb + (int64_t)blockIdx.x * kTrsmCols + c;
    const bool live = col < ce;
    for (int i = g; i < kk; i += 16) xs[i * kTrsmCols + c] = live ? A[col * lda + r0 + i] : 0.0;
    for (int j = 0; j < kk - 1; j++) {
        __syncthreads();
        const double xj = xs[j * kTrsmCols + c];
        const double* Lj = A + (r0 + j) * lda + r0;     // column j of L
        for (int i = j + 1 + g; i < kk; i += 16) xs[i * kTrsmCols + c] = fma(-Lj[i], xj, xs[i * kTrsmCols + c]);
    }
    __syncthreads();
    if (live)
        for (int i = g; i < kk; i += 16) A[col * lda + r0 + i] = xs[i * kTrsmCols + c];
}

// ---------------------------------------------------------------------------
// DGEMM: C -= A * B in FP64 with DFMA. TB x TB CTA tile (64, or 32 when
// 64-wide tiles would leave SMs idle: one 64 x 64 x 64 tile is ~60 us of a
// single SM's FP64 pipe, so small trailing matrices want more, smaller
// tiles), k-step 16, 256 threads with a (TB/16)^2 register tile, cp.async
// double buffering. C is loaded into the accumulators first so every entry
// sees c - sum(a*b) accumulated in increasing k, as in the unblocked
// elimination; the result does not depend on TB.
constexpr int kGB = 64, kGK = 16;

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    int sz = pred ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int TB>
__global__ void __launch_bounds__(256) k_dgemm_sub(int64_t m, int64_t nn, int64_t kk, const double* __restrict__ A,
                                                   int64_t lda, const double* __restrict__ B, int64_t ldb,
                                                   double* __restrict__ C, int64_t ldc) {
    constexpr int R = TB / 16;                     // register tile R x R
    constexpr int LQ = TB * kGK / 256;             // elements of a k-slab each thread loads per operand
    __shared__ __align__(16) double As[2][kGK][TB + 1];
    __shared__ __align__(16) double Bs[2][kGK][TB + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * TB, col0 = (int64_t)blockIdx.y * TB;

    auto load_tile = [&](int buf, int64_t k0) {
#pragma unroll
        for (int q = 0; q < LQ; q++) {
            int e = tid + 256 * q;
            int kq = e / TB, r = e % TB;
            bool ok = (row0 + r < m) && (k0 + kq < kk);
            const double* g = ok ? A + (k0 + kq) * lda + row0 + r : A;
            cp_async8(&As[buf][kq][r], g, ok);
        }
#pragma unroll
        for (int q = 0; q < LQ; q++) {
            int e = tid + 256 * q;
            int c = e >> 4, kq = e & 15;
            bool ok = (col0 + c < nn) && (k0 + kq < kk);
            const double* g = ok ? B + (col0 + c) * ldb + k0 + kq : B;
            cp_async8(&Bs[buf][kq][c], g, ok);
        }
        cp_async_commit();
    };

    double acc[R][R];
#pragma unroll
    for (int j = 0; j < R; j++)
#pragma unroll
        for (int i = 0; i < R; i++) {
            int64_t r = row0 + tx + 16 * i, c = col0 + ty + 16 * j;
            acc[i][j] = (r < m && c < nn) ? C[c * ldc + r] : 0.0;
        }

    const int ntiles = (int)((kk + kGK - 1) / kGK);
    load_tile(0, 0);
    for (int t = 0; t < ntiles; t++) {
        const int buf = t & 1;
        if (t + 1 < ntiles) {
            load_tile(buf ^ 1, (int64_t)(t + 1) * kGK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kq = 0; kq < kGK; kq++) {
            double a[R], b[R];
#pragma unroll
            for (int i = 0; i < R; i++) a[i] = As[buf][kq][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < R; j++) b[j] = Bs[buf][kq][ty + 16 * j];
#pragma unroll
            for (int j = 0; j < R; j++)
#pragma unroll
                for (int i = 0; i < R; i++) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < R; j++)
#pragma unroll
        for (int i = 0; i < R; i++) {
            int64_t r = row0 + tx + 16 * i, c = col0 + ty + 16 * j;
            if (r < m && c < nn) C[c * ldc + r] = acc[i][j];
        }
}

__global__ void k_lu_finish(hpl_info* info, const PanelSync* sync, const int* emu_err) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (sync->abort || *emu_err) info->status = HPL_ERR_TIMEOUT;
        else if (info->info != 0) info->status = HPL_ERR_SINGULAR;
        else info->status = HPL_OK;
    }
}

// ---------------------------------------------------------------------------
// Trailing update with FP64 accuracy on the BF16 tensor cores (sliced products
// after Ozaki, Ogita, Oishi & Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", 2012; not
// in the paper). Row i of L21 is 2^eA_i sum_s a_s 2^-6s and column j of U12 is
// 2^eB_j sum_t b_t 2^-6t, with integer slices |a_s|, |b_t| < 64 (exact in
// BF16) truncated from the 66 bits below the top bit of the row / column (so
// that entries well below their row's or column's largest still keep about
// 53 bits). A group g = s + t of slice products summed over at most
// (g-1) kb <= 11 * 256 terms stays below 2^24, so one BF16 tensor-core product
// with FP32 accumulation per group is exact; the groups are combined in 64-bit
// integers and rounded to FP64:
//   C(i,j) -= 2^(eA_i + eB_j) sum_{g=2..12} 2^-6g C_g(i,j).
// Products with s + t > 12 are left out (below 2^(eA_i+eB_j-72) kb in size).

__device__ __forceinline__ int emu_exp(unsigned long long absbits) {   // |x| < 2^e for the largest |x|
    return absbits ? (int)(absbits >> 52) - 1022 : 0;
}

// 66-bit fixed-point magnitude of x relative to 2^e (|x| < 2^e), truncated,
// as hi (the top 36 bits, slices 1..6) and lo (the next 30 bits, slices 7..11)
__device__ __forceinline__ void emu_fixed(double x, int e, unsigned long long& hi, unsigned long long& lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    const int E = (int)(u >> 52);
    hi = lo = 0ull;
    if (E == 0) return;                            // zero and subnormals: below 2^-1022
    const unsigned long long mant = (u & 0xfffffffffffffull) | (1ull << 52);
    // x / 2^e = mant * 2^(E - 1075 - e); the 66-bit fixed point F = mant * 2^(E - 1009 - e)
    const int sh = E - 1009 - e;                   // <= 13 since |x| < 2^e
    // F = (hi << 30) | lo with hi < 2^36, lo < 2^30
    if (sh >= 0) {                                 // F = mant << sh (< 2^66)
        hi = mant >> (30 - sh);
        lo = (mant << sh) & ((1ull << 30) - 1);
    } else if (sh > -53) {
        const unsigned long long f = mant >> (-sh);    // < 2^53: fits 64 bits
        hi = f >> 30;
        lo = f & ((1ull << 30) - 1);
    }
}

// One warp per row i of L21 (m x kb, column-major): exponent and the
// kEmuSlices slices into sA[i][s * kbp + q] (zeros for q >= kb).
__global__ void __launch_bounds__(256) k_emu_slice_rows(int64_t m, int kb, int kbp, const double* __restrict__ L,
                                                        int64_t ldl, __nv_bfloat16* __restrict__ sA, int64_t lds,
                                                        int* __restrict__ eA) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= m) return;
    unsigned long long mx = 0;
    for (int q = lane; q < kb; q += 32) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(L[(int64_t)q * ldl + i]) & 0x7fffffffffffffffull;
        mx = u > mx ? u : mx;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    const int e = emu_exp(mx);
    if (lane == 0) eA[i] = e;
    __nv_bfloat16* row = sA + i * lds;
    for (int q = lane; q < kbp; q += 32) {
        const double x = q < kb ? L[(int64_t)q * ldl + i] : 0.0;
        unsigned long long fh, fl;
        emu_fixed(x, e, fh, fl);
        const bool neg = x < 0.0;
#pragma unroll
        for (int sl = 1; sl <= kEmuSlices; sl++) {
            const int a = sl <= 6 ? (int)((fh >> (36 - kEmuBits * sl)) & 63ull)
                                  : (int)((fl >> (30 - kEmuBits * (sl - 6))) & 63ull);
            row[(sl - 1) * kbp + q] = __int2bfloat16_rn(neg ? -a : a);
        }
    }
}

// One warp per column j of U12 (kb x nn, column-major): exponent and slices
// into sB[j][(kEmuSlices - t) * kbp + q] (slot order reversed, so that the
// B operand of group g is the last g-1 slots).
__global__ void __launch_bounds__(256) k_emu_slice_cols(int64_t nn, int kb, int kbp, const double* __restrict__ U,
                                                        int64_t ldu, __nv_bfloat16* __restrict__ sB, int64_t lds,
                                                        int* __restrict__ eB) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= nn) return;
    const double* col = U + j * ldu;
    unsigned long long mx = 0;
    for (int q = lane; q < kb; q += 32) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(col[q]) & 0x7fffffffffffffffull;
        mx = u > mx ? u : mx;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    const int e = emu_exp(mx);
    if (lane == 0) eB[j] = e;
    __nv_bfloat16* out = sB + j * lds;
    for (int q = lane; q < kbp; q += 32) {
        const double x = q < kb ? col[q] : 0.0;
        unsigned long long fh, fl;
        emu_fixed(x, e, fh, fl);
        const bool neg = x < 0.0;
#pragma unroll
        for (int t = 1; t <= kEmuSlices; t++) {
            const int b = t <= 6 ? (int)((fh >> (36 - kEmuBits * t)) & 63ull)
                                 : (int)((fl >> (30 - kEmuBits * (t - 6))) & 63ull);
            out[(kEmuSlices - t) * kbp + q] = __int2bfloat16_rn(neg ? -b : b);
        }
    }
}

// C(i, j) -= 2^(eA_i + eB_j) sum_g 2^-6g C_g(i, j) for an m x nc block; the
// group products are exact integers below 2^24 in FP32 (cg[g-2], ld m).
__global__ void __launch_bounds__(256) k_emu_combine(int64_t m, int64_t nc, const float* __restrict__ cg,
                                                     const int* __restrict__ eA, const int* __restrict__ eB,
                                                     double* __restrict__ C, int64_t ldc) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x, j = blockIdx.y;
    if (i >= m || j >= nc) return;
    const int64_t stride = m * nc, at = j * m + i;
    long long hi = 0, lo = 0;          // in units of 2^-36 (g = 2..6) and 2^-72 (g = 7..12)
#pragma unroll
    for (int g = 2; g <= 6; g++) hi += (long long)__float2int_rn(cg[(g - 2) * stride + at]) * (1ll << (kEmuBits * (6 - g)));
#pragma unroll
    for (int g = 7; g <= kEmuSlices + 1; g++)
        lo += (long long)__float2int_rn(cg[(g - 2) * stride + at]) * (1ll << (kEmuBits * (kEmuSlices + 1 - g)));
    const double v = fma((double)lo, 0x1p-36, (double)hi);               // sum in units of 2^-36
    const int e = eA[i] + eB[j] - 36;
    const double scale = (e > -1022 && e < 1024) ? __longlong_as_double((long long)(e + 1023) << 52)   // 2^e
                                                 : ldexp(1.0, e);
    double* c = C + j * ldc + i;
    *c = fma(-v, scale, *c);
}

int launch_gemm_bf16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                     float* C, int64_t ldc, int sub, int* err, int64_t timeout_ns, int max_ctas, cudaStream_t s);

// Slices of one step: L21 (m x kb, ld ldl) and the kb x nn block row U12 (ld ldu).
static int emu_slice(const LuWs& w, int64_t m, int64_t nn, int kb, const double* L, int64_t ldl, const double* U,
                     int64_t ldu, cudaStream_t s) {
    const int kbp = (int)emu_kbp(kb);
    const int64_t lds = (int64_t)kEmuSlices * kbp;
    if (m > 0) {
        k_emu_slice_rows<<<(unsigned)((m + 7) / 8), 256, 0, s>>>(m, kb, kbp, L, ldl, (__nv_bfloat16*)w.sA, lds, w.eA);
        HPL_LAUNCH_CHECK();
    }
    if (nn > 0) {
        k_emu_slice_cols<<<(unsigned)((nn + 7) / 8), 256, 0, s>>>(nn, kb, kbp, U, ldu, (__nv_bfloat16*)w.sB, lds, w.eB);
        HPL_LAUNCH_CHECK();
    }
    return HPL_OK;
}

// C (m x nn, ld ldc) -= L21 U12 for the block-row columns col0 .. col0+nn of
// the sliced step, with FP64 accuracy on the tensor cores.
static int emu_update(const LuWs& w, int64_t m, int64_t nn, int kb, int64_t col0, double* C, int64_t ldc, int* err,
                      int64_t timeout_ns, cudaStream_t s) {
    if (m <= 0 || nn <= 0 || kb <= 0) return HPL_OK;
    const int kbp = (int)emu_kbp(kb);
    const int64_t lds = (int64_t)kEmuSlices * kbp;
    for (int64_t j0 = 0; j0 < nn; j0 += kEmuChunk) {
        const int64_t nc = std::min<int64_t>(kEmuChunk, nn - j0);
        for (int g = 2; g <= kEmuSlices + 1; g++) {
            const int64_t K = (int64_t)(g - 1) * kbp;
            const uint16_t* Bg = w.sB + (col0 + j0) * lds + (int64_t)(kEmuSlices - (g - 1)) * kbp;
            int st = launch_gemm_bf16(m, nc, K, w.sA, lds, Bg, lds, w.cg + (int64_t)(g - 2) * m * nc, m, 0, err,
                                      timeout_ns, 0, s);
            if (st) return st;
        }
        k_emu_combine<<<dim3((unsigned)((m + 255) / 256), (unsigned)nc), 256, 0, s>>>(m, nc, w.cg, w.eA,
                                                                                      w.eB + col0 + j0,
                                                                                      C + j0 * ldc, ldc);
        HPL_LAUNCH_CHECK();
    }
    return HPL_OK;
}

// ---------------------------------------------------------------------------
// Host-side launch helpers.

int launch_dgemm_sub(int64_t m, int64_t nn, int64_t kk, const double* A, int64_t lda, const double* B, int64_t ldb,
                     double* C, int64_t ldc, cudaStream_t s) {
    if (m <= 0 || nn <= 0 || kk <= 0) return HPL_OK;
    dim3 grid((unsigned)((m + kGB - 1) / kGB), (unsigned)((nn + kGB - 1) / kGB));
    if ((int64_t)grid.x * grid.y < 4 * kNumSMsGB300) {
        // fewer than four waves of 64-wide tiles: quarter-size tiles fill the SMs
        dim3 g32((unsigned)((m + 31) / 32), (unsigned)((nn + 31) / 32));
        if (g32.y > 65535) return HPL_ERR_INVALID;
        k_dgemm_sub<32><<<g32, 256, 0, s>>>(m, nn, kk, A, lda, B, ldb, C, ldc);
        HPL_LAUNCH_CHECK();
        return HPL_OK;
    }
    if (grid.y > 65535) return HPL_ERR_INVALID;
    k_dgemm_sub<64><<<grid, 256, 0, s>>>(m, nn, kk, A, lda, B, ldb, C, ldc);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

// TRSM of the FP64 LU: one kernel (0) or blocked by 64 with DFMA updates (1,
// the default: measured on GB300 at n = 32768, NB = 256, TRSM phase 161.5 ->
// 131.7 ms, factorization 18.90 -> 18.86 s); a measurement switch
// (hplgb_lu_config), the same bits either way.
static int g_trsm_blocked = 1;

static int launch_trsm(double* A, int64_t lda, int64_t r0, int kk, int64_t cb, int64_t ce, cudaStream_t s) {
    if (ce <= cb || kk <= 1) return HPL_OK;
    if (kk <= 64) {
        if ((ce - cb) / 16 >= kNumSMsGB300) {
            k_trsm_lunit_small<16><<<(unsigned)((ce - cb + 15) / 16), 256, 0, s>>>(A, lda, r0, kk, cb, ce);
        } else {
            k_trsm_lunit_small<8><<<(unsigned)((ce - cb + 7) / 8), 256, 0, s>>>(A, lda, r0, kk, cb, ce);
        }
        HPL_LAUNCH_CHECK();
        return HPL_OK;
    }
    if (g_trsm_blocked) {
        // Blocked by 64: each diagonal block solved by the shared-memory TRSM,
        // the rows below it updated by the DFMA product. Every x_i still
        // receives fma(-L_ij, x_j, x_i) for j = 0, 1, ... in order (both
        // kernels accumulate in place, in k order), so the result is
        // bit-identical to the one-kernel TRSM; three quarters of the flops
        // (kk = 256) run on the update kernel's tiles.
        for (int b0 = 0; b0 < kk; b0 += 64) {
            const int bk = std::min(64, kk - b0);
            int st = launch_trsm(A, lda, r0 + b0, bk, cb, ce, s);
            if (st) return st;
            if (b0 + bk < kk) {
                st = launch_dgemm_sub(kk - b0 - bk, ce - cb, bk, A + (r0 + b0) * lda + r0 + b0 + bk, lda,
                                      A + cb * lda + r0 + b0, lda, A + cb * lda + r0 + b0 + bk, lda, s);
                if (st) return st;
            }
        }
        return HPL_OK;
    }
    size_t smem = sizeof(double) * kk * kTrsmCols;
    unsigned grid = (unsigned)((ce - cb + kTrsmCols - 1) / kTrsmCols);
    k_trsm_lunit<<<grid, 256, smem, s>>>(A, lda, r0, kk, cb, ce);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

struct PanelPlan {
    int max_coop;   // co-resident leaf CTAs
    int max_cluster;  // largest cluster the cluster leaf may use (0: none)
};

constexpr int kClusterLeafRows = 64;             // rows per CTA the cluster leaf aims for
constexpr size_t kClusterLeafSmem = 200 * 1024;  // dynamic shared memory bound per CTA

// The cluster leaf for columns [c0, c0+w) when the panel's rows fit; returns
// 1 (nothing launched) when they do not.
static int launch_leaf_cluster(int64_t n, double* A, int64_t lda, int64_t c0, int w, int64_t pc0, int64_t pw,
                               int32_t* ipiv, hpl_info* info, const PanelPlan& pp, cudaStream_t s) {
    if (pp.max_cluster < 1 || w > 64) return 1;
    const int64_t m = n - c0;
    const int W = w <= 32 ? 32 : 64;
    const size_t row_bytes = sizeof(double) * (W + 1);
    const int64_t cap_rows = (int64_t)(kClusterLeafSmem / row_bytes);
    int C = (int)std::min<int64_t>((m + kClusterLeafRows - 1) / kClusterLeafRows, pp.max_cluster);
    if (C < 1) C = 1;
    int64_t rows_per = (m + C - 1) / C;
    if (rows_per > cap_rows) {
        C = pp.max_cluster;
        rows_per = (m + C - 1) / C;
        if (rows_per > cap_rows) return 1;
    }
    const size_t smem = row_bytes * (size_t)std::max<int64_t>(rows_per, 1);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kLeafThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int rp = (int)rows_per;
    if (W == 32)
        HPL_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel_leaf_cl<32>, n, A, lda, c0, w, rp, pc0, pw, ipiv, info));
    else
        HPL_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel_leaf_cl<64>, n, A, lda, c0, w, rp, pc0, pw, ipiv, info));
    count_launch();
    return HPL_OK;
}

static int launch_leaf(int64_t n, double* A, int64_t lda, int64_t c0, int w, int64_t pc0, int64_t pw,
                       int32_t* ipiv, const LuWs& ws, hpl_info* info, int64_t timeout_ns, const PanelPlan& pp,
                       cudaStream_t s) {
    int64_t m = n - c0;
    int P = (int)std::min<int64_t>((m + 255) / 256, (int64_t)pp.max_coop);
    if (P < 1) P = 1;
    int rows_per = (int)((m + P - 1) / P);
    P = (int)((m + rows_per - 1) / rows_per);
    size_t smem = sizeof(double) * (size_t)rows_per * kLeafStride;
    if (smem > 200 * 1024) return HPL_ERR_INVALID;     // matrix too tall for the FP64 panel
    void* args[] = {&n, &A, &lda, &c0, &w, &rows_per, &pc0, &pw, &ipiv, (void*)&ws.slots, (void*)&ws.drow,
                    (void*)&ws.sync, &info, &timeout_ns};
    HPL_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_panel_leaf, dim3(P), dim3(kLeafThreads), args, smem, s));
    count_launch();
    return HPL_OK;
}

// Recursive PFACT of the panel columns [c0, c0+w) (rows [c0, n)) inside the
// NB panel [pc0, pc0+pw): left half, TRSM + GEMM on the right half, right half.
static int panel_rec(int64_t n, double* A, int64_t lda, int64_t c0, int w, int64_t pc0, int64_t pw, int32_t* ipiv,
                     const LuWs& ws, hpl_info* info, int64_t timeout_ns, const PanelPlan& pp, cudaStream_t s) {
    if (w <= 64 && n - c0 <= HPLGB_CLUSTER_LEAF_MAX_ROWS) {
        int st = launch_leaf_cluster(n, A, lda, c0, w, pc0, pw, ipiv, info, pp, s);
        if (st != 1) return st;
    }
    if (w <= kLeafW) return launch_leaf(n, A, lda, c0, w, pc0, pw, ipiv, ws, info, timeout_ns, pp, s);
    int w1 = ((w / 2 + kLeafW - 1) / kLeafW) * kLeafW;
    if (w1 >= w) w1 = kLeafW;
    int st = panel_rec(n, A, lda, c0, w1, pc0, pw, ipiv, ws, info, timeout_ns, pp, s);
    if (st) return st;
    st = launch_trsm(A, lda, c0, w1, c0 + w1, c0 + w, s);
    if (st) return st;
    st = launch_dgemm_sub(n - c0 - w1, w - w1, w1, A + c0 * lda + c0 + w1, lda, A + (c0 + w1) * lda + c0, lda,
                          A + (c0 + w1) * lda + c0 + w1, lda, s);
    if (st) return st;
    return panel_rec(n, A, lda, c0 + w1, w - w1, pc0, pw, ipiv, ws, info, timeout_ns, pp, s);
}

// Largest cluster (16, else the portable 8) on which the cluster leaf can run
// with its largest shared-memory footprint; 0 when none can.
static int max_leaf_cluster() {
    static std::atomic<int> cache[kMaxDevices];      // cluster size + 1; 0: not yet known
    const int dv = device_slot();
    if (dv < 0) return 0;
    if (const int c = cache[dv].load()) return c - 1;
    int best = 0;
    const void* fns[2] = {(const void*)k_panel_leaf_cl<32>, (const void*)k_panel_leaf_cl<64>};
    for (const void* f : fns) {
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterLeafSmem);
        cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    for (int c : {16, 8}) {
        bool ok = true;
        for (const void* f : fns) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)c;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3((unsigned)c);
            cfg.blockDim = dim3(kLeafThreads);
            cfg.dynamicSmemBytes = kClusterLeafSmem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, f, &cfg) != cudaSuccess || nclusters < 1) ok = false;
        }
        cudaGetLastError();
        if (ok) { best = c; break; }
    }
    cache[dv].store(best + 1);
    return best;
}

static int max_coop_leaf_ctas(int num_sms, int64_t n) {
    // the leaf's dynamic SMEM depends on rows_per; size the bound for the
    // tallest panel (rows_per <= ceil(n / P)) with one CTA per SM.
    int per_sm = 0;
    size_t smem_guess = sizeof(double) * 256 * kLeafStride;
    cudaFuncSetAttribute((const void*)k_panel_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_panel_leaf, kLeafThreads, smem_guess);
    int64_t need = (n + 255) / 256;
    int64_t cap = (int64_t)num_sms * std::max(per_sm, 1);
    if (need > cap) {
        // fewer CTAs, more rows each; one CTA per SM is always co-resident
        cap = num_sms;
    }
    return (int)std::min<int64_t>(std::min<int64_t>(need, cap), kMaxPanelCtas);
}

}  // namespace hplgb

using namespace hplgb;

extern "C" size_t lu_factor_workspace_size(int64_t n, const hpl_opts* opts) {
    Opts o = resolve_opts(opts, 256);
    return lu_ws_layout(o.nb, nullptr, nullptr, o.fp64_emulation ? std::max<int64_t>(n, 0) : 0);
}

extern "C" int lu_factor(int64_t n, double* A, int64_t lda, int32_t* ipiv, const hpl_opts* opts, void* ws,
                         size_t ws_bytes, hpl_info* info, void* stream) {
    if (n < 0 || lda < (n > 1 ? n : 1) || !info) return HPL_ERR_INVALID;
    if (n > 0 && (!A || !ipiv)) return HPL_ERR_INVALID;
    if (n > 0x7fffffff) return HPL_ERR_INVALID;
    Opts o = resolve_opts(opts, 256);
    if (o.nb < 1 || o.nb > 512) return HPL_ERR_INVALID;
    const bool emu = o.fp64_emulation != 0;
    if (o.fp64_emulation < 0 || o.fp64_emulation > 1 || (emu && o.nb > 256)) return HPL_ERR_INVALID;
    if (o.pfact < 0 || o.pfact > 1) return HPL_ERR_INVALID;
    const int64_t n_emu = emu ? n : 0;
    size_t need = lu_ws_layout(o.nb, nullptr, nullptr, n_emu);
    if (!ws || ws_bytes < need) return HPL_ERR_NOMEM;
    if ((uintptr_t)ws & 255) return HPL_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    HPL_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(hpl_info), s));
    if (n == 0) return HPL_OK;
    LuWs w;
    lu_ws_layout(o.nb, &w, (char*)ws, n_emu);
    HPL_CUDA_TRY(cudaMemsetAsync(ws, 0, w.base_bytes, s));

    DeviceCtx* ctx = nullptr;
    int st = get_ctx(&ctx);
    if (st) return st;
    PanelPlan pp;
    pp.max_coop = max_coop_leaf_ctas(ctx->num_sms, n);
    pp.max_cluster = o.pfact == 0 ? max_leaf_cluster() : 0;
    HPL_CUDA_TRY(cudaFuncSetAttribute((const void*)k_trsm_lunit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * 512 * kTrsmCols)));

    const int64_t nb = o.nb;
    const int64_t nsteps = (n + nb - 1) / nb;
    const bool la = o.lookahead != 0;
    cudaStream_t ps = la ? ctx->side : s;                // panel stream
    cudaEvent_t ev_fork = ctx->ev[0], ev_panel = ctx->ev[1], ev_la = ctx->ev[2], ev_join = ctx->ev[3];
    if (la) {
        HPL_CUDA_TRY(cudaEventRecord(ev_fork, s));
        HPL_CUDA_TRY(cudaStreamWaitEvent(ps, ev_fork, 0));
    }
    auto panel = [&](int64_t k) -> int {
        int64_t c0 = k * nb;
        int kb = (int)std::min(nb, n - c0);
        const double pm = (double)(n - c0);
        int slot = phase_begin(ps);
        int r = panel_rec(n, A, lda, c0, kb, c0, kb, ipiv, w, info, o.timeout_ns, pp, ps);
        if (r) return r;
        int par = (int)(k & 1);
        k_perm_pairs<<<1, 32, perm_pairs_smem(kb), ps>>>(ipiv, c0, kb, c0 + kb, n, w.perm_cnt + par,
                                                           w.perm_dst + par * 2 * nb, w.perm_src + par * 2 * nb);
        HPL_LAUNCH_CHECK();
        // getrf of an m x kb panel: m kb^2 - kb^3/3 flops (leading terms)
        phase_end(slot, ps, PH_PANEL, pm * kb * kb - (double)kb * kb * kb / 3.0, (int)k);
        return HPL_OK;
    };

    st = panel(0);
    if (st) return st;
    for (int64_t k = 0; k < nsteps; k++) {
        const int64_t c0 = k * nb;
        const int kb = (int)std::min(nb, n - c0);
        const int64_t c1 = c0 + kb;                      // first trailing column
        const int par = (int)(k & 1);
        if (la) {
            HPL_CUDA_TRY(cudaEventRecord(ev_panel, ps));
            HPL_CUDA_TRY(cudaStreamWaitEvent(s, ev_panel, 0));
        }
        // SWAP on every column outside the panel
        int64_t ncols_out = c0 + (n - c1);
        if (ncols_out > 0) {
            unsigned g = (unsigned)((ncols_out + kSwapCols - 1) / kSwapCols);
            int slot = phase_begin(s);
            k_laswp_gather<<<g, 256, 0, s>>>(A, lda, c0, c1, n, w.perm_cnt + par, w.perm_dst + par * 2 * nb,
                                             w.perm_src + par * 2 * nb);
            HPL_LAUNCH_CHECK();
            // at most 2 kb rows move: read + write of each moved element
            phase_end(slot, s, PH_SWAP, 2.0 * 2.0 * kb * (double)ncols_out * sizeof(double), (int)k);
        }
        if (c1 < n) {
            // DTRSM on the block row, then DGEMM: look-ahead columns first
            const int64_t m2 = n - c1;
            int slot = phase_begin(s);
            st = launch_trsm(A, lda, c0, kb, c1, n, s);
            if (st) return st;
            phase_end(slot, s, PH_TRSM, (double)kb * (kb - 1) * (double)m2, (int)k);
            const int64_t la_cols = la ? std::min(nb, n - c1) : n - c1;   // no look-ahead: one update
            slot = phase_begin(s);
            if (emu) {
                st = emu_slice(w, m2, n - c1, kb, A + c0 * lda + c1, lda, A + c1 * lda + c0, lda, s);
                if (st) return st;
                st = emu_update(w, m2, la_cols, kb, 0, A + c1 * lda + c1, lda, w.emu_err, o.timeout_ns, s);
            } else {
                st = launch_dgemm_sub(m2, la_cols, kb, A + c0 * lda + c1, lda, A + c1 * lda + c0, lda,
                                      A + c1 * lda + c1, lda, s);
            }
            if (st) return st;
            phase_end(slot, s, PH_UPDATE, 2.0 * m2 * la_cols * kb, (int)k);
            if (la) {
                HPL_CUDA_TRY(cudaEventRecord(ev_la, s));
                HPL_CUDA_TRY(cudaStreamWaitEvent(ps, ev_la, 0));
                st = panel(k + 1);
                if (st) return st;
            }
            if (n - c1 - la_cols > 0) {
                slot = phase_begin(s);
                if (emu)
                    st = emu_update(w, m2, n - c1 - la_cols, kb, la_cols, A + (c1 + la_cols) * lda + c1, lda,
                                    w.emu_err, o.timeout_ns, s);
                else
                    st = launch_dgemm_sub(m2, n - c1 - la_cols, kb, A + c0 * lda + c1, lda,
                                          A + (c1 + la_cols) * lda + c0, lda, A + (c1 + la_cols) * lda + c1, lda, s);
                if (st) return st;
                phase_end(slot, s, PH_UPDATE, 2.0 * m2 * (n - c1 - la_cols) * kb, (int)k);
            }
            if (!la) {
                st = panel(k + 1);
                if (st) return st;
            }
        }
    }
    if (la) {
        HPL_CUDA_TRY(cudaEventRecord(ev_join, ps));
        HPL_CUDA_TRY(cudaStreamWaitEvent(s, ev_join, 0));
    }
    k_lu_finish<<<1, 32, 0, s>>>(info, w.sync, w.emu_err);
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

namespace hplgb {
extern int g_solve_wave;         // solve64.cu
extern int g_solve_wave_grid;
}  // namespace hplgb

extern "C" int hplgb_lu_config(int what, long long value) {
    switch (what) {
        case 0:
            if (value < 0 || value > 1) return HPL_ERR_INVALID;
            hplgb::g_trsm_blocked = (int)value;
            return HPL_OK;
        case 1:
            if (value < 0 || value > 1) return HPL_ERR_INVALID;
            hplgb::g_solve_wave = (int)value;
            return HPL_OK;
        case 2:
            if (value < 0 || value > 4096) return HPL_ERR_INVALID;
            hplgb::g_solve_wave_grid = (int)value;
            return HPL_OK;
        default:
            return HPL_ERR_INVALID;
    }
}
