// lu_solve: the triangular solves that follow the factorization (paper
// Sec. III-A.1, "followed by triangular solves"), FP64.
//
// Interchanges: the pivot vector is cut into blocks of 256; one warp per block
// turns its sequential swaps into (dst, src) pairs (done in parallel for all
// blocks), then one CTA per right-hand side applies the blocks in order
// (reverse order, inverse pairs, for the transposed solve).
// Triangles: blocked substitution with 64-row diagonal blocks. A diagonal
// block is solved by one warp per right-hand side with shuffles; the rows
// below (forward) or above (backward) are then updated by a GEMV/GEMM kernel.
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

static size_t solve_ws_layout(int64_t n, int** cnt, int** dst, int** src, char* base) {
    int64_t nblk = (n + kPivBlock - 1) / kPivBlock;
    size_t off = 0;
    size_t o_cnt = off; off = align_up(off + sizeof(int) * nblk, 256);
    size_t o_dst = off; off = align_up(off + sizeof(int) * nblk * 2 * kPivBlock, 256);
    size_t o_src = off; off = align_up(off + sizeof(int) * nblk * 2 * kPivBlock, 256);
    if (base) {
        *cnt = (int*)(base + o_cnt);
        *dst = (int*)(base + o_dst);
        *src = (int*)(base + o_src);
    }
    return std::max<size_t>(off, 256);
}

// Both triangles for one right-hand side (no transpose, P b applied) on one
// thread-block cluster: the latency-bound case of a small matrix, where the
// per-block kernel launches of tri_solve dominate. Blocks of 64 rows are
// dealt round-robin to the C CTAs (CTA c owns blocks c, c + C, ...; its part
// of the right-hand side stays in shared memory throughout). Step by step
// (forward: block 0 up; backward: the last block down) the owner solves the
// diagonal block with one warp (upper: reciprocals of the diagonal taken once
// per block), one cluster barrier publishes the solved block, every CTA reads
// it through distributed shared memory and subtracts its product with the
// off-diagonal blocks of the rows it owns. A solved block is never written
// again, so no publication needs a second buffer.
__global__ void __launch_bounds__(256) k_trsv_cluster(int64_t n, const double* __restrict__ LU, int64_t lda,
                                                      double* __restrict__ b) {
    extern __shared__ double xs[];            // this CTA's blocks of b / x, 64 each
    __shared__ double T[kTB][kTB + 1];
    __shared__ double xb[kTB];
    __shared__ double part[4][kTB];
    __shared__ double rinv[kTB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned C = gridDim.x, me = cluster_rank();
    const int nblk = (int)((n + kTB - 1) / kTB);
    for (int q = (int)me, lq = 0; q < nblk; q += (int)C, lq++)
        for (int i = tid; i < kTB; i += 256) xs[lq * kTB + i] = (int64_t)q * kTB + i < n ? b[(int64_t)q * kTB + i] : 0.0;
    __syncthreads();
    for (int phase = 0; phase < 2; phase++) {
        const bool lower = phase == 0;
        for (int st = 0; st < nblk; st++) {
            const int blk = lower ? st : nblk - 1 - st;
            const unsigned owner = (unsigned)(blk % (int)C);
            const int bs = (int)std::min<int64_t>(kTB, n - (int64_t)blk * kTB);
            const int64_t b0 = (int64_t)blk * kTB;
            if (me == owner) {
                for (int idx = tid; idx < bs * bs; idx += 256) {
                    const int j = idx / bs, i = idx - j * bs;
                    T[i][j] = LU[(b0 + j) * lda + b0 + i];
                }
                __syncthreads();
                if (!lower && tid < bs) rinv[tid] = 1.0 / T[tid][tid];
                __syncthreads();
                if (warp == 0) {
                    double* y = xs + (blk / (int)C) * kTB;
                    double v0 = lane < bs ? y[lane] : 0.0, v1 = lane + 32 < bs ? y[lane + 32] : 0.0;
                    if (lower) {
                        for (int j = 0; j < bs; j++) {
                            const double xj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
                            if (lane > j && lane < bs) v0 = fma(-T[lane][j], xj, v0);
                            if (lane + 32 > j && lane + 32 < bs) v1 = fma(-T[lane + 32][j], xj, v1);
                        }
                    } else {
                        for (int j = bs - 1; j >= 0; j--) {
                            if (lane == (j & 31)) {
                                if (j < 32) v0 *= rinv[j];
                                else v1 *= rinv[j];
                            }
                            const double xj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
                            if (lane < j) v0 = fma(-T[lane][j], xj, v0);
                            if (lane + 32 < j) v1 = fma(-T[lane + 32][j], xj, v1);
                        }
                    }
                    if (lane < bs) y[lane] = v0;
                    if (lane + 32 < bs) y[lane + 32] = v1;
                }
            }
            cluster_sync_all();
            if (tid < bs) xb[tid] = ld_cluster_f64(cluster_addr(&xs[(blk / (int)C) * kTB + tid], owner));
            __syncthreads();
            for (int q = (int)me, lq = 0; q < nblk; q += (int)C, lq++) {
                if (lower ? q <= blk : q >= blk) continue;
                const int rs = (int)std::min<int64_t>(kTB, n - (int64_t)q * kTB);
                const int i = tid & 63, g = tid >> 6;
                double acc = 0.0;
                if (i < rs)
                    for (int j = g * 16; j < g * 16 + 16 && j < bs; j++)
                        acc = fma(LU[(b0 + j) * lda + (int64_t)q * kTB + i], xb[j], acc);
                part[g][i] = acc;
                __syncthreads();
                if (tid < rs) xs[lq * kTB + tid] -= (part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]);
                __syncthreads();
            }
        }
        cluster_sync_all();          // every read of this phase's publications is done
    }
    for (int q = (int)me, lq = 0; q < nblk; q += (int)C, lq++)
        for (int i = tid; i < kTB; i += 256)
            if ((int64_t)q * kTB + i < n) b[(int64_t)q * kTB + i] = xs[lq * kTB + i];
}

constexpr int kTrsvClusterBlocksPerCta = 8;

// Cluster size for k_trsv_cluster (16, else the portable 8; 0 = unavailable).
static int trsv_cluster_max() {
    static std::atomic<int> cache[kMaxDevices];      // cluster size + 1; 0: not yet known
    const int dv = device_slot();
    if (dv < 0) return 0;
    if (const int c = cache[dv].load()) return c - 1;
    int best = 0;
    const void* f = (const void*)k_trsv_cluster;
    cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = sizeof(double) * kTB * kTrsvClusterBlocksPerCta;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, f, &cfg) == cudaSuccess && nc >= 1) {
            best = c;
            break;
        }
    }
    cudaGetLastError();
    cache[dv].store(best + 1);
    return best;
}

// One launch for both triangles when the system fits one cluster; returns 1
// (nothing launched) otherwise.
static int solve_cluster(int64_t n, const double* LU, int64_t lda, double* b, cudaStream_t s) {
    const int cmax = trsv_cluster_max();
    const int64_t nblk = (n + kTB - 1) / kTB;
    if (cmax < 1 || nblk > (int64_t)cmax * kTrsvClusterBlocksPerCta) return 1;
    const int C = (int)std::min<int64_t>(nblk, cmax);
    const int R = (int)((nblk + C - 1) / C);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sizeof(double) * kTB * R;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HPL_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_trsv_cluster, n, LU, lda, b));
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
    return solve_ws_layout(n > 0 ? n : 1, nullptr, nullptr, nullptr, nullptr);
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
    size_t need = solve_ws_layout(n, nullptr, nullptr, nullptr, nullptr);
    if (!ws || ws_bytes < need) return HPL_ERR_NOMEM;
    if ((uintptr_t)ws & 255) return HPL_ERR_INVALID;
    int *cnt, *dst, *src;
    solve_ws_layout(n, &cnt, &dst, &src, (char*)ws);
    const int nblk = (int)((n + kPivBlock - 1) / kPivBlock);
    k_perm_pairs<<<nblk, 32, sizeof(int) * 5 * kPivBlock, s>>>(ipiv, 0, kPivBlock, n, n, cnt, dst, src);
    HPL_LAUNCH_CHECK();
    if (info) {
        k_check_udiag<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(n, LU, lda, info);
        HPL_LAUNCH_CHECK();
    }
    if (!trans) {
        k_apply_perm<<<(unsigned)nrhs, 512, 0, s>>>(n, nblk, cnt, dst, src, 0, B, ldb);
        HPL_LAUNCH_CHECK();
        if (nrhs == 1) {
            int st = solve_cluster(n, LU, lda, B, s);
            if (st != 1) return st;
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
