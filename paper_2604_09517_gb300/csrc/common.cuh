// Shared helpers of the GPU library (host and device). Not used by the oracle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

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
    PH_COUNT = 8
};
int phase_begin(cudaStream_t s);                                   // -1 when timing is off
void phase_end(int slot, cudaStream_t s, int phase, double work, int step = -1);  // work: flops or bytes

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Align a byte offset up.
__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace hplgb
