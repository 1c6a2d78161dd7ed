// lu_factor_noalloc: lu_factor for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they factor: code
// that runs under an allocator it does not own (a framework's caching
// allocator or a memory budget fixed at start-up), or a host thread that must
// not block on a driver allocation in the middle of its work. This entry
// point takes no workspace. The scratch that lu_factor needs (its grid-barrier
// words, pivot-candidate slots and row-interchange pairs; its size depends on
// the panel width only, not on n) lives in the file-scope device array below,
// which every GPU that loads the library keeps until the process exits.
//
// Host code cannot use the array's name as a device address, so on the first
// call on each device (with that device current) the address is looked up
// once with cudaGetSymbolAddress and cached; make that first call before any
// stream capture. All calls on a device share the one array and each call
// clears it on its stream before use (lu_factor zeroes its workspace), so
// calls whose GPU work overlaps (different streams, or host threads) race on
// it and must be serialised by the caller.
#include <mutex>

#include "common.cuh"

static constexpr size_t kNoAllocScratchBytes = 320 * 1024;   // enough for any NB <= 512 (FP64 update)

static __device__ __align__(256) unsigned char g_lu_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_mu;
void* g_scratch_addr[64];

int scratch_address(void** out) {
    int dev = 0;
    HPL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return HPL_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        HPL_CUDA_TRY(cudaGetSymbolAddress(&p, g_lu_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HPL_OK;
}

}  // namespace

extern "C" size_t lu_factor_noalloc_max_scratch(void) { return kNoAllocScratchBytes; }

extern "C" int lu_factor_noalloc(int64_t n, double* A, int64_t lda, int32_t* ipiv, const hpl_opts* opts,
                                 hpl_info* info, void* stream) {
    // Options lu_factor itself refuses get its HPL_ERR_INVALID here too, before
    // any size test, so HPL_ERR_NOMEM only ever means "valid options whose
    // scratch does not fit the array".
    hplgb::Opts o = hplgb::resolve_opts(opts, 256);
    if (o.nb < 1 || o.nb > 512 || o.pfact < 0 || o.pfact > 1 || o.fp64_emulation < 0 || o.fp64_emulation > 1) {
        hplgb_internal_set_message("lu_factor_noalloc: invalid options (NB must be 1..512, pfact 0 or 1)");
        return HPL_ERR_INVALID;
    }
    // The FP64-emulated update keeps sliced copies of L21 and U12 whose size
    // grows with n, which no fixed array can hold for every n: refused.
    if (o.fp64_emulation) {
        hplgb_internal_set_message("lu_factor_noalloc: opts.fp64_emulation is not available without a "
                                   "workspace (its scratch grows with n); use lu_factor");
        return HPL_ERR_INVALID;
    }
    size_t need = lu_factor_workspace_size(n, opts);
    if (need > kNoAllocScratchBytes) {
        hplgb_internal_set_message("lu_factor_noalloc: these options need more scratch than the fixed "
                                   "device array holds");
        return HPL_ERR_NOMEM;
    }
    void* scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st) return st;
    return lu_factor(n, A, lda, ipiv, opts, scratch, kNoAllocScratchBytes, info, stream);
}
