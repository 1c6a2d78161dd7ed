// Status strings, options, per-device context and last-error text.
#include <atomic>
#include <mutex>
#include <string.h>
#include <vector>

#include "common.cuh"

static char g_last_error[512];
static std::mutex g_err_mu;

extern "C" void hplgb_internal_set_error(cudaError_t e, const char* what, const char* file, int line) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    snprintf(g_last_error, sizeof(g_last_error), "%s (%d) at %s:%d in %s", cudaGetErrorString(e), (int)e,
             file, line, what);
}

// Record a plain message as the last error text.
extern "C" void hplgb_internal_set_message(const char* msg) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

// Text of the last CUDA error met by the library (thread-shared, diagnostic only).
extern "C" const char* hplgb_last_error(void) { return g_last_error; }

extern "C" const char* hpl_status_string(int status) {
    switch (status) {
        case HPL_OK: return "HPL_OK";
        case HPL_ERR_INVALID: return "HPL_ERR_INVALID";
        case HPL_ERR_SINGULAR: return "HPL_ERR_SINGULAR";
        case HPL_ERR_NONFINITE: return "HPL_ERR_NONFINITE";
        case HPL_ERR_NOT_CONVERGED: return "HPL_ERR_NOT_CONVERGED";
        case HPL_ERR_TIMEOUT: return "HPL_ERR_TIMEOUT";
        case HPL_ERR_NOMEM: return "HPL_ERR_NOMEM";
        case HPL_ERR_CUDA: return "HPL_ERR_CUDA";
        default: return "HPL_ERR_UNKNOWN";
    }
}

extern "C" void hpl_default_opts(hpl_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->nb = 0;
    o->lookahead = 1;
    o->prec = HPL_PREC_BF16;
    o->refine = HPL_REFINE_GMRES;
    o->max_iter = 50;
    o->gmres_m = 30;
    o->ns_iters = 2;
    o->tol = 16.0;
    o->timeout_ns = hplgb::kDefaultTimeoutNs;
}

namespace hplgb {

Opts resolve_opts(const hpl_opts* o, int64_t default_nb) {
    hpl_opts d;
    hpl_default_opts(&d);
    if (!o) o = &d;
    Opts r;
    r.nb = o->nb > 0 ? o->nb : default_nb;
    r.lookahead = o->lookahead;
    r.prec = o->prec;
    r.refine = o->refine;
    r.max_iter = o->max_iter > 0 ? o->max_iter : d.max_iter;
    r.gmres_m = o->gmres_m > 0 ? o->gmres_m : d.gmres_m;
    r.ns_iters = o->ns_iters > 0 ? o->ns_iters : d.ns_iters;
    r.tol = o->tol > 0 ? o->tol : d.tol;
    r.timeout_ns = o->timeout_ns > 0 ? o->timeout_ns : d.timeout_ns;
    r.fp64_emulation = o->fp64_emulation;
    r.pfact = o->pfact;
    r.storage = o->storage;
    r.inner = o->inner;
    return r;
}

static std::mutex g_ctx_mu;
static DeviceCtx* g_ctx[kMaxDevices];

int get_ctx(DeviceCtx** out) {
    int dev = 0;
    HPL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return HPL_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    if (!g_ctx[dev]) {
        DeviceCtx* c = new DeviceCtx();
        c->device = dev;
        HPL_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
        int lo = 0, hi = 0;
        HPL_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        HPL_CUDA_TRY(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi));
        for (int i = 0; i < 4; i++) HPL_CUDA_TRY(cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming));
        g_ctx[dev] = c;
    }
    *out = g_ctx[dev];
    return HPL_OK;
}

}  // namespace hplgb

// ---------------------------------------------------------------------------
// Launch counter and phase timers.
namespace hplgb {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct PhaseRec {
    cudaEvent_t a, b;
    int phase;
    int step;      // factorization step k, or -1
    double work;
    bool used;
};
static std::mutex g_ph_mu;
static std::vector<PhaseRec> g_ph;
static size_t g_ph_next = 0;
static int g_ph_on = 0;

int phase_begin(cudaStream_t s) {
    if (!g_ph_on) return -1;
    std::lock_guard<std::mutex> lk(g_ph_mu);
    if (g_ph_next == g_ph.size()) {
        PhaseRec r{};
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
        g_ph.push_back(r);
    }
    int idx = (int)g_ph_next++;
    g_ph[idx].used = false;
    if (cudaEventRecord(g_ph[idx].a, s) != cudaSuccess) return -1;
    return idx;
}

void phase_end(int slot, cudaStream_t s, int phase, double work, int step) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_ph_mu);
    PhaseRec& r = g_ph[slot];
    r.phase = phase;
    r.step = step;
    r.work = work;
    r.used = cudaEventRecord(r.b, s) == cudaSuccess;
}

}  // namespace hplgb

extern "C" long long hplgb_launch_count(void) { return hplgb::g_launches.load(); }

extern "C" void hplgb_set_phase_timing(int on) {
    std::lock_guard<std::mutex> lk(hplgb::g_ph_mu);
    hplgb::g_ph_on = on;
    hplgb::g_ph_next = 0;
}

extern "C" int hplgb_phase_records(int32_t* phase, int32_t* step, double* start_ms, double* ms, double* work,
                                   long long cap, long long* count) {
    using namespace hplgb;
    std::lock_guard<std::mutex> lk(g_ph_mu);
    long long k = 0;
    int first = -1;
    for (size_t i = 0; i < g_ph_next; i++) {
        PhaseRec& r = g_ph[i];
        if (!r.used) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return HPL_ERR_CUDA;
        if (first < 0) first = (int)i;
        if (k < cap) {
            float t = 0.0f, t0 = 0.0f;
            if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return HPL_ERR_CUDA;
            if (cudaEventElapsedTime(&t0, g_ph[first].a, r.a) != cudaSuccess) return HPL_ERR_CUDA;
            if (phase) phase[k] = r.phase;
            if (step) step[k] = r.step;
            if (start_ms) start_ms[k] = t0;
            if (ms) ms[k] = t;
            if (work) work[k] = r.work;
        }
        k++;
    }
    if (count) *count = k;
    return HPL_OK;
}

extern "C" int hplgb_phase_times(double* ms, double* work, long long* count) {
    using namespace hplgb;
    std::lock_guard<std::mutex> lk(g_ph_mu);
    for (int p = 0; p < PH_COUNT; p++) {
        if (ms) ms[p] = 0.0;
        if (work) work[p] = 0.0;
        if (count) count[p] = 0;
    }
    for (size_t i = 0; i < g_ph_next; i++) {
        PhaseRec& r = g_ph[i];
        if (!r.used) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return HPL_ERR_CUDA;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return HPL_ERR_CUDA;
        if (ms) ms[r.phase] += t;
        if (work) work[r.phase] += r.work;
        if (count) count[r.phase] += 1;
    }
    g_ph_next = 0;
    return HPL_OK;
}
