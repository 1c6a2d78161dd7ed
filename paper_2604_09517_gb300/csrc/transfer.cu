// hpl_upload / hpl_download: an FP64 column-major matrix between page-locked
// host memory and device memory, copied by a kernel that reads (upload) or
// writes (download) the host buffer through its mapped device address (over
// the CPU-GPU link) instead of by the copy engine. On GB300 the copy engine's
// host-to-device copies of a large buffer sometimes stall for hundreds of
// milliseconds after the GPU has been busy or idle for a while (measured:
// 8.6 GB in 41 ms back to back, 302 and 814 ms after such stretches), while
// the kernel copy kept 41-49 ms every time.
#include <algorithm>

#include "common.cuh"

namespace hplgb {

// Contiguous source and destination: 16-byte copies over a grid-stride loop.
__global__ void __launch_bounds__(512) k_upload_flat(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                     size_t n16) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Column by column (leading dimensions lds, ldd): blockIdx.y strides over the
// columns, the threads of x over the rows, two values per thread when both
// columns are 16-byte aligned.
__global__ void __launch_bounds__(512) k_upload_cols(const double* __restrict__ src, int64_t lds,
                                                     double* __restrict__ dst, int64_t ldd, int64_t m, int64_t n,
                                                     int vec2) {
    for (int64_t c = blockIdx.y; c < n; c += gridDim.y) {
        const double* s = src + c * lds;
        double* d = dst + c * ldd;
        if (vec2) {
            const int64_t m2 = m / 2;
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m2;
                 i += (int64_t)gridDim.x * blockDim.x)
                reinterpret_cast<double2*>(d)[i] = reinterpret_cast<const double2*>(s)[i];
            if ((m & 1) && blockIdx.x == 0 && threadIdx.x == 0) d[m - 1] = s[m - 1];
        } else {
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
                 i += (int64_t)gridDim.x * blockDim.x)
                d[i] = s[i];
        }
    }
}

// The copy between two device-addressable matrices (both addresses already
// device addresses).
static int copy_kernel(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd,
                       cudaStream_t s) {
    int dev = 0, sms = kNumSMsGB300;
    HPL_CUDA_TRY(cudaGetDevice(&dev));
    HPL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t bytes = (size_t)m * (size_t)n * sizeof(double);
    const bool flat = lds == m && ldd == m && (((uintptr_t)src | (uintptr_t)dst) & 15) == 0 && bytes % 16 == 0;
    if (flat) {
        const size_t n16 = bytes / 16;
        const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((n16 + 511) / 512, (size_t)sms * 8));
        k_upload_flat<<<blocks, 512, 0, s>>>((const uint4*)src, (uint4*)dst, n16);
    } else {
        const int vec2 = (((uintptr_t)src | (uintptr_t)dst) & 15) == 0 && lds % 2 == 0 && ldd % 2 == 0;
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 1023) / 1024, 8));
        const unsigned gy = (unsigned)std::min<int64_t>(n, 65535);
        k_upload_cols<<<dim3(gx, gy), 512, 0, s>>>(src, lds, dst, ldd, m, n, vec2);
    }
    HPL_LAUNCH_CHECK();
    return HPL_OK;
}

// Device address of a host buffer, or nullptr (message set) when the device
// cannot address it.
static void* host_device_ptr(const double* p, const char* who) {
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, const_cast<double*>(p), 0) != cudaSuccess || !d) {
        cudaGetLastError();
        hplgb_internal_set_message(who);
        return nullptr;
    }
    return d;
}

}  // namespace hplgb

extern "C" int hpl_upload(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd,
                          void* stream) {
    if (m < 0 || n < 0 || lds < (m > 1 ? m : 1) || ldd < (m > 1 ? m : 1)) return HPL_ERR_INVALID;
    if (m == 0 || n == 0) return HPL_OK;
    if (!src || !dst) return HPL_ERR_INVALID;
    void* dsrc = hplgb::host_device_ptr(src, "hpl_upload: the device cannot address this host buffer (page-lock "
                                             "it: cudaHostAlloc or cudaHostRegister; torch pin_memory)");
    if (!dsrc) return HPL_ERR_INVALID;
    return hplgb::copy_kernel(m, n, (const double*)dsrc, lds, dst, ldd, (cudaStream_t)stream);
}

extern "C" int hpl_download(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd,
                            void* stream) {
    if (m < 0 || n < 0 || lds < (m > 1 ? m : 1) || ldd < (m > 1 ? m : 1)) return HPL_ERR_INVALID;
    if (m == 0 || n == 0) return HPL_OK;
    if (!src || !dst) return HPL_ERR_INVALID;
    void* ddst = hplgb::host_device_ptr(dst, "hpl_download: the device cannot address this host buffer (page-lock "
                                             "it: cudaHostAlloc or cudaHostRegister; torch pin_memory)");
    if (!ddst) return HPL_ERR_INVALID;
    return hplgb::copy_kernel(m, n, src, lds, (double*)ddst, ldd, (cudaStream_t)stream);
}
