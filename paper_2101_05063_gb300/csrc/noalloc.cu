// hsein_solve_noalloc: the solve of hsein_solve without a caller-provided
// workspace, for callers that cannot allocate device memory -- plug-ins whose
// host framework owns all device memory and forbids raw cudaMalloc, or
// real-time paths that must not call an allocator once they are running.
//
// The workspace is a file-scope __device__ array of kNoAllocBytes bytes.  The
// CUDA runtime creates it on every device that loads this library and keeps
// it until the process exits.  In host code the array's name is only a
// host-side stand-in, so its device address is looked up once per device
// (cudaGetSymbolAddress, with that device current) on the first call made on
// that device, cached, and that address is what the kernels receive.  The
// cache is not refreshed: after cudaDeviceReset the cached address of that
// device is stale, so this entry point must not be used across a reset.
//
// Every call shares the one array.  The solve re-initializes all state it
// reads (status word, norms, exponents, bounds) at its start, so the previous
// call's contents do not matter; but two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array.
#include "../../include/hsein.h"
#include "common.cuh"

#include <mutex>

namespace hsein {
int plan_device(const hsein_plan_s* p);
}

namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// device address of the scratch array on device dev, which must be current
// (nullptr on error)
void* scratch_on_device(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[dev] = ptr;
    }
    return g_scratch_ptr[dev];
}

}  // namespace

extern "C" {

hsein_status hsein_solve_noalloc(hsein_plan_t plan, const double* dH, int ldh, const double* dWr,
                                 const double* dWi, const double* dB, int ldb, double* dX, int ldx,
                                 int* dStatus, void* stream) {
    if (!plan) return HSEIN_EARG;
    size_t need = 0;
    hsein_status s = hsein_plan_info(plan, nullptr, nullptr, nullptr, nullptr, nullptr, &need);
    if (s != HSEIN_OK) return s;
    if (need > kNoAllocBytes) return HSEIN_ENOMEM;  // beyond the fixed device array
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return HSEIN_ECUDA;
    // the array is per device: the call runs on the current device, which
    // must be the one the plan was made on
    if (dev != hsein::plan_device(plan)) return HSEIN_EARG;
    void* scratch = scratch_on_device(dev);
    if (!scratch) return HSEIN_ECUDA;
    return hsein_solve(plan, dH, ldh, dWr, dWi, dB, ldb, dX, ldx, dStatus, scratch, kNoAllocBytes,
                       stream);
}

}  // extern "C"
