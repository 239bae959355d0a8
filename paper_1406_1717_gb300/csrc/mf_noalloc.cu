// mf_noalloc.cu -- mf_filter_noalloc: the median filter without any device
// allocation, for callers that cannot call cudaMalloc.
//
// The regular entry points keep their scratch in a workspace the handle
// allocates on first use.  Some callers cannot allow that: applications whose
// device memory is handed out only by their own pool or arena and must see no
// foreign allocation, and real-time loops where an allocation's unbounded
// latency is not acceptable.  For them
// this file holds the scratch in a fixed, file-scope device array that exists
// for as long as the library is loaded.  The caller still passes its own
// input and output buffers.
#include <cuda_runtime.h>
#include <climits>
#include <cstdint>
#include <mutex>

#include "mf.h"
#include "mf_internal.h"

namespace {

// 32 MiB of scratch, resident on every GPU that loads this library.
constexpr size_t kNoAllocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSlot {
    bool ready = false;
    void* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 0;
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return na && nb && pa < pb + nb && pb < pa + na;
}

// Per-device set-up, done by the first call on each device with that device
// current: look up the array's device address (the symbol's name in host
// code is only a stand-in), check the GPU, set the kernels' shared-memory
// limits.  None of this allocates.
mf_status device_slot(int dev, DeviceSlot** out) {
    if (dev < 0 || dev >= kMaxDevices) return MF_ERR_DEVICE;
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSlot& s = g_slots[dev];
    if (!s.ready) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return MF_ERR_CUDA;
        if (prop.major != 10 || prop.minor != 3) return MF_ERR_DEVICE;
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return MF_ERR_CUDA;
        }
        if (mf::pipeline_setup() != cudaSuccess) return MF_ERR_CUDA;
        s.scratch = ptr;
        s.num_sms = prop.multiProcessorCount;
        s.ready = true;
    }
    *out = &s;
    return MF_OK;
}

}  // namespace

extern "C" mf_status mf_filter_noalloc(mf_dtype dtype, const void* x, int64_t n, int32_t k,
                                       void* y, int32_t* argmed, void* cuda_stream) {
    if (!x || !y) return MF_ERR_NULL;
    if (dtype != MF_INT32 && dtype != MF_FLOAT32) return MF_ERR_DTYPE;
    if (n < 1) return MF_ERR_BAD_N;
    if (k < 1) return MF_ERR_K_GT_N;
    if (k % 2 == 0) return MF_ERR_EVEN_K;
    if ((int64_t)k > n) return MF_ERR_K_GT_N;
    if (argmed && n > (int64_t)INT32_MAX) return MF_ERR_BAD_N;
    if (k > mf::pipeline_max_k()) return MF_ERR_UNSUPPORTED;
    const size_t m = (size_t)(n - k + 1);
    if (ranges_overlap(x, 4 * (size_t)n, y, 4 * m)) return MF_ERR_OVERLAP;
    if (argmed && (ranges_overlap(x, 4 * (size_t)n, argmed, 4 * m) ||
                   ranges_overlap(y, 4 * m, argmed, 4 * m)))
        return MF_ERR_OVERLAP;
    const size_t need = mf::pipeline_workspace_bytes(n, k);
    if (need > kNoAllocScratchBytes) return MF_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MF_ERR_CUDA;
    DeviceSlot* slot = nullptr;
    mf_status st = device_slot(dev, &slot);
    if (st != MF_OK) return st;
    // Every element of the scratch that the kernels read is written earlier in
    // the same call, so nothing has to be cleared between calls.
    mf::Elem el;
    el.is_float = dtype == MF_FLOAT32;
    el.wide = false;
    const cudaError_t e = mf::launch_pipeline(x, n, k, (k - 1) / 2, el, y, argmed, slot->scratch,
                                              kNoAllocScratchBytes, slot->num_sms,
                                              (cudaStream_t)cuda_stream, nullptr);
    return e == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}
