// mf_internal.h -- declarations shared by the library's translation units
// (kernel parameter blocks and host launchers).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace mf {

constexpr int kFusedThreads = 256;                 // 8 warps per CTA
constexpr int kMaxSmemBytes = 227 * 1024;          // opt-in dynamic shared memory per CTA

struct FusedParams {
    const uint32_t* x;        // input bits (int32 or float32)
    uint32_t* y;              // output bits
    int32_t* argmed;          // optional output indices
    int64_t n;
    int64_t npairs;           // b - 1
    int k, h, G, bpg;
    bool is_float;
    uint32_t off_keyA, off_keyB, off_valA, off_valB, off_hist;
    uint32_t off_rec, off_jpos, off_info;
    uint32_t rec_stride, jpos_stride, info_stride;
};

bool fused_plan(int k, int G, FusedParams* p, size_t* smem_bytes);
int fused_max_k();
cudaError_t fused_setup();
cudaError_t launch_fused(const uint32_t* x, int64_t n, int k, bool is_float,
                         uint32_t* y, int32_t* argmed, int num_sms, cudaStream_t stream,
                         uint64_t* launches);

cudaError_t backward_setup();
cudaError_t launch_backward(const float* gy, const int32_t* argmed, int64_t n, int k,
                            float* gx, cudaStream_t stream, uint64_t* launches);

}  // namespace mf
