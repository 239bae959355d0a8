// mf_gen.cu -- synthetic request payloads drawn on the device.
//
// Element i of a payload is output i+1 of SplitMix64 (Steele, Lea and Flood,
// OOPSLA 2014) started at state `seed`: state_i = seed + i * 0x9E3779B97F4A7C15
// (mod 2^64), finalised by xor-shift 30, multiply by 0xBF58476D1CE4E5B9,
// xor-shift 27, multiply by 0x94D049BB133111EB, xor-shift 31.  int32 samples
// are the top 16 bits (uniform on [0, 65536)); float32 samples the top 24
// bits times 2^-24 (uniform on [0, 1)).  Not part of the median filter: the
// request server uses it to create the inputs of served requests in place.
#include <cuda_runtime.h>
#include <cstdint>
#include "mf.h"
#include "mf_gen.h"

namespace mf {

__device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256)
fill_splitmix_kernel(uint32_t* __restrict__ x, int64_t n, uint64_t seed, bool is_float)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t z = splitmix_out(seed, (uint64_t)i);
        uint32_t v;
        if (is_float) {
            const float f = (float)(uint32_t)(z >> 40) * 5.9604644775390625e-8f;   // 2^-24
            v = __float_as_uint(f);
        } else {
            v = (uint32_t)(z >> 48);
        }
        x[i] = v;
    }
}

}  // namespace mf

extern "C" mf_status mf_fill_splitmix(mf_dtype dtype, void* x, int64_t n, uint64_t seed,
                                      void* cuda_stream)
{
    if (!x) return MF_ERR_NULL;
    if (dtype != MF_INT32 && dtype != MF_FLOAT32) return MF_ERR_DTYPE;
    if (n < 0) return MF_ERR_BAD_N;
    if (n == 0) return MF_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MF_ERR_CUDA;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    mf::fill_splitmix_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(
        (uint32_t*)x, n, seed, dtype == MF_FLOAT32);
    return cudaGetLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}
