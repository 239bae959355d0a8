// mf_backward.cu -- gradient of y = median_filter(x) with respect to x.
//
// y[i] is the element x[argmed[i]] (the median is always an input element,
// paper Section 1), so where the window's values are distinct dy[i]/dx[j] is
// 1 for j = argmed[i] and 0 otherwise, and
//     gx[j] = sum over { i : argmed[i] == j } of gy[i].
// argmed[i] lies in [i, i+k-1], so the outputs that can reach j are
// i in [j-k+1, j].  Each thread owns one j and adds the matching gy[i] in
// ascending i from a shared-memory tile: no atomics, a fixed summation order,
// bit-reproducible results.  Rows (independent signals of the same n and k,
// argmed local to the row) run in one launch: grid y strides over them.
#include <cuda_runtime.h>
#include <cstdint>
#include "mf_internal.h"

namespace mf {

constexpr int kBwdThreads = 256;

__global__ void __launch_bounds__(kBwdThreads)
backward_kernel(const float* __restrict__ gy_all, const int32_t* __restrict__ argmed_all,
                int64_t rows, int64_t n, int k, float* __restrict__ gx_all)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t m = n - k + 1;
    const int64_t j0 = (int64_t)blockIdx.x * kBwdThreads;
    const int64_t i0 = j0 - (k - 1);                        // first output that can reach j0
    const int span = kBwdThreads + k - 1;
    int32_t* sa = reinterpret_cast<int32_t*>(smem);
    float* sg = reinterpret_cast<float*>(smem + sizeof(int32_t) * (size_t)span);
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const float* gy = gy_all + row * m;
        const int32_t* argmed = argmed_all + row * m;
        for (int t = threadIdx.x; t < span; t += blockDim.x) {
            const int64_t i = i0 + t;
            const bool ok = i >= 0 && i < m;
            sa[t] = ok ? argmed[i] : -1;
            sg[t] = ok ? gy[i] : 0.0f;
        }
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        if (j < n) {
            const int32_t jj = (int32_t)j;
            float acc = 0.0f;
            for (int t = threadIdx.x; t < threadIdx.x + k; ++t)  // i = j-k+1 .. j, ascending
                if (sa[t] == jj) acc += sg[t];
            gx_all[row * n + j] = acc;
        }
        __syncthreads();                                     // the tile is reused by the next row
    }
}

cudaError_t backward_setup()
{
    return cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxSmemBytes);
}

cudaError_t launch_backward(const float* gy, const int32_t* argmed, int64_t rows, int64_t n, int k,
                            float* gx, cudaStream_t stream, uint64_t* launches)
{
    const int span = kBwdThreads + k - 1;
    const size_t smem = (sizeof(int32_t) + sizeof(float)) * (size_t)span;
    if (smem > (size_t)kMaxSmemBytes) return cudaErrorInvalidValue;
    const int64_t grid = (n + kBwdThreads - 1) / kBwdThreads;
    const dim3 g((unsigned)grid, (unsigned)(rows < 65535 ? rows : 65535));
    backward_kernel<<<g, kBwdThreads, smem, stream>>>(gy, argmed, rows, n, k, gx);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace mf
