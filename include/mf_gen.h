/* mf_gen.h -- synthetic request payloads for the request server.
 *
 * Not part of the paper's method (the paper has no counterpart): the request
 * server in paper_1406_1717_gb300/serve.py creates each served request's
 * samples on the device with this call instead of copying them from the host.
 */
#pragma once
#include <stdint.h>
#include "mf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Write n samples of `dtype` to the device pointer x on `cuda_stream`
 * (cudaStream_t, NULL = legacy default stream of the current device).
 * Sample i is derived from output i+1 of SplitMix64 (Steele, Lea and Flood,
 * OOPSLA 2014) started at state `seed` (state_i = seed + i * 0x9E3779B97F4A7C15
 * mod 2^64, then the published finaliser): MF_INT32 takes the top 16 bits
 * (uniform on [0, 65536)), MF_FLOAT32 the top 24 bits times 2^-24 (uniform on
 * [0, 1), exact).  Asynchronous.
 * Errors: MF_ERR_NULL (x), MF_ERR_DTYPE, MF_ERR_BAD_N (n < 0), MF_ERR_CUDA. */
mf_status mf_fill_splitmix(mf_dtype dtype, void* x, int64_t n, uint64_t seed, void* cuda_stream);

#ifdef __cplusplus
}
#endif
