// mf_api.cu -- the C ABI declared in include/mf.h: handle, argument checks,
// workspace, dispatch to the CUDA kernels.  No CPU fallback: every result is
// computed by the kernels of this library.
#include <cuda_runtime.h>
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <new>
#include <vector>

#include "mf.h"
#include "mf_internal.h"

struct mf_ctx {
    int device;
    cudaStream_t stream;
    size_t max_ws;
    void* ws;
    size_t ws_size;
    int num_sms;
    int max_k;
    int large_from_k;         // k >= this runs the large-k tier (k above the
                              // shared-memory pipeline's limit always does)
    mf::LaunchStats stats;
    bool events_made;
    mf::Tuning tune[mf::kNumTuneClasses];
    // pinned staging of batched descriptor tables; a buffer that a captured
    // call used belongs to that graph and is kept until mf_destroy
    void* stage;
    size_t stage_size;
    bool stage_in_graph;
    cudaEvent_t stage_done;
    std::vector<void*> retired;
    // copy-in and copy-out streams of the chunked host entry point, the
    // fork / join events and, per buffer slot, the events that chain a
    // chunk's copy-in, filter and copy-out
    cudaStream_t aux = nullptr, aux2 = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    static constexpr int kHostSlots = 3;
    cudaEvent_t ev_in[kHostSlots] = {}, ev_done[kHostSlots] = {}, ev_out[kHostSlots] = {};
};

namespace {

// Make `dev` current for the scope of a call and restore the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return na && nb && pa < pb + nb && pb < pa + na;
}

bool dtype_ok(int dtype) {
    return dtype == MF_INT32 || dtype == MF_FLOAT32 || dtype == MF_INT64 || dtype == MF_FLOAT64;
}

mf::Elem elem_of(int dtype) {
    mf::Elem e;
    e.is_float = dtype == MF_FLOAT32 || dtype == MF_FLOAT64;
    e.wide = dtype == MF_INT64 || dtype == MF_FLOAT64;
    return e;
}

mf_status check_common(mf_handle h, int dtype, const void* x, int64_t n, int32_t k, const void* y) {
    if (!h || !x || !y) return MF_ERR_NULL;
    if (!dtype_ok(dtype)) return MF_ERR_DTYPE;
    if (n < 1) return MF_ERR_BAD_N;
    if (k < 1) return MF_ERR_K_GT_N;
    if (k % 2 == 0) return MF_ERR_EVEN_K;
    if ((int64_t)k > n) return MF_ERR_K_GT_N;
    return MF_OK;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) { cudaGetLastError(); return false; }
    return st == cudaStreamCaptureStatusActive;
}

mf_status ensure_workspace(mf_handle h, size_t bytes) {
    if (h->ws_size >= bytes) return MF_OK;
    if (h->max_ws && bytes > h->max_ws) return MF_ERR_OOM;
    if (capturing(h->stream)) return MF_ERR_OOM;      // allocate before capturing
    if (h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_size = 0;
    }
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return MF_ERR_OOM;
    }
    h->ws_size = bytes;
    return MF_OK;
}

mf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MF_OK : MF_ERR_CUDA; }

// Workspace of one signal: shared-memory pipeline up to pipeline_max_k(),
// the global-memory large-k tier above it.
bool use_large(mf_handle h, int k, bool wide) {
    return k >= h->large_from_k || k > mf::pipeline_max_k(wide);
}

size_t signal_workspace_bytes(mf_handle h, int64_t n, int k, bool wide) {
    return use_large(h, k, wide) ? mf::large_workspace_bytes(n, k, wide)
                                 : mf::pipeline_workspace_bytes(n, k);
}

// Workspace of a batched call: the pipeline group and, reusing the same
// memory afterwards, the large-k group (all its signals at once).
size_t batched_need(mf_handle h, const mf_segment* segs, int32_t nseg, bool wide) {
    std::vector<int64_t> nn, bn;
    std::vector<int32_t> kk, bk;
    for (int32_t s = 0; s < nseg; ++s) {
        if (use_large(h, segs[s].k, wide)) {
            bn.push_back(segs[s].n);
            bk.push_back(segs[s].k);
        } else {
            nn.push_back(segs[s].n);
            kk.push_back(segs[s].k);
        }
    }
    const size_t small_need =
        kk.empty() ? 0 : mf::pipeline_batched_workspace_bytes(nn.data(), kk.data(), (int)kk.size());
    const size_t big_need =
        bk.empty() ? 0 : mf::large_batched_workspace_bytes(bn.data(), bk.data(), (int)bk.size(), wide);
    return std::max(small_need, big_need);
}

cudaError_t launch_signal(mf_handle h, const void* x, int64_t n, int k, int rank,
                          mf::Elem el, void* y, int32_t* argmed, void* ws, size_t ws_bytes,
                          cudaStream_t stream) {
    if (!use_large(h, k, el.wide))
        return mf::launch_pipeline(x, n, k, rank, el, y, argmed, ws, ws_bytes, h->num_sms,
                                   stream, &h->stats);
    return mf::launch_large(x, n, k, rank, el, y, argmed, ws, ws_bytes, stream, &h->stats);
}

// argmed of a chunk is relative to the chunk's first input; shift it to the
// whole signal's numbering
__global__ void add_offset_kernel(int32_t* a, int64_t count, int32_t off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] += off;
}

// Shared body of mf_filter / mf_filter_rank after the window checks.
mf_status filter_device(mf_handle h, mf_dtype dtype, const void* x, int64_t n, int32_t k,
                        int32_t rank, void* y, int32_t* argmed) {
    if (argmed && n > (int64_t)INT32_MAX) return MF_ERR_BAD_N;
    if (k > h->max_k) return MF_ERR_UNSUPPORTED;
    const size_t m = (size_t)(n - k + 1);
    const mf::Elem el = elem_of(dtype);
    const size_t eb = (size_t)el.bytes();
    if (overlaps(x, eb * (size_t)n, y, eb * m)) return MF_ERR_OVERLAP;
    if (argmed && (overlaps(x, eb * (size_t)n, argmed, 4 * m) || overlaps(y, eb * m, argmed, 4 * m)))
        return MF_ERR_OVERLAP;
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    const size_t need = signal_workspace_bytes(h, n, k, el.wide);
    mf_status st = ensure_workspace(h, need);
    if (st != MF_OK) return st;
    return cuda_status(launch_signal(h, x, n, k, rank, el, y, argmed, h->ws, need, h->stream));
}

}  // namespace

extern "C" {

mf_status mf_create(mf_handle* out, int device, void* cuda_stream, size_t max_workspace_bytes) {
    if (!out) return MF_ERR_NULL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) { cudaGetLastError(); return MF_ERR_DEVICE; }
    if (device < 0 || device >= count) return MF_ERR_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return MF_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return MF_ERR_DEVICE;
    DeviceGuard g(device);
    if (!g.ok) return MF_ERR_CUDA;
    if (mf::pipeline_setup() != cudaSuccess || mf::large_setup() != cudaSuccess ||
        mf::backward_setup() != cudaSuccess)
        return MF_ERR_CUDA;
    mf_ctx* h = new (std::nothrow) mf_ctx();
    if (!h) return MF_ERR_OOM;
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    h->max_ws = max_workspace_bytes;
    h->ws = nullptr;
    h->ws_size = 0;
    h->num_sms = prop.multiProcessorCount;
    h->max_k = mf::kLargeMaxK;
    h->large_from_k = std::min(mf::kLargeFromK, mf::pipeline_max_k() + 1);
    h->events_made = false;
    for (int c = 0; c < mf::kNumTuneClasses; ++c) h->tune[c] = mf::Tuning{0, 0, 0};
    h->stats.tune = h->tune;
    h->stage = nullptr;
    h->stage_size = 0;
    h->stage_in_graph = false;
    if (cudaEventCreateWithFlags(&h->stage_done, cudaEventDisableTiming) != cudaSuccess) {
        delete h;
        return MF_ERR_CUDA;
    }
    *out = h;
    return MF_OK;
}

mf_status mf_set_stream(mf_handle h, void* cuda_stream) {
    if (!h) return MF_ERR_NULL;
    h->stream = (cudaStream_t)cuda_stream;
    return MF_OK;
}

mf_status mf_filter(mf_handle h, mf_dtype dtype, const void* x, int64_t n, int32_t k,
                    void* y, int32_t* argmed) {
    mf_status st = check_common(h, dtype, x, n, k, y);
    if (st != MF_OK) return st;
    return filter_device(h, dtype, x, n, k, (k - 1) / 2, y, argmed);
}

mf_status mf_filter_rank(mf_handle h, mf_dtype dtype, const void* x, int64_t n, int32_t k,
                         int32_t rank, void* y, int32_t* argmed) {
    if (!h || !x || !y) return MF_ERR_NULL;
    if (!dtype_ok(dtype)) return MF_ERR_DTYPE;
    if (n < 1) return MF_ERR_BAD_N;
    if (k < 1 || (int64_t)k > n) return MF_ERR_K_GT_N;
    if (rank < 0 || rank >= k) return MF_ERR_BAD_RANK;
    return filter_device(h, dtype, x, n, k, rank, y, argmed);
}

// Outputs per chunk of the host entry point: about 1/8 of the signal, at
// least 2^20 outputs, a multiple of k.  The chunks run as a pipeline on three
// streams -- copy-in, filter (the handle's stream), copy-out -- chained by one
// event per step, with kHostSlots device buffer slots in flight; so the
// copies of one chunk overlap the filtering of its neighbours, and H2D and
// D2H (separate copy engines) overlap each other.
static int64_t host_chunk_outputs(int64_t m, int k) {
    const int64_t target = std::max<int64_t>((m + 7) / 8, (int64_t)1 << 20);
    return (target + k - 1) / k * k;
}

mf_status mf_filter_host(mf_handle h, mf_dtype dtype, const void* x_host, int64_t n, int32_t k,
                         void* y_host, int32_t* argmed_host) {
    mf_status st = check_common(h, dtype, x_host, n, k, y_host);
    if (st != MF_OK) return st;
    if (argmed_host && n > (int64_t)INT32_MAX) return MF_ERR_BAD_N;
    if (k > h->max_k) return MF_ERR_UNSUPPORTED;
    const int64_t m = n - k + 1;
    const mf::Elem el = elem_of(dtype);
    const size_t eb = (size_t)el.bytes();
    const int rank = (k - 1) / 2;
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    // Chunk c filters inputs [c L, c L + L + k - 1) into outputs [c L, c L + L):
    // every window lies inside one chunk, so the results equal one whole call.
    const int64_t L = host_chunk_outputs(m, k);
    const int64_t nchunks = (m + L - 1) / L;
    constexpr int R = mf_ctx::kHostSlots;
    const int nslots = (int)std::min<int64_t>(nchunks, R);
    const int64_t cin = std::min<int64_t>(n, L + k - 1);
    const size_t xb = (eb * (size_t)cin + 255) & ~size_t(255);
    const size_t yb = (eb * (size_t)L + 255) & ~size_t(255);
    const size_t ab = argmed_host ? ((4 * (size_t)L + 255) & ~size_t(255)) : 0;
    const size_t need = signal_workspace_bytes(h, cin, k, el.wide);
    const size_t slot_bytes = xb + yb + ab;
    const size_t ws_off = slot_bytes * (size_t)nslots;   // one filter workspace, after the slots
    st = ensure_workspace(h, ws_off + ((need + 255) & ~size_t(255)));
    if (st != MF_OK) return st;
    if (!h->aux) {
        bool ok = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h->aux2, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) == cudaSuccess;
        for (int r = 0; ok && r < R; ++r)
            ok = cudaEventCreateWithFlags(&h->ev_in[r], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_done[r], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_out[r], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return MF_ERR_CUDA;
        }
    }
    cudaStream_t sin = h->aux, sfl = h->stream, sout = h->aux2;
    // both copy streams start after the work already on the handle's stream
    cudaError_t e = cudaEventRecord(h->fork_ev, sfl);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, h->fork_ev, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, h->fork_ev, 0);
    void* wsd = (char*)h->ws + ws_off;
    for (int64_t c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int slot = (int)(c % R);
        char* base = (char*)h->ws + slot_bytes * slot;
        void* xd = base;
        void* yd = base + xb;
        int32_t* ad = argmed_host ? (int32_t*)(base + xb + yb) : nullptr;
        const int64_t off = c * L;
        const int64_t out = std::min(L, m - off);
        const int64_t in = out + k - 1;
        // copy-in, once the slot's previous chunk has been copied out
        if (c >= R) e = cudaStreamWaitEvent(sin, h->ev_out[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(xd, (const char*)x_host + eb * off, eb * (size_t)in,
                                cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[slot], sin);
        // filter
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sfl, h->ev_in[slot], 0);
        if (e == cudaSuccess) e = launch_signal(h, xd, in, k, rank, el, yd, ad, wsd, need, sfl);
        if (e == cudaSuccess && ad && off > 0) {
            add_offset_kernel<<<(unsigned)((out + 255) / 256), 256, 0, sfl>>>(ad, out, (int32_t)off);
            h->stats.launches += 1;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_done[slot], sfl);
        // copy-out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, h->ev_done[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)y_host + eb * off, yd, eb * (size_t)out,
                                cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess && ad)
            e = cudaMemcpyAsync(argmed_host + off, ad, 4 * (size_t)out, cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[slot], sout);
    }
    // the handle's stream waits for the last copy-out (and the copy-in stream)
    const cudaError_t e2 = cudaEventRecord(h->join_ev, sout);
    if (e2 == cudaSuccess) cudaStreamWaitEvent(sfl, h->join_ev, 0);
    if (e == cudaSuccess) e = e2;
    const cudaError_t e3 = cudaStreamSynchronize(sfl);
    const cudaError_t e4 = cudaStreamSynchronize(sin);
    if (e == cudaSuccess) e = e3;
    if (e == cudaSuccess) e = e4;
    return cuda_status(e);
}

mf_status mf_filter_batched(mf_handle h, mf_dtype dtype, const void* x, void* y,
                            const mf_segment* segs, int32_t nseg, int32_t* argmed) {
    if (!h || !x || !y || (!segs && nseg > 0)) return MF_ERR_NULL;
    if (!dtype_ok(dtype)) return MF_ERR_DTYPE;
    if (nseg < 0) return MF_ERR_BAD_SEGMENT;
    const mf::Elem el = elem_of(dtype);
    const size_t eb = (size_t)el.bytes();
    int64_t xext = 0, yext = 0;
    std::vector<std::pair<int64_t, int64_t>> yr;
    yr.reserve((size_t)nseg);
    for (int32_t s = 0; s < nseg; ++s) {
        const mf_segment& d = segs[s];
        if (d.pad != 0 || d.x_off < 0 || d.y_off < 0 || d.n < 1 || d.k < 1 || d.k % 2 == 0 ||
            (int64_t)d.k > d.n || d.k > h->max_k)
            return MF_ERR_BAD_SEGMENT;
        if (argmed && d.n > (int64_t)INT32_MAX) return MF_ERR_BAD_SEGMENT;
        const int64_t m = d.n - d.k + 1;
        xext = std::max(xext, d.x_off + d.n);
        yext = std::max(yext, d.y_off + m);
        yr.emplace_back(d.y_off, d.y_off + m);
    }
    std::sort(yr.begin(), yr.end());
    for (size_t i = 1; i < yr.size(); ++i)
        if (yr[i].first < yr[i - 1].second) return MF_ERR_OVERLAP;
    if (overlaps(x, eb * (size_t)xext, y, eb * (size_t)yext)) return MF_ERR_OVERLAP;
    if (argmed && (overlaps(x, eb * (size_t)xext, argmed, 4 * (size_t)yext) ||
                   overlaps(y, eb * (size_t)yext, argmed, 4 * (size_t)yext)))
        return MF_ERR_OVERLAP;
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    if (nseg == 0) return MF_OK;
    // signals of the shared-memory pipeline go into one batched launch group
    // (one launch per kernel and window class), then the large-k ones into one
    // launch sequence of the global-memory tier, reusing the same workspace;
    // the number of launches depends on neither the number of signals nor the
    // number of large-k signals
    std::vector<int64_t> xo, nn, yo, bxo, bnn, byo;
    std::vector<int32_t> kk, bkk;
    for (int32_t s = 0; s < nseg; ++s) {
        const mf_segment& d = segs[s];
        if (use_large(h, d.k, el.wide)) {
            bxo.push_back(d.x_off); bnn.push_back(d.n); byo.push_back(d.y_off); bkk.push_back(d.k);
        } else {
            xo.push_back(d.x_off); nn.push_back(d.n); yo.push_back(d.y_off); kk.push_back(d.k);
        }
    }
    const int32_t nsmall = (int32_t)kk.size(), nbig = (int32_t)bkk.size();
    const size_t need = batched_need(h, segs, nseg, el.wide);
    mf_status st = ensure_workspace(h, need);
    if (st != MF_OK) return st;
    // pinned staging: the pipeline's descriptors, then the large tier's
    const size_t small_stage = ((size_t)nsmall * sizeof(mf::PipeParams) + 255) & ~size_t(255);
    const size_t stage_need = small_stage + (size_t)nbig * mf::large_descriptor_bytes();
    const bool cap = capturing(h->stream);
    if (!cap) {
        if (h->stage_in_graph) {                      // leave that buffer to its graph
            h->retired.push_back(h->stage);
            h->stage = nullptr;
            h->stage_size = 0;
            h->stage_in_graph = false;
        } else if (h->stage) {
            cudaEventSynchronize(h->stage_done);      // previous copy has read the buffer
        }
        if (h->stage_size < stage_need) {
            if (h->stage) cudaFreeHost(h->stage);
            h->stage = nullptr;
            h->stage_size = 0;
            if (cudaMallocHost(&h->stage, stage_need) != cudaSuccess) { cudaGetLastError(); return MF_ERR_OOM; }
            h->stage_size = stage_need;
        }
    } else if (h->stage_size < stage_need || h->stage_in_graph) {
        return MF_ERR_OOM;                            // make one uncaptured call of this size first
    }
    cudaError_t e = cudaSuccess;
    if (nsmall > 0)
        e = mf::launch_pipeline_batched(x, y, argmed, el, xo.data(), nn.data(), yo.data(),
                                        kk.data(), nsmall, h->ws, need, h->stage, small_stage,
                                        h->num_sms, h->stream, &h->stats);
    if (e == cudaSuccess && nbig > 0)
        e = mf::launch_large_batched(x, y, argmed, el, bxo.data(), bnn.data(), byo.data(), bkk.data(),
                                     nbig, h->ws, need, (char*)h->stage + small_stage,
                                     stage_need - small_stage, h->stream, &h->stats);
    if (e != cudaSuccess) return MF_ERR_CUDA;
    if (cap) h->stage_in_graph = true;
    else cudaEventRecord(h->stage_done, h->stream);
    return MF_OK;
}

mf_status mf_filter_backward_rows(mf_handle h, const float* gy, const int32_t* argmed,
                                  int64_t rows, int64_t n, int32_t k, float* gx) {
    if (!h || !gy || !argmed || !gx) return MF_ERR_NULL;
    if (rows < 1 || n < 1 || n > (int64_t)INT32_MAX) return MF_ERR_BAD_N;
    if (k < 1) return MF_ERR_K_GT_N;
    if (k % 2 == 0) return MF_ERR_EVEN_K;
    if ((int64_t)k > n) return MF_ERR_K_GT_N;
    const size_t m = (size_t)(n - k + 1);
    const size_t gxb = 4 * (size_t)n * (size_t)rows, inb = 4 * m * (size_t)rows;
    if (overlaps(gx, gxb, gy, inb) || overlaps(gx, gxb, argmed, inb)) return MF_ERR_OVERLAP;
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    cudaError_t e = mf::launch_backward(gy, argmed, rows, n, k, gx, h->stream, &h->stats.launches);
    if (e == cudaErrorInvalidValue) return MF_ERR_UNSUPPORTED;
    return cuda_status(e);
}

mf_status mf_filter_backward(mf_handle h, const float* gy, const int32_t* argmed,
                             int64_t n, int32_t k, float* gx) {
    return mf_filter_backward_rows(h, gy, argmed, 1, n, k, gx);
}

mf_status mf_sync(mf_handle h) {
    if (!h) return MF_ERR_NULL;
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(h->stream));
}

mf_status mf_debug_take(mf_handle h, uint32_t* count, uint32_t* site, uint64_t* value) {
    if (!h || !count || !site || !value) return MF_ERR_NULL;
    *count = 0;
    *site = 0;
    *value = 0;
#ifdef MF_DEBUG
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    cudaError_t e = cudaDeviceSynchronize();          // kernels of every stream, aux included
    using Take = cudaError_t (*)(uint32_t*, uint32_t*, uint64_t*);
    const Take takes[] = {mf::debug_take_sortlist, mf::debug_take_pipeline, mf::debug_take_large};
    for (Take t : takes) {
        uint32_t c = 0, st = 0;
        uint64_t v = 0;
        if (e == cudaSuccess) e = t(&c, &st, &v);
        if (c > 0 && *count == 0) {
            *site = st;
            *value = v;
        }
        *count += c;
    }
    return cuda_status(e);
#else
    return MF_ERR_UNSUPPORTED;
#endif
}

mf_status mf_debug_selftest(mf_handle h) {
    if (!h) return MF_ERR_NULL;
#ifdef MF_DEBUG
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    return cuda_status(mf::debug_selftest(h->stream));
#else
    return MF_ERR_UNSUPPORTED;
#endif
}

mf_status mf_launch_count(mf_handle h, uint64_t* count) {
    if (!h || !count) return MF_ERR_NULL;
    *count = h->stats.launches;
    return MF_OK;
}

mf_status mf_set_tuning(mf_handle h, int32_t k, int32_t sort_pairs_per_cta, int32_t store_pairs_per_cta) {
    if (!h) return MF_ERR_NULL;
    if (k < 1) return MF_ERR_K_GT_N;
    mf::Tuning& t = h->tune[mf::tune_class_of(k)];
    t.sort_G = sort_pairs_per_cta > 0 ? sort_pairs_per_cta : 0;
    t.epi_G = store_pairs_per_cta > 0 ? store_pairs_per_cta : 0;
    return MF_OK;
}

mf_status mf_set_sort_variant(mf_handle h, int32_t k, int32_t variant) {
    if (!h) return MF_ERR_NULL;
    if (k < 1) return MF_ERR_K_GT_N;
    if (variant < 0 || variant > 3) return MF_ERR_UNSUPPORTED;
    h->tune[mf::tune_class_of(k)].variant = variant;
    return MF_OK;
}

mf_status mf_batched_workspace_bytes(mf_handle h, mf_dtype dtype, const mf_segment* segs,
                                     int32_t nseg, size_t* bytes) {
    if (!h || !bytes || (!segs && nseg > 0)) return MF_ERR_NULL;
    if (!dtype_ok(dtype)) return MF_ERR_DTYPE;
    if (nseg < 0) return MF_ERR_BAD_SEGMENT;
    for (int32_t s = 0; s < nseg; ++s) {
        const mf_segment& d = segs[s];
        if (d.pad != 0 || d.n < 1 || d.k < 1 || d.k % 2 == 0 || (int64_t)d.k > d.n || d.k > h->max_k)
            return MF_ERR_BAD_SEGMENT;
    }
    *bytes = batched_need(h, segs, nseg, elem_of(dtype).wide);
    return MF_OK;
}

mf_status mf_workspace_size(mf_handle h, size_t* bytes) {
    if (!h || !bytes) return MF_ERR_NULL;
    *bytes = h->ws_size;
    return MF_OK;
}

mf_status mf_release_workspace(mf_handle h) {
    if (!h) return MF_ERR_NULL;
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    if (capturing(h->stream)) return MF_ERR_UNSUPPORTED;
    if (!h->ws) return MF_OK;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return MF_ERR_CUDA;
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_size = 0;
    return MF_OK;
}

mf_status mf_set_tier_threshold(mf_handle h, int32_t k) {
    if (!h) return MF_ERR_NULL;
    if (k < 0) return MF_ERR_K_GT_N;
    const int lim = mf::pipeline_max_k() + 1;
    h->large_from_k = k == 0 ? std::min(mf::kLargeFromK, lim) : std::min(k, lim);
    return MF_OK;
}

mf_status mf_get_tier_threshold(mf_handle h, int32_t* k) {
    if (!h || !k) return MF_ERR_NULL;
    *k = h->large_from_k;
    return MF_OK;
}

mf_status mf_set_timing(mf_handle h, int enable) {
    if (!h) return MF_ERR_NULL;
    if (enable && !h->events_made) {
        DeviceGuard g(h->device);
        if (!g.ok) return MF_ERR_CUDA;
        for (int r = 0; r < mf::LaunchStats::kRing; ++r)
            for (int j = 0; j < 5; ++j)
                if (cudaEventCreate(&h->stats.ev[r][j]) != cudaSuccess) return MF_ERR_CUDA;
        h->events_made = true;
    }
    h->stats.timing = enable != 0;
    h->stats.ring_pos = 0;
    return MF_OK;
}

mf_status mf_kernel_times(mf_handle h, int32_t ncalls, float* ms) {
    if (!h || !ms) return MF_ERR_NULL;
    for (int j = 0; j < 4; ++j) ms[j] = 0.0f;
    if (!h->events_made || ncalls < 1) return MF_OK;
    DeviceGuard g(h->device);
    if (!g.ok) return MF_ERR_CUDA;
    const uint64_t have = h->stats.ring_pos;
    uint64_t use = (uint64_t)ncalls;
    if (use > have) use = have;
    if (use > (uint64_t)mf::LaunchStats::kRing) use = mf::LaunchStats::kRing;
    for (uint64_t c = have - use; c < have; ++c) {
        cudaEvent_t* ev = h->stats.ev[c % mf::LaunchStats::kRing];
        if (cudaEventSynchronize(ev[4]) != cudaSuccess) return MF_ERR_CUDA;
        for (int j = 0; j < 4; ++j) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, ev[j], ev[j + 1]) != cudaSuccess) return MF_ERR_CUDA;
            ms[j] += t;
        }
    }
    return MF_OK;
}

const char* mf_status_str(mf_status s) {
    switch (s) {
        case MF_OK: return "MF_OK";
        case MF_ERR_NULL: return "MF_ERR_NULL: a required pointer or the handle is NULL";
        case MF_ERR_BAD_N: return "MF_ERR_BAD_N: n < 1 or too large";
        case MF_ERR_EVEN_K: return "MF_ERR_EVEN_K: window size must be odd";
        case MF_ERR_K_GT_N: return "MF_ERR_K_GT_N: need 1 <= k <= n";
        case MF_ERR_DTYPE: return "MF_ERR_DTYPE: unknown dtype";
        case MF_ERR_OOM: return "MF_ERR_OOM: workspace allocation failed or above the cap";
        case MF_ERR_CUDA: return "MF_ERR_CUDA: a CUDA call or kernel failed";
        case MF_ERR_UNSUPPORTED: return "MF_ERR_UNSUPPORTED: not served by this library variant";
        case MF_ERR_OVERLAP: return "MF_ERR_OVERLAP: output overlaps an input";
        case MF_ERR_DEVICE: return "MF_ERR_DEVICE: no such device or not compute capability 10.3";
        case MF_ERR_BAD_SEGMENT: return "MF_ERR_BAD_SEGMENT: invalid batched segment descriptor";
        case MF_ERR_TOO_LARGE: return "MF_ERR_TOO_LARGE: request exceeds the fixed no-alloc scratch";
        case MF_ERR_BAD_RANK: return "MF_ERR_BAD_RANK: rank outside 0 .. k-1";
    }
    return "MF_ERR_UNKNOWN";
}

mf_status mf_destroy(mf_handle h) {
    if (!h) return MF_ERR_NULL;
    {
        DeviceGuard g(h->device);
        if (g.ok) {
            cudaStreamSynchronize(h->stream);
            if (h->ws) cudaFree(h->ws);
            if (h->events_made)
                for (int r = 0; r < mf::LaunchStats::kRing; ++r)
                    for (int j = 0; j < 5; ++j) cudaEventDestroy(h->stats.ev[r][j]);
            cudaEventDestroy(h->stage_done);
            if (h->aux) {
                cudaStreamSynchronize(h->aux);
                cudaStreamSynchronize(h->aux2);
                cudaStreamDestroy(h->aux);
                cudaStreamDestroy(h->aux2);
                cudaEventDestroy(h->fork_ev);
                cudaEventDestroy(h->join_ev);
                for (int r = 0; r < mf_ctx::kHostSlots; ++r) {
                    cudaEventDestroy(h->ev_in[r]);
                    cudaEventDestroy(h->ev_done[r]);
                    cudaEventDestroy(h->ev_out[r]);
                }
            }
            if (h->stage) cudaFreeHost(h->stage);
            for (void* r : h->retired) cudaFreeHost(r);
        }
    }
    delete h;
    return MF_OK;
}

}  // extern "C"
