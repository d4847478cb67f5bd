// Forward evaluation from host buffers: a chunked three-stage pipeline
// (host->device copy, kernel, device->host copy) over a caller-provided
// device workspace, on three library-owned streams per device, ordered after
// the caller's stream on entry and before it on exit.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "sph_internal.h"

namespace sph {
namespace {

constexpr int kHostMaxDevices = 64;
constexpr int kStages = 2;  // double-buffered device chunks

struct HostPipe {
    cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    cudaEvent_t h2d_ev[kStages] = {}, comp_ev[kStages] = {}, free_ev[kStages] = {};
    bool ready = false;
    bool used = false;  // `done` marks the previous call's last copy
};
std::mutex g_pipe_mu;
HostPipe g_pipe[kHostMaxDevices];

cudaError_t pipe_for(int dev, HostPipe** out) {
    HostPipe& p = g_pipe[dev];
    if (!p.ready) {
        cudaError_t e = cudaStreamCreateWithFlags(&p.h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.comp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.d2h, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming);
        for (int b = 0; b < kStages && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&p.h2d_ev[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.comp_ev[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.free_ev[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
        p.ready = true;
    }
    *out = &p;
    return cudaSuccess;
}

}  // namespace
}  // namespace sph

using namespace sph;

extern "C" int sphericart_compute_host(const void* xyz_host, int64_t n, int l_max, int normalized, int dtype,
                                       int out, void* sph_host, void* dsph_host, void* workspace,
                                       size_t workspace_bytes, int64_t chunk_points, void* stream) {
    if (n < 0 || l_max < 0 || l_max > SPH_MAX_L || (dtype != SPH_F32 && dtype != SPH_F64) ||
        (out != SPH_OUT_SAME && out != SPH_OUT_BF16) || (dtype == SPH_F64 && out == SPH_OUT_BF16)) {
        set_error("compute_host: bad n, l_max, dtype or out");
        return SPH_EINVAL;
    }
    if (n == 0) return SPH_OK;
    if (!xyz_host || !sph_host || !workspace) {
        set_error("compute_host: xyz_host, sph_host and workspace must be non-NULL");
        return SPH_EINVAL;
    }
    const size_t ein = dtype == SPH_F64 ? 8 : 4;
    const size_t eo = dtype == SPH_F64 ? 8 : (out == SPH_OUT_BF16 ? 2 : 4);
    const size_t K = size_t(l_max + 1) * (l_max + 1);
    const bool grad = dsph_host != nullptr;
    // One stage holds xyz, sph and (dsph) of `chunk` points, each 256-byte aligned.
    auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    auto stage_bytes = [&](size_t c) {
        return a256(c * 3 * ein) + a256(c * K * eo) + (grad ? a256(c * 3 * K * eo) : 0);
    };
    size_t chunk = chunk_points > 0 ? size_t(chunk_points) : size_t(1) << 20;
    chunk = std::min(chunk, size_t(n));
    chunk = (chunk + 31) / 32 * 32;
    while (chunk > 32 && kStages * stage_bytes(chunk) > workspace_bytes) chunk = (chunk / 2 + 31) / 32 * 32;
    if (kStages * stage_bytes(chunk) > workspace_bytes) {
        set_error("compute_host: workspace of %zu bytes is smaller than two 32-point stages (%zu bytes)",
                  workspace_bytes, kStages * stage_bytes(chunk));
        return SPH_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) {
        set_error("compute_host: workspace must be 256-byte aligned");
        return SPH_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kHostMaxDevices) {
        cudaGetLastError();
        set_error("compute_host: no usable CUDA device");
        return SPH_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_pipe_mu);  // one pipeline per device at a time
    HostPipe* P = nullptr;
    cudaError_t e = pipe_for(dev, &P);
    if (e != cudaSuccess) {
        set_error("compute_host: stream/event creation failed: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    const size_t sb = stage_bytes(chunk);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    e = cudaEventRecord(P->start, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->h2d, P->start, 0);
    // the stages are shared with the previous call on this device: wait for its last copy
    if (e == cudaSuccess && P->used) e = cudaStreamWaitEvent(P->h2d, P->done, 0);
    const int64_t nchunks = (n + int64_t(chunk) - 1) / int64_t(chunk);
    for (int64_t c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int b = int(c % kStages);
        const int64_t p0 = c * int64_t(chunk);
        const int64_t cnt = std::min<int64_t>(int64_t(chunk), n - p0);
        unsigned char* st = ws + size_t(b) * sb;
        void* dx = st;
        void* ds = st + a256(chunk * 3 * ein);
        void* dd = grad ? st + a256(chunk * 3 * ein) + a256(chunk * K * eo) : nullptr;
        // stage b is free once the device->host copies of chunk c - kStages finished
        if (c >= kStages) e = cudaStreamWaitEvent(P->h2d, P->free_ev[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dx, static_cast<const unsigned char*>(xyz_host) + size_t(p0) * 3 * ein,
                                size_t(cnt) * 3 * ein, cudaMemcpyHostToDevice, P->h2d);
        if (e == cudaSuccess) e = cudaEventRecord(P->h2d_ev[b], P->h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->comp, P->h2d_ev[b], 0);
        if (e == cudaSuccess) {
            const int stt = sphericart_compute_ex(dx, cnt, l_max, normalized, dtype, out, SPH_Q_NATIVE,
                                                  SPH_KERNEL_AUTO, nullptr, ds, dd, nullptr, P->comp);
            if (stt != SPH_OK) return stt;  // message already set
        }
        if (e == cudaSuccess) e = cudaEventRecord(P->comp_ev[b], P->comp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->d2h, P->comp_ev[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<unsigned char*>(sph_host) + size_t(p0) * K * eo, ds, size_t(cnt) * K * eo,
                                cudaMemcpyDeviceToHost, P->d2h);
        if (e == cudaSuccess && grad)
            e = cudaMemcpyAsync(static_cast<unsigned char*>(dsph_host) + size_t(p0) * 3 * K * eo, dd,
                                size_t(cnt) * 3 * K * eo, cudaMemcpyDeviceToHost, P->d2h);
        if (e == cudaSuccess) e = cudaEventRecord(P->free_ev[b], P->d2h);
    }
    if (e == cudaSuccess) e = cudaEventRecord(P->done, P->d2h);
    if (e == cudaSuccess) P->used = true;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, P->done, 0);
    if (e != cudaSuccess) {
        set_error("compute_host: %s", cudaGetErrorString(e));
        return SPH_ECUDA;
    }
    return SPH_OK;
}
