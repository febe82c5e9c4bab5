// host.h -- host-side helpers shared by the C ABI translation units: error
// recording (thread-local last error), CUDA call checks, launch context.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace hp {

extern thread_local std::string g_last_error;

inline hpeel_status fail(hpeel_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
inline hpeel_status fail(hpeel_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define HP_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::hp::fail(HPEEL_ERR_CUDA, "%s failed: %s (%s:%d)", #call,               \
                              cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

#define HP_TRY(expr)                                                                        \
    do {                                                                                    \
        hpeel_status s_ = (expr);                                                           \
        if (s_ != HPEEL_OK) return s_;                                                      \
    } while (0)

inline hpeel_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(HPEEL_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return HPEEL_OK;
}

// Per-device properties the launches need (cached).
struct DeviceInfo {
    int sms = 0;
    int smem_per_sm = 0;     // bytes
    int smem_optin = 0;      // largest dynamic shared memory of one block
};

inline hpeel_status device_info(int dev, DeviceInfo *out) {
    static std::mutex mu;
    static DeviceInfo cache[64];
    if (dev < 0 || dev >= 64) return fail(HPEEL_ERR_INVALID_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev].sms == 0) {
        DeviceInfo d;
        HP_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        HP_CUDA(cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                       dev));
        HP_CUDA(cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cache[dev] = d;
    }
    *out = cache[dev];
    return HPEEL_OK;
}

inline hpeel_status make_launch(void *stream, Launch *L) {
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    DeviceInfo d;
    HP_TRY(device_info(dev, &d));
    L->sms = d.sms;
    L->stream = (cudaStream_t)stream;
    return HPEEL_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace hp
