// Error reporting, device memory and copy helpers shared by the liblds sources.
#include <cstdarg>
#include <mutex>

#include "common.cuh"

namespace lds {

namespace {
thread_local std::string t_last_error;
}

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
}

const char* last_error() { return t_last_error.c_str(); }

int g_fail_alloc_countdown = 0;
std::atomic<long long> g_launches{0};

void* dev_alloc(size_t bytes, cudaStream_t s) {
    if (g_fail_alloc_countdown > 0) {
        if (--g_fail_alloc_countdown == 0) {
            set_error("device allocation of %zu bytes failed (injected)", bytes);
            throw Error{LDS_ENOMEM};
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        throw Error{e == cudaErrorMemoryAllocation ? LDS_ENOMEM : LDS_ECUDA};
    }
    return p;
}

void dev_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int num_sms() {
    static int sms = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 132;
        sms = v;
    });
    return sms;
}

void copy_out(void* dst, lds_mem where, const void* src_dev, size_t bytes, cudaStream_t s) {
    if (!bytes || !dst) return;
    LDS_CUDA(cudaMemcpyAsync(dst, src_dev, bytes,
                             where == LDS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
}

void copy_in(void* dst_dev, const void* src, lds_mem where, size_t bytes, cudaStream_t s) {
    if (!bytes) return;
    LDS_CUDA(cudaMemcpyAsync(dst_dev, src, bytes,
                             where == LDS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
}

}  // namespace lds

extern "C" {

const char* lds_version(void) { return "liblds 0.1 (sm_103a)"; }

const char* lds_last_error(void) { return lds::last_error(); }

int32_t lds_device_count(void) {
    int c = 0;
    if (cudaGetDeviceCount(&c) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return c;
}

int64_t lds_launch_count(void) { return (int64_t)lds::g_launches.load(); }

void lds_debug_fail_alloc_after(int32_t k) { lds::g_fail_alloc_countdown = k > 0 ? k : 0; }

}  // extern "C"
