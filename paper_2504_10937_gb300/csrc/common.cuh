// Shared definitions for the liblds CUDA sources: status handling, device
// memory, launch geometry.  Host code never throws across the C-ABI; every
// entry point converts failures into an lds_status plus a thread-local message.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "lds.h"

namespace lds {

// ---------------------------------------------------------------- errors

void set_error(const char* fmt, ...);
const char* last_error();

struct Error {
    lds_status st;
};

#define LDS_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e__ = (call);                                                   \
        if (e__ != cudaSuccess) {                                                   \
            ::lds::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call,            \
                             cudaGetErrorString(e__));                              \
            throw ::lds::Error{e__ == cudaErrorMemoryAllocation ? LDS_ENOMEM        \
                                                                : LDS_ECUDA};       \
        }                                                                           \
    } while (0)

#define LDS_CHECK_LAUNCH() LDS_CUDA(cudaGetLastError())

// Number of kernels this library has launched since it was loaded.
extern std::atomic<long long> g_launches;

// Launch, check, count.  Every kernel of the library goes through this macro.
#define LDS_LAUNCH(kernel, grid, block, smem, stream, ...)                          \
    do {                                                                            \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                 \
        LDS_CHECK_LAUNCH();                                                         \
        ::lds::g_launches.fetch_add(1, std::memory_order_relaxed);                  \
    } while (0)

#define LDS_REQUIRE(cond, status, ...)                                              \
    do {                                                                            \
        if (!(cond)) {                                                              \
            ::lds::set_error(__VA_ARGS__);                                          \
            throw ::lds::Error{status};                                             \
        }                                                                           \
    } while (0)

// Wraps an entry point body: returns LDS_OK or the status of the first failure.
template <class F>
lds_status guard(F&& f) {
    try {
        f();
        return LDS_OK;
    } catch (const Error& e) {
        return e.st;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LDS_ENOMEM;
    } catch (...) {
        set_error("unexpected host exception");
        return LDS_ECUDA;
    }
}

// ---------------------------------------------------------------- memory

// Test hook: when > 0, the n-th device allocation from now fails (host-side
// fault injection for the LDS_ENOMEM path).
extern int g_fail_alloc_countdown;

void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// RAII device buffer allocated stream-ordered.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(size_t count, cudaStream_t stream) { alloc(count, stream); }
    void alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        p = count ? static_cast<T*>(dev_alloc(count * sizeof(T), stream)) : nullptr;
    }
    void release() {
        if (p) dev_free(p, s);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    T* get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// ---------------------------------------------------------------- launch

int num_sms();

inline unsigned grid_for(int64_t work, int block, int per_thread = 1) {
    int64_t g = (work + (int64_t)block * per_thread - 1) / ((int64_t)block * per_thread);
    if (g < 1) g = 1;
    int64_t cap = (int64_t)num_sms() * 32;
    return (unsigned)(g < cap ? g : cap);
}

inline unsigned grid_exact(int64_t work, int block) {
    int64_t g = (work + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

// Copy helpers between host / device buffers described by lds_mem.
void copy_out(void* dst, lds_mem where, const void* src_dev, size_t bytes, cudaStream_t s);
void copy_in(void* dst_dev, const void* src, lds_mem where, size_t bytes, cudaStream_t s);

inline int bit_length_u64(uint64_t x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

}  // namespace lds
