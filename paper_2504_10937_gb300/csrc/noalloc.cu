// lds_fw_exact_noalloc: the exact Frank-Wolfe iteration for edge density
// without any device allocation.
//
// Some callers cannot allocate device memory themselves: a host framework
// that owns the whole device heap and forbids allocations from plugins, a
// latency-critical loop that cannot afford the implicit synchronisation of
// cudaMalloc / cudaFree, or a memory budget that must be fixed when the
// process starts.  This entry point serves them: the caller passes the edge
// list and the output buffers, and the only scratch memory (one counter per
// vertex plus an error word) is a file-scope device array of fixed size that
// every GPU loading this library holds until the process exits.
//
// Limits and behaviour (also in include/lds.h):
//   * at most LDS_NOALLOC_MAX_VERTICES vertices; larger n is rejected;
//   * on each device, the first call resolves the array's device address with
//     cudaGetSymbolAddress while that device is current; that first call
//     should come before any stream capture.  The address is kept per device
//     ordinal for the life of the process, which assumes the device's primary
//     context lives as long: after cudaDeviceReset, or with another context
//     current on the same ordinal, the kept address is stale;
//   * every call on a device shares the array and leaves its last contents in
//     it; each call clears the part it uses first, so calls that overlap on the
//     GPU (different streams, concurrent host threads) race and must not be
//     issued.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int32_t kMaxVertices = LDS_NOALLOC_MAX_VERTICES;
constexpr int32_t kErrorWord = kMaxVertices;     // index of the error word

// counters for every vertex, then the error word (and padding)
static __device__ __align__(256) int32_t g_noalloc_scratch[kMaxVertices + 64];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set up once per device).
int32_t* scratch_for_current_device() {
    int dev = 0;
    LDS_CUDA(cudaGetDevice(&dev));
    LDS_REQUIRE(dev >= 0 && dev < kMaxDevices, LDS_ECUDA, "lds_fw_exact_noalloc: device ordinal %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        LDS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = static_cast<int32_t*>(p);
    }
    return g_scratch_ptr[dev];
}

__global__ void noalloc_clear_kernel(int32_t* scratch, int64_t* R, int32_t n) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        scratch[x] = 0;
        R[x] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) scratch[kErrorWord] = 0;
}

// R_x = deg(x) (alpha = 1/2 scaled by D_0 = 2), W_e = 1; flags ids that are out
// of range or not ordered u < v, and edges that are not strictly after the
// previous one in (u, v) order (a repeat or an unsorted list).
__global__ void noalloc_init_kernel(const int32_t* u, const int32_t* v, int64_t m, int32_t n, int64_t* R, int64_t* W,
                                    int32_t* scratch) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int32_t a = u[e], b = v[e];
        const bool ordered = e == 0 || u[e - 1] < a || (u[e - 1] == a && v[e - 1] < b);
        if (a < 0 || b >= n || a >= b || !ordered) {
            atomicOr(scratch + kErrorWord, 1);
            continue;
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(R + a), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(R + b), 1ull);
        W[e] = 1;
    }
}

// Iteration i: edge (u, v) goes to u iff R_u < R_v (ties to v, the larger id);
// W += 2(i+1) when u receives; the receiver's counter grows by one.
__global__ void noalloc_pass_kernel(const int32_t* u, const int32_t* v, int64_t m, const int64_t* R, int64_t* W,
                                    int64_t inc, int32_t* scratch) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int32_t a = u[e], b = v[e];
        bool to_u = R[a] < R[b];
        if (to_u) W[e] += inc;
        atomicAdd(scratch + (to_u ? a : b), 1);
    }
}

__global__ void noalloc_update_kernel(int64_t* R, int32_t n, int64_t inc, int32_t* scratch) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        int32_t c = scratch[x];
        if (c) {
            R[x] += inc * (int64_t)c;
            scratch[x] = 0;
        }
    }
}

}  // namespace

using namespace lds;

extern "C" lds_status lds_fw_exact_noalloc(int32_t n, int64_t m, const int32_t* u, const int32_t* v, int32_t iters,
                                           int64_t* R, int64_t* W, void* stream) {
    return guard([&] {
        LDS_REQUIRE(n >= 0 && m >= 0 && iters >= 0, LDS_EINVAL, "lds_fw_exact_noalloc: negative size or iters");
        LDS_REQUIRE(n <= kMaxVertices, LDS_EINVAL,
                    "lds_fw_exact_noalloc: n = %d exceeds the fixed scratch limit of %d vertices", n, kMaxVertices);
        LDS_REQUIRE(iters <= 60000, LDS_EINVAL, "lds_fw_exact_noalloc: iters = %d out of range", iters);
        LDS_REQUIRE(m == 0 || (u && v && W), LDS_EINVAL, "lds_fw_exact_noalloc: NULL edge or weight pointer");
        LDS_REQUIRE(n == 0 || R, LDS_EINVAL, "lds_fw_exact_noalloc: NULL load pointer");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int32_t* scratch = scratch_for_current_device();
        const int blk = 256;
        LDS_LAUNCH(noalloc_clear_kernel, grid_for(std::max(n, 1), blk), blk, 0, s, scratch, R, n);
        if (m) LDS_LAUNCH(noalloc_init_kernel, grid_for(m, blk), blk, 0, s, u, v, m, n, R, W, scratch);
        int32_t bad = 0;
        LDS_CUDA(cudaMemcpyAsync(&bad, scratch + kErrorWord, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        LDS_REQUIRE(!bad, LDS_EINVAL,
                    "lds_fw_exact_noalloc: edges must satisfy 0 <= u < v < n and be distinct and sorted by (u, v)");
        for (int32_t i = 1; i <= iters && m; ++i) {
            const int64_t inc = 2 * (int64_t)(i + 1);
            LDS_LAUNCH(noalloc_pass_kernel, grid_for(m, blk), blk, 0, s, u, v, m, R, W, inc, scratch);
            LDS_LAUNCH(noalloc_update_kernel, grid_for(std::max(n, 1), blk), blk, 0, s, R, n, inc, scratch);
        }
        LDS_CUDA(cudaStreamSynchronize(s));
    });
}
