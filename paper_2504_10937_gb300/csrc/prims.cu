// Exclusive scans and a stable LSD radix sort (see prims.cuh).
#include "prims.cuh"

namespace lds {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class In>
__device__ __forceinline__ int64_t load_as_i64(const In* p, int64_t i, int64_t n) {
    return i < n ? (int64_t)p[i] : 0;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t x, int64_t* excl) {
    constexpr int NW = SCAN_THREADS / 32;
    __shared__ int64_t warp_tot[NW];
    __shared__ int64_t block_total;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < NW ? warp_tot[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) warp_tot[lane] = wi - w;
        if (lane == NW - 1) block_total = wi;
    }
    __syncthreads();
    *excl = warp_tot[warp] + incl - x;
    int64_t t = block_total;
    __syncthreads();
    return t;
}

template <class In>
__global__ void scan_reduce_kernel(const In* in, int64_t n, int64_t* block_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) s += load_as_i64(in, base + k, n);
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, &excl);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

template <class In>
__global__ void scan_apply_kernel(const In* in, int64_t* out, int64_t n, const int64_t* block_offsets) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = load_as_i64(in, base + k, n);
        s += v[k];
    }
    int64_t excl;
    block_exclusive_scan(s, &excl);
    int64_t run = excl + (block_offsets ? block_offsets[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

template <class In>
void scan_impl(const In* in, int64_t* out, int64_t n, int64_t* total_dev, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) LDS_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
        return;
    }
    int64_t nblocks = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nblocks == 1) {
        // the total is taken before the in-place apply may overwrite the input
        if (total_dev) {
            LDS_LAUNCH(scan_reduce_kernel<In>, 1, SCAN_THREADS, 0, s, in, n, total_dev);
            LDS_CHECK_LAUNCH();
        }
        LDS_LAUNCH(scan_apply_kernel<In>, 1, SCAN_THREADS, 0, s, in, out, n, nullptr);
        LDS_CHECK_LAUNCH();
        return;
    }
    DevBuf<int64_t> sums(nblocks, s);
    LDS_LAUNCH(scan_reduce_kernel<In>, (unsigned)nblocks, SCAN_THREADS, 0, s, in, n, sums.get());
    LDS_CHECK_LAUNCH();
    DevBuf<int64_t> offs(nblocks, s);
    scan_impl<int64_t>(sums.get(), offs.get(), nblocks, total_dev, s);
    LDS_LAUNCH(scan_apply_kernel<In>, (unsigned)nblocks, SCAN_THREADS, 0, s, in, out, n, offs.get());
    LDS_CHECK_LAUNCH();
}

}  // namespace

void exclusive_scan_i64_dev(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                            cudaStream_t s) {
    scan_impl<int64_t>(in, out, n, total_dev, s);
}

int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    DevBuf<int64_t> tot(1, s);
    scan_impl<int64_t>(in, out, n, tot.get(), s);
    int64_t h = 0;
    LDS_CUDA(cudaMemcpyAsync(&h, tot.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    return h;
}

int64_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    DevBuf<int64_t> tot(1, s);
    scan_impl<int32_t>(in, out, n, tot.get(), s);
    int64_t h = 0;
    LDS_CUDA(cudaMemcpyAsync(&h, tot.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    return h;
}

// ------------------------------------------------------------------ radix sort

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;                       // keys per thread per tile
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;     // 4096 keys per tile
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void rs_histogram_kernel(const uint64_t* keys, int64_t n, int shift, int64_t ntiles,
                                    int64_t* counts) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ROUNDS; ++j) {
        int64_t i = base + (int64_t)j * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter_kernel(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                  uint32_t* vals_out, int64_t n, int shift, int64_t ntiles,
                                  const int64_t* offsets) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wcnt[RS_WARPS][256];
    __shared__ int64_t s_goff[256];
    int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    s_base[t] = 0;
    s_goff[t] = offsets[(int64_t)t * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) s_wcnt[w][t] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ROUNDS; ++j) {
        int64_t i = base + (int64_t)j * RS_THREADS + t;
        bool valid = i < n;
        uint64_t key = valid ? keys_in[i] : 0;
        uint32_t val = (valid && vals_in) ? vals_in[i] : 0;
        int d = valid ? (int)((key >> shift) & 0xFF) : 256;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) s_wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t below = 0;
            for (int w = 0; w < warp; ++w) below += s_wcnt[w][d];
            int64_t pos = s_goff[d] + s_base[d] + below + rank;
            keys_out[pos] = key;
            if (vals_out) vals_out[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            add += s_wcnt[w][t];
            s_wcnt[w][t] = 0;
        }
        s_base[t] += add;
        __syncthreads();
    }
}

__global__ void gather_u32_kernel(const uint32_t* in, const uint32_t* idx, uint32_t* out, int64_t n) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = in[idx[i]];
}

}  // namespace

void radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    int passes = (bits + 7) / 8;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    DevBuf<uint64_t> kbuf(n, s);
    DevBuf<uint32_t> vbuf;
    if (vals) vbuf.alloc(n, s);
    DevBuf<int64_t> counts(256 * ntiles, s);
    uint64_t* kin = keys;
    uint64_t* kout = kbuf.get();
    uint32_t* vin = vals;
    uint32_t* vout = vals ? vbuf.get() : nullptr;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        LDS_LAUNCH(rs_histogram_kernel, (unsigned)ntiles, RS_THREADS, 0, s, kin, n, shift, ntiles, counts.get());
        LDS_CHECK_LAUNCH();
        exclusive_scan_i64_dev(counts.get(), counts.get(), 256 * ntiles, nullptr, s);
        LDS_LAUNCH(rs_scatter_kernel, (unsigned)ntiles, RS_THREADS, 0, s, kin, vin, kout, vout, n, shift, ntiles,
                                                                counts.get());
        LDS_CHECK_LAUNCH();
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    if (kin != keys) {
        LDS_CUDA(cudaMemcpyAsync(keys, kin, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) LDS_CUDA(cudaMemcpyAsync(vals, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

void gather_u32(const uint32_t* in, const uint32_t* idx, uint32_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    LDS_LAUNCH(gather_u32_kernel, grid_for(n, 256), 256, 0, s, in, idx, out, n);
    LDS_CHECK_LAUNCH();
}

}  // namespace lds
