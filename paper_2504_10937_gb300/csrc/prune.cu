// Pruning (Alg. 3): Pruning rule 1 (Cor. 1) and Pruning rule 2 (Lemma 5,
// Lemma 6) on the GPU.
//
// Bounds are exact rationals num / den per vertex (den > 0); comparisons use
// 128-bit cross products.  Rule 1 marks every vertex x with an edge (x, y) such
// that ub(x) < lb(y), all decided on the bounds before any removal.  Rule 2
// then repeats: core (tr-core) numbers of G[kept], remove every kept vertex
// with core < lb, until nothing is removed.  The loop ends at the unique largest
// set in which every vertex's core number reaches its lower bound (core numbers
// only grow with the graph), whatever the removal order, so removing all
// violators of a round at once is the same as Alg. 3's one-at-a-time loop.
#include <cstdio>
#include <cstdlib>

#include "prune.cuh"

namespace lds {

namespace {

typedef __int128 i128;

__device__ __forceinline__ bool frac_lt(int64_t a, int64_t b, int64_t c, int64_t d) {
    return (i128)a * (i128)d < (i128)c * (i128)b;
}

__global__ void rule1_kernel(const int32_t* eu, const int32_t* ev, int64_t m, const int64_t* ubn, const int64_t* ubd,
                             const int64_t* lbn, const int64_t* lbd, uint8_t* status) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int32_t a = eu[e], b = ev[e];
        if (frac_lt(ubn[a], ubd[a], lbn[b], lbd[b])) status[a] = 1;
        if (frac_lt(ubn[b], ubd[b], lbn[a], lbd[a])) status[b] = 1;
    }
}

__global__ void kept_mask_kernel(const uint8_t* status, int32_t n, uint8_t* kept) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) kept[x] = status[x] == 0;
}

// kept vertices whose core number is below the lower bound are removed (status 2)
__global__ void rule2_kernel(const int64_t* core, int32_t nact, int32_t n, const int64_t* lbn, const int64_t* lbd,
                             uint8_t* status, int32_t* removed) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int32_t c = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        if (status[x]) continue;
        int64_t k = x < nact ? core[x] : 0;             // isolated vertices have core number 0
        if ((i128)k * (i128)lbd[x] < (i128)lbn[x]) {
            status[x] = 2;
            ++c;
        }
    }
    if (c) atomicAdd(removed, c);
}

__global__ void gather_orig_i64_kernel(const int64_t* in_orig, const int32_t* to_orig, int32_t n, int64_t* out_int) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) out_int[x] = in_orig[to_orig[x]];
}
__global__ void scatter_orig_u8_kernel(const uint8_t* in_int, const int32_t* to_orig, int32_t n, uint8_t* out_orig) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) out_orig[to_orig[x]] = in_int[x];
}
}  // namespace

void prune(lds_graph* g, bool tri, const int64_t* ubn, const int64_t* ubd, const int64_t* lbn, const int64_t* lbd,
           uint8_t* status) {
    cudaStream_t s = g->stream;
    const int blk = 256;
    const int32_t n = g->n, nact = g->nact;
    if (n == 0) return;
    LDS_CUDA(cudaMemsetAsync(status, 0, n, s));
    if (g->m) LDS_LAUNCH(rule1_kernel, grid_for(g->m, blk), blk, 0, s, g->eu.get(), g->ev.get(), g->m, ubn, ubd, lbn, lbd, status);
    DevBuf<uint8_t> kept(n, s);
    DevBuf<int64_t> core(std::max(nact, 1), s);
    DevBuf<int32_t> removed(1, s);
    for (int round = 0;; ++round) {
        LDS_LAUNCH(kept_mask_kernel, grid_for(n, blk), blk, 0, s, status, n, kept.get());
        core_numbers(g, tri, core.get(), kept.get());
        LDS_CUDA(cudaMemsetAsync(removed.get(), 0, sizeof(int32_t), s));
        LDS_LAUNCH(rule2_kernel, grid_for(n, blk), blk, 0, s, core.get(), nact, n, lbn, lbd, status, removed.get());
        int32_t hr = 0;
        LDS_CUDA(cudaMemcpyAsync(&hr, removed.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        const char* vb = getenv("LDS_VERBOSE");
        if (vb && vb[0] == '1') fprintf(stderr, "[prune] n=%d round %d removed %d\n", n, round, hr);
        if (hr == 0) break;
        LDS_REQUIRE(round < n + 1, LDS_ETIMEOUT, "prune: rule 2 did not settle");
    }
}

}  // namespace lds

using namespace lds;

extern "C" lds_status lds_prune(lds_graph* g, lds_density d, const int64_t* ub_num, const int64_t* ub_den,
                                const int64_t* lb_num, const int64_t* lb_den, uint8_t* status) {
    return guard([&] {
        LDS_REQUIRE(g && ub_num && ub_den && lb_num && lb_den && status, LDS_EINVAL, "lds_prune: NULL argument");
        LDS_REQUIRE(d == LDS_EDGE || d == LDS_TRIANGLE, LDS_EINVAL, "lds_prune: bad density");
        const int32_t n = g->n;
        if (n == 0) return;
        for (int32_t x = 0; x < n; ++x)
            LDS_REQUIRE(ub_den[x] > 0 && lb_den[x] > 0, LDS_EINVAL, "lds_prune: bound denominators must be positive");
        cudaStream_t s = g->stream;
        const int blk = 256;
        DevBuf<int64_t> h[4];
        const int64_t* src[4] = {ub_num, ub_den, lb_num, lb_den};
        DevBuf<int64_t> dv[4];
        for (int k = 0; k < 4; ++k) {
            h[k].alloc(n, s);
            dv[k].alloc(n, s);
            copy_in(h[k].get(), src[k], LDS_MEM_HOST, n * sizeof(int64_t), s);
            LDS_LAUNCH(gather_orig_i64_kernel, grid_for(n, blk), blk, 0, s, h[k].get(), g->to_orig.get(), n, dv[k].get());
        }
        DevBuf<uint8_t> st(n, s), so(n, s);
        prune(g, d == LDS_TRIANGLE, dv[0].get(), dv[1].get(), dv[2].get(), dv[3].get(), st.get());
        LDS_LAUNCH(scatter_orig_u8_kernel, grid_for(n, blk), blk, 0, s, st.get(), g->to_orig.get(), n, so.get());
        copy_out(status, LDS_MEM_HOST, so.get(), n, s);
        LDS_CUDA(cudaStreamSynchronize(s));
    });
}
