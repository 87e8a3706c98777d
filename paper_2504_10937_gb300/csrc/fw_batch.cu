// Frank-Wolfe (Alg. 1, edge density) for many small graphs in one persistent
// launch.
//
// One CTA of 1024 threads per SM takes graphs from a shared queue (largest
// first).  A graph whose active vertices fit in shared memory (8 bytes each:
// a 32-bit load word and a 32-bit count) runs all N iterations there: per
// iteration every edge (u, v), u < v, goes to the endpoint with the smaller
// load (ties to v, the larger id), counts are added in shared memory, then
// every load is updated: exact R <- R + 2(i+1) c, or binary32
// r <- (1 - gamma) r + gamma c with gamma = 2 / (i + 2) and each operation
// rounded on its own.  W = D_i alpha of the edge's lower endpoint grows by
// 2(i+1) whenever u takes the edge.  These are the same iterates, the same
// tie rule and the same rounding as the single-graph path, so the state left
// in each handle is identical to what lds_fw would leave: W and R = D_N r as
// exact integers, r in binary64.  Graphs that do not fit run the single-graph
// path.
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <unordered_set>
#include <vector>

#include "graph.cuh"

namespace lds {

namespace {

constexpr int FB_THREADS = 1024;                // threads per graph unless tuned
constexpr int32_t ONCHIP_MAX_V = 24576;          // 8 B of shared memory per vertex
constexpr int kOnchipSmemMax = ONCHIP_MAX_V * 8;
constexpr int kThreadChoices[] = {128, 256, 512, 1024};

// threads per graph (warps per graph x 32) chosen per size bucket: the bit
// length of the graph's active vertex count
std::mutex g_fwb_mu;
std::map<int, int> g_fwb_threads;

int fwb_bucket(int32_t nact) {
    int b = 0;
    while (nact) { ++b; nact >>= 1; }
    return b;
}

int fwb_threads_for(int bucket) {
    std::lock_guard<std::mutex> lk(g_fwb_mu);
    auto it = g_fwb_threads.find(bucket);
    return it == g_fwb_threads.end() ? FB_THREADS : it->second;
}

struct GraphJob {
    const int32_t* eu;
    const int32_t* ev;
    const int64_t* rowptr;
    int64_t m;
    int32_t nact, n;
    uint32_t* wt;       // [m] working W (32 bits)
    int64_t* W;         // [m] out: W per canonical edge
    int64_t* R;         // [n] out: exact loads
    double* r;          // [n] out: reported loads
};

// ---- one mid-size graph on a thread-block cluster.  Every CTA of the cluster
// keeps all load words in its shared memory and takes 1/CL_SIZE of the edges;
// each counts its edges' receipts in its own shared memory.  After the pass,
// CTA c owns the vertex slice c: it sums the slice's counts over the cluster's
// shared memories (distributed shared memory), computes the new loads and
// writes them into every CTA's copy.  Three cluster barriers per iteration
// (after the pass, after the reads of the counts, after the broadcast) replace
// grid-wide barriers.  Same iterates, ties and rounding as lds_fw.
constexpr int CL_SIZE = 8;
constexpr int CL_THREADS = 1024;
constexpr int CL_SLICE = 4;       // vertices of the slice per thread (24,576 / 8 / 1,024 = 3)
// 8 SMs against 152: past this many edges the grid-wide cooperative form wins
// (measured at 500 iterations: 2.5 against 3.3 ms at 32k edges, 4.4 against
// 4.3 ms at 64k, 12.7 against 5.1 ms at 348k)
constexpr int64_t kClusterMaxEdges = 49152;

template <bool FP32>
__global__ void __launch_bounds__(CL_THREADS, 1) fw_cluster_kernel(GraphJob g, int32_t N, uint8_t* last) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) uint32_t sm[];
    const int32_t nv = g.nact;
    uint32_t* L = sm;          // load words: R, or the bits of r in binary32
    uint32_t* C = sm + nv;     // this CTA's counts
    const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
    const int tid = threadIdx.x, bd = blockDim.x;
    const int64_t e0 = g.m * rank / cs, e1 = g.m * (rank + 1) / cs;
    const int32_t v0 = (int32_t)((int64_t)nv * rank / cs), v1 = (int32_t)((int64_t)nv * (rank + 1) / cs);
    for (int32_t x = tid; x < nv; x += bd) {
        const uint32_t d = (uint32_t)(g.rowptr[x + 1] - g.rowptr[x]);
        L[x] = FP32 ? __float_as_uint(__fmul_rn((float)d, 0.5f)) : d;     // r0 = deg / 2, R0 = D_0 r0 = deg
        C[x] = 0;
    }
    for (int64_t e = e0 + tid; e < e1; e += bd) g.wt[e] = 1u;             // W0 = D_0 / 2
    cl.sync();
    for (int32_t i = 1; i <= N; ++i) {
        const uint32_t inc = 2u * (uint32_t)(i + 1);
        for (int64_t e = e0 + tid; e < e1; e += bd) {
            const int32_t u = g.eu[e], v = g.ev[e];
            const uint32_t lu = L[u], lv = L[v];
            const bool to_u = FP32 ? (__uint_as_float(lu) < __uint_as_float(lv)) : (lu < lv);
            atomicAdd(C + (to_u ? u : v), 1u);
            if (to_u) g.wt[e] += inc;
            if (last && i == N) last[e] = to_u ? 1 : 0;
        }
        cl.sync();
        uint32_t nl[CL_SLICE];
        {
            int j = 0;
            for (int32_t x = v0 + tid; x < v1; x += bd, ++j) {
                uint32_t c = 0;
                for (unsigned r = 0; r < cs; ++r) c += cl.map_shared_rank(C, r)[x];
                if (FP32) {
                    const float gam = __fdiv_rn(2.0f, (float)(i + 2));
                    const float om = __fsub_rn(1.0f, gam);
                    nl[j] = __float_as_uint(__fadd_rn(__fmul_rn(om, __uint_as_float(L[x])), __fmul_rn(gam, (float)c)));
                } else {
                    nl[j] = L[x] + inc * c;
                }
            }
        }
        cl.sync();                               // every CTA has read the counts of its slice
        for (int32_t x = tid; x < nv; x += bd) C[x] = 0;
        {
            int j = 0;
            for (int32_t x = v0 + tid; x < v1; x += bd, ++j)
                for (unsigned r = 0; r < cs; ++r) cl.map_shared_rank(L, r)[x] = nl[j];
        }
        cl.sync();
    }
    // outputs: W, R = the incident shares of W (D_N - W for the upper endpoint), r
    const uint32_t D = (uint32_t)(N + 1) * (uint32_t)(N + 2);
    for (int64_t e = e0 + tid; e < e1; e += bd) {
        const uint32_t w = g.wt[e];
        g.W[e] = (int64_t)w;
        atomicAdd(C + g.eu[e], w);
        atomicAdd(C + g.ev[e], D - w);
    }
    cl.sync();
    for (int32_t x = v0 + tid; x < v1; x += bd) {
        uint32_t c = 0;
        for (unsigned r = 0; r < cs; ++r) c += cl.map_shared_rank(C, r)[x];
        g.R[x] = (int64_t)c;
        g.r[x] = FP32 ? (double)__uint_as_float(L[x]) : (double)L[x] / (double)D;
    }
    if (rank == 0)
        for (int32_t x = nv + tid; x < g.n; x += bd) {
            g.R[x] = 0;
            g.r[x] = 0.0;
        }
    cl.sync();                                   // no CTA leaves while others read its counts
}

template <bool FP32>
__global__ void __launch_bounds__(FB_THREADS)
    fw_batch_kernel(const GraphJob* __restrict__ jobs, int32_t njobs, int32_t* next, int32_t N) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ int32_t job;
    const int tid = threadIdx.x, bd = blockDim.x;
    for (;;) {
        if (tid == 0) job = atomicAdd(next, 1);
        __syncthreads();
        const int32_t j = job;
        __syncthreads();
        if (j >= njobs) return;
        const GraphJob g = jobs[j];
        const int32_t nv = g.nact;
        uint32_t* L = sm;          // load words: R, or the bits of r in binary32
        uint32_t* C = sm + nv;     // counts
        for (int32_t x = tid; x < nv; x += bd) {
            const uint32_t d = (uint32_t)(g.rowptr[x + 1] - g.rowptr[x]);
            L[x] = FP32 ? __float_as_uint(__fmul_rn((float)d, 0.5f)) : d;     // r0 = deg / 2, R0 = D_0 r0 = deg
            C[x] = 0;
        }
        for (int64_t e = tid; e < g.m; e += bd) g.wt[e] = 1u;                // W0 = D_0 / 2
        __syncthreads();
        for (int32_t i = 1; i <= N; ++i) {
            const uint32_t inc = 2u * (uint32_t)(i + 1);
            for (int64_t e = tid; e < g.m; e += bd) {
                const int32_t u = g.eu[e], v = g.ev[e];
                const uint32_t lu = L[u], lv = L[v];
                const bool to_u = FP32 ? (__uint_as_float(lu) < __uint_as_float(lv)) : (lu < lv);
                atomicAdd(C + (to_u ? u : v), 1u);
                if (to_u) g.wt[e] += inc;
            }
            __syncthreads();
            if (FP32) {
                const float gam = 2.0f / (float)(i + 2);
                const float om = 1.0f - gam;
                for (int32_t x = tid; x < nv; x += bd) {
                    const uint32_t c = C[x];
                    L[x] = __float_as_uint(__fadd_rn(__fmul_rn(om, __uint_as_float(L[x])), __fmul_rn(gam, (float)c)));
                    C[x] = 0;
                }
            } else {
                for (int32_t x = tid; x < nv; x += bd) {
                    const uint32_t c = C[x];
                    if (c) {
                        L[x] += inc * c;
                        C[x] = 0;
                    }
                }
            }
            __syncthreads();
        }
        // outputs: W, R = the incident shares of W (D_N - W for the upper endpoint), r
        const uint32_t D = (uint32_t)(N + 1) * (uint32_t)(N + 2);
        for (int64_t e = tid; e < g.m; e += bd) {
            const uint32_t w = g.wt[e];
            g.W[e] = (int64_t)w;
            atomicAdd(C + g.eu[e], w);
            atomicAdd(C + g.ev[e], D - w);
        }
        __syncthreads();
        for (int32_t x = tid; x < g.n; x += bd) {
            if (x < nv) {
                g.R[x] = (int64_t)C[x];
                g.r[x] = FP32 ? (double)__uint_as_float(L[x]) : (double)L[x] / (double)D;
            } else {
                g.R[x] = 0;
                g.r[x] = 0.0;
            }
        }
        __syncthreads();
    }
}

void launch_bucket(const GraphJob* jobs, int32_t njobs, int32_t* next, int32_t maxv, int threads, bool fp32,
                   int32_t iters, cudaStream_t s) {
    const size_t smem = (size_t)maxv * 8;
    int per_sm = 0;
    // the limit is the largest any launch asks for: a per-launch value could be
    // lowered by another thread between its setting and this launch
    if (fp32) {
        LDS_CUDA(cudaFuncSetAttribute(fw_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOnchipSmemMax));
        LDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_batch_kernel<true>, threads, smem));
    } else {
        LDS_CUDA(cudaFuncSetAttribute(fw_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOnchipSmemMax));
        LDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_batch_kernel<false>, threads, smem));
    }
    const int grid = std::max(1, std::min(num_sms() * std::max(per_sm, 1), (int)njobs));
    if (fp32) LDS_LAUNCH(fw_batch_kernel<true>, grid, threads, smem, s, jobs, njobs, next, iters);
    else LDS_LAUNCH(fw_batch_kernel<false>, grid, threads, smem, s, jobs, njobs, next, iters);
}

bool fits_on_chip(const lds_graph* g, int32_t N, lds_precision p);

}  // namespace

// Runs lds_fw's edge-density iterations of g on one cluster when its active
// vertices fit in shared memory (exact or binary32); fills the handle's R, r, W
// and, when `last` is given, the last iteration's choices.  False when the graph
// does not fit or no cluster of CL_SIZE CTAs can be resident.
bool fw_cluster_run(lds_graph* g, int32_t N, lds_precision p, uint8_t* last, bool any_size) {
    static_assert(ONCHIP_MAX_V / CL_SIZE <= CL_SLICE * CL_THREADS, "a CTA's vertex slice exceeds its registers");
    if (!fits_on_chip(g, N, p) || (!any_size && g->m > kClusterMaxEdges)) return false;
    cudaStream_t s = g->stream;
    const bool fp32 = p == LDS_FP32;
    const size_t smem = (size_t)std::max(g->nact, 1) * 8;
    const void* fn = fp32 ? (const void*)fw_cluster_kernel<true> : (const void*)fw_cluster_kernel<false>;
    LDS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kOnchipSmemMax));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL_SIZE);
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL_SIZE;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return false;
    }
    DevBuf<uint32_t> wt(std::max<int64_t>(g->m, 1), s);
    g->fw_W.alloc(std::max<int64_t>(g->m, 1), s);
    GraphJob job{g->eu.get(), g->ev.get(), g->rowptr.get(), g->m, g->nact, g->n, wt.get(), g->fw_W.get(),
                 g->fw_R.get(), g->fw_r.get()};
    int32_t iters = N;
    void* args[] = {(void*)&job, (void*)&iters, (void*)&last};
    LDS_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return true;
}

namespace {

bool fits_on_chip(const lds_graph* g, int32_t N, lds_precision p) {
    if (p != LDS_EXACT && p != LDS_FP32) return false;
    if (N < 1 || g->m < 1 || g->nact > ONCHIP_MAX_V) return false;
    const unsigned __int128 D = (unsigned __int128)(N + 1) * (unsigned __int128)(N + 2);
    // every load and every share sum must fit 32 bits
    return (unsigned __int128)std::max(g->info.max_degree, 1) * D < ((unsigned __int128)1 << 32);
}

}  // namespace

}  // namespace lds

using namespace lds;

namespace lds {

// lds_fw_batch's body; force_threads > 0 overrides the tuned threads per graph
void fw_batch_run(int32_t count, lds_graph** graphs, int32_t iters, lds_precision p, int32_t* onchip,
                  int force_threads) {
    {
        LDS_REQUIRE(count >= 0 && (count == 0 || graphs), LDS_EINVAL, "lds_fw_batch: bad graph list");
        LDS_REQUIRE(iters >= 0 && iters <= 60000, LDS_EINVAL, "lds_fw_batch: iters = %d out of range", iters);
        LDS_REQUIRE(p == LDS_EXACT || p == LDS_FP32 || p == LDS_FP64, LDS_EINVAL, "lds_fw_batch: bad precision");
        std::unordered_set<const lds_graph*> seen;
        for (int32_t i = 0; i < count; ++i) {
            LDS_REQUIRE(graphs[i], LDS_EINVAL, "lds_fw_batch: graph %d is NULL", i);
            LDS_REQUIRE(seen.insert(graphs[i]).second, LDS_EINVAL, "lds_fw_batch: graph %d appears twice", i);
        }
        if (onchip) *onchip = 0;
        std::vector<lds_graph*> on, off;
        for (int32_t i = 0; i < count; ++i) (fits_on_chip(graphs[i], iters, p) ? on : off).push_back(graphs[i]);
        // the rest run the single-graph path
        for (lds_graph* g : off) {
            fw_run(g, LDS_EDGE, iters, p, false);
            g->fw_reuse = true;
        }
        if (on.empty()) return;
        // size buckets contiguous (largest first), largest graphs first inside a bucket
        std::sort(on.begin(), on.end(), [](const lds_graph* a, const lds_graph* b) {
            const int ba = fwb_bucket(a->nact), bb = fwb_bucket(b->nact);
            return ba != bb ? ba > bb : a->m > b->m;
        });
        // each handle's buffers are allocated on its own stream, then everything runs on the first one
        int64_t total_m = 0;
        for (lds_graph* g : on) total_m += g->m;
        cudaStream_t s = on.front()->stream;
        DevBuf<uint32_t> wt(total_m, s);
        std::vector<GraphJob> jobs;
        int64_t off_m = 0;
        int32_t maxv = 1;
        for (lds_graph* g : on) {
            cudaStream_t gs = g->stream;
            LDS_CUDA(cudaStreamSynchronize(gs));
            g->fw_valid = false;
            g->fw_last.release();
            g->fw_R.alloc(std::max(g->n, 1), gs);
            g->fw_r.alloc(std::max(g->n, 1), gs);
            g->fw_W.alloc(std::max<int64_t>(g->m, 1), gs);
            LDS_CUDA(cudaStreamSynchronize(gs));
            jobs.push_back(GraphJob{g->eu.get(), g->ev.get(), g->rowptr.get(), g->m, g->nact, g->n,
                                   wt.get() + off_m, g->fw_W.get(), g->fw_R.get(), g->fw_r.get()});
            off_m += g->m;
            maxv = std::max(maxv, g->nact);
        }
        (void)maxv;
        DevBuf<GraphJob> djobs(jobs.size(), s);
        DevBuf<int32_t> next(64, s);
        LDS_CUDA(cudaMemcpyAsync(djobs.get(), jobs.data(), jobs.size() * sizeof(GraphJob), cudaMemcpyHostToDevice, s));
        LDS_CUDA(cudaMemsetAsync(next.get(), 0, 64 * sizeof(int32_t), s));
        const auto t0 = std::chrono::steady_clock::now();
        // one launch per size bucket (jobs are sorted by size, so buckets are contiguous):
        // its own threads per graph and shared memory sized to its largest graph, as
        // many CTAs per SM as fit
        size_t lo = 0;
        int launch = 0;
        while (lo < on.size()) {
            const int bk = fwb_bucket(on[lo]->nact);
            size_t hi = lo;
            int32_t bmax = 1;
            while (hi < on.size() && fwb_bucket(on[hi]->nact) == bk) bmax = std::max(bmax, on[hi++]->nact);
            const int threads = force_threads > 0 ? force_threads : fwb_threads_for(bk);
            launch_bucket(djobs.get() + lo, (int32_t)(hi - lo), next.get() + (launch++ % 64), bmax, threads,
                          p == LDS_FP32, iters, s);
            lo = hi;
        }
        LDS_CUDA(cudaStreamSynchronize(s));
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        const int64_t Dn = (int64_t)(iters + 1) * (iters + 2);
        for (lds_graph* g : on) {
            g->fw_valid = true;
            g->fw_density = LDS_EDGE;
            g->fw_prec = p;
            g->fw_iters = iters;
            g->fw_D = Dn;
            g->fw_reuse = true;
            g->fw_ms = ms;
            g->pass_us = 0.0;
            g->pass_launches = 0;
            g->pass_bytes = 0;
            g->pass_kernel = "fw_batch_kernel";
        }
        if (onchip) *onchip = (int32_t)on.size();
    }
}

// Times the on-chip Frank-Wolfe of `count` graphs with every threads-per-graph
// choice, per size bucket, and keeps the fastest choice of each bucket.
void fw_batch_autotune(int32_t count, lds_graph** graphs, int32_t iters, lds_precision p) {
    std::map<int, std::vector<lds_graph*>> byb;
    for (int32_t i = 0; i < count; ++i)
        if (fits_on_chip(graphs[i], iters, p)) byb[fwb_bucket(graphs[i]->nact)].push_back(graphs[i]);
    for (auto& kv : byb) {
        {
            std::lock_guard<std::mutex> lk(g_fwb_mu);
            if (g_fwb_threads.count(kv.first)) continue;
        }
        double best = 1e300;
        int best_t = FB_THREADS;
        for (int t : kThreadChoices) {
            const auto t0 = std::chrono::steady_clock::now();
            fw_batch_run((int32_t)kv.second.size(), kv.second.data(), iters, p, nullptr, t);
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (ms < best) {
                best = ms;
                best_t = t;
            }
        }
        std::lock_guard<std::mutex> lk(g_fwb_mu);
        g_fwb_threads[kv.first] = best_t;
    }
}

int32_t fw_batch_threads(int32_t nact) { return fwb_threads_for(fwb_bucket(nact)); }

}  // namespace lds

extern "C" lds_status lds_fw_batch(int32_t count, lds_graph** graphs, int32_t iters, lds_precision p,
                                   int32_t* onchip) {
    return guard([&] { fw_batch_run(count, graphs, iters, p, onchip, 0); });
}

extern "C" int32_t lds_fw_batch_threads(int32_t nact) {
    try {
        return fw_batch_threads(nact);
    } catch (...) {
        return 0;
    }
}
