// Maximum flow and maximal minimum cut of the pattern network (Alg. 8) on the
// GPU, by push-relabel.
//
// Network: source s, sink t, one node per pattern (a set of 1-3 vertices: an
// edge, a loop, a triangle or the part of one), one node per vertex.  Arcs
// s -> pattern with capacity q, pattern -> each of its vertices with capacity
// q, vertex -> t with capacity p, where rho = p / q (all capacities scaled by
// q so that they are integers).  The arcs live in a CSR by tail node with the
// index of each arc's twin, built directly from the pattern lists.
//
// Algorithm: the preflow phase of push-relabel (Goldberg and Tarjan 1988) in
// its lock-free form for many threads (Hong 2008): every active node (positive
// excess, label below the node count) pushes to its lowest neighbour along a
// residual arc when its label is higher, else relabels itself to that label
// plus one; capacities and excesses change by atomic adds only.  A global
// relabel (breadth-first search from t over residual arcs) runs before every
// batch of pulses.  When no active node is left, excess(t) is the maximum flow
// value and the nodes that cannot reach t in the residual graph (the last
// search leaves them unlabelled) form the largest source side of a minimum
// cut, the cut that Lemma 9 uses.  Every loop is bounded; running out of the
// bound returns LDS_ETIMEOUT.
#include <algorithm>

#include "flow.cuh"
#include "prims.cuh"

namespace lds {

namespace {

constexpr int FBLK = 256;

__global__ void pf_vertex_count_kernel(const int64_t* pptr, const int32_t* pidx, int32_t np, int32_t* vdeg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride)
        for (int64_t k = pptr[j]; k < pptr[j + 1]; ++k) atomicAdd(vdeg + pidx[k], 1);
}

__global__ void pf_arcs_kernel(const int64_t* pptr, const int32_t* pidx, int32_t np, int32_t nv, int64_t pat_base,
                               const int64_t* vstart, int32_t* cursor, int64_t q, int32_t* head, int64_t* cap,
                               int64_t* rev) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int32_t pn = 2 + (int32_t)j;
        const int64_t a0 = pat_base + pptr[j] + j;          // first arc of pattern j
        // s -> pattern j (arc j) and its twin pattern j -> s (arc a0)
        head[j] = pn;
        cap[j] = q;
        rev[j] = a0;
        head[a0] = 0;
        cap[a0] = 0;
        rev[a0] = j;
        for (int64_t k = pptr[j]; k < pptr[j + 1]; ++k) {
            const int32_t v = pidx[k];
            const int64_t a = a0 + 1 + (k - pptr[j]);       // pattern j -> v
            const int64_t b = vstart[v] + 1 + atomicAdd(cursor + v, 1);   // v -> pattern j
            head[a] = 2 + np + v;
            cap[a] = q;
            rev[a] = b;
            head[b] = pn;
            cap[b] = 0;
            rev[b] = a;
        }
    }
}

__global__ void pf_sink_arcs_kernel(int32_t np, int32_t nv, const int64_t* vstart, int64_t p, int32_t* head,
                                    int64_t* cap, int64_t* rev) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        const int64_t a = vstart[v];                        // v -> t
        const int64_t b = np + v;                           // t -> v
        head[a] = 1;
        cap[a] = p;
        rev[a] = b;
        head[b] = 2 + np + (int32_t)v;
        cap[b] = 0;
        rev[b] = a;
    }
}

__global__ void pf_node_ptr_kernel(const int64_t* pptr, int32_t np, int32_t nv, const int64_t* vstart,
                                   int64_t pat_base, int64_t total, int64_t* nptr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t N = 2 + (int64_t)np + nv;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= N; x += stride) {
        int64_t v;
        if (x == 0) v = 0;                                   // s
        else if (x == 1) v = np;                             // t
        else if (x < 2 + np) v = pat_base + pptr[x - 2] + (x - 2);
        else if (x < N) v = vstart[x - 2 - np];
        else v = total;
        nptr[x] = v;
    }
}

__global__ void pf_init_kernel(int32_t np, int64_t q, int64_t* cap, const int64_t* rev, int64_t* excess, int64_t N) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        cap[j] = 0;                 // saturate s -> pattern
        cap[rev[j]] = q;
        excess[2 + j] = q;
    }
}

// global relabel: level-synchronous search from t over residual arcs (x -> y with cap > 0, y labelled)
__global__ void gr_level_kernel(const int64_t* nptr, const int32_t* head, const int64_t* cap, const int64_t* rev,
                                const int32_t* frontier, int32_t fsize, int32_t* label, int32_t level,
                                int32_t* next, int32_t* nsize) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < fsize; i += stride) {
        const int32_t y = frontier[i];
        for (int64_t a = nptr[y]; a < nptr[y + 1]; ++a) {
            const int32_t x = head[a];
            if (cap[rev[a]] > 0 && label[x] < 0) {
                if (atomicCAS(label + x, -1, level + 1) == -1) next[atomicAdd(nsize, 1)] = x;
            }
        }
    }
}

__global__ void gr_reset_kernel(int64_t N, int32_t* label) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride) label[x] = x == 1 ? 0 : -1;
}

__global__ void gr_apply_kernel(int64_t N, const int32_t* label, int32_t* height) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride)
        height[x] = (x == 0 || label[x] < 0) ? (int32_t)N : label[x];
}

// Values written by other blocks' atomics are read through L2 (__ldcg), never a
// possibly stale L1 line.
__global__ void pr_pulse_kernel(const int64_t* nptr, const int32_t* head, int64_t* cap, const int64_t* rev,
                                int64_t* excess, int32_t* height, int64_t N, int pulses, int32_t* active) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int32_t act = 0;
    for (int64_t x = 2 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride) {
        for (int it = 0; it < pulses; ++it) {
            int64_t e = __ldcg(excess + x);
            int32_t hx = __ldcg(height + x);
            if (e <= 0 || hx >= N) break;
            int64_t best = -1, capb = 0;
            int32_t hmin = INT32_MAX;
            for (int64_t a = nptr[x]; a < nptr[x + 1]; ++a) {
                int64_t c = __ldcg(cap + a);
                if (c > 0) {
                    int32_t hy = __ldcg(height + head[a]);
                    if (hy < hmin) {
                        hmin = hy;
                        best = a;
                        capb = c;
                    }
                }
            }
            if (best < 0) {
                height[x] = (int32_t)N;        // no residual arc: x cannot push now
                break;
            }
            if (hx > hmin) {
                // only x lowers its own arcs' capacities and its own excess, so d stays available
                int64_t d = min(e, capb);
                atomicAdd((unsigned long long*)(cap + best), (unsigned long long)(-d));
                atomicAdd((unsigned long long*)(cap + rev[best]), (unsigned long long)d);
                atomicAdd((unsigned long long*)(excess + x), (unsigned long long)(-d));
                atomicAdd((unsigned long long*)(excess + head[best]), (unsigned long long)d);
            } else {
                height[x] = hmin + 1;
            }
        }
        if (__ldcg(excess + x) > 0 && __ldcg(height + x) < N) ++act;
    }
    if (act) atomicAdd(active, act);
}

__global__ void add_one_kernel(const int32_t* in, int32_t nv, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= nv; v += stride) out[v] = v < nv ? in[v] + 1 : 0;
}

__global__ void add_offset_kernel(int64_t* p, int64_t k, int64_t off) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) p[i] += off;
}

__global__ void count_active_kernel(const int64_t* excess, const int32_t* height, int64_t N, int32_t* active) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int32_t c = 0;
    for (int64_t x = 2 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride)
        c += (excess[x] > 0 && height[x] < N);
    if (c) atomicAdd(active, c);
}

__global__ void pf_side_kernel(const int32_t* label, int32_t np, int32_t nv, uint8_t* side) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride)
        side[v] = label[2 + np + v] < 0 ? 1 : 0;
}

}  // namespace

int64_t pattern_max_flow(const int64_t* pptr, const int32_t* pidx, int32_t np, int32_t nv, int64_t p, int64_t q,
                         uint8_t* side, cudaStream_t s) {
    const int64_t N = 2 + (int64_t)np + nv;
    int64_t npidx = 0;
    if (np) LDS_CUDA(cudaMemcpyAsync(&npidx, pptr + np, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    // arcs: s: np; t: nv; patterns: np + npidx; vertices: nv + npidx
    const int64_t pat_base = np + nv;
    const int64_t vert_base = pat_base + np + npidx;
    const int64_t total = vert_base + nv + npidx;
    DevBuf<int32_t> vdeg(std::max(nv, 1) + 1, s);
    LDS_CUDA(cudaMemsetAsync(vdeg.get(), 0, (std::max(nv, 1) + 1) * sizeof(int32_t), s));
    if (np) LDS_LAUNCH(pf_vertex_count_kernel, grid_for(np, FBLK), FBLK, 0, s, pptr, pidx, np, vdeg.get());
    // vertex v's arcs start at vert_base + (v + sum of earlier degrees)
    DevBuf<int32_t> vlen(std::max(nv, 1) + 1, s);
    DevBuf<int64_t> vstart(std::max(nv, 1) + 1, s);
    LDS_LAUNCH(add_one_kernel, grid_for(nv + 1, FBLK), FBLK, 0, s, vdeg.get(), nv, vlen.get());
    exclusive_scan_i32_to_i64(vlen.get(), vstart.get(), nv + 1, s);
    LDS_LAUNCH(add_offset_kernel, grid_for(nv + 1, FBLK), FBLK, 0, s, vstart.get(), nv + 1, vert_base);
    DevBuf<int32_t> head(total, s), cursor(std::max(nv, 1), s);
    DevBuf<int64_t> cap(total, s), rev(total, s), nptr(N + 1, s), excess(N, s);
    DevBuf<int32_t> height(N, s), label(N, s), fa(N, s), fb(N, s), cnt(1, s);
    LDS_CUDA(cudaMemsetAsync(cursor.get(), 0, std::max(nv, 1) * sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(excess.get(), 0, N * sizeof(int64_t), s));
    if (np)
        LDS_LAUNCH(pf_arcs_kernel, grid_for(np, FBLK), FBLK, 0, s, pptr, pidx, np, nv, pat_base, vstart.get(),
                   cursor.get(), q, head.get(), cap.get(), rev.get());
    if (nv) LDS_LAUNCH(pf_sink_arcs_kernel, grid_for(nv, FBLK), FBLK, 0, s, np, nv, vstart.get(), p, head.get(), cap.get(), rev.get());
    LDS_LAUNCH(pf_node_ptr_kernel, grid_for(N + 1, FBLK), FBLK, 0, s, pptr, np, nv, vstart.get(), pat_base, total, nptr.get());
    if (np) LDS_LAUNCH(pf_init_kernel, grid_for(np, FBLK), FBLK, 0, s, np, q, cap.get(), rev.get(), excess.get(), N);

    auto global_relabel = [&]() {
        LDS_LAUNCH(gr_reset_kernel, grid_for(N, FBLK), FBLK, 0, s, N, label.get());
        int32_t one = 1;
        LDS_CUDA(cudaMemcpyAsync(fa.get(), &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));  // frontier = {t}
        int32_t fsize = 1, level = 0;
        int32_t* cur = fa.get();
        int32_t* nxt = fb.get();
        while (fsize > 0) {
            LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
            LDS_LAUNCH(gr_level_kernel, grid_for(fsize, FBLK), FBLK, 0, s, nptr.get(), head.get(), cap.get(), rev.get(),
                       cur, fsize, label.get(), level, nxt, cnt.get());
            LDS_CUDA(cudaMemcpyAsync(&fsize, cnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
            std::swap(cur, nxt);
            ++level;
            LDS_REQUIRE(level <= N + 1, LDS_ETIMEOUT, "max flow: global relabel did not finish");
        }
        LDS_LAUNCH(gr_apply_kernel, grid_for(N, FBLK), FBLK, 0, s, N, label.get(), height.get());
    };

    const int pulses = 16;
    int64_t rounds = 0;
    const int64_t max_rounds = 4 * N + 1000;
    while (true) {
        // exact labels, then stop when no node with excess can still reach t
        global_relabel();
        LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
        LDS_LAUNCH(count_active_kernel, grid_for(N, FBLK), FBLK, 0, s, excess.get(), height.get(), N, cnt.get());
        int32_t active = 0;
        LDS_CUDA(cudaMemcpyAsync(&active, cnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        if (active == 0) break;
        LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
        LDS_LAUNCH(pr_pulse_kernel, grid_for(N, FBLK), FBLK, 0, s, nptr.get(), head.get(), cap.get(), rev.get(),
                   excess.get(), height.get(), N, pulses, cnt.get());
        LDS_REQUIRE(++rounds < max_rounds, LDS_ETIMEOUT, "max flow: push-relabel did not finish");
    }
    // the labels of the last search tell which nodes still reach t
    int64_t flow = 0;
    LDS_CUDA(cudaMemcpyAsync(&flow, excess.get() + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (side && nv) LDS_LAUNCH(pf_side_kernel, grid_for(nv, FBLK), FBLK, 0, s, label.get(), np, nv, side);
    LDS_CUDA(cudaStreamSynchronize(s));
    return flow;
}

}  // namespace lds

using namespace lds;

extern "C" lds_status lds_pattern_max_flow(int32_t nv, int32_t np, const int64_t* pat_ptr, const int32_t* pat_idx,
                                           int64_t p, int64_t q, int64_t* flow, uint8_t* source_side) {
    return guard([&] {
        LDS_REQUIRE(nv >= 0 && np >= 0 && p >= 0 && q > 0, LDS_EINVAL, "lds_pattern_max_flow: bad sizes or capacities");
        LDS_REQUIRE(flow && (np == 0 || (pat_ptr && pat_idx)), LDS_EINVAL, "lds_pattern_max_flow: NULL argument");
        LDS_REQUIRE(lds_device_count() > 0, LDS_ECUDA, "lds_pattern_max_flow: no CUDA device");
        for (int32_t j = 0; j < np; ++j)
            LDS_REQUIRE(pat_ptr[j + 1] >= pat_ptr[j], LDS_EINVAL, "lds_pattern_max_flow: pat_ptr not ascending");
        const int64_t k = np ? pat_ptr[np] : 0;
        for (int64_t i = 0; i < k; ++i)
            LDS_REQUIRE(pat_idx[i] >= 0 && pat_idx[i] < nv, LDS_EINVAL, "lds_pattern_max_flow: vertex index out of range");
        cudaStream_t s = nullptr;
        DevBuf<int64_t> dp(np + 1, s);
        DevBuf<int32_t> di(std::max<int64_t>(k, 1), s);
        DevBuf<uint8_t> side(std::max(nv, 1), s);
        if (np) copy_in(dp.get(), pat_ptr, LDS_MEM_HOST, (np + 1) * sizeof(int64_t), s);
        else LDS_CUDA(cudaMemsetAsync(dp.get(), 0, sizeof(int64_t), s));
        if (k) copy_in(di.get(), pat_idx, LDS_MEM_HOST, k * sizeof(int32_t), s);
        *flow = pattern_max_flow(dp.get(), di.get(), np, nv, p, q, side.get(), s);
        if (source_side && nv) {
            copy_out(source_side, LDS_MEM_HOST, side.get(), nv, s);
            LDS_CUDA(cudaStreamSynchronize(s));
        }
    });
}
