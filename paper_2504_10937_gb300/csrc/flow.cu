// Maximum flow and maximal minimum cut of the pattern network (Alg. 8) on the
// GPU, by push-relabel from a warm-started preflow.
//
// Network.  Alg. 8's network has a source s, a sink t, a node per pattern (a
// set of 1-3 vertices: an edge, a loop, a triangle or the part of one) and a
// node per vertex; arcs s -> pattern and pattern -> member have capacity q,
// vertex -> t has capacity p (rho = p / q).  Every capacity is multiplied by a
// power of two K (the cut structure is unchanged) so that a fractional split
// of each pattern's unit among its members can be written in integers.
//
// The preflow saturates every s -> pattern arc and splits each pattern's qK
// units among its members (in proportion to `share`, e.g. the Frank-Wolfe
// weights alpha, so that a near-optimal split leaves little excess); each
// vertex sends what it receives to t up to pK and keeps the rest as excess.
// Pattern nodes then hold no excess, and they are contracted where that is
// exact:
//   * a one-member pattern (a loop) only feeds its member: no node, no arc;
//   * a two-member pattern {a, b} with split (f_a, f_b) becomes the arc pair
//     a -> b (residual f_a) and b -> a (residual f_b): moving d units of the
//     pattern from a to b is a push along a -> b.  For a vertex set A on the
//     source side this pair adds f_a + f_b = qK to the cut exactly when one
//     member is in A and the other is not, which is what the pattern node's
//     arcs cost in Alg. 8's network, so every cut, the maximum flow and the
//     maximal minimum cut are unchanged;
//   * a pattern with three or more members keeps its node, with arcs
//     pattern -> member (residual qK - f) and member -> pattern (residual f).
// Excess that would return to s is never moved: it stays on nodes that cannot
// reach t, which is all the maximum flow and the largest source side need.
//
// Algorithm.  The preflow phase of push-relabel (Goldberg and Tarjan 1988) in
// the lock-free form for many threads (Hong 2008): an active node (positive
// excess, label below DEAD) pushes to its lowest residual neighbour when its
// label is higher, else relabels itself to that label plus one; capacities
// and excesses change by atomic adds only.  One warp serves one active node
// and scans its arcs 32 at a time (vertex nodes have hundreds of arcs).  Only
// active nodes are visited: a push that activates a node appends it to the
// next round's work list.  A global relabel (breadth-first search from t over
// residual arcs) runs first and whenever the relabels since the last one
// exceed the node count; nodes it does not reach are DEAD.  When no active
// node is left after a global relabel, the flow into t is the maximum flow and
// the DEAD vertices are the largest source side of a minimum cut (the cut that
// Lemma 9 uses).  Excess on a DEAD node can never reach t: a push into a DEAD
// node needs a label above DEAD, and valid labels of nodes that reach t stay
// below the node count.  Every loop is bounded; running out of the bound
// returns LDS_ETIMEOUT.
#include <algorithm>
#include <utility>

#include "flow.cuh"
#include "prims.cuh"

namespace lds {

namespace {

constexpr int FB = 256;
constexpr int32_t DEAD = 0x3fffffff;       // label of nodes that cannot reach t
constexpr unsigned FULL = 0xffffffffu;

typedef unsigned long long ull;
typedef __int128 i128;

struct Net {
    int32_t nv;            // vertex nodes 0..nv-1 (they alone have sink arcs)
    int32_t nn;            // all nodes (vertex nodes, then pattern nodes)
    const int64_t* ptr;    // [nn + 1] arcs of node x at ptr[x] .. ptr[x+1]
    const int32_t* head;   // [A]
    int64_t* cap;          // [A] residual capacities
    const int64_t* rev;    // [A] twin arc
    int64_t* tcap;         // [nv] residual capacity to t
    int64_t* excess;       // [nn]
    int32_t* height;       // [nn]
};

// split of every pattern's qK units among its members; big[j] = pattern j keeps a node
__global__ void split_kernel(const int64_t* pptr, int32_t np, const int64_t* share, int64_t qK, int64_t* f,
                             int32_t* big) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int64_t b = pptr[j], e = pptr[j + 1], len = e - b;
        big[j] = len >= 3;
        if (len == 0) continue;
        i128 tot = 0;
        if (share)
            for (int64_t k = b; k < e; ++k) tot += (i128)(share[k] > 0 ? share[k] : (int64_t)0);
        int64_t given = 0;
        for (int64_t k = b; k < e; ++k) {
            int64_t v;
            if (k == e - 1) v = qK - given;
            else if (tot > 0) v = (int64_t)((i128)qK * (i128)(share[k] > 0 ? share[k] : (int64_t)0) / tot);
            else v = qK / len;
            f[k] = v;
            given += v;
        }
    }
}

// node degrees and the flow each vertex receives
__global__ void degree_kernel(const int64_t* pptr, const int32_t* pidx, int32_t np, const int64_t* f,
                              const int64_t* bigpos, int32_t nv, int32_t* deg, ull* in) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int64_t b = pptr[j], e = pptr[j + 1], len = e - b;
        for (int64_t k = b; k < e; ++k) {
            atomicAdd(in + pidx[k], (ull)f[k]);
            if (len >= 2) atomicAdd(deg + pidx[k], 1);
        }
        if (len >= 3) deg[nv + bigpos[j]] = (int32_t)len;
    }
}

__global__ void fill_kernel(const int64_t* pptr, const int32_t* pidx, int32_t np, const int64_t* f,
                            const int64_t* bigpos, int32_t nv, int64_t qK, const int64_t* ptr, int32_t* cursor,
                            int32_t* head, int64_t* cap, int64_t* rev) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int64_t b = pptr[j], e = pptr[j + 1], len = e - b;
        if (len == 2) {
            const int32_t x = pidx[b], y = pidx[b + 1];
            const int64_t ax = ptr[x] + atomicAdd(cursor + x, 1);
            const int64_t ay = ptr[y] + atomicAdd(cursor + y, 1);
            head[ax] = y;
            cap[ax] = f[b];
            rev[ax] = ay;
            head[ay] = x;
            cap[ay] = f[b + 1];
            rev[ay] = ax;
        } else if (len >= 3) {
            const int32_t node = nv + (int32_t)bigpos[j];
            for (int64_t k = b; k < e; ++k) {
                const int32_t v = pidx[k];
                const int64_t ap = ptr[node] + (k - b);
                const int64_t av = ptr[v] + atomicAdd(cursor + v, 1);
                head[ap] = v;
                cap[ap] = qK - f[k];
                rev[ap] = av;
                head[av] = node;
                cap[av] = f[k];
                rev[av] = ap;
            }
        }
    }
}

__global__ void init_kernel(Net net, const ull* in, int64_t pK, ull* flow_t) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    ull acc = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < net.nn; x += stride) {
        if (x < net.nv) {
            const int64_t r = (int64_t)in[x];
            const int64_t toT = min(r, pK);
            net.tcap[x] = pK - toT;
            net.excess[x] = r - toT;
            acc += (ull)toT;
        } else {
            net.excess[x] = 0;
        }
    }
    if (acc) atomicAdd(flow_t, acc);
}

// ---- global relabel

__global__ void gr_init_kernel(Net net, int32_t* frontier, int32_t* fcnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < net.nn; x += stride) {
        const bool hit = x < net.nv && net.tcap[x] > 0;
        net.height[x] = hit ? 1 : DEAD;
        if (hit) frontier[atomicAdd(fcnt, 1)] = (int32_t)x;
    }
}

// one level: x joins at level + 1 when it has a residual arc to a frontier node y
__global__ void gr_level_kernel(Net net, const int32_t* frontier, const int32_t* fcnt, int32_t level, int32_t* next,
                                int32_t* ncnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nf = *fcnt;
    for (int64_t i = warp; i < nf; i += nwarps) {
        const int32_t y = frontier[i];
        for (int64_t a = net.ptr[y] + lane; a < net.ptr[y + 1]; a += 32) {
            const int32_t x = net.head[a];
            if (__ldcg(net.height + x) == DEAD && net.cap[net.rev[a]] > 0)
                if (atomicCAS(net.height + x, DEAD, level + 1) == DEAD) next[atomicAdd(ncnt, 1)] = x;
        }
    }
}

// after a global relabel: work list of the active nodes, count of stuck excess
__global__ void gr_finish_kernel(Net net, int32_t* list, int32_t* lcnt, int32_t* inq, int32_t tag, int32_t* stuck) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int32_t st = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < net.nn; x += stride) {
        if (net.excess[x] <= 0) continue;
        if (net.height[x] < DEAD) {
            inq[x] = tag;
            list[atomicAdd(lcnt, 1)] = (int32_t)x;
        } else {
            ++st;
        }
    }
    if (st) atomicAdd(stuck, st);
}

// ---- push-relabel round: one warp per node of the current work list.  The
// lists and counts were written by earlier launches; values that other warps
// change during the round are read through L2 (__ldcg) or by atomics.
__global__ void __launch_bounds__(FB) pr_round_kernel(Net net, const int32_t* cur, const int32_t* cur_cnt, int32_t* nxt,
                                                     int32_t* nxt_cnt, int32_t* clear_cnt, int32_t* inq, int32_t tag,
                                                     int pulses, ull* flow_t, int32_t* relabels) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *clear_cnt = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t ncur = *cur_cnt;
    int32_t nrel = 0;
    for (int64_t i = warp; i < ncur; i += nwarps) {
        const int32_t x = cur[i];
        const int64_t a0 = net.ptr[x], a1 = net.ptr[x + 1];
        for (int it = 0; it < pulses; ++it) {
            const int64_t e = __ldcg(net.excess + x);
            const int32_t hx = __ldcg(net.height + x);
            if (e <= 0 || hx >= DEAD) break;
            if (x < net.nv) {
                const int64_t tc = __ldcg(net.tcap + x);
                if (tc > 0) {          // t (label 0) is the lowest neighbour
                    if (lane == 0) {
                        const int64_t d = min(e, tc);
                        atomicAdd((ull*)(net.tcap + x), (ull)(-d));
                        atomicAdd((ull*)(net.excess + x), (ull)(-d));
                        atomicAdd(flow_t, (ull)d);
                    }
                    __syncwarp();
                    continue;
                }
            }
            int32_t hmin = INT32_MAX;
            int64_t best = -1, capb = 0;
            for (int64_t a = a0 + lane; a < a1; a += 32) {
                const int64_t c = __ldcg(net.cap + a);
                if (c > 0) {
                    const int32_t hy = __ldcg(net.height + net.head[a]);
                    if (hy < hmin) {
                        hmin = hy;
                        best = a;
                        capb = c;
                    }
                }
            }
            const int32_t gmin = (int32_t)__reduce_min_sync(FULL, (unsigned)hmin);
            if (gmin == INT32_MAX) {           // no residual arc left
                if (lane == 0) net.height[x] = DEAD;
                __syncwarp();
                break;
            }
            const int src = __ffs(__ballot_sync(FULL, hmin == gmin)) - 1;
            best = __shfl_sync(FULL, best, src);
            capb = __shfl_sync(FULL, capb, src);
            if (hx > gmin) {
                if (lane == 0) {
                    // only x lowers its own arcs' capacities and its own excess, so d stays available
                    const int64_t d = min(e, capb);
                    const int32_t y = net.head[best];
                    atomicAdd((ull*)(net.cap + best), (ull)(-d));
                    atomicAdd((ull*)(net.cap + net.rev[best]), (ull)d);
                    atomicAdd((ull*)(net.excess + x), (ull)(-d));
                    const long long old = (long long)atomicAdd((ull*)(net.excess + y), (ull)d);
                    if (old <= 0 && atomicExch(inq + y, tag) != tag) nxt[atomicAdd(nxt_cnt, 1)] = y;
                }
            } else {
                if (lane == 0) net.height[x] = min(gmin + 1, DEAD);
                ++nrel;
            }
            __syncwarp();
        }
        if (lane == 0 && (long long)atomicAdd((ull*)(net.excess + x), 0ull) > 0 && __ldcg(net.height + x) < DEAD &&
            atomicExch(inq + x, tag) != tag)
            nxt[atomicAdd(nxt_cnt, 1)] = x;
    }
    if (lane == 0 && nrel) atomicAdd(relabels, nrel);
}

__global__ void side_kernel(const int32_t* height, int32_t nv, uint8_t* side) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) side[v] = height[v] >= DEAD;
}

// blocks for a warp-per-item launch, at most 8 blocks per SM
int warps_grid(int64_t items) {
    const int64_t cap = (int64_t)num_sms() * 8;
    const int64_t b = (items * 32 + FB - 1) / FB;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

}  // namespace

int64_t pattern_max_flow(const int64_t* pptr, const int32_t* pidx, int32_t np, int32_t nv, int64_t p, int64_t q,
                         const int64_t* share, uint8_t* side, bool stop_if_short, cudaStream_t s) {
    LDS_REQUIRE(q > 0 && p >= 0 && np >= 0 && nv >= 0, LDS_EINVAL, "max flow: bad network");
    // K: the largest power of two up to 2^20 with np q K <= 2^61, so every sum of flows fits
    int64_t K = 1;
    const i128 unit = (i128)std::max<int64_t>(np, 1) * q;
    while (K < (1 << 20) && unit * (K * 2) <= ((i128)1 << 61)) K *= 2;
    LDS_REQUIRE(unit * K <= ((i128)1 << 62) && (i128)p * K <= ((i128)1 << 62), LDS_EOVERFLOW,
                "max flow: capacities overflow");
    const int64_t qK = q * K, pK = p * K;
    int64_t nidx = 0;
    if (np) {
        LDS_CUDA(cudaMemcpyAsync(&nidx, pptr + np, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
    }
    DevBuf<int64_t> f(std::max<int64_t>(nidx, 1), s);
    DevBuf<int32_t> big(np + 1, s);
    DevBuf<int64_t> bigpos(np + 1, s);
    LDS_CUDA(cudaMemsetAsync(big.get(), 0, (np + 1) * sizeof(int32_t), s));
    int64_t n3 = 0;
    if (np) {
        LDS_LAUNCH(split_kernel, grid_for(np, FB), FB, 0, s, pptr, np, share, qK, f.get(), big.get());
        n3 = exclusive_scan_i32_to_i64(big.get(), bigpos.get(), np + 1, s);
    }
    LDS_REQUIRE((int64_t)nv + n3 < (int64_t)DEAD, LDS_EOVERFLOW, "max flow: too many nodes");
    const int32_t nn = nv + (int32_t)n3;
    const int32_t nnp = std::max(nn, 1);
    DevBuf<int32_t> deg(nnp + 1, s), cursor(nnp, s);
    DevBuf<ull> in(nnp, s);
    LDS_CUDA(cudaMemsetAsync(deg.get(), 0, (nnp + 1) * sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(cursor.get(), 0, nnp * sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(in.get(), 0, nnp * sizeof(ull), s));
    if (np) LDS_LAUNCH(degree_kernel, grid_for(np, FB), FB, 0, s, pptr, pidx, np, f.get(), bigpos.get(), nv, deg.get(), in.get());
    DevBuf<int64_t> ptr(nnp + 1, s);
    const int64_t A = exclusive_scan_i32_to_i64(deg.get(), ptr.get(), nn + 1, s);
    DevBuf<int32_t> head(std::max<int64_t>(A, 1), s);
    DevBuf<int64_t> cap(std::max<int64_t>(A, 1), s), rev(std::max<int64_t>(A, 1), s);
    if (np)
        LDS_LAUNCH(fill_kernel, grid_for(np, FB), FB, 0, s, pptr, pidx, np, f.get(), bigpos.get(), nv, qK, ptr.get(),
                   cursor.get(), head.get(), cap.get(), rev.get());
    DevBuf<int64_t> tcap(std::max(nv, 1), s), excess(nnp, s);
    DevBuf<int32_t> height(nnp, s), inq(nnp, s);
    DevBuf<int32_t> la(nnp, s), lb(nnp, s), cnt(4, s), gcnt(3, s);
    DevBuf<ull> flow_t(1, s);
    LDS_CUDA(cudaMemsetAsync(inq.get(), 0, nnp * sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(flow_t.get(), 0, sizeof(ull), s));
    Net net{nv, nn, ptr.get(), head.get(), cap.get(), rev.get(), tcap.get(), excess.get(), height.get()};
    if (nn) LDS_LAUNCH(init_kernel, grid_for(nn, FB), FB, 0, s, net, in.get(), pK, flow_t.get());

    int32_t tag = 0;
    // cnt: [0..2] work-list counts (triple-buffered), [3] relabels;
    // gcnt: [0..1] breadth-first frontier counts, [2] nodes with stuck excess
    auto global_relabel = [&]() -> std::pair<int32_t, int32_t> {
        LDS_CUDA(cudaMemsetAsync(gcnt.get(), 0, 3 * sizeof(int32_t), s));
        if (nn) LDS_LAUNCH(gr_init_kernel, grid_for(nn, FB), FB, 0, s, net, la.get(), gcnt.get());
        int32_t fsize = 0;
        LDS_CUDA(cudaMemcpyAsync(&fsize, gcnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        int32_t* cur = la.get();
        int32_t* nxt = lb.get();
        int32_t* ccur = gcnt.get();
        int32_t* cnxt = gcnt.get() + 1;
        for (int32_t level = 1; fsize > 0; ++level) {
            LDS_REQUIRE(level <= nn + 1, LDS_ETIMEOUT, "max flow: global relabel did not finish");
            LDS_CUDA(cudaMemsetAsync(cnxt, 0, sizeof(int32_t), s));
            LDS_LAUNCH(gr_level_kernel, warps_grid(fsize), FB, 0, s, net, cur, ccur, level, nxt, cnxt);
            LDS_CUDA(cudaMemcpyAsync(&fsize, cnxt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
            std::swap(cur, nxt);
            std::swap(ccur, cnxt);
        }
        // the work list goes to la with its count in cnt[0]
        LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, 4 * sizeof(int32_t), s));
        LDS_CUDA(cudaMemsetAsync(gcnt.get() + 2, 0, sizeof(int32_t), s));
        ++tag;
        if (nn) LDS_LAUNCH(gr_finish_kernel, grid_for(nn, FB), FB, 0, s, net, la.get(), cnt.get(), inq.get(), tag, gcnt.get() + 2);
        int32_t h[2] = {0, 0};
        LDS_CUDA(cudaMemcpyAsync(&h[0], cnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaMemcpyAsync(&h[1], gcnt.get() + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        return {h[0], h[1]};
    };

    const int pulses = 8;
    const int batch = 8;
    const int64_t max_rounds = 64 * (int64_t)nn + 100000;
    const int round_grid = warps_grid(nn);
    int64_t rounds = 0;
    while (true) {
        const std::pair<int32_t, int32_t> gr = global_relabel();
        if (stop_if_short && gr.second > 0) return -1;
        if (gr.first == 0) break;
        // rounds until the list empties or enough relabels pile up for a new global relabel
        int32_t* lists[2] = {la.get(), lb.get()};
        for (int r = 0;;) {
            for (int b = 0; b < batch; ++b, ++r) {
                ++tag;
                LDS_LAUNCH(pr_round_kernel, round_grid, FB, 0, s, net, lists[r & 1], cnt.get() + (r % 3),
                           lists[(r + 1) & 1], cnt.get() + ((r + 1) % 3), cnt.get() + ((r + 2) % 3), inq.get(), tag,
                           pulses, flow_t.get(), cnt.get() + 3);
            }
            int32_t h[2];
            LDS_CUDA(cudaMemcpyAsync(&h[0], cnt.get() + (r % 3), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaMemcpyAsync(&h[1], cnt.get() + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
            rounds += batch;
            LDS_REQUIRE(rounds < max_rounds, LDS_ETIMEOUT, "max flow: push-relabel did not finish");
            if (h[0] == 0 || h[1] > nn) break;
        }
    }
    ull ft = 0;
    LDS_CUDA(cudaMemcpyAsync(&ft, flow_t.get(), sizeof(ull), cudaMemcpyDeviceToHost, s));
    if (side && nv) LDS_LAUNCH(side_kernel, grid_for(nv, FB), FB, 0, s, height.get(), nv, side);
    LDS_CUDA(cudaStreamSynchronize(s));
    // every cut of the network is a multiple of K
    LDS_REQUIRE((int64_t)ft % K == 0, LDS_ECUDA, "max flow: flow value %llu is not a multiple of the scale", ft);
    return (int64_t)ft / K;
}

}  // namespace lds

using namespace lds;

extern "C" lds_status lds_pattern_max_flow(int32_t nv, int32_t np, const int64_t* pat_ptr, const int32_t* pat_idx,
                                           int64_t p, int64_t q, int64_t* flow, uint8_t* source_side) {
    return guard([&] {
        LDS_REQUIRE(nv >= 0 && np >= 0 && p >= 0 && q > 0, LDS_EINVAL, "lds_pattern_max_flow: bad sizes or capacities");
        LDS_REQUIRE(flow && (np == 0 || (pat_ptr && pat_idx)), LDS_EINVAL, "lds_pattern_max_flow: NULL argument");
        LDS_REQUIRE(lds_device_count() > 0, LDS_ECUDA, "lds_pattern_max_flow: no CUDA device");
        LDS_REQUIRE(np == 0 || pat_ptr[0] == 0, LDS_EINVAL, "lds_pattern_max_flow: pat_ptr[0] must be 0");
        for (int32_t j = 0; j < np; ++j)
            LDS_REQUIRE(pat_ptr[j + 1] >= pat_ptr[j], LDS_EINVAL, "lds_pattern_max_flow: pat_ptr not ascending");
        const int64_t k = np ? pat_ptr[np] : 0;
        for (int64_t i = 0; i < k; ++i)
            LDS_REQUIRE(pat_idx[i] >= 0 && pat_idx[i] < nv, LDS_EINVAL, "lds_pattern_max_flow: vertex index out of range");
        for (int32_t j = 0; j < np; ++j)
            for (int64_t a = pat_ptr[j]; a < pat_ptr[j + 1]; ++a)
                for (int64_t b = a + 1; b < pat_ptr[j + 1]; ++b)
                    LDS_REQUIRE(pat_idx[a] != pat_idx[b], LDS_EINVAL, "lds_pattern_max_flow: pattern %d repeats a vertex", j);
        cudaStream_t s = nullptr;
        DevBuf<int64_t> dp(np + 1, s);
        DevBuf<int32_t> di(std::max<int64_t>(k, 1), s);
        DevBuf<uint8_t> side(std::max(nv, 1), s);
        if (np) copy_in(dp.get(), pat_ptr, LDS_MEM_HOST, (np + 1) * sizeof(int64_t), s);
        else LDS_CUDA(cudaMemsetAsync(dp.get(), 0, sizeof(int64_t), s));
        if (k) copy_in(di.get(), pat_idx, LDS_MEM_HOST, k * sizeof(int32_t), s);
        *flow = pattern_max_flow(dp.get(), di.get(), np, nv, p, q, nullptr, side.get(), false, s);
        if (source_side && nv) {
            copy_out(source_side, LDS_MEM_HOST, side.get(), nv, s);
            LDS_CUDA(cudaStreamSynchronize(s));
        }
    });
}
