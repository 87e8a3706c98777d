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
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
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

// ---- vertex-node form (no pattern nodes)
//
// After the preflow every pattern P holds its qK units split among its members
// (f_{P,x}).  In Alg. 8's network the residual path x -> P -> y exists exactly
// when f_{P,x} > 0, and pushing d units along it is f_{P,x} -= d, f_{P,y} += d.
// So the network needs no pattern nodes: x has a hyper-arc to every other
// member y of P, all of them drawing on the same capacity f_{P,x}.  Labels
// stay valid under such a push: if h(x) = h(y) + 1 and the push makes y -> z
// through P residual for a third member z, then x -> z through P was residual,
// so h(x) <= h(z) + 1 and h(y) <= h(z).  The vertices that cannot reach t in
// this residual structure are exactly those that cannot reach t in Alg. 8's
// network, so the DEAD vertices at the end are the largest source side.
//
// Layout: the incidences of every vertex are contiguous (vptr); incidence i
// holds f (its vertex's share of the pattern) and the incidences / vertices of
// the pattern's other members (at most two; -1 where absent).  Loops (one
// member) only feed their vertex and have no incidence.
struct HNet {
    int32_t nv;
    const int64_t* vptr;   // [nv + 1]
    int64_t* f;            // [ninc]
    const int32_t* o1;     // [ninc] incidence of another member, -1 if none
    const int32_t* o2;
    const int32_t* w1;     // [ninc] vertex of that member, -1 if none
    const int32_t* w2;
    int64_t* tcap;         // [nv] residual capacity to t
    int64_t* excess;       // [nv]
    int32_t* h;            // [nv] exact distance to t (DEAD: cannot reach it)
};

// widths above 3 are refused; count[v] = incidences of v; in[v] = flow v receives
__global__ void hyper_degree_kernel(const int64_t* pptr, const int32_t* pidx, int32_t np, const int64_t* f,
                                    int32_t* deg, ull* in, int32_t* wide) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int64_t b = pptr[j], e = pptr[j + 1], len = e - b;
        if (len > 3) {
            *wide = 1;
            continue;
        }
        for (int64_t k = b; k < e; ++k) {
            atomicAdd(in + pidx[k], (ull)f[k]);
            if (len >= 2) atomicAdd(deg + pidx[k], 1);
        }
    }
}

// position of every slot (of a pattern with >= 2 members) in its vertex's incidence list
__global__ void hyper_pos_kernel(const int64_t* pptr, const int32_t* pidx, int32_t np, const int64_t* vptr,
                                 int32_t* cursor, int32_t* pos) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int64_t b = pptr[j], e = pptr[j + 1];
        if (e - b < 2 || e - b > 3) continue;
        for (int64_t k = b; k < e; ++k) pos[k] = (int32_t)(vptr[pidx[k]] + atomicAdd(cursor + pidx[k], 1));
    }
}

__global__ void hyper_fill_kernel(const int64_t* pptr, const int32_t* pidx, int32_t np, const int64_t* fslot,
                                  const int32_t* pos, HNet net) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int64_t b = pptr[j], e = pptr[j + 1], len = e - b;
        if (len < 2 || len > 3) continue;
        for (int64_t k = b; k < e; ++k) {
            const int64_t a = k == b ? b + 1 : b;                  // the other members, in slot order
            const int64_t c = len == 3 ? (k == e - 1 ? e - 2 : e - 1) : -1;
            const int32_t i = pos[k];
            net.f[i] = fslot[k];
            ((int32_t*)net.o1)[i] = pos[a];
            ((int32_t*)net.w1)[i] = pidx[a];
            ((int32_t*)net.o2)[i] = c >= 0 ? pos[c] : -1;
            ((int32_t*)net.w2)[i] = c >= 0 ? pidx[c] : -1;
        }
    }
}

__global__ void hyper_init_kernel(HNet net, const ull* in, int64_t pK, ull* flow_t) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    ull acc = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < net.nv; x += stride) {
        const int64_t r = (int64_t)in[x];
        const int64_t toT = min(r, pK);
        net.tcap[x] = pK - toT;
        net.excess[x] = r - toT;
        acc += (ull)toT;
    }
    if (acc) atomicAdd(flow_t, acc);
}

// hyper_flow_kernel control words
enum : int {
    HC_LEVEL = 0,      // [0..2] vertices labelled per breadth-first level (three rotating counters)
    HC_ACTIVE = 3,     // vertices with excess and a label
    HC_STUCK = 4,      // vertices with excess and no path to t
    HC_LMAX = 5,       // highest label holding excess
    HC_FLOW = 6,       // flow into t
    HC_STATUS = 7,     // 0 finished, 1 phase bound hit, 2 stopped: some excess cannot reach t
    HC_PHASES = 8,
    HC_LEVELS = 9,     // breadth-first levels run in all
    HC_WORDS = 10
};

// One cooperative launch runs the whole preflow phase.  Each phase computes
// exact distance labels by a breadth-first search from t over the residual
// hyper-arcs (a global relabel), then sweeps the labels from the highest one
// that holds excess down to 1: every vertex at label L with excess pushes it
// along its admissible hyper-arcs (to members at label L - 1), in incidence
// order, until the excess or those arcs run out; vertices at label 1 push into
// t.  Within a label no two vertices touch the same share from below (a share
// is lowered only by its own vertex, and vertices at label L receive nothing
// while label L is swept), so a push needs atomics only on the target's share
// and excess.  After the sweep every vertex that still holds excess has no
// admissible hyper-arc, and since no push shortens a distance, its label rises
// in the next phase; labels are at most nv, so there are at most nv^2 + 1
// phases.  One warp serves one vertex; `max_phases` bounds the loop (status 1).
__global__ void __launch_bounds__(FB) hyper_flow_kernel(HNet net, ull* ctrl, int64_t max_phases, int stop_if_short) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t warp = tid >> 5, nwarps = nthreads >> 5;
    const int32_t nv = net.nv;
    for (int64_t phase = 0;; ++phase) {
        if (phase >= max_phases) {
            if (tid == 0) ctrl[HC_STATUS] = 1;
            return;
        }
        if (tid == 0) {
            ctrl[HC_LEVEL] = ctrl[HC_LEVEL + 1] = ctrl[HC_LEVEL + 2] = 0;
            ctrl[HC_ACTIVE] = ctrl[HC_STUCK] = ctrl[HC_LMAX] = 0;
            ctrl[HC_PHASES] = (ull)phase + 1;
        }
        for (int64_t v = tid; v < nv; v += nthreads) net.h[v] = __ldcg(net.tcap + v) > 0 ? 1 : DEAD;
        grid.sync();
        // breadth-first levels: an unlabelled vertex joins level L + 1 when one of its
        // hyper-arcs (share > 0) leads to a member at level L
        for (int32_t L = 1;; ++L) {
            for (int64_t v = warp; v < nv; v += nwarps) {
                if (__ldcg(net.h + v) != DEAD) continue;
                const int64_t b0 = net.vptr[v], b1 = net.vptr[v + 1];
                bool found = false;
                for (int64_t base = b0; base < b1 && !found; base += 32) {
                    const int64_t i = base + lane;
                    bool hit = false;
                    if (i < b1 && __ldcg(net.f + i) > 0) {
                        const int32_t a = net.w1[i], c = net.w2[i];
                        hit = (a >= 0 && __ldcg(net.h + a) == L) || (c >= 0 && __ldcg(net.h + c) == L);
                    }
                    found = __any_sync(FULL, hit);
                }
                if (found && lane == 0) {
                    net.h[v] = L + 1;
                    atomicAdd(ctrl + HC_LEVEL + (L % 3), 1ull);
                }
            }
            grid.sync();
            const ull added = __ldcg(ctrl + HC_LEVEL + (L % 3));
            if (tid == 0) {
                ctrl[HC_LEVEL + ((L + 2) % 3)] = 0;
                ctrl[HC_LEVELS] += 1;
            }
            if (added == 0) break;
        }
        // vertices holding excess: with a label (active) or without (stuck)
        {
            ull act = 0, stk = 0;
            int32_t lmax = 0;
            for (int64_t v = tid; v < nv; v += nthreads) {
                if (__ldcg(net.excess + v) > 0) {
                    const int32_t hv = __ldcg(net.h + v);
                    if (hv < DEAD) {
                        ++act;
                        lmax = max(lmax, hv);
                    } else {
                        ++stk;
                    }
                }
            }
            for (int o = 16; o; o >>= 1) {
                act += __shfl_xor_sync(FULL, act, o);
                stk += __shfl_xor_sync(FULL, stk, o);
                lmax = max(lmax, __shfl_xor_sync(FULL, lmax, o));
            }
            if (lane == 0) {
                if (act) atomicAdd(ctrl + HC_ACTIVE, act);
                if (stk) atomicAdd(ctrl + HC_STUCK, stk);
                if (lmax) atomicMax(ctrl + HC_LMAX, (ull)lmax);
            }
        }
        grid.sync();
        const ull act = __ldcg(ctrl + HC_ACTIVE), stk = __ldcg(ctrl + HC_STUCK);
        const int32_t lmax = (int32_t)__ldcg(ctrl + HC_LMAX);
        if (stop_if_short && stk > 0) {
            if (tid == 0) ctrl[HC_STATUS] = 2;
            return;
        }
        if (act == 0) {
            if (tid == 0) ctrl[HC_STATUS] = 0;
            return;
        }
        // downhill sweep
        for (int32_t L = lmax; L >= 1; --L) {
            for (int64_t v = warp; v < nv; v += nwarps) {
                if (__ldcg(net.h + v) != L) continue;
                const int64_t e = __ldcg(net.excess + v);
                if (e <= 0) continue;
                if (L == 1) {
                    if (lane == 0) {
                        const int64_t tc = __ldcg(net.tcap + v);
                        const int64_t d = min(e, tc);
                        if (d > 0) {
                            net.tcap[v] = tc - d;
                            net.excess[v] = e - d;
                            atomicAdd(ctrl + HC_FLOW, (ull)d);
                        }
                    }
                    continue;
                }
                const int64_t b0 = net.vptr[v], b1 = net.vptr[v + 1];
                int64_t rem = e;
                for (int64_t base = b0; base < b1 && rem > 0; base += 32) {
                    const int64_t i = base + lane;
                    int64_t cap = 0;
                    int32_t to_i = -1, to_v = -1;
                    if (i < b1) {
                        const int64_t fi = __ldcg(net.f + i);
                        if (fi > 0) {
                            const int32_t a = net.w1[i], c = net.w2[i];
                            if (a >= 0 && __ldcg(net.h + a) == L - 1) {
                                cap = fi;
                                to_i = net.o1[i];
                                to_v = a;
                            } else if (c >= 0 && __ldcg(net.h + c) == L - 1) {
                                cap = fi;
                                to_i = net.o2[i];
                                to_v = c;
                            }
                        }
                    }
                    // shares of all incidences sum to at most np q K <= 2^61: no overflow
                    int64_t incl = cap;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int64_t t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += t;
                    }
                    const int64_t d = max((int64_t)0, min(cap, rem - (incl - cap)));
                    if (d > 0) {
                        net.f[i] -= d;
                        atomicAdd((ull*)(net.f + to_i), (ull)d);
                        atomicAdd((ull*)(net.excess + to_v), (ull)d);
                    }
                    rem -= min(rem, __shfl_sync(FULL, incl, 31));
                }
                if (lane == 0 && rem != e) net.excess[v] = rem;
            }
            grid.sync();
        }
    }
}

}  // namespace

std::atomic<int> g_flow_variant{0};

// The vertex-node form of the maximum flow, from the split f of every slot.
static int64_t hyper_max_flow(const int64_t* pptr, const int32_t* pidx, int32_t np, int32_t nv, int64_t nidx,
                              const int64_t* fslot, int64_t pK, int64_t K, uint8_t* side, bool stop_if_short,
                              cudaStream_t s) {
    const int32_t nvp = std::max(nv, 1);
    DevBuf<int32_t> deg(nvp + 1, s), cursor(nvp, s), wide(1, s);
    DevBuf<ull> in(nvp, s), ctrl(HC_WORDS, s);
    LDS_CUDA(cudaMemsetAsync(deg.get(), 0, (nvp + 1) * sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(cursor.get(), 0, nvp * sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(wide.get(), 0, sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(in.get(), 0, nvp * sizeof(ull), s));
    LDS_CUDA(cudaMemsetAsync(ctrl.get(), 0, HC_WORDS * sizeof(ull), s));
    if (np)
        LDS_LAUNCH(hyper_degree_kernel, grid_for(np, FB), FB, 0, s, pptr, pidx, np, fslot, deg.get(), in.get(),
                   wide.get());
    DevBuf<int64_t> vptr(nvp + 1, s);
    const int64_t ninc = exclusive_scan_i32_to_i64(deg.get(), vptr.get(), (int64_t)nv + 1, s);
    int32_t hwide = 0;
    LDS_CUDA(cudaMemcpyAsync(&hwide, wide.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    LDS_REQUIRE(hwide == 0, LDS_EINVAL, "max flow: a pattern has more than three members");
    LDS_REQUIRE(ninc < (int64_t)INT32_MAX, LDS_EOVERFLOW, "max flow: %lld incidences exceed the 32-bit index",
                (long long)ninc);
    DevBuf<int32_t> pos(std::max<int64_t>(nidx, 1), s);
    DevBuf<int64_t> f(std::max<int64_t>(ninc, 1), s), tcap(nvp, s), excess(nvp, s);
    DevBuf<int32_t> o1(std::max<int64_t>(ninc, 1), s), o2(std::max<int64_t>(ninc, 1), s);
    DevBuf<int32_t> w1(std::max<int64_t>(ninc, 1), s), w2(std::max<int64_t>(ninc, 1), s), h(nvp, s);
    HNet net{nv, vptr.get(), f.get(), o1.get(), o2.get(), w1.get(), w2.get(), tcap.get(), excess.get(), h.get()};
    if (np) {
        LDS_LAUNCH(hyper_pos_kernel, grid_for(np, FB), FB, 0, s, pptr, pidx, np, vptr.get(), cursor.get(), pos.get());
        LDS_LAUNCH(hyper_fill_kernel, grid_for(np, FB), FB, 0, s, pptr, pidx, np, fslot, pos.get(), net);
    }
    if (nv) LDS_LAUNCH(hyper_init_kernel, grid_for(nv, FB), FB, 0, s, net, in.get(), pK, ctrl.get() + HC_FLOW);
    if (nv) {
        int per_sm = 0;
        LDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hyper_flow_kernel, FB, 0));
        LDS_REQUIRE(per_sm > 0, LDS_ECUDA, "max flow: the flow kernel cannot be resident");
        // one warp per vertex; no more blocks than can be resident at once
        const int64_t want = ((int64_t)nv * 32 + FB - 1) / FB;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * std::min(per_sm, 4)));
        const int64_t max_phases = std::min<int64_t>((int64_t)nv * nv + 2, (int64_t)1 << 40);
        int stop = stop_if_short ? 1 : 0;
        ull* cp = ctrl.get();
        void* args[] = {(void*)&net, (void*)&cp, (void*)&max_phases, (void*)&stop};
        LDS_CUDA(cudaLaunchCooperativeKernel((void*)hyper_flow_kernel, dim3(grid), dim3(FB), args, 0, s));
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    ull hc[HC_WORDS];
    LDS_CUDA(cudaMemcpyAsync(hc, ctrl.get(), sizeof(hc), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    LDS_REQUIRE(hc[HC_STATUS] != 1, LDS_ETIMEOUT, "max flow: phase bound hit");
    if (hc[HC_STATUS] == 2) return -1;
    if (side && nv) LDS_LAUNCH(side_kernel, grid_for(nv, FB), FB, 0, s, h.get(), nv, side);
    LDS_CUDA(cudaStreamSynchronize(s));
    const ull ft = hc[HC_FLOW];
    LDS_REQUIRE((int64_t)ft % K == 0, LDS_ECUDA, "max flow: flow value %llu is not a multiple of the scale", ft);
    return (int64_t)ft / K;
}

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
    // the vertex-node form is the default (variant 0)
    const int variant = g_flow_variant.load(std::memory_order_relaxed);
    if (variant != 1)
        return hyper_max_flow(pptr, pidx, np, nv, nidx, f.get(), pK, K, side, stop_if_short, s);
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

extern "C" lds_status lds_set_flow_variant(int32_t variant) {
    return guard([&] {
        LDS_REQUIRE(variant >= 0 && variant <= 2, LDS_EINVAL, "lds_set_flow_variant: %d is not 0, 1 or 2", variant);
        g_flow_variant.store(variant, std::memory_order_relaxed);
    });
}

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
