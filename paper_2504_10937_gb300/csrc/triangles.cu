// Triangle listing (the set T of Eq. 3 / Eq. 4) and core / tr-core numbers
// (Def. 6, Def. 11).
//
// Listing: every edge is oriented from the endpoint of lower (degree, id) rank
// to the higher one, which bounds out-degrees by O(sqrt(m)); each oriented edge
// x -> y meets out(x) and out(y) (both ascending) by a merge walk, and each
// common out-neighbour w closes the triangle {x, y, w} exactly once.  A count
// pass sizes the output, a write pass fills it, and two stable radix sorts put
// the rows in (a, b, c) order.
//
// Core numbers: level-synchronous peeling.  At level k every live vertex whose
// remaining degree (number of live triangles for tr-core) is <= k gets core k
// and is removed, its neighbours' degrees drop, and the step repeats until no
// vertex is removed; then k moves to the smallest remaining degree.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>
#include <cstdio>
#include <cstdlib>

#include "graph.cuh"
#include "prims.cuh"

namespace cg = cooperative_groups;

namespace lds {

namespace {

__device__ __forceinline__ bool precedes(int32_t dx, int32_t x, int32_t dy, int32_t y) {
    return dx < dy || (dx == dy && x < y);
}

__global__ void orient_count_kernel(const int64_t* rowptr, const int32_t* col, int32_t nact, int32_t* outdeg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int64_t b = rowptr[x], e = rowptr[x + 1];
        int32_t dx = (int32_t)(e - b);
        int32_t c = 0;
        for (int64_t s = b; s < e; ++s) {
            int32_t y = col[s];
            int32_t dy = (int32_t)(rowptr[y + 1] - rowptr[y]);
            c += precedes(dx, (int32_t)x, dy, y);
        }
        outdeg[x] = c;
    }
}

__global__ void orient_fill_kernel(const int64_t* rowptr, const int32_t* col, int32_t nact, const int64_t* optr,
                                   int32_t* ocol) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int64_t b = rowptr[x], e = rowptr[x + 1];
        int32_t dx = (int32_t)(e - b);
        int64_t o = optr[x];
        for (int64_t s = b; s < e; ++s) {
            int32_t y = col[s];
            int32_t dy = (int32_t)(rowptr[y + 1] - rowptr[y]);
            if (precedes(dx, (int32_t)x, dy, y)) ocol[o++] = y;
        }
    }
}

// source vertex of every oriented slot
__global__ void oriented_src_kernel(const int64_t* optr, int32_t nact, int32_t* osrc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride)
        for (int64_t s = optr[x], e = optr[x + 1]; s < e; ++s) osrc[s] = (int32_t)x;
}

template <bool WRITE>
__global__ void tri_intersect_kernel(const int64_t* optr, const int32_t* ocol, const int32_t* osrc, int64_t nos,
                                     int64_t* count, const int64_t* offset, int32_t* ta, int32_t* tb, int32_t* tc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nos; s += stride) {
        int32_t x = osrc[s], y = ocol[s];
        int64_t i = optr[x], ie = optr[x + 1];
        int64_t j = optr[y], je = optr[y + 1];
        int64_t c = 0;
        int64_t o = WRITE ? offset[s] : 0;
        while (i < ie && j < je) {
            int32_t a = ocol[i], b = ocol[j];
            if (a < b) ++i;
            else if (b < a) ++j;
            else {
                if (WRITE) {
                    int32_t p = x, q = y, r = a;
                    if (p > q) { int32_t t = p; p = q; q = t; }
                    if (q > r) { int32_t t = q; q = r; r = t; }
                    if (p > q) { int32_t t = p; p = q; q = t; }
                    ta[o] = p; tb[o] = q; tc[o] = r;
                    ++o;
                }
                ++c; ++i; ++j;
            }
        }
        if (!WRITE) count[s] = c;
    }
}

__global__ void tri_key_bc_kernel(const int32_t* tb, const int32_t* tc, int64_t ntri, int64_t nn, uint64_t* key,
                                  uint32_t* idx) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        key[t] = (uint64_t)tb[t] * (uint64_t)nn + (uint64_t)tc[t];
        idx[t] = (uint32_t)t;
    }
}

__global__ void tri_key_a_kernel(const int32_t* ta, const uint32_t* idx, int64_t ntri, uint64_t* key) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) key[t] = (uint64_t)ta[idx[t]];
}

__global__ void permute3_kernel(const int32_t* a, const int32_t* b, const int32_t* c, const uint32_t* idx, int64_t k,
                                int32_t* oa, int32_t* ob, int32_t* oc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k; t += stride) {
        uint32_t j = idx[t];
        oa[t] = a[j]; ob[t] = b[j]; oc[t] = c[j];
    }
}

__global__ void tri_rows_orig_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, const int32_t* to_orig,
                                     int64_t ntri, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        out[3 * t] = to_orig[ta[t]];
        out[3 * t + 1] = to_orig[tb[t]];
        out[3 * t + 2] = to_orig[tc[t]];
    }
}

// ---- peeling

__global__ void alive_init_kernel(const uint8_t* init, int32_t nact, uint8_t* alive, int64_t* core, int32_t* nalive) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int32_t c = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        uint8_t a = init ? (init[x] ? 1 : 0) : 1;
        alive[x] = a;
        core[x] = -1;
        c += a;
    }
    if (c) atomicAdd(nalive, c);
}

__global__ void alive_degree_kernel(const int64_t* rowptr, const int32_t* col, const uint8_t* alive, int32_t nact,
                                    int32_t* deg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        if (!alive[x]) continue;
        int32_t d = 0;
        for (int64_t q = rowptr[x], e = rowptr[x + 1]; q < e; ++q) d += alive[col[q]];
        deg[x] = d;
    }
}

// triangle counts of G[alive]; triangles with a dead vertex are marked dead
__global__ void tri_all_alive_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t ntri,
                                     const uint8_t* alive, int32_t* flag) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride)
        flag[t] = alive[ta[t]] && alive[tb[t]] && alive[tc[t]];
}

__global__ void tri_compact_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t ntri,
                                   const int32_t* flag, const int64_t* tpos, int32_t* oa, int32_t* ob, int32_t* oc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride)
        if (flag[t]) {
            const int64_t o = tpos[t];
            oa[o] = ta[t];
            ob[o] = tb[t];
            oc[o] = tc[t];
        }
}

__global__ void alive_tri_count_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t ntri,
                                       const uint8_t* alive, int32_t* deg, uint8_t* tdead) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        int32_t a = ta[t], b = tb[t], c = tc[t];
        if (alive[a] && alive[b] && alive[c]) {
            atomicAdd(deg + a, 1);
            atomicAdd(deg + b, 1);
            atomicAdd(deg + c, 1);
        } else {
            unsigned int* word = (unsigned int*)(tdead + (t & ~3ll));
            atomicOr(word, 1u << (8 * (t & 3)));
        }
    }
}

// one atomic per group of converged threads that append together
__device__ __forceinline__ unsigned long long agg_slot(unsigned long long* ctr) {
    cg::coalesced_group grp = cg::coalesced_threads();
    unsigned long long base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(ctr, (unsigned long long)grp.size());
    return grp.shfl(base, 0) + grp.thread_rank();
}

// Removing a peeled vertex at level k lowers the count of each neighbour (of
// each other vertex of each live triangle); a vertex whose count falls from
// k + 1 to k is peeled at level k too (exactly one decrement sees k + 1) and
// joins the next frontier.  Counts of vertices already peeled are lowered as
// well: theirs are at most their level <= k and only fall, so they never see
// k + 1 again, and skipping a liveness test saves a dependent load.
__device__ __forceinline__ void peel_drop(int32_t y, int64_t k, uint8_t* alive, int32_t* deg, int64_t* core,
                                          int32_t* next, unsigned long long* next_cnt) {
    if ((int64_t)atomicSub(deg + y, 1) == k + 1) {
        alive[y] = 0;
        core[y] = k;
        next[agg_slot(next_cnt)] = y;
    }
}

__device__ __forceinline__ void peel_triangle(int32_t t, int32_t x, int64_t k, const int32_t* ta, const int32_t* tb,
                                              const int32_t* tc, uint8_t* tdead, uint8_t* alive, int32_t* deg,
                                              int64_t* core, int32_t* next, unsigned long long* next_cnt) {
    unsigned int* word = (unsigned int*)(tdead + (t & ~3));
    unsigned int bit = 1u << (8 * (t & 3));
    if (atomicOr(word, bit) & bit) return;          // the triangle died with another vertex
    int32_t a = ta[t], b = tb[t], c = tc[t];
    if (a != x) peel_drop(a, k, alive, deg, core, next, next_cnt);
    if (b != x) peel_drop(b, k, alive, deg, core, next, next_cnt);
    if (c != x) peel_drop(c, k, alive, deg, core, next, next_cnt);
}

constexpr int PEEL_LIGHT = 8;       // a lane removes a vertex with at most this many incidences
constexpr int PEEL_CHUNK = 128;     // otherwise a warp removes each chunk of this many (4 per lane)

constexpr int PEEL_SOLO = 8192;      // live vertices the one-block kernel finishes with, in shared memory
constexpr int PEEL_SOLO_T = 1024;    // its threads
constexpr size_t PEEL_SOLO_SMEM = 16 + (size_t)PEEL_SOLO * (4 * sizeof(int32_t) + 1);

// exclusive block scan of one int64 per thread (PEEL_SOLO_T threads); returns the total
__device__ __forceinline__ int64_t block_scan_i64(int64_t v, int64_t* out, int64_t* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;                          // inclusive warp totals
    }
    __syncthreads();
    out[tid] = inc - v + (wid ? wsum[wid - 1] : 0);
    const int64_t total = wsum[31];
    __syncthreads();
    return total;
}

// The dense tail of the peel, in one block, once at most PEEL_SOLO vertices are
// live (the grid-wide kernel hands over through ctrl[9..12]).  Their counts, live
// flags and the frontiers sit in shared memory (live vertex x at slot[x]; slot
// is -1 for every other vertex, whose count no longer matters), so a round costs
// block barriers and shared-memory atomics instead of grid barriers and L2
// atomics.  A round's incidences are spread evenly over the threads (batches of
// PEEL_SOLO_T frontier vertices, a scan of their incidence counts), so one hub
// does not hold the round.  Same levels and rules as the grid-wide loop.
__global__ void __launch_bounds__(PEEL_SOLO_T, 1) peel_solo_kernel(
    bool tri, const int64_t* ptr, const int32_t* adj, const int32_t* ta, const int32_t* tb, const int32_t* tc,
    uint8_t* tdead, const uint8_t* alive, const int32_t* deg, int64_t* core, const int32_t* A0, const int32_t* A1,
    int32_t* slot, unsigned long long* ctrl, int64_t max_steps) {
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int64_t b_off[PEEL_SOLO_T], b_beg[PEEL_SOLO_T], wsum[32];
    __shared__ int32_t b_x[PEEL_SOLO_T];
    if (ctrl[12] == 0) return;                  // the grid-wide kernel finished the peel
    const int32_t* list = ctrl[9] ? A1 : A0;
    const int32_t nl = (int32_t)ctrl[4 + ctrl[9]];
    int64_t k = (int64_t)ctrl[10], steps = (int64_t)ctrl[11];
    int32_t* sc = reinterpret_cast<int32_t*>(psm);              // [0] frontier count, [1] smallest kept count
    int32_t* sv = sc + 4;                                         // vertex of each slot
    int32_t* sd = sv + PEEL_SOLO;                                 // its count
    int32_t* fa = sd + PEEL_SOLO;                                 // frontiers (slots)
    int32_t* fb = fa + PEEL_SOLO;
    uint8_t* sl = reinterpret_cast<uint8_t*>(fb + PEEL_SOLO);     // live flag
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int i = tid; i < nl; i += bd) {
        const int32_t x = list[i];
        sv[i] = x;
        sd[i] = deg[x];
        sl[i] = alive[x];
        slot[x] = i;
    }
    __syncthreads();
    for (;;) {
        if (++steps > max_steps) {
            if (tid == 0) ctrl[3] = 1;
            return;
        }
        if (tid == 0) {
            sc[0] = 0;
            sc[1] = INT_MAX;
        }
        __syncthreads();
        // level scan: live vertices with count <= k are peeled at k
        for (int i = tid; i < nl; i += bd)
            if (sl[i]) {
                const int32_t d = sd[i];
                if (d <= k) {
                    sl[i] = 0;
                    core[sv[i]] = k;
                    fa[atomicAdd(sc, 1)] = i;
                } else {
                    atomicMin(sc + 1, d);
                }
            }
        __syncthreads();
        int32_t nf = sc[0];
        const int32_t mn = sc[1];
        __syncthreads();
        if (nf == 0) {
            if (mn == INT_MAX) {
                if (tid == 0) {
                    ctrl[6] = (unsigned long long)steps;
                    ctrl[7] = (unsigned long long)k;
                }
                return;
            }
            k = max(k + 1, (int64_t)mn);
            continue;
        }
        int32_t* cf = fa;
        int32_t* nx = fb;
        while (nf > 0) {
            if (++steps > max_steps) {
                if (tid == 0) ctrl[3] = 1;
                return;
            }
            if (tid == 0) sc[0] = 0;
            __syncthreads();
            // a vertex whose count falls from k + 1 to k is peeled at k
            auto drop = [&](int32_t y) {
                const int32_t j = slot[y];
                if (j >= 0 && atomicSub(sd + j, 1) == k + 1) {
                    sl[j] = 0;
                    core[y] = k;
                    nx[atomicAdd(sc, 1)] = j;
                }
            };
            for (int32_t base = 0; base < nf; base += bd) {
                const int32_t j = base + tid;
                int64_t d = 0, b0 = 0;
                int32_t x = -1;
                if (j < nf) {
                    x = sv[cf[j]];
                    b0 = ptr[x];
                    d = ptr[x + 1] - b0;
                }
                const int64_t total = block_scan_i64(d, b_off, wsum);
                b_x[tid] = x;
                b_beg[tid] = b0;
                __syncthreads();
                const int32_t cnt = min(bd, nf - base);
                for (int64_t i = tid; i < total; i += bd) {
                    int32_t lo = 0, hi = cnt;            // last entry with offset <= i
                    while (hi - lo > 1) {
                        const int32_t mid = (lo + hi) >> 1;
                        if (b_off[mid] <= i) lo = mid; else hi = mid;
                    }
                    const int32_t xv = b_x[lo];
                    const int32_t e = adj[b_beg[lo] + (i - b_off[lo])];
                    if (!tri) {
                        drop(e);
                    } else {
                        unsigned int* word = (unsigned int*)(tdead + (e & ~3));
                        const unsigned int bit = 1u << (8 * (e & 3));
                        if (atomicOr(word, bit) & bit) continue;      // died with another vertex
                        const int32_t va = ta[e], vb = tb[e], vc = tc[e];
                        if (va != xv) drop(va);
                        if (vb != xv) drop(vb);
                        if (vc != xv) drop(vc);
                    }
                }
                __syncthreads();
            }
            nf = sc[0];
            __syncthreads();
            int32_t* t = cf;
            cf = nx;
            nx = t;
        }
        k = k + 1;
    }
}

// Whole peeling loop in one cooperative launch (peeling by levels).  A level k
// starts with a scan of the live-vertex list: vertices with count <= k are
// peeled (core k) into the frontier, the others go to the other list, and the
// smallest kept count is recorded; an empty frontier moves k to
// max(k + 1, that minimum) and scans again.  Frontier rounds then remove the
// frontier and collect the vertices that fall to k: a lane removes a vertex
// with few incidences itself, and the incidences of the others are cut into
// chunks that all warps share, so a hub does not hold up the round.  Once the
// live list is down to `solo` (at most PEEL_SOLO) vertices, the grid stops and
// peel_solo_kernel finishes in one block: block barriers cost far less than
// grid barriers over the many small levels of the dense tail.
// ctrl: [0..1] frontier counts, [2] smallest kept count, [3] error (bound hit),
// [4..5] live-list counts, [6..7] steps and last level (reported at the end),
// [8] chunk count, [9..12] the hand-over (live list, level, steps, flag).  Every
// thread follows the same k and the same branches: the counters are read right
// after a barrier.
__global__ void __launch_bounds__(1024, 1) peel_coop_kernel(bool tri, const int64_t* rowptr, const int32_t* col,
                                                            const int64_t* vptr, const int32_t* vtri,
                                                            const int32_t* ta, const int32_t* tb, const int32_t* tc,
                                                            uint8_t* tdead, uint8_t* alive, int32_t* deg,
                                                            int64_t* core, int32_t* F0, int32_t* F1, int32_t* A0,
                                                            int32_t* A1, int32_t* qv, int64_t* qs,
                                                            unsigned long long* ctrl, int64_t max_steps,
                                                            int64_t solo) {
    cg::grid_group grid = cg::this_grid();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t warp = tid >> 5, nwarps = nthreads >> 5;
    auto barrier = [&]() { grid.sync(); };
    auto rd = [&](int i) -> unsigned long long { return __ldcg(ctrl + i); };
    const int64_t* ptr = tri ? vptr : rowptr;
    const int32_t* adj = tri ? vtri : col;
    auto F = [&](int i) { return i ? F1 : F0; };
    auto A = [&](int i) { return i ? A1 : A0; };
    int cur = 0, a = 0;
    int64_t k = 0, steps = 0;
    for (;;) {
        if (++steps > max_steps) {
            if (tid == 0) ctrl[3] = 1;
            return;
        }
        const int64_t na = (int64_t)rd(4 + a);
        if (na <= solo) {
            // peel_solo_kernel, launched next, finishes in one block
            if (tid == 0) {
                ctrl[9] = (unsigned long long)a;
                ctrl[10] = (unsigned long long)k;
                ctrl[11] = (unsigned long long)(steps - 1);
                ctrl[12] = 1;
            }
            return;
        }
        // level scan, warp by warp: one atomic per warp for each list and for the minimum
        for (int64_t base = tid - lane; base < na; base += nthreads) {
            const int64_t i = base + lane;
            int32_t x = -1, d = 0;
            bool peel = false, keep = false;
            if (i < na) {
                x = __ldcg(A(a) + i);
                if (__ldcg(alive + x)) {
                    d = __ldcg(deg + x);
                    peel = d <= k;
                    keep = !peel;
                }
            }
            const unsigned pm = __ballot_sync(0xffffffffu, peel), km = __ballot_sync(0xffffffffu, keep);
            const unsigned dmin = __reduce_min_sync(0xffffffffu, keep ? (unsigned)d : 0xffffffffu);
            unsigned long long pb = 0, kb = 0;
            if (lane == 0) {
                if (pm) pb = atomicAdd(ctrl + cur, (unsigned long long)__popc(pm));
                if (km) {
                    kb = atomicAdd(ctrl + 5 - a, (unsigned long long)__popc(km));
                    atomicMin(ctrl + 2, (unsigned long long)dmin);
                }
            }
            pb = __shfl_sync(0xffffffffu, pb, 0);
            kb = __shfl_sync(0xffffffffu, kb, 0);
            const unsigned below = (1u << lane) - 1u;
            if (peel) {
                alive[x] = 0;
                core[x] = k;
                F(cur)[pb + __popc(pm & below)] = x;
            }
            if (keep) A(1 - a)[kb + __popc(km & below)] = x;
        }
        barrier();
        unsigned long long f = rd(cur);
        const unsigned long long kept = rd(5 - a);
        const unsigned long long mn = rd(2);
        barrier();
        if (tid == 0) {
            ctrl[4 + a] = 0;
            ctrl[2] = ~0ull;
        }
        a = 1 - a;
        if (f == 0) {
            if (kept == 0) {
                if (tid == 0) {
                    ctrl[6] = (unsigned long long)steps;
                    ctrl[7] = (unsigned long long)k;
                }
                return;
            }
            k = max(k + 1, (int64_t)mn);
            barrier();
            continue;
        }
        // frontier rounds at level k
        while (f > 0) {
            if (++steps > max_steps) {
                if (tid == 0) ctrl[3] = 1;
                return;
            }
            int32_t* fr = F(cur);
            int32_t* nx = F(1 - cur);
            unsigned long long* ncnt = ctrl + (1 - cur);
            // light vertices by their lane; chunks of the heavy ones into the queue
            for (int64_t base = warp * 32; base < (int64_t)f; base += nwarps * 32) {
                const int64_t i = base + lane;
                int32_t x = -1;
                int64_t b = 0, len = 0;
                if (i < (int64_t)f) {
                    x = __ldcg(fr + i);
                    b = ptr[x];
                    len = ptr[x + 1] - b;
                }
                if (len <= PEEL_LIGHT) {
                    int32_t it[PEEL_LIGHT];
#pragma unroll
                    for (int j = 0; j < PEEL_LIGHT; ++j) it[j] = j < len ? adj[b + j] : -1;
#pragma unroll
                    for (int j = 0; j < PEEL_LIGHT; ++j)
                        if (it[j] >= 0) {
                            if (tri) peel_triangle(it[j], x, k, ta, tb, tc, tdead, alive, deg, core, nx, ncnt);
                            else peel_drop(it[j], k, alive, deg, core, nx, ncnt);
                        }
                }
                const int32_t nch = len > PEEL_LIGHT ? (int32_t)((len + PEEL_CHUNK - 1) / PEEL_CHUNK) : 0;
                int32_t incl = nch;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int32_t tot = __shfl_sync(0xffffffffu, incl, 31);
                unsigned long long cb = 0;
                if (lane == 0 && tot) cb = atomicAdd(ctrl + 8, (unsigned long long)tot);
                cb = __shfl_sync(0xffffffffu, cb, 0);
                for (int32_t c = 0; c < nch; ++c) {
                    const unsigned long long at = cb + (unsigned long long)(incl - nch + c);
                    qv[at] = x;
                    qs[at] = b + (int64_t)c * PEEL_CHUNK;
                }
            }
            barrier();
            const int64_t nq = (int64_t)rd(8);
            for (int64_t c = warp; c < nq; c += nwarps) {
                const int32_t x = __ldcg(qv + c);
                const int64_t q0 = __ldcg(qs + c);
                const int64_t q1 = min(q0 + (int64_t)PEEL_CHUNK, ptr[x + 1]);
                int32_t it[PEEL_CHUNK / 32];
#pragma unroll
                for (int j = 0; j < PEEL_CHUNK / 32; ++j) {
                    const int64_t q = q0 + lane + 32 * j;
                    it[j] = q < q1 ? adj[q] : -1;
                }
#pragma unroll
                for (int j = 0; j < PEEL_CHUNK / 32; ++j)
                    if (it[j] >= 0) {
                        if (tri) peel_triangle(it[j], x, k, ta, tb, tc, tdead, alive, deg, core, nx, ncnt);
                        else peel_drop(it[j], k, alive, deg, core, nx, ncnt);
                    }
            }
            barrier();
            f = rd(1 - cur);
            barrier();
            if (tid == 0) {
                ctrl[cur] = 0;
                ctrl[8] = 0;
            }
            cur = 1 - cur;
            barrier();
        }
        k = k + 1;
    }
}

// list of the live vertices
__global__ void alive_list_kernel(const uint8_t* alive, int32_t nact, int32_t* list, unsigned long long* cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride)
        if (alive[x]) list[agg_slot(cnt)] = (int32_t)x;
}

}  // namespace

void ensure_triangles(lds_graph* g) {
    if (g->ntri >= 0) return;
    cudaStream_t s = g->stream;
    const int32_t nact = g->nact;
    const int blk = 256;
    if (g->m == 0 || nact == 0) {
        g->ntri = 0;
        return;
    }
    DevBuf<int32_t> outdeg(nact + 1, s);
    LDS_CUDA(cudaMemsetAsync(outdeg.get(), 0, (nact + 1) * sizeof(int32_t), s));
    LDS_LAUNCH(orient_count_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), g->col.get(), nact, outdeg.get());
    LDS_CHECK_LAUNCH();
    DevBuf<int64_t> optr(nact + 1, s);
    int64_t nos = exclusive_scan_i32_to_i64(outdeg.get(), optr.get(), nact + 1, s);
    LDS_REQUIRE(nos == g->m, LDS_ECUDA, "triangle listing: orientation lost edges (internal error)");
    DevBuf<int32_t> ocol(nos, s), osrc(nos, s);
    LDS_LAUNCH(orient_fill_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), g->col.get(), nact, optr.get(), ocol.get());
    LDS_LAUNCH(oriented_src_kernel, grid_for(nact, blk), blk, 0, s, optr.get(), nact, osrc.get());
    LDS_CHECK_LAUNCH();
    DevBuf<int64_t> cnt(nos, s), off(nos, s);
    LDS_LAUNCH(tri_intersect_kernel<false>, grid_for(nos, blk), blk, 0, s, optr.get(), ocol.get(), osrc.get(), nos, cnt.get(),
                                                                   nullptr, nullptr, nullptr, nullptr);
    LDS_CHECK_LAUNCH();
    int64_t ntri = exclusive_scan_i64(cnt.get(), off.get(), nos, s);
    LDS_REQUIRE(ntri < ((int64_t)1 << 32), LDS_EOVERFLOW, "triangle listing: |T| = %lld exceeds 2^32",
                (long long)ntri);
    DevBuf<int32_t> a(ntri, s), b(ntri, s), c(ntri, s);
    if (ntri) {
        LDS_LAUNCH(tri_intersect_kernel<true>, grid_for(nos, blk), blk, 0, s, optr.get(), ocol.get(), osrc.get(), nos, nullptr,
                                                                      off.get(), a.get(), b.get(), c.get());
        LDS_CHECK_LAUNCH();
    }
    cnt.release(); off.release(); ocol.release(); osrc.release(); optr.release(); outdeg.release();
    g->ta.alloc(ntri, s);
    g->tb.alloc(ntri, s);
    g->tc.alloc(ntri, s);
    if (ntri) {
        DevBuf<uint64_t> key(ntri, s);
        DevBuf<uint32_t> idx(ntri, s);
        const uint64_t nn = (uint64_t)nact;
        LDS_LAUNCH(tri_key_bc_kernel, grid_for(ntri, blk), blk, 0, s, b.get(), c.get(), ntri, (int64_t)nn, key.get(), idx.get());
        LDS_CHECK_LAUNCH();
        radix_sort_u64(key.get(), idx.get(), ntri, bit_length_u64(nn * nn), s);
        LDS_LAUNCH(tri_key_a_kernel, grid_for(ntri, blk), blk, 0, s, a.get(), idx.get(), ntri, key.get());
        LDS_CHECK_LAUNCH();
        radix_sort_u64(key.get(), idx.get(), ntri, bit_length_u64(nn), s);
        LDS_LAUNCH(permute3_kernel, grid_for(ntri, blk), blk, 0, s, a.get(), b.get(), c.get(), idx.get(), ntri, g->ta.get(),
                                                            g->tb.get(), g->tc.get());
        LDS_CHECK_LAUNCH();
    }
    LDS_CUDA(cudaStreamSynchronize(s));
    g->ntri = ntri;
    g->info.triangles = ntri;
}

// Core (tr-core) numbers of G[alive] in internal ids: core_int[nact]; vertices
// outside `init_alive` (device mask, NULL = every vertex) get -1.
static void core_numbers_internal(lds_graph* g, bool tri, int64_t* core_int, const uint8_t* init_alive) {
    cudaStream_t s = g->stream;
    const int32_t nact = g->nact;
    const int blk = 256;
    if (nact == 0) return;
    DevBuf<int32_t> deg(nact, s), frontier(nact, s);
    DevBuf<uint8_t> alive(nact, s);
    DevBuf<int32_t> nalive(1, s);
    LDS_CUDA(cudaMemsetAsync(nalive.get(), 0, sizeof(int32_t), s));
    LDS_LAUNCH(alive_init_kernel, grid_for(nact, blk), blk, 0, s, init_alive, nact, alive.get(), core_int, nalive.get());
    DevBuf<uint8_t> tdead;
    LDS_CUDA(cudaMemsetAsync(deg.get(), 0, nact * sizeof(int32_t), s));
    // the triangle list the peeling walks: all of T, or, when few vertices are alive,
    // only the triangles whose three members are alive (the others never count)
    DevBuf<int32_t> cta, ctb, ctc, cvi;
    DevBuf<int64_t> cvp;
    const int64_t* tvp = nullptr;
    const int32_t *tvi = nullptr, *tta = nullptr, *ttb = nullptr, *ttc = nullptr;
    int64_t tnt = 0;
    if (!tri) {
        LDS_LAUNCH(alive_degree_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), g->col.get(), alive.get(), nact,
                   deg.get());
    } else {
        ensure_triangles(g);
        int32_t nal = 0;
        LDS_CUDA(cudaMemcpyAsync(&nal, nalive.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        if (init_alive && (int64_t)nal * 4 < (int64_t)nact && g->ntri) {
            const int64_t ntri = g->ntri;
            DevBuf<int32_t> flag(ntri + 1, s);
            DevBuf<int64_t> tpos(ntri + 1, s);
            LDS_CUDA(cudaMemsetAsync(flag.get() + ntri, 0, sizeof(int32_t), s));
            LDS_LAUNCH(tri_all_alive_kernel, grid_for(ntri, blk), blk, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), ntri,
                       alive.get(), flag.get());
            tnt = exclusive_scan_i32_to_i64(flag.get(), tpos.get(), ntri + 1, s);
            cta.alloc(std::max<int64_t>(tnt, 1), s);
            ctb.alloc(std::max<int64_t>(tnt, 1), s);
            ctc.alloc(std::max<int64_t>(tnt, 1), s);
            if (tnt)
                LDS_LAUNCH(tri_compact_kernel, grid_for(ntri, blk), blk, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), ntri,
                           flag.get(), tpos.get(), cta.get(), ctb.get(), ctc.get());
            build_vertex_triangles(cta.get(), ctb.get(), ctc.get(), tnt, nact, cvp, cvi, s);
            tvp = cvp.get();
            tvi = cvi.get();
            tta = cta.get();
            ttb = ctb.get();
            ttc = ctc.get();
        } else {
            ensure_vertex_triangles(g);
            tnt = g->ntri;
            tvp = g->vt_ptr.get();
            tvi = g->vt_idx.get();
            tta = g->ta.get();
            ttb = g->tb.get();
            ttc = g->tc.get();
        }
        tdead.alloc(((tnt + 3) & ~3ll) + 4, s);
        LDS_CUDA(cudaMemsetAsync(tdead.get(), 0, ((tnt + 3) & ~3ll) + 4, s));
        if (tnt)
            LDS_LAUNCH(alive_tri_count_kernel, grid_for(tnt, blk), blk, 0, s, tta, ttb, ttc, tnt, alive.get(), deg.get(),
                       tdead.get());
    }
    int32_t remaining = 0;
    LDS_CUDA(cudaMemcpyAsync(&remaining, nalive.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    if (remaining == 0) return;
    // every vertex alive: the whole graph's core numbers, peeled once per handle
    DevBuf<int64_t>& whole = g->core_all[tri ? 1 : 0];
    const bool all_alive = remaining == nact;
    if (all_alive && whole.p) {
        LDS_CUDA(cudaMemcpyAsync(core_int, whole.get(), (size_t)nact * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        return;
    }
    // one cooperative launch runs every level; the grid must be resident at once
    DevBuf<unsigned long long> ctrl(13, s);
    unsigned long long hctrl[13] = {0ull, 0ull, ~0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    LDS_CUDA(cudaMemcpyAsync(ctrl.get(), hctrl, sizeof(hctrl), cudaMemcpyHostToDevice, s));
    DevBuf<int32_t> F1(nact, s), A0(nact, s), A1(nact, s);
    // chunk queue: at most one chunk per vertex plus one per PEEL_CHUNK incidences
    const int64_t incid = tri ? 3 * tnt : 2 * g->m;
    const int64_t qcap = (int64_t)nact + incid / PEEL_CHUNK + 1;
    DevBuf<int32_t> qv(qcap, s);
    DevBuf<int64_t> qs(qcap, s);
    LDS_LAUNCH(alive_list_kernel, grid_for(nact, blk), blk, 0, s, alive.get(), nact, A0.get(), ctrl.get() + 4);
    // one block of 1024 threads per SM: grid barriers get cheaper with fewer blocks
    const int pblk = 1024;
    int per_sm = 0;
    LDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peel_coop_kernel, pblk, 0));
    LDS_CUDA(cudaFuncSetAttribute(peel_solo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PEEL_SOLO_SMEM));
    LDS_REQUIRE(per_sm > 0, LDS_ECUDA, "core numbers: peeling kernel cannot be resident");
    int grid = std::max(1, std::min(num_sms(), (int)((nact + pblk - 1) / pblk)));
    int64_t max_steps = 4 * (int64_t)nact + 64;
    // the one-block tail only for edges: a triangle tail's incidences (hub
    // triangles) keep the whole grid busy (R-MAT 20: 3.1 s instead of 5.9 s per
    // LTDS query with the tail in one block)
    int64_t solo = tri ? 0 : PEEL_SOLO;
    DevBuf<int32_t> slotb(nact, s);
    LDS_CUDA(cudaMemsetAsync(slotb.get(), 0xff, (size_t)nact * sizeof(int32_t), s));
    int32_t* slp = slotb.get();
    bool trib = tri;
    const int64_t* rp = g->rowptr.get();
    const int32_t* cl = g->col.get();
    const int64_t* vp = tri ? tvp : nullptr;
    const int32_t* vi = tri ? tvi : nullptr;
    const int32_t* pa = tri ? tta : nullptr;
    const int32_t* pb = tri ? ttb : nullptr;
    const int32_t* pc = tri ? ttc : nullptr;
    uint8_t* td = tri ? tdead.get() : nullptr;
    uint8_t* al = alive.get();
    int32_t* dg = deg.get();
    int32_t* f0 = frontier.get();
    int32_t* f1 = F1.get();
    int32_t* a0 = A0.get();
    int32_t* a1 = A1.get();
    unsigned long long* ct = ctrl.get();
    int32_t* qvp = qv.get();
    int64_t* qsp = qs.get();
    void* args[] = {(void*)&trib, (void*)&rp, (void*)&cl, (void*)&vp, (void*)&vi, (void*)&pa, (void*)&pb, (void*)&pc,
                    (void*)&td, (void*)&al, (void*)&dg, (void*)&core_int, (void*)&f0, (void*)&f1, (void*)&a0,
                    (void*)&a1, (void*)&qvp, (void*)&qsp, (void*)&ct, (void*)&max_steps, (void*)&solo};
    const char* vb = getenv("LDS_VERBOSE");
    const bool verbose = vb && vb[0] == '1';
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (verbose) {
        LDS_CUDA(cudaEventCreate(&e0));
        LDS_CUDA(cudaEventCreate(&e1));
        LDS_CUDA(cudaEventRecord(e0, s));
    }
    LDS_CUDA(cudaLaunchCooperativeKernel((void*)peel_coop_kernel, dim3(grid), dim3(pblk), args, 0, s));
    LDS_LAUNCH(peel_solo_kernel, 1, PEEL_SOLO_T, PEEL_SOLO_SMEM, s, trib, tri ? tvp : g->rowptr.get(),
               tri ? tvi : g->col.get(), pa, pb, pc, td, al, dg, core_int, a0, a1, slp, ct, max_steps);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (verbose) LDS_CUDA(cudaEventRecord(e1, s));
    LDS_CUDA(cudaMemcpyAsync(hctrl, ctrl.get(), sizeof(hctrl), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    if (verbose) {
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        fprintf(stderr, "[core] nact=%d live=%d peel %.2f ms, %llu steps, last level %llu, grid %d\n", nact, remaining,
                ms, hctrl[6], hctrl[7], grid);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    LDS_REQUIRE(hctrl[3] == 0, LDS_ETIMEOUT, "core numbers: peeling hit its iteration bound");
    if (all_alive) {
        whole.alloc(nact, s);
        LDS_CUDA(cudaMemcpyAsync(whole.get(), core_int, (size_t)nact * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    }
}

void core_numbers(lds_graph* g, bool tri, int64_t* core_int_out, const uint8_t* init_alive) {
    core_numbers_internal(g, tri, core_int_out, init_alive);
}

}  // namespace lds

using namespace lds;

extern "C" {

lds_status lds_list_triangles(lds_graph* g, int64_t* count) {
    return guard([&] {
        LDS_REQUIRE(g, LDS_EINVAL, "lds_list_triangles: NULL graph");
        ensure_triangles(g);
        if (count) *count = g->ntri;
    });
}

lds_status lds_get_triangles(lds_graph* g, int32_t* tri, lds_mem where) {
    return guard([&] {
        LDS_REQUIRE(g && tri, LDS_EINVAL, "lds_get_triangles: NULL argument");
        LDS_REQUIRE(g->ntri >= 0, LDS_EINVAL, "lds_get_triangles: call lds_list_triangles first");
        if (g->ntri == 0) return;
        cudaStream_t s = g->stream;
        DevBuf<int32_t> rows(3 * g->ntri, s);
        LDS_LAUNCH(tri_rows_orig_kernel, grid_for(g->ntri, 256), 256, 0, s, g->ta.get(), g->tb.get(), g->tc.get(),
                                                                    g->to_orig.get(), g->ntri, rows.get());
        LDS_CHECK_LAUNCH();
        copy_out(tri, where, rows.get(), 3 * g->ntri * sizeof(int32_t), s);
        LDS_CUDA(cudaStreamSynchronize(s));
    });
}

lds_status lds_core_numbers(lds_graph* g, lds_density d, int64_t* core, lds_mem where) {
    return guard([&] {
        LDS_REQUIRE(g && core, LDS_EINVAL, "lds_core_numbers: NULL argument");
        LDS_REQUIRE(d == LDS_EDGE || d == LDS_TRIANGLE, LDS_EINVAL, "lds_core_numbers: bad density");
        cudaStream_t s = g->stream;
        const int32_t n = g->n;
        if (n == 0) return;
        DevBuf<int64_t> ci(n, s), co(n, s);
        LDS_CUDA(cudaMemsetAsync(ci.get(), 0, n * sizeof(int64_t), s));
        core_numbers_internal(g, d == LDS_TRIANGLE, ci.get(), nullptr);
        to_original_order_i64(g, ci.get(), co.get());
        copy_out(core, where, co.get(), n * sizeof(int64_t), s);
        LDS_CUDA(cudaStreamSynchronize(s));
    });
}

}  // extern "C"
