// Candidate verification on the GPU: IsDensest (Sec. 5.4), IsLDS (Alg. 4),
// IsLTDS (Alg. 7) with ExtMaximal (Alg. 8), plus the helpers the driver needs
// (connected components of G[S], subgraph handles, exact compact numbers of a
// small vertex set).
//
// IsDensest(S): G[S] is its own densest subgraph iff the pattern network over
// S (patterns E(S) or T(S), rho = density) saturates every source arc, i.e.
// the maximum flow is q |P| for rho = p / q.
//
// IsLDS(S): rho = |E(S)| / |S|.  A neighbour w outside S with lb(w) > rho
// rejects S at once (phi(w) > rho, Lemma 3).  Otherwise U is grown from S over
// neighbours w with lb(w) <= rho <= ub(w) (a level-synchronous search; the set
// does not depend on the visiting order), every edge from a U vertex v to a
// vertex w outside U with lb(w) > rho becomes a loop pattern {v}, and the
// maximum flow over U with patterns E(U) plus the loops yields A, the largest
// source side (= {u in U : phi(u) >= rho}, Lemma 9).  S is an LDS iff S is a
// connected component of G[A].  When U = S no flow is needed.
//
// IsLTDS(S): the same with tr-density; the patterns are, for every triangle
// with a vertex in U and all three upper bounds >= rho, its vertices with
// lb <= rho (Alg. 7).  Those vertices are reached by the edge search as well,
// so U is the same edge-grown set.
#include <cooperative_groups.h>

#include <algorithm>
#include <numeric>

#include "flow.cuh"
#include "prims.cuh"
#include "verify.cuh"

namespace lds {

namespace {

typedef __int128 i128;
constexpr int VB = 256;

// num / den compared with p / q
__device__ __forceinline__ bool gt_rho(int64_t num, int64_t den, int64_t p, int64_t q) {
    return (i128)num * q > (i128)p * den;
}
__device__ __forceinline__ bool lt_rho(int64_t num, int64_t den, int64_t p, int64_t q) {
    return (i128)num * q < (i128)p * den;
}

__global__ void mark_kernel(const int32_t* list, int32_t k, uint8_t* flag, int32_t* local) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        flag[list[i]] = 1;
        if (local) local[list[i]] = (int32_t)i;
    }
}

__global__ void unmark_kernel(const int32_t* list, int32_t k, uint8_t* flag) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) flag[list[i]] = 0;
}

// Warp-per-member helpers: lane l takes slots l, l + 32, ... of the member's row;
// outputs keep the row's order (ballot + prefix popcount), as one thread would.
#define WARP_MEMBER_LOOP(k)                                                        \
    const int lane = threadIdx.x & 31;                                             \
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;                \
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < (k); i += wstride)

__device__ __forceinline__ unsigned lanes_below(int lane) { return (1u << lane) - 1u; }

// per member x: number of edge patterns it owns (neighbours y in the set with y > x)
__global__ void edge_pat_count_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* rowptr,
                                      const int32_t* col, const uint8_t* in, int32_t* cnt) {
    WARP_MEMBER_LOOP(k) {
        const int32_t x = list[i];
        int32_t c = 0;
        if (x < nact)
            for (int64_t q = rowptr[x] + lane; q < rowptr[x + 1]; q += 32) {
                const int32_t y = col[q];
                c += (y > x && in[y]);
            }
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[i] = c;
    }
}

// share (optional): the Frank-Wolfe split of each edge, W = D alpha for its
// lower endpoint x and D - W for y
__global__ void edge_pat_fill_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* rowptr,
                                     const int32_t* col, const uint8_t* in, const int32_t* local, const int64_t* off,
                                     int32_t* pidx, const int64_t* slot_edge, const int64_t* W, int64_t D,
                                     int64_t* share) {
    WARP_MEMBER_LOOP(k) {
        const int32_t x = list[i];
        if (x >= nact) continue;
        int64_t o = off[i];
        const int64_t b = rowptr[x], e = rowptr[x + 1];
        for (int64_t q0 = b; q0 < e; q0 += 32) {
            const int64_t q = q0 + lane;
            bool take = false;
            int32_t y = 0;
            if (q < e) {
                y = col[q];
                take = y > x && in[y];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int64_t at = o + __popc(bal & lanes_below(lane));
                pidx[2 * at] = (int32_t)i;
                pidx[2 * at + 1] = local[y];
                if (share) {
                    const int64_t w = W[slot_edge[q]];
                    share[2 * at] = w;
                    share[2 * at + 1] = D - w;
                }
            }
            o += __popc(bal);
        }
    }
}

// loops: members v with neighbours w outside the set and lb(w) > rho
__global__ void loop_count_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* rowptr, const int32_t* col,
                                  const uint8_t* in, const int64_t* ln, const int64_t* ld, int64_t p, int64_t q,
                                  int32_t* cnt) {
    WARP_MEMBER_LOOP(k) {
        const int32_t x = list[i];
        int32_t c = 0;
        if (x < nact)
            for (int64_t r = rowptr[x] + lane; r < rowptr[x + 1]; r += 32) {
                const int32_t w = col[r];
                c += (!in[w] && gt_rho(ln[w], ld[w], p, q));
            }
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void uniform_pat_ptr_kernel(int64_t np, int64_t width, int64_t* pptr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= np; j += stride) pptr[j] = j * width;
}

__global__ void loop_fill_kernel(const int32_t* cnt, const int64_t* off, int32_t k, int32_t* pidx, int64_t base,
                                 int64_t* share) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride)
        for (int32_t c = 0; c < cnt[i]; ++c) {
            pidx[base + off[i] + c] = (int32_t)i;
            if (share) share[base + off[i] + c] = 1;
        }
}

// ---- triangle patterns over the incidences of the set: one work item per
// (member, incident triangle) pair, so that hubs with millions of triangles
// are shared by the whole grid.  ioff is the exclusive prefix of the members'
// triangle counts.  A triangle is taken by its smallest member in the set.

__global__ void tri_inc_count_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* vt_ptr,
                                     int32_t* icnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        const int32_t x = list[i];
        icnt[i] = x < nact ? (int32_t)(vt_ptr[x + 1] - vt_ptr[x]) : 0;
    }
}

__device__ __forceinline__ int32_t tri_inc_member(const int64_t* ioff, int32_t k, int64_t item) {
    int32_t lo = 0, hi = k;                  // last i with ioff[i] <= item
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (ioff[mid] <= item) lo = mid; else hi = mid;
    }
    return lo;
}

// members of triangle t that form its pattern (mask of columns), 0 when t is not
// taken by x: all three in the set (all_in), else Alg. 7's reduction (all
// ub >= rho; the members in the set with lb <= rho)
__device__ __forceinline__ int tri_pattern_mask(int32_t x, int32_t t, const int32_t* ta, const int32_t* tb,
                                                const int32_t* tc, const uint8_t* in, bool all_in,
                                                const int64_t* un, const int64_t* ud, const int64_t* ln,
                                                const int64_t* ld, int64_t p, int64_t q) {
    const int32_t v[3] = {ta[t], tb[t], tc[t]};
    int32_t owner = -1;
    for (int j = 0; j < 3; ++j)
        if (in[v[j]] && (owner < 0 || v[j] < owner)) owner = v[j];
    if (owner != x) return 0;
    if (all_in) return (in[v[0]] && in[v[1]] && in[v[2]]) ? 7 : 0;
    for (int j = 0; j < 3; ++j)
        if (lt_rho(un[v[j]], ud[v[j]], p, q)) return 0;
    int mask = 0;
    for (int j = 0; j < 3; ++j)
        if (in[v[j]] && !gt_rho(ln[v[j]], ld[v[j]], p, q)) mask |= 1 << j;
    return mask;
}

// per item: 1 if it takes a pattern, and the pattern's length
__global__ void tri_item_count_kernel(const int32_t* list, int32_t k, const int64_t* ioff, int64_t nitems,
                                      const int64_t* vt_ptr, const int32_t* vt_idx, const int32_t* ta,
                                      const int32_t* tb, const int32_t* tc, const uint8_t* in, bool all_in,
                                      const int64_t* un, const int64_t* ud, const int64_t* ln, const int64_t* ld,
                                      int64_t p, int64_t q, int32_t* take, int32_t* len) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nitems; it += stride) {
        const int32_t i = tri_inc_member(ioff, k, it);
        const int32_t x = list[i];
        const int32_t t = vt_idx[vt_ptr[x] + (it - ioff[i])];
        const int mask = tri_pattern_mask(x, t, ta, tb, tc, in, all_in, un, ud, ln, ld, p, q);
        take[it] = mask != 0;
        if (len) len[it] = __popc(mask);
    }
}

// per taking item: its pattern's start (slot offset) and members, with the
// Frank-Wolfe split of each member when share is given
__global__ void tri_item_fill_kernel(const int32_t* list, int32_t k, const int64_t* ioff, int64_t nitems,
                                     const int64_t* vt_ptr, const int32_t* vt_idx, const int32_t* ta,
                                     const int32_t* tb, const int32_t* tc, const uint8_t* in, const int32_t* local,
                                     bool all_in, const int64_t* un, const int64_t* ud, const int64_t* ln,
                                     const int64_t* ld, int64_t p, int64_t q, const int64_t* patpos,
                                     const int64_t* slotpos, int64_t* pptr, int32_t* pidx, const int64_t* W,
                                     int64_t* share) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nitems; it += stride) {
        const int32_t i = tri_inc_member(ioff, k, it);
        const int32_t x = list[i];
        const int32_t t = vt_idx[vt_ptr[x] + (it - ioff[i])];
        const int mask = tri_pattern_mask(x, t, ta, tb, tc, in, all_in, un, ud, ln, ld, p, q);
        if (!mask) continue;
        const int32_t v[3] = {ta[t], tb[t], tc[t]};
        int64_t at = slotpos ? slotpos[it] : 3 * patpos[it];
        if (pptr) pptr[patpos[it]] = at;
        for (int j = 0; j < 3; ++j)
            if (mask & (1 << j)) {
                if (share) share[at] = W[3 * (int64_t)t + j];
                pidx[at++] = local[v[j]];
            }
    }
}

__global__ void add_offset_i64_kernel(int64_t* p, int64_t k, int64_t off) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) p[i] += off;
}

__global__ void widen_i32_u64_kernel(const int32_t* in, int64_t k, uint64_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = (uint64_t)in[i];
}

__global__ void narrow_u64_i32_kernel(const uint64_t* in, int64_t k, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = (int32_t)in[i];
}

// one level of the search that grows U over neighbours with lb <= rho <= ub
// (with use_lb = false: over neighbours with ub >= rho, the IsLDS-core search)
__global__ void grow_level_kernel(const int32_t* frontier, int32_t fsize, int32_t nact, const int64_t* rowptr,
                                  const int32_t* col, uint8_t* inU, const int64_t* un, const int64_t* ud,
                                  const int64_t* ln, const int64_t* ld, int64_t p, int64_t q, bool use_lb,
                                  int32_t* next, int32_t* nsize) {
    WARP_MEMBER_LOOP(fsize) {
        const int32_t x = frontier[i];
        if (x >= nact) continue;
        for (int64_t r = rowptr[x] + lane; r < rowptr[x + 1]; r += 32) {
            const int32_t w = col[r];
            if (inU[w]) continue;
            if (use_lb && gt_rho(ln[w], ld[w], p, q)) continue;   // loop side, never joins U
            if (lt_rho(un[w], ud[w], p, q)) continue;         // phi(w) < rho
            unsigned int* word = (unsigned int*)(inU + (w & ~3));
            unsigned int bit = 1u << (8 * (w & 3));
            if (!(atomicOr(word, bit) & bit)) next[atomicAdd(nsize, 1)] = w;
        }
    }
}

// any neighbour outside S with lb > rho
__global__ void denser_neighbour_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* rowptr,
                                        const int32_t* col, const uint8_t* inS, const int64_t* ln, const int64_t* ld,
                                        int64_t p, int64_t q, int32_t* flag) {
    WARP_MEMBER_LOOP(k) {
        const int32_t x = list[i];
        if (x >= nact) continue;
        for (int64_t r = rowptr[x] + lane; r < rowptr[x + 1]; r += 32) {
            const int32_t w = col[r];
            if (!inS[w] && gt_rho(ln[w], ld[w], p, q)) {
                atomicOr(flag, 1);
                break;
            }
        }
    }
}

__global__ void iota_i32_kernel(int32_t* out, int32_t n) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (int32_t)i;
}

__global__ void collect_kernel(const uint8_t* flag, int32_t n, int32_t* out, int32_t* cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        if (flag[x]) out[atomicAdd(cnt, 1)] = (int32_t)x;
}

// S must lie in A and have no neighbour in A outside S
__global__ void component_check_kernel(const int32_t* S, int32_t k, int32_t nact, const int64_t* rowptr,
                                       const int32_t* col, const uint8_t* inS, const uint8_t* inA, int32_t* bad) {
    WARP_MEMBER_LOOP(k) {
        const int32_t x = S[i];
        if (!inA[x]) {
            if (lane == 0) atomicOr(bad, 1);
            continue;
        }
        if (x >= nact) continue;
        for (int64_t r = rowptr[x] + lane; r < rowptr[x + 1]; r += 32) {
            const int32_t w = col[r];
            if (inA[w] && !inS[w]) {
                atomicOr(bad, 1);
                break;
            }
        }
    }
}

__global__ void side_to_flag_kernel(const int32_t* U, int32_t nu, const uint8_t* side, uint8_t* inA) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += stride) inA[U[i]] = side[i];
}

// ---- components

__global__ void cc_init_kernel(const int32_t* list, int32_t k, int32_t* label) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) label[list[i]] = list[i];
}

// Every sweep of label propagation in one cooperative launch: each sweep lowers
// every member's label to the smallest label among its in-set neighbours (atomic
// minimum, so labels only fall), a grid barrier, and a stop when a sweep changed
// nothing.  flags[0..1] alternate as the sweeps' change flags; flags[2] is set
// when the sweep bound is hit.
__global__ void cc_coop_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* rowptr,
                               const int32_t* col, const uint8_t* in, int32_t* label, int32_t* flags,
                               int64_t max_sweeps) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t sweep = 0;; ++sweep) {
        if (sweep >= max_sweeps) {
            if (tid == 0) flags[2] = 1;
            return;
        }
        int32_t* changed = flags + (sweep & 1);
        // one warp per member: the lanes share its row
        const int lane = threadIdx.x & 31;
        for (int64_t i = tid >> 5; i < k; i += nthreads >> 5) {
            const int32_t x = list[i];
            if (x >= nact) continue;
            const int32_t lx = __ldcg(label + x);
            int32_t best = lx;
            for (int64_t r = rowptr[x] + lane; r < rowptr[x + 1]; r += 32) {
                const int32_t w = col[r];
                if (in[w]) best = min(best, __ldcg(label + w));
            }
            for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
            if (lane == 0 && best < lx) {
                atomicMin(label + x, best);
                *changed = 1;
            }
        }
        grid.sync();
        const int32_t c = __ldcg(changed);
        // the other flag is cleared for the next sweep; every thread has read this one
        if (tid == 0) flags[(sweep + 1) & 1] = 0;
        grid.sync();
        if (!c) return;
    }
}

__global__ void cc_keys_kernel(const int32_t* list, int32_t k, const int32_t* label, int bits, uint64_t* key) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride)
        key[i] = ((uint64_t)label[list[i]] << bits) | (uint64_t)list[i];
}

__global__ void cc_unpack_kernel(const uint64_t* key, int32_t k, int bits, int32_t* members, int32_t* starts,
                                 int32_t* nstart) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint64_t mask = (1ull << bits) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        members[i] = (int32_t)(key[i] & mask);
        if (i == 0 || (key[i] >> bits) != (key[i - 1] >> bits)) starts[atomicAdd(nstart, 1)] = (int32_t)i;
    }
}

// ---- subgraph

__global__ void sub_edges_count_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* rowptr,
                                       const int32_t* col, const uint8_t* in, int32_t* cnt) {
    WARP_MEMBER_LOOP(k) {
        const int32_t x = list[i];
        int32_t c = 0;
        if (x < nact)
            for (int64_t r = rowptr[x] + lane; r < rowptr[x + 1]; r += 32) c += (col[r] > x && in[col[r]]);
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void sub_edges_fill_kernel(const int32_t* list, int32_t k, int32_t nact, const int64_t* rowptr,
                                      const int32_t* col, const uint8_t* in, const int32_t* local, const int64_t* off,
                                      int32_t* su, int32_t* sv) {
    WARP_MEMBER_LOOP(k) {
        const int32_t x = list[i];
        if (x >= nact) continue;
        int64_t o = off[i];
        const int64_t b = rowptr[x], e = rowptr[x + 1];
        for (int64_t q0 = b; q0 < e; q0 += 32) {
            const int64_t r = q0 + lane;
            bool take = false;
            int32_t y = 0;
            if (r < e) {
                y = col[r];
                take = y > x && in[y];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int64_t at = o + __popc(bal & lanes_below(lane));
                su[at] = (int32_t)i;
                sv[at] = local[y];
            }
            o += __popc(bal);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

Scratch::Scratch(lds_graph* g) : s(g->stream) {
    in.alloc(std::max(g->n, 1) + 4, s);
    in2.alloc(std::max(g->n, 1) + 4, s);
    local.alloc(std::max(g->n, 1), s);
    LDS_CUDA(cudaMemsetAsync(in.get(), 0, std::max(g->n, 1) + 4, s));
    LDS_CUDA(cudaMemsetAsync(in2.get(), 0, std::max(g->n, 1) + 4, s));
}

static int64_t scan_counts(const int32_t* cnt, int64_t k, DevBuf<int64_t>& off, cudaStream_t s) {
    off.alloc(k + 1, s);
    DevBuf<int32_t> c1(k + 1, s);
    LDS_CUDA(cudaMemsetAsync(c1.get(), 0, (k + 1) * sizeof(int32_t), s));
    if (k) LDS_CUDA(cudaMemcpyAsync(c1.get(), cnt, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return exclusive_scan_i32_to_i64(c1.get(), off.get(), k + 1, s);
}

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Builds the pattern lists over `list` (k members, marked in sc.in with local
// indices in sc.local).  Edge density: E(list) (+ loops when `loops` is set);
// triangle density: T(list) when all_in, else Alg. 7's reduced patterns.
// With `share`, it also receives the Frank-Wolfe split of every pattern
// (aligned with pidx) when g holds Frank-Wolfe weights of the same density,
// else it is released (the flow then splits evenly).
static int64_t build_patterns(lds_graph* g, bool tri, const int32_t* list, int32_t k, Scratch& sc, bool all_in,
                              bool loops, const Bounds* b, int64_t p, int64_t q, DevBuf<int64_t>& pptr,
                              DevBuf<int32_t>& pidx, int64_t* n_main, DevBuf<int64_t>* share = nullptr) {
    cudaStream_t s = g->stream;
    const int32_t nact = g->nact;
    const bool warm = share && g->fw_valid && g->fw_density == (tri ? LDS_TRIANGLE : LDS_EDGE);
    if (share) share->release();
    DevBuf<int32_t> cnt(std::max(k, 1), s), len(std::max(k, 1), s);
    DevBuf<int64_t> off;
    if (!tri) {
        if (k) LDS_LAUNCH(edge_pat_count_kernel, grid_for((int64_t)k * 32, VB), VB, 0, s, list, k, nact, g->rowptr.get(), g->col.get(),
                          sc.in.get(), cnt.get());
        int64_t ne = scan_counts(cnt.get(), k, off, s);
        int64_t nl = 0;
        DevBuf<int32_t> lcnt(std::max(k, 1), s);
        DevBuf<int64_t> loff;
        if (loops) {
            if (k) LDS_LAUNCH(loop_count_kernel, grid_for((int64_t)k * 32, VB), VB, 0, s, list, k, nact, g->rowptr.get(), g->col.get(),
                              sc.in.get(), b->ln.get(), b->ld.get(), p, q, lcnt.get());
            nl = scan_counts(lcnt.get(), k, loff, s);
        }
        const int64_t np = ne + nl;
        pptr.alloc(np + 1, s);
        pidx.alloc(std::max<int64_t>(2 * ne + nl, 1), s);
        if (warm) {
            ensure_slot_edge(g);
            share->alloc(std::max<int64_t>(2 * ne + nl, 1), s);
        }
        int64_t* sh = warm ? share->get() : nullptr;
        // edge patterns first (width 2), then loops (width 1)
        LDS_LAUNCH(uniform_pat_ptr_kernel, grid_for(ne + 1, VB), VB, 0, s, ne, 2, pptr.get());
        if (nl) {
            DevBuf<int64_t> tail(nl + 1, s);
            LDS_LAUNCH(uniform_pat_ptr_kernel, grid_for(nl + 1, VB), VB, 0, s, nl, 1, tail.get());
            LDS_LAUNCH(add_offset_i64_kernel, grid_for(nl + 1, VB), VB, 0, s, tail.get(), nl + 1, 2 * ne);
            LDS_CUDA(cudaMemcpyAsync(pptr.get() + ne, tail.get(), (nl + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        }
        if (k && ne)
            LDS_LAUNCH(edge_pat_fill_kernel, grid_for((int64_t)k * 32, VB), VB, 0, s, list, k, nact, g->rowptr.get(), g->col.get(),
                       sc.in.get(), sc.local.get(), off.get(), pidx.get(), warm ? g->slot_edge.get() : nullptr,
                       warm ? g->fw_W.get() : nullptr, g->fw_D, sh);
        if (k && nl)
            LDS_LAUNCH(loop_fill_kernel, grid_for(k, VB), VB, 0, s, lcnt.get(), loff.get(), k, pidx.get(), 2 * ne, sh);
        if (n_main) *n_main = ne;
        return np;
    }
    ensure_vertex_triangles(g);
    const Bounds* bb = b;
    const int64_t* un = bb ? bb->un.get() : nullptr;
    const int64_t* ud = bb ? bb->ud.get() : nullptr;
    const int64_t* ln = bb ? bb->ln.get() : nullptr;
    const int64_t* ld = bb ? bb->ld.get() : nullptr;
    {
        // items = (member, incident triangle) pairs
        DevBuf<int64_t> ioff;
        if (k) LDS_LAUNCH(tri_inc_count_kernel, grid_for(k, VB), VB, 0, s, list, k, nact, g->vt_ptr.get(), cnt.get());
        const int64_t nitems = scan_counts(cnt.get(), k, ioff, s);
        DevBuf<int32_t> take(nitems + 1, s), plen(all_in ? 0 : nitems + 1, s);
        if (nitems)
            LDS_LAUNCH(tri_item_count_kernel, grid_for(nitems, VB), VB, 0, s, list, k, ioff.get(), nitems,
                       g->vt_ptr.get(), g->vt_idx.get(), g->ta.get(), g->tb.get(), g->tc.get(), sc.in.get(), all_in, un,
                       ud, ln, ld, p, q, take.get(), all_in ? (int32_t*)nullptr : plen.get());
        LDS_CUDA(cudaMemsetAsync(take.get() + nitems, 0, sizeof(int32_t), s));
        DevBuf<int64_t> patpos(nitems + 1, s), slotpos;
        const int64_t np = exclusive_scan_i32_to_i64(take.get(), patpos.get(), nitems + 1, s);
        int64_t nidx = 3 * np;
        if (!all_in) {
            LDS_CUDA(cudaMemsetAsync(plen.get() + nitems, 0, sizeof(int32_t), s));
            slotpos.alloc(nitems + 1, s);
            nidx = exclusive_scan_i32_to_i64(plen.get(), slotpos.get(), nitems + 1, s);
        }
        pptr.alloc(np + 1, s);
        pidx.alloc(std::max<int64_t>(nidx, 1), s);
        if (warm) share->alloc(std::max<int64_t>(nidx, 1), s);
        if (all_in) LDS_LAUNCH(uniform_pat_ptr_kernel, grid_for(np + 1, VB), VB, 0, s, np, 3, pptr.get());
        else LDS_CUDA(cudaMemcpyAsync(pptr.get() + np, &nidx, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (nitems && np)
            LDS_LAUNCH(tri_item_fill_kernel, grid_for(nitems, VB), VB, 0, s, list, k, ioff.get(), nitems,
                       g->vt_ptr.get(), g->vt_idx.get(), g->ta.get(), g->tb.get(), g->tc.get(), sc.in.get(),
                       sc.local.get(), all_in, un, ud, ln, ld, p, q, patpos.get(),
                       all_in ? (const int64_t*)nullptr : slotpos.get(), all_in ? (int64_t*)nullptr : pptr.get(),
                       pidx.get(), warm ? (const int64_t*)g->fw_W.get() : (const int64_t*)nullptr,
                       warm ? share->get() : (int64_t*)nullptr);
        LDS_CUDA(cudaStreamSynchronize(s));      // nidx (host) is read by the copy above
        if (n_main) *n_main = np;
        return np;
    }
}

int64_t build_all_patterns(lds_graph* h, bool tri, const int32_t* list, int32_t k, Scratch& sc,
                           DevBuf<int64_t>& pptr, DevBuf<int32_t>& pidx) {
    cudaStream_t s = h->stream;
    if (k) LDS_LAUNCH(mark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get(), sc.local.get());
    int64_t np = build_patterns(h, tri, list, k, sc, true, false, nullptr, 0, 1, pptr, pidx, nullptr);
    if (k) LDS_LAUNCH(unmark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get());
    LDS_CUDA(cudaStreamSynchronize(s));
    return np;
}

bool is_densest(lds_graph* g, bool tri, const int32_t* list, int32_t k, Scratch& sc, int64_t* npat) {
    cudaStream_t s = g->stream;
    *npat = 0;
    if (k == 0) return false;
    LDS_LAUNCH(mark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get(), sc.local.get());
    DevBuf<int64_t> pptr, share;
    DevBuf<int32_t> pidx;
    int64_t np = build_patterns(g, tri, list, k, sc, true, false, nullptr, 0, 1, pptr, pidx, nullptr, &share);
    *npat = np;
    bool ok = true;
    // a connected edge set with |E| = |S| - 1 is a tree: every proper subset has
    // density (j - 1) / j or less, so it is its own densest subgraph
    const bool tree = !tri && np == (int64_t)k - 1;
    if (np > 0 && !tree) {
        int64_t gg = gcd64(np, k);
        int64_t p = np / gg, q = k / gg;
        int64_t f = pattern_max_flow(pptr.get(), pidx.get(), (int32_t)np, k, p, q, share.get(), nullptr, true, s);
        ok = f == q * np;
    }
    LDS_LAUNCH(unmark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get());
    LDS_CUDA(cudaStreamSynchronize(s));
    return ok;
}

bool is_lds(lds_graph* g, bool tri, const int32_t* list, int32_t k, int64_t npat, const Bounds& b, Scratch& sc,
            VerifyStats* st, lds_verify mode) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n, nact = g->nact;
    int64_t gg = gcd64(npat, k);
    const int64_t p = npat / gg, q = k / gg;
    LDS_LAUNCH(mark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get(), (int32_t*)nullptr);
    DevBuf<int32_t> flag(1, s);
    int32_t hflag = 0;
    if (mode == LDS_VERIFY_BOUNDS) {
        LDS_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int32_t), s));
        LDS_LAUNCH(denser_neighbour_kernel, grid_for((int64_t)k * 32, VB), VB, 0, s, list, k, nact, g->rowptr.get(), g->col.get(),
                   sc.in.get(), b.ln.get(), b.ld.get(), p, q, flag.get());
        LDS_CUDA(cudaMemcpyAsync(&hflag, flag.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        if (hflag) {
            LDS_LAUNCH(unmark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get());
            if (st) ++st->denser_neighbour;
            return false;
        }
    }
    // grow U from S (sc.in2 marks U); the whole-graph baseline takes U = V
    DevBuf<int32_t> fa(std::max(n, 1), s), fb(std::max(n, 1), s), cnt(1, s);
    DevBuf<int32_t> U(std::max(n, 1), s);
    int32_t usize = k;
    if (mode == LDS_VERIFY_WHOLE) {
        usize = n;
        if (n) {
            LDS_LAUNCH(iota_i32_kernel, grid_for(n, VB), VB, 0, s, U.get(), n);
            LDS_LAUNCH(mark_kernel, grid_for(n, VB), VB, 0, s, U.get(), n, sc.in2.get(), (int32_t*)nullptr);
        }
    } else {
        LDS_LAUNCH(mark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in2.get(), (int32_t*)nullptr);
        LDS_CUDA(cudaMemcpyAsync(fa.get(), list, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        int32_t fsize = k;
        int32_t* cur = fa.get();
        int32_t* nxt = fb.get();
        LDS_CUDA(cudaMemcpyAsync(U.get(), list, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        while (fsize > 0) {
            LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t), s));
            LDS_LAUNCH(grow_level_kernel, grid_for((int64_t)fsize * 32, VB), VB, 0, s, cur, fsize, nact, g->rowptr.get(),
                       g->col.get(), sc.in2.get(), b.un.get(), b.ud.get(), b.ln.get(), b.ld.get(), p, q,
                       mode == LDS_VERIFY_BOUNDS, nxt, cnt.get());
            LDS_CUDA(cudaMemcpyAsync(&fsize, cnt.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
            if (fsize)
                LDS_CUDA(cudaMemcpyAsync(U.get() + usize, nxt, fsize * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            usize += fsize;
            std::swap(cur, nxt);
        }
    }
    bool result;
    if (usize == k) {
        result = true;                   // U = S: no denser neighbour, no loop, nothing to add
    } else {
        // sort U ascending so local indices are deterministic
        {
            DevBuf<uint64_t> key(usize, s);
            LDS_LAUNCH(widen_i32_u64_kernel, grid_for(usize, VB), VB, 0, s, U.get(), usize, key.get());
            radix_sort_u64(key.get(), nullptr, usize, bit_length_u64((uint64_t)std::max(n, 1)), s);
            LDS_LAUNCH(narrow_u64_i32_kernel, grid_for(usize, VB), VB, 0, s, key.get(), usize, U.get());
        }
        // patterns over U: swap marks so that sc.in marks U with local indices
        LDS_LAUNCH(unmark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get());
        LDS_LAUNCH(mark_kernel, grid_for(usize, VB), VB, 0, s, U.get(), usize, sc.in.get(), sc.local.get());
        // Alg. 4 / Alg. 7 networks (loops for denser outside neighbours, triangles reduced
        // to members with lb <= rho); the core and whole-graph forms hold every vertex
        // with ub >= rho that the search reaches (or all of V), so their patterns are
        // those inside U and there are no loops
        const bool bounds = mode == LDS_VERIFY_BOUNDS;
        DevBuf<int64_t> pptr, share;
        DevBuf<int32_t> pidx;
        int64_t np = build_patterns(g, tri, U.get(), usize, sc, !bounds, bounds && !tri, &b, p, q, pptr, pidx, nullptr,
                                    &share);
        DevBuf<uint8_t> side(usize, s);
        pattern_max_flow(pptr.get(), pidx.get(), (int32_t)np, usize, p, q, share.get(), side.get(), false, s);
        if (st) ++st->flows;
        // A = source side; S must be a connected component of G[A]
        LDS_LAUNCH(unmark_kernel, grid_for(usize, VB), VB, 0, s, U.get(), usize, sc.in.get());
        LDS_LAUNCH(side_to_flag_kernel, grid_for(usize, VB), VB, 0, s, U.get(), usize, side.get(), sc.in.get());
        // sc.in now marks A; sc.in2 is reused to mark S
        LDS_LAUNCH(unmark_kernel, grid_for(usize, VB), VB, 0, s, U.get(), usize, sc.in2.get());
        LDS_LAUNCH(mark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in2.get(), (int32_t*)nullptr);
        LDS_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int32_t), s));
        LDS_LAUNCH(component_check_kernel, grid_for((int64_t)k * 32, VB), VB, 0, s, list, k, nact, g->rowptr.get(), g->col.get(),
                   sc.in2.get(), sc.in.get(), flag.get());
        LDS_CUDA(cudaMemcpyAsync(&hflag, flag.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        result = hflag == 0;
        LDS_LAUNCH(unmark_kernel, grid_for(usize, VB), VB, 0, s, U.get(), usize, sc.in.get());
        LDS_LAUNCH(unmark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in2.get());
        LDS_CUDA(cudaStreamSynchronize(s));
        return result;
    }
    LDS_LAUNCH(unmark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get());
    LDS_LAUNCH(unmark_kernel, grid_for(usize, VB), VB, 0, s, U.get(), usize, sc.in2.get());
    LDS_CUDA(cudaStreamSynchronize(s));
    return result;
}

void components(lds_graph* g, const int32_t* list, int32_t k, Scratch& sc, DevBuf<int32_t>& members,
                std::vector<int32_t>& starts) {
    cudaStream_t s = g->stream;
    starts.clear();
    members.alloc(std::max(k, 1), s);
    if (k == 0) return;
    DevBuf<int32_t> label(std::max(g->n, 1), s), flags(3, s);
    LDS_LAUNCH(mark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get(), (int32_t*)nullptr);
    LDS_LAUNCH(cc_init_kernel, grid_for(k, VB), VB, 0, s, list, k, label.get());
    {
        // all sweeps in one cooperative launch
        LDS_CUDA(cudaMemsetAsync(flags.get(), 0, 3 * sizeof(int32_t), s));
        int per_sm = 0;
        LDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cc_coop_kernel, VB, 0));
        LDS_REQUIRE(per_sm > 0, LDS_ECUDA, "components: the sweep kernel cannot be resident");
        const int grid =
            (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)k * 32 + VB - 1) / VB, (int64_t)num_sms() * per_sm));
        const int32_t* lp = list;
        int32_t kk = k, na = g->nact;
        const int64_t* rp = g->rowptr.get();
        const int32_t* cp = g->col.get();
        const uint8_t* ip = sc.in.get();
        int32_t* lab = label.get();
        int32_t* fl = flags.get();
        int64_t max_sweeps = (int64_t)k + 2;
        void* args[] = {(void*)&lp, (void*)&kk, (void*)&na, (void*)&rp, (void*)&cp, (void*)&ip, (void*)&lab,
                        (void*)&fl, (void*)&max_sweeps};
        LDS_CUDA(cudaLaunchCooperativeKernel((void*)cc_coop_kernel, dim3(grid), dim3(VB), args, 0, s));
        g_launches.fetch_add(1, std::memory_order_relaxed);
        int32_t hf[3] = {0, 0, 0};
        LDS_CUDA(cudaMemcpyAsync(hf, flags.get(), sizeof(hf), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        LDS_REQUIRE(hf[2] == 0, LDS_ETIMEOUT, "components: label propagation did not settle");
    }
    LDS_LAUNCH(unmark_kernel, grid_for(k, VB), VB, 0, s, list, k, sc.in.get());
    const int bits = std::max(1, bit_length_u64((uint64_t)std::max(g->n, 1)));
    DevBuf<uint64_t> key(k, s);
    LDS_LAUNCH(cc_keys_kernel, grid_for(k, VB), VB, 0, s, list, k, label.get(), bits, key.get());
    radix_sort_u64(key.get(), nullptr, k, 2 * bits, s);
    DevBuf<int32_t> st(k, s), ns(1, s);
    LDS_CUDA(cudaMemsetAsync(ns.get(), 0, sizeof(int32_t), s));
    LDS_LAUNCH(cc_unpack_kernel, grid_for(k, VB), VB, 0, s, key.get(), k, bits, members.get(), st.get(), ns.get());
    int32_t hn = 0;
    LDS_CUDA(cudaMemcpyAsync(&hn, ns.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    starts.resize(hn);
    LDS_CUDA(cudaMemcpyAsync(starts.data(), st.get(), hn * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    std::sort(starts.begin(), starts.end());
    starts.push_back(k);
}

lds_graph* subgraph(lds_graph* g, const int32_t* list, int32_t k, Scratch& sc) {
    cudaStream_t s = g->stream;
    LDS_LAUNCH(mark_kernel, grid_for(std::max(k, 1), VB), VB, 0, s, list, k, sc.in.get(), sc.local.get());
    DevBuf<int32_t> cnt(std::max(k, 1), s);
    DevBuf<int64_t> off;
    if (k) LDS_LAUNCH(sub_edges_count_kernel, grid_for((int64_t)k * 32, VB), VB, 0, s, list, k, g->nact, g->rowptr.get(), g->col.get(),
                      sc.in.get(), cnt.get());
    int64_t me = scan_counts(cnt.get(), k, off, s);
    DevBuf<int32_t> su(std::max<int64_t>(me, 1), s), sv(std::max<int64_t>(me, 1), s);
    if (k && me)
        LDS_LAUNCH(sub_edges_fill_kernel, grid_for((int64_t)k * 32, VB), VB, 0, s, list, k, g->nact, g->rowptr.get(), g->col.get(),
                   sc.in.get(), sc.local.get(), off.get(), su.get(), sv.get());
    LDS_LAUNCH(unmark_kernel, grid_for(std::max(k, 1), VB), VB, 0, s, list, k, sc.in.get());
    LDS_CUDA(cudaStreamSynchronize(s));
    lds_graph* h = nullptr;
    lds_status stt = lds_create_graph(k, me, su.get(), sv.get(), LDS_MEM_DEVICE, s, &h);
    LDS_REQUIRE(stt == LDS_OK, stt, "subgraph: %s", lds_last_error());
    return h;
}

}  // namespace lds
