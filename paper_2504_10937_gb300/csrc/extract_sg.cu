// ExtractSG (Alg. 2): stable groups and compact-number bounds from the exact
// feasible solution of the last Frank-Wolfe run on a handle.
//
// 1. Vertices are sorted by exact load R = D r descending, ties by id
//    ascending (one radix sort of (Rmax - R, id) keys).
// 2. e_j, the number of patterns (edges or triangles) inside the first j
//    vertices, is a histogram over each pattern's largest position plus a scan.
// 3. Position j is a cut point when e_j / j is strictly larger than e_j' / j'
//    for every j' > j (argmax over j' >= j with ties to the larger j').  A tile
//    reduction, a suffix pass over tiles and a per-tile suffix scan compare the
//    fractions exactly with 128-bit cross products.
// 4. Candidates (segments between cut points) are checked against Def. 5
//    (Def. 12 for triangles) on a modified feasible solution: every pattern that
//    touches the segment S and has a vertex after S (in Z) gives its weight to
//    its lowest-load Z vertex; otherwise, if it has a vertex before S (in X),
//    to its lowest-load S vertex; for an edge that is "all weight to the other
//    endpoint".  S is accepted when every X vertex stays above max_S r' and
//    every Z vertex below min_S r'; a failed candidate merges with the next one
//    (Alg. 2's loop).  Each check walks the incidences (edges, triangles) of
//    the segment's vertices, one work item per incidence so that hubs are
//    shared by the whole grid; the S-side changes go to a per-position array
//    and the outside changes become (segment, vertex) records that are sorted
//    and summed.  The first round checks every candidate at once; a failure is
//    followed by single checks of the growing merged segment.
// 5. Accepted groups give lo = min_S R', hi = max_S R' (over the denominator D);
//    by Lemma 4 / Lemma 8 lo <= D phi(u) <= hi for u in the group.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstdlib>

#include "extract_sg.cuh"
#include "prims.cuh"

namespace lds {

namespace {

typedef __int128 i128;

// a/b > c/d for b, d > 0 (the numerator -1 stands for minus infinity)
__device__ __forceinline__ bool frac_gt(int64_t a, int64_t b, int64_t c, int64_t d) {
    return (i128)a * (i128)d > (i128)c * (i128)b;
}

__global__ void rmax_kernel(const int64_t* R, int32_t n, unsigned long long* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long m = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        m = max(m, (unsigned long long)R[x]);
    if (m) atomicMax(out, m);
}

// ties are broken by the original id (internal ids put isolated vertices last)
__global__ void sg_keys_kernel(const int64_t* R, const int32_t* to_orig, int32_t n, uint64_t rmax, int bits,
                               uint64_t* key) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        key[x] = ((rmax - (uint64_t)R[x]) << bits) | (uint64_t)to_orig[x];
}

__global__ void sg_order_kernel(const uint64_t* key, const int32_t* to_int, int32_t n, uint64_t mask, int32_t* order,
                                int32_t* pos) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        int32_t x = to_int[(int32_t)(key[p] & mask)];
        order[p] = x;
        pos[x] = (int32_t)p;
    }
}

__global__ void sg_hist_edges_kernel(const int32_t* eu, const int32_t* ev, int64_t m, const int32_t* pos, int32_t* h) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        atomicAdd(h + max(pos[eu[e]], pos[ev[e]]), 1);
}

__global__ void sg_hist_tris_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t nt,
                                    const int32_t* pos, int32_t* h) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride)
        atomicAdd(h + max(pos[ta[t]], max(pos[tb[t]], pos[tc[t]])), 1);
}

constexpr int CUT_THREADS = 256;
constexpr int CUT_ITEMS = 4;
constexpr int CUT_TILE = CUT_THREADS * CUT_ITEMS;

// excl_prefix[p] = patterns inside positions < p; e_{p+1} = excl_prefix[p] + h[p].
__device__ __forceinline__ void frac_max(int64_t& a, int64_t& b, int64_t c, int64_t d) {
    if (frac_gt(c, d, a, b)) { a = c; b = d; }
}

__global__ void cut_tilemax_kernel(const int64_t* incl, int32_t n, int64_t* tnum, int64_t* tden) {
    __shared__ int64_t sn[CUT_THREADS], sd[CUT_THREADS];
    int64_t base = (int64_t)blockIdx.x * CUT_TILE + threadIdx.x * CUT_ITEMS;
    int64_t bn = -1, bd = 1;
    for (int k = 0; k < CUT_ITEMS; ++k) {
        int64_t p = base + k;
        if (p < n) frac_max(bn, bd, incl[p], p + 1);
    }
    sn[threadIdx.x] = bn;
    sd[threadIdx.x] = bd;
    __syncthreads();
    for (int o = CUT_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            int64_t a = sn[threadIdx.x], b = sd[threadIdx.x];
            frac_max(a, b, sn[threadIdx.x + o], sd[threadIdx.x + o]);
            sn[threadIdx.x] = a;
            sd[threadIdx.x] = b;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tnum[blockIdx.x] = sn[0];
        tden[blockIdx.x] = sd[0];
    }
}

// suffix max over tiles, exclusive: sfx[b] = max over tiles > b (one thread; tiles are few)
__global__ void cut_tile_suffix_kernel(const int64_t* tnum, const int64_t* tden, int64_t ntiles, int64_t* snum,
                                       int64_t* sden) {
    if (blockIdx.x || threadIdx.x) return;
    int64_t a = -1, b = 1;
    for (int64_t t = ntiles - 1; t >= 0; --t) {
        snum[t] = a;
        sden[t] = b;
        frac_max(a, b, tnum[t], tden[t]);
    }
}

__global__ void cut_flags_kernel(const int64_t* incl, int32_t n, const int64_t* snum, const int64_t* sden,
                                 int32_t* flag) {
    __shared__ int64_t sn[CUT_THREADS], sd[CUT_THREADS];
    const int t = threadIdx.x;
    int64_t base = (int64_t)blockIdx.x * CUT_TILE + t * CUT_ITEMS;
    // max of this thread's items
    int64_t mn = -1, md = 1;
    for (int k = 0; k < CUT_ITEMS; ++k) {
        int64_t p = base + k;
        if (p < n) frac_max(mn, md, incl[p], p + 1);
    }
    sn[t] = mn;
    sd[t] = md;
    __syncthreads();
    // exclusive suffix max over threads t+1.. (Hillis-Steele on a reversed scan)
    int64_t an = mn, ad = md;       // inclusive suffix value
    for (int o = 1; o < CUT_THREADS; o <<= 1) {
        int64_t cn = -1, cd = 1;
        if (t + o < CUT_THREADS) { cn = sn[t + o]; cd = sd[t + o]; }
        __syncthreads();
        frac_max(an, ad, cn, cd);
        sn[t] = an;
        sd[t] = ad;
        __syncthreads();
    }
    int64_t rn = snum[blockIdx.x], rd = sden[blockIdx.x];
    if (t + 1 < CUT_THREADS) frac_max(rn, rd, sn[t + 1], sd[t + 1]);
    for (int k = CUT_ITEMS - 1; k >= 0; --k) {
        int64_t p = base + k;
        if (p >= n) continue;
        int64_t en = incl[p], ed = p + 1;
        flag[p] = frac_gt(en, ed, rn, rd) ? 1 : 0;
        frac_max(rn, rd, en, ed);
    }
}

__global__ void cut_list_kernel(const int32_t* flag, const int64_t* excl, int32_t n, int64_t* cuts) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        if (flag[p]) cuts[excl[p]] = p + 1;
}

// ---- checks

__global__ void seg_of_pos_kernel(const int64_t* sa, const int64_t* sb, int32_t nseg, int32_t plo, int32_t phi,
                                  int32_t* segof) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = plo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < phi; p += stride) {
        int lo = 0, hi = nseg;            // last segment with sa <= p
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (sa[mid] <= p) lo = mid + 1; else hi = mid;
        }
        int s = lo - 1;
        segof[p] = (s >= 0 && p <= sb[s]) ? s : -1;
    }
}

// ---- checks spread over incidences: every (position, incident edge or
// triangle) pair of the checked positions is one work item, so a hub with
// millions of incidences is shared by the whole grid.  ioff[p - plo] is the
// exclusive prefix of the checked positions' incidence counts; records take
// their slots from one counter (they are sorted by key and summed afterwards,
// so their order does not matter).

__global__ void inc_count_kernel(const int32_t* order, const int32_t* segof, int32_t plo, int32_t phi,
                                 const int64_t* ptr, int32_t nact, int64_t* icnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = plo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < phi; p += stride) {
        const int32_t x = order[p];
        icnt[p - plo] = ((!segof || segof[p] >= 0) && x < nact) ? ptr[x + 1] - ptr[x] : 0;
    }
}

// position of incidence i: the last p with ioff[p - plo] <= i
__device__ __forceinline__ int64_t inc_position(const int64_t* ioff, int32_t plo, int32_t phi, int64_t i) {
    int64_t lo = 0, hi = phi - plo;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (ioff[mid] <= i) lo = mid; else hi = mid;
    }
    return plo + lo;
}

__global__ void check_edges_flat_kernel(const int32_t* order, const int32_t* pos, const int32_t* segof,
                                        const int64_t* sa, const int64_t* sb, int32_t plo, int32_t phi,
                                        const int64_t* ioff, int64_t ninc, const int64_t* rowptr, const int32_t* col,
                                        const int64_t* slot_edge, const int32_t* eu, const int64_t* W, int64_t Dn,
                                        int32_t n, unsigned long long* deltaS, uint64_t* rkey, int64_t* rval,
                                        unsigned long long* nrec) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ninc; i += stride) {
        const int64_t p = inc_position(ioff, plo, phi, i);
        const int32_t s = segof[p];
        const int32_t x = order[p];
        const int64_t q = rowptr[x] + (i - ioff[p - plo]);
        const int32_t y = col[q];
        const int64_t py = pos[y], a = sa[s], b = sb[s];
        if (py >= a && py <= b) continue;
        const int64_t ed = slot_edge[q];
        const int64_t share_x = (eu[ed] == x) ? W[ed] : Dn - W[ed];
        const int64_t share_y = Dn - share_x;
        const unsigned long long o = atomicAdd(nrec, 1ull);
        rkey[o] = (uint64_t)s * (uint64_t)n + (uint64_t)y;
        if (py < a) {                                // y in X: the edge goes to x
            atomicAdd(deltaS + (p - plo), (unsigned long long)share_y);
            rval[o] = -share_y;
        } else {                                     // y in Z: the edge goes to y
            atomicAdd(deltaS + (p - plo), (unsigned long long)(-share_x));
            rval[o] = share_x;
        }
    }
}

// a triangle touching segment s is handled by its member of s with the largest position
__global__ void check_tris_flat_kernel(const int32_t* order, const int32_t* pos, const int32_t* segof,
                                       const int64_t* sa, const int64_t* sb, int32_t plo, int32_t phi,
                                       const int64_t* ioff, int64_t ninc, const int64_t* vt_ptr,
                                       const int32_t* vt_idx, const int32_t* ta, const int32_t* tb, const int32_t* tc,
                                       const int64_t* W, int32_t n, unsigned long long* deltaS, uint64_t* rkey,
                                       int64_t* rval, unsigned long long* nrec) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ninc; i += stride) {
        const int64_t p = inc_position(ioff, plo, phi, i);
        const int32_t s = segof[p];
        const int32_t x = order[p];
        const int32_t t = vt_idx[vt_ptr[x] + (i - ioff[p - plo])];
        const int64_t a = sa[s], b = sb[s];
        const int32_t v[3] = {ta[t], tb[t], tc[t]};
        const int64_t pp[3] = {pos[v[0]], pos[v[1]], pos[v[2]]};
        int64_t best = -1;
        for (int k = 0; k < 3; ++k)
            if (pp[k] >= a && pp[k] <= b && pp[k] > best) best = pp[k];
        if (best != p) continue;
        int zt = -1, st = -1;
        bool anyx = false;
        for (int k = 0; k < 3; ++k) {
            if (pp[k] > b) { if (zt < 0 || pp[k] > pp[zt]) zt = k; }
            else if (pp[k] < a) anyx = true;
            else if (st < 0 || pp[k] > pp[st]) st = k;
        }
        int tgt;
        if (zt >= 0) tgt = zt;
        else if (anyx) tgt = st;
        else continue;
        int64_t moved = 0;
        for (int k = 0; k < 3; ++k) {
            const bool mover = (zt >= 0) ? !(pp[k] > b) : (pp[k] < a);
            if (!mover) continue;
            const int64_t w = W[3 * (int64_t)t + k];
            moved += w;
            if (pp[k] >= a && pp[k] <= b) {
                atomicAdd(deltaS + (pp[k] - plo), (unsigned long long)(-w));
            } else {
                const unsigned long long o = atomicAdd(nrec, 1ull);
                rkey[o] = (uint64_t)s * (uint64_t)n + (uint64_t)v[k];
                rval[o] = -w;
            }
        }
        if (pp[tgt] >= a && pp[tgt] <= b) {
            atomicAdd(deltaS + (pp[tgt] - plo), (unsigned long long)moved);
        } else {
            const unsigned long long o = atomicAdd(nrec, 1ull);
            rkey[o] = (uint64_t)s * (uint64_t)n + (uint64_t)v[tgt];
            rval[o] = moved;
        }
    }
}

// ---- incremental chain checks.  For a fixed start a the candidate segment S =
// [a, b] grows; a pattern's change of the loads (its "delta") depends only on
// which of its members lie before S (X), in S or after S (Z):
//   * no member in S: unchanged;
//   * a member in Z: every member outside Z gives its weight to the Z member of
//     largest position (the lowest load in Z);
//   * else a member in X: every X member gives its weight to the S member of
//     largest position;
//   * else (all in S): unchanged.
// Growing S from [a, b] to [a, b'] changes the category of the members in
// (b, b'] only, so the per-position deltas are updated by (new - old) for the
// patterns with a member there, each pattern once (by its member of largest
// position in (b, b']).

__device__ __forceinline__ void pattern_delta(int k, const int64_t* pp, const int64_t* w, int64_t a, int64_t b,
                                              int64_t* d) {
    int zt = -1, st = -1;
    bool anyx = false, anys = false;
    for (int j = 0; j < k; ++j) {
        d[j] = 0;
        if (pp[j] > b) { if (zt < 0 || pp[j] > pp[zt]) zt = j; }
        else if (pp[j] < a) anyx = true;
        else { anys = true; if (st < 0 || pp[j] > pp[st]) st = j; }
    }
    if (!anys || (zt < 0 && !anyx)) return;
    const int tgt = zt >= 0 ? zt : st;
    int64_t moved = 0;
    for (int j = 0; j < k; ++j) {
        const bool mover = zt >= 0 ? !(pp[j] > b) : (pp[j] < a);
        if (mover) {
            d[j] -= w[j];
            moved += w[j];
        }
    }
    d[tgt] += moved;
}

// incidence r of the vertex at position p: if the pattern's member of largest
// position in (b0, b1] is p, add its (new - old) change of the loads to delta
__device__ __forceinline__ void chain_incidence(bool tri, int64_t p, int64_t r, const int32_t* order,
                                                const int32_t* pos, int64_t a, int64_t b0, int64_t b1,
                                                const int64_t* rowptr, const int32_t* col, const int64_t* slot_edge,
                                                const int32_t* eu, const int64_t* vt_ptr, const int32_t* vt_idx,
                                                const int32_t* ta, const int32_t* tb, const int32_t* tc,
                                                const int64_t* W, int64_t Dn, unsigned long long* delta) {
    const int32_t x = order[p];
    int k;
    int64_t pp[3], w[3];
    if (tri) {
        const int32_t t = vt_idx[vt_ptr[x] + r];
        const int32_t v[3] = {ta[t], tb[t], tc[t]};
        k = 3;
        for (int j = 0; j < 3; ++j) {
            pp[j] = pos[v[j]];
            w[j] = W[3 * (int64_t)t + j];
        }
    } else {
        const int64_t q = rowptr[x] + r;
        const int32_t y = col[q];
        const int64_t ed = slot_edge[q];
        k = 2;
        pp[0] = p;
        pp[1] = pos[y];
        w[0] = (eu[ed] == x) ? W[ed] : Dn - W[ed];
        w[1] = Dn - w[0];
    }
    int64_t best = -1;
    for (int j = 0; j < k; ++j)
        if (pp[j] > b0 && pp[j] <= b1 && pp[j] > best) best = pp[j];
    if (best != p) return;
    int64_t dn[3], dold[3];
    pattern_delta(k, pp, w, a, b1, dn);
    pattern_delta(k, pp, w, a, b0, dold);
    for (int j = 0; j < k; ++j)
        if (dn[j] != dold[j]) atomicAdd(delta + pp[j], (unsigned long long)(dn[j] - dold[j]));
}

// ---- one chain of merged candidates walked on the device (graphs of any size).
// Positions in chunks of CW_CHUNK, chunks in super-chunks of CW_SUPER.  Along a
// chain with fixed start a, X = [0, a) loads only fall, the loads of S members
// already in S only rise and Z loads only rise (pattern_delta moves weight from
// X to S or Z and from S to Z only), so min X and max S are running extremes, max
// Z is a chunk maximum kept by atomics (plus the partial chunk after b), and min S
// is recomputed only for chunks that changed.
constexpr int CW_CHUNK = 256;
constexpr int CW_SUPER = 256;

// chunk c of S changed: listed once until its minimum is recomputed (dirty is
// padded to whole 32-bit words)
__device__ __forceinline__ void mark_dirty(int64_t c, uint8_t* dirty, int32_t* dlist, int32_t* nd) {
    unsigned int* word = reinterpret_cast<unsigned int*>(dirty + (c & ~3ll));
    const unsigned int bit = 1u << (8 * (c & 3));
    if (!(atomicOr(word, bit) & bit)) dlist[atomicAdd(nd, 1)] = (int32_t)c;
}

// chain_incidence, also keeping the extremes: X -> running min, old S -> running
// max and a dirty chunk, Z -> chunk and super-chunk maxima
__device__ __forceinline__ void chain_track(bool tri, int64_t p, int64_t r, const int32_t* order, const int32_t* pos,
                                            int64_t a, int64_t b0, int64_t b1, const int64_t* rowptr,
                                            const int32_t* col, const int64_t* slot_edge, const int32_t* eu,
                                            const int64_t* vt_ptr, const int32_t* vt_idx, const int32_t* ta,
                                            const int32_t* tb, const int32_t* tc, const int64_t* W, int64_t Dn,
                                            const int64_t* R, unsigned long long* delta, unsigned long long* minX,
                                            unsigned long long* maxS, unsigned long long* cZ, unsigned long long* sZ,
                                            uint8_t* dirty, int32_t* dlist, int32_t* nd) {
    const int32_t x = order[p];
    int k;
    int64_t pp[3], w[3];
    if (tri) {
        const int32_t t = vt_idx[vt_ptr[x] + r];
        const int32_t v[3] = {ta[t], tb[t], tc[t]};
        k = 3;
        for (int j = 0; j < 3; ++j) {
            pp[j] = pos[v[j]];
            w[j] = W[3 * (int64_t)t + j];
        }
    } else {
        const int64_t q = rowptr[x] + r;
        const int32_t y = col[q];
        const int64_t ed = slot_edge[q];
        k = 2;
        pp[0] = p;
        pp[1] = pos[y];
        w[0] = (eu[ed] == x) ? W[ed] : Dn - W[ed];
        w[1] = Dn - w[0];
    }
    int64_t best = -1;
    for (int j = 0; j < k; ++j)
        if (pp[j] > b0 && pp[j] <= b1 && pp[j] > best) best = pp[j];
    if (best != p) return;
    int64_t dn[3], dold[3];
    pattern_delta(k, pp, w, a, b1, dn);
    pattern_delta(k, pp, w, a, b0, dold);
    for (int j = 0; j < k; ++j) {
        if (dn[j] == dold[j]) continue;
        const int64_t q = pp[j];
        const unsigned long long ch = (unsigned long long)(dn[j] - dold[j]);
        const unsigned long long v = (unsigned long long)R[order[q]] + atomicAdd(delta + q, ch) + ch;
        if (q < a) {
            atomicMin(minX, v);
        } else if (q <= b0) {
            atomicMax(maxS, v);
            mark_dirty(q / CW_CHUNK, dirty, dlist, nd);
        } else if (q > b1) {
            atomicMax(cZ + q / CW_CHUNK, v);
            atomicMax(sZ + q / ((int64_t)CW_CHUNK * CW_SUPER), v);
        }
    }
}

// exclusive scan of one int64 per thread over a block of 1024 threads; returns the total
__device__ __forceinline__ int64_t cw_block_scan(int64_t v, int64_t* out, int64_t* wsum) {
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
        wsum[lane] = w;
    }
    __syncthreads();
    out[tid] = inc - v + (wid ? wsum[wid - 1] : 0);
    const int64_t total = wsum[31];
    __syncthreads();
    return total;
}

// Chain state kept in device memory between launches (cws, 8 words): [0] min X,
// [1] max S (running), [2] listed dirty chunks, [3] end b of S, [4] next
// candidate, [5] 1 when that candidate's patterns are already applied, [6] steps,
// [7] 1 once the chunk maxima of Z are set up.
constexpr int64_t CW_HEAVY = 16384;   // a step with more incidences runs grid-wide

// One chain of merged candidates with start a (S = [a, cb[k]] for k = cws[4],
// cws[4] + 1, ...), in one CTA: stops at the first candidate whose two checks
// pass (status 0), at the first X-side failure (status 1), after the last
// candidate (status 2), or before a step with more than CW_HEAVY incidences
// (status 3: the host applies them grid-wide, chain_heavy_kernel, and launches
// this kernel again).  The caller clears delta and dirty once per chain.
// out = {k_end, status, minS, maxS, minX, maxZ}.
__global__ void __launch_bounds__(1024) chain_walk_kernel(
    bool tri, const int32_t* order, const int32_t* pos, int32_t n, int32_t nact, int64_t a, int32_t ncand,
    const int64_t* cb, const int64_t* R, const int64_t* rowptr, const int32_t* col, const int64_t* slot_edge,
    const int32_t* eu, const int64_t* vt_ptr, const int32_t* vt_idx, const int32_t* ta, const int32_t* tb,
    const int32_t* tc, const int64_t* W, int64_t Dn, unsigned long long* delta, unsigned long long* csmin,
    unsigned long long* cZ, unsigned long long* sZ, uint8_t* dirty, int32_t* dlist, long long* cws, long long* out) {
    __shared__ unsigned long long s_minX, s_maxS;
    __shared__ unsigned long long red[2][32];
    __shared__ long long s_cnt;
    __shared__ int32_t s_nd, s_done;
    __shared__ int64_t s_off[1024], s_wsum[32];
    const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = bd >> 5;
    const int64_t nchunks = ((int64_t)n + CW_CHUNK - 1) / CW_CHUNK;
    const int64_t nsuper = (nchunks + CW_SUPER - 1) / CW_SUPER;
    if (cws[7] == 0) {
        // unmodified maxima: the first position of a chunk holds its largest load
        for (int64_t c = tid; c < nchunks; c += bd) cZ[c] = (unsigned long long)R[order[c * CW_CHUNK]];
        for (int64_t c = tid; c < nsuper; c += bd) sZ[c] = (unsigned long long)R[order[c * CW_CHUNK * CW_SUPER]];
    }
    if (tid == 0) {
        const bool first = cws[7] == 0;
        s_minX = first ? (a > 0 ? (unsigned long long)R[order[a - 1]] : ~0ull) : (unsigned long long)cws[0];
        s_maxS = first ? 0ull : (unsigned long long)cws[1];
        s_nd = first ? 0 : (int32_t)cws[2];
        s_done = 0;
    }
    __syncthreads();
    int64_t b = cws[3], steps = cws[6];
    bool applied = cws[5] != 0;
    int32_t k = (int32_t)cws[4];
    for (; k < ncand; ++k) {
        const int64_t b0 = b, b1 = cb[k];
        if (!applied) {
            // incidences of the added positions: past CW_HEAVY the grid takes them
            if (tid == 0) s_cnt = 0;
            __syncthreads();
            long long c = 0;
            for (int64_t p = b0 + 1 + tid; p <= b1; p += bd) {
                const int32_t x = order[p];
                if (x < nact) c += tri ? vt_ptr[x + 1] - vt_ptr[x] : rowptr[x + 1] - rowptr[x];
            }
            for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0 && c) atomicAdd(reinterpret_cast<unsigned long long*>(&s_cnt), (unsigned long long)c);
            __syncthreads();
            if (s_cnt > CW_HEAVY) {
                if (tid == 0) {
                    cws[0] = (long long)s_minX;
                    cws[1] = (long long)s_maxS;
                    cws[2] = s_nd;
                    cws[3] = b;
                    cws[4] = k;
                    cws[5] = 0;
                    cws[6] = steps;
                    cws[7] = 1;
                    out[1] = 3;
                }
                return;
            }
            // one position by the whole block, several by one warp each
            if (b1 == b0 + 1) {
                const int32_t x = order[b1];
                if (x < nact) {
                    const int64_t deg = tri ? vt_ptr[x + 1] - vt_ptr[x] : rowptr[x + 1] - rowptr[x];
                    for (int64_t r = tid; r < deg; r += bd)
                        chain_track(tri, b1, r, order, pos, a, b0, b1, rowptr, col, slot_edge, eu, vt_ptr, vt_idx, ta,
                                    tb, tc, W, Dn, R, delta, &s_minX, &s_maxS, cZ, sZ, dirty, dlist, &s_nd);
                }
            } else {
                // several positions: their incidences spread evenly over the block, in
                // batches of one position per thread (scan of the incidence counts)
                for (int64_t base = b0 + 1; base <= b1; base += bd) {
                    const int64_t p = base + tid;
                    int64_t d = 0;
                    if (p <= b1) {
                        const int32_t x = order[p];
                        if (x < nact) d = tri ? vt_ptr[x + 1] - vt_ptr[x] : rowptr[x + 1] - rowptr[x];
                    }
                    const int64_t total = cw_block_scan(d, s_off, s_wsum);
                    const int32_t cnt = (int32_t)min((int64_t)bd, b1 - base + 1);
                    for (int64_t i = tid; i < total; i += bd) {
                        int32_t lo = 0, hi = cnt;            // last position with offset <= i
                        while (hi - lo > 1) {
                            const int32_t mid = (lo + hi) >> 1;
                            if (s_off[mid] <= i) lo = mid; else hi = mid;
                        }
                        chain_track(tri, base + lo, i - s_off[lo], order, pos, a, b0, b1, rowptr, col, slot_edge, eu,
                                    vt_ptr, vt_idx, ta, tb, tc, W, Dn, R, delta, &s_minX, &s_maxS, cZ, sZ, dirty, dlist,
                                    &s_nd);
                    }
                    __syncthreads();
                }
            }
        }
        applied = false;
        for (int64_t p = b0 + 1 + tid; p <= b1; p += bd)
            if (p == b0 + 1 || p % CW_CHUNK == 0) mark_dirty(p / CW_CHUNK, dirty, dlist, &s_nd);
        __syncthreads();
        // the new members' loads, and the minima of the changed chunks of S
        for (int64_t p = b0 + 1 + tid; p <= b1; p += bd)
            atomicMax(&s_maxS, (unsigned long long)R[order[p]] + delta[p]);
        const int32_t nd = s_nd;
        for (int32_t i = wid; i < nd; i += nw) {
            const int64_t c = dlist[i];
            const int64_t lo = max(c * CW_CHUNK, a), hi = min(c * CW_CHUNK + CW_CHUNK - 1, b1);
            unsigned long long m = ~0ull;
            for (int64_t p = lo + lane; p <= hi; p += 32) m = min(m, (unsigned long long)R[order[p]] + delta[p]);
            for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) {
                csmin[c] = m;
                dirty[c] = 0;
            }
        }
        __syncthreads();
        if (tid == 0) s_nd = 0;
        // min S over its chunks; max Z over the rest of b's chunk, the chunks to the
        // end of its super-chunk and the super-chunks after
        unsigned long long mS = ~0ull, mZ = 0;
        for (int64_t c = a / CW_CHUNK + tid; c <= b1 / CW_CHUNK; c += bd) mS = min(mS, csmin[c]);
        if (b1 < n - 1) {
            const int64_t cz = b1 / CW_CHUNK, sz = cz / CW_SUPER;
            const int64_t pend = min((int64_t)n, (cz + 1) * CW_CHUNK);
            for (int64_t p = b1 + 1 + tid; p < pend; p += bd)
                mZ = max(mZ, (unsigned long long)R[order[p]] + delta[p]);
            const int64_t cend = min(nchunks, (sz + 1) * CW_SUPER);
            for (int64_t c = cz + 1 + tid; c < cend; c += bd) mZ = max(mZ, cZ[c]);
            for (int64_t c = sz + 1 + tid; c < nsuper; c += bd) mZ = max(mZ, sZ[c]);
        }
        for (int o = 16; o; o >>= 1) {
            mS = min(mS, __shfl_xor_sync(0xffffffffu, mS, o));
            mZ = max(mZ, __shfl_xor_sync(0xffffffffu, mZ, o));
        }
        if (lane == 0) {
            red[0][wid] = mS;
            red[1][wid] = mZ;
        }
        __syncthreads();
        if (tid == 0) {
            for (int j = 1; j < nw; ++j) {
                mS = min(mS, red[0][j]);
                mZ = max(mZ, red[1][j]);
            }
            ++steps;
            const long long lo = (long long)mS, hi = (long long)s_maxS;
            const long long mx = s_minX == ~0ull ? LLONG_MAX : (long long)s_minX;
            const long long mz = b1 == n - 1 ? LLONG_MIN : (long long)mZ;
            const bool xok = a == 0 || mx > hi;
            const bool zok = b1 == n - 1 || mz < lo;
            if (!xok || zok) {
                out[0] = k;
                out[1] = xok ? 0 : 1;
                out[2] = lo;
                out[3] = hi;
                out[4] = mx;
                out[5] = mz;
                s_done = 1;
            }
        }
        __syncthreads();
        if (s_done) break;
        b = b1;
    }
    if (tid == 0) {
        if (!s_done) {
            out[0] = ncand;
            out[1] = 2;
        }
        cws[6] = steps;
    }
}

// the patterns of positions (b0, b1] of a chain grid-wide: one work item per
// incidence, the same tracking as in chain_walk_kernel, the running extremes
// and the dirty count in cws
__global__ void chain_heavy_kernel(bool tri, const int32_t* order, const int32_t* pos, int64_t a, int64_t b0, int64_t b1,
                                   const int64_t* ioff, int64_t ninc, const int64_t* rowptr, const int32_t* col,
                                   const int64_t* slot_edge, const int32_t* eu, const int64_t* vt_ptr,
                                   const int32_t* vt_idx, const int32_t* ta, const int32_t* tb, const int32_t* tc,
                                   const int64_t* W, int64_t Dn, const int64_t* R, unsigned long long* delta,
                                   unsigned long long* cZ, unsigned long long* sZ, uint8_t* dirty, int32_t* dlist,
                                   long long* cws) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int32_t plo = (int32_t)(b0 + 1), phi = (int32_t)(b1 + 1);
    unsigned long long* gX = reinterpret_cast<unsigned long long*>(cws);
    unsigned long long* gS = reinterpret_cast<unsigned long long*>(cws + 1);
    int32_t* gnd = reinterpret_cast<int32_t*>(cws + 2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ninc; i += stride) {
        const int64_t p = inc_position(ioff, plo, phi, i);
        chain_track(tri, p, i - ioff[p - plo], order, pos, a, b0, b1, rowptr, col, slot_edge, eu, vt_ptr, vt_idx, ta,
                    tb, tc, W, Dn, R, delta, gX, gS, cZ, sZ, dirty, dlist, gnd);
    }
}

// The whole walk of Alg. 2's merge loop in one CTA, for small graphs: candidate k
// starting at the current start takes its single check (precomputed); any other
// extends the chain of the current start (chain_incidence) and takes the block's
// min / max over X, S and Z.  Writes the accepted groups' ends and bounds.
__global__ void __launch_bounds__(1024) sg_walk_small_kernel(
    bool tri, const int32_t* order, const int32_t* pos, int32_t n, int32_t nact, int32_t ncand, const int64_t* ca,
    const int64_t* cb, const long long* mnS, const long long* mxS, const long long* mnX, const long long* mxZ,
    const int64_t* R, const int64_t* rowptr, const int32_t* col, const int64_t* slot_edge, const int32_t* eu,
    const int64_t* vt_ptr, const int32_t* vt_idx, const int32_t* ta, const int32_t* tb, const int32_t* tc,
    const int64_t* W, int64_t Dn, unsigned long long* delta, int64_t* gend, long long* glo, long long* ghi,
    int32_t* ngroups, int64_t* chain_checks, bool fresh) {
    __shared__ unsigned long long red[4][32];
    __shared__ long long res[4];
    __shared__ int64_t s_start, s_a, s_b;
    __shared__ int32_t s_ng, s_stop;
    __shared__ int64_t s_checks;
    const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        s_start = 0;
        s_a = -1;
        s_b = -1;
        s_ng = 0;
        s_stop = 0;
        s_checks = 0;
    }
    __syncthreads();
    for (int32_t k = 0; k < ncand; ++k) {
        const int64_t start = s_start;
        long long lo, hi, mx, mz;
        if (ca[k] == start && !fresh) {
            lo = mnS[k]; hi = mxS[k]; mx = mnX[k]; mz = mxZ[k];
        } else {
            // (fresh: a single check is the first step of a chain from its start)
            if (s_a != start) {
                for (int32_t p = tid; p < n; p += bd) delta[p] = 0;
                __syncthreads();
                if (tid == 0) { s_a = start; s_b = start - 1; }
                __syncthreads();
            }
            const int64_t b0 = s_b, b1 = cb[k];
            // positions (b0, b1]: each one's incidences spread over the block
            for (int64_t p = b0 + 1; p <= b1; ++p) {
                const int32_t x = order[p];
                if (x >= nact) continue;
                const int64_t deg = tri ? vt_ptr[x + 1] - vt_ptr[x] : rowptr[x + 1] - rowptr[x];
                for (int64_t r = tid; r < deg; r += bd)
                    chain_incidence(tri, p, r, order, pos, start, b0, b1, rowptr, col, slot_edge, eu, vt_ptr, vt_idx,
                                    ta, tb, tc, W, Dn, delta);
            }
            __syncthreads();
            unsigned long long e0 = ~0ull, e1 = 0, e2 = ~0ull, e3 = 0;
            for (int32_t p = tid; p < n; p += bd) {
                const unsigned long long v = (unsigned long long)(R[order[p]] + (int64_t)delta[p]);
                if (p < start) e2 = min(e2, v);
                else if (p <= b1) { e0 = min(e0, v); e1 = max(e1, v); }
                else e3 = max(e3, v);
            }
            for (int o = 16; o; o >>= 1) {
                e0 = min(e0, __shfl_xor_sync(0xffffffffu, e0, o));
                e1 = max(e1, __shfl_xor_sync(0xffffffffu, e1, o));
                e2 = min(e2, __shfl_xor_sync(0xffffffffu, e2, o));
                e3 = max(e3, __shfl_xor_sync(0xffffffffu, e3, o));
            }
            if (lane == 0) { red[0][wid] = e0; red[1][wid] = e1; red[2][wid] = e2; red[3][wid] = e3; }
            __syncthreads();
            if (tid == 0) {
                for (int j = 1; j < (bd + 31) / 32; ++j) {
                    e0 = min(e0, red[0][j]); e1 = max(e1, red[1][j]);
                    e2 = min(e2, red[2][j]); e3 = max(e3, red[3][j]);
                }
                res[0] = (long long)e0;
                res[1] = (long long)e1;
                res[2] = e2 == ~0ull ? LLONG_MAX : (long long)e2;
                res[3] = b1 == n - 1 ? LLONG_MIN : (long long)e3;
                s_b = b1;
                ++s_checks;
            }
            __syncthreads();
            lo = res[0]; hi = res[1]; mx = res[2]; mz = res[3];
        }
        const bool xok = start == 0 || mx > hi;
        const bool zok = cb[k] == n - 1 || mz < lo;
        __syncthreads();
        if (tid == 0) {
            if (xok && zok) {
                gend[s_ng] = cb[k] + 1;
                glo[s_ng] = lo;
                ghi[s_ng] = hi;
                ++s_ng;
                s_start = cb[k] + 1;
            } else if (!xok) {
                s_stop = 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
    }
    if (tid == 0) {
        *ngroups = s_ng;
        *chain_checks = s_checks;
    }
}

__global__ void iota_u32_kernel(uint32_t* p, int64_t k) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) p[i] = (uint32_t)i;
}

__global__ void fill_i32_range_kernel(int32_t* p, int32_t lo, int32_t hi, int32_t v) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += stride) p[i] = v;
}

__global__ void rec_gather_vals_kernel(const int64_t* val, const uint32_t* idx, int64_t k, int64_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = val[idx[i]];
}

__global__ void rec_reduce_kernel(const uint64_t* key, const int64_t* val, int64_t k, int32_t n, const int64_t* R,
                                  const int32_t* pos, const int64_t* sa, long long* minX, long long* maxZ) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        uint64_t kk = key[i];
        if (i > 0 && key[i - 1] == kk) continue;
        int64_t tot = 0;
        for (int64_t j = i; j < k && key[j] == kk; ++j) tot += val[j];
        int32_t s = (int32_t)(kk / (uint64_t)n);
        int32_t y = (int32_t)(kk % (uint64_t)n);
        long long v = (long long)(R[y] + tot);
        if (pos[y] < sa[s]) atomicMin(minX + s, v);
        else atomicMax(maxZ + s, v);
    }
}

__global__ void side_s_kernel(const int32_t* order, const int32_t* segof, int32_t npos_lo, int32_t npos_hi,
                              const int64_t* R, const int64_t* deltaS, long long* minS, long long* maxS) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = npos_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npos_hi; p += stride) {
        int32_t s = segof[p];
        if (s < 0) continue;
        long long v = (long long)(R[order[p]] + deltaS[p - npos_lo]);
        atomicMin(minS + s, v);
        atomicMax(maxS + s, v);
    }
}

__global__ void side_init_kernel(const int64_t* sa, const int64_t* sb, int32_t nseg, int32_t n, const int32_t* order,
                                 const int64_t* R, long long* minS, long long* maxS, long long* minX, long long* maxZ) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += stride) {
        minS[s] = LLONG_MAX;
        maxS[s] = LLONG_MIN;
        minX[s] = sa[s] > 0 ? (long long)R[order[sa[s] - 1]] : LLONG_MAX;
        maxZ[s] = sb[s] < n - 1 ? (long long)R[order[sb[s] + 1]] : LLONG_MIN;
    }
}

__global__ void vt_key_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t nt, uint64_t* key,
                              uint32_t* tid) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nt; i += stride) {
        int64_t t = i / 3;
        int k = (int)(i % 3);
        key[i] = (uint64_t)(k == 0 ? ta[t] : (k == 1 ? tb[t] : tc[t]));
        tid[i] = (uint32_t)t;
    }
}

__global__ void vt_ptr_kernel(const uint64_t* key, int64_t k3, int32_t nact, int64_t* ptr) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k3; i += stride) {
        int64_t x = (int64_t)key[i];
        int64_t prev = i == 0 ? -1 : (int64_t)key[i - 1];
        for (int64_t r = prev + 1; r <= x; ++r) ptr[r] = i;
        if (i == k3 - 1)
            for (int64_t r = x + 1; r <= nact; ++r) ptr[r] = k3;
    }
}

__global__ void u32_to_i32_kernel(const uint32_t* in, int64_t k, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = (int32_t)in[i];
}

}  // namespace

void build_vertex_triangles(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t nt, int32_t nact,
                            DevBuf<int64_t>& vt_ptr, DevBuf<int32_t>& vt_idx, cudaStream_t s) {
    const int blk = 256;
    vt_ptr.alloc(nact + 1, s);
    vt_idx.alloc(std::max<int64_t>(3 * nt, 1), s);
    if (nt == 0) {
        LDS_CUDA(cudaMemsetAsync(vt_ptr.get(), 0, (nact + 1) * sizeof(int64_t), s));
        LDS_CUDA(cudaStreamSynchronize(s));
        return;
    }
    DevBuf<uint64_t> key(3 * nt, s);
    DevBuf<uint32_t> tid(3 * nt, s);
    LDS_LAUNCH(vt_key_kernel, grid_for(3 * nt, blk), blk, 0, s, ta, tb, tc, nt, key.get(), tid.get());
    radix_sort_u64(key.get(), tid.get(), 3 * nt, bit_length_u64((uint64_t)nact), s);
    LDS_LAUNCH(vt_ptr_kernel, grid_for(3 * nt, blk), blk, 0, s, key.get(), 3 * nt, nact, vt_ptr.get());
    LDS_LAUNCH(u32_to_i32_kernel, grid_for(3 * nt, blk), blk, 0, s, tid.get(), 3 * nt, vt_idx.get());
    LDS_CUDA(cudaStreamSynchronize(s));
}

void ensure_vertex_triangles(lds_graph* g) {
    if (g->vt_ptr.p) return;
    ensure_triangles(g);
    build_vertex_triangles(g->ta.get(), g->tb.get(), g->tc.get(), g->ntri, g->nact, g->vt_ptr, g->vt_idx, g->stream);
}

// Checks the given disjoint segments (positions, inclusive) and returns
// (minS, maxS, minX, maxZ) per segment.
// segof (device, all -1 between calls) maps positions to checked segments.
static void check_segments(lds_graph* g, const SgState& st, int32_t* segof, const std::vector<int64_t>& ha,
                           const std::vector<int64_t>& hb, std::vector<long long>& minS, std::vector<long long>& maxS,
                           std::vector<long long>& minX, std::vector<long long>& maxZ) {
    cudaStream_t s = g->stream;
    const int blk = 256;
    const int32_t n = g->n;
    const int32_t nseg = (int32_t)ha.size();
    const bool tri = g->fw_density == LDS_TRIANGLE;
    DevBuf<int64_t> sa(nseg, s), sb(nseg, s);
    copy_in(sa.get(), ha.data(), LDS_MEM_HOST, nseg * sizeof(int64_t), s);
    copy_in(sb.get(), hb.data(), LDS_MEM_HOST, nseg * sizeof(int64_t), s);
    const int32_t plo = (int32_t)ha.front(), phi = (int32_t)hb.back() + 1;
    LDS_LAUNCH(seg_of_pos_kernel, grid_for(phi - plo, blk), blk, 0, s, sa.get(), sb.get(), nseg, plo, phi, segof);
    DevBuf<int64_t> deltaS(phi - plo, s);
    LDS_CUDA(cudaMemsetAsync(deltaS.get(), 0, (phi - plo) * sizeof(int64_t), s));
    const int64_t* W = g->fw_W.get();
    const int32_t nact = g->nact;
    // every incidence of a checked position is one work item; each emits at most one
    // record (edges) or owns at most one triangle, which emits at most two
    DevBuf<uint64_t> rkey;
    DevBuf<int64_t> rval;
    int64_t nrec = 0;
    const bool have = tri ? g->ntri > 0 : g->m > 0;
    if (have) {
        if (tri) ensure_vertex_triangles(g);
        else ensure_slot_edge(g);
        const int64_t* iptr = tri ? g->vt_ptr.get() : g->rowptr.get();
        DevBuf<int64_t> icnt(phi - plo, s), ioff(phi - plo, s);
        LDS_LAUNCH(inc_count_kernel, grid_for(phi - plo, blk), blk, 0, s, st.order.get(), segof, plo, phi, iptr, nact,
                   icnt.get());
        const int64_t ninc = exclusive_scan_i64(icnt.get(), ioff.get(), phi - plo, s);
        if (ninc) {
            const int64_t cap = tri ? 2 * ninc : ninc;
            rkey.alloc(cap, s);
            rval.alloc(cap, s);
            DevBuf<unsigned long long> dn(1, s);
            LDS_CUDA(cudaMemsetAsync(dn.get(), 0, sizeof(unsigned long long), s));
            if (tri)
                LDS_LAUNCH(check_tris_flat_kernel, grid_for(ninc, blk), blk, 0, s, st.order.get(), st.pos.get(), segof,
                           sa.get(), sb.get(), plo, phi, ioff.get(), ninc, g->vt_ptr.get(), g->vt_idx.get(), g->ta.get(),
                           g->tb.get(), g->tc.get(), W, n, (unsigned long long*)deltaS.get(), rkey.get(), rval.get(),
                           dn.get());
            else
                LDS_LAUNCH(check_edges_flat_kernel, grid_for(ninc, blk), blk, 0, s, st.order.get(), st.pos.get(), segof,
                           sa.get(), sb.get(), plo, phi, ioff.get(), ninc, g->rowptr.get(), g->col.get(),
                           g->slot_edge.get(), g->eu.get(), W, g->fw_D, n, (unsigned long long*)deltaS.get(),
                           rkey.get(), rval.get(), dn.get());
            unsigned long long hn = 0;
            LDS_CUDA(cudaMemcpyAsync(&hn, dn.get(), sizeof(hn), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
            nrec = (int64_t)hn;
            LDS_REQUIRE(nrec <= cap, LDS_ECUDA, "extract_sg: record buffer overrun");
        }
    }
    DevBuf<long long> dminS(nseg, s), dmaxS(nseg, s), dminX(nseg, s), dmaxZ(nseg, s);
    LDS_LAUNCH(side_init_kernel, grid_for(nseg, blk), blk, 0, s, sa.get(), sb.get(), nseg, n, st.order.get(),
               g->fw_R.get(), dminS.get(), dmaxS.get(), dminX.get(), dmaxZ.get());
    if (nrec) {
        DevBuf<uint32_t> idx(nrec, s);
        DevBuf<int64_t> sval(nrec, s);
        // sort the records by (segment, vertex), carrying their index
        LDS_LAUNCH(iota_u32_kernel, grid_for((int64_t)nrec, blk), blk, 0, s, idx.get(), (int64_t)nrec);
        radix_sort_u64(rkey.get(), idx.get(), (int64_t)nrec, bit_length_u64((uint64_t)nseg * (uint64_t)n), s);
        LDS_LAUNCH(rec_gather_vals_kernel, grid_for((int64_t)nrec, blk), blk, 0, s, rval.get(), idx.get(), (int64_t)nrec,
                   sval.get());
        LDS_LAUNCH(rec_reduce_kernel, grid_for((int64_t)nrec, blk), blk, 0, s, rkey.get(), sval.get(), (int64_t)nrec, n,
                   g->fw_R.get(), st.pos.get(), sa.get(), dminX.get(), dmaxZ.get());
    }
    LDS_LAUNCH(side_s_kernel, grid_for(phi - plo, blk), blk, 0, s, st.order.get(), segof, plo, phi, g->fw_R.get(),
               deltaS.get(), dminS.get(), dmaxS.get());
    LDS_LAUNCH(fill_i32_range_kernel, grid_for(phi - plo, blk), blk, 0, s, segof, plo, phi, -1);
    minS.resize(nseg);
    maxS.resize(nseg);
    minX.resize(nseg);
    maxZ.resize(nseg);
    LDS_CUDA(cudaMemcpyAsync(minS.data(), dminS.get(), nseg * sizeof(long long), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaMemcpyAsync(maxS.data(), dmaxS.get(), nseg * sizeof(long long), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaMemcpyAsync(minX.data(), dminX.get(), nseg * sizeof(long long), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaMemcpyAsync(maxZ.data(), dmaxZ.get(), nseg * sizeof(long long), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
}

// graphs up to this many vertices run the check walk in one CTA (sg_walk_small_kernel)
constexpr int32_t kSmallWalk = 65536;
// 0: by size; 1: the walk of large graphs (host loop, device chains) at every size
std::atomic<int> g_sg_variant{0};

void extract_sg(lds_graph* g, SgState& st) {
    LDS_REQUIRE(g->fw_valid, LDS_EINVAL, "extract_sg: run lds_fw on this graph first");
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t s = g->stream;
    const int blk = 256;
    const int32_t n = g->n;
    const bool tri = g->fw_density == LDS_TRIANGLE;
    st.D = g->fw_D;
    st.order.alloc(std::max(n, 1), s);
    st.pos.alloc(std::max(n, 1), s);
    st.cuts.clear();
    st.group_end.clear();
    st.lo.clear();
    st.hi.clear();
    if (n == 0) return;
    // 1. order by (R desc, id asc)
    DevBuf<unsigned long long> rmax(1, s);
    LDS_CUDA(cudaMemsetAsync(rmax.get(), 0, sizeof(unsigned long long), s));
    LDS_LAUNCH(rmax_kernel, grid_for(n, blk), blk, 0, s, g->fw_R.get(), n, rmax.get());
    unsigned long long hrmax = 0;
    LDS_CUDA(cudaMemcpyAsync(&hrmax, rmax.get(), sizeof(hrmax), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    const int idbits = std::max(1, bit_length_u64((uint64_t)std::max(n - 1, 1)));
    const int rbits = bit_length_u64(hrmax);
    LDS_REQUIRE(rbits + idbits <= 64, LDS_EOVERFLOW, "extract_sg: loads too large for the sort key");
    {
        DevBuf<uint64_t> key(n, s);
        LDS_LAUNCH(sg_keys_kernel, grid_for(n, blk), blk, 0, s, g->fw_R.get(), g->to_orig.get(), n, (uint64_t)hrmax,
                   idbits, key.get());
        radix_sort_u64(key.get(), nullptr, n, rbits + idbits, s);
        LDS_LAUNCH(sg_order_kernel, grid_for(n, blk), blk, 0, s, key.get(), g->to_int.get(), n, (1ull << idbits) - 1ull,
                   st.order.get(), st.pos.get());
    }
    // 2. e_j
    DevBuf<int32_t> h(n, s);
    LDS_CUDA(cudaMemsetAsync(h.get(), 0, n * sizeof(int32_t), s));
    if (!tri && g->m)
        LDS_LAUNCH(sg_hist_edges_kernel, grid_for(g->m, blk), blk, 0, s, g->eu.get(), g->ev.get(), g->m, st.pos.get(), h.get());
    if (tri && g->ntri)
        LDS_LAUNCH(sg_hist_tris_kernel, grid_for(g->ntri, blk), blk, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), g->ntri,
                   st.pos.get(), h.get());
    DevBuf<int64_t> incl(n + 1, s);
    {
        DevBuf<int32_t> h1(n + 1, s);
        LDS_CUDA(cudaMemsetAsync(h1.get(), 0, (n + 1) * sizeof(int32_t), s));
        LDS_CUDA(cudaMemcpyAsync(h1.get(), h.get(), n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        // exclusive scan of [h0, h1, ..., 0]: entry p + 1 is the inclusive prefix up to p
        exclusive_scan_i32_to_i64(h1.get(), incl.get(), n + 1, s);
    }
    const int64_t* inclp = incl.get() + 1;     // inclp[p] = e_{p+1}
    // 3. cut points
    const int64_t ntiles = (n + CUT_TILE - 1) / CUT_TILE;
    DevBuf<int64_t> tn(ntiles, s), td(ntiles, s), sn(ntiles, s), sd(ntiles, s);
    LDS_LAUNCH(cut_tilemax_kernel, (unsigned)ntiles, CUT_THREADS, 0, s, inclp, n, tn.get(), td.get());
    LDS_LAUNCH(cut_tile_suffix_kernel, 1, 1, 0, s, tn.get(), td.get(), ntiles, sn.get(), sd.get());
    DevBuf<int32_t> flag(n, s);
    LDS_LAUNCH(cut_flags_kernel, (unsigned)ntiles, CUT_THREADS, 0, s, inclp, n, sn.get(), sd.get(), flag.get());
    DevBuf<int64_t> fex(n, s);
    int64_t ncut = exclusive_scan_i32_to_i64(flag.get(), fex.get(), n, s);
    DevBuf<int64_t> dcuts(std::max<int64_t>(ncut, 1), s);
    LDS_LAUNCH(cut_list_kernel, grid_for(n, blk), blk, 0, s, flag.get(), fex.get(), n, dcuts.get());
    st.cuts.resize(ncut);
    LDS_CUDA(cudaMemcpyAsync(st.cuts.data(), dcuts.get(), ncut * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    const double ms_cuts = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    // 4. checks: every candidate alone first, then the merged segments of failures
    std::vector<int64_t> ca, cb;
    int64_t prev = 0;
    for (int64_t c : st.cuts) {
        ca.push_back(prev);
        cb.push_back(c - 1);
        prev = c;
    }
    DevBuf<int32_t> segof(n, s);
    LDS_LAUNCH(fill_i32_range_kernel, grid_for(n, blk), blk, 0, s, segof.get(), 0, n, -1);
    // Single-candidate checks are independent of one another; they are run
    // lazily, in batches of growing size, because the walk below often stops
    // long before the last candidate.
    const size_t ncand = ca.size();
    std::vector<long long> mnS(ncand), mxS(ncand), mnX(ncand), mxZ(ncand);
    size_t checked = 0, batch = 16;
    auto ensure_checked = [&](size_t k) {
        while (checked <= k) {
            const size_t hi = std::min(ncand, checked + batch);
            std::vector<int64_t> a(ca.begin() + checked, ca.begin() + hi), b(cb.begin() + checked, cb.begin() + hi);
            std::vector<long long> r1, r2, r3, r4;
            check_segments(g, st, segof.get(), a, b, r1, r2, r3, r4);
            std::copy(r1.begin(), r1.end(), mnS.begin() + checked);
            std::copy(r2.begin(), r2.end(), mxS.begin() + checked);
            std::copy(r3.begin(), r3.end(), mnX.begin() + checked);
            std::copy(r4.begin(), r4.end(), mxZ.begin() + checked);
            checked = hi;
            batch = std::min<size_t>(batch * 4, (size_t)1 << 22);
        }
    };
    // For a fixed start, growing the segment only lowers the X vertices' modified
    // loads and only raises max_S r': once the X-side test fails it fails for
    // every longer merge, so the whole rest is the unaccepted remainder.
    // Small graphs (refinement rounds on G[C]): every single check at once, then the
    // whole walk, chains included, in one CTA.
    if (n <= kSmallWalk && ncand > 0 && g_sg_variant.load(std::memory_order_relaxed) == 0) {
        // few candidates: each single check is a chain step inside the walk (one
        // reset of the n chain deltas per start), no batched checks at all
        const bool fresh = (int64_t)ncand * n <= ((int64_t)1 << 26);
        if (!fresh) ensure_checked(ncand - 1);
        const bool tri_g = tri;
        if (tri_g) ensure_vertex_triangles(g);
        else if (g->m) ensure_slot_edge(g);
        DevBuf<int64_t> dca(ncand, s), dcb(ncand, s), dgend(ncand, s), dchk(1, s);
        DevBuf<long long> d1(ncand, s), d2(ncand, s), d3(ncand, s), d4(ncand, s), dlo(ncand, s), dhi(ncand, s);
        DevBuf<unsigned long long> delta(n, s);
        DevBuf<int32_t> dng(1, s);
        copy_in(dca.get(), ca.data(), LDS_MEM_HOST, ncand * sizeof(int64_t), s);
        copy_in(dcb.get(), cb.data(), LDS_MEM_HOST, ncand * sizeof(int64_t), s);
        copy_in(d1.get(), mnS.data(), LDS_MEM_HOST, ncand * sizeof(long long), s);
        copy_in(d2.get(), mxS.data(), LDS_MEM_HOST, ncand * sizeof(long long), s);
        copy_in(d3.get(), mnX.data(), LDS_MEM_HOST, ncand * sizeof(long long), s);
        copy_in(d4.get(), mxZ.data(), LDS_MEM_HOST, ncand * sizeof(long long), s);
        LDS_LAUNCH(sg_walk_small_kernel, 1, 1024, 0, s, tri_g, st.order.get(), st.pos.get(), n, g->nact,
                   (int32_t)ncand, dca.get(), dcb.get(), d1.get(), d2.get(), d3.get(), d4.get(), g->fw_R.get(),
                   g->rowptr.get(), g->col.get(), tri_g ? nullptr : g->slot_edge.get(), g->eu.get(),
                   tri_g ? g->vt_ptr.get() : nullptr, tri_g ? g->vt_idx.get() : nullptr, g->ta.get(), g->tb.get(),
                   g->tc.get(), g->fw_W.get(), g->fw_D, delta.get(), dgend.get(), dlo.get(), dhi.get(), dng.get(),
                   dchk.get(), fresh);
        int32_t ng = 0;
        int64_t chk = 0;
        LDS_CUDA(cudaMemcpyAsync(&ng, dng.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaMemcpyAsync(&chk, dchk.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        st.group_end.resize(ng);
        st.lo.resize(ng);
        st.hi.resize(ng);
        if (ng) {
            LDS_CUDA(cudaMemcpyAsync(st.group_end.data(), dgend.get(), ng * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaMemcpyAsync(st.lo.data(), dlo.get(), ng * sizeof(long long), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaMemcpyAsync(st.hi.data(), dhi.get(), ng * sizeof(long long), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
        }
        st.chain_checks = chk;
        const char* vb0 = getenv("LDS_VERBOSE");
        if (vb0 && vb0[0] == '1')
            fprintf(stderr, "[extract_sg] n=%d candidates=%zu groups=%zu chain_checks=%lld (one-CTA walk); "
                            "sort+cuts %.2f ms, checks %.2f ms\n",
                    n, ca.size(), st.group_end.size(), (long long)st.chain_checks, ms_cuts,
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count() -
                        ms_cuts);
        return;
    }
    // A chain of merged candidates (the single check at the start failed on the Z
    // side) is walked on the device in one launch (chain_walk_kernel): each step
    // only walks the patterns of the positions it adds.
    const int64_t nchunks = ((int64_t)n + CW_CHUNK - 1) / CW_CHUNK;
    const int64_t nsuper = (nchunks + CW_SUPER - 1) / CW_SUPER;
    DevBuf<unsigned long long> cw_delta, cw_smin, cw_z, cw_sz;
    DevBuf<uint8_t> cw_dirty;
    DevBuf<int32_t> cw_list;
    DevBuf<int64_t> cw_cb;
    DevBuf<long long> cw_out, cw_state;
    int64_t start = 0;
    for (size_t k = 0; k < ca.size(); ++k) {
        long long lo, hi, mx, mz;
        if (ca[k] == start) {
            ensure_checked(k);
            lo = mnS[k]; hi = mxS[k]; mx = mnX[k]; mz = mxZ[k];
        } else {
            if (!cw_out.p) {
                cw_delta.alloc(n, s);
                cw_smin.alloc(nchunks, s);
                cw_z.alloc(nchunks, s);
                cw_sz.alloc(nsuper, s);
                cw_dirty.alloc((nchunks + 3) & ~3ll, s);
                cw_list.alloc(nchunks, s);
                cw_cb.alloc(ca.size(), s);
                cw_out.alloc(8, s);
                cw_state.alloc(8, s);
                copy_in(cw_cb.get(), cb.data(), LDS_MEM_HOST, cb.size() * sizeof(int64_t), s);
                if (tri) ensure_vertex_triangles(g);
                else if (g->m) ensure_slot_edge(g);
            }
            LDS_CUDA(cudaMemsetAsync(cw_delta.get(), 0, (size_t)n * sizeof(unsigned long long), s));
            LDS_CUDA(cudaMemsetAsync(cw_dirty.get(), 0, (nchunks + 3) & ~3ll, s));
            const long long init[8] = {0, 0, 0, (long long)start - 1, (long long)k, 0, 0, 0};
            copy_in(cw_state.get(), init, LDS_MEM_HOST, sizeof(init), s);
            long long h[8], cs[8];
            for (;;) {
                LDS_LAUNCH(chain_walk_kernel, 1, 1024, 0, s, tri, st.order.get(), st.pos.get(), n, g->nact, start,
                           (int32_t)ca.size(), cw_cb.get(), g->fw_R.get(), g->rowptr.get(), g->col.get(),
                           tri ? nullptr : g->slot_edge.get(), g->eu.get(), tri ? g->vt_ptr.get() : nullptr,
                           tri ? g->vt_idx.get() : nullptr, g->ta.get(), g->tb.get(), g->tc.get(), g->fw_W.get(),
                           g->fw_D, cw_delta.get(), cw_smin.get(), cw_z.get(), cw_sz.get(), cw_dirty.get(),
                           cw_list.get(), cw_state.get(), cw_out.get());
                LDS_CUDA(cudaMemcpyAsync(h, cw_out.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
                LDS_CUDA(cudaMemcpyAsync(cs, cw_state.get(), sizeof(cs), cudaMemcpyDeviceToHost, s));
                LDS_CUDA(cudaStreamSynchronize(s));
                if (h[1] != 3) break;
                // a heavy step: its incidences grid-wide, then the walk goes on
                const int64_t b0 = cs[3], b1 = cb[cs[4]];
                const int32_t plo = (int32_t)(b0 + 1), phi = (int32_t)(b1 + 1);
                const int64_t* iptr = tri ? g->vt_ptr.get() : g->rowptr.get();
                DevBuf<int64_t> icnt(phi - plo, s), ioff(phi - plo, s);
                LDS_LAUNCH(inc_count_kernel, grid_for(phi - plo, blk), blk, 0, s, st.order.get(),
                           (const int32_t*)nullptr, plo, phi, iptr, g->nact, icnt.get());
                const int64_t ninc = exclusive_scan_i64(icnt.get(), ioff.get(), phi - plo, s);
                if (ninc)
                    LDS_LAUNCH(chain_heavy_kernel, grid_for(ninc, blk), blk, 0, s, tri, st.order.get(), st.pos.get(),
                               start, b0, b1, ioff.get(), ninc, g->rowptr.get(), g->col.get(),
                               tri ? nullptr : g->slot_edge.get(), g->eu.get(), tri ? g->vt_ptr.get() : nullptr,
                               tri ? g->vt_idx.get() : nullptr, g->ta.get(), g->tb.get(), g->tc.get(), g->fw_W.get(),
                               g->fw_D, g->fw_R.get(), cw_delta.get(), cw_z.get(), cw_sz.get(), cw_dirty.get(),
                               cw_list.get(), cw_state.get());
                const long long one = 1;
                copy_in(cw_state.get() + 5, &one, LDS_MEM_HOST, sizeof(one), s);
            }
            st.chain_checks += cs[6];
            if (h[1] == 2) break;                 // no candidate left: the rest is the remainder
            k = (size_t)h[0];
            lo = h[2]; hi = h[3]; mx = h[4]; mz = h[5];
        }
        const bool xok = start == 0 || mx > hi;
        const bool zok = cb[k] == n - 1 || mz < lo;
        if (xok && zok) {
            st.group_end.push_back(cb[k] + 1);
            st.lo.push_back(lo);
            st.hi.push_back(hi);
            start = cb[k] + 1;
        } else if (!xok) {
            break;
        }
    }
    const char* vb = getenv("LDS_VERBOSE");
    if (vb && vb[0] == '1')
        fprintf(stderr, "[extract_sg] n=%d candidates=%zu groups=%zu chain_checks=%lld; sort+cuts %.2f ms, checks %.2f ms\n",
                n, ca.size(), st.group_end.size(), (long long)st.chain_checks, ms_cuts,
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count() - ms_cuts);
}

}  // namespace lds

using namespace lds;

extern "C" lds_status lds_set_extract_variant(int32_t variant) {
    return guard([&] {
        LDS_REQUIRE(variant == 0 || variant == 1, LDS_EINVAL, "lds_set_extract_variant: %d is not 0 or 1", variant);
        g_sg_variant.store(variant, std::memory_order_relaxed);
    });
}

extern "C" lds_status lds_extract_sg(lds_graph* g, int32_t* order, int32_t* ngroups, int64_t* group_end,
                                     int64_t* lo_num, int64_t* hi_num, int64_t* D, int32_t* ncuts, int64_t* cuts) {
    return guard([&] {
        LDS_REQUIRE(g && ngroups, LDS_EINVAL, "lds_extract_sg: NULL argument");
        SgState st;
        extract_sg(g, st);
        const int32_t n = g->n;
        *ngroups = (int32_t)st.group_end.size();
        if (D) *D = st.D;
        if (ncuts) *ncuts = (int32_t)st.cuts.size();
        if (order && n) {
            DevBuf<int32_t> o(n, g->stream);
            map_ids(st.order.get(), g->to_orig.get(), n, o.get(), g->stream);
            copy_out(order, LDS_MEM_HOST, o.get(), n * sizeof(int32_t), g->stream);
            LDS_CUDA(cudaStreamSynchronize(g->stream));
        }
        for (size_t k = 0; k < st.group_end.size(); ++k) {
            if (group_end) group_end[k] = st.group_end[k];
            if (lo_num) lo_num[k] = st.lo[k];
            if (hi_num) hi_num[k] = st.hi[k];
        }
        if (cuts)
            for (size_t k = 0; k < st.cuts.size(); ++k) cuts[k] = st.cuts[k];
    });
}
