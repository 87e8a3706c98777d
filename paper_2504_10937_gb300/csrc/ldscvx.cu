// The LDScvx / LTDScvx driver (Alg. 5 and its triangle extension, Sec. 6)
// orchestrated on the host; every step over vertices, edges, triangles or flow
// networks runs in the library's kernels.
//
// Readings (the same as the CPU oracle's driver):
//   * Initial reduction: ub = core number, lb = core / 2 (tr-core, tr-core / 3).
//   * The first round (FW, ExtractSG, Pruning) runs on G itself, so its bounds
//     hold for G.  Refinement rounds run on G[C] for a component C of a group:
//     their lower bounds are lifted to G, their upper bounds stay in the round.
//   * Every popped group is split into connected components.  A component that
//     is self-densest is certified by IsLDS / IsLTDS on G (or dropped); one that
//     is not is refined.  A refinement that returns the component unchanged is
//     retried with 2N, 4N, 8N iterations and then settled exactly (compact
//     numbers of G[C] by a divide and conquer of maximum flows over the
//     density-friendly decomposition, LDSs of G[C] by their level sets, each
//     certified on G).
//   * Completeness: every group is processed, except that once k sets are
//     certified a group whose vertices all have ub < rho_k is skipped.
//   * Output: density descending, ties by smallest member id.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <unordered_map>

#include "extract_sg.cuh"
#include "flow.cuh"
#include "prims.cuh"
#include "prune.cuh"
#include "verify.cuh"

namespace lds {

namespace {

typedef __int128 i128;
constexpr int DB = 256;

__global__ void init_bounds_kernel(const int64_t* core, int32_t nact, int32_t n, int64_t div, int64_t* un, int64_t* ud,
                                   int64_t* ln, int64_t* ld) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        int64_t c = x < nact ? core[x] : 0;
        un[x] = c;
        ud[x] = 1;
        ln[x] = c;
        ld[x] = div;
    }
}

// a/b reduced to lowest terms is not needed: comparisons cross-multiply
__device__ __forceinline__ bool fr_lt(int64_t a, int64_t b, int64_t c, int64_t d) {
    return (i128)a * d < (i128)c * b;
}

// tighten the bounds of the vertices of every accepted group
__global__ void apply_groups_kernel(const int32_t* order, const int64_t* gend, const int64_t* lo, const int64_t* hi,
                                    int32_t ng, int64_t Dn, int64_t npos, int64_t* un, int64_t* ud, int64_t* ln,
                                    int64_t* ld) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npos; p += stride) {
        int lo_i = 0, hi_i = ng;                  // first group with end > p
        while (lo_i < hi_i) {
            int mid = (lo_i + hi_i) >> 1;
            if (gend[mid] > p) hi_i = mid; else lo_i = mid + 1;
        }
        int gi = lo_i;
        if (gi >= ng) continue;
        int32_t x = order[p];
        if (fr_lt(hi[gi], Dn, un[x], ud[x])) { un[x] = hi[gi]; ud[x] = Dn; }
        if (fr_lt(ln[x], ld[x], lo[gi], Dn)) { ln[x] = lo[gi]; ld[x] = Dn; }
    }
}

// group id of every position (accepted groups 0..ng-1, remainder ng) and kept flag
__global__ void group_keys_kernel(const int32_t* order, const int64_t* gend, int32_t ng, int32_t n, const uint8_t* status,
                                  int32_t* gid, int32_t* keep, int32_t* gcount) {
    // warp-uniform loop; lanes of one group add their count with one atomic
    const int lane = threadIdx.x & 31;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; p0 < n; p0 += stride) {
        const int64_t p = p0 + lane;
        int key = -1;
        if (p < n) {
            int lo_i = 0, hi_i = ng;
            while (lo_i < hi_i) {
                int mid = (lo_i + hi_i) >> 1;
                if (gend[mid] > p) hi_i = mid; else lo_i = mid + 1;
            }
            int32_t k = status[order[p]] == 0;
            gid[p] = lo_i;
            keep[p] = k;
            if (k) key = lo_i;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(gcount + key, __popc(peers));
    }
}

__global__ void group_compact_kernel(const int32_t* order, const int32_t* keep, const int64_t* kpos, int32_t n,
                                     int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        if (keep[p]) out[kpos[p]] = order[p];
}

// sub-round bounds: ub_sub = min(core_sub, ub_G of the same vertex)
__global__ void sub_bounds_kernel(const int32_t* sub_to_orig, const int32_t* comp, int32_t nsub, const int64_t* unG,
                                  const int64_t* udG, int64_t* un, int64_t* ud) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nsub; x += stride) {
        int32_t gx = comp[sub_to_orig[x]];
        if (fr_lt(unG[gx], udG[gx], un[x], ud[x])) { un[x] = unG[gx]; ud[x] = udG[gx]; }
    }
}

// lift lower bounds of a sub-round to G
__global__ void lift_lb_kernel(const int32_t* sub_to_orig, const int32_t* comp, int32_t nsub, const int64_t* ln,
                               const int64_t* ld, int64_t* lnG, int64_t* ldG) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nsub; x += stride) {
        int32_t gx = comp[sub_to_orig[x]];
        if (fr_lt(lnG[gx], ldG[gx], ln[x], ld[x])) { lnG[gx] = ln[x]; ldG[gx] = ld[x]; }
    }
}

// members given in sub internal ids -> G internal ids
__global__ void to_parent_kernel(const int32_t* in, int64_t k, const int32_t* sub_to_orig, const int32_t* comp,
                                 int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = comp[sub_to_orig[in[i]]];
}

// 1 if some vertex of the list has ub >= num / den
__global__ void any_ub_ge_kernel(const int32_t* list, int32_t k, const int64_t* un, const int64_t* ud, int64_t num,
                                 int64_t den, int32_t* flag) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        int32_t x = list[i];
        if (!fr_lt(un[x], ud[x], num, den)) *flag = 1;
    }
}

__global__ void sort_keys_kernel(const int32_t* in, int64_t k, uint64_t* key) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) key[i] = (uint64_t)in[i];
}

__global__ void unsort_keys_kernel(const uint64_t* key, int64_t k, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = (int32_t)key[i];
}

// ---- exact settle: compact numbers of G[C] by divide and conquer over the
// density-friendly decomposition.  A sub-problem is a vertex set F with every
// vertex of a higher level settled above it and every vertex of a lower level
// below it; its patterns are those inside (above + F) with a member in F, each
// reduced to its members in F.  Vertex states:
constexpr uint8_t ES_BELOW = 0, ES_ABOVE = 1, ES_IN = 2;
constexpr unsigned ES_FULL = 0xffffffffu;

// incidences: deg[v] = patterns with member v
__global__ void es_inc_count_kernel(const int32_t* pidx, int64_t nnz, int32_t* deg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nnz; a += stride) atomicAdd(deg + pidx[a], 1);
}

__global__ void es_inc_fill_kernel(const int64_t* pptr, const int32_t* pidx, int64_t np, const int64_t* vptr,
                                   int32_t* cursor, int32_t* vinc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride)
        for (int64_t a = pptr[j]; a < pptr[j + 1]; ++a) {
            const int32_t v = pidx[a];
            vinc[vptr[v] + atomicAdd(cursor + v, 1)] = (int32_t)j;
        }
}

// members of F enter the sub-problem (state, local index) or leave it
__global__ void es_enter_kernel(const int32_t* F, int32_t nf, uint8_t* st, int32_t* freeidx) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += stride) {
        st[F[i]] = ES_IN;
        freeidx[F[i]] = (int32_t)i;
    }
}

__global__ void es_leave_kernel(const int32_t* F, int32_t nf, uint8_t* st, uint8_t to, int64_t p, int64_t q,
                                int64_t* phin, int64_t* phid) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += stride) {
        st[F[i]] = to;
        if (to == ES_ABOVE) {
            phin[F[i]] = p;
            phid[F[i]] = q;
        }
    }
}

// one warp per member v of F: the sub-problem's patterns through v that no member
// below it touches and whose smallest member in F is v (each pattern once);
// FILL writes their ids in incidence order
template <bool FILL>
__global__ void es_emit_kernel(const int32_t* F, int32_t nf, const int64_t* vptr, const int32_t* vinc,
                               const int64_t* pptr, const int32_t* pidx, const uint8_t* st, int32_t* cnt,
                               const int64_t* off, int32_t* out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nf; i += nwarps) {
        const int32_t v = F[i];
        const int64_t a1 = vptr[v + 1];
        int64_t o = FILL ? off[i] : 0;
        for (int64_t base = vptr[v]; base < a1; base += 32) {
            const int64_t a = base + lane;
            bool keep = false;
            int32_t j = 0;
            if (a < a1) {
                j = vinc[a];
                keep = true;
                for (int64_t b = pptr[j]; b < pptr[j + 1]; ++b) {
                    const int32_t w = pidx[b];
                    const uint8_t sw = st[w];
                    if (sw == ES_BELOW || (sw == ES_IN && w < v)) {
                        keep = false;
                        break;
                    }
                }
            }
            const unsigned bal = __ballot_sync(ES_FULL, keep);
            if (FILL && keep) out[o + __popc(bal & ((1u << lane) - 1u))] = j;
            o += __popc(bal);
        }
        if (!FILL && lane == 0) cnt[i] = (int32_t)o;
    }
}

// reduced patterns: their members in F as local indices
__global__ void es_len_kernel(const int32_t* pats, int64_t nr, const int64_t* pptr, const int32_t* pidx,
                              const uint8_t* st, int32_t* len) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += stride) {
        const int32_t j = pats[r];
        int32_t c = 0;
        for (int64_t b = pptr[j]; b < pptr[j + 1]; ++b) c += st[pidx[b]] == ES_IN;
        len[r] = c;
    }
}

__global__ void es_fill_kernel(const int32_t* pats, int64_t nr, const int64_t* pptr, const int32_t* pidx,
                               const uint8_t* st, const int32_t* freeidx, const int64_t* dptr, int32_t* ridx) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += stride) {
        const int32_t j = pats[r];
        int64_t o = dptr[r];
        for (int64_t b = pptr[j]; b < pptr[j + 1]; ++b)
            if (st[pidx[b]] == ES_IN) ridx[o++] = freeidx[pidx[b]];
    }
}

__global__ void es_iota_kernel(int32_t* out, int32_t n) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (int32_t)i;
}

__global__ void u8_to_i32_kernel(const uint8_t* in, int64_t k, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = in[i] != 0;
}

// F split by the cut side: side 1 to X (in order), side 0 to Y (in order)
__global__ void es_split_kernel(const int32_t* F, int32_t nf, const int32_t* side, const int64_t* pos, int32_t* X,
                                int32_t* Y) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += stride) {
        if (side[i]) X[pos[i]] = F[i];
        else Y[i - pos[i]] = F[i];
    }
}

// one warp per vertex x (local id): 1 if a neighbour of x in G[C] has a higher
// compact number (no LDS of G[C] contains x then)
__global__ void es_higher_kernel(const int32_t* all, int32_t n, int32_t nact, const int64_t* rowptr, const int32_t* col,
                                 const int32_t* to_local, const int64_t* phin, const int64_t* phid, uint8_t* flag) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int32_t xi = all[x];
        bool hi = false;
        if (xi < nact) {
            const i128 a = phin[x], b = phid[x];
            for (int64_t e = rowptr[xi] + lane; e < rowptr[xi + 1] && !hi; e += 32) {
                const int32_t y = to_local[col[e]];
                hi = (i128)phin[y] * b > a * (i128)phid[y];
            }
        }
        hi = __any_sync(ES_FULL, hi);
        if (lane == 0) flag[x] = hi;
    }
}

// component id of every member (components listed back to back, offsets off)
__global__ void comp_id_kernel(const int32_t* cm, const int32_t* off, int32_t ncomp, int32_t* compid) {
    const int64_t total = off[ncomp];
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        int32_t lo = 0, hi = ncomp;              // last component with off <= i
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid;
        }
        compid[cm[i]] = lo;
    }
}

// one warp per member: its component is open if the member has a neighbour in G
// outside it
__global__ void comp_open_kernel(const int32_t* cm, int64_t total, const int32_t* compid, int32_t nact,
                                 const int64_t* rowptr, const int32_t* col, uint8_t* open) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < total; i += nwarps) {
        const int32_t x = cm[i];
        if (x >= nact) continue;
        const int32_t c = compid[x];
        bool out = false;
        for (int64_t e = rowptr[x] + lane; e < rowptr[x + 1] && !out; e += 32) out = compid[col[e]] != c;
        if (__any_sync(0xffffffffu, out) && lane == 0) open[c] = 1;
    }
}

}  // namespace

struct Timers {
    double fw = 0, sg = 0, prune = 0, verify = 0, refine = 0, total = 0;
    double init = 0, comps = 0, sub = 0, sub_init = 0;     // host-clock split of the rest
};

static double ms_since(std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

struct Driver {
    lds_graph* G;
    bool tri;
    int32_t k;
    int32_t N;
    lds_precision prec;
    bool include_zero;
    lds_verify vmode;
    Bounds bG;
    Scratch sc;
    VerifyStats vst;
    lds_topk_stats_t stats{};
    Timers tm;
    struct Found {
        int64_t num, den;
        std::vector<int32_t> members;          // G internal ids, ascending
    };
    std::vector<Found> found;

    Driver(lds_graph* g, bool t, int32_t kk, int32_t n, lds_precision p, bool iz, lds_verify vm)
        : G(g), tri(t), k(kk), N(n), prec(p), include_zero(iz), vmode(vm), sc(g) {}

    cudaStream_t st() const { return G->stream; }

    void init_bounds(lds_graph* g, Bounds& b) {
        cudaStream_t s = g->stream;
        const int32_t n = g->n;
        b.un.alloc(std::max(n, 1), s);
        b.ud.alloc(std::max(n, 1), s);
        b.ln.alloc(std::max(n, 1), s);
        b.ld.alloc(std::max(n, 1), s);
        DevBuf<int64_t> core(std::max(g->nact, 1), s);
        core_numbers(g, tri, core.get(), nullptr);
        if (n) LDS_LAUNCH(init_bounds_kernel, grid_for(n, DB), DB, 0, s, core.get(), g->nact, n, tri ? 3 : 2, b.un.get(),
                          b.ud.get(), b.ln.get(), b.ld.get());
    }

    // FW + ExtractSG + Pruning on handle h with bounds b (tightened in place).
    // Returns the kept members of every group (h internal ids) and group offsets.
    void round(lds_graph* h, Bounds& b, int32_t iters, DevBuf<int32_t>& members, std::vector<int64_t>& offs) {
        cudaStream_t s = h->stream;
        auto t0 = std::chrono::steady_clock::now();
        // a state left by lds_fw_batch for exactly this round is taken as it is
        const lds_density dd = tri ? LDS_TRIANGLE : LDS_EDGE;
        const bool reuse = h->fw_reuse && h->fw_valid && h->fw_density == dd && h->fw_iters == iters &&
                           h->fw_prec == prec;
        h->fw_reuse = false;
        if (!reuse) fw_run(h, dd, iters, prec, false);
        ++stats.fw_rounds;
        stats.fw_edge_updates += (tri ? h->ntri : h->m) * (int64_t)iters;
        auto t1 = std::chrono::steady_clock::now();
        SgState sg;
        extract_sg(h, sg);
        const int32_t n = h->n;
        const int32_t ng = (int32_t)sg.group_end.size();
        DevBuf<int64_t> gend(std::max(ng, 1), s), lo(std::max(ng, 1), s), hi(std::max(ng, 1), s);
        if (ng) {
            std::vector<int64_t> l(sg.lo.begin(), sg.lo.end()), hh(sg.hi.begin(), sg.hi.end());
            copy_in(gend.get(), sg.group_end.data(), LDS_MEM_HOST, ng * sizeof(int64_t), s);
            copy_in(lo.get(), l.data(), LDS_MEM_HOST, ng * sizeof(int64_t), s);
            copy_in(hi.get(), hh.data(), LDS_MEM_HOST, ng * sizeof(int64_t), s);
            int64_t npos = sg.group_end.back();
            LDS_LAUNCH(apply_groups_kernel, grid_for(npos, DB), DB, 0, s, sg.order.get(), gend.get(), lo.get(), hi.get(),
                       ng, sg.D, npos, b.un.get(), b.ud.get(), b.ln.get(), b.ld.get());
        }
        auto t2 = std::chrono::steady_clock::now();
        DevBuf<uint8_t> status(std::max(n, 1), s);
        prune(h, tri, b.un.get(), b.ud.get(), b.ln.get(), b.ld.get(), status.get());
        // kept members per group (the remainder is one more group)
        DevBuf<int32_t> gid(std::max(n, 1), s), keep(std::max(n, 1), s), gcount(ng + 1, s);
        LDS_CUDA(cudaMemsetAsync(gcount.get(), 0, (ng + 1) * sizeof(int32_t), s));
        if (n) LDS_LAUNCH(group_keys_kernel, grid_for(n, DB), DB, 0, s, sg.order.get(), gend.get(), ng, n, status.get(),
                          gid.get(), keep.get(), gcount.get());
        DevBuf<int64_t> kpos(std::max(n, 1), s);
        int64_t nk = exclusive_scan_i32_to_i64(keep.get(), kpos.get(), n, s);
        members.alloc(std::max<int64_t>(nk, 1), s);
        if (n) LDS_LAUNCH(group_compact_kernel, grid_for(n, DB), DB, 0, s, sg.order.get(), keep.get(), kpos.get(), n,
                          members.get());
        std::vector<int32_t> hc(ng + 1);
        LDS_CUDA(cudaMemcpyAsync(hc.data(), gcount.get(), (ng + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        offs.assign(1, 0);
        for (int32_t c : hc)
            if (c) offs.push_back(offs.back() + c);
        auto t3 = std::chrono::steady_clock::now();
        tm.fw += std::chrono::duration<double, std::milli>(t1 - t0).count();
        tm.sg += std::chrono::duration<double, std::milli>(t2 - t1).count();
        tm.prune += std::chrono::duration<double, std::milli>(t3 - t2).count();
    }

    bool kth(int64_t& num, int64_t& den) {
        if ((int32_t)found.size() < k) return false;
        std::vector<std::pair<int64_t, int64_t>> ds;
        for (auto& f : found) ds.push_back({f.num, f.den});
        std::sort(ds.begin(), ds.end(), [](auto& a, auto& b) { return (i128)a.first * b.second > (i128)b.first * a.second; });
        num = ds[k - 1].first;
        den = ds[k - 1].second;
        return true;
    }

    // closed: S is a whole connected component of G.  With no neighbour outside, a
    // self-densest G[S] is rho-compact (every T in S has density <= rho, which is
    // the compactness inequality for U = S - T) and no connected proper supergraph
    // exists, so S is an LDS (LTDS) without a flow.
    void certify(const int32_t* comp, int32_t csize, int64_t npat, bool closed = false) {
        if (npat == 0 && !include_zero) return;
        bool ok = closed || is_lds(G, tri, comp, csize, npat, bG, sc, &vst, vmode);
        if (ok) {
            Found f;
            int64_t g = std::gcd(npat, (int64_t)csize);
            f.num = npat / g;
            f.den = csize / g;
            f.members.resize(csize);
            LDS_CUDA(cudaMemcpyAsync(f.members.data(), comp, csize * sizeof(int32_t), cudaMemcpyDeviceToHost, st()));
            LDS_CUDA(cudaStreamSynchronize(st()));
            found.push_back(std::move(f));
            ++stats.certified;
        } else {
            ++stats.failed;
        }
    }

    // 1 for every component (listed back to back in cm, offsets cs) that is a whole
    // connected component of G
    std::vector<uint8_t> closed_components(const int32_t* cm, const std::vector<int32_t>& cs) {
        cudaStream_t s = st();
        const int32_t nc = (int32_t)cs.size() - 1;
        std::vector<uint8_t> closed(std::max(nc, 0), 0);
        if (nc <= 0) return closed;
        const int64_t total = cs.back();
        DevBuf<int32_t> off(nc + 1, s), compid(std::max(G->n, 1), s);
        DevBuf<uint8_t> open(nc, s);
        copy_in(off.get(), cs.data(), LDS_MEM_HOST, (nc + 1) * sizeof(int32_t), s);
        LDS_CUDA(cudaMemsetAsync(compid.get(), 0xff, std::max(G->n, 1) * sizeof(int32_t), s));
        LDS_CUDA(cudaMemsetAsync(open.get(), 0, nc, s));
        if (total) {
            LDS_LAUNCH(comp_id_kernel, grid_for(total, DB), DB, 0, s, cm, off.get(), nc, compid.get());
            LDS_LAUNCH(comp_open_kernel, grid_for(total * 32, DB), DB, 0, s, cm, total, compid.get(), G->nact,
                       G->rowptr.get(), G->col.get(), open.get());
        }
        LDS_CUDA(cudaMemcpyAsync(closed.data(), open.get(), nc, cudaMemcpyDeviceToHost, s));
        LDS_CUDA(cudaStreamSynchronize(s));
        for (auto& c : closed) c = !c;
        return closed;
    }

    // Compact numbers of G[comp] by the density-friendly decomposition, then the
    // LDSs of G[comp] (level-set components with no denser neighbour inside
    // comp), each certified on G.
    void exact_settle(const int32_t* comp, int32_t csize);

    void run();
};

// Compact numbers of every vertex of h (Thm. 1 / Thm. 4: the optimal loads r*),
// exactly, as reduced fractions phin / phid indexed by h's original ids, through
// the density-friendly decomposition.  `all` receives h's internal id of every
// original id.  Returns the number of maximum flows run.
int64_t exact_compact_numbers(lds_graph* h, bool tri, DevBuf<int32_t>& all, DevBuf<int64_t>& phin,
                              DevBuf<int64_t>& phid) {
    cudaStream_t s = h->stream;
    if (tri) ensure_triangles(h);
    const int32_t n = h->n;
    int64_t flows = 0;
    // patterns of G[comp] over local ids (h's original ids = positions in comp)
    Scratch shc(h);
    all.alloc(std::max(n, 1), s);
    {
        std::vector<int32_t> ids(n);
        std::iota(ids.begin(), ids.end(), 0);
        DevBuf<int32_t> orig(std::max(n, 1), s);
        copy_in(orig.get(), ids.data(), LDS_MEM_HOST, n * sizeof(int32_t), s);
        map_ids(orig.get(), h->to_int.get(), n, all.get(), s);   // internal ids of h, in original order
        LDS_CUDA(cudaStreamSynchronize(s));
    }
    DevBuf<int64_t> pptr;
    DevBuf<int32_t> pidx;
    const int64_t np = build_all_patterns(h, tri, all.get(), n, shc, pptr, pidx);
    int64_t nnz = 0;
    if (np) LDS_CUDA(cudaMemcpyAsync(&nnz, pptr.get() + np, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    // vertex -> pattern incidences
    DevBuf<int32_t> ideg(n + 1, s), cursor(std::max(n, 1), s), vinc(std::max<int64_t>(nnz, 1), s);
    DevBuf<int64_t> vptr(n + 1, s);
    LDS_CUDA(cudaMemsetAsync(ideg.get(), 0, (n + 1) * sizeof(int32_t), s));
    LDS_CUDA(cudaMemsetAsync(cursor.get(), 0, std::max(n, 1) * sizeof(int32_t), s));
    if (nnz) LDS_LAUNCH(es_inc_count_kernel, grid_for(nnz, DB), DB, 0, s, pidx.get(), nnz, ideg.get());
    exclusive_scan_i32_to_i64(ideg.get(), vptr.get(), n + 1, s);
    if (np) LDS_LAUNCH(es_inc_fill_kernel, grid_for(np, DB), DB, 0, s, pptr.get(), pidx.get(), np, vptr.get(),
                       cursor.get(), vinc.get());
    // divide and conquer: at the ratio rho_0 = |P_F| / |F| of a sub-problem, the largest
    // maximiser of |P_F(X)| - rho_0 |X| is {x in F : phi(x) >= rho_0}.  Its value is 0
    // exactly when F is one level (every phi = rho_0, the mean of phi over F); otherwise
    // it is a proper nonempty subset, settled before the rest of F (highest first).
    DevBuf<uint8_t> state(std::max(n, 1), s), side(std::max(n, 1), s);
    DevBuf<int32_t> freeidx(std::max(n, 1), s);
    phin.alloc(std::max(n, 1), s);
    phid.alloc(std::max(n, 1), s);
    LDS_CUDA(cudaMemsetAsync(state.get(), ES_BELOW, std::max(n, 1), s));
    struct Sub {
        std::shared_ptr<DevBuf<int32_t>> list;
        int32_t size;
    };
    std::vector<Sub> todo;
    {
        auto l0 = std::make_shared<DevBuf<int32_t>>(std::max(n, 1), s);
        if (n) LDS_LAUNCH(es_iota_kernel, grid_for(n, DB), DB, 0, s, l0->get(), n);
        if (n) todo.push_back({l0, n});
    }
    const int64_t max_subs = 2 * (int64_t)n + 2;
    int64_t subs = 0;
    while (!todo.empty()) {
        Sub F = todo.back();
        todo.pop_back();
        ++subs;
        LDS_REQUIRE(subs <= max_subs, LDS_ETIMEOUT, "exact settle: decomposition did not terminate");
        const int32_t nf = F.size;
        const int32_t* Fp = F.list->get();
        LDS_LAUNCH(es_enter_kernel, grid_for(nf, DB), DB, 0, s, Fp, nf, state.get(), freeidx.get());
        DevBuf<int32_t> cnt(nf + 1, s);
        DevBuf<int64_t> off(nf + 1, s);
        LDS_CUDA(cudaMemsetAsync(cnt.get() + nf, 0, sizeof(int32_t), s));
        LDS_LAUNCH(es_emit_kernel<false>, grid_for((int64_t)nf * 32, DB), DB, 0, s, Fp, nf, vptr.get(), vinc.get(),
                   pptr.get(), pidx.get(), state.get(), cnt.get(), nullptr, nullptr);
        const int64_t nr = exclusive_scan_i32_to_i64(cnt.get(), off.get(), nf + 1, s);
        int64_t p = 0, q = 1;
        bool leaf = nr == 0;                      // no pattern: every phi in F is 0
        if (!leaf) {
            DevBuf<int32_t> pats(nr, s), len(nr + 1, s);
            LDS_LAUNCH(es_emit_kernel<true>, grid_for((int64_t)nf * 32, DB), DB, 0, s, Fp, nf, vptr.get(), vinc.get(),
                       pptr.get(), pidx.get(), state.get(), nullptr, off.get(), pats.get());
            LDS_CUDA(cudaMemsetAsync(len.get() + nr, 0, sizeof(int32_t), s));
            LDS_LAUNCH(es_len_kernel, grid_for(nr, DB), DB, 0, s, pats.get(), nr, pptr.get(), pidx.get(), state.get(),
                       len.get());
            DevBuf<int64_t> dptr(nr + 1, s);
            const int64_t rn = exclusive_scan_i32_to_i64(len.get(), dptr.get(), nr + 1, s);
            DevBuf<int32_t> ridx(std::max<int64_t>(rn, 1), s);
            LDS_LAUNCH(es_fill_kernel, grid_for(nr, DB), DB, 0, s, pats.get(), nr, pptr.get(), pidx.get(), state.get(),
                       freeidx.get(), dptr.get(), ridx.get());
            const int64_t g = std::gcd(nr, (int64_t)nf);
            p = nr / g;
            q = nf / g;
            LDS_REQUIRE(nr <= (int64_t)INT32_MAX, LDS_EOVERFLOW, "exact settle: %lld patterns", (long long)nr);
            const int64_t f = pattern_max_flow(dptr.get(), ridx.get(), (int32_t)nr, nf, p, q, nullptr, side.get(), false, s);
            ++flows;
            leaf = q * nr - f == 0;
            if (!leaf) {
                DevBuf<int32_t> sd(nf + 1, s);
                DevBuf<int64_t> pos(nf + 1, s);
                LDS_LAUNCH(u8_to_i32_kernel, grid_for(nf, DB), DB, 0, s, side.get(), nf, sd.get());
                LDS_CUDA(cudaMemsetAsync(sd.get() + nf, 0, sizeof(int32_t), s));
                const int64_t xs = exclusive_scan_i32_to_i64(sd.get(), pos.get(), nf + 1, s);
                LDS_REQUIRE(xs > 0 && xs < nf, LDS_ETIMEOUT, "exact settle: the cut at the mean ratio did not split");
                auto X = std::make_shared<DevBuf<int32_t>>(xs, s);
                auto Y = std::make_shared<DevBuf<int32_t>>(nf - xs, s);
                LDS_LAUNCH(es_split_kernel, grid_for(nf, DB), DB, 0, s, Fp, nf, sd.get(), pos.get(), X->get(), Y->get());
                LDS_LAUNCH(es_leave_kernel, grid_for(nf, DB), DB, 0, s, Fp, nf, state.get(), ES_BELOW, 0, 1, phin.get(),
                           phid.get());
                todo.push_back({Y, (int32_t)(nf - xs)});
                todo.push_back({X, (int32_t)xs});
                LDS_CUDA(cudaStreamSynchronize(s));
                continue;
            }
        }
        LDS_LAUNCH(es_leave_kernel, grid_for(nf, DB), DB, 0, s, Fp, nf, state.get(), ES_ABOVE, p, q, phin.get(),
                   phid.get());
        LDS_CUDA(cudaStreamSynchronize(s));
    }
    return flows;
}

void Driver::exact_settle(const int32_t* comp, int32_t csize) {
    ++stats.exact_settled;
    cudaStream_t s = st();
    lds_graph* h = subgraph(G, comp, csize, sc);
    struct Free { lds_graph* h; ~Free() { lds_free(h); } } fr{h};
    const int32_t n = h->n;
    DevBuf<int32_t> all;
    DevBuf<int64_t> phin, phid;
    vst.flows += exact_compact_numbers(h, tri, all, phin, phid);
    // LDSs of G[comp]: components of level sets with no neighbour of higher phi inside comp
    DevBuf<uint8_t> hflag(std::max(n, 1), s);
    if (n) LDS_LAUNCH(es_higher_kernel, grid_for((int64_t)n * 32, DB), DB, 0, s, all.get(), n, h->nact, h->rowptr.get(),
                      h->col.get(), h->to_orig.get(), phin.get(), phid.get(), hflag.get());
    std::vector<int64_t> hn(n), hd(n);
    std::vector<uint8_t> hf(n);
    std::vector<int32_t> hcomp(csize);
    LDS_CUDA(cudaMemcpyAsync(hn.data(), phin.get(), n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaMemcpyAsync(hd.data(), phid.get(), n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaMemcpyAsync(hf.data(), hflag.get(), n, cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaMemcpyAsync(hcomp.data(), comp, csize * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    // levels holding a vertex with no higher neighbour (the others hold no LDS)
    std::vector<std::pair<std::pair<int64_t, int64_t>, int32_t>> byl;     // ((num, den), local id)
    for (int32_t x = 0; x < n; ++x) {
        const int64_t g = std::gcd(hn[x], hd[x]);
        byl.push_back({{hn[x] / (g ? g : 1), hd[x] / (g ? g : 1)}, x});
    }
    std::sort(byl.begin(), byl.end());
    std::unordered_map<int32_t, int32_t> local;            // G internal id -> local id
    for (size_t a0 = 0; a0 < byl.size();) {
        size_t a1 = a0;
        bool any_free = false;
        while (a1 < byl.size() && byl[a1].first == byl[a0].first) any_free |= !hf[byl[a1++].second];
        const auto lv = byl[a0].first;
        if (any_free && (lv.first != 0 || include_zero)) {
            std::vector<int32_t> memb;
            for (size_t t = a0; t < a1; ++t) {
                memb.push_back(hcomp[byl[t].second]);
                local[hcomp[byl[t].second]] = byl[t].second;
            }
            DevBuf<int32_t> dm(memb.size(), s);
            copy_in(dm.get(), memb.data(), LDS_MEM_HOST, memb.size() * sizeof(int32_t), s);
            DevBuf<int32_t> cm;
            std::vector<int32_t> cs;
            components(G, dm.get(), (int32_t)memb.size(), sc, cm, cs);
            std::vector<int32_t> hm(cs.back());
            LDS_CUDA(cudaMemcpyAsync(hm.data(), cm.get(), hm.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
            for (size_t c = 0; c + 1 < cs.size(); ++c) {
                bool ok = true;
                for (int32_t t = cs[c]; t < cs[c + 1] && ok; ++t) ok = !hf[local[hm[t]]];
                if (!ok) continue;
                int64_t npat = 0;
                const int32_t* cp = cm.get() + cs[c];
                const int32_t csz = cs[c + 1] - cs[c];
                if (is_densest(G, tri, cp, csz, sc, &npat)) certify(cp, csz, npat);
            }
        }
        a0 = a1;
    }
}

void Driver::run() {
    auto T0 = std::chrono::steady_clock::now();
    const char* vb = getenv("LDS_VERBOSE");
    const bool verbose = vb && vb[0] == '1';
    auto elapsed = [&] { return std::chrono::duration<double>(std::chrono::steady_clock::now() - T0).count(); };
    cudaStream_t s = st();
    if (tri) ensure_triangles(G);
    {
        auto ti = std::chrono::steady_clock::now();
        init_bounds(G, bG);
        LDS_CUDA(cudaStreamSynchronize(s));
        tm.init += ms_since(ti);
    }
    if (verbose) fprintf(stderr, "[lds_topk] initial bounds at %.3fs\n", elapsed());
    DevBuf<int32_t> members;
    std::vector<int64_t> offs;
    round(G, bG, N, members, offs);
    if (verbose)
        fprintf(stderr, "[lds_topk] first round: fw %.1f ms, extract %.1f ms, prune %.1f ms\n", tm.fw, tm.sg, tm.prune);
    struct Item {
        std::shared_ptr<DevBuf<int32_t>> buf;
        int64_t off, size;
    };
    std::vector<Item> stack;
    auto mshared = std::make_shared<DevBuf<int32_t>>(std::move(members));
    for (size_t gidx = offs.size() - 1; gidx-- > 0;)
        stack.push_back({mshared, offs[gidx], offs[gidx + 1] - offs[gidx]});
    if (verbose)
        fprintf(stderr, "[lds_topk] first round done at %.3fs: %zu groups\n", elapsed(), stack.size());
    int64_t popped = 0;
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        const int32_t* S = it.buf->get() + it.off;
        const int32_t ssz = (int32_t)it.size;
        ++popped;
        if (verbose && (popped < 50 || popped % 1000 == 0))
            fprintf(stderr, "[lds_topk] %.3fs pop #%lld size %d stack %zu found %zu refined %lld flows %lld\n",
                    elapsed(), (long long)popped, ssz, stack.size(), found.size(), (long long)stats.refined,
                    (long long)vst.flows);
        int64_t rkn, rkd;
        if (kth(rkn, rkd)) {
            DevBuf<int32_t> flag(1, s);
            LDS_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int32_t), s));
            LDS_LAUNCH(any_ub_ge_kernel, grid_for(ssz, DB), DB, 0, s, S, ssz, bG.un.get(), bG.ud.get(), rkn, rkd, flag.get());
            int32_t hf = 0;
            LDS_CUDA(cudaMemcpyAsync(&hf, flag.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LDS_CUDA(cudaStreamSynchronize(s));
            if (!hf) {
                ++stats.skipped_by_bound;
                continue;
            }
        }
        // components of G[S], members ascending
        DevBuf<int32_t> sorted(std::max(ssz, 1), s);
        {
            DevBuf<uint64_t> key(std::max(ssz, 1), s);
            LDS_LAUNCH(sort_keys_kernel, grid_for(ssz, DB), DB, 0, s, S, ssz, key.get());
            radix_sort_u64(key.get(), nullptr, ssz, bit_length_u64((uint64_t)std::max(G->n, 1)), s);
            LDS_LAUNCH(unsort_keys_kernel, grid_for(ssz, DB), DB, 0, s, key.get(), ssz, sorted.get());
        }
        DevBuf<int32_t> cm;
        std::vector<int32_t> cs;
        auto tv0 = std::chrono::steady_clock::now();
        components(G, sorted.get(), ssz, sc, cm, cs);
        tm.comps += ms_since(tv0);
        if (verbose)
            fprintf(stderr, "[lds_topk]   %zu components in %.1f ms\n", cs.size() - 1,
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tv0).count());
        double small_ms = 0;
        int small_n = 0;
        const std::vector<uint8_t> closed = closed_components(cm.get(), cs);
        auto cmh = std::make_shared<DevBuf<int32_t>>(std::move(cm));
        for (size_t c = 0; c + 1 < cs.size(); ++c) {
            const int32_t* comp = cmh->get() + cs[c];
            const int32_t csize = cs[c + 1] - cs[c];
            int64_t npat = 0;
            auto tv1 = std::chrono::steady_clock::now();
            // a connected set of one vertex (of two, for triangles) holds no pattern: density 0,
            // never reported; a connected pair is one edge, its own densest subgraph
            const bool trivial = csize == 1 || csize == 2;
            if (trivial && (csize == 1 || tri) && !include_zero) continue;
            bool dens;
            if (trivial) {
                npat = (csize == 2 && !tri) ? 1 : 0;
                dens = true;
            } else {
                dens = is_densest(G, tri, comp, csize, sc, &npat);
            }
            auto tv2 = std::chrono::steady_clock::now();
            if (dens) {
                certify(comp, csize, npat, closed[c] != 0);
                auto tv3 = std::chrono::steady_clock::now();
                tm.verify += std::chrono::duration<double, std::milli>(tv3 - tv1).count();
                if (verbose && csize > 2)
                    fprintf(stderr, "[lds_topk]   component %d (|P|=%lld): densest %.1f ms, certify %.1f ms\n", csize,
                            (long long)npat, std::chrono::duration<double, std::milli>(tv2 - tv1).count(),
                            std::chrono::duration<double, std::milli>(tv3 - tv2).count());
                if (csize <= 2) {
                    small_ms += std::chrono::duration<double, std::milli>(tv3 - tv1).count();
                    ++small_n;
                }
                continue;
            }
            if (verbose)
                fprintf(stderr, "[lds_topk]   component %d (|P|=%lld): not densest %.1f ms\n", csize, (long long)npat,
                        std::chrono::duration<double, std::milli>(tv2 - tv1).count());
            tm.verify += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tv1).count();
            // refine on G[comp] (one handle for every retry: its whole-graph core
            // numbers are peeled once)
            int32_t n_try = N;
            auto tsub = std::chrono::steady_clock::now();
            lds_graph* h = subgraph(G, comp, csize, sc);
            struct Free { lds_graph* h; ~Free() { lds_free(h); } } fr{h};
            tm.sub += ms_since(tsub);
            while (true) {
                ++stats.refined;
                auto ts = std::chrono::steady_clock::now();
                Bounds bs;
                init_bounds(h, bs);
                LDS_CUDA(cudaStreamSynchronize(s));
                tm.sub_init += ms_since(ts);
                if (h->n)
                    LDS_LAUNCH(sub_bounds_kernel, grid_for(h->n, DB), DB, 0, s, h->to_orig.get(), comp, h->n,
                               bG.un.get(), bG.ud.get(), bs.un.get(), bs.ud.get());
                DevBuf<int32_t> sm;
                std::vector<int64_t> so;
                round(h, bs, n_try, sm, so);
                if (h->n)
                    LDS_LAUNCH(lift_lb_kernel, grid_for(h->n, DB), DB, 0, s, h->to_orig.get(), comp, h->n, bs.ln.get(),
                               bs.ld.get(), bG.ln.get(), bG.ld.get());
                const int64_t nsub = so.back();
                bool progress = !(so.size() == 2 && nsub == csize);
                if (progress) {
                    auto mp = std::make_shared<DevBuf<int32_t>>(std::max<int64_t>(nsub, 1), s);
                    if (nsub)
                        LDS_LAUNCH(to_parent_kernel, grid_for(nsub, DB), DB, 0, s, sm.get(), nsub, h->to_orig.get(), comp,
                                   mp->get());
                    LDS_CUDA(cudaStreamSynchronize(s));
                    for (size_t gidx = so.size() - 1; gidx-- > 0;)
                        stack.push_back({mp, so[gidx], so[gidx + 1] - so[gidx]});
                    break;
                }
                if (n_try >= 8 * N) {
                    exact_settle(comp, csize);
                    break;
                }
                n_try *= 2;
            }
            if (verbose)
                fprintf(stderr, "[lds_topk]   refined component %d in %.1f ms\n", csize,
                        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tv2).count());
        }
        if (verbose && small_n)
            fprintf(stderr, "[lds_topk]   %d components of size <= 2 verified in %.1f ms\n", small_n, small_ms);
        tm.refine += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tv0).count();
    }
    stats.flows = vst.flows;
    stats.denser_neighbour = vst.denser_neighbour;
    tm.total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - T0).count();
    if (verbose)
        fprintf(stderr,
                "[lds_topk] total %.1f ms: fw %.1f, extract %.1f, prune %.1f, verify %.1f, initial bounds %.1f, "
                "components %.1f, subgraph handles %.1f, their bounds %.1f\n",
                tm.total, tm.fw, tm.sg, tm.prune, tm.verify, tm.init, tm.comps, tm.sub, tm.sub_init);
    stats.ms_total = tm.total;
    stats.ms_fw = tm.fw;
    stats.ms_extract = tm.sg;
    stats.ms_prune = tm.prune;
    stats.ms_verify = tm.verify;
}

}  // namespace lds

using namespace lds;

namespace {
thread_local lds_topk_stats_t t_last_stats{};
}

extern "C" {

static void topk_run(lds_graph* g, int32_t k, lds_density d, int32_t iters, lds_precision p, bool include_zero,
                     lds_verify vmode, lds_result** out);

lds_status lds_topk(lds_graph* g, int32_t k, lds_density d, int32_t iters, lds_precision p, lds_result** out) {
    return guard([&] {
        LDS_REQUIRE(g && out, LDS_EINVAL, "lds_topk: NULL argument");
        topk_run(g, k, d, iters, p, false, LDS_VERIFY_BOUNDS, out);
    });
}

lds_status lds_topk_ex(lds_graph* g, int32_t k, lds_density d, int32_t iters, const lds_options* opt,
                       lds_result** out) {
    return guard([&] {
        LDS_REQUIRE(g && out, LDS_EINVAL, "lds_topk_ex: NULL argument");
        lds_options o{LDS_EXACT, nullptr, 0, LDS_VERIFY_BOUNDS};
        if (opt) o = *opt;
        LDS_REQUIRE(o.verify == LDS_VERIFY_BOUNDS || o.verify == LDS_VERIFY_CORE || o.verify == LDS_VERIFY_WHOLE,
                    LDS_EINVAL, "lds_topk_ex: bad verify value %d", (int)o.verify);
        cudaStream_t cs = static_cast<cudaStream_t>(o.cuda_stream);
        if (!cs || cs == g->stream) {
            topk_run(g, k, d, iters, o.prec, o.include_zero_density != 0, o.verify, out);
            return;
        }
        // the handle and its buffers follow the call's stream for the call, so that every
        // stream-ordered free is ordered after the work that used the buffer
        cudaStream_t own = g->stream;
        LDS_CUDA(cudaStreamSynchronize(own));
        set_stream(g, cs);
        struct Back {
            lds_graph* g;
            cudaStream_t own, cs;
            ~Back() {
                cudaStreamSynchronize(cs);
                set_stream(g, own);
            }
        } back{g, own, cs};
        topk_run(g, k, d, iters, o.prec, o.include_zero_density != 0, o.verify, out);
    });
}

static void topk_run(lds_graph* g, int32_t k, lds_density d, int32_t iters, lds_precision p, bool include_zero,
                     lds_verify vmode, lds_result** out) {
    {
        LDS_REQUIRE(k >= 1, LDS_EINVAL, "lds_topk: k = %d < 1", k);
        LDS_REQUIRE(d == LDS_EDGE || d == LDS_TRIANGLE, LDS_EINVAL, "lds_topk: bad density");
        LDS_REQUIRE(iters >= 1 && iters <= (d == LDS_EDGE ? 7000 : 3500), LDS_EINVAL,
                    "lds_topk: iters = %d out of range (refinement may run 8x iters)", iters);
        LDS_REQUIRE(p == LDS_EXACT || p == LDS_FP32 || p == LDS_FP64, LDS_EINVAL, "lds_topk: bad precision");
        *out = nullptr;
        Driver drv(g, d == LDS_TRIANGLE, k, iters, p, include_zero, vmode);
        drv.run();
        // order: density descending, ties by smallest member id (original ids)
        struct R {
            int64_t num, den;
            std::vector<int32_t> orig;
        };
        std::vector<R> rs;
        std::vector<int32_t> to_orig(g->n);
        if (g->n) {
            LDS_CUDA(cudaMemcpyAsync(to_orig.data(), g->to_orig.get(), g->n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                     g->stream));
            LDS_CUDA(cudaStreamSynchronize(g->stream));
        }
        for (auto& f : drv.found) {
            R r{f.num, f.den, {}};
            for (int32_t x : f.members) r.orig.push_back(to_orig[x]);
            std::sort(r.orig.begin(), r.orig.end());
            rs.push_back(std::move(r));
        }
        std::sort(rs.begin(), rs.end(), [](const R& a, const R& b) {
            i128 l = (i128)a.num * b.den, r = (i128)b.num * a.den;
            if (l != r) return l > r;
            return a.orig[0] < b.orig[0];
        });
        if ((int32_t)rs.size() > k) rs.resize(k);
        lds_result* res = (lds_result*)calloc(1, sizeof(lds_result));
        LDS_REQUIRE(res, LDS_ENOMEM, "lds_topk: host allocation failed");
        int64_t total = 0;
        for (auto& r : rs) total += (int64_t)r.orig.size();
        res->count = (int32_t)rs.size();
        res->dens_num = (int64_t*)malloc(sizeof(int64_t) * std::max<size_t>(rs.size(), 1));
        res->dens_den = (int64_t*)malloc(sizeof(int64_t) * std::max<size_t>(rs.size(), 1));
        res->offsets = (int64_t*)malloc(sizeof(int64_t) * (rs.size() + 1));
        res->vertices = (int32_t*)malloc(sizeof(int32_t) * std::max<int64_t>(total, 1));
        if (!res->dens_num || !res->dens_den || !res->offsets || !res->vertices) {
            lds_result_free(res);
            LDS_REQUIRE(false, LDS_ENOMEM, "lds_topk: host allocation failed");
        }
        res->offsets[0] = 0;
        for (size_t i = 0; i < rs.size(); ++i) {
            res->dens_num[i] = rs[i].num;
            res->dens_den[i] = rs[i].den;
            std::memcpy(res->vertices + res->offsets[i], rs[i].orig.data(), rs[i].orig.size() * sizeof(int32_t));
            res->offsets[i + 1] = res->offsets[i] + (int64_t)rs[i].orig.size();
        }
        t_last_stats = drv.stats;
        *out = res;
    }
}

void lds_result_free(lds_result* r) {
    if (!r) return;
    free(r->dens_num);
    free(r->dens_den);
    free(r->offsets);
    free(r->vertices);
    free(r);
}

lds_status lds_topk_last_stats(lds_topk_stats_t* st) {
    return guard([&] {
        LDS_REQUIRE(st, LDS_EINVAL, "lds_topk_last_stats: NULL argument");
        *st = t_last_stats;
    });
}

lds_status lds_compact_numbers(lds_graph* g, lds_density d, int64_t* num, int64_t* den, lds_mem where) {
    return guard([&] {
        LDS_REQUIRE(g && num && den, LDS_EINVAL, "lds_compact_numbers: NULL argument");
        LDS_REQUIRE(d == LDS_EDGE || d == LDS_TRIANGLE, LDS_EINVAL, "lds_compact_numbers: bad density");
        if (g->n == 0) return;
        DevBuf<int32_t> all;
        DevBuf<int64_t> phin, phid;
        exact_compact_numbers(g, d == LDS_TRIANGLE, all, phin, phid);
        copy_out(num, where, phin.get(), g->n * sizeof(int64_t), g->stream);
        copy_out(den, where, phid.get(), g->n * sizeof(int64_t), g->stream);
        LDS_CUDA(cudaStreamSynchronize(g->stream));
    });
}

}  // extern "C"
