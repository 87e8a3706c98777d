// Oriented, key-based Frank-Wolfe pass for CP(G) (Alg. 1), exact and binary32.
//
// Layout (the "FW view", built once per graph).  Vertices are relabelled by
// (degree descending, id ascending).  Every edge is stored once, in the row of
// its lower-ranked endpoint, as the fw id of its higher-ranked endpoint; on a
// power-law graph most stored targets are therefore high-degree vertices.
// Each vertex carries one 64-bit key: (load << B) | (2^B - 1 - id), B = bits of
// the vertex count, load = R (exact form) or the bit pattern of the binary32
// load.  Keys are distinct, and key_x < key_y exactly when r_x < r_y or
// (r_x == r_y and x > y): Alg. 1's choice with ties sent to the larger id.
//
// Pass.  Every block first copies the keys of the HOT highest-ranked vertices
// into shared memory (they receive most of the gathers) and zeroes shared
// counters for them.  Warps then stream 32-slot chunks: lane l of chunk g
// holds slot 32 g + l, finds its row from the chunk's first non-empty row and
// the row-start bits, compares the two keys, and the chunk's 32 decisions
// become one ballot word of this iteration's bit plane.  The row endpoint's
// count is the popcount of its lanes (one atomic per row segment); the
// target's count goes to shared memory for hot targets (flushed once per
// block) and to a global atomic otherwise.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "fw_internal.cuh"
#include "prims.cuh"

namespace lds {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int OP_THREADS = 1024;
constexpr int OP_UNROLL = 3;
constexpr int HOT = 16384;                       // hot vertices staged per block
constexpr size_t OP_SMEM = (size_t)HOT * 8 + (size_t)HOT * 4;

__device__ __forceinline__ uint32_t lanes_le(int lane) { return lane == 31 ? FULL : ((2u << lane) - 1u); }

// ---------------------------------------------------------------- view build

__global__ void rank_keys_kernel(const int64_t* rowptr, int32_t nact, int32_t maxdeg, int bits, uint64_t* key) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int64_t d = rowptr[x + 1] - rowptr[x];
        key[x] = ((uint64_t)(maxdeg - d) << bits) | (uint64_t)x;
    }
}

__global__ void perm_from_keys_kernel(const uint64_t* key, int32_t nact, uint64_t mask, int32_t* perm, int32_t* pos) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        int32_t x = (int32_t)(key[p] & mask);
        perm[p] = x;
        pos[x] = (int32_t)p;
    }
}

__global__ void slot_keys_kernel(const int32_t* eu, const int32_t* ev, int64_t m, const int32_t* pos, int64_t nact,
                                 uint64_t* key, uint32_t* eid) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int64_t a = pos[eu[e]], b = pos[ev[e]];
        int64_t src = a > b ? a : b, tgt = a > b ? b : a;
        key[e] = (uint64_t)(src * nact + tgt);
        eid[e] = (uint32_t)e;
    }
}

__global__ void slot_rows_kernel(const uint64_t* key, int64_t m, int64_t nact, int32_t* col, int32_t* start) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        uint64_t k = key[s];
        int64_t src = (int64_t)(k / (uint64_t)nact);
        bool st = s == 0 || (int64_t)(key[s - 1] / (uint64_t)nact) != src;
        col[s] = (int32_t)(k % (uint64_t)nact) | (st ? (int32_t)0x80000000 : 0);
        start[s] = st ? 1 : 0;
    }
}

__global__ void nz_rows_kernel(const uint64_t* key, const int32_t* start, const int64_t* rank_excl, int64_t m, int64_t nact,
                               int32_t* nzrow, int32_t* chunk_nz0) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        int64_t ridx = rank_excl[s] + start[s] - 1;
        if (start[s]) nzrow[ridx] = (int32_t)(key[s] / (uint64_t)nact);
        if ((s & 31) == 0) chunk_nz0[s >> 5] = (int32_t)ridx;
    }
}

// slots per row (rows are the fw ids of the lower-ranked endpoints)
__global__ void row_count_kernel(const uint64_t* key, int64_t m, int64_t nact, int32_t* cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride)
        atomicAdd(cnt + (int64_t)(key[s] / (uint64_t)nact), 1);
}

__global__ void widen_eid_kernel(const uint32_t* in, int64_t m, int64_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) out[i] = in[i];
}

__global__ void narrow_i64_i32_kernel(const int64_t* in, int64_t k, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = (int32_t)in[i];
}

// ---------------------------------------------------------------- iteration kernels

__global__ void okey_init_kernel(const int64_t* rowptr, const int32_t* perm, int32_t nact, int bits, bool fp32,
                                 uint64_t* key, float* r32) {
    const uint64_t lowmask = (bits >= 64) ? ~0ull : ((1ull << bits) - 1ull);
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        int32_t x = perm[p];
        int64_t d = rowptr[x + 1] - rowptr[x];
        uint64_t low = lowmask - (uint64_t)x;
        if (fp32) {
            float r = __fmul_rn((float)d, 0.5f);
            r32[p] = r;
            key[p] = ((uint64_t)__float_as_uint(r) << bits) | low;
        } else {
            key[p] = ((uint64_t)d << bits) | low;
        }
    }
}

template <int U>
__global__ void __launch_bounds__(OP_THREADS, 1)
    fw_opass_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ chunk_nz0,
                    const int32_t* __restrict__ nzrow, int64_t nslots, int64_t nchunks,
                    const uint64_t* __restrict__ key, int32_t nhot, int32_t* __restrict__ cnt,
                    uint32_t* __restrict__ plane) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* hkey = reinterpret_cast<uint64_t*>(smem);
    uint32_t* hcnt = reinterpret_cast<uint32_t*>(smem + (size_t)HOT * 8);
    {
        // stage the hot keys with 16-byte loads (key is 256-byte aligned)
        const uint4* k4 = reinterpret_cast<const uint4*>(key);
        uint4* h4 = reinterpret_cast<uint4*>(hkey);
        const int n4 = nhot >> 1;
#pragma unroll 8
        for (int i = threadIdx.x; i < n4; i += blockDim.x) h4[i] = __ldg(k4 + i);
        if ((nhot & 1) && threadIdx.x == 0) hkey[nhot - 1] = __ldg(key + nhot - 1);
        uint4* c4 = reinterpret_cast<uint4*>(hcnt);
        for (int i = threadIdx.x; i < (nhot + 3) >> 2; i += blockDim.x) c4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    // generic pointers select shared (hot) or global (cold) storage without
    // divergent branches: one load / one atomic per lane
    int32_t* const hcnt_i = reinterpret_cast<int32_t*>(hcnt);
    const int lane = threadIdx.x & 31;
    const uint32_t nch = (uint32_t)nchunks;            // slots and chunks fit 32 bits (m < 2^31)
    const uint32_t nsl = (uint32_t)nslots;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t le = lanes_le(lane);
    const uint32_t ge = ~((1u << lane) - 1u);
    int32_t cn[U], zn[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        uint32_t g = warp * U + k;
        uint32_t sl = (g << 5) + lane;
        cn[k] = (g < nch && sl < nsl) ? __ldg(col + sl) : 0;
        zn[k] = (g < nch) ? __ldg(chunk_nz0 + g) : 0;
    }
    for (uint32_t g0 = warp * U; g0 < nch; g0 += nwarps * U) {
        int32_t c[U], z0[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            c[k] = cn[k];
            z0[k] = zn[k];
            uint32_t g = g0 + nwarps * U + k;
            uint32_t sl = (g << 5) + lane;
            cn[k] = (g < nch && sl < nsl) ? __ldg(col + sl) : 0;
            zn[k] = (g < nch) ? __ldg(chunk_nz0 + g) : 0;
        }
        uint32_t f[U];
        int32_t src[U], tgt[U];
        bool valid[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            uint32_t sl = ((g0 + k) << 5) + lane;
            valid[k] = (g0 + k < nch) && sl < nsl;
            f[k] = __ballot_sync(FULL, c[k] < 0);
            tgt[k] = c[k] & 0x7fffffff;
            src[k] = valid[k] ? __ldg(nzrow + (z0[k] + __popc(f[k] & le) - (int)(f[k] & 1u))) : 0;
        }
        uint64_t ks[U], kt[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint64_t* ps = src[k] < nhot ? hkey + src[k] : key + src[k];
            const uint64_t* pt = tgt[k] < nhot ? hkey + tgt[k] : key + tgt[k];
            ks[k] = valid[k] ? *ps : 0;
            kt[k] = valid[k] ? *pt : 0;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t g = g0 + k;
            const bool srecv = valid[k] && ks[k] < kt[k];
            const uint32_t bal = __ballot_sync(FULL, srecv);
            if (lane == 0 && g < nch) plane[g] = bal;
            if (valid[k] && (lane == 0 || ((f[k] >> lane) & 1u))) {
                const uint32_t above = f[k] & ~le;
                const uint32_t below_end = above ? ((above & (0u - above)) - 1u) : FULL;
                const int cs = __popc(bal & ge & below_end);
                if (cs) atomicAdd(src[k] < nhot ? hcnt_i + src[k] : cnt + src[k], cs);
            }
            if (valid[k] && !srecv) atomicAdd(tgt[k] < nhot ? hcnt_i + tgt[k] : cnt + tgt[k], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nhot; i += blockDim.x) {
        uint32_t v = hcnt[i];
        if (v) atomicAdd(cnt + i, (int)v);
    }
}

// ---- 32-bit load words (used whenever every scaled load fits 32 bits and no
// degree reaches 65536).  The hot set doubles: HOT32 words of 4 bytes plus
// 16-bit counters packed two per word.  Ties (equal words) are rare and are
// broken by the internal ids, looked up only then.
constexpr int HOT32 = 32768;
// cooperative FW: hot vertices' global counts packed two per word (one atomic per
// word in the flush), and the grid sized to the work (chunks per block; 0: one
// block per SM whatever the size).  Both measured slower on the 1M-vertex graph
// and its refinement subgraphs, so both are off.
constexpr bool kPackedHot = false;
constexpr int kCoopChunksPerBlock = 0;
constexpr size_t OP32_SMEM = (size_t)HOT32 * 4 + (size_t)HOT32 * 2;

// One pass over every stored slot.  ROWS: the row endpoints' counts are left
// out of the pass; the vertex update takes them as popcounts of each row's bit
// range in this iteration's plane.  COOP: the body runs inside a cooperative
// kernel whose other blocks rewrite the load words between passes, so words
// are read through L2 (never the read-only data path).
template <int U, class Word, bool ROWS, bool COOP>
__device__ __forceinline__ void opass32_body(const int32_t* __restrict__ col, const int32_t* __restrict__ chunk_nz0,
                                             const int32_t* __restrict__ nzrow, int64_t nslots, int64_t nchunks,
                                             const Word* word, const int32_t* __restrict__ perm, int32_t nhot,
                                             int32_t* cnt, uint32_t* plane, Word* hword, uint32_t* hcnt2,
                                             uint32_t* hglob = nullptr) {
    {
        const uint4* w4 = reinterpret_cast<const uint4*>(word);
        uint4* h4 = reinterpret_cast<uint4*>(hword);
        const int n4 = nhot >> 2;
#pragma unroll 8
        for (int i = threadIdx.x; i < n4; i += blockDim.x) h4[i] = COOP ? __ldcg(w4 + i) : __ldg(w4 + i);
        for (int i = (n4 << 2) + threadIdx.x; i < nhot; i += blockDim.x) hword[i] = COOP ? __ldcg(word + i) : __ldg(word + i);
        uint4* c4 = reinterpret_cast<uint4*>(hcnt2);
        for (int i = threadIdx.x; i < (nhot + 7) >> 3; i += blockDim.x) c4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t nch = (uint32_t)nchunks;
    const uint32_t nsl = (uint32_t)nslots;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t le = lanes_le(lane);
    const uint32_t ge = ~((1u << lane) - 1u);
    int32_t cn[U], zn[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        uint32_t g = warp * U + k;
        uint32_t sl = (g << 5) + lane;
        cn[k] = (g < nch && sl < nsl) ? __ldg(col + sl) : 0;
        zn[k] = (g < nch) ? __ldg(chunk_nz0 + g) : 0;
    }
    for (uint32_t g0 = warp * U; g0 < nch; g0 += nwarps * U) {
        int32_t c[U], z0[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            c[k] = cn[k];
            z0[k] = zn[k];
            uint32_t g = g0 + nwarps * U + k;
            uint32_t sl = (g << 5) + lane;
            cn[k] = (g < nch && sl < nsl) ? __ldg(col + sl) : 0;
            zn[k] = (g < nch) ? __ldg(chunk_nz0 + g) : 0;
        }
        uint32_t f[U];
        int32_t src[U], tgt[U];
        bool valid[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            uint32_t sl = ((g0 + k) << 5) + lane;
            valid[k] = (g0 + k < nch) && sl < nsl;
            f[k] = __ballot_sync(FULL, c[k] < 0);
            tgt[k] = c[k] & 0x7fffffff;
            src[k] = valid[k] ? __ldg(nzrow + (z0[k] + __popc(f[k] & le) - (int)(f[k] & 1u))) : 0;
        }
        Word ws[U], wt[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const Word* ps = src[k] < nhot ? hword + src[k] : word + src[k];
            const Word* pt = tgt[k] < nhot ? hword + tgt[k] : word + tgt[k];
            ws[k] = valid[k] ? *ps : Word(0);
            wt[k] = valid[k] ? *pt : Word(0);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t g = g0 + k;
            bool srecv = valid[k] && ws[k] < wt[k];
            if (valid[k] && ws[k] == wt[k]) srecv = __ldg(perm + src[k]) > __ldg(perm + tgt[k]);
            const uint32_t bal = __ballot_sync(FULL, srecv);
            if (lane == 0 && g < nch) plane[g] = bal;
            if (!ROWS && valid[k] && (lane == 0 || ((f[k] >> lane) & 1u))) {
                const uint32_t above = f[k] & ~le;
                const uint32_t below_end = above ? ((above & (0u - above)) - 1u) : FULL;
                const int cs = __popc(bal & ge & below_end);
                if (cs) {
                    if (src[k] < nhot) atomicAdd(hcnt2 + (src[k] >> 1), (uint32_t)cs << ((src[k] & 1) << 4));
                    else atomicAdd(cnt + src[k], cs);
                }
            }
            if (valid[k] && !srecv) {
                if (ROWS) {
                    // one generic atomic: a packed shared counter for a hot target, else its global one
                    const bool hot = tgt[k] < nhot;
                    uint32_t* pc = hot ? hcnt2 + (tgt[k] >> 1) : reinterpret_cast<uint32_t*>(cnt + tgt[k]);
                    atomicAdd(pc, hot ? 1u << ((tgt[k] & 1) << 4) : 1u);
                } else if (tgt[k] < nhot) {
                    atomicAdd(hcnt2 + (tgt[k] >> 1), 1u << ((tgt[k] & 1) << 4));
                } else {
                    atomicAdd(cnt + tgt[k], 1);
                }
            }
        }
    }
    __syncthreads();
    // hglob: the hot vertices' global counts, packed like the shared ones (a vertex
    // receives at most its degree < 2^16 per iteration, so halves never carry)
    for (int i = threadIdx.x; i < (nhot + 1) >> 1; i += blockDim.x) {
        uint32_t v = hcnt2[i];
        if (v) {
            if (hglob) {
                atomicAdd(hglob + i, v);
            } else {
                if (v & 0xffffu) atomicAdd(cnt + 2 * i, (int)(v & 0xffffu));
                if (v >> 16) atomicAdd(cnt + 2 * i + 1, (int)(v >> 16));
            }
        }
    }
}

template <int U, class Word, bool ROWS>
__global__ void __launch_bounds__(OP_THREADS, 1)
    fw_opass32_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ chunk_nz0,
                      const int32_t* __restrict__ nzrow, int64_t nslots, int64_t nchunks,
                      const Word* __restrict__ word, const int32_t* __restrict__ perm, int32_t nhot,
                      int32_t* __restrict__ cnt, uint32_t* __restrict__ plane) {
    extern __shared__ __align__(16) unsigned char smem[];
    Word* hword = reinterpret_cast<Word*>(smem);
    uint32_t* hcnt2 = reinterpret_cast<uint32_t*>(smem + (size_t)HOT32 * 4);   // two 16-bit counters per word
    opass32_body<U, Word, ROWS, false>(col, chunk_nz0, nzrow, nslots, nchunks, word, perm, nhot, cnt, plane, hword,
                                       hcnt2);
}

__global__ void oword_init_kernel(const int64_t* rowptr, const int32_t* perm, int32_t nact, bool fp32, uint32_t* w32,
                                  float* r32) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        int64_t d = rowptr[perm[p] + 1] - rowptr[perm[p]];
        if (fp32) r32[p] = __fmul_rn((float)d, 0.5f);
        else w32[p] = (uint32_t)d;
    }
}

__global__ void oword_update_exact_kernel(uint32_t* __restrict__ w, int32_t* __restrict__ cnt, int32_t nact,
                                          uint32_t inc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        int32_t c = cnt[p];
        if (c) {
            w[p] += inc * (uint32_t)c;
            cnt[p] = 0;
        }
    }
}

// receipts of fw id p as a row endpoint in this iteration: the set bits of the
// plane over its row's slots [a, b)
__device__ __forceinline__ int32_t row_receipts(const int32_t* __restrict__ rowptr, const uint32_t* __restrict__ plane,
                                                int64_t p) {
    const int32_t a = rowptr[p], b = rowptr[p + 1];
    int32_t c = 0;
    if (a < b) {
        const int32_t wa = a >> 5, wb = (b - 1) >> 5;
        for (int32_t q = wa; q <= wb; ++q) {
            uint32_t bits = plane[q];
            if (q == wa) bits &= FULL << (a & 31);
            if (q == wb) bits &= lanes_le((b - 1) & 31);
            c += __popc(bits);
        }
    }
    return c;
}

__global__ void oword_update_rows_exact_kernel(uint32_t* __restrict__ w, int32_t* __restrict__ cnt,
                                               const int32_t* __restrict__ rowptr, const uint32_t* __restrict__ plane,
                                               int32_t nact, uint32_t inc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        const int32_t t = cnt[p];
        const int32_t c = t + row_receipts(rowptr, plane, p);
        if (c) w[p] += inc * (uint32_t)c;
        if (t) cnt[p] = 0;
    }
}

__global__ void oword_update_rows_fp32_kernel(float* __restrict__ r32, int32_t* __restrict__ cnt,
                                              const int32_t* __restrict__ rowptr, const uint32_t* __restrict__ plane,
                                              int32_t nact, float gam, float one_minus) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        const int32_t t = cnt[p];
        const int32_t c = t + row_receipts(rowptr, plane, p);
        r32[p] = __fadd_rn(__fmul_rn(one_minus, r32[p]), __fmul_rn(gam, (float)c));
        if (t) cnt[p] = 0;
    }
}

// Iterations i_first .. i_first + K - 1 in one cooperative launch: each runs
// the pass (targets' receipts; choice plane it of `planes`), a grid barrier,
// the vertex update (row endpoints' receipts from the plane, then R += 2(i+1) c
// for the exact words or r <- (1 - gamma) r + gamma c in binary32 with gamma =
// fl(2 / (i + 2))), and a second barrier before the next pass stages the new
// words.  Same iterates, ties and rounding as the per-iteration launches.
template <class Word>
__global__ void __launch_bounds__(OP_THREADS, 1)
    fw_coop32_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ chunk_nz0,
                     const int32_t* __restrict__ nzrow, int64_t nslots, int64_t nchunks, Word* word,
                     const int32_t* __restrict__ perm, int32_t nhot, int32_t* cnt, const int32_t* __restrict__ rowptr,
                     uint32_t* planes, int32_t nact, int32_t i_first, int32_t K, uint32_t* hglob) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    extern __shared__ __align__(16) unsigned char smem[];
    Word* hword = reinterpret_cast<Word*>(smem);
    uint32_t* hcnt2 = reinterpret_cast<uint32_t*>(smem + (size_t)HOT32 * 4);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int32_t it = 0; it < K; ++it) {
        const int32_t i = i_first + it;
        uint32_t* plane = planes + (int64_t)it * nchunks;
        opass32_body<OP_UNROLL, Word, true, true>(col, chunk_nz0, nzrow, nslots, nchunks, word, perm, nhot, cnt, plane,
                                                  hword, hcnt2, kPackedHot ? hglob : nullptr);
        grid.sync();
        // update: one work item per packed word of hot counts (two vertices), then one
        // per cold vertex; without packing, one item per vertex
        const int32_t hw = kPackedHot ? (nhot + 1) >> 1 : 0;
        const int64_t items = (int64_t)hw + (nact - (kPackedHot ? nhot : 0));
        for (int64_t it = tid; it < items; it += nthreads) {
            int32_t p0, np;
            uint32_t packed = 0;
            int32_t tc = 0;
            if (it < hw) {
                p0 = (int32_t)(2 * it);
                np = min(2, nhot - p0);
                packed = __ldcg(hglob + it);
                if (packed) hglob[it] = 0;
            } else {
                p0 = (kPackedHot ? nhot : 0) + (int32_t)(it - hw);
                np = 1;
                tc = __ldcg(cnt + p0);
                if (tc) cnt[p0] = 0;
            }
            for (int32_t j = 0; j < np; ++j) {
                const int32_t p = p0 + j;
                int32_t c = it < hw ? (int32_t)((packed >> (16 * j)) & 0xffffu) : tc;
                const int32_t a = rowptr[p], b = rowptr[p + 1];
                if (a < b) {
                    const int32_t wa = a >> 5, wb = (b - 1) >> 5;
                    for (int32_t q = wa; q <= wb; ++q) {
                        uint32_t bits = __ldcg(plane + q);
                        if (q == wa) bits &= FULL << (a & 31);
                        if (q == wb) bits &= lanes_le((b - 1) & 31);
                        c += __popc(bits);
                    }
                }
                if constexpr (std::is_same<Word, float>::value) {
                    const float gam = __fdiv_rn(2.0f, (float)(i + 2));
                    const float om = __fsub_rn(1.0f, gam);
                    word[p] = __fadd_rn(__fmul_rn(om, word[p]), __fmul_rn(gam, (float)c));
                } else {
                    if (c) word[p] += (uint32_t)(2 * (i + 1)) * (uint32_t)c;
                }
            }
        }
        grid.sync();
    }
}

__global__ void oword_update_fp32_kernel(float* __restrict__ r32, int32_t* __restrict__ cnt, int32_t nact, float gam,
                                         float one_minus) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        int32_t c = cnt[p];
        r32[p] = __fadd_rn(__fmul_rn(one_minus, r32[p]), __fmul_rn(gam, (float)c));
        if (c) cnt[p] = 0;
    }
}

__global__ void owords_to_internal_kernel(const uint32_t* w32, const float* r32, const int32_t* perm, int32_t nact,
                                          double Dn, bool fp32, double* r_int) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride)
        r_int[perm[p]] = fp32 ? (double)r32[p] : (double)w32[p] / Dn;
}

__global__ void okey_update_exact_kernel(uint64_t* __restrict__ key, int32_t* __restrict__ cnt, int32_t nact,
                                         int64_t inc, int bits) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        int32_t c = cnt[p];
        if (c) {
            key[p] += (uint64_t)(inc * (int64_t)c) << bits;
            cnt[p] = 0;
        }
    }
}

__global__ void okey_update_fp32_kernel(uint64_t* __restrict__ key, float* __restrict__ r32, int32_t* __restrict__ cnt,
                                        int32_t nact, float gam, float one_minus, int bits) {
    const uint64_t lowmask = (1ull << bits) - 1ull;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        int32_t c = cnt[p];
        float r = __fadd_rn(__fmul_rn(one_minus, r32[p]), __fmul_rn(gam, (float)c));
        r32[p] = r;
        key[p] = ((uint64_t)__float_as_uint(r) << bits) | (key[p] & lowmask);
        if (c) cnt[p] = 0;
    }
}

__global__ void fill_u32_kernel(uint32_t* p, int64_t n, uint32_t v) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

// ---------------------------------------------------------------- fold

constexpr int FOLD_TILE = 32;   // planes per tile and chunks per block

__global__ void __launch_bounds__(1024) fold_tiled_kernel(const uint32_t* __restrict__ planes, int nplanes,
                                                          int64_t nchunks, int64_t nitems, int64_t i_first,
                                                          int64_t mult, uint32_t* __restrict__ W) {
    __shared__ uint32_t tile[FOLD_TILE][FOLD_TILE + 1];
    const int t = threadIdx.x;
    const int c = t >> 5, l = t & 31;
    for (int64_t g0 = (int64_t)blockIdx.x * FOLD_TILE; g0 < nchunks; g0 += (int64_t)gridDim.x * FOLD_TILE) {
        const int64_t item = (g0 + c) * 32 + l;
        uint32_t acc = 0;
        for (int k0 = 0; k0 < nplanes; k0 += FOLD_TILE) {
            // thread t loads plane k0 + c, chunk g0 + l (coalesced along chunks)
            int kp = k0 + c;
            int64_t gc = g0 + l;
            tile[c][l] = (kp < nplanes && gc < nchunks) ? __ldg(planes + (int64_t)kp * nchunks + gc) : 0u;
            __syncthreads();
            int kmax = min(FOLD_TILE, nplanes - k0);
            for (int j = 0; j < kmax; ++j) {
                uint32_t b = (tile[j][c] >> l) & 1u;
                acc += b * (uint32_t)(mult * (i_first + k0 + j + 1));
            }
            __syncthreads();
        }
        if (item < nitems) W[item] += acc;
    }
}

// ---------------------------------------------------------------- outputs

__global__ void oloads_from_w_kernel(const int32_t* col, const int32_t* chunk_nz0, const int32_t* nzrow, int64_t m,
                                     const uint32_t* W, uint32_t Dn, unsigned long long* R) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        // row of slot s: the chunk's first row plus the row starts after it, up to s
        int64_t g = s >> 5;
        int64_t ridx = chunk_nz0[g];
        for (int64_t q = (g << 5) + 1; q <= s; ++q)
            if (col[q] < 0) ++ridx;
        int32_t src = nzrow[ridx];
        int32_t tgt = col[s] & 0x7fffffff;
        atomicAdd(R + src, (unsigned long long)W[s]);
        atomicAdd(R + tgt, (unsigned long long)(Dn - W[s]));
    }
}

__global__ void oedge_outputs_kernel(const int32_t* col, const int32_t* chunk_nz0, const int32_t* nzrow,
                                     const int64_t* slot_edge, int64_t m, const int32_t* pos, const int32_t* eu,
                                     const uint32_t* W, uint32_t Dn, const uint32_t* last_plane, int64_t* Wout,
                                     uint8_t* last) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += stride) {
        int64_t g = s >> 5;
        int64_t ridx = chunk_nz0[g];
        for (int64_t q = (g << 5) + 1; q <= s; ++q)
            if (col[q] < 0) ++ridx;
        int32_t src = nzrow[ridx];
        int64_t e = slot_edge[s];
        bool u_is_src = pos[eu[e]] == src;
        if (Wout) Wout[e] = u_is_src ? (int64_t)W[s] : (int64_t)(Dn - W[s]);
        if (last) {
            uint32_t b = (last_plane[g] >> (s & 31)) & 1u;
            last[e] = (uint8_t)(u_is_src ? b : 1u - b);
        }
    }
}

__global__ void okeys_to_internal_kernel(const uint64_t* key, const float* r32, const int32_t* perm, int32_t nact,
                                         int bits, double Dn, bool fp32, double* r_int) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) {
        double r = fp32 ? (double)r32[p] : (double)(int64_t)(key[p] >> bits) / Dn;
        r_int[perm[p]] = r;
    }
}

__global__ void permute_back_i64_kernel(const unsigned long long* in, const int32_t* perm, int32_t nact, int64_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += stride) out[perm[p]] = (int64_t)in[p];
}

}  // namespace

void fold_planes(const uint32_t* planes, int nplanes, int64_t nchunks, int64_t nitems, int64_t i_first, int64_t mult,
                 uint32_t* W, cudaStream_t s) {
    if (nitems <= 0 || nplanes <= 0) return;
    int64_t blocks = (nchunks + FOLD_TILE - 1) / FOLD_TILE;
    unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms() * 2));
    LDS_LAUNCH(fold_tiled_kernel, grid, 1024, 0, s, planes, nplanes, nchunks, nitems, i_first, mult, W);
}

void ensure_fw_view(lds_graph* g) {
    if (g->fwv_built) return;
    cudaStream_t s = g->stream;
    const int32_t nact = g->nact;
    const int64_t m = g->m;
    const int blk = 256;
    int bits = std::max(1, bit_length_u64((uint64_t)std::max(nact, 1)));
    g->fwv_bits = bits;
    g->fwv_perm.alloc(std::max(nact, 1), s);
    g->fwv_pos.alloc(std::max(nact, 1), s);
    if (nact > 0) {
        DevBuf<uint64_t> rk(nact, s);
        int32_t maxdeg = g->info.max_degree;
        LDS_LAUNCH(rank_keys_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), nact, maxdeg, bits, rk.get());
        radix_sort_u64(rk.get(), nullptr, nact, bits + bit_length_u64((uint64_t)maxdeg), s);
        uint64_t mask = (1ull << bits) - 1ull;
        LDS_LAUNCH(perm_from_keys_kernel, grid_for(nact, blk), blk, 0, s, rk.get(), nact, mask, g->fwv_perm.get(),
                   g->fwv_pos.get());
    }
    g->fwv_col.alloc(std::max<int64_t>(m, 1), s);
    g->fwv_chunk_nz0.alloc(std::max<int64_t>((m + 31) / 32, 1), s);
    g->fwv_edge.alloc(std::max<int64_t>(m, 1), s);
    if (m > 0) {
        DevBuf<uint64_t> key(m, s);
        DevBuf<uint32_t> eid(m, s);
        LDS_LAUNCH(slot_keys_kernel, grid_for(m, blk), blk, 0, s, g->eu.get(), g->ev.get(), m, g->fwv_pos.get(),
                   (int64_t)nact, key.get(), eid.get());
        radix_sort_u64(key.get(), eid.get(), m, bit_length_u64((uint64_t)nact * (uint64_t)nact), s);
        DevBuf<int32_t> start(m, s);
        DevBuf<int64_t> rexcl(m, s);
        LDS_LAUNCH(slot_rows_kernel, grid_for(m, blk), blk, 0, s, key.get(), m, (int64_t)nact, g->fwv_col.get(),
                   start.get());
        int64_t nz = exclusive_scan_i32_to_i64(start.get(), rexcl.get(), m, s);
        g->fwv_nz = nz;
        g->fwv_nzrow.alloc(std::max<int64_t>(nz, 1), s);
        LDS_LAUNCH(nz_rows_kernel, grid_for(m, blk), blk, 0, s, key.get(), start.get(), rexcl.get(), m, (int64_t)nact,
                   g->fwv_nzrow.get(), g->fwv_chunk_nz0.get());
        LDS_LAUNCH(widen_eid_kernel, grid_for(m, blk), blk, 0, s, eid.get(), m, g->fwv_edge.get());
        DevBuf<int32_t> rc(nact + 1, s);
        DevBuf<int64_t> rp64(nact + 1, s);
        LDS_CUDA(cudaMemsetAsync(rc.get(), 0, (nact + 1) * sizeof(int32_t), s));
        LDS_LAUNCH(row_count_kernel, grid_for(m, blk), blk, 0, s, key.get(), m, (int64_t)nact, rc.get());
        exclusive_scan_i32_to_i64(rc.get(), rp64.get(), (int64_t)nact + 1, s);
        g->fwv_rowptr.alloc(nact + 1, s);
        LDS_LAUNCH(narrow_i64_i32_kernel, grid_for(nact + 1, blk), blk, 0, s, rp64.get(), (int64_t)nact + 1,
                   g->fwv_rowptr.get());
    } else {
        g->fwv_rowptr.alloc(std::max(nact, 0) + 1, s);
        LDS_CUDA(cudaMemsetAsync(g->fwv_rowptr.get(), 0, (std::max(nact, 0) + 1) * sizeof(int32_t), s));
    }
    LDS_CUDA(cudaStreamSynchronize(s));
    g->fwv_built = true;
}

// Folds, loads and outputs shared by both word widths.
static void oriented_outputs(lds_graph* g, int N, const uint32_t* W, const uint32_t* last_plane, int64_t nchunks,
                             bool want_w, bool want_last, EdgeFwOut& out) {
    cudaStream_t s = g->stream;
    const int blk = 256;
    const int32_t n = g->n, nact = g->nact;
    const int64_t m = g->m;
    const int64_t Dn = (int64_t)(N + 1) * (N + 2);
    out.R_int.alloc(std::max(n, 1), s);
    LDS_CUDA(cudaMemsetAsync(out.R_int.get(), 0, std::max(n, 1) * sizeof(int64_t), s));
    if (nact) {
        DevBuf<unsigned long long> Rfw(nact, s);
        LDS_CUDA(cudaMemsetAsync(Rfw.get(), 0, nact * sizeof(unsigned long long), s));
        if (m)
            LDS_LAUNCH(oloads_from_w_kernel, grid_for(m, blk), blk, 0, s, g->fwv_col.get(), g->fwv_chunk_nz0.get(),
                       g->fwv_nzrow.get(), m, W, (uint32_t)Dn, Rfw.get());
        LDS_LAUNCH(permute_back_i64_kernel, grid_for(nact, blk), blk, 0, s, Rfw.get(), g->fwv_perm.get(), nact,
                   out.R_int.get());
    }
    if ((want_w || want_last) && m) {
        if (want_w) out.W_edge.alloc(m, s);
        if (want_last) out.last_edge.alloc(m, s);
        LDS_LAUNCH(oedge_outputs_kernel, grid_for(m, blk), blk, 0, s, g->fwv_col.get(), g->fwv_chunk_nz0.get(),
                   g->fwv_nzrow.get(), g->fwv_edge.get(), m, g->fwv_pos.get(), g->eu.get(), W, (uint32_t)Dn, last_plane,
                   want_w ? out.W_edge.get() : nullptr, want_last ? out.last_edge.get() : nullptr);
        if (want_last && N == 0) LDS_CUDA(cudaMemsetAsync(out.last_edge.get(), 0, m, s));
    }
}

bool run_edge_fw_oriented(lds_graph* g, int N, lds_precision p, bool want_w, bool want_last, EdgeFwOut& out,
                          PassTimer& timer) {
    if (p != LDS_EXACT && p != LDS_FP32) return false;
    const int32_t nact = g->nact;
    const int64_t m = g->m;
    const int bits = std::max(1, bit_length_u64((uint64_t)std::max(nact, 1)));
    const int64_t maxdeg = std::max(g->info.max_degree, 1);
    const int64_t Dn = (int64_t)(N + 1) * (N + 2);
    // 32-bit words: every scaled load below 2^32 and per-block hot counts below 2^16
    extern int g_fw_variant;
    // variant 3 keeps the row endpoints' counts inside the pass; variant 4 counts them
    // in the vertex update but launches pass and update once per iteration; the
    // default runs many iterations per cooperative launch
    const bool rows = g_fw_variant != 3;
    const bool coop = g_fw_variant == 0 || g_fw_variant == 5 || g_fw_variant == 6;
    bool use32 = g_fw_variant != 2 && maxdeg < 65536 && (p == LDS_FP32 || (unsigned __int128)maxdeg * (unsigned __int128)Dn < ((unsigned __int128)1 << 32));
    if (!use32) {
        if (p == LDS_EXACT) {
            unsigned __int128 maxR = (unsigned __int128)maxdeg * (unsigned __int128)Dn;
            int rbits = 0;
            while (maxR) { ++rbits; maxR >>= 1; }
            if (rbits + bits > 63) return false;
        } else if (32 + bits > 64) {
            return false;
        }
    }
    ensure_fw_view(g);
    cudaStream_t s = g->stream;
    const int blk = 256;
    const bool fp32 = p == LDS_FP32;
    const int64_t nchunks = (m + 31) / 32;
    DevBuf<float> r32(fp32 ? std::max(nact, 1) : 0, s);
    DevBuf<int32_t> cnt(std::max(nact, 1), s);
    LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, std::max(nact, 1) * sizeof(int32_t), s));
    const int K = planes_capacity(nchunks, N);
    DevBuf<uint32_t> planes(std::max<int64_t>(1, (int64_t)K * nchunks), s);
    DevBuf<uint32_t> W(std::max<int64_t>(m, 1), s);
    if (m) LDS_LAUNCH(fill_u32_kernel, grid_for(m, blk), blk, 0, s, W.get(), m, 1u);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms(), (nchunks + 31) / 32));
    DevBuf<uint64_t> key(use32 ? 0 : std::max(nact, 1), s);
    DevBuf<uint32_t> w32(use32 && !fp32 ? std::max(nact, 1) : 0, s);
    int32_t nhot;
    if (use32) {
        nhot = std::min(nact, HOT32);
        if (nact)
            LDS_LAUNCH(oword_init_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), g->fwv_perm.get(), nact, fp32,
                       w32.get(), r32.get());
        LDS_CUDA(cudaFuncSetAttribute(fw_coop32_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)OP32_SMEM));
        LDS_CUDA(cudaFuncSetAttribute(fw_coop32_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)OP32_SMEM));
        LDS_CUDA(cudaFuncSetAttribute(fw_opass32_kernel<OP_UNROLL, float, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OP32_SMEM));
        LDS_CUDA(cudaFuncSetAttribute(fw_opass32_kernel<OP_UNROLL, uint32_t, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OP32_SMEM));
        LDS_CUDA(cudaFuncSetAttribute(fw_opass32_kernel<OP_UNROLL, float, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OP32_SMEM));
        LDS_CUDA(cudaFuncSetAttribute(fw_opass32_kernel<OP_UNROLL, uint32_t, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OP32_SMEM));
        g->pass_kernel = "fw_opass32_kernel";
    } else {
        nhot = std::min(nact, HOT);
        if (nact)
            LDS_LAUNCH(okey_init_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), g->fwv_perm.get(), nact, bits,
                       fp32, key.get(), r32.get());
        LDS_CUDA(cudaFuncSetAttribute(fw_opass_kernel<OP_UNROLL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)OP_SMEM));
        g->pass_kernel = "fw_opass_kernel";
    }
    int stored = 0;
    int64_t first_i = 1;
    int64_t last_plane = 0;
    if (use32 && coop && nchunks) {
        int per_sm = 0;
        if (fp32) LDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_coop32_kernel<float>, OP_THREADS,
                                                                         OP32_SMEM));
        else LDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_coop32_kernel<uint32_t>, OP_THREADS,
                                                                    OP32_SMEM));
        LDS_REQUIRE(per_sm >= 1, LDS_ECUDA, "fw: the cooperative pass cannot be resident");
        g->pass_kernel = "fw_coop32_kernel";
        const unsigned cgrid =
            kCoopChunksPerBlock > 0
                ? (unsigned)std::max<int64_t>(
                      1, std::min<int64_t>(grid, (nchunks + kCoopChunksPerBlock - 1) / kCoopChunksPerBlock))
                : grid;
        DevBuf<uint32_t> hglob(((nhot + 1) >> 1) + 1, s);
        LDS_CUDA(cudaMemsetAsync(hglob.get(), 0, (((nhot + 1) >> 1) + 1) * sizeof(uint32_t), s));
        int i = 1;
        while (i <= N) {
            int32_t kk = std::min(K - stored, N - i + 1);
            uint32_t* pl = planes.get() + (int64_t)stored * nchunks;
            const int32_t* pcol = g->fwv_col.get();
            const int32_t* pz = g->fwv_chunk_nz0.get();
            const int32_t* pnz = g->fwv_nzrow.get();
            const int32_t* pperm = g->fwv_perm.get();
            const int32_t* prow = g->fwv_rowptr.get();
            int32_t* pcnt = cnt.get();
            int64_t nsl = m, nch = nchunks;
            int32_t nh = nhot, na = nact, i0 = i;
            void* wp = fp32 ? (void*)r32.get() : (void*)w32.get();
            uint32_t* hg = hglob.get();
            void* args[] = {(void*)&pcol, (void*)&pz, (void*)&pnz, (void*)&nsl, (void*)&nch, (void*)&wp, (void*)&pperm,
                            (void*)&nh, (void*)&pcnt, (void*)&prow, (void*)&pl, (void*)&na, (void*)&i0, (void*)&kk,
                            (void*)&hg};
            timer.start(s);
            if (fp32)
                LDS_CUDA(cudaLaunchCooperativeKernel((void*)fw_coop32_kernel<float>, dim3(cgrid), dim3(OP_THREADS),
                                                     args, OP32_SMEM, s));
            else
                LDS_CUDA(cudaLaunchCooperativeKernel((void*)fw_coop32_kernel<uint32_t>, dim3(cgrid), dim3(OP_THREADS),
                                                     args, OP32_SMEM, s));
            g_launches.fetch_add(1, std::memory_order_relaxed);
            timer.stop(s, kk);
            stored += kk;
            i += kk;
            if (stored == K || i > N) {
                fold_planes(planes.get(), stored, nchunks, m, first_i, 2, W.get(), s);
                last_plane = stored - 1;
                if (i <= N) {
                    stored = 0;
                    first_i = i;
                }
            }
        }
    }
    for (int i = (use32 && coop && nchunks) ? N + 1 : 1; i <= N; ++i) {
        uint32_t* plane = planes.get() + (int64_t)stored * nchunks;
        if (nchunks) {
            const float gam = 2.0f / (float)(i + 2);
            const float om = 1.0f - gam;
            timer.start(s);
            if (use32 && rows && fp32)
                LDS_LAUNCH((fw_opass32_kernel<OP_UNROLL, float, true>), grid, OP_THREADS, OP32_SMEM, s,
                           g->fwv_col.get(), g->fwv_chunk_nz0.get(), g->fwv_nzrow.get(), m, nchunks, r32.get(),
                           g->fwv_perm.get(), nhot, cnt.get(), plane);
            else if (use32 && rows)
                LDS_LAUNCH((fw_opass32_kernel<OP_UNROLL, uint32_t, true>), grid, OP_THREADS, OP32_SMEM, s,
                           g->fwv_col.get(), g->fwv_chunk_nz0.get(), g->fwv_nzrow.get(), m, nchunks, w32.get(),
                           g->fwv_perm.get(), nhot, cnt.get(), plane);
            else if (use32 && fp32)
                LDS_LAUNCH((fw_opass32_kernel<OP_UNROLL, float, false>), grid, OP_THREADS, OP32_SMEM, s,
                           g->fwv_col.get(), g->fwv_chunk_nz0.get(), g->fwv_nzrow.get(), m, nchunks, r32.get(),
                           g->fwv_perm.get(), nhot, cnt.get(), plane);
            else if (use32)
                LDS_LAUNCH((fw_opass32_kernel<OP_UNROLL, uint32_t, false>), grid, OP_THREADS, OP32_SMEM, s,
                           g->fwv_col.get(), g->fwv_chunk_nz0.get(), g->fwv_nzrow.get(), m, nchunks, w32.get(),
                           g->fwv_perm.get(), nhot, cnt.get(), plane);
            else
                LDS_LAUNCH(fw_opass_kernel<OP_UNROLL>, grid, OP_THREADS, OP_SMEM, s, g->fwv_col.get(),
                           g->fwv_chunk_nz0.get(), g->fwv_nzrow.get(), m, nchunks, key.get(), nhot, cnt.get(), plane);
            timer.stop(s);
            if (use32 && rows && fp32)
                LDS_LAUNCH(oword_update_rows_fp32_kernel, grid_for(nact, blk), blk, 0, s, r32.get(), cnt.get(),
                           g->fwv_rowptr.get(), plane, nact, gam, om);
            else if (use32 && rows)
                LDS_LAUNCH(oword_update_rows_exact_kernel, grid_for(nact, blk), blk, 0, s, w32.get(), cnt.get(),
                           g->fwv_rowptr.get(), plane, nact, (uint32_t)(2 * (i + 1)));
            else if (use32 && fp32)
                LDS_LAUNCH(oword_update_fp32_kernel, grid_for(nact, blk), blk, 0, s, r32.get(), cnt.get(), nact, gam, om);
            else if (use32)
                LDS_LAUNCH(oword_update_exact_kernel, grid_for(nact, blk), blk, 0, s, w32.get(), cnt.get(), nact,
                           (uint32_t)(2 * (i + 1)));
            else if (!fp32)
                LDS_LAUNCH(okey_update_exact_kernel, grid_for(nact, blk), blk, 0, s, key.get(), cnt.get(), nact,
                           2 * (int64_t)(i + 1), bits);
            else
                LDS_LAUNCH(okey_update_fp32_kernel, grid_for(nact, blk), blk, 0, s, key.get(), r32.get(), cnt.get(),
                           nact, gam, om, bits);
        }
        ++stored;
        if (stored == K || i == N) {
            fold_planes(planes.get(), stored, nchunks, m, first_i, 2, W.get(), s);
            last_plane = stored - 1;
            if (i < N) {
                stored = 0;
                first_i = i + 1;
            }
        }
    }
    const int32_t n = g->n;
    out.r_int.alloc(std::max(n, 1), s);
    LDS_CUDA(cudaMemsetAsync(out.r_int.get(), 0, std::max(n, 1) * sizeof(double), s));
    if (nact) {
        if (use32)
            LDS_LAUNCH(owords_to_internal_kernel, grid_for(nact, blk), blk, 0, s, w32.get(), r32.get(), g->fwv_perm.get(),
                       nact, (double)Dn, fp32, out.r_int.get());
        else
            LDS_LAUNCH(okeys_to_internal_kernel, grid_for(nact, blk), blk, 0, s, key.get(), r32.get(), g->fwv_perm.get(),
                       nact, bits, (double)Dn, fp32, out.r_int.get());
    }
    oriented_outputs(g, N, W.get(), planes.get() + last_plane * nchunks, nchunks, want_w, want_last, out);
    LDS_CUDA(cudaStreamSynchronize(s));
    return true;
}

}  // namespace lds
