// Frank-Wolfe iterations for CP(G) (Eq. 2, Alg. 1) and for the triangle
// program (Eq. 4, Alg. 6).
//
// Edge pass (one launch per iteration).  The symmetric CSR is streamed in
// 32-slot chunks, one chunk per warp step.  Slot (x, y) decides whether x
// receives the edge {x, y} in this iteration: r_x < r_y, or r_x == r_y and
// x > y (Alg. 1 with u < v orientation; ties to the larger id).  The 32
// decisions of a chunk are one ballot word, stored as this iteration's bit
// plane; the per-row count of received edges is the popcount of the ballot
// over the row's lanes, added with one atomic per (row, chunk).  The first slot
// of every row carries bit 31 in the column array, so a lane finds its row from
// the chunk's first row plus a popcount of the row starts before it.
//
// Vertex pass: R_x += 2(i+1) c_x (exact form, D_i = (i+1)(i+2)) or
// r_x = (1 - gamma) r_x + gamma c_x in binary32 (every operation rounded,
// matching the oracle).  Weights are not touched during the iterations: the bit
// planes are folded into per-slot weights W = D_N alpha every K iterations:
// W_slot += sum_i 2(i+1) bit_i.
//
// Triangle pass: one thread per triangle (a < b < c): the receiving vertex is
// the lowest-load one, ties to the larger id (later column); the column is
// stored as two bit planes and the count is added with warp-aggregated atomics.
//
// The binary64 path is Alg. 1 literally: one alpha per slot updated as
// alpha = (1 - gamma) alpha + gamma alpha_hat, then r_x summed over row x left
// to right by one thread per row.
#include <algorithm>
#include <cmath>

#include "fw_internal.cuh"
#include "prims.cuh"

namespace lds {

int g_fw_variant = 0;

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int FW_THREADS = 256;
constexpr int FW_UNROLL = 4;

__device__ __forceinline__ uint32_t lanes_le(int lane) { return lane == 31 ? FULL : ((2u << lane) - 1u); }

template <class L>
__device__ __forceinline__ bool receives(L rx, L ry, int32_t x, int32_t y) {
    return (rx < ry) || (rx == ry && x > y);
}

// One edge pass over all slots.  plane[g] receives the ballot of chunk g.
template <class L>
__global__ void __launch_bounds__(FW_THREADS) fw_edge_pass_kernel(const int32_t* __restrict__ fwcol,
                                                                  const int32_t* __restrict__ chunk_row0,
                                                                  int64_t nslots, int64_t nchunks,
                                                                  const L* __restrict__ R, int32_t* __restrict__ cnt,
                                                                  uint32_t* __restrict__ plane) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t le = lanes_le(lane);
    const uint32_t ge = ~((1u << lane) - 1u);
    for (int64_t g0 = warp * FW_UNROLL; g0 < nchunks; g0 += nwarps * FW_UNROLL) {
        int32_t c[FW_UNROLL], r0[FW_UNROLL];
#pragma unroll
        for (int k = 0; k < FW_UNROLL; ++k) {
            int64_t g = g0 + k;
            int64_t s = (g << 5) + lane;
            c[k] = (s < nslots) ? __ldg(fwcol + s) : 0;
            r0[k] = (g < nchunks) ? __ldg(chunk_row0 + g) : 0;
        }
        L ru[FW_UNROLL], rv[FW_UNROLL];
        int32_t uu[FW_UNROLL], vv[FW_UNROLL];
        uint32_t f[FW_UNROLL];
#pragma unroll
        for (int k = 0; k < FW_UNROLL; ++k) {
            int64_t s = ((g0 + k) << 5) + lane;
            f[k] = __ballot_sync(FULL, c[k] < 0);
            vv[k] = c[k] & 0x7fffffff;
            uu[k] = r0[k] + __popc(f[k] & le) - (int)(f[k] & 1u);
            if (s < nslots) {
                ru[k] = __ldg(R + uu[k]);
                rv[k] = __ldg(R + vv[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < FW_UNROLL; ++k) {
            int64_t g = g0 + k;
            int64_t s = (g << 5) + lane;
            bool valid = s < nslots;
            bool recv = valid && receives<L>(ru[k], rv[k], uu[k], vv[k]);
            uint32_t bal = __ballot_sync(FULL, recv);
            if (g < nchunks) {
                if (lane == 0) plane[g] = bal;
                bool starts = lane == 0 || ((f[k] >> lane) & 1u);
                if (valid && starts) {
                    uint32_t above = f[k] & ~le;
                    uint32_t below_end = above ? ((above & (0u - above)) - 1u) : FULL;
                    int cntk = __popc(bal & ge & below_end);
                    if (cntk) atomicAdd(cnt + uu[k], cntk);
                }
            }
        }
    }
}

__global__ void fw_update_exact_kernel(int64_t* __restrict__ R, int32_t* __restrict__ cnt, int32_t nact, int64_t inc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int32_t cx = cnt[x];
        if (cx) {
            R[x] += inc * (int64_t)cx;
            cnt[x] = 0;
        }
    }
}

__global__ void fw_update_fp32_kernel(float* __restrict__ r, int32_t* __restrict__ cnt, int32_t nact, float gam,
                                      float one_minus) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int32_t cx = cnt[x];
        r[x] = __fadd_rn(__fmul_rn(one_minus, r[x]), __fmul_rn(gam, (float)cx));
        if (cx) cnt[x] = 0;
    }
}

// W_slot[s] += sum over stored planes k of bit_k(s) * (mult * (i_first + k + 1))
__global__ void fw_fold_kernel(const uint32_t* __restrict__ planes, int nplanes, int64_t nchunks, int64_t nslots,
                               int64_t i_first, int64_t mult, uint32_t* __restrict__ W) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += stride) {
        int64_t g = s >> 5;
        int lane = (int)(s & 31);
        uint32_t acc = 0;
        for (int k = 0; k < nplanes; ++k) {
            uint32_t b = (__ldg(planes + (int64_t)k * nchunks + g) >> lane) & 1u;
            acc += b * (uint32_t)(mult * (i_first + k + 1));
        }
        W[s] += acc;
    }
}

__global__ void fill_u32_kernel(uint32_t* p, int64_t n, uint32_t v) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

__global__ void fill_f64_kernel(double* p, int64_t n, double v) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

__global__ void init_loads_edge_kernel(const int64_t* rowptr, int32_t nact, int64_t* R, float* r32) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int64_t d = rowptr[x + 1] - rowptr[x];
        if (R) R[x] = d;
        if (r32) r32[x] = __fmul_rn((float)d, 0.5f);
    }
}

// ---- binary64 literal path

__global__ void __launch_bounds__(FW_THREADS) fw64_slot_kernel(const int32_t* __restrict__ fwcol,
                                                               const int32_t* __restrict__ chunk_row0, int64_t nslots,
                                                               int64_t nchunks, const double* __restrict__ r,
                                                               double* __restrict__ alpha, double gam, double one_minus,
                                                               uint32_t* __restrict__ plane) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t le = lanes_le(lane);
    for (int64_t g = warp; g < nchunks; g += nwarps) {
        int64_t s = (g << 5) + lane;
        bool valid = s < nslots;
        int32_t c = valid ? fwcol[s] : 0;
        uint32_t f = __ballot_sync(FULL, c < 0);
        int32_t v = c & 0x7fffffff;
        int32_t u = chunk_row0[g] + __popc(f & le) - (int)(f & 1u);
        bool recv = false;
        if (valid) {
            recv = receives<double>(r[u], r[v], u, v);
            double a = alpha[s];
            alpha[s] = __dadd_rn(__dmul_rn(one_minus, a), __dmul_rn(gam, recv ? 1.0 : 0.0));
        }
        uint32_t bal = __ballot_sync(FULL, recv);
        if (lane == 0 && plane) plane[g] = bal;
    }
}

__global__ void fw64_rowsum_kernel(const int64_t* __restrict__ rowptr, const double* __restrict__ alpha, int32_t nact,
                                   double* __restrict__ r) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        double acc = 0.0;
        for (int64_t s = rowptr[x], e = rowptr[x + 1]; s < e; ++s) acc = __dadd_rn(acc, alpha[s]);
        r[x] = acc;
    }
}

__global__ void fw64_weights_kernel(const double* __restrict__ alpha, int64_t nslots, double Dn, uint32_t* W) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += stride)
        W[s] = (uint32_t)llrint(alpha[s] * Dn);
}

// ---- outputs

// R_x = sum of x's slot weights (exact loads of the returned weights)
__global__ void loads_from_slots_kernel(const int64_t* rowptr, const uint32_t* W, int32_t nact, int64_t* R) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int64_t acc = 0;
        for (int64_t s = rowptr[x], e = rowptr[x + 1]; s < e; ++s) acc += W[s];
        R[x] = acc;
    }
}

// canonical edge e sits at slot slot_of_edge[e] in row u
__global__ void edge_weights_kernel(const int64_t* rowptr, const int32_t* col, const int32_t* eu, const int32_t* ev,
                                    int64_t m, const uint32_t* W, const uint32_t* planes_last, int64_t* Wout,
                                    uint8_t* last) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int32_t u = eu[e], v = ev[e];
        int64_t lo = rowptr[u], hi = rowptr[u + 1];
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (col[mid] < v) lo = mid + 1; else hi = mid;
        }
        if (Wout) Wout[e] = W[lo];
        if (last) last[e] = (uint8_t)((planes_last[lo >> 5] >> (lo & 31)) & 1u);
    }
}

template <class L>
__global__ void loads_to_double_kernel(const L* in, int32_t nact, int32_t n, double scale_div, double* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        out[x] = x < nact ? (double)in[x] / scale_div : 0.0;
}

__global__ void pad_i64_kernel(int64_t* p, int32_t from, int32_t to) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < to; x += stride) p[x] = 0;
}

// ---- triangles

template <class L>
__global__ void __launch_bounds__(FW_THREADS) fw_tri_pass_kernel(const int32_t* __restrict__ ta,
                                                                 const int32_t* __restrict__ tb,
                                                                 const int32_t* __restrict__ tc, int64_t ntri,
                                                                 const L* __restrict__ R, int32_t* __restrict__ cnt,
                                                                 uint32_t* __restrict__ plane0,
                                                                 uint32_t* __restrict__ plane1) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (ntri + 31) >> 5;
    for (int64_t g0 = warp * FW_UNROLL; g0 < nchunks; g0 += nwarps * FW_UNROLL) {
        int32_t a[FW_UNROLL], b[FW_UNROLL], c[FW_UNROLL];
#pragma unroll
        for (int k = 0; k < FW_UNROLL; ++k) {
            int64_t t = ((g0 + k) << 5) + lane;
            bool ok = t < ntri;
            a[k] = ok ? __ldg(ta + t) : 0;
            b[k] = ok ? __ldg(tb + t) : 0;
            c[k] = ok ? __ldg(tc + t) : 0;
        }
        L ra[FW_UNROLL], rb[FW_UNROLL], rc[FW_UNROLL];
#pragma unroll
        for (int k = 0; k < FW_UNROLL; ++k) {
            int64_t t = ((g0 + k) << 5) + lane;
            if (t < ntri) {
                ra[k] = __ldg(R + a[k]);
                rb[k] = __ldg(R + b[k]);
                rc[k] = __ldg(R + c[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < FW_UNROLL; ++k) {
            int64_t g = g0 + k;
            int64_t t = (g << 5) + lane;
            bool ok = t < ntri;
            int best = 2;
            int32_t w = c[k];
            if (ok) {
                L bv = rc[k];
                if (rb[k] < bv) { best = 1; bv = rb[k]; w = b[k]; }
                if (ra[k] < bv) { best = 0; w = a[k]; }
            }
            uint32_t b0 = __ballot_sync(FULL, ok && (best & 1));
            uint32_t b1 = __ballot_sync(FULL, ok && (best & 2));
            if (g < nchunks && lane == 0) {
                plane0[g] = b0;
                plane1[g] = b1;
            }
            uint32_t okmask = __ballot_sync(FULL, ok);
            if (ok) {
                uint32_t peers = __match_any_sync(okmask, w);
                if ((peers & ((1u << lane) - 1u)) == 0) atomicAdd(cnt + w, __popc(peers));
            }
        }
    }
}

// Wt[3t + k] += sum_planes [column == k] * (mult * (i_first + j + 1))
__global__ void fw_tri_fold_kernel(const uint32_t* __restrict__ planes, int nplanes, int64_t nchunks, int64_t ntri,
                                   int64_t i_first, int64_t mult, uint32_t* __restrict__ Wt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        int64_t g = t >> 5;
        int lane = (int)(t & 31);
        uint32_t acc[3] = {0, 0, 0};
        for (int j = 0; j < nplanes; ++j) {
            uint32_t p0 = (__ldg(planes + (2 * (int64_t)j) * nchunks + g) >> lane) & 1u;
            uint32_t p1 = (__ldg(planes + (2 * (int64_t)j + 1) * nchunks + g) >> lane) & 1u;
            uint32_t col = p0 | (p1 << 1);
            uint32_t inc = (uint32_t)(mult * (i_first + j + 1));
            acc[0] += col == 0 ? inc : 0u;
            acc[1] += col == 1 ? inc : 0u;
            acc[2] += col == 2 ? inc : 0u;
        }
        Wt[3 * t] += acc[0];
        Wt[3 * t + 1] += acc[1];
        Wt[3 * t + 2] += acc[2];
    }
}

__global__ void tri_counts_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t ntri, int32_t* tcount) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        atomicAdd(tcount + ta[t], 1);
        atomicAdd(tcount + tb[t], 1);
        atomicAdd(tcount + tc[t], 1);
    }
}

__global__ void init_loads_tri_kernel(const int32_t* tcount, int32_t nact, int64_t* R, float* r32) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nact; x += stride) {
        int32_t t = tcount[x];
        if (R) R[x] = 2 * (int64_t)t;
        if (r32) r32[x] = __fdiv_rn((float)t, 3.0f);
    }
}

__global__ void tri_loads_from_w_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t ntri,
                                        const uint32_t* Wt, unsigned long long* R) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        atomicAdd(R + ta[t], (unsigned long long)Wt[3 * t]);
        atomicAdd(R + tb[t], (unsigned long long)Wt[3 * t + 1]);
        atomicAdd(R + tc[t], (unsigned long long)Wt[3 * t + 2]);
    }
}

__global__ void tri_last_kernel(const uint32_t* plane0, const uint32_t* plane1, int64_t ntri, uint8_t* last) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        uint32_t p0 = (plane0[t >> 5] >> (t & 31)) & 1u, p1 = (plane1[t >> 5] >> (t & 31)) & 1u;
        last[t] = (uint8_t)(p0 | (p1 << 1));
    }
}

__global__ void widen_u32_kernel(const uint32_t* in, int64_t k, int64_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = in[i];
}

int fw_grid(int64_t chunks) {
    int64_t want = (chunks + FW_UNROLL - 1) / FW_UNROLL;         // warps
    int64_t blocks = (want * 32 + FW_THREADS - 1) / FW_THREADS;
    int64_t cap = (int64_t)num_sms() * 8;                        // 8 resident blocks of 256 per SM
    return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

}  // namespace

bool g_pass_profiling = false;

// ---------------------------------------------------------------- edge FW

struct EdgeFwState {
    DevBuf<int64_t> R;       // EXACT loads (internal ids)
    DevBuf<float> r32;       // FP32 loads
    DevBuf<double> r64;      // FP64 loads
    DevBuf<double> alpha;    // FP64 alpha per slot
    DevBuf<uint32_t> W;      // per-slot scaled weights
    DevBuf<uint32_t> planes; // last stored planes
    int64_t last_plane = -1; // index of the plane holding the last iteration
};

static void run_edge_fw(lds_graph* g, int N, lds_precision p, EdgeFwState& st, PassTimer& timer) {
    cudaStream_t s = g->stream;
    const int64_t nslots = 2 * g->m;
    const int64_t nchunks = (nslots + 31) / 32;
    const int32_t nact = g->nact;
    const int blk = 256;
    DevBuf<int32_t> cnt(std::max<int32_t>(nact, 1), s);
    LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, std::max<int32_t>(nact, 1) * sizeof(int32_t), s));
    const int K = planes_capacity(nchunks, N);
    st.planes.alloc(std::max<int64_t>(1, (int64_t)K * nchunks), s);
    st.W.alloc(std::max<int64_t>(nslots, 1), s);
    const int grid = fw_grid(nchunks);

    if (p == LDS_FP64) {
        st.alpha.alloc(std::max<int64_t>(nslots, 1), s);
        st.r64.alloc(std::max<int32_t>(nact, 1), s);
        if (nslots) LDS_LAUNCH(fill_f64_kernel, grid_for(nslots, blk), blk, 0, s, st.alpha.get(), nslots, 0.5);
        if (nact) LDS_LAUNCH(fw64_rowsum_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), st.alpha.get(), nact, st.r64.get());
        LDS_CHECK_LAUNCH();
        for (int i = 1; i <= N; ++i) {
            double gam = 2.0 / (double)(i + 2);
            double om = 1.0 - gam;
            if (nchunks) {
                timer.start(s);
                LDS_LAUNCH(fw64_slot_kernel, grid, FW_THREADS, 0, s, g->fwcol.get(), g->chunk_row0.get(), nslots, nchunks,
                                                             st.r64.get(), st.alpha.get(), gam, om, st.planes.get());
                timer.stop(s);
                LDS_LAUNCH(fw64_rowsum_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), st.alpha.get(), nact, st.r64.get());
                LDS_CHECK_LAUNCH();
            }
        }
        st.last_plane = 0;
        double Dn = (double)((int64_t)(N + 1) * (N + 2));
        if (nslots) LDS_LAUNCH(fw64_weights_kernel, grid_for(nslots, blk), blk, 0, s, st.alpha.get(), nslots, Dn, st.W.get());
        LDS_CHECK_LAUNCH();
        return;
    }

    if (nslots) LDS_LAUNCH(fill_u32_kernel, grid_for(nslots, blk), blk, 0, s, st.W.get(), nslots, 1u);
    if (p == LDS_EXACT) {
        st.R.alloc(std::max<int32_t>(nact, 1), s);
        if (nact) LDS_LAUNCH(init_loads_edge_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), nact, st.R.get(), nullptr);
    } else {
        st.r32.alloc(std::max<int32_t>(nact, 1), s);
        if (nact) LDS_LAUNCH(init_loads_edge_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), nact, nullptr, st.r32.get());
    }
    LDS_CHECK_LAUNCH();
    int stored = 0;
    int64_t first_i = 1;
    for (int i = 1; i <= N; ++i) {
        uint32_t* plane = st.planes.get() + (int64_t)stored * nchunks;
        if (nchunks) {
            timer.start(s);
            if (p == LDS_EXACT)
                LDS_LAUNCH(fw_edge_pass_kernel<int64_t>, grid, FW_THREADS, 0, s, g->fwcol.get(), g->chunk_row0.get(), nslots,
                                                                        nchunks, st.R.get(), cnt.get(), plane);
            else
                LDS_LAUNCH(fw_edge_pass_kernel<float>, grid, FW_THREADS, 0, s, g->fwcol.get(), g->chunk_row0.get(), nslots,
                                                                      nchunks, st.r32.get(), cnt.get(), plane);
            timer.stop(s);
            LDS_CHECK_LAUNCH();
            if (p == LDS_EXACT) {
                LDS_LAUNCH(fw_update_exact_kernel, grid_for(nact, blk), blk, 0, s, st.R.get(), cnt.get(), nact, 2 * (int64_t)(i + 1));
            } else {
                float gam = 2.0f / (float)(i + 2);
                float om = 1.0f - gam;
                LDS_LAUNCH(fw_update_fp32_kernel, grid_for(nact, blk), blk, 0, s, st.r32.get(), cnt.get(), nact, gam, om);
            }
            LDS_CHECK_LAUNCH();
        }
        ++stored;
        if (stored == K || i == N) {
            if (nslots) {
                LDS_LAUNCH(fw_fold_kernel, grid_for(nslots, blk), blk, 0, s, st.planes.get(), stored, nchunks, nslots, first_i, 2,
                                                                    st.W.get());
                LDS_CHECK_LAUNCH();
            }
            st.last_plane = stored - 1;
            if (i < N) {
                stored = 0;
                first_i = i + 1;
            }
        }
    }
}

// ---------------------------------------------------------------- triangle FW

// ---- Alg. 6 literally in binary64: one alpha per (vertex, triangle) pair,
// alpha <- (1 - gamma) alpha + gamma alpha_hat with every operation rounded on
// its own (no fused multiply-add), and r_v summed left to right over v's
// triangles in ascending triangle order, starting from 0.

__global__ void tri_alpha_init64_kernel(double* alpha, int64_t n3) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += stride) alpha[i] = 1.0 / 3.0;
}

__global__ void tri_rsum64_kernel(const int64_t* vt_ptr, const int32_t* vt_idx, const int32_t* ta, const int32_t* tb,
                                  const double* alpha, int32_t nact, double* r) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nact; v += stride) {
        double acc = 0.0;
        for (int64_t q = vt_ptr[v]; q < vt_ptr[v + 1]; ++q) {
            const int32_t t = vt_idx[q];
            const int k = ta[t] == v ? 0 : (tb[t] == v ? 1 : 2);
            acc = __dadd_rn(acc, alpha[3 * (int64_t)t + k]);
        }
        r[v] = acc;
    }
}

// receiving column: the lowest load, ties to the later column (the larger id)
__global__ void tri_pass64_kernel(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t ntri,
                                  const double* r, double gam, double om, double* alpha, uint8_t* last) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        const double ra = r[ta[t]], rb = r[tb[t]], rc = r[tc[t]];
        int best = 2;
        double bv = rc;
        if (rb < bv) { best = 1; bv = rb; }
        if (ra < bv) best = 0;
        for (int k = 0; k < 3; ++k)
            alpha[3 * t + k] = __dadd_rn(__dmul_rn(om, alpha[3 * t + k]), __dmul_rn(gam, k == best ? 1.0 : 0.0));
        if (last) last[t] = (uint8_t)best;
    }
}

// an exactly feasible integer solution: every weight rint(alpha D), except that the
// member with the largest alpha (the first on ties) takes D minus the other two
__global__ void tri_w_from_alpha64_kernel(const double* alpha, int64_t ntri, int64_t Dn3, uint32_t* W) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += stride) {
        int64_t w[3];
        int j = 0;
        for (int k = 0; k < 3; ++k) {
            w[k] = llrint(__dmul_rn(alpha[3 * t + k], (double)Dn3));
            if (alpha[3 * t + k] > alpha[3 * t + j]) j = k;
        }
        w[j] = Dn3 - (w[0] + w[1] + w[2] - w[j]);
        for (int k = 0; k < 3; ++k) W[3 * t + k] = (uint32_t)w[k];
    }
}

struct TriFwState {
    DevBuf<int64_t> R;
    DevBuf<float> r32;
    DevBuf<double> r64;        // binary64 form
    DevBuf<uint8_t> last64;    // binary64 form: receiving column of the last iteration
    DevBuf<uint32_t> W;        // [3 ntri]
    DevBuf<uint32_t> planes;   // 2 planes per stored iteration
    int64_t last_pair = -1;
};

static void run_tri_fw64(lds_graph* g, int N, TriFwState& st, PassTimer& timer) {
    cudaStream_t s = g->stream;
    const int64_t ntri = g->ntri;
    const int32_t nact = g->nact;
    const int blk = 256;
    ensure_vertex_triangles(g);
    DevBuf<double> alpha(std::max<int64_t>(3 * ntri, 1), s);
    st.r64.alloc(std::max<int32_t>(nact, 1), s);
    st.last64.alloc(std::max<int64_t>(ntri, 1), s);
    st.W.alloc(std::max<int64_t>(3 * ntri, 1), s);
    if (ntri) LDS_LAUNCH(tri_alpha_init64_kernel, grid_for(3 * ntri, blk), blk, 0, s, alpha.get(), 3 * ntri);
    if (ntri) LDS_CUDA(cudaMemsetAsync(st.last64.get(), 2, ntri, s));
    if (nact)
        LDS_LAUNCH(tri_rsum64_kernel, grid_for(nact, blk), blk, 0, s, g->vt_ptr.get(), g->vt_idx.get(), g->ta.get(),
                   g->tb.get(), alpha.get(), nact, st.r64.get());
    for (int i = 1; i <= N && ntri; ++i) {
        const double gam = 2.0 / (double)(i + 2);
        const double om = 1.0 - gam;
        timer.start(s);
        LDS_LAUNCH(tri_pass64_kernel, grid_for(ntri, blk), blk, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), ntri,
                   st.r64.get(), gam, om, alpha.get(), i == N ? st.last64.get() : (uint8_t*)nullptr);
        timer.stop(s);
        LDS_LAUNCH(tri_rsum64_kernel, grid_for(nact, blk), blk, 0, s, g->vt_ptr.get(), g->vt_idx.get(), g->ta.get(),
                   g->tb.get(), alpha.get(), nact, st.r64.get());
    }
    const int64_t Dn3 = 3 * (int64_t)(N + 1) * (N + 2);
    if (ntri) LDS_LAUNCH(tri_w_from_alpha64_kernel, grid_for(ntri, blk), blk, 0, s, alpha.get(), ntri, Dn3, st.W.get());
}

static void run_tri_fw(lds_graph* g, int N, lds_precision p, TriFwState& st, PassTimer& timer) {
    cudaStream_t s = g->stream;
    const int64_t ntri = g->ntri;
    const int64_t nchunks = (ntri + 31) / 32;
    const int32_t nact = g->nact;
    const int blk = 256;
    DevBuf<int32_t> cnt(std::max<int32_t>(nact, 1), s);
    LDS_CUDA(cudaMemsetAsync(cnt.get(), 0, std::max<int32_t>(nact, 1) * sizeof(int32_t), s));
    DevBuf<int32_t> tcount(std::max<int32_t>(nact, 1), s);
    LDS_CUDA(cudaMemsetAsync(tcount.get(), 0, std::max<int32_t>(nact, 1) * sizeof(int32_t), s));
    if (ntri) LDS_LAUNCH(tri_counts_kernel, grid_for(ntri, blk), blk, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), ntri, tcount.get());
    LDS_CHECK_LAUNCH();
    const int K = planes_capacity(2 * nchunks, N);
    st.planes.alloc(std::max<int64_t>(1, 2 * (int64_t)K * nchunks), s);
    st.W.alloc(std::max<int64_t>(3 * ntri, 1), s);
    if (ntri) LDS_LAUNCH(fill_u32_kernel, grid_for(3 * ntri, blk), blk, 0, s, st.W.get(), 3 * ntri, 2u);
    if (p == LDS_EXACT) {
        st.R.alloc(std::max<int32_t>(nact, 1), s);
        if (nact) LDS_LAUNCH(init_loads_tri_kernel, grid_for(nact, blk), blk, 0, s, tcount.get(), nact, st.R.get(), nullptr);
    } else {
        st.r32.alloc(std::max<int32_t>(nact, 1), s);
        if (nact) LDS_LAUNCH(init_loads_tri_kernel, grid_for(nact, blk), blk, 0, s, tcount.get(), nact, nullptr, st.r32.get());
    }
    LDS_CHECK_LAUNCH();
    const int grid = fw_grid(nchunks);
    int stored = 0;
    int64_t first_i = 1;
    for (int i = 1; i <= N; ++i) {
        uint32_t* p0 = st.planes.get() + (2 * (int64_t)stored) * nchunks;
        uint32_t* p1 = p0 + nchunks;
        if (nchunks) {
            timer.start(s);
            if (p == LDS_EXACT)
                LDS_LAUNCH(fw_tri_pass_kernel<int64_t>, grid, FW_THREADS, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), ntri,
                                                                       st.R.get(), cnt.get(), p0, p1);
            else
                LDS_LAUNCH(fw_tri_pass_kernel<float>, grid, FW_THREADS, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), ntri,
                                                                     st.r32.get(), cnt.get(), p0, p1);
            timer.stop(s);
            LDS_CHECK_LAUNCH();
            if (p == LDS_EXACT) {
                LDS_LAUNCH(fw_update_exact_kernel, grid_for(nact, blk), blk, 0, s, st.R.get(), cnt.get(), nact, 6 * (int64_t)(i + 1));
            } else {
                float gam = 2.0f / (float)(i + 2);
                float om = 1.0f - gam;
                LDS_LAUNCH(fw_update_fp32_kernel, grid_for(nact, blk), blk, 0, s, st.r32.get(), cnt.get(), nact, gam, om);
            }
            LDS_CHECK_LAUNCH();
        }
        ++stored;
        if (stored == K || i == N) {
            if (ntri) {
                LDS_LAUNCH(fw_tri_fold_kernel, grid_for(ntri, blk), blk, 0, s, st.planes.get(), stored, nchunks, ntri, first_i, 6,
                                                                      st.W.get());
                LDS_CHECK_LAUNCH();
            }
            st.last_pair = stored - 1;
            if (i < N) {
                stored = 0;
                first_i = i + 1;
            }
        }
    }
}

void fw_run(lds_graph* g, lds_density d, int32_t iters, lds_precision p, bool want_last) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n, nact = g->nact;
    const int blk = 256;
    PassTimer timer;
    timer.on = g_pass_profiling;
    cudaEvent_t e0, e1;
    LDS_CUDA(cudaEventCreate(&e0));
    LDS_CUDA(cudaEventCreate(&e1));
    struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{e0, e1};

    g->fw_valid = false;
    const int64_t Dn = (int64_t)(iters + 1) * (iters + 2) * (d == LDS_TRIANGLE ? 3 : 1);
    g->fw_R.alloc(std::max(n, 1), s);
    g->fw_r.alloc(std::max(n, 1), s);
    g->fw_last.release();
    DevBuf<int64_t>& R_int = g->fw_R;
    DevBuf<double>& r_int = g->fw_r;

    if (d == LDS_EDGE) {
        EdgeFwOut fo;
        LDS_CUDA(cudaEventRecord(e0, s));
        // graphs whose active vertices fit in shared memory run on one thread-block cluster
        bool clus = false;
        if ((g_fw_variant == 0 || g_fw_variant == 6) && (p == LDS_EXACT || p == LDS_FP32)) {
            if (want_last) g->fw_last.alloc(std::max<int64_t>(g->m, 1), s);
            timer.start(s);
            clus = fw_cluster_run(g, iters, p, want_last ? g->fw_last.get() : nullptr, g_fw_variant == 6);
            if (clus) timer.stop(s, iters);
            else g->fw_last.release();
        }
        bool fast = !clus && g_fw_variant != 1 && run_edge_fw_oriented(g, iters, p, true, want_last, fo, timer);
        if (clus) {
            LDS_CUDA(cudaEventRecord(e1, s));
            g->pass_kernel = "fw_cluster_kernel";
            g->pass_bytes = 12 * g->m + 8 * (int64_t)nact;
        } else if (fast) {
            LDS_CUDA(cudaEventRecord(e1, s));
            const std::string pk(g->pass_kernel);
            g->pass_bytes = 4 * g->m + 8 * ((g->m + 31) / 32) + 4 * g->fwv_nz +
                            (pk == "fw_opass32_kernel" || pk == "fw_coop32_kernel" ? 4 : 8) * (int64_t)nact;
            // the cooperative kernel also runs the vertex update: words and counts read and
            // written, row ranges read, the plane read again
            if (pk == "fw_coop32_kernel") g->pass_bytes += 20 * (int64_t)nact + 4 * ((g->m + 31) / 32);
            R_int = std::move(fo.R_int);
            r_int = std::move(fo.r_int);
            g->fw_W = std::move(fo.W_edge);
            if (want_last) g->fw_last = std::move(fo.last_edge);
        } else {
            EdgeFwState st;
            run_edge_fw(g, iters, p, st, timer);
            LDS_CUDA(cudaEventRecord(e1, s));
            const int64_t nslots = 2 * g->m, nc = (nslots + 31) / 32;
            if (p == LDS_FP64) {
                g->pass_kernel = "fw64_slot_kernel";
                g->pass_bytes = 4 * nslots + 8 * nc + 16 * nslots + 8 * (int64_t)nact;
            } else {
                g->pass_kernel = "fw_edge_pass_kernel";
                g->pass_bytes = 4 * nslots + 8 * nc + (p == LDS_EXACT ? 8 : 4) * (int64_t)nact;
            }
            if (nact) LDS_LAUNCH(loads_from_slots_kernel, grid_for(nact, blk), blk, 0, s, g->rowptr.get(), st.W.get(), nact, R_int.get());
            if (n > nact) LDS_LAUNCH(pad_i64_kernel, grid_for(n - nact, blk), blk, 0, s, R_int.get(), nact, n);
            if (n) {
                if (p == LDS_EXACT)
                    LDS_LAUNCH(loads_to_double_kernel<int64_t>, grid_for(n, blk), blk, 0, s, st.R.get(), nact, n, (double)Dn, r_int.get());
                else if (p == LDS_FP32)
                    LDS_LAUNCH(loads_to_double_kernel<float>, grid_for(n, blk), blk, 0, s, st.r32.get(), nact, n, 1.0, r_int.get());
                else
                    LDS_LAUNCH(loads_to_double_kernel<double>, grid_for(n, blk), blk, 0, s, st.r64.get(), nact, n, 1.0, r_int.get());
            }
            g->fw_W.alloc(std::max<int64_t>(g->m, 1), s);
            if (want_last) g->fw_last.alloc(std::max<int64_t>(g->m, 1), s);
            if (g->m) {
                const uint32_t* lastp = st.planes.get() + std::max<int64_t>(st.last_plane, 0) * nc;
                LDS_LAUNCH(edge_weights_kernel, grid_for(g->m, blk), blk, 0, s, g->rowptr.get(), g->col.get(), g->eu.get(),
                           g->ev.get(), g->m, st.W.get(), lastp, g->fw_W.get(), want_last ? g->fw_last.get() : nullptr);
                if (want_last && iters == 0) LDS_CUDA(cudaMemsetAsync(g->fw_last.get(), 0, g->m, s));
            }
        }
    } else {
        ensure_triangles(g);
        TriFwState st;
        LDS_CUDA(cudaEventRecord(e0, s));
        if (p == LDS_FP64) run_tri_fw64(g, iters, st, timer);
        else run_tri_fw(g, iters, p, st, timer);
        LDS_CUDA(cudaEventRecord(e1, s));
        if (p == LDS_FP64) {
            g->pass_kernel = "tri_pass64_kernel";
            g->pass_bytes = 12 * g->ntri + 48 * g->ntri + 24 * (int64_t)nact;
        } else {
            g->pass_kernel = "fw_tri_pass_kernel";
            g->pass_bytes = 12 * g->ntri + 8 * ((g->ntri + 31) / 32) + (p == LDS_EXACT ? 8 : 4) * (int64_t)nact;
        }
        const int64_t ntri = g->ntri;
        LDS_CUDA(cudaMemsetAsync(R_int.get(), 0, std::max(n, 1) * sizeof(int64_t), s));
        if (ntri)
            LDS_LAUNCH(tri_loads_from_w_kernel, grid_for(ntri, blk), blk, 0, s, g->ta.get(), g->tb.get(), g->tc.get(), ntri,
                       st.W.get(), (unsigned long long*)R_int.get());
        if (n) {
            if (p == LDS_EXACT)
                LDS_LAUNCH(loads_to_double_kernel<int64_t>, grid_for(n, blk), blk, 0, s, st.R.get(), nact, n, (double)Dn, r_int.get());
            else if (p == LDS_FP64)
                LDS_LAUNCH(loads_to_double_kernel<double>, grid_for(n, blk), blk, 0, s, st.r64.get(), nact, n, 1.0, r_int.get());
            else
                LDS_LAUNCH(loads_to_double_kernel<float>, grid_for(n, blk), blk, 0, s, st.r32.get(), nact, n, 1.0, r_int.get());
        }
        g->fw_W.alloc(std::max<int64_t>(3 * ntri, 1), s);
        if (ntri) LDS_LAUNCH(widen_u32_kernel, grid_for(3 * ntri, blk), blk, 0, s, st.W.get(), 3 * ntri, g->fw_W.get());
        if (want_last) {
            g->fw_last.alloc(std::max<int64_t>(ntri, 1), s);
            int64_t nch = (ntri + 31) / 32;
            const uint32_t* p0 = st.planes.get() + 2 * std::max<int64_t>(st.last_pair, 0) * nch;
            if (ntri) {
                if (p == LDS_FP64)
                    LDS_CUDA(cudaMemcpyAsync(g->fw_last.get(), st.last64.get(), ntri, cudaMemcpyDeviceToDevice, s));
                else if (iters == 0) LDS_CUDA(cudaMemsetAsync(g->fw_last.get(), 2, ntri, s));
                else LDS_LAUNCH(tri_last_kernel, grid_for(ntri, blk), blk, 0, s, p0, p0 + nch, ntri, g->fw_last.get());
            }
        }
    }
    LDS_CUDA(cudaStreamSynchronize(s));
    float ms = 0;
    LDS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    g->fw_ms = ms;
    // per iteration: a cooperative launch covers many iterations
    g->pass_launches = timer.iters;
    g->pass_us = timer.iters ? 1000.0 * timer.total_ms() / (double)timer.iters : 0.0;
    g->fw_valid = true;
    g->fw_density = d;
    g->fw_prec = p;
    g->fw_reuse = false;
    g->fw_iters = iters;
    g->fw_D = Dn;
}

}  // namespace lds

using namespace lds;

extern "C" {

lds_status lds_fw(lds_graph* g, lds_density d, int32_t iters, lds_precision p, lds_mem where, lds_fw_result* out) {
    return guard([&] {
        LDS_REQUIRE(g && out, LDS_EINVAL, "lds_fw: NULL argument");
        LDS_REQUIRE(d == LDS_EDGE || d == LDS_TRIANGLE, LDS_EINVAL, "lds_fw: bad density");
        LDS_REQUIRE(p == LDS_EXACT || p == LDS_FP32 || p == LDS_FP64, LDS_EINVAL, "lds_fw: bad precision");
        LDS_REQUIRE(iters >= 0 && iters <= (d == LDS_EDGE ? 60000 : 30000), LDS_EINVAL,
                    "lds_fw: iters = %d out of range", iters);
        LDS_REQUIRE(where == LDS_MEM_HOST || where == LDS_MEM_DEVICE, LDS_EINVAL, "lds_fw: bad lds_mem");
        fw_run(g, d, iters, p, out->last != nullptr);
        copy_fw_state(g, d, where, out);
    });
}

lds_status lds_fw_state(lds_graph* g, lds_mem where, lds_fw_result* out) {
    return guard([&] {
        LDS_REQUIRE(g && out, LDS_EINVAL, "lds_fw_state: NULL argument");
        LDS_REQUIRE(g->fw_valid, LDS_EINVAL, "lds_fw_state: no Frank-Wolfe state on this graph");
        LDS_REQUIRE(where == LDS_MEM_HOST || where == LDS_MEM_DEVICE, LDS_EINVAL, "lds_fw_state: bad lds_mem");
        LDS_REQUIRE(out->last == nullptr || g->fw_last.get() != nullptr, LDS_EINVAL,
                    "lds_fw_state: the last choices were not kept for this state");
        copy_fw_state(g, g->fw_density, where, out);
    });
}

}  // extern "C"

namespace lds {

// r, R, W (and the last choices) of the handle's state into the caller's buffers
void copy_fw_state(lds_graph* g, lds_density d, lds_mem where, lds_fw_result* out) {
    {
        cudaStream_t s = g->stream;
        const int32_t n = g->n;
        out->D = g->fw_D;
        if (out->r && n) {
            DevBuf<double> r_orig(n, s);
            to_original_order_f64(g, g->fw_r.get(), r_orig.get());
            copy_out(out->r, where, r_orig.get(), n * sizeof(double), s);
            LDS_CUDA(cudaStreamSynchronize(s));
        }
        if (out->R && n) {
            DevBuf<int64_t> R_orig(n, s);
            to_original_order_i64(g, g->fw_R.get(), R_orig.get());
            copy_out(out->R, where, R_orig.get(), n * sizeof(int64_t), s);
            LDS_CUDA(cudaStreamSynchronize(s));
        }
        const int64_t npat = d == LDS_EDGE ? g->m : g->ntri;
        if (out->W && npat) copy_out(out->W, where, g->fw_W.get(), (d == LDS_EDGE ? 1 : 3) * npat * sizeof(int64_t), s);
        if (out->last && npat) copy_out(out->last, where, g->fw_last.get(), npat, s);
        LDS_CUDA(cudaStreamSynchronize(s));
    }
}

}  // namespace lds

extern "C" {

lds_status lds_fw_last_timing(const lds_graph* g, double* fw_ms, double* pass_us, int64_t* pass_launches,
                              int64_t* pass_bytes, const char** pass_kernel) {
    return guard([&] {
        LDS_REQUIRE(g, LDS_EINVAL, "lds_fw_last_timing: NULL graph");
        if (fw_ms) *fw_ms = g->fw_ms;
        if (pass_us) *pass_us = g->pass_us;
        if (pass_launches) *pass_launches = g->pass_launches;
        if (pass_bytes) *pass_bytes = g->pass_bytes;
        if (pass_kernel) *pass_kernel = g->pass_kernel;
    });
}

void lds_set_pass_profiling(int32_t on) { g_pass_profiling = on != 0; }

lds_status lds_set_fw_variant(int32_t variant) {
    return guard([&] {
        LDS_REQUIRE(variant >= 0 && variant <= 6, LDS_EINVAL, "lds_set_fw_variant: variant must be 0 to 6");
        g_fw_variant = variant;
    });
}

}  // extern "C"
