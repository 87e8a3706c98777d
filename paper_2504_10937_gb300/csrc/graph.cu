// Graph ingest: raw (src, dst) pairs -> canonical edge list and symmetric CSR
// on the device (the simple undirected G = (V, E) of Sec. 3).
//
// One stable radix sort of the 2m directed keys x*n + y (self-loops mapped to a
// key above every real one) gives, after removing repeats, the symmetric CSR in
// row-major order; the slots with row < col, in order, are the canonical edges.
#include "graph.cuh"
#include "prims.cuh"

namespace lds {

namespace {

__global__ void validate_kernel(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, int* bad) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n) atomicOr(bad, 1);
    }
}

__global__ void directed_keys_kernel(const int32_t* src, const int32_t* dst, int64_t m, int64_t n,
                                     uint64_t loop_key, uint64_t* keys, unsigned long long* loops) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        int64_t a = src[i], b = dst[i];
        if (a == b) {
            keys[2 * i] = loop_key;
            keys[2 * i + 1] = loop_key;
            ++local;
        } else {
            keys[2 * i] = (uint64_t)(a * n + b);
            keys[2 * i + 1] = (uint64_t)(b * n + a);
        }
    }
    if (local) atomicAdd(loops, local);
}

__global__ void unique_flags_kernel(const uint64_t* keys, int64_t k, uint64_t loop_key, int32_t* flag) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        uint64_t x = keys[i];
        flag[i] = (x != loop_key && (i == 0 || keys[i - 1] != x)) ? 1 : 0;
    }
}

__global__ void compact_degree_kernel(const uint64_t* keys, const int32_t* flag, const int64_t* pos, int64_t k,
                                      int64_t n, uint64_t* out, int32_t* deg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        if (flag[i]) {
            uint64_t x = keys[i];
            out[pos[i]] = x;
            atomicAdd(&deg[(int64_t)(x / (uint64_t)n)], 1);
        }
    }
}

__global__ void nonisolated_flag_kernel(const int32_t* deg, int32_t n, int32_t* flag) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) flag[i] = deg[i] > 0;
}

__global__ void id_maps_kernel(const int32_t* deg, const int64_t* nz_rank, int32_t n, int32_t nact,
                               int32_t* to_int, int32_t* to_orig, int32_t* deg_int, int* maxdeg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int32_t dmax = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int32_t d = deg[i];
        int32_t id = d > 0 ? (int32_t)nz_rank[i] : (int32_t)(nact + (i - nz_rank[i]));
        to_int[i] = id;
        to_orig[id] = (int32_t)i;
        if (d > 0) {
            deg_int[id] = d;
            dmax = max(dmax, d);
        }
    }
    if (dmax) atomicMax(maxdeg, dmax);
}

__global__ void fill_csr_kernel(const uint64_t* ukeys, int64_t k2, int64_t n, const int32_t* to_int,
                                int32_t* col, int32_t* upper_flag) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k2; s += stride) {
        uint64_t x = ukeys[s];
        int32_t r = to_int[(int64_t)(x / (uint64_t)n)];
        int32_t c = to_int[(int64_t)(x % (uint64_t)n)];
        col[s] = c;
        upper_flag[s] = r < c;
    }
}

__global__ void canonical_edges_kernel(const uint64_t* ukeys, const int32_t* upper_flag, const int64_t* epos,
                                       int64_t k2, int64_t n, const int32_t* to_int, int32_t* eu, int32_t* ev) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k2; s += stride) {
        if (upper_flag[s]) {
            uint64_t x = ukeys[s];
            int64_t e = epos[s];
            eu[e] = to_int[(int64_t)(x / (uint64_t)n)];
            ev[e] = to_int[(int64_t)(x % (uint64_t)n)];
        }
    }
}

__global__ void row_marks_kernel(const int64_t* rowptr, int32_t nact, const int32_t* col, int32_t* fwcol,
                                 int32_t* chunk_row0) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nact; r += stride) {
        int64_t b = rowptr[r], e = rowptr[r + 1];
        fwcol[b] = col[b] | (int32_t)0x80000000;
        // chunks whose first slot lies in [b, e)
        for (int64_t g = (b + 31) >> 5; (g << 5) < e; ++g) chunk_row0[g] = (int32_t)r;
    }
}

__global__ void copy_unflagged_kernel(const int32_t* col, int32_t* fwcol, int64_t k2) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k2; s += stride) fwcol[s] = col[s];
}

// upper slot of edge e = (u, v), u < v: row u lists its lower neighbours first, then
// its upper ones in edge order, so the slot is rowptr[u] + low(u) + (e - eptr[u])
__global__ void slot_edge_upper_kernel(const int32_t* eu, int64_t m, const int64_t* rowptr, const int64_t* updeg,
                                       const int64_t* eptr, int64_t* slot_edge) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t u = eu[e];
        const int64_t low = rowptr[u + 1] - rowptr[u] - updeg[u];
        slot_edge[rowptr[u] + low + (e - eptr[u])] = e;
    }
}

__global__ void second_endpoint_keys_kernel(const int32_t* ev, int64_t m, uint64_t* key, uint32_t* eid) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        key[e] = (uint64_t)ev[e];
        eid[e] = (uint32_t)e;
    }
}

// lower slots: the edges sorted (stably) by their upper endpoint v, so by u within v;
// the i-th of v's group sits at slot rowptr[v] + (i - gstart[v])
__global__ void slot_edge_lower_kernel(const uint64_t* key, const uint32_t* eid, int64_t m, const int64_t* rowptr,
                                       const int64_t* gstart, int64_t* slot_edge) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int64_t v = (int64_t)key[i];
        slot_edge[rowptr[v] + (i - gstart[v])] = (int64_t)eid[i];
    }
}

__global__ void lower_degree_kernel(const int64_t* rowptr, const int64_t* updeg, int32_t nact, int64_t* low) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nact; r += stride)
        low[r] = rowptr[r + 1] - rowptr[r] - updeg[r];
}

__global__ void upper_degree_kernel(const int64_t* rowptr, const int32_t* col, int32_t nact, int64_t* updeg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nact; r += stride) {
        int64_t lo = rowptr[r], hi = rowptr[r + 1], e = hi;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (col[mid] <= r) lo = mid + 1; else hi = mid;
        }
        updeg[r] = e - lo;
    }
}

__global__ void map_ids_kernel(const int32_t* in, const int32_t* map, int64_t k, int32_t* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) out[i] = map[in[i]];
}

template <class T>
__global__ void scatter_orig_kernel(const T* in, const int32_t* to_orig, int32_t n, T* out) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[to_orig[i]] = in[i];
}

}  // namespace

void map_ids(const int32_t* in, const int32_t* map, int64_t k, int32_t* out, cudaStream_t s) {
    if (k <= 0) return;
    LDS_LAUNCH(map_ids_kernel, grid_for(k, 256), 256, 0, s, in, map, k, out);
    LDS_CHECK_LAUNCH();
}

void ensure_slot_edge(lds_graph* g) {
    if (g->slot_edge.p || g->m == 0) return;
    cudaStream_t s = g->stream;
    DevBuf<int64_t> updeg(g->nact, s), eptr(g->nact, s);
    LDS_LAUNCH(upper_degree_kernel, grid_for(g->nact, 256), 256, 0, s, g->rowptr.get(), g->col.get(), g->nact, updeg.get());
    LDS_CHECK_LAUNCH();
    exclusive_scan_i64_dev(updeg.get(), eptr.get(), g->nact, nullptr, s);
    g->slot_edge.alloc(2 * g->m, s);
    const int64_t m = g->m;
    LDS_LAUNCH(slot_edge_upper_kernel, grid_for(m, 256), 256, 0, s, g->eu.get(), m, g->rowptr.get(), updeg.get(),
               eptr.get(), g->slot_edge.get());
    DevBuf<int64_t> low(g->nact, s), gstart(g->nact, s);
    LDS_LAUNCH(lower_degree_kernel, grid_for(g->nact, 256), 256, 0, s, g->rowptr.get(), updeg.get(), g->nact, low.get());
    exclusive_scan_i64_dev(low.get(), gstart.get(), g->nact, nullptr, s);
    DevBuf<uint64_t> key(m, s);
    DevBuf<uint32_t> eid(m, s);
    LDS_LAUNCH(second_endpoint_keys_kernel, grid_for(m, 256), 256, 0, s, g->ev.get(), m, key.get(), eid.get());
    radix_sort_u64(key.get(), eid.get(), m, std::max(1, bit_length_u64((uint64_t)g->nact)), s);
    LDS_LAUNCH(slot_edge_lower_kernel, grid_for(m, 256), 256, 0, s, key.get(), eid.get(), m, g->rowptr.get(),
               gstart.get(), g->slot_edge.get());
}

void to_original_order_i64(const lds_graph* g, const int64_t* in_int, int64_t* out_orig) {
    if (g->n <= 0) return;
    LDS_LAUNCH(scatter_orig_kernel<int64_t>, grid_for(g->n, 256), 256, 0, g->stream, in_int, g->to_orig.get(), g->n, out_orig);
    LDS_CHECK_LAUNCH();
}

void to_original_order_f64(const lds_graph* g, const double* in_int, double* out_orig) {
    if (g->n <= 0) return;
    LDS_LAUNCH(scatter_orig_kernel<double>, grid_for(g->n, 256), 256, 0, g->stream, in_int, g->to_orig.get(), g->n, out_orig);
    LDS_CHECK_LAUNCH();
}

static void build_graph(lds_graph* g, int32_t n, int64_t m_in, const int32_t* src, const int32_t* dst, lds_mem where) {
    cudaStream_t s = g->stream;
    g->n = n;
    g->info.n = n;
    g->info.input_pairs = m_in;
    g->info.triangles = -1;
    const int32_t* dsrc = src;
    const int32_t* ddst = dst;
    DevBuf<int32_t> hsrc, hdst;
    if (where == LDS_MEM_HOST && m_in > 0) {
        hsrc.alloc(m_in, s);
        hdst.alloc(m_in, s);
        copy_in(hsrc.get(), src, LDS_MEM_HOST, m_in * sizeof(int32_t), s);
        copy_in(hdst.get(), dst, LDS_MEM_HOST, m_in * sizeof(int32_t), s);
        dsrc = hsrc.get();
        ddst = hdst.get();
    }
    DevBuf<int> bad(1, s);
    LDS_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    if (m_in > 0) {
        LDS_LAUNCH(validate_kernel, grid_for(m_in, 256), 256, 0, s, dsrc, ddst, m_in, n, bad.get());
        LDS_CHECK_LAUNCH();
    }
    int hbad = 0;
    LDS_CUDA(cudaMemcpyAsync(&hbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    LDS_REQUIRE(!hbad, LDS_EINVAL, "lds_create_graph: vertex id outside [0, %d)", n);

    const uint64_t nn = (uint64_t)n * (uint64_t)n;
    const int bits = bit_length_u64(nn);           // 2^bits > n*n - 1, every real key fits
    const uint64_t loop_key = bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
    const int64_t K = 2 * m_in;

    DevBuf<uint64_t> keys(K, s);
    DevBuf<unsigned long long> loops(1, s);
    LDS_CUDA(cudaMemsetAsync(loops.get(), 0, sizeof(unsigned long long), s));
    if (m_in > 0) {
        LDS_LAUNCH(directed_keys_kernel, grid_for(m_in, 256), 256, 0, s, dsrc, ddst, m_in, n, loop_key, keys.get(), loops.get());
        LDS_CHECK_LAUNCH();
    }
    hsrc.release();
    hdst.release();
    radix_sort_u64(keys.get(), nullptr, K, bits, s);

    DevBuf<int32_t> flag(K, s);
    DevBuf<int64_t> pos(K, s);
    if (K > 0) {
        LDS_LAUNCH(unique_flags_kernel, grid_for(K, 256), 256, 0, s, keys.get(), K, loop_key, flag.get());
        LDS_CHECK_LAUNCH();
    }
    int64_t K2 = exclusive_scan_i32_to_i64(flag.get(), pos.get(), K, s);
    LDS_REQUIRE(K2 % 2 == 0, LDS_ECUDA, "lds_create_graph: asymmetric key set (internal error)");
    g->m = K2 / 2;
    DevBuf<uint64_t> ukeys(K2, s);
    DevBuf<int32_t> deg(n, s);
    LDS_CUDA(cudaMemsetAsync(deg.get(), 0, n * sizeof(int32_t), s));
    if (K > 0) {
        LDS_LAUNCH(compact_degree_kernel, grid_for(K, 256), 256, 0, s, keys.get(), flag.get(), pos.get(), K, n, ukeys.get(),
                                                               deg.get());
        LDS_CHECK_LAUNCH();
    }
    keys.release();
    flag.release();
    pos.release();

    unsigned long long hloops = 0;
    LDS_CUDA(cudaMemcpyAsync(&hloops, loops.get(), sizeof(hloops), cudaMemcpyDeviceToHost, s));

    // id maps
    DevBuf<int32_t> nzflag(n, s);
    DevBuf<int64_t> nzrank(n, s);
    if (n > 0) {
        LDS_LAUNCH(nonisolated_flag_kernel, grid_for(n, 256), 256, 0, s, deg.get(), n, nzflag.get());
        LDS_CHECK_LAUNCH();
    }
    int64_t nact = exclusive_scan_i32_to_i64(nzflag.get(), nzrank.get(), n, s);
    g->nact = (int32_t)nact;
    g->to_int.alloc(n, s);
    g->to_orig.alloc(n, s);
    DevBuf<int32_t> deg_int(nact + 1, s);
    DevBuf<int> maxdeg(1, s);
    LDS_CUDA(cudaMemsetAsync(maxdeg.get(), 0, sizeof(int), s));
    if (n > 0) {
        LDS_LAUNCH(id_maps_kernel, grid_for(n, 256), 256, 0, s, deg.get(), nzrank.get(), n, g->nact, g->to_int.get(),
                                                        g->to_orig.get(), deg_int.get(), maxdeg.get());
        LDS_CHECK_LAUNCH();
    }
    g->rowptr.alloc(nact + 1, s);
    {
        DevBuf<int64_t> deg64(nact + 1, s);
        LDS_CUDA(cudaMemsetAsync(deg64.get(), 0, (nact + 1) * sizeof(int64_t), s));
        // widen deg_int to int64 via the scan input (int32 -> int64 scan)
        LDS_CUDA(cudaMemsetAsync(deg_int.get() + nact, 0, sizeof(int32_t), s));
        exclusive_scan_i32_to_i64(deg_int.get(), g->rowptr.get(), nact + 1, s);
    }
    g->col.alloc(K2, s);
    DevBuf<int32_t> upper(K2, s);
    DevBuf<int64_t> epos(K2, s);
    if (K2 > 0) {
        LDS_LAUNCH(fill_csr_kernel, grid_for(K2, 256), 256, 0, s, ukeys.get(), K2, n, g->to_int.get(), g->col.get(),
                                                          upper.get());
        LDS_CHECK_LAUNCH();
    }
    int64_t mm = exclusive_scan_i32_to_i64(upper.get(), epos.get(), K2, s);
    LDS_REQUIRE(mm == g->m, LDS_ECUDA, "lds_create_graph: edge count mismatch (internal error)");
    g->eu.alloc(g->m, s);
    g->ev.alloc(g->m, s);
    if (K2 > 0) {
        LDS_LAUNCH(canonical_edges_kernel, grid_for(K2, 256), 256, 0, s, ukeys.get(), upper.get(), epos.get(), K2, n,
                                                                 g->to_int.get(), g->eu.get(), g->ev.get());
        LDS_CHECK_LAUNCH();
    }
    ukeys.release();
    upper.release();
    epos.release();

    // FW layout: flagged column copy and the first row of each 32-slot chunk
    g->fwcol.alloc(K2, s);
    int64_t nchunks = (K2 + 31) / 32;
    g->chunk_row0.alloc(nchunks, s);
    if (K2 > 0) {
        LDS_LAUNCH(copy_unflagged_kernel, grid_for(K2, 256), 256, 0, s, g->col.get(), g->fwcol.get(), K2);
        LDS_CHECK_LAUNCH();
        LDS_LAUNCH(row_marks_kernel, grid_for(nact, 256), 256, 0, s, g->rowptr.get(), g->nact, g->col.get(), g->fwcol.get(),
                                                             g->chunk_row0.get());
        LDS_CHECK_LAUNCH();
    }
    int hmax = 0;
    LDS_CUDA(cudaMemcpyAsync(&hmax, maxdeg.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    LDS_CUDA(cudaStreamSynchronize(s));
    g->info.m = g->m;
    g->info.self_loops = (int64_t)hloops;
    g->info.duplicates = m_in - (int64_t)hloops - g->m;
    g->info.max_degree = hmax;
    g->info.isolated = n - g->nact;
}

void set_stream(lds_graph* g, cudaStream_t s) {
    g->stream = s;
    g->to_orig.s = s;
    g->to_int.s = s;
    g->eu.s = s;
    g->ev.s = s;
    g->rowptr.s = s;
    g->col.s = s;
    g->fwcol.s = s;
    g->chunk_row0.s = s;
    g->slot_edge.s = s;
    g->ta.s = s;
    g->tb.s = s;
    g->tc.s = s;
    g->vt_ptr.s = s;
    g->vt_idx.s = s;
    g->core_all[0].s = s;
    g->core_all[1].s = s;
    g->fwv_perm.s = s;
    g->fwv_pos.s = s;
    g->fwv_col.s = s;
    g->fwv_nzrow.s = s;
    g->fwv_chunk_nz0.s = s;
    g->fwv_edge.s = s;
    g->fwv_rowptr.s = s;
    g->fwv_ta.s = s;
    g->fwv_tb.s = s;
    g->fwv_tc.s = s;
    g->fw_R.s = s;
    g->fw_r.s = s;
    g->fw_W.s = s;
    g->fw_last.s = s;
}

}  // namespace lds

using namespace lds;

extern "C" {

lds_status lds_create_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, lds_mem where,
                            void* stream, lds_graph** out) {
    return guard([&] {
        LDS_REQUIRE(out != nullptr, LDS_EINVAL, "lds_create_graph: out is NULL");
        *out = nullptr;
        LDS_REQUIRE(n >= 0 && n <= 0x7ffffffe, LDS_EINVAL, "lds_create_graph: n = %d out of range", n);
        LDS_REQUIRE(m >= 0, LDS_EINVAL, "lds_create_graph: m = %lld < 0", (long long)m);
        LDS_REQUIRE(m == 0 || (src && dst), LDS_EINVAL, "lds_create_graph: src / dst is NULL");
        LDS_REQUIRE(where == LDS_MEM_HOST || where == LDS_MEM_DEVICE, LDS_EINVAL, "lds_create_graph: bad lds_mem");
        LDS_REQUIRE(lds_device_count() > 0, LDS_ECUDA, "lds_create_graph: no CUDA device");
        lds_graph* g = new lds_graph();
        g->stream = (cudaStream_t)stream;
        try {
            build_graph(g, n, m, src, dst, where);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

void lds_free(lds_graph* g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    delete g;
    cudaStreamSynchronize(nullptr);
}

lds_status lds_graph_info(const lds_graph* g, lds_graph_info_t* info) {
    return guard([&] {
        LDS_REQUIRE(g && info, LDS_EINVAL, "lds_graph_info: NULL argument");
        *info = g->info;
        info->triangles = g->ntri;
    });
}

lds_status lds_get_edges(const lds_graph* g, int32_t* u, int32_t* v, lds_mem where) {
    return guard([&] {
        LDS_REQUIRE(g && u && v, LDS_EINVAL, "lds_get_edges: NULL argument");
        cudaStream_t s = g->stream;
        if (g->m == 0) return;
        DevBuf<int32_t> ou(g->m, s), ov(g->m, s);
        // internal -> original ids (monotone, so the order is kept)
        map_ids(g->eu.get(), g->to_orig.get(), g->m, ou.get(), s);
        map_ids(g->ev.get(), g->to_orig.get(), g->m, ov.get(), s);
        copy_out(u, where, ou.get(), g->m * sizeof(int32_t), s);
        copy_out(v, where, ov.get(), g->m * sizeof(int32_t), s);
        LDS_CUDA(cudaStreamSynchronize(s));
    });
}

}  // extern "C"

