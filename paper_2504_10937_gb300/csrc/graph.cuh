// The graph handle and its device layout.
//
// Internal ids: the non-isolated vertices keep their relative order and are
// numbered 0..nact-1; isolated vertices follow.  The map is monotone on
// non-isolated vertices, so comparisons by id (the FW tie rule, the (u, v)
// order of edges, the (a, b, c) order of triangles) are the same in internal
// and original ids, and every row 0..nact-1 of the CSR is non-empty.
#pragma once

#include "common.cuh"

struct lds_graph {
    int32_t n = 0;        // vertices (original id space)
    int32_t nact = 0;     // non-isolated vertices (internal ids 0..nact-1)
    int64_t m = 0;        // distinct undirected edges
    cudaStream_t stream = nullptr;
    lds_graph_info_t info{};

    lds::DevBuf<int32_t> to_orig;     // [n] internal -> original
    lds::DevBuf<int32_t> to_int;      // [n] original -> internal
    lds::DevBuf<int32_t> eu, ev;      // [m] canonical edges, internal ids, u < v
    lds::DevBuf<int64_t> rowptr;      // [nact + 1]
    lds::DevBuf<int32_t> col;         // [2m] internal ids, ascending in each row
    lds::DevBuf<int32_t> fwcol;       // [2m] col with bit 31 set on the first slot of each row
    lds::DevBuf<int32_t> chunk_row0;  // [ceil(2m / 32)] row of slot 32 g
    lds::DevBuf<int64_t> slot_edge;   // [2m] canonical edge id of each slot (lazy)

    // triangles (lazy): internal ids a < b < c, triangle order
    int64_t ntri = -1;
    lds::DevBuf<int32_t> ta, tb, tc;
    // vertex -> triangle incidence (lazy): triangles of x at vt_idx[vt_ptr[x] .. vt_ptr[x+1]), ascending
    lds::DevBuf<int64_t> vt_ptr;      // [nact + 1]
    lds::DevBuf<int32_t> vt_idx;      // [3 |T|]
    // core numbers of the whole graph (lazy), [0] edge, [1] triangle: a peel with
    // every vertex alive is the same every time the handle asks
    lds::DevBuf<int64_t> core_all[2];

    // FW view: vertices relabelled by (degree descending, id ascending); every
    // edge stored once, in the row of its lower-ranked endpoint, pointing to the
    // higher-ranked one (so most targets are high-degree vertices).
    bool fwv_built = false;
    int32_t fwv_bits = 0;              // B = bit length of nact (tie bits of a key)
    int64_t fwv_nz = 0;                // non-empty rows
    lds::DevBuf<int32_t> fwv_perm;     // [nact] fw id -> internal id
    lds::DevBuf<int32_t> fwv_pos;      // [nact] internal id -> fw id
    lds::DevBuf<int32_t> fwv_col;      // [m] target fw id; bit 31 on the first slot of each row
    lds::DevBuf<int32_t> fwv_nzrow;    // [fwv_nz] fw id of each non-empty row, ascending
    lds::DevBuf<int32_t> fwv_chunk_nz0;// [ceil(m / 32)] non-empty-row index of slot 32 g
    lds::DevBuf<int64_t> fwv_edge;     // [m] canonical edge id of each slot
    lds::DevBuf<int32_t> fwv_rowptr;   // [nact + 1] slots of the row of fw id p: rowptr[p] .. rowptr[p+1]
    lds::DevBuf<int32_t> fwv_ta, fwv_tb, fwv_tc;  // triangles in fw ids (lazy)

    // state of the most recent Frank-Wolfe run (internal ids), read by the later stages
    bool fw_valid = false;
    lds_density fw_density = LDS_EDGE;
    lds_precision fw_prec = LDS_EXACT;
    bool fw_reuse = false;            // set by lds_fw_batch: the next query's first round takes this state
    int32_t fw_iters = 0;
    int64_t fw_D = 0;
    lds::DevBuf<int64_t> fw_R;        // [n] exact loads of the weights below (R = D r)
    lds::DevBuf<double> fw_r;         // [n] reported loads
    lds::DevBuf<int64_t> fw_W;        // [m] D alpha_{u,v} per canonical edge, or [3 |T|] per triangle row
    lds::DevBuf<uint8_t> fw_last;     // [m] or [|T|] last-iteration choices

    // timing of the most recent lds_fw
    double fw_ms = 0.0, pass_us = 0.0;
    int64_t pass_launches = 0;
    int64_t pass_bytes = 0;
    const char* pass_kernel = "";
};

namespace lds {

// Points the handle and every buffer it owns at stream s: later work and the
// buffers' stream-ordered frees then follow s.  The caller makes sure that no
// work on the previous stream is pending.
void set_stream(lds_graph* g, cudaStream_t s);

// Builds slot_edge (canonical edge id of every CSR slot) if not present.
void ensure_slot_edge(lds_graph* g);

// Runs `iters` Frank-Wolfe iterations and leaves the results in g->fw_*.
void fw_run(lds_graph* g, lds_density d, int32_t iters, lds_precision p, bool want_last);

// Copies r, R, W (and the last choices when asked) of the handle's state out.
void copy_fw_state(lds_graph* g, lds_density d, lds_mem where, lds_fw_result* out);

// Builds the FW view (see lds_graph) if not present.
void ensure_fw_view(lds_graph* g);

// Builds the vertex -> triangle incidence (ascending triangle order) if not present.
void ensure_vertex_triangles(lds_graph* g);
// The same incidence for any triangle list (vt_idx indexes that list).
void build_vertex_triangles(const int32_t* ta, const int32_t* tb, const int32_t* tc, int64_t nt, int32_t nact,
                            DevBuf<int64_t>& vt_ptr, DevBuf<int32_t>& vt_idx, cudaStream_t s);

// Core (tr-core) numbers of G[alive] (internal ids, -1 outside the mask).
void core_numbers(lds_graph* g, bool tri, int64_t* core_int, const uint8_t* init_alive);

// Lists triangles into g->ta/tb/tc if not present.
void ensure_triangles(lds_graph* g);

// out[i] = map[in[i]] for i < k.
void map_ids(const int32_t* in, const int32_t* map, int64_t k, int32_t* out, cudaStream_t s);

// Scatter a per-internal-vertex array to original ids: out[to_orig[i]] = in[i].
void to_original_order_i64(const lds_graph* g, const int64_t* in_int, int64_t* out_orig);
void to_original_order_f64(const lds_graph* g, const double* in_int, double* out_orig);

// Batched on-chip Frank-Wolfe (fw_batch.cu): tunes the threads per graph of every
// size bucket among the given graphs (kept for the process), and reports the choice.
void fw_batch_autotune(int32_t count, lds_graph** graphs, int32_t iters, lds_precision p);
// lds_fw's edge-density iterations of one small graph on a thread-block cluster
// (fw_batch.cu); false when the graph does not fit, or (unless `any_size`) has
// more edges than the cluster form beats the grid-wide form on (the caller runs
// another path).
bool fw_cluster_run(lds_graph* g, int32_t N, lds_precision p, uint8_t* last, bool any_size);
int32_t fw_batch_threads(int32_t nact);

}  // namespace lds
