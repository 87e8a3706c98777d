// Verification stage and driver helpers.
#pragma once

#include <vector>

#include "graph.cuh"

namespace lds {

// Bounds on compact numbers, num / den per internal vertex id (device).
struct Bounds {
    DevBuf<int64_t> un, ud, ln, ld;
};

// Per-graph scratch flags and local index map (all flags zero between uses).
struct Scratch {
    cudaStream_t s;
    DevBuf<uint8_t> in, in2;
    DevBuf<int32_t> local;
    explicit Scratch(lds_graph* g);
};

struct VerifyStats {
    int64_t flows = 0;
    int64_t denser_neighbour = 0;
};

// IsDensest on G[list] (list: k internal ids on the device); npat receives |E(S)| or |T(S)|.
bool is_densest(lds_graph* g, bool tri, const int32_t* list, int32_t k, Scratch& sc, int64_t* npat);

// IsLDS (edge) / IsLTDS (triangle) of the connected set `list` with |E(S)| (|T(S)|) = npat.
// mode: the network of Alg. 4 / Alg. 7 (LDS_VERIFY_BOUNDS), the upper-bound-only
// network of the Sec. 7 ablation (LDS_VERIFY_CORE), or the whole graph (LDS_VERIFY_WHOLE).
bool is_lds(lds_graph* g, bool tri, const int32_t* list, int32_t k, int64_t npat, const Bounds& b, Scratch& sc,
            VerifyStats* st, lds_verify mode = LDS_VERIFY_BOUNDS);

// Connected components of G[list]: members (device) grouped by component, each
// component's members ascending, components ordered by smallest member;
// starts[c] .. starts[c+1] delimit component c.
void components(lds_graph* g, const int32_t* list, int32_t k, Scratch& sc, DevBuf<int32_t>& members,
                std::vector<int32_t>& starts);

// Patterns E(list) or T(list) over all of `list` with local index = position in list.
int64_t build_all_patterns(lds_graph* h, bool tri, const int32_t* list, int32_t k, Scratch& sc,
                           DevBuf<int64_t>& pptr, DevBuf<int32_t>& pidx);

// A new handle for G[list] (list ascending): vertex i of the subgraph is list[i].
lds_graph* subgraph(lds_graph* g, const int32_t* list, int32_t k, Scratch& sc);

}  // namespace lds
