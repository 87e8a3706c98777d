// ExtractSG state shared by the pipeline stages.
#pragma once

#include <vector>

#include "graph.cuh"

namespace lds {

struct SgState {
    int64_t D = 0;                        // denominator of the loads
    DevBuf<int32_t> order;                // [n] internal ids by (load desc, id asc)
    DevBuf<int32_t> pos;                  // [n] position of each internal id
    std::vector<int64_t> cuts;            // 1-based cut positions (ascending)
    std::vector<int64_t> group_end;       // exclusive end position of each accepted group
    std::vector<long long> lo, hi;        // min / max modified load of each group (over D)
    int64_t chain_checks = 0;             // single checks of merged candidates
};

// Alg. 2 on the last Frank-Wolfe run of g (g->fw_*).
void extract_sg(lds_graph* g, SgState& st);

}  // namespace lds
