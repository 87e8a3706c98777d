// Pruning (Alg. 3) shared by the pipeline.
#pragma once

#include "graph.cuh"

namespace lds {

// status[x] (internal ids, device): 0 kept, 1 removed by rule 1, 2 removed by
// rule 2.  Bounds are device arrays num / den in internal ids.
void prune(lds_graph* g, bool tri, const int64_t* ub_num, const int64_t* ub_den, const int64_t* lb_num,
           const int64_t* lb_den, uint8_t* status);

}  // namespace lds
