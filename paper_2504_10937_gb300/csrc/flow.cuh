// Pattern-network maximum flow (Alg. 8) shared by the verification stages.
#pragma once

#include "graph.cuh"

namespace lds {

// Patterns j = 0..np-1 list vertices pidx[pptr[j] .. pptr[j+1]) in 0..nv-1
// (device arrays).  Capacities: source -> pattern q, pattern -> vertex q,
// vertex -> sink p.  Returns the maximum flow; side[v] (device, optional) is 1
// for vertices on the largest source side of a minimum cut.
int64_t pattern_max_flow(const int64_t* pptr, const int32_t* pidx, int32_t np, int32_t nv, int64_t p, int64_t q,
                         uint8_t* side, cudaStream_t s);

}  // namespace lds
