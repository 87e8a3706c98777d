// Pattern-network maximum flow (Alg. 8) shared by the verification stages.
#pragma once

#include "graph.cuh"

namespace lds {

// Patterns j = 0..np-1 list vertices pidx[pptr[j] .. pptr[j+1]) in 0..nv-1
// (device arrays).  The network is Alg. 8's: source -> pattern q, pattern ->
// each member q, vertex -> sink p (rho = p / q).  Returns the maximum flow;
// side[v] (device, optional) is 1 for vertices on the largest source side of a
// minimum cut.
//
// share (device, optional, aligned with pidx): nonnegative weights that split
// each pattern's unit among its members for the initial preflow (a warm start
// from the Frank-Wolfe weights); null or an all-zero pattern splits evenly.
// The result does not depend on it.
//
// stop_if_short: return -1 as soon as some excess is proven unable to reach
// the sink (the maximum flow is then below q * np); side is not written.
int64_t pattern_max_flow(const int64_t* pptr, const int32_t* pidx, int32_t np, int32_t nv, int64_t p, int64_t q,
                         const int64_t* share, uint8_t* side, bool stop_if_short, cudaStream_t s);

}  // namespace lds
