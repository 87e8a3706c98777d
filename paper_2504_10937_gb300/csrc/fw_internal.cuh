// Pieces shared by the Frank-Wolfe sources.
#pragma once

#include <algorithm>
#include <vector>

#include "graph.cuh"

namespace lds {

// Event pairs around every pass launch, read after the final synchronisation.
struct PassTimer {
    std::vector<cudaEvent_t> ev;
    int used = 0;
    bool on = false;
    void start(cudaStream_t s) {
        if (!on) return;
        if ((int)ev.size() < used + 2) {
            cudaEvent_t a, b;
            LDS_CUDA(cudaEventCreate(&a));
            LDS_CUDA(cudaEventCreate(&b));
            ev.push_back(a);
            ev.push_back(b);
        }
        LDS_CUDA(cudaEventRecord(ev[used], s));
    }
    int64_t iters = 0;     // iterations the timed launches covered (one per launch unless given)
    void stop(cudaStream_t s, int64_t covered = 1) {
        if (!on) return;
        LDS_CUDA(cudaEventRecord(ev[used + 1], s));
        used += 2;
        iters += covered;
    }
    double total_ms() {
        double t = 0;
        for (int i = 0; i < used; i += 2) {
            float ms = 0;
            LDS_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            t += ms;
        }
        return t;
    }
    ~PassTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

// Number of iterations whose bit planes are kept before folding: at most
// ~2 GiB of planes, between 32 and 512 iterations, never more than N.
inline int planes_capacity(int64_t plane_words, int N) {
    int64_t budget = (int64_t)2 << 30;
    int64_t cap = plane_words > 0 ? budget / (plane_words * 4) : N;
    cap = std::max<int64_t>(32, std::min<int64_t>(cap, 512));
    return (int)std::min<int64_t>(cap, std::max(N, 1));
}

// Folds `nplanes` bit planes (plane k at planes + k * nchunks, bit l of word g
// for item 32 g + l) into W: W[item] += mult * (i_first + k + 1) per set bit.
void fold_planes(const uint32_t* planes, int nplanes, int64_t nchunks, int64_t nitems, int64_t i_first,
                 int64_t mult, uint32_t* W, cudaStream_t s);

// Results of an edge FW run in internal ids.
struct EdgeFwOut {
    DevBuf<int64_t> R_int;     // [n] exact loads of the returned weights (internal ids)
    DevBuf<double> r_int;      // [n] reported loads (internal ids)
    DevBuf<int64_t> W_edge;    // [m] D alpha_{u,v} per canonical edge (if wanted)
    DevBuf<uint8_t> last_edge; // [m] alpha_hat_{u,v} of the last iteration (if wanted)
};

// Oriented, key-based edge FW (exact and binary32).  Returns false when the
// scaled loads would not fit the 64-bit keys (the caller then uses the
// symmetric-slot kernel).
bool run_edge_fw_oriented(lds_graph* g, int N, lds_precision p, bool want_w, bool want_last, EdgeFwOut& out,
                          PassTimer& timer);

}  // namespace lds
