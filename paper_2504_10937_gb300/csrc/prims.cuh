// Device-wide primitives written for this library: exclusive scans and a
// stable LSD radix sort.  All run on the given stream; temporary memory comes
// from dev_alloc.
#pragma once

#include "common.cuh"

namespace lds {

// out[i] = sum_{j < i} in[i]; returns the total (copied to the host, which
// synchronises the stream).  in and out may alias.  n may be 0.
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Same, without the host read-back: the total is written to *total_dev.
void exclusive_scan_i64_dev(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                            cudaStream_t s);
// int32 input flags / counts, int64 exclusive sums.
int64_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of uint64 keys on bits [0, bits), 8 bits per pass,
// with an optional uint32 payload.  keys / vals are sorted in place (a
// temporary ping-pong buffer is allocated).  vals may be null.
void radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s);

// Gathers: out[i] = in[idx[i]].
void gather_u32(const uint32_t* in, const uint32_t* idx, uint32_t* out, int64_t n, cudaStream_t s);

}  // namespace lds
