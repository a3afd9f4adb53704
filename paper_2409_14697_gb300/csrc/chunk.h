// K2 chunk pass: argument block and launcher.
#pragma once

#include "kops.cuh"
#include "qs_internal.h"

namespace qs {

struct ChunkArgs {
    int32_t m;          // local qubits (tile = 2^m amplitudes)
    int32_t c0;         // local bits 0..c0-1 are contiguous (runs of 2^c0 amplitudes)
    int32_t nlh;        // m - c0
    int32_t lhigh[24];  // global positions of the other local bits, ascending
    int32_t n_ops;
    uint64_t n_tiles;   // 2^(n-m)
};

// One pass over the state: tiles over the local bit set `lmask`, applying `kops`
// (tile-local positions; their reals in `mats`) in order.
void launch_chunk_pass(DeviceState &st, uint64_t lmask, const std::vector<KOp> &kops,
                       const std::vector<double> &mats);

}  // namespace qs
