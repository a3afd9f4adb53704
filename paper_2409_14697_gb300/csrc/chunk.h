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
    // staged = 1: the pass's ops and reals are copied once per CTA into dynamic shared
    // memory after the tile, at byte offsets ops_off and reals_off
    int32_t staged;
    uint32_t ops_off, reals_off, n_reals;
};

// One pass over the state: tiles over the local bit set `lmask`, applying `kops`
// (tile-local positions; their reals in `mats`) in order.
void launch_chunk_pass(DeviceState &st, uint64_t lmask, const std::vector<KOp> &kops,
                       const std::vector<double> &mats);

// Tensor-core variant (complex64): ops of kind F_TC index bmats (B operands built by
// build_tc_operand; b_floats = largest B part of the pass, in floats).
void launch_chunk_pass_tc(DeviceState &st, uint64_t lmask, const std::vector<KOp> &kops,
                          const std::vector<double> &mats, const std::vector<float> &bmats, uint32_t b_floats);
// True if a k-qubit block can run on the tensor cores in a tile of 2^m amplitudes.
bool tc_available(int m, int k);
// Appends the TF32 hi/lo B operand of the complex D x D block G (D = 2^k) to out.
void build_tc_operand(const std::vector<cd> &G, int k, std::vector<float> &out, int &off, int &count);

}  // namespace qs
