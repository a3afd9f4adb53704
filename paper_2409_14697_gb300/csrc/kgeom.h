// Host: lowered Op -> KOp (kernel-side op) in a given index space.
#pragma once

#include "kops.cuh"
#include "qs_internal.h"

namespace qs {

// Builds the KOp of `op`; pos[q] is the bit position of qubit q in the target index
// space (identity for the whole state, tile-local position for a chunk pass).  The
// op's matrix entries are appended to `mats` (as re, im doubles; KOp.mat indexes them).
KOp make_kop(const Op &op, const int *pos, std::vector<double> &mats);

// complex64 passes: replaces runs of consecutive one- and two-bit ops whose positions fit
// in 4 tile positions by F_RGROUP ops (applied in registers, one shared-memory sweep per
// run); member matrices are appended to `mats`.  m = tile bits.
std::vector<KOp> group_registers(const std::vector<KOp> &in, std::vector<double> &mats, int m);

// Fraction of the state's bytes one streaming application reads and writes, counting
// whole DRAM sectors of 2^sector_bits elements.
double kop_touched_fraction(const KOp &k, int sector_bits);

}  // namespace qs
