// Host: lowered Op -> KOp (kernel-side op) in a given index space.
#pragma once

#include "kops.cuh"
#include "qs_internal.h"

namespace qs {

// Builds the KOp of `op`; pos[q] is the bit position of qubit q in the target index
// space (identity for the whole state, tile-local position for a chunk pass).  The
// op's matrix entries are appended to `mats` (as re, im doubles; KOp.mat indexes them).
KOp make_kop(const Op &op, const int *pos, std::vector<double> &mats);

// The same for the shared-memory tile kernels: a diagonal on 3 or more qubits whose entries
// are 1 unless some qubits ("controls") are set becomes F_CDIAGK, which touches only the
// elements with every control set.
KOp make_tile_kop(const Op &op, const int *pos, std::vector<double> &mats);

// complex128 FP64 tile programs: an unscaled Hadamard (F_H with scale 1) directly followed
// by an F_CDIAGK whose only control is the Hadamard's position becomes one F_HCDIAGK (the
// block multiplies only the elements the butterfly's difference lands on, so both fit
// one sweep of the tile; a QFT target and its controlled phases).
std::vector<KOp> join_h_cdiag(const std::vector<KOp> &kops, const std::vector<double> &mats);

// complex64 tiles of 2^m amplitudes with 2^thread_bits threads: true if register phases
// apply (m = thread_bits + kRpBits).
bool rphase_applicable(int m, int thread_bits);
// Packs the pass's ops (logical qubits, tile position of qubit q = pos[q]) into register
// phases (F_RPHASE KOps; their programs appended to `mats`).  Ops no phase can hold
// (swaps, wider dense or diagonal blocks) become ordinary KOps in their place in the
// order.  n_phases (optional) receives the number of phases.
std::vector<KOp> build_register_phases(const std::vector<Op> &ops, const int *pos, int m, int thread_bits,
                                       std::vector<double> &mats, int *n_phases = nullptr);

// Fraction of the state's bytes one streaming application reads and writes, counting
// whole DRAM sectors of 2^sector_bits elements.
double kop_touched_fraction(const KOp &k, int sector_bits);

}  // namespace qs
