// K6 batched persistent execution: host-side batch object and device pass descriptor.
#pragma once

#include "kops.cuh"
#include "qs_internal.h"

namespace qs {

// Device descriptor of one pass of one circuit in the batch's global work list.
struct BatchPass {
    int32_t circuit;
    int32_t self;        // index of this pass (its completion counter)
    int32_t m, c0, nlh;  // tile geometry as in the chunk kernel
    int32_t lhigh[24];
    int32_t n_ops;
    int32_t init_zero;   // first pass of the circuit: the tile starts as |0...0>
    int32_t dep;         // completion counter to wait for (-1: none)
    uint32_t dep_need;   // tiles that counter must reach
    uint32_t n_tiles;
    uint64_t state_off;  // element offset of the circuit's state in the batch arena
    uint64_t tile_start; // global work index of this pass's tile 0
    uint64_t ops_off;    // first KOp of the pass
    uint64_t mats_off;   // first matrix real of the pass
    uint32_t n_reals;    // matrix reals of the pass
    int32_t staged;      // 1: ops and reals are copied into shared memory once per work item
};

struct Batch {
    int dtype = QS_C64;
    std::vector<int> nq;
    std::vector<uint64_t> state_off;
    std::vector<int> total_passes_per_circuit;
    std::vector<BatchPass> passes;
    uint64_t state_elems = 0, total_items = 0;
    int max_m = 0, grid = 0;
    size_t prog_bytes = 0;  // largest staged pass program (ops + reals), in bytes
    long long wait_limit_ns = 2000000000ll;
    cudaStream_t stream = nullptr;
    bool owns_stream = true;
    cudaGraphExec_t exec = nullptr;
    void *d_states = nullptr, *d_mats = nullptr;
    BatchPass *d_passes = nullptr;
    KOp *d_ops = nullptr;
    unsigned long long *d_counter = nullptr;
    unsigned int *d_done = nullptr;
    int *d_err = nullptr, *d_abort = nullptr;
};

// Plans every circuit, lays out the work list and uploads all tables.
void batch_build(Batch &b, const std::vector<std::vector<Op>> &circ_ops, const std::vector<int> &nq,
                 const qs_options &o);
// Captures {counter resets, persistent kernel} into b.exec.
void batch_capture(Batch &b);

}  // namespace qs
