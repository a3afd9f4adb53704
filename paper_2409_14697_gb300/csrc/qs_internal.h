// Internal declarations of the state-vector library (host side + kernel launchers).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <memory>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "qs.h"

namespace qs {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------------
// Errors: every internal failure throws qs::Error; the C entry points translate it to
// a return code and the thread-local message.
struct Error {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const std::string &msg);
void cuda_check(cudaError_t e, const char *what);
#define QS_CUDA(x) ::qs::cuda_check((x), #x)

// Counts kernel launches of this library (process-wide).
void count_launch(uint64_t n = 1);

// ---------------------------------------------------------------------------------
// Lowered operations (host IR).  Every gate record becomes one Op: its operand qubits
// (first = most significant of the group index, Eq. 3's row order) and a structural
// kind that tells the kernels which amplitudes of each group it touches.
enum OpKind : int32_t {
    K_H = 0,       // Hadamard on q[0]
    K_PERM1,       // X on q[0]: exchange the pair
    K_DIAG1,       // diag(d0, d1) on q[0]
    K_DENSE1,      // 2x2 on q[0]
    K_CTRL1,       // control q[0] = 1, 2x2 matrix u on target q[1]
    K_SWAP,        // exchange |01>,|10> of (q[0], q[1])
    K_DIAG,        // diagonal on k qubits: m holds the 2^k diagonal entries
    K_DENSE,       // dense 2^k x 2^k on k qubits (k >= 2), m row-major
    K_PHASEFN,     // merged run of diagonal gates on any qubits (pf; k = 0, mask in wide_mask)
};

struct PhaseFn;

// A factor of a diagonal block that depends on a qubit outside the pass's local set (whose
// bit is fixed within a tile): when bit h of the tile is 1, the entries of the block with
// local qubit t set (every entry for t = -1) are multiplied by f.
struct HiTerm {
    int t;
    int h;
    cd f;
};
constexpr int kMaxHiTerms = 64;

struct Op {
    OpKind kind;
    int k = 0;          // operand count
    int q[8] = {0};     // operands
    std::vector<cd> m;  // K_DIAG1: 2 entries; K_DENSE1/K_CTRL1: 4; K_DIAG: 2^k; K_DENSE: 4^k;
                        // K_H: empty (1/sqrt2) or {scale} (gate-by-gate deferred scale)
    std::shared_ptr<const PhaseFn> pf;  // K_PHASEFN
    uint64_t wide_mask = 0;             // K_PHASEFN: every qubit the function reads
    std::vector<HiTerm> hi;             // K_DIAG blocks of a chunk pass: non-local factors
    // The full 2^k x 2^k matrix of the op on q[0..k-1] (row-major).
    std::vector<cd> full() const;
    uint64_t qmask() const {
        uint64_t r = wide_mask;
        for (int j = 0; j < k; j++) r |= 1ull << q[j];
        return r;
    }
};

// Validates one gate record against an n-qubit state (throws QS_ERR_INVALID).
void validate_gate(const qs_gate &g, int n);
// Lowers a validated record to an Op (own gate definitions, FP64).
Op lower_gate(const qs_gate &g);

// Gate fusion (Sec. II-B "Gate Fusion", Sec. III-A tier 5): greedily merges runs of
// consecutive ops into dense (or, if every member is diagonal, diagonal) blocks on at most
// fuse_k qubits.  FP64 host products.  The paper leaves the merge decision to a cost
// function; here, with sweep_flops >= 0, a merge is taken only if the fused block costs at
// most the flops per amplitude of its members applied one by one plus sweep_flops (the
// value of one saved pass over the tile).  sweep_flops < 0 merges whenever the width fits.
// lmask != 0: ops with a qubit outside lmask (a chunk pass's local set) are not fused.
std::vector<Op> fuse_ops(std::vector<Op> ops, int fuse_k, double sweep_flops = -1.0, uint64_t lmask = 0);
// Merges runs of consecutive diagonal gates into diagonal blocks of at most max_k qubits
// where that costs fewer FP64 operations per amplitude in a shared-memory pass (a block
// multiplies only the elements whose "control" qubits, those on whose 0-half every entry
// is 1, are set; sweep_cost is added per separate sweep).  FP64 host products; blocks
// that come out as the identity are dropped.
//
// With lmask != 0 (the pass's local qubits), two-qubit diagonals with one qubit outside
// lmask are taken too: d(x_a, x_h) = d(x_a, 0) * [x_h ? d(x_a, 1) / d(x_a, 0) : 1], so the
// block's table gets the x_h = 0 slice on its local qubit a and the rest becomes HiTerms
// (g0 = d(0,1)/d(0,0) on every entry, g1/g0 with g1 = d(1,1)/d(1,0) on the entries with a
// set).  A block's table covers its non-control qubits: at most 2^max_k entries, and
// 2^(max_k - 1) with HiTerms (at most 64), so that table and terms fit one op's reals.
std::vector<Op> merge_tile_diagonals(std::vector<Op> ops, int max_k, double sweep_cost, uint64_t lmask = 0);
// Qubits of a two-qubit diagonal (no zero entry) that may be its only local qubit in a
// chunk pass: a with d(0, x) = 1 for both x (the gate is then a phase on a's 1-half chosen
// by the other bit, which keeps a a control of the block: CP, CZ, controlled RZ).  0 if none.
uint64_t hi_local_choices(const Op &op);
// True for ops that are diagonal in the computational basis (they commute with each other).
bool op_is_diagonal(const Op &op);
// Gate-by-gate form of a circuit: every one-qubit diagonal diag(d0, d1) with d0 != 1 (RZ)
// but the last becomes diag(1, d1 / d0), which changes only the amplitudes with the
// target bit set; the product of the factored d0 (a global phase) is multiplied into the
// last one, applied in full.  The product of the ops is unchanged (FP64 host arithmetic),
// so the state is exact again when the last op has run.
std::vector<Op> fold_global_phases(const std::vector<Op> &ops);
// complex128 form of the Hadamards of a circuit (gate-by-gate FP64 calls, and the ops of a
// chunk pass): all but the last (and
// every (kMaxUnscaledH + 1)-th) become the unscaled butterfly (a + b, a - b), 2 FP64
// additions per amplitude instead of 3 FP64 instructions; the collected factor 2^(-k/2) is
// carried by the next scaled one (K_H with m = {scale}), so the state is exact again when
// the last Hadamard has run.  Between, amplitudes grow by at most 2^(kMaxUnscaledH / 2).
constexpr int kMaxUnscaledH = 63;
void defer_hadamard_scale(std::vector<Op> &ops);
// complex128 FP64 chunk passes of 256 tiles or more: a one-qubit matrix with a real first
// entry and complex others (U3) is P(phi) R P(lambda) with R = [[a, -s], [s, a]] real (4
// FP64 instructions per amplitude instead of 7) and P(x) = diag(1, e^{ix}).  For each run
// of such ops on distinct qubits the P(lambda) of all come first, then the R, then the
// P(phi) (ops on distinct qubits commute), so the phases join the neighbouring diagonal
// gates (a CZ layer) in one run that merge_tile_diagonals applies as a few table
// multiplies.  Ops whose matrix the split does not reproduce to 1e-14 are kept.
std::vector<Op> split_one_qubit_phases(const std::vector<Op> &ops);
// Structure class (D1_GENERAL, D1_R0, D1_REAL, D1_RX of kops.cuh) of a 2x2 matrix,
// row-major: the cheapest form the complex128 kernels apply it with.
int32_t d1_class(const std::vector<cd> &u);
// Real flops per amplitude of applying op alone (structure-aware: the complex128 forms of
// one-qubit matrices, the unscaled Hadamard, the elements a controlled op touches).
double op_flops(const Op &op);

// ---------------------------------------------------------------------------------
// Device-side geometry of a streaming application: each group is one base index with
// the fixed bits (sorted ascending, in element units) cleared; set_mask bits forced
// to one; the op touches nt elements at base | set_mask | off[t].
struct StreamGeom {
    int nf;             // number of fixed bits (1..3)
    int fb[3];          // fixed bits, ascending (element index space)
    uint64_t set_mask;  // forced-one bits (element index space)
    int nt;             // touched elements per group (1, 2 or 4)
    uint64_t off[4];    // offsets of the touched elements
    uint64_t n_groups;  // 2^(n_elem_bits - nf)
};

// Parameter arenas per state, used in turn by successive qs_apply_circuit calls: a call
// waits (on the host) only for the call kArenas - 1 before it, so a caller can queue that
// many calls on a state whose stream waits for other work without stalling.
constexpr int kArenas = 16;

// Tensor Product Booster: most groups of one product pass (k_tpb.cu, tpb.cpp).
constexpr int kTpbMaxGroups = 4;

struct DeviceState {
    void *psi = nullptr;  // amplitudes
    int n = 0;            // qubits
    int dtype = QS_C128;
    int prec = QS_PREC_FP64;  // complex128 arithmetic: QS_PREC_FP64 or QS_PREC_DF32
    bool ix = false;          // complex128 one-qubit dense and diagonal ops (streaming and
                              // chunk passes): integer products (QS_PREC_IX64)
    bool reg_phases = true;   // complex64 chunk passes: register phases (2^13-amplitude tiles)
    cudaStream_t stream = nullptr;
    // scratch for reductions (owned by the state; stream-ordered allocation on `stream`)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    int num_sms = 0;
    // parameter arenas (a ring, one per qs_apply_circuit call)
    void *arena_dev[kArenas] = {};
    void *arena_host[kArenas] = {};
    size_t arena_cap[kArenas] = {};
    size_t arena_used = 0;
    int arena_cur = 0;
    cudaEvent_t arena_ev[kArenas] = {};
    std::vector<std::pair<void *, void *>> arena_retired[kArenas];  // outgrown (device, pinned) buffers
    std::vector<void *> pinned_retired;  // outgrown page-locked buffers, freed with the state
    // device error word written by bounded waits (QS_ERR_TIMEOUT), checked on sync
    int *dev_err = nullptr;
    // two FP64 squared norms (before / after) for the norm-preserving correction
    double *dev_norms = nullptr;
    // the amplitudes are |0...0> (set by launch_set_zero_state; cleared by every other
    // write): qs_apply_circuit may then build a prefix as a tensor product
    bool known_zero = false;
    // Tensor Product Booster: group sub-states (small states of their own) and their memory
    DeviceState *tpb_sub[kTpbMaxGroups] = {};
    void *tpb_buf = nullptr;
    size_t tpb_buf_bytes = 0;
};

// Executor: runs one lowered circuit on d.stream (mode, fusion and planning from o).
void run_circuit(DeviceState &d, const std::vector<Op> &ops, const qs_options &o, qs_stats &st);
// Frees everything DeviceState owns except psi and the stream.
void free_device_state(DeviceState &d);
// Frees the booster's sub-states and memory (part of free_device_state).
void tpb_free(DeviceState &d);
// Creates the booster's sub-states of d now, each with parameter arenas of `arena_bytes`
// (so that a later call needs no page-locked allocation).
void tpb_reserve(DeviceState &d, size_t arena_bytes);
void arena_begin(DeviceState &st);
void arena_end(DeviceState &st);
// Gives every parameter arena of st at least `bytes` of capacity now, so that later calls
// with programs that fit never grow one (growing frees memory later, and cudaFree waits for
// the whole device).
void arena_reserve(DeviceState &st, size_t bytes);

// Launchers (kernels live in the .cu files).  All are asynchronous on st.stream.
void launch_stream_op(DeviceState &st, const Op &op);           // K1, one op, one pass
void launch_phasefn(DeviceState &st, const Op &op);             // merged diagonal run, one pass
void launch_set_zero_state(DeviceState &st);                    // |0..0>
// psi[x] = prod_g tables[g][pext(x, masks[g])]: one write pass (masks partition the qubits)
void launch_tpb_product(DeviceState &st, const void *const *tables, const uint64_t *masks, int groups);
void launch_scale(DeviceState &st, double f);                   // psi *= f
// Reductions (K4).  expz may be null (norm only).  Results are copied to host.
void reduce_expz(DeviceState &st, double *norm, double *expz);
void top_k(DeviceState &st, uint32_t k, uint64_t *idx, double *amp);
// Asynchronous forms (no host wait): results land in device memory.  reduce_expz_async
// writes out_dev[0] = squared norm, out_dev[1 + q] = <Z_q>; top_k_async writes k indices
// and 2k doubles.  Scratch must have been sized by the caller (scratch_expz_bytes /
// scratch_topk_bytes) before any capture or concurrent use.
void reduce_expz_async(DeviceState &st, double *out_dev);
// Squared norm into out_dev[0] (asynchronous); psi *= sqrt(norms[0] / norms[1]).
void reduce_norm_async(DeviceState &st, double *out_dev);
void launch_scale_ratio(DeviceState &st, const double *norms_dev);
void top_k_async(DeviceState &st, uint32_t k, uint64_t *idx_dev, double *amp_dev);
size_t scratch_expz_bytes(int n);
size_t scratch_topk_bytes(int n, uint32_t k);

// Host <-> device copy of `bytes` on st.stream (asynchronous).  Ranges of page-locked host
// memory mapped into the device (cudaHostAlloc, registered memory) of 4 MiB or more are
// copied by a kernel that reads or writes them over the CPU-GPU link: on GB300 copy-engine
// transfers were measured to run at 20-46 GB/s for their first gigabytes now and then
// before reaching the link rate (211 GB/s in, 194 GB/s out), while SM copies hold that
// rate from the start.  ctas: the copy kernel's grid (0: 8 per SM, for copies the caller
// waits for), or kCopyEngines: cudaMemcpyAsync on the copy engines, for copies meant to run
// under kernels of other streams (a copy kernel there waits for SM slots that persistent
// kernels hold, and a slow start of a copy-engine transfer is hidden).  Other host memory:
// cudaMemcpyAsync.
void copy_host(DeviceState &st, void *dst, const void *src, size_t bytes, bool to_device, int ctas);
constexpr int kCopyEngines = -1;

// Algorithmic bytes of one streaming application of op on an n-qubit state.
double stream_bytes(const Op &op, int n, int dtype);

// Persistent grid: SMs x resident blocks of kernel fn at this block size / smem, capped
// by the number of work blocks.  Inside a LaunchYield scope of the calling thread, grids
// grow so that no block loops over more than `iters` work blocks: the grid-stride kernels
// compute the same results with any grid, and their blocks then end every few hundred
// microseconds, which lets the CTA scheduler start pending blocks of higher-priority
// streams (the serving loop's small requests) instead of waiting for a whole launch.
int persistent_grid(const void *fn, int threads, size_t smem, uint64_t work_blocks);
struct LaunchYield {
    explicit LaunchYield(int iters);
    ~LaunchYield();
    int prev;
};

// Copies `bytes` of host data into the state's device parameter arena (asynchronously,
// ordered on st.stream before any later launch) and returns the device address.
void *upload_params(DeviceState &st, const void *host, size_t bytes);

// Waits for st.stream and raises QS_ERR_TIMEOUT if a kernel's bounded wait gave up.
void sync_and_check(DeviceState &st);

// Scratch helper: makes sure st.scratch holds at least `bytes`.
void ensure_scratch(DeviceState &st, size_t bytes);
int device_sm_count();

}  // namespace qs
