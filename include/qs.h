/*
 * qs.h — C interface of the GB300 (sm_103a) state-vector quantum-circuit simulator.
 *
 * The operation implemented is the one of QueenV2 (arXiv 2409.14697):
 *   - Sec. II-A, Eq. 1: an N-qubit state is the vector of 2^N complex amplitudes a_i,
 *     i in [0, 2^N).  Qubit q is bit q of i (qubit 0 least significant, so low qubits
 *     are contiguous in memory; Sec. II-B speaks of moving qubits to the "least
 *     significant bits" for locality).
 *   - Sec. II-A, Eq. 2: a one-qubit gate G replaces every pair (a_{..0_q..}, a_{..1_q..})
 *     by G times the pair.
 *   - Sec. II-A, Eq. 3 and the sentence before it: a k-qubit gate is a 2^k x 2^k matrix
 *     applied to every group of 2^k amplitudes that differ only in its operand bits.
 *     For operands (q_0, ..., q_{k-1}) the row index inside the group is
 *     s = sum_j bit(q_j) * 2^(k-1-j): the first operand is the most significant, the
 *     row order of Eq. 3, whose printed CNOT matrix makes the first operand the control.
 *   - Sec. II-B / III: gate fusion, qubit reordering and in-cache (block-by-block)
 *     execution are how the library schedules that work; they never change the result
 *     beyond floating-point rounding.
 *
 * Conventions for every function:
 *   - Return value: QS_OK (0) on success, a negative QS_ERR_* code on failure
 *     (QS_NOT_READY = 1 only from qs_poll).  On failure a message is available from
 *     qs_last_error() (thread-local, valid until the next call on the same thread).
 *   - Ownership: the caller owns every host array it passes; the library copies what it
 *     needs before returning.  The library owns all device memory it allocates.  Output
 *     arrays are allocated by the caller.
 *   - Amplitude layout (host and device): interleaved (re, im), index i at element i;
 *     complex128 = two doubles (16 bytes), complex64 = two floats (8 bytes).
 *   - Thread safety: a qs_state must be used by one thread at a time; a qs_server is
 *     thread-safe.  Calls are synchronous unless stated otherwise.
 *   - Failure detection: no device code traps or asserts.  Device-side bounded waits
 *     return QS_ERR_TIMEOUT; CUDA errors return QS_ERR_CUDA with the CUDA message.
 */
#ifndef QSIM_QS_H_
#define QSIM_QS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QS_ABI_VERSION 4
#define QS_MAX_QUBITS 36      /* index arithmetic limit; memory is the real limit */
#define QS_MAX_GATE_QUBITS 8  /* operands per gate record */

typedef struct qs_state qs_state;   /* opaque: one state vector resident in HBM */
typedef struct qs_server qs_server; /* opaque: serving runtime (continuous batching) */

typedef enum { QS_C64 = 1, QS_C128 = 2 } qs_dtype;

enum {
    QS_OK = 0,
    QS_NOT_READY = 1,
    QS_ERR_INVALID = -1,     /* bad argument: qubit out of range, repeated operand, ... */
    QS_ERR_NOMEM = -2,       /* device memory or admission budget exhausted */
    QS_ERR_CUDA = -3,        /* a CUDA runtime/driver call failed */
    QS_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    QS_ERR_BUSY = -5,        /* object still has work in flight */
    QS_ERR_UNSUPPORTED = -6  /* valid request the library does not implement */
};

/* Gate types.  Matrices (first operand most significant in the group index):
 *   H = [[1,1],[1,-1]]/sqrt2      X, Y, Z = Pauli       S = diag(1,i)   T = diag(1,e^{i pi/4})
 *   RX(t) = exp(-i t X/2)  RY(t) = exp(-i t Y/2)  RZ(t) = exp(-i t Z/2) (global phase kept)
 *   P(l) = diag(1, e^{i l})
 *   U3(t,p,l) = [[cos(t/2), -e^{il} sin(t/2)], [e^{ip} sin(t/2), e^{i(p+l)} cos(t/2)]]
 *   CNOT(c,t) = Eq. 3           CZ = diag(1,1,1,-1)       SWAP exchanges |01>,|10>
 *   CU3(c,t; t,p,l) = |0><0| (x) I + |1><1| (x) U3        CP(l) = diag(1,1,1,e^{il})
 *   RZZ(t) = exp(-i t Z(x)Z/2)
 *   DENSE: the caller's 2^nq x 2^nq matrix, row-major, interleaved (re, im) doubles. */
typedef enum {
    QS_H = 0, QS_X = 1, QS_Y = 2, QS_Z = 3, QS_S = 4, QS_T = 5,
    QS_RX = 6, QS_RY = 7, QS_RZ = 8, QS_P = 9, QS_U3 = 10,
    QS_CNOT = 11, QS_CZ = 12, QS_SWAP = 13, QS_CU3 = 14, QS_CP = 15, QS_RZZ = 16,
    QS_DENSE = 17
} qs_gate_type;

/* One gate record (72 bytes).  q[0..nq-1] are distinct qubits < n; p[] holds the angles
 * (theta, phi, lambda) of the parametrised types; m is read only for QS_DENSE (nq <= 6)
 * and must stay valid for the duration of the call that receives the record. */
typedef struct {
    int32_t type;
    int32_t nq;
    int32_t q[QS_MAX_GATE_QUBITS];
    double p[3];
    const double *m;
} qs_gate;

/* Execution modes for qs_apply_circuit. */
enum {
    QS_MODE_AUTO = 0,     /* fuse + plan in-cache chunk passes (default) */
    QS_MODE_GATE = 1,     /* plain gate by gate: one streaming launch per gate */
    QS_MODE_CHUNK = 2,    /* every gate through in-shared-memory chunk passes */
    QS_MODE_FUSED = 3     /* fuse to dense k-qubit blocks, one full pass per block */
};
/* Arithmetic used for complex128 gate updates (complex64 always uses FP32).  The state
 * is stored as IEEE doubles in every mode. */
enum {
    QS_PREC_DEFAULT = 0,  /* QS_PREC_IX64 */
    QS_PREC_FP64 = 1,     /* native FP64 instructions */
    QS_PREC_DF32 = 2,     /* double-float: FP32 pairs with compensated products and sums
                             (TwoProd/TwoSum); each update is within ~2^-46 of the sum of
                             |matrix entry x amplitude| of the exact value.  Applies to
                             the streaming and the in-cache (chunk) passes. */
    QS_PREC_IX64 = 3      /* one-qubit dense gates and diagonal ops with constant factors
                             (streaming launches and chunk passes), and the factor multiply
                             of merged diagonal runs: each real output as a dot product of
                             64-bit integer significand products, aligned to its largest
                             term in one signed 64-bit accumulator and rounded once to a
                             double: within 0.5 ulp + 2^-56.4 x the largest |matrix entry x
                             amplitude| of the exact value (a chain of FP64 multiply-adds:
                             about one ulp of each partial sum per term).  About one value
                             in four of every thread runs the native FP64 form, so both
                             pipes work.  Inputs below 2^-1022 in magnitude count as 0 and
                             outputs below 2^-959 flush to 0.  Other ops (Hadamards,
                             table-driven diagonal blocks, dense blocks of 2+ qubits) as
                             QS_PREC_FP64. */
};

/* Bits of qs_options.flags (all off by default). */
enum {
    QS_OPT_NO_REG_PHASES = 1,   /* complex64 passes over 2^13-amplitude tiles: one shared-memory
                                   sweep per op instead of register phases (runs of one-qubit,
                                   controlled and at most two-qubit diagonal gates applied to
                                   amplitudes held in registers, one sweep per run) */
    QS_OPT_NO_DIAG_MERGE = 2,   /* QS_MODE_AUTO / QS_MODE_CHUNK: never merge runs of diagonal
                                   gates into one phase-function pass (by default both plans are
                                   built and the one with fewer passes over the state runs) */
    QS_OPT_NO_TC_NORM_FIX = 4,  /* no norm-preserving correction after complex64 circuits that
                                   used tensor-core blocks (by default the squared norm before
                                   the circuit is restored, removing the small systematic shrink
                                   of FP32 accumulation inside the MMA) */
    QS_OPT_NO_TPB = 8           /* QS_MODE_AUTO / QS_MODE_CHUNK: no Tensor Product Booster.  By
                                   default (states of 20 qubits or more) a call on a state that
                                   holds |0...0> (after qs_create or qs_reset, before anything
                                   else writes it) builds the longest prefix of the circuit whose
                                   gates keep the qubits in independent groups as a tensor
                                   product of the groups' small sub-states, in one write pass,
                                   when that saves passes (Sec. III-A tier 1).  Amplitudes
                                   written through the device pointer of qs_info are not seen:
                                   call qs_set_amplitudes, or pass this flag, after such
                                   writes. */
};

/* Options for qs_apply_circuit; pass NULL for defaults.  Zero fields mean "choose". */
typedef struct {
    int32_t mode;         /* QS_MODE_* */
    int32_t fuse_k;       /* max qubits of a fused block (0: choose; 1 disables fusion) */
    int32_t chunk_m;      /* local qubits of a chunk pass (0: choose) */
    int32_t precision;    /* QS_PREC_* */
    uint32_t flags;       /* QS_OPT_* bits */
    /* reserved[0], reserved[1]: batched-launch wait limit in microseconds and a test hook
     * (qs_batch_create); reserved[2], reserved[3]: zero. */
    int32_t reserved[4];
} qs_options;

/* Statistics of the last qs_apply_circuit on a state. */
typedef struct {
    int64_t gates_in;      /* gate records received */
    int64_t ops_after_fuse;/* operations after fusion */
    int64_t passes;        /* full state-vector passes launched (each = 1 read + 1 write) */
    int64_t launches;      /* kernel launches */
    double bytes;          /* algorithmic HBM bytes of those launches */
    int64_t tile_sweeps;   /* shared-memory sweeps of the tiles in chunk passes, summed over
                              passes (a register phase is one sweep for all its ops) */
    int64_t tc_blocks;     /* dense blocks applied on the tensor cores (tcgen05), summed over
                              passes */
    int64_t tpb_gates;     /* gates built by the Tensor Product Booster (QS_OPT_NO_TPB) */
    double tc_flops;       /* floating-point operations of the tensor-core blocks: a k-qubit
                              block on n qubits is 2^(n+k+2) real multiply-adds per TF32
                              product, three products (hi x hi, hi x lo, lo x hi) */
} qs_stats;

/* ---- library ------------------------------------------------------------------ */

/* Thread-local message of the last failure on this thread ("" if none). */
const char *qs_last_error(void);
/* Number of kernel launches this library has issued in the process so far. */
uint64_t qs_launch_count(void);
/* ABI version (QS_ABI_VERSION) and the CUDA device count; no allocation. */
int qs_version(int32_t *abi, int32_t *device_count);

/* ---- state lifetime (Eq. 1) --------------------------------------------------- */

/* Allocates a 2^n_qubits-amplitude state of dtype dt on the current CUDA device and
 * sets it to |0...0> (a_0 = 1).  1 <= n_qubits <= QS_MAX_QUBITS.  The state gets its own
 * non-blocking CUDA stream.  QS_ERR_NOMEM if 2^n * bytes-per-amplitude does not fit. */
int qs_create(int n_qubits, qs_dtype dt, qs_state **out);
/* As qs_create, but over caller-owned device memory dev_ptr of `bytes` bytes (at least
 * 2^n * bytes-per-amplitude, 256-byte aligned), e.g. a PyTorch tensor, on the caller's
 * CUDA stream `stream` (cudaStream_t, may be NULL for the legacy stream).  The memory is
 * NOT initialised and NOT freed by qs_destroy. */
int qs_create_on(int n_qubits, qs_dtype dt, void *dev_ptr, uint64_t bytes, void *stream,
                 qs_state **out);
/* Waits for the state's stream and frees what the library allocated. */
int qs_destroy(qs_state *s);
/* Makes later launches of this state run on `stream` (cudaStream_t). */
int qs_set_stream(qs_state *s, void *stream);
/* Blocks until all work queued on the state's stream is done. */
int qs_synchronize(qs_state *s);
/* Sets the state to |0...0> (asynchronous on the state's stream). */
int qs_reset(qs_state *s);
/* Number of qubits, dtype and the device pointer of the amplitudes (for inspection). */
int qs_info(const qs_state *s, int32_t *n_qubits, int32_t *dtype, void **dev_ptr);

/* ---- gates (Eq. 2, Eq. 3, Sec. II-B, Sec. III) --------------------------------- */

/* Applies gates[0..n_gates-1] in order to the state.  The records are validated first
 * (QS_ERR_INVALID: unknown type, wrong nq, operand out of range or repeated, dense
 * matrix missing); nothing is applied if any record is invalid.  The call queues the
 * work on the state's stream and returns once it is queued (use qs_synchronize, or any
 * reading call, to wait).  Options: see qs_options. */
int qs_apply_circuit(qs_state *s, const qs_gate *gates, size_t n_gates, const qs_options *opt);
/* Statistics of the last qs_apply_circuit on s. */
int qs_last_stats(const qs_state *s, qs_stats *out);

/* Host-only dry run of the chunk planner of QS_MODE_AUTO (Sec. II-B "Qubit Reordering"
 * and "In-cache Operations"; Sec. III-A tier 4): no GPU is touched.  For an n-qubit state
 * of dtype dt, writes for each gate the index of the pass that executes it into
 * pass_of_gate[n_gates]; for each pass p < *n_passes (at most n_gates passes), its local
 * qubit mask into pass_lmask[p] (0 for a pass run by the streaming kernel).  Every qubit
 * of a gate is in its pass's mask, except that complex128 passes take a controlled phase
 * (CP, CZ, CU3 with theta = 0) with one of its qubits in the mask and the other outside
 * (a per-tile factor).  The caller allocates both arrays with n_gates entries.  Errors as
 * qs_apply_circuit. */
int qs_plan(int n_qubits, qs_dtype dt, const qs_gate *gates, size_t n_gates, const qs_options *opt,
            int32_t *pass_of_gate, uint64_t *pass_lmask, int64_t *n_passes);

/* ---- amplitudes and reductions -------------------------------------------------- */

/* Copies cnt amplitudes [off, off+cnt) from host memory (the state's dtype, interleaved)
 * into the state; synchronous.  QS_ERR_INVALID if the range exceeds 2^n.  Page-locked
 * host buffers (cudaHostAlloc / cudaHostRegister) of 4 MiB or more, 8-byte aligned, are
 * read by a copy kernel over the CPU-GPU link; other memory by cudaMemcpyAsync.  The
 * caller keeps ownership of host_src, which must hold cnt amplitudes. */
int qs_set_amplitudes(qs_state *s, uint64_t off, uint64_t cnt, const void *host_src);
/* Copies cnt amplitudes [off, off+cnt) of the state to host memory (state's dtype);
 * synchronous (waits for queued gates).  Same copy paths as qs_set_amplitudes. */
int qs_amplitudes(qs_state *s, uint64_t off, uint64_t cnt, void *host_dst);
/* Stream-ordered forms of the two copies above: enqueued on the state's stream after the
 * work queued so far, they return at once.  The caller keeps host_src (unchanged) and
 * host_dst (unread) alive until qs_synchronize(s) returns; a timeout of earlier queued
 * work is reported there.  Both use cudaMemcpyAsync on the copy engines, which need no
 * SMs, so they run under kernels of other streams: asynchronous for page-locked buffers;
 * for pageable memory the call waits as cudaMemcpyAsync does.  With two states on two
 * streams, the copies of one run under the gates of the other. */
int qs_set_amplitudes_async(qs_state *s, uint64_t off, uint64_t cnt, const void *host_src);
int qs_amplitudes_async(qs_state *s, uint64_t off, uint64_t cnt, void *host_dst);
/* Squared norm sum_i |a_i|^2, accumulated in FP64 in a fixed order (deterministic). */
int qs_norm(qs_state *s, double *out);
/* <Z_q> = sum_i |a_i|^2 (1 - 2 bit_q(i)) for q = 0..n-1 into out[0..n-1] (FP64, fixed
 * order, not divided by the norm); also the squared norm into *norm_out if non-NULL. */
int qs_expectation_z(qs_state *s, double *out, double *norm_out);
/* The k amplitudes with the largest |a_i|^2 (ties: lower index first), sorted; idx[k]
 * receives indices, amp[2k] the interleaved amplitudes as doubles.  k <= min(2^n, 4096). */
int qs_top_amplitudes(qs_state *s, uint32_t k, uint64_t *idx, double *amp);
/* Scales the state by 1/sqrt(norm) (norm computed in FP64); returns the old norm. */
int qs_renormalize(qs_state *s, double *old_norm);

/* Allocation-free <Z_q> and squared norm.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc, e.g. a host program that has handed all device
 * memory to its own pool allocator, or a latency-critical loop that cannot afford
 * cudaMalloc's implicit device synchronisation.  Same results as qs_expectation_z (FP64,
 * fixed summation order): bit for bit up to 30 qubits; at 31 and 32 qubits the state is
 * split into fewer, larger blocks, so the last bits may differ.
 *   dev_psi   device pointer to 2^n_qubits amplitudes of dtype dt (caller's memory,
 *             16-byte aligned), left unchanged;
 *   stream    cudaStream_t to run on (NULL: legacy default stream); the results are
 *             copied to the host, and the call returns once its stream has finished them;
 *   out_expz  host array of n_qubits doubles (or NULL), out_norm host double (or NULL).
 * Scratch: a file-scope device array of about 2.5 MB that every GPU loading this library
 * holds until process exit; nothing is allocated per call.  The first call on a device
 * does a one-time set-up: it looks up that array's device address (cudaGetSymbolAddress)
 * with that device current; make this first call before any stream capture begins.  The
 * address is kept for the life of the process: after a cudaDeviceReset of that device it
 * is stale, so do not call this entry point again in a process that has reset the device.
 * All calls share the one array and it keeps the last call's contents;
 * every value a call reads it has written itself, so nothing needs clearing, but calls
 * that overlap on the GPU (on different streams or host threads) race.
 * Errors: QS_ERR_INVALID for NULL pointers, an unknown dtype or n_qubits outside 1..32
 * (the scratch's limit); QS_ERR_CUDA if a launch or copy fails. */
int qs_expectation_z_noalloc(const void *dev_psi, int n_qubits, qs_dtype dt, void *stream,
                             double *out_expz, double *out_norm);

/* ---- serving: continuous batching of circuit requests -------------------------- */
/* The paper has no serving layer; this is the request loop around the operation of
 * Eq. 1-3.  Requests enter a FIFO queue; a worker thread admits the queue head when a
 * slot is free and the admitted states' bytes (2^n x bytes per amplitude) stay within
 * hbm_budget_bytes.  Every slot has its own CUDA stream, so admitted requests overlap on
 * the device.  A request runs its circuit (QS_MODE_* of `mode`, planned by default) from
 * |0...0> or from the caller's amplitudes, then returns <Z_q> for every qubit, the squared
 * norm and its top_k amplitudes.  Results are bitwise identical whatever else runs.
 * Large requests are admitted in submission order.  Small requests (small_max_qubits) may
 * overtake them: they take a free small slot, else a free regular one, as soon as the
 * budget allows, so a burst of large states does not hold them back.  Their streams have
 * the device's highest priority.  Slots only overlap on the device if their streams get
 * hardware queues of their own: set CUDA_DEVICE_MAX_CONNECTIONS (default 8, at most 32)
 * to at least the number of slots before the process first uses CUDA. */

typedef struct {
    uint64_t hbm_budget_bytes;  /* admission budget for the states in flight */
    int32_t max_slots;          /* requests in flight at once (1..256) */
    int32_t small_slots;        /* extra slots that only small requests use (0..256; 0: none);
                                   their buffers are sized at creation for small_max_qubits,
                                   so serving a small request frees no memory (cudaFree waits
                                   for the whole device) */
    int32_t small_max_qubits;   /* a request of at most this many qubits is small */
    int32_t reserved[3];
} qs_server_config;

/* Bits of qs_request.flags. */
enum {
    QS_REQ_BORROW_INIT = 1  /* init_amplitudes is not copied at submission: the caller keeps
                               the buffer alive and unchanged until qs_poll has returned QS_OK
                               (or an error) for the ticket, and the request's stream copies
                               straight from it when the request starts.  Several requests may
                               borrow one buffer.  A page-locked buffer (cudaHostAlloc,
                               cudaHostRegister) keeps that copy asynchronous on the copy
                               engines; pageable memory makes the worker wait for it. */
};

typedef struct {
    int32_t n_qubits;
    int32_t dtype;                 /* QS_C64 or QS_C128 */
    const qs_gate *gates;          /* copied by qs_submit */
    uint64_t n_gates;
    const void *init_amplitudes;   /* 2^n amplitudes of dtype (copied unless borrowed, see
                                      QS_REQ_BORROW_INIT), or NULL for |0...0> */
    uint32_t top_k;                /* amplitudes to return, <= min(2^n, 4096) */
    int32_t mode;                  /* QS_MODE_* for the circuit */
    int32_t precision;             /* QS_PREC_* for complex128 requests */
    uint32_t flags;                /* QS_REQ_* bits (0: copy init_amplitudes at submission) */
} qs_request;

typedef struct {
    int64_t submitted, completed, failed, queued, in_flight;
    uint64_t bytes_in_use, peak_bytes;
} qs_server_stats_t;

/* Creates the server on the current CUDA device and starts its worker thread. */
int qs_server_create(const qs_server_config *cfg, qs_server **out);
/* Queues a request and returns its ticket.  QS_ERR_NOMEM only if the request can never
 * fit the budget; QS_ERR_INVALID for bad records (nothing is queued). */
int qs_submit(qs_server *sv, const qs_request *req, uint64_t *ticket);
/* QS_NOT_READY while the request runs; QS_OK once done, copying <Z_q> (n doubles),
 * the squared norm, top_k indices and 2*top_k doubles (interleaved amplitudes) and the
 * latency from submission to completion in seconds (any pointer may be NULL).  A ticket
 * is returned once; afterwards (or never issued) it is QS_ERR_INVALID. */
int qs_poll(qs_server *sv, uint64_t ticket, double *expz, double *norm, uint64_t *top_idx,
            double *top_amp, double *latency_s);
int qs_server_stats(qs_server *sv, qs_server_stats_t *out);
/* Waits until every submitted request has completed; QS_ERR_TIMEOUT after timeout_s. */
int qs_server_drain(qs_server *sv, double timeout_s);
/* QS_ERR_BUSY while requests are queued or in flight. */
int qs_server_destroy(qs_server *sv);

/* ---- batched execution: many small circuits in one persistent launch ------------ */

typedef struct qs_batch qs_batch;  /* opaque */

/* One circuit of a batch: its qubit count and its gate records (copied at creation). */
typedef struct {
    int32_t n_qubits;
    int32_t reserved;
    const qs_gate *gates;
    uint64_t n_gates;
} qs_circuit;

typedef struct {
    int64_t circuits;
    int64_t passes;       /* tile passes over all circuits */
    int64_t work_items;   /* tiles handed out by the persistent kernel per run */
    int64_t grid;         /* persistent CTAs */
    uint64_t state_bytes; /* device bytes of all states together */
} qs_batch_stats;

/* Plans every circuit (gate semantics of Eq. 2 / Eq. 3; passes and fusion as in
 * qs_apply_circuit, Sec. II-B / III-A), lays all states out in one device arena (every
 * circuit starts from |0...0>), uploads every table and captures one CUDA graph holding a
 * single persistent kernel launch.  All circuits share dtype dt.  Options: chunk_m (tile
 * width), fuse_k (fusion width inside a pass); reserved[0] = wait limit of the kernel's
 * dependency waits in microseconds (0: 2 s); reserved[1] = 1 is a test hook that makes one
 * dependency unsatisfiable, so that a run ends with QS_ERR_TIMEOUT instead of hanging.
 * QS_ERR_UNSUPPORTED for dense blocks wider than 4 qubits. */
int qs_batch_create(const qs_circuit *circuits, size_t count, qs_dtype dt, const qs_options *opt,
                    qs_batch **out);
/* Replays the graph (all circuits from |0...0>) on the batch's stream; asynchronous. */
int qs_batch_run(qs_batch *b);
/* Waits for the batch's stream; QS_ERR_TIMEOUT if a bounded device wait gave up. */
int qs_batch_synchronize(qs_batch *b);
/* Makes later runs use `stream` (cudaStream_t). */
int qs_batch_set_stream(qs_batch *b, void *stream);
/* Copies amplitudes [off, off+cnt) of circuit i (batch dtype, interleaved) to host memory. */
int qs_batch_amplitudes(qs_batch *b, uint64_t i, uint64_t off, uint64_t cnt, void *host_dst);
int qs_batch_info(const qs_batch *b, qs_batch_stats *out);
int qs_batch_destroy(qs_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_QS_H_ */
