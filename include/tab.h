/*
 * tab.h -- C ABI of libtab: a GB300 (sm_103a) stabilizer-tableau simulator.
 *
 * The operation is the Clifford-circuit backend of Qibo 0.2.9 (arXiv:2408.00384,
 * section "Simulation of Clifford circuits"), which is built on the phase-space
 * (stabilizer tableau) formalism of Aaronson & Gottesman, PRA 70, 052328 (2004),
 * Sec. III: an n-qubit state is held as n destabilizer and n stabilizer rows of
 * X|Z bits plus a sign bit; a Clifford gate updates one or two bit columns of
 * every row; a Z measurement either draws a random outcome (pivot row, then
 * rowsum of the pivot into every row that anticommutes with Z_a) or reads a
 * deterministic one (product of stabilizer rows selected by the destabilizers).
 *
 * Conventions shared by every call:
 *  - Return value: TAB_OK (0) on success, a negative tab_status on error; the
 *    message of the last error on the calling thread is tab_last_error().
 *  - Qubit indices are 0-based.  A tableau has 2n rows: rows 0..n-1 are the
 *    destabilizers, rows n..2n-1 the stabilizers; row i is the Pauli
 *    (-1)^r_i (x)_j P(x_ij, z_ij) with P(0,0)=I, P(1,0)=X, P(1,1)=Y, P(0,1)=Z.
 *  - Host buffers passed in are borrowed for the duration of the call only.
 *    Device memory belongs to the handle, except with tab_create_on, where the
 *    caller owns it and must keep it alive until tab_destroy.
 *  - Work is enqueued on the handle's CUDA stream (default: the legacy default
 *    stream) and runs asynchronously unless a call says it synchronizes.
 *    Device-side errors (a wait that timed out, a phase-parity violation) are
 *    latched on the device and reported by the next synchronizing call as
 *    TAB_ETIMEOUT / TAB_EDEVICE.
 *  - Random outcomes: the k-th measurement op (k counted from 0 over every
 *    MZ/MZR of the handle since tab_set_rng, deterministic ones included) of
 *    (circuit_id, shot) uses bit 0 of word 0 of Philox4x32-10 (Salmon et al.,
 *    SC'11) with counter (k, shot, circuit_id lo, circuit_id hi) and key
 *    (seed lo, seed hi).  The bit is used only when the outcome is random.
 *  - Pivot choice: the smallest stabilizer row with x_pa = 1.  These two
 *    choices make every outcome and every tableau bit reproducible.
 */
#ifndef TAB_H_
#define TAB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tab_s *tab_t;

/* Gate word: bits 63..56 op, 55..28 first qubit, 27..0 second qubit (0 for
 * one-qubit ops).  A gate list is in program order.  The library may reorder
 * gates that act on disjoint qubits (they commute), which never changes a
 * result.  TAB_BARRIER is a hint with no effect on results. */
typedef uint64_t tab_gate;

enum tab_op {
  TAB_I = 0, TAB_X = 1, TAB_Y = 2, TAB_Z = 3, TAB_H = 4, TAB_S = 5, TAB_SDG = 6,
  TAB_CNOT = 7, /* first qubit is the control */
  TAB_CZ = 8, TAB_SWAP = 9,
  TAB_MZ = 10,  /* measure Z; outcome appended to the handle's outcome log */
  TAB_MZR = 11, /* measure Z, then apply X when the outcome is 1 (reset to |0>) */
  TAB_BARRIER = 12,
  /* Extended ops, accepted by tab_apply, batches and the server, and (all
   * but the noise ops) by tab_prog_create.  MX / MY are lowered to the ops
   * above on the host; noise ops are drawn per shot (below). */
  TAB_MX = 13,     /* measure X: H, TAB_MZ, H (outcome logged like TAB_MZ) */
  TAB_MY = 14,     /* measure Y: S^dag, H, TAB_MZ, H, S */
  TAB_DEPOL1 = 15, /* depolarizing noise on q1: X, Y or Z with total probability p */
  TAB_XERR = 16,   /* X on q1 with probability p */
  TAB_ZERR = 17    /* Z on q1 with probability p */
};

/* Noise ops carry p in the second-qubit field as a 28-bit fraction (p = field
 * / 2^28).  Noise op j -- counted per handle from 0 after tab_set_rng or
 * tab_reset, in program order -- draws r = Philox4x32-10 with counter
 * (j, shot, circuit_id lo, circuit_id hi) and key (seed lo, seed hi XOR
 * 0x4E4F4953).  It fires when (r.x >> 4) < field; TAB_DEPOL1 then applies
 * X, Y or Z for floor(r.y * 3 / 2^32) = 0, 1 or 2.  The noise of a circuit
 * does not depend on its state, so tab_apply and the server take the draws on
 * the host when they compile the list (a fired noise op costs one Pauli gate,
 * an unfired one nothing; the server compiles each shot of a noisy request
 * apart), while a batch keeps its noise ops and every shot draws its own on
 * the device (the counter starts at 0 in every shot, and the gates a batch
 * runs once for all shots end at the circuit's first measurement or noise
 * op).  At most 16,383 noise ops per batch circuit. */

enum tab_status {
  TAB_OK = 0,
  TAB_EINVAL = -1,   /* malformed argument (unknown op, q1 == q2, null pointer) */
  TAB_ERANGE = -2,   /* qubit index >= n, or n outside [1, TAB_MAX_QUBITS] */
  TAB_ENOMEM = -3,   /* device or host allocation failed, or caller memory too small */
  TAB_ECUDA = -4,    /* a CUDA runtime call failed */
  TAB_EDEVICE = -5,  /* a kernel reported an internal inconsistency */
  TAB_ETIMEOUT = -6, /* a device-side wait exceeded its limit; the handle is unusable */
  TAB_ESTATE = -7    /* call not valid in the handle's state (e.g. capacity exceeded) */
};

#define TAB_MAX_QUBITS 16384
#define TAB_BATCH_MAX_QUBITS 640 /* largest n of the single-CTA engine */

static inline tab_gate tab_make_gate(uint32_t op, uint32_t q1, uint32_t q2) {
  return ((uint64_t)op << 56) | ((uint64_t)(q1 & 0xFFFFFFFu) << 28) | (uint64_t)(q2 & 0xFFFFFFFu);
}

/* ---- handles (Aaronson-Gottesman Sec. III: the tableau) ------------------ */

/* Bytes of device memory tab_create_on needs for n qubits (tableau planes plus
 * the handle's measurement workspace).  0 if n is out of range. */
size_t tab_bytes_required(int32_t n);

/* Allocate a tableau for n qubits (1 <= n <= TAB_MAX_QUBITS) in |0^n>
 * (destabilizer i = +X_i, stabilizer i = +Z_i).  *out receives the handle.
 * TAB_ERANGE for bad n, TAB_ENOMEM if device memory runs out. */
int tab_create(int32_t n, tab_t *out);

/* As tab_create, but the tableau and workspace live in caller-owned device
 * memory dev_ptr of at least tab_bytes_required(n) bytes, 256-byte aligned
 * (e.g. a torch uint8 CUDA tensor).  cuda_stream (a cudaStream_t, may be NULL)
 * becomes the handle's stream.  The memory must outlive the handle. */
int tab_create_on(int32_t n, void *dev_ptr, size_t bytes, void *cuda_stream, tab_t *out);

/* Release the handle (and its device memory unless caller-owned).  Waits for
 * the handle's pending work.  NULL is accepted. */
int tab_destroy(tab_t h);

int tab_num_qubits(tab_t h, int32_t *n);

/* Bind the handle to a CUDA stream (cudaStream_t; NULL = default stream).
 * Later work is enqueued there; earlier work is not moved.  When the stream
 * changes, the call first waits for the work already enqueued on the
 * previous one (TAB_ECUDA if that work failed). */
int tab_set_stream(tab_t h, void *cuda_stream);

/* Set (seed, circuit_id, shot) of the outcome stream and reset the
 * measurement counter k to 0.  Defaults: seed 1, circuit 0, shot 0. */
int tab_set_rng(tab_t h, uint64_t seed, uint64_t circuit_id, uint32_t shot);

/* Put the tableau back to |0^n> (Sec. III initial tableau); clears the
 * outcome log; keeps the RNG settings but resets k to 0.  Asynchronous. */
int tab_reset(tab_t h);

/* Host only (no device work): the base-op list that tab_apply runs for a list
 * holding extended ops, under RNG context (seed, circuit_id, shot) and noise
 * counter *noise_counter (advanced; NULL: noise ops are TAB_EINVAL).  MX / MY
 * become Z measurements between basis changes; a run of consecutive
 * measurement ops on distinct qubits shares one block of pre-rotations and
 * one of post-rotations (the same tableau as op by op).  *out_count is the
 * number of words; TAB_ENOMEM (nothing written) when it exceeds out_cap. */
int tab_lower_ops(int32_t n, const tab_gate *gates, int64_t count, uint64_t seed,
                  uint64_t circuit_id, uint32_t shot, uint64_t *noise_counter, tab_gate *out,
                  int64_t out_cap, int64_t *out_count);

/* ---- gates and measurements --------------------------------------------- */

/* Apply `count` gate words (host memory, program order, TAB_MZ/TAB_MZR
 * allowed) to the tableau.  Every qubit index is validated on the host before
 * anything is launched (TAB_ERANGE / TAB_EINVAL: nothing is applied).  Gates
 * are the column updates of AG Sec. III (CNOT, H, S) and their products;
 * measurements are AG's two cases, their outcomes appended to the handle's
 * outcome log (tab_read_outcomes).  Asynchronous: the host list is copied
 * before the call returns. */
int tab_apply(tab_t h, const tab_gate *gates, int64_t count);

/* Expectation values <psi|P_i|psi> of k Pauli strings on the handle's
 * stabilizer state (AG Sec. III: +-P is in the stabilizer group exactly when
 * P commutes with every stabilizer row, and then it is the product of the
 * stabilizer rows whose destabilizer partners anticommute with P).
 * `paulis`: k x n host bytes, row-major; entry j of string i is the Pauli on
 * qubit j: 0 = I, 1 = X, 2 = Z, 3 = Y (bit 0 = x, bit 1 = z).  `out`: k host
 * bytes, each -1, 0 or +1.  The state is not changed and no measurement index
 * is used.  Synchronous.  TAB_EINVAL on a code above 3 or a null pointer
 * (nothing launched); TAB_EDEVICE if a product fails its consistency checks. */
int tab_expect(tab_t h, const uint8_t *paulis, int32_t k, int8_t *out);

/* State vector of the handle's state, for n <= TAB_SV_MAX_QUBITS.
 * `amps`: host array of at least 2^(n+1) floats, filled with the 2^n complex
 * amplitudes as (re, im) pairs; basis index bit q is qubit q.  The global
 * phase is fixed so that the nonzero amplitude of smallest index is real and
 * positive.  Computed on the device as prod_i (I + S_i)/2 |b> over the
 * stabilizer rows S_i, normalised, with b a basis state in the support (the Z
 * outcomes of a copy of the tableau).  The handle's state, outcome log and
 * counters are unchanged.  Synchronous.  TAB_ERANGE if n is above the limit,
 * TAB_EINVAL if `amps` is null or too short. */
#define TAB_SV_MAX_QUBITS 26
int tab_statevector(tab_t h, float *amps, int64_t len);

/* ---- one tableau split by rows over shards ---------------------------------- */

/* A tableau whose qubit-row indices are split over `shards` shards (shard s
 * holds destabilizer i and stabilizer n+i for its range of i, every column;
 * 1 <= shards <= ceil(n/32)), each driven by its own host thread.  Gates need
 * no exchange (AG Sec. III: rows are independent).  A Z measurement
 * exchanges, between launches: the minimum of the shards' pivot candidates;
 * in the random case the pivot row (2n bits and a sign), broadcast by its
 * owner; in the deterministic case the shards' partial products of selected
 * stabilizer rows, gathered on shard 0 and multiplied in shard order; then
 * the outcome.  Results are identical to a single tableau's (same Philox
 * outcome stream).  The handle owns its device memory; calls on one handle
 * are not concurrent-safe. */
typedef struct tab_shard_s *tab_shard_t;
int tab_sharded_create(int32_t n, int32_t shards, tab_shard_t *out);
int tab_sharded_destroy(tab_shard_t h);
/* as tab_set_rng: (seed, circuit_id, shot) of the outcome stream, counter k = 0 */
int tab_sharded_set_rng(tab_shard_t h, uint64_t seed, uint64_t circuit_id, uint32_t shot);
/* as tab_apply, synchronous; base ops only (the extended ops are TAB_EINVAL) */
int tab_sharded_apply(tab_shard_t h, const tab_gate *gates, int64_t count);
int tab_sharded_read_outcomes(tab_shard_t h, uint8_t *out, int64_t max, int64_t *count);
/* as tab_export: rows 0..2n-1 unpacked, gathered from the shards */
int tab_sharded_export(tab_shard_t h, uint8_t *x, uint8_t *z, uint8_t *r);

/* A gate list compiled once (validated, grouped into layers of disjoint gates,
 * uploaded to device memory) and replayable on any handle with the same n. */
typedef struct tab_prog_s *tab_prog_t;

int tab_prog_create(int32_t n, const tab_gate *gates, int64_t count, tab_prog_t *out);
int tab_prog_destroy(tab_prog_t p);
/* number of gate ops, measurement ops and gate layers in the program */
int tab_prog_info(tab_prog_t p, int64_t *n_gates, int64_t *n_meas, int64_t *n_layers);
/* Run a compiled program on the handle (asynchronous; nothing is copied from
 * the host).  TAB_EINVAL if the program's n differs from the handle's. */
int tab_run(tab_t h, tab_prog_t p);

/* Measure Z on k qubits in the given order (AG Sec. III), with `seed` as the
 * Philox key for this call (circuit_id, shot and k continue from the handle).
 * Synchronizes; out_bits[i] receives outcome i as 0 or 1.  Outcomes are also
 * appended to the outcome log. */
int tab_measure(tab_t h, const int32_t *qubits, int32_t k, uint64_t seed, uint8_t *out_bits);

/* As tab_measure with the handle's seed, without synchronizing: outcome i is
 * written, as one byte, to dev_out_bits[i] (device memory, >= k bytes, kept
 * alive by the caller until the stream reaches this point). */
int tab_measure_async(tab_t h, const int32_t *qubits, int32_t k, uint8_t *dev_out_bits);

/* Measurement that allocates no device memory.  (The paper has no
 * counterpart: this is a deployment variant of tab_measure_async.)
 *
 * tab_create, tab_measure and tab_measure_async all allocate device memory.
 * Some callers cannot: a process whose device memory is owned by another
 * allocator (a framework that reserved the whole heap up front, where
 * cudaMalloc fails or fragments its pool), or a latency-critical loop that
 * must not pay for, or synchronize on, an allocation after start-up.  With a
 * tableau in caller-owned memory (tab_create_on), this call lets them measure
 * with no allocation at all.
 *
 * Measures Z on the k host-listed qubits in order (MZR when reset != 0),
 * exactly as tab_measure_async does (same outcomes and tableau, same
 * outcome-stream counter, which advances by k), writing outcome i as one byte
 * to dev_out_bits[i] (caller-owned device memory, >= k bytes).  The outcomes
 * are not added to the handle's outcome log.  Asynchronous on the handle's
 * stream; device errors surface at the next synchronizing call.  The host
 * qubit list is read only during the call: the qubit codes travel to the
 * device as kernel parameters, with no host buffer and no host-to-device copy.
 *
 * Scratch: a file-scope device array of TAB_NOALLOC_SCRATCH_BYTES (1 MiB) per
 * device, held by every process that loads the library until it exits.  A
 * call uses at most k + (2G + 2)W + 2G + 128 of its 32-bit words (W = 2 * the handle's
 * words per half-column, G = CTAs of the measurement launch, lowered as far
 * as 1 to fit); TAB_ERANGE if it does not fit with G = 1.  Every call shares
 * the array: calls whose GPU work may overlap (different streams) race, so
 * serialise them on one stream.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with the handle's device
 * current); make that first call before any stream capture.  TAB_EINVAL if
 * the handle's device is not current, TAB_ERANGE for a bad qubit (nothing is
 * launched). */
#define TAB_NOALLOC_SCRATCH_BYTES (1u << 20)
int tab_measure_noalloc(tab_t h, const int32_t *qubits, int32_t k, int32_t reset,
                        uint8_t *dev_out_bits);

/* Synchronize and copy the outcome log (every outcome since the last
 * tab_reset / tab_clear_outcomes, in program order, one byte each) into out
 * (capacity max).  *count receives the number of outcomes in the log. */
int tab_read_outcomes(tab_t h, uint8_t *out, int64_t max, int64_t *count);
int tab_clear_outcomes(tab_t h);

/* Execution engine for tab_apply / tab_run / tab_measure on this handle.
 * TAB_ENGINE_SINGLE_CTA keeps the whole tableau in one CTA's shared memory
 * (n <= TAB_BATCH_MAX_QUBITS; one launch per call).  The other engines apply
 * gate runs with the block gate kernel (one CTA per 32-row word of the
 * tableau) and differ in how a run of measurements executes:
 *   TAB_ENGINE_GRID     tableau in the shared memory of a cooperative grid
 *                       of one CTA per SM (n up to about 7,900), else
 *                       streamed from HBM/L2;
 *   TAB_ENGINE_STREAM   always streamed from HBM/L2 by a cooperative grid.
 * TAB_ENGINE_AUTO (default) picks by size: single-CTA for n <= 256, else
 * grid-resident where it fits, else streaming.  Results are bit-identical
 * across engines.  TAB_ERANGE if SINGLE_CTA is asked for
 * n > TAB_BATCH_MAX_QUBITS; TAB_EINVAL for any other value (3 is unused). */
enum tab_engine {
  TAB_ENGINE_AUTO = 0, TAB_ENGINE_SINGLE_CTA = 1, TAB_ENGINE_GRID = 2, TAB_ENGINE_STREAM = 4
};
int tab_set_engine(tab_t h, int engine);

/* The engine a run of Z measurements takes on this handle under its selected
 * engine and size (TAB_ENGINE_SINGLE_CTA, _GRID or _STREAM; never
 * _AUTO) in *engine, and the CTAs it launches in *ctas.  GRID falls back to
 * STREAM for a tableau that no cooperative grid holds in shared memory; this
 * call shows which one runs.  No device work.  TAB_EINVAL on null pointers. */
int tab_engine_resolved(tab_t h, int* engine, int* ctas);

/* Bytes this handle has copied host -> device (compiled programs, imports)
 * and device -> host (outcomes, exports) for its callers since creation.
 * Either pointer may be null.  No device work. */
int tab_transfer_bytes(tab_t h, int64_t* h2d, int64_t* d2h);

/* Number of CUDA kernels this handle has launched since creation. */
int tab_kernel_launches(tab_t h, int64_t *count);

/* Work counters of the streaming measurement engine, for stating a run's
 * algorithmic bytes exactly (the work model of AG Sec. III's measurement:
 * a random outcome's rowsum touches the columns where the pivot row p is not
 * I -- its support -- and a deterministic outcome multiplies the stabilizer
 * rows n+i with x_ia = 1).  The paper has no counterpart.  tab_count_work(h,
 * 1) zeroes the counters and starts counting on h's later streaming-engine
 * runs (one atomic add per CTA and measurement); 0 stops it.  Other engines
 * leave the counters alone.  tab_work_counts synchronizes h's stream and
 * writes counts[0] = the support columns summed over random-outcome
 * measurements, counts[1] = the rows multiplied summed over deterministic
 * ones, counts[2] / counts[3] = the random / deterministic measurements
 * counted (all 0 if counting never started).  TAB_ENOMEM when the 32-byte
 * counter buffer cannot be allocated. */
int tab_count_work(tab_t h, int32_t on);
int tab_work_counts(tab_t h, int64_t *counts);

/* ---- state transfer (checkpoint / oracle comparison) --------------------- */

/* Synchronize and unpack the tableau into row-major host arrays: x and z of
 * 2n*n bytes (row i, qubit j at [i*n + j]), r of 2n bytes; values 0/1. */
int tab_export(tab_t h, uint8_t *x, uint8_t *z, uint8_t *r);

/* Load a tableau from the same layout (values are taken mod 2) and set the
 * measurement counter k.  The rows must form a valid tableau (symplectic);
 * this is not checked.  Synchronizes. */
int tab_import(tab_t h, const uint8_t *x, const uint8_t *z, const uint8_t *r,
               uint64_t meas_counter);

/* Wait for the handle's work; returns latched device errors. */
int tab_sync(tab_t h);

/* Message of the last error on this thread ("" if none). */
const char *tab_last_error(void);

/* ---- batched runs: many independent circuits and shots, one launch ------- */

typedef struct {
  int32_t n;              /* qubits, 1..TAB_BATCH_MAX_QUBITS */
  const tab_gate *gates;  /* host gate list, program order */
  int64_t n_gates;        /* number of gate words */
  int32_t shots;          /* >= 1 independent runs from |0^n> */
  uint64_t circuit_id;    /* Philox counter words 2..3 */
} tab_circuit;

/* Run m circuits, each for its number of shots, with Philox key `seed`.
 * Outcomes of (circuit c, shot s) go, in program order, to
 * out_bits[out_offsets[c] + s * n_meas(c) ...] where n_meas(c) counts the
 * MZ, MZR, MX and MY ops of circuit c (tab_meas_counts); out_offsets may be
 * NULL, meaning circuits are packed back to back in order.  All shots of a
 * circuit share the gates before its first measurement (gates do not depend
 * on outcomes).  Large lists are cut into chunks (tab_config.batch_chunks)
 * that the host compiles while the device runs the chunk before; with
 * packed output in pinned host memory each chunk's outcomes are copied back
 * behind its launch.  Uses the current CUDA device and streams of its own;
 * synchronizes before returning.  The outcomes do not depend on the
 * chunking. */
int tab_batch_run(const tab_circuit *circuits, int32_t m, uint64_t seed,
                  uint8_t *out_bits, const int64_t *out_offsets);
/* tab_batch_run with packed output into a caller buffer of out_capacity
 * bytes, without counting the outcomes first: counts (NULL: not wanted)
 * receives n_meas(c) of every circuit as the chunks are compiled.
 * TAB_ERANGE when the outcomes would pass out_capacity; the chunks launched
 * before that point have written their bytes (all within the buffer) and
 * nothing is written past it.  TAB_EINVAL for out_capacity < 0. */
int tab_batch_run_packed(const tab_circuit *circuits, int32_t m, uint64_t seed,
                         uint8_t *out_bits, int64_t out_capacity, int64_t *counts);

/* A batch compiled once (gate lists validated, layered, uploaded, work items
 * sorted by cost) and replayable with tab_batch_exec; replays are captured in
 * a CUDA graph on first use. */
typedef struct tab_batch_s *tab_batch_t;

int tab_batch_create(const tab_circuit *circuits, int32_t m, tab_batch_t *out);
/* tab_batch_create with options.  TAB_BATCH_SAMPLE_TERMINAL: a circuit whose
 * measurements all come after its gates (Z without reset) runs them once,
 * with every sign kept as an affine form over the run's random outcome bits,
 * and every shot is then evaluated from its own Philox bits -- the same
 * outcome bits as running each shot (the "shot sampler"; see
 * tab_batch_sampled for how many circuits qualified).  Other circuits run
 * per shot as usual.  TAB_EINVAL on unknown flags. */
enum { TAB_BATCH_SAMPLE_TERMINAL = 1 };
int tab_batch_create_ex(const tab_circuit *circuits, int32_t m, uint32_t flags,
                        tab_batch_t *out);
/* Circuits of the batch that run through the terminal-measurement sampler. */
int tab_batch_sampled(tab_batch_t b, int32_t *circuits);
int tab_batch_destroy(tab_batch_t b);
/* totals: gate ops (once per circuit), measurement ops (over all shots),
 * outcome bytes needed */
int tab_batch_info(tab_batch_t b, int64_t *n_gates, int64_t *n_meas, int64_t *out_bytes);
/* n_meas(c) of every circuit: counts[c] for c < m (the caller's array). */
int tab_batch_meas_counts(tab_batch_t b, int64_t *counts);
/* n_meas(c) of m host gate lists (MZ, MZR, MX, MY words), counted on the
 * host's worker threads without compiling anything: the sizes tab_batch_run
 * writes.  TAB_EINVAL on a null array. */
int tab_meas_counts(const tab_circuit *circuits, int32_t m, int64_t *counts);
/* Enqueue one run of the whole batch on cuda_stream: outcomes (packed back to
 * back per circuit and shot) go to dev_out (device memory, >= out_bytes). */
int tab_batch_exec(tab_batch_t b, uint64_t seed, uint8_t *dev_out, void *cuda_stream);
/* Bytes of compiled tables (circuit descriptors, segments, gate codes, layer
 * offsets, work items) the batch copied host -> device when it was created;
 * tab_batch_run copies the same amount per call. */
int tab_batch_h2d_bytes(tab_batch_t b, int64_t *bytes);
/* Size classes.  The batch's circuits are grouped by qubit count into size
 * classes -- runs of 32-qubit groups (one tableau word per 32 qubits) whose
 * tableaus take the same number of CTAs per SM -- and each class runs as a
 * persistent launch of its own, shaped for it (threads per CTA, shared
 * memory for its largest tableau, as many CTAs as fit); tab_batch_exec
 * launches the classes in one CUDA graph, the largest qubit counts first,
 * each class's launch starting once every CTA of the one before is running
 * (its CTAs then take SMs as the earlier classes finish).  tab_batch_classes: their number; tab_batch_class:
 * class k's range and shape. */
typedef struct {
  int32_t lo_n, max_n;   /* qubit counts of the class: lo_n .. max_n */
  int32_t threads, ctas; /* launch shape */
  int64_t smem_bytes;    /* dynamic shared memory per CTA */
  int64_t items;         /* work items (prefix and shot items) */
} tab_batch_class_info;
int tab_batch_classes(tab_batch_t b, int32_t *count);
int tab_batch_class(tab_batch_t b, int32_t k, tab_batch_class_info *out);
/* Number of kernels one tab_batch_exec launches (one per non-empty class). */
int tab_batch_launches(tab_batch_t b, int64_t *count);
/* Work counters of the batched kernel (as tab_count_work, for stating a
 * run's algorithmic work exactly; the paper has no counterpart).
 * tab_batch_count_work(b, 1) zeroes them and makes b's later execs count:
 * those launch the kernel's counting instances (one atomic add per
 * measurement) one size class after another, outside the batch's graph,
 * and the timed instances carry no counting code; 0 stops it.
 * tab_batch_work_counts, once those runs have finished, writes counts[0] =
 * the random-outcome measurements' pivot-row supports, each times its
 * tableau's 32-row words per column (2 ceil(n/32)), summed over every
 * (circuit, shot); counts[1] = the rows the deterministic outcomes multiply,
 * times the same words per column; counts[2] / counts[3] = the random /
 * deterministic measurements (all 0 if counting never started). */
int tab_batch_count_work(tab_batch_t b, int32_t on);
int tab_batch_work_counts(tab_batch_t b, int64_t *counts);
/* Autotuner: runs each size class's launch alone once per CTA size the
 * persistent kernel is built for (128, 256, 512 or 1024 threads per CTA;
 * shared memory sized to the class's largest tableau; as many CTAs as fit on
 * the GPU), timed with events on cuda_stream, and keeps the fastest per
 * class for later tab_batch_exec replays.  Each run writes the outcomes an
 * exec with this seed writes for that class (dev_out as for tab_batch_exec).
 * Synchronises cuda_stream.  *threads_out gets the first (largest-qubit)
 * class's choice and *best_ms_out the sum of the classes' best times (either
 * may be null).  TAB_EDEVICE / TAB_ETIMEOUT if a run reports a device
 * error. */
int tab_batch_tune(tab_batch_t b, uint64_t seed, uint8_t *dev_out, void *cuda_stream,
                   int32_t *threads_out, float *best_ms_out);
/* Launch shape of the first (largest-qubit) size class. */
int tab_batch_config(tab_batch_t b, int32_t *threads, int32_t *ctas, int64_t *smem_bytes);

/* ---- serving: continuous batching of circuit requests -------------------- */

/* A request server keeps many tableaus resident on the device at once.  A
 * submitted circuit waits in a FIFO until a slot is free and its tableau fits
 * the memory budget; it is then compiled and its whole program (gate runs,
 * mid-circuit measurement runs, outcome copy) is enqueued on one of the
 * server's streams, overlapping with other requests.  When it completes, its
 * slot and memory go to the next waiting request.  Outcomes of a request
 * depend only on its own circuit, circuit_id and shots (Philox key = the
 * server's seed), never on the mix it ran in.  A worker thread owns the
 * device work; the calls below are thread-safe. */
typedef struct tab_server_s *tab_server_t;

typedef struct {
  uint64_t mem_budget_bytes;  /* device bytes for resident tableaus (admission cap) */
  int32_t max_inflight;       /* requests on the device at once (>= 1) */
  int32_t n_streams;          /* CUDA streams the requests are spread over (>= 1) */
  int32_t meas_ctas;          /* CTAs per grid-engine measurement launch; 0 = default */
  double request_timeout_s;   /* fail a running request not completed by then; 0 = none */
  uint64_t seed;              /* Philox key of every request */
  int32_t max_grid_inflight;  /* requests with n > TAB_BATCH_MAX_QUBITS (which spread over
                                 many SMs) on the device at once; 0 = 1.  Smaller requests
                                 run on one SM each and fill the rest of the GPU. */
} tab_server_config;

enum tab_req_state { TAB_REQ_PENDING = 0, TAB_REQ_RUNNING = 1, TAB_REQ_DONE = 2, TAB_REQ_FAILED = 3 };

/* Host-side fault injection for tests: drop the completion of a request, so
 * that it fails with TAB_ETIMEOUT at its deadline and its slot is reclaimed. */
enum tab_fault { TAB_FAULT_DROP_COMPLETION = 1 };

typedef struct {
  int64_t submitted, completed, failed, rejected;
  int64_t inflight, queued, peak_inflight;
  uint64_t mem_used, peak_mem;
} tab_server_stats;

int tab_server_create(const tab_server_config *cfg, tab_server_t *out);
/* Validate and enqueue a request (gates are copied).  Invalid gates are
 * refused here (TAB_ERANGE / TAB_EINVAL) and never reach the device.
 * *ticket identifies the request. */
int tab_server_submit(tab_server_t s, const tab_circuit *c, int64_t *ticket);
/* Current tab_req_state of a request. */
int tab_server_query(tab_server_t s, int64_t ticket, int *state);
/* Wait (timeout_s < 0: forever) for a request; copy up to cap outcome bytes
 * (shot 0's outcomes, then shot 1's, ...) to out, set *count to the total
 * and *latency_s to submit-to-completion seconds, and forget the ticket.
 * Returns the request's status: TAB_OK, TAB_ENOMEM (larger than the whole
 * budget), TAB_ETIMEOUT (deadline passed), or TAB_ESTATE if timeout_s
 * passed first (the ticket stays valid). */
int tab_server_wait(tab_server_t s, int64_t ticket, double timeout_s, uint8_t *out, int64_t cap,
                    int64_t *count, double *latency_s);
int tab_server_inject(tab_server_t s, int64_t ticket, int kind);
int tab_server_stats_get(tab_server_t s, tab_server_stats *out);
/* Finish every submitted request, then stop the worker and free the server. */
int tab_server_destroy(tab_server_t s);

/* ---- autotuner of the plain path --------------------------------------
 * The paper has no counterpart.  tab_tune times `reps` runs (3 if reps is
 * 0) of the compiled program p from |0^n> on handle h, with the handle's RNG
 * settings, under each launch shape the kernels are built for: the
 * measurement engine (single-CTA, grid-resident, streaming, where each holds
 * n qubits), the grid-resident engine's measurements per batch (8, 16, 32),
 * then the block gate kernel's threads per CTA (128, 256, 512) with the best
 * engine.  It keeps the fastest shape for later runs on h (tab_set_engine
 * and the handle's launch shape) and returns it in *out.  Every run's
 * outcomes must equal the first run's; TAB_EDEVICE if a shape disagrees.
 * With TAB_AUTOTUNE_CACHE naming a file, a shape stored there for the same
 * (GPU name, n rounded up to a power of two, log2 of gates per qubit, log2 of
 * measurements + 1) is applied without timing (from_cache = 1) unless reps <
 * 0, and a tuning run adds its shape to the file.  Leaves the tableau reset
 * to |0^n> and the outcome log empty.  Synchronizes. */
typedef struct {
  int32_t engine;         /* TAB_ENGINE_* the measurement runs take */
  int32_t block_threads;  /* block gate kernel threads per CTA (0: the default by n) */
  int32_t meas_batch;     /* grid-resident measurements per batch (0: the largest that fits) */
  int32_t from_cache;     /* 1: taken from the TAB_AUTOTUNE_CACHE file, no timing */
  int32_t tried;          /* shapes timed */
  float best_ms;          /* mean time of one run of p with the kept shape */
} tab_tuned;
int tab_tune(tab_t h, tab_prog_t p, int32_t reps, tab_tuned *out);

/* ---- run-time configuration (process-wide) ------------------------------
 * Launch-shape knobs (0 = the library's choice by size), the limit of the
 * device-side grid-barrier waits, and test-only fault injection.  The
 * paper has no counterpart.  Initial values come from the environment
 * (TAB_BLOCK_THREADS, TAB_MEAS_BATCH, TAB_GRID_CTAS, TAB_BATCH_CHUNKS), read on
 * first use.
 * tab_set_config applies to launches issued after it returns; grid_ctas
 * applies to handles created after it.  TAB_EINVAL (nothing changed) for an
 * out-of-range field. */
typedef struct {
  int32_t block_threads;  /* block gate kernel threads per CTA: 0, 128, 256, 512 */
  int32_t meas_batch;     /* grid-resident engine measurements per batch: 0 or 1..32 (power of 2) */
  int32_t grid_ctas;      /* grid-resident engine CTAs: 0 = one per SM */
  uint32_t debug;         /* TAB_DEBUG_* bits */
  uint64_t wait_limit_ns; /* limit of each grid-barrier wait in the measurement
                             engines; 0 = 2 s.  A wait that runs out latches a
                             device error reported as TAB_ETIMEOUT */
  int32_t batch_chunks;   /* tab_batch_run: pieces the circuit list is cut into,
                             each compiled on the host while the device runs
                             the one before; 0 = by size (five for large
                             lists, a small first one), else 1..64 pieces of
                             equal gate count */
  int32_t reserved;       /* 0 */
} tab_config;
/* Test-only: in every grid-resident measurement launch the last CTA skips its
 * first grid-barrier arrival and leaves, so the other CTAs' bounded waits run
 * out (TAB_ETIMEOUT at the next synchronizing call).  Nothing hangs or
 * faults: every CTA returns once its wait has run out. */
#define TAB_DEBUG_SKIP_BARRIER_ARRIVAL 1u
int tab_get_config(tab_config *out);
int tab_set_config(const tab_config *cfg);

/* ---- debug build ---------------------------------------------------------
 * The same library compiled with -DTAB_DEBUG (libtab_debug.so, built by
 * `python -m paper_2408_00384_gb300.build --debug`; the Python binding loads
 * it when the environment variable TAB_DEBUG is 1).  In it every qubit index
 * a kernel reads from its inputs (gate and measurement codes, block records,
 * the batch's work items) is checked against the tableau's size on the
 * device; an index out of range latches a device error, reported as
 * TAB_EDEVICE ("index out of range") by the next synchronizing call, and is
 * replaced by 0, so no kernel touches memory outside its tableau.  Nothing
 * traps.  Host-side validation is the same in both builds.
 *
 * tab_debug_build: 1 in the debug build, 0 otherwise.
 * tab_debug_check: runs the device check once, on `index` against `limit`,
 *   in a one-thread kernel on the current device; *checked gets the index
 *   the kernel went on with.  Returns TAB_OK (index in range, or a release
 *   build, where the check is compiled out and the index passes unchanged),
 *   TAB_EDEVICE (debug build, index out of range: the error latched), or
 *   TAB_ECUDA. */
int tab_debug_build(void);
int tab_debug_check(uint32_t index, uint32_t limit, uint32_t *checked);

/* ---- roofline ceilings of the current device ---------------------------
 * The paper has no counterpart: these are the ceilings the kernels above are
 * measured against.  Every kernel here is GF(2) logic on words held in shared
 * memory, L2 or HBM, so its roofline is the integer logic pipe, the shared
 * memory port, L2 or HBM; the measurement engines also wait on chains of grid
 * barriers.  tab_measure_peaks times one launch of each microbenchmark with
 * CUDA events after a warm-up launch (about 0.2 s in all), on a stream of its
 * own, and changes no device setting.  It allocates (and frees) 128 MiB of
 * device memory.  TAB_ECUDA if a launch fails; TAB_ETIMEOUT if the barrier
 * benchmark's bounded wait ran out (then grid_barrier_us is 0). */
typedef struct {
  int32_t sms;                  /* multiprocessors of the current device */
  double sm_clock_mhz;          /* SM clock during the logic run (clock64 over globaltimer) */
  double logic_tops;            /* lop3.b32 per second, all SMs (1e12) */
  double logic_ops_per_clk_sm;  /* the same per SM per clock */
  double logic_ms;              /* duration of the logic run */
  double smem_gbs;              /* ld.shared.v4 bytes per second, all SMs, no bank conflicts */
  double smem_bytes_per_clk_sm; /* the same per SM per clock */
  double l2_read_gbs;           /* ld.global.cg bytes per second over a 64 MiB set */
  double l2_rw_gbs;             /* read + write bytes per second over a 64 MiB set */
  double grid_barrier_us;       /* one bounded grid barrier, one CTA per SM */
} tab_peaks;
int tab_measure_peaks(tab_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* TAB_H_ */
