// tab_internal.h -- device layout, compiled-program format and launch
// declarations shared by the kernels and the C-ABI layer of libtab.
//
// Device tableau layout ("qubit-major, bit-packed"):
//   Wh = ceil(n/32) rounded up to a multiple of 4 words per half-column,
//   W  = 2*Wh words per column.  Word w of a column holds 32 rows: bit b of
//   word w is packed row 32*w + b.  Destabilizer i is packed row i, stabilizer
//   i is packed row 32*Wh + i, so a stabilizer and its paired destabilizer sit
//   at the same bit of words w and w - Wh.  Pad rows are all-zero with sign 0,
//   and every gate keeps them so.
//   X plane: X[a*W + w], Z plane: Z[a*W + w] (a = qubit), sign: R[w].
// A gate therefore touches whole contiguous columns (coalesced sweeps), and a
// measurement's pivot search reads one contiguous half-column.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/tab.h"

namespace tab {

// ---- device op codes: op<<28 | q1<<14 | q2 (q < 2^14) --------------------
enum : uint32_t {
  OP_I = 0, OP_X = 1, OP_Y = 2, OP_Z = 3, OP_H = 4, OP_S = 5, OP_SDG = 6,
  OP_CNOT = 7, OP_CZ = 8, OP_SWAP = 9, OP_MZ = 10, OP_MZR = 11,
  // a Pauli noise op resolved per shot on the device: q1 = qubit, q2 = its
  // ordinal among the circuit's noise ops (index into the noise table, whose
  // entry is kind << 28 | 28-bit probability, kind 0 DEPOL1, 1 XERR, 2 ZERR)
  OP_NOISE = 12
};
__host__ __device__ __forceinline__ uint32_t dcode(uint32_t op, uint32_t a, uint32_t b) {
  return (op << 28) | (a << 14) | b;
}
__host__ __device__ __forceinline__ uint32_t dop(uint32_t c) { return c >> 28; }
__host__ __device__ __forceinline__ uint32_t dq1(uint32_t c) { return (c >> 14) & 0x3FFFu; }
__host__ __device__ __forceinline__ uint32_t dq2(uint32_t c) { return c & 0x3FFFu; }

inline int half_words(int n) { return (((n + 31) / 32) + 3) & ~3; }

// ---- device error word values ---------------------------------------------
enum : int { DERR_NONE = 0, DERR_TIMEOUT = 1, DERR_PHASE = 2, DERR_BOUNDS = 3 };

// ---- debug builds (compiled with -DTAB_DEBUG: libtab_debug.so) ---------------
// Every qubit index a kernel takes from its inputs goes through dbg_index.  In
// a debug build an index at or past `lim` latches DERR_BOUNDS in the error
// word and is replaced by 0, so the kernel finishes without touching memory
// outside its tableau and the next synchronizing call reports the error; in a
// release build the index passes unchanged and the check compiles away.
#ifdef TAB_DEBUG
constexpr bool kDebugBuild = true;
#else
constexpr bool kDebugBuild = false;
#endif
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t dbg_index(uint32_t i, uint32_t lim, int* err) {
  if (kDebugBuild && i >= lim) {
    if (err) atomicCAS(err, 0, DERR_BOUNDS);
    return 0u;
  }
  return i;
}
// A gate or measurement code with its qubit fields checked against n
// (dbg_index; the second field only for two-qubit gates).
__device__ __forceinline__ uint32_t dbg_code(uint32_t c, uint32_t n, int* err) {
  if (!kDebugBuild) return c;
  const uint32_t op = dop(c);
  const uint32_t q1 = dbg_index(dq1(c), n, err);
  const uint32_t q2 = (op == OP_CNOT || op == OP_CZ || op == OP_SWAP) ? dbg_index(dq2(c), n, err) : dq2(c);
  return (c & 0xF0000000u) | (q1 << 14) | q2;
}
#endif

// ---- compiled program ----------------------------------------------------------
// ops[] holds gate segments (gates grouped by layer; a layer's gates act on
// pairwise-disjoint qubits) and measurement segments (MZ/MZR codes in program
// order).  layer_off[] holds absolute op offsets of layer boundaries.
struct Seg {
  uint32_t kind;       // 0 = gates, 1 = measurements
  uint32_t op_begin, op_end;
  uint32_t layer_begin, layer_end;  // gates: layers [layer_begin, layer_end)
  uint32_t meas_before;             // measurement ops preceding this segment
  uint32_t blk_begin, blk_end;      // gates: block super-layers [blk_begin, blk_end)
};

// Compile forms of gate runs (build_program's mode, either or both):
//   kProgLayers  ASAP layers of gate codes (ops, layer_off): the single-CTA
//                engine;
//   kProgBlocks  two-qubit blocks in super-layers (blk, blk_off): the block
//                gate kernel of the multi-CTA engines (blocks.cpp).
//   kProgNoise   (with kProgLayers only) Pauli noise ops are kept as OP_NOISE
//                codes and listed in `noise`, for per-shot draws on the device.
//   kProgBankOrder  (with kProgBlocks) order each super-layer's records so
//                that a warp's 32 lanes touch distinct shared-memory banks
//                where the layer allows: about twice the host compile time,
//                so it is used where a program is compiled once and replayed
//                (tab_prog_create), not on the per-call paths.
enum : int { kProgLayers = 1, kProgBlocks = 2, kProgNoise = 4, kProgBankOrder = 8 };

struct HostProgram {
  int32_t n = 0;
  int mode = kProgLayers;
  int64_t n_gates = 0, n_meas = 0;
  // block records: lo = qa | qb<<14 | has_b<<28 | ent<<29 (0 none, 1 CNOT
  // with its control in register 0, 2 CZ); hi = U0 | U1<<7 | V0<<14 |
  // V1<<21 | swap<<28 (7-bit single-qubit Cliffords, clifford1.h)
  std::vector<uint2> blk;
  std::vector<uint32_t> blk_off;  // absolute record offsets of super-layer bounds
  std::vector<uint32_t> ops;
  std::vector<uint32_t> layer_off;  // size = layers + 1 when any gate exists
  std::vector<uint32_t> noise;      // kProgNoise: kind << 28 | probability, per noise op
  std::vector<Seg> segs;
  // empty program for n qubits (the arrays keep their capacity)
  void clear(int32_t n_) {
    n = n_;
    mode = kProgLayers;
    n_gates = n_meas = 0;
    blk.clear();
    blk_off.clear();
    ops.clear();
    layer_off.clear();
    noise.clear();
    segs.clear();
  }
};

// Validate and compile a gate list into the forms `mode` asks for (see
// kProgLayers etc.; measurement runs are always MZ/MZR codes in ops).
// Returns TAB_OK or an error (message set).
int build_program(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out,
                  int mode = kProgLayers);
// Lower a validated list with extended ops to base ops for a batch or a
// request: MX / MY become Z measurements between basis changes (as in
// tab_apply); noise ops are kept as they are (keep_noise: drawn per shot on
// the device) or resolved for (seed, cid, shot) with the noise counter
// starting at 0.
int lower_for_runs(int32_t n, const tab_gate* g, int64_t count, bool keep_noise, uint64_t seed,
                   uint64_t cid, uint32_t shot, std::vector<tab_gate>& out);
// Validate a gate list (in parallel on the host pool): TAB_OK, or the error of
// the first bad word in list order (message set).  With `ext` given, the
// extended ops (TAB_MX .. TAB_ZERR) are accepted and *ext counts them;
// without it they are errors.
int validate_program(int32_t n, const tab_gate* gates, int64_t count, int64_t* ext = nullptr);
// Compile an already validated gate list (validate_program returned TAB_OK
// with no extended ops) in one of build_program's modes, on this thread.
int build_validated(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out, int mode);
// Compile an already validated piece of a gate list into blocks (kProgBlocks).
int build_validated_blocks(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out);
// Concatenate part[0..T) -- programs compiled for consecutive pieces of one
// gate list, in list order -- into P: each piece's arrays copied and its
// offsets shifted (pieces in parallel on the host pool).  Consecutive gate
// runs keep adjacent super-layer offsets: the last bound of one run equals
// the first of the next.  With with_blk false the block records are not
// copied (P.blk stays empty; the offsets are those of the full concatenation).
void concat_programs(HostProgram& P, const HostProgram* part, size_t T, bool with_blk = true);

// Block compiler for one gate run at a time (blocks.cpp).
struct BlkRec {
  uint16_t qa, qb;
  int32_t layer;
  uint8_t has_b, ent, dir, swp, dead;
  uint8_t U[2], V[2];
};
class BlockBuilder {
 public:
  void reset(int32_t n, size_t hint);             // start a gate run (hint: blocks)
  void add(uint32_t op, uint32_t a, uint32_t b);  // next gate of the run (tab_op)
  void emit(HostProgram& P, Seg& s);              // append the run's blocks
  bool bank_order_on = false;                     // kProgBankOrder
 private:
  struct QSlot {
    int32_t cur;     // latest block of the qubit in this run
    uint32_t stamp;  // run id of `cur` / `role`
    uint32_t role;   // register of that block holding the qubit
  };
  std::vector<QSlot> q_;
  uint32_t seg_ = 0;
  const uint8_t* comp_ = nullptr;  // single-qubit code composition table
  const uint8_t* code_ = nullptr;  // code of each one-qubit op
  std::vector<BlkRec> blk_;
  std::vector<uint32_t> key_, cnt_;  // emit scratch: sort key per block, bucket counts
  std::vector<uint2> rec_;           // emit scratch: packed record per block
};

// ---- global grid barrier state ----------------------------------------------------
struct GridBar {
  unsigned int count;
  unsigned int gen;
};

// ---- measurement workspace (per handle) ---------------------------------------------
struct MeasWork {
  uint32_t* ph;     // [G][2][W] per-CTA partial phases (lo plane, hi plane)
  uint32_t* r4;     // [2][W]    base phase (lo, hi), owned by CTA 0
  uint32_t* dp;     // [2][G]    deterministic partials, double-buffered
  GridBar* bar;
  int* err;
  int max_ctas;
  // work counters (tab_count_work; null: off): [0] support columns of the
  // random-outcome pivot rows, [1] stabilizer rows the deterministic
  // outcomes multiply, [2] random and [3] deterministic measurements
  unsigned long long* work = nullptr;
};

// ---- launches (kernels_*.cu) ---------------------------------------------------------
void launch_init(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh, cudaStream_t s);
// Gate layers (single-CTA engine) and block super-layers hold at most
// kMaxLayerOps entries; device op and record buffers extend at least kOpsPad
// entries past their last one.
constexpr int kMaxLayerOps = 2048;
constexpr int kOpsPad = 1024;
// Block gate kernel: super-layers of at most kMaxLayerOps records, the
// device record buffer padded by kOpsPad records past its end.
int gates_block_max_n();
// threads: 128, 256 or 512 per CTA, 0 for the default by n
cudaError_t launch_gates_block(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int W,
                               const uint2* blk, const uint32_t* blk_off, int nlayers,
                               int* err, cudaStream_t s, int threads = 0);
cudaError_t launch_measure(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh,
                           const uint32_t* mops, int nm, uint64_t k0, uint64_t seed,
                           uint64_t cid, uint32_t shot, uint8_t* out, const MeasWork& mw,
                           int ctas, cudaStream_t s);
int measure_ctas_for(int n, int sm_count, int max_ctas);
// Grid-resident measurement engine (kernels_resident.cu): CTA count for n
// qubits (0 if the tableau does not fit the GPU's shared memory), its global
// workspace in words, and the launch.
int resident_ctas_for(int n, int Wh, int sm_count);
size_t resident_work_words(int n, int max_ctas);
// batch: largest measurements per batch (a power of two), 0 for the default
cudaError_t launch_measure_resident(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh,
                                    const uint32_t* mops, int nm, uint64_t k0, uint64_t seed,
                                    uint64_t cid, uint32_t shot, uint8_t* out, int* err,
                                    uint32_t* work, GridBar* bar, int G, cudaStream_t s,
                                    int batch = 0);
size_t measure_work_words(int n, int max_ctas);
cudaError_t launch_expect(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int Wh,
                          const uint8_t* codes, int k, int8_t* out, int* err, cudaStream_t s);
size_t sv_work_bytes(int n);
cudaError_t launch_statevector(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n,
                               int Wh, uint32_t b, float2* v, void* work, cudaStream_t s);
cudaError_t launch_pack(uint32_t* X, uint32_t* Z, uint32_t* R, const uint8_t* xs,
                        const uint8_t* zs, const uint8_t* rs, int n, int Wh, cudaStream_t s);
cudaError_t launch_unpack(const uint32_t* X, const uint32_t* Z, const uint32_t* R,
                          uint8_t* xs, uint8_t* zs, uint8_t* rs, int n, int Wh,
                          cudaStream_t s);

// thread-local error message
void set_error(const char* fmt, ...);

// Process-wide run-time configuration (config.cpp): a copy of the current
// settings, and the grid-barrier wait limit in effect.
constexpr unsigned long long kDefaultWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kMaxBatchChunks = 64;  // tab_config.batch_chunks upper bound

// tab_batch_run's chunks of a circuit list: contiguous runs of circuits cut
// where the running gate count first reaches each target -- first_share of
// all gates for the first chunk, then equal parts of the rest -- so at most
// K chunks, none empty.  Returns the bounds: 0, ..., m (one entry, 0, for
// m = 0).
inline std::vector<int32_t> batch_chunk_cuts(const tab_circuit* circuits, int32_t m, int K,
                                             double first_share) {
  int64_t gates = 0;
  for (int32_t c = 0; c < m; ++c) gates += circuits[c].n_gates > 0 ? circuits[c].n_gates : 0;
  std::vector<int32_t> cut(1, 0);
  int64_t before = 0;
  for (int32_t c = 0, k = 1; c < m && k < K; ++c) {
    before += circuits[c].n_gates > 0 ? circuits[c].n_gates : 0;
    const double target =
        (double)gates * (first_share + (1.0 - first_share) * (double)(k - 1) / (double)(K - 1));
    if ((double)before >= target) {
      cut.push_back(c + 1);
      ++k;
    }
  }
  if (cut.back() != m) cut.push_back(m);
  return cut;
}
tab_config run_config();
unsigned long long run_wait_limit_ns();

// Raise fn's dynamic shared-memory limit to `bytes` on the current device,
// once per (kernel, device, limit).  Thread-safe; never allocates.
cudaError_t ensure_smem_limit(const void* fn, int bytes);

// Read-only view of a handle for entry points outside tab_api.cpp.
struct HandleView {
  int n, Wh, dev;
  uint32_t *X, *Z, *R;
  cudaStream_t stream;
  uint64_t seed, cid, k;
  uint32_t shot;
  int* err;
  int meas_ctas;
};
int handle_view(tab_t h, HandleView* v);     // TAB_OK, or the handle's error
void handle_advance_k(tab_t h, uint64_t dk);  // count dk more measurement ops
// Launch shape of a handle's plain-path kernels (0: the library's default):
// block gate kernel threads per CTA, grid-resident measurements per batch.
void handle_set_shape(tab_t h, int block_threads, int meas_batch);
void handle_get_shape(tab_t h, int* block_threads, int* meas_batch);

}  // namespace tab
