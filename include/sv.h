/*
 * sv.h -- C ABI of the GB300 state-vector simulator core (libsv.so).
 *
 * The library applies quantum gates to a state vector held in GPU memory and
 * reduces measurement probabilities and Pauli-string expectation values, as
 * the state-vector primitives of the cuQuantum paper describe them (arXiv
 * 2308.01999, Sec. II-A, Table I; gate fusion Sec. II-B and Sec. II-D-1).
 *
 * Conventions (the paper fixes only that each index bit is one qubit, Sec. II-C):
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - a state of n qubits is 2^n amplitudes, interleaved (re, im):
 *     SV_C64 = two floats (8 bytes), SV_C128 = two doubles (16 bytes);
 *   - a gate matrix is HOST memory, row-major, 2^k x 2^k complex128 given as
 *     interleaved (re, im) doubles; row/column index bit j belongs to targets[j];
 *   - a controlled gate applies its matrix where every control qubit equals its
 *     control value (all 1 when control_values is NULL), identity elsewhere.
 *
 * Memory ownership (Sec. II-A, "relaxed memory model" and "small memory
 * footprint"): the state vector belongs to the caller, who allocates it in GPU
 * memory; the library only borrows the pointer. Every operation runs in place.
 * A handle owns one small device workspace (SV_WORKSPACE_BYTES) and one small
 * pinned host buffer, allocated by sv_create and freed by sv_destroy. Host
 * arrays passed to any call (matrices, qubit lists, Pauli strings) are read
 * before the call returns and may be freed right after.
 *
 * Streams: work is enqueued on the handle's CUDA stream and returns without
 * waiting, except the calls documented as synchronising (they return host
 * values and wait for the stream).
 *
 * Errors: every call returns an sv_status_t; nothing is thrown across the ABI.
 * A call that returns an error has enqueued no work, except SV_ERR_CUDA, which
 * reports a failed CUDA call or launch (cudaGetLastError is cleared by then).
 */
#ifndef SV_GB300_SV_H
#define SV_GB300_SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SV_API __attribute__((visibility("default")))
#else
#define SV_API
#endif

#define SV_MAX_TARGETS 6         /* largest dense gate, 64 x 64 */
#define SV_MAX_CONTROLS 24       /* control qubits of one gate */
#define SV_MAX_QUBITS 36         /* 2^36 c64 amplitudes = 512 GiB: beyond one GPU */
#define SV_WORKSPACE_BYTES (32u << 20)  /* device workspace per handle ("a few tens of MB", Table I) */

typedef struct sv_ctx *sv_handle_t;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype_t;

typedef enum {
    SV_OK = 0,
    SV_ERR_INVALID_ARGUMENT = 1,    /* bad qubit index, duplicate qubit, k out of range, NULL pointer */
    SV_ERR_NOT_SUPPORTED = 2,       /* e.g. tensor-core precision on a complex128 state */
    SV_ERR_INSUFFICIENT_WORKSPACE = 3,
    SV_ERR_CUDA = 4,                /* a CUDA call or kernel launch failed */
    SV_ERR_TIMEOUT = 5,             /* a bounded device-side wait gave up (see sv_check_device_status) */
    SV_ERR_ALLOC = 6                /* the handle's workspace could not be allocated */
} sv_status_t;

/* Arithmetic of fused gates of 5-6 qubits on a complex64 state (Sec. II-B).
 * NATIVE: FP32 complex arithmetic on CUDA cores.
 * TF32: tensor cores, operands rounded to TF32, FP32 accumulation.
 * SPLIT_BF16: tensor cores, each operand split into a BF16 high and low part,
 *   three products (hi*hi + hi*lo + lo*hi), FP32 accumulation. */
typedef enum { SV_PREC_NATIVE = 0, SV_PREC_TF32 = 1, SV_PREC_SPLIT_BF16 = 2 } sv_precision_t;

typedef enum { SV_PAULI_I = 0, SV_PAULI_X = 1, SV_PAULI_Y = 2, SV_PAULI_Z = 3 } sv_pauli_t;

/* One gate of a circuit, as sv_apply_fused and sv_fuse_plan read it. */
typedef struct {
    int n_targets;                        /* 1..SV_MAX_TARGETS */
    int targets[SV_MAX_TARGETS];
    int n_controls;                       /* 0..SV_MAX_CONTROLS */
    int controls[SV_MAX_CONTROLS];
    int control_values[SV_MAX_CONTROLS];  /* each 0 or 1 */
    const double *matrix;                 /* host, row-major 2^k x 2^k complex128 (re, im) */
} sv_gate_t;

/* Create a handle for an n-qubit state of the given dtype at d_state (device
 * memory, 2^n amplitudes, at least 16-byte aligned, owned by the caller).
 * stream: a cudaStream_t (NULL = the legacy default stream). Allocates the
 * handle's workspace on the current device. The state's contents are not
 * touched. Errors: INVALID_ARGUMENT (n outside 1..SV_MAX_QUBITS, NULL pointers,
 * misaligned d_state), ALLOC, CUDA. (Table I, "Resource management".) */
SV_API sv_status_t sv_create(int n_qubits, sv_dtype_t dtype, void *d_state, void *stream, sv_handle_t *out);

/* Wait for the handle's stream, then free the workspace; never frees the state. */
SV_API sv_status_t sv_destroy(sv_handle_t h);

/* Enqueue later work on another stream (a cudaStream_t). */
SV_API sv_status_t sv_set_stream(sv_handle_t h, void *stream);

/* Point the handle at another state of the same size and dtype. */
SV_API sv_status_t sv_set_state_pointer(sv_handle_t h, void *d_state);

/* Point the handle at another state of n_qubits qubits and the given dtype
 * (device memory, 2^n_qubits amplitudes, 16-byte aligned, caller-owned). The
 * workspace does not depend on the state's size, so a handle can serve states
 * of any size in turn without allocating: a pool of handles, one per stream,
 * replaces sv_create / sv_destroy per state (Table I, "Resource management").
 * Work already enqueued keeps the state it was given. Errors:
 * INVALID_ARGUMENT as sv_create. */
SV_API sv_status_t sv_set_state(sv_handle_t h, int n_qubits, sv_dtype_t dtype, void *d_state);

/* psi <- |index> (one amplitude 1, the rest 0). Asynchronous. */
SV_API sv_status_t sv_set_basis_state(sv_handle_t h, uint64_t index);

/* Accessor (Table I) without qubit reordering: copy the whole state between a
 * host buffer of 2^n amplitudes and the device. Pinned host memory makes the
 * copy faster. Both synchronise the stream before returning. */
SV_API sv_status_t sv_copy_from_host(sv_handle_t h, const void *host);
SV_API sv_status_t sv_copy_to_host(sv_handle_t h, void *host);

/* The same copies, only enqueued on the handle's stream (they return at once).
 * The host buffer must stay valid, and must not be reused, until the stream
 * has passed the copy; with pinned host memory the copy overlaps work on other
 * streams (e.g. a second state's gates), with pageable memory the CUDA runtime
 * stages it and the call may block. Errors: INVALID_ARGUMENT for NULL
 * pointers, CUDA. */
SV_API sv_status_t sv_copy_from_host_async(sv_handle_t h, const void *host);
SV_API sv_status_t sv_copy_to_host_async(sv_handle_t h, void *host);

/* Gate application (Table I; Sec. II-B): psi <- G psi with G the 2^k x 2^k
 * matrix on targets (k = n_targets, 1..6), applied where the controls hold.
 * adjoint != 0 applies the conjugate transpose. The library inspects the
 * matrix exactly (no tolerance) and takes the cheapest exact form: target
 * bits on which the matrix is the identity in one half become controls, a
 * diagonal matrix scales only the amplitudes it changes, and a generalized
 * permutation matrix (one nonzero per row and column, e.g. X, CNOT) moves
 * amplitudes without a matrix product (Sec. II-D-1). Asynchronous.
 * Errors: INVALID_ARGUMENT for a qubit outside [0, n), a qubit listed twice
 * (among targets and controls together), k outside 1..6, more than
 * SV_MAX_CONTROLS controls, a control value other than 0/1, NULL pointers. */
SV_API sv_status_t sv_apply_matrix(sv_handle_t h, const int *targets, int n_targets,
                            const int *controls, const int *control_values, int n_controls,
                            const double *matrix, int adjoint);

/* Gate fusion (Sec. II-B; qsim's max_fused_gate_size, Sec. II-D-1): the gates
 * are grouped greedily, in program order and moving a gate only past gates on
 * disjoint qubits, into blocks of at most max_fused_qubits qubits (1..6); each
 * block's matrix is composed on the host in FP64 and applied once. Blocks of
 * 5-6 qubits run in `prec` (tensor cores for TF32 / SPLIT_BF16), smaller ones
 * in native precision. With a tensor-core precision, when at least 6 wide
 * blocks would have a target on qubit 0 or 1 (the slower tensor-core variant),
 * the call first relabels qubits (Sec. II-C, qubit reordering: one index-bit
 * swap pass moving the qubits that the fewest wide blocks use down to bits 0-1),
 * applies the blocks in the new labels and swaps back; the result is the same.
 * *n_fused_out (may be NULL) receives the block count. Asynchronous. Errors:
 * as sv_apply_matrix for each gate; NOT_SUPPORTED for a tensor-core precision
 * on a complex128 state. */
SV_API sv_status_t sv_apply_fused(sv_handle_t h, const sv_gate_t *gates, int n_gates,
                           int max_fused_qubits, sv_precision_t prec, int *n_fused_out);

/* Index-bit swap (Table I, "Index bit swap", single-GPU version; Sec. II-C,
 * qubit reordering): for each of the n_pairs disjoint pairs
 * (bit_pairs[2k], bit_pairs[2k+1]) exchange those two bits of every amplitude
 * index, i.e. psi'[swap(i)] = psi[i]. This relabels the paired qubits (qubit a
 * of the new state is qubit b of the old one). In place, one pass over the
 * amplitudes whose paired bits differ. Asynchronous. Errors: INVALID_ARGUMENT
 * for a bit outside [0, n), a bit used twice, a pair of equal bits, or
 * n_pairs outside 1..18. */
SV_API sv_status_t sv_swap_index_bits(sv_handle_t h, const int *bit_pairs, int n_pairs);

/* Fusion options: max_fused_qubits as above (1..6); max_fused_diagonal_qubits
 * (0 = off, else 1..6) sends diagonal gates (CZ, CRZ, phases, controlled
 * diagonals) to separate diagonal blocks of up to that many qubits, applied by
 * the diagonal kernel (Sec. II-D-1: dense/diagonal fusion with
 * max_fused_gate_size and max_fused_diagonal_gate_size); precision as above. */
typedef struct {
    int max_fused_qubits;
    int max_fused_diagonal_qubits;
    sv_precision_t precision;
} sv_fusion_options_t;

/* sv_apply_fused with explicit options (sv_apply_fused is this call with
 * max_fused_diagonal_qubits = 0). Errors as sv_apply_fused, and
 * INVALID_ARGUMENT for an option out of range or a NULL opt. */
SV_API sv_status_t sv_apply_fused_ex(sv_handle_t h, const sv_gate_t *gates, int n_gates,
                                     const sv_fusion_options_t *opt, int *n_fused_out);

/* Host-only view of the fusion pass, for inspection and tests (no GPU needed).
 * Writes at most max_blocks blocks: block b acts on block_k[b] qubits
 * block_targets[6*b .. 6*b+k-1] (bit j of its matrix index is target j) with
 * the 2^k x 2^k complex128 matrix at block_matrices + b * 64*64*2 doubles
 * (row-major, leading dimension 2^k). Blocks are applied in order.
 * Errors: INVALID_ARGUMENT; INSUFFICIENT_WORKSPACE if more than max_blocks. */
SV_API sv_status_t sv_fuse_plan(const sv_gate_t *gates, int n_gates, int n_qubits, int max_fused_qubits,
                         int max_blocks, int *n_blocks_out, int *block_k, int *block_targets,
                         double *block_matrices);

/* sv_fuse_plan with explicit fusion options (the precision field is ignored). */
SV_API sv_status_t sv_fuse_plan_ex(const sv_gate_t *gates, int n_gates, int n_qubits, const sv_fusion_options_t *opt,
                                   int max_blocks, int *n_blocks_out, int *block_k, int *block_targets,
                                   double *block_matrices);

/* Pauli-string expectation values (Table I, "Expectation"):
 * out[s] = Re <psi| P_s |psi>, P_s = prod_i paulis[s*n_sites + i] on qubit
 * sites[s*n_sites + i]. Not divided by <psi|psi>. Products are formed in the
 * state's precision. complex128: accumulated in FP64. complex64: each thread
 * adds up to 8 terms in FP32, accumulates those partials in FP32 with
 * compensation (Neumaier), and everything across threads and blocks is
 * summed in FP64 in a fixed order (bitwise reproducible); the absolute error
 * stays below about 1.2e-6 <psi|psi> (the terms' magnitudes sum to at most
 * <psi|psi>) and is typically far smaller. out is host memory of n_strings
 * doubles. Synchronises the stream. Errors: INVALID_ARGUMENT for a site outside
 * [0, n), a site repeated within a string, a code outside 0..3. */
SV_API sv_status_t sv_expectation_pauli(sv_handle_t h, const int *paulis, const int *sites,
                                 int n_sites, int n_strings, double *out);

#define SV_NOALLOC_MAX_STRINGS 4096  /* strings per sv_expectation_pauli_noalloc call */

/* Pauli-string expectation values without a handle and without allocating
 * anything (this entry point has no counterpart in the paper). It is for
 * callers that cannot call cudaMalloc: a process whose device memory is
 * already owned by another allocator (for example a framework's caching
 * allocator, or a memory pool sized to the whole GPU), where a new allocation
 * would fail or force that allocator to give memory back, and latency-critical
 * loops that cannot afford cudaMalloc/cudaFree, which may synchronise the
 * device. Results equal sv_expectation_pauli's for the same state and strings.
 * d_state: device memory, 2^n_qubits amplitudes of `dtype`, 16-byte aligned,
 * caller-owned; stream: a cudaStream_t (NULL = legacy default stream); paulis,
 * sites, n_sites, n_strings, out: as sv_expectation_pauli (out is host memory).
 * Scratch space is one file-scope device array of 160 KiB that every GPU which
 * loads the library holds until the process exits; at most
 * SV_NOALLOC_MAX_STRINGS strings per call (more: SV_ERR_INSUFFICIENT_WORKSPACE,
 * before any work is enqueued). The first call on a device, made with that
 * device current, looks up the array's device address (cudaGetSymbolAddress)
 * and caches it. All calls
 * share the array: calls whose work overlaps on the GPU race, so the caller
 * must order them (one stream, or synchronise between them). Synchronises the
 * stream. Errors: INVALID_ARGUMENT as sv_expectation_pauli, or for a NULL or
 * misaligned d_state or a bad dtype; CUDA. */
SV_API sv_status_t sv_expectation_pauli_noalloc(int n_qubits, sv_dtype_t dtype, const void *d_state, void *stream,
                                                const int *paulis, const int *sites, int n_sites, int n_strings,
                                                double *out);

/* Pauli rotation (Table I, "Pauli rotation"): psi <- exp(i theta P) psi =
 * cos(theta) psi + i sin(theta) P psi, P = prod_i paulis[i] on qubit sites[i]
 * (codes as sv_expectation_pauli). In place, one pass over the state.
 * Asynchronous. Errors: INVALID_ARGUMENT for a bad code or site, a repeated
 * site, a non-finite theta. */
SV_API sv_status_t sv_apply_pauli_rotation(sv_handle_t h, double theta, const int *paulis, const int *sites,
                                           int n_sites);

/* Sampler (Table I, "Sampler"): measurement outcomes of all qubits without
 * collapsing the state. For each randnums[t] in [0, 1), out[t] is the basis
 * index i at which the cumulative probability sum_{k<=i} |psi_k|^2 first
 * exceeds randnums[t] * <psi|psi> (probabilities summed in FP64). out is host
 * memory of n_samples int64. Synchronises the stream. Errors:
 * INVALID_ARGUMENT for a random number outside [0, 1) or NULL pointers. */
SV_API sv_status_t sv_sample(sv_handle_t h, const double *randnums, int n_samples, int64_t *out);

/* Probabilities of a measurement in the Z-product basis of `qubits` (Table I,
 * "Measurement"): p_even/p_odd = sum of |psi_i|^2 over basis states whose
 * measured bits have even/odd parity, in FP64. Synchronises the stream. */
SV_API sv_status_t sv_measure_probs(sv_handle_t h, const int *qubits, int n_qubits,
                             double *p_even, double *p_odd);

/* Collapse onto one parity outcome (Table I: collapse is separate from the
 * probability computation): amplitudes of the other parity become 0, the rest
 * are scaled by 1/sqrt(prob). Asynchronous. INVALID_ARGUMENT unless prob > 0. */
SV_API sv_status_t sv_collapse(sv_handle_t h, const int *qubits, int n_qubits, int parity, double prob);

/* Measurement: parity 0 iff randnum < p_even / (p_even + p_odd); with collapse
 * != 0 the state collapses onto that outcome. randnum in [0, 1). Synchronises. */
SV_API sv_status_t sv_measure(sv_handle_t h, const int *qubits, int n_qubits, double randnum,
                       int collapse, int *parity_out);

/* <psi|psi> in FP64. Synchronises the stream. */
SV_API sv_status_t sv_norm2(sv_handle_t h, double *out);

/* Synchronise the stream and report whether a bounded device-side wait gave
 * up since the last call (SV_ERR_TIMEOUT), then clear the flag. */
SV_API sv_status_t sv_check_device_status(sv_handle_t h);

/* Diagnostic of device-side failure detection: launch one wait that nothing
 * completes, bounded to `cycles` SM clock ticks (1e3..4e9), then report the
 * device status as sv_check_device_status does. A working build returns
 * SV_ERR_TIMEOUT (and clears the flag); the context stays usable. The
 * tensor-core kernel bounds every one of its waits the same way. */
SV_API sv_status_t sv_check_bounded_wait(sv_handle_t h, long long cycles);

/* Number of kernels this handle has launched since sv_create. */
SV_API sv_status_t sv_launch_count(sv_handle_t h, uint64_t *out);

/* ---- Batched state vectors ----
 * Many independent circuits advanced by one persistent launch (gate
 * application and expectation values of Table I, with gate fusion of
 * Sec. II-B, on a batch). Each state of up to SV_BATCH_TILE_QUBITS qubits
 * lives in GPU shared memory of one CTA for its whole circuit; larger ones (up
 * to SV_BATCH_MAX_QUBITS) are processed in passes over 2^14-amplitude tiles
 * that each hold every gate of the pass, and the tiles of a pass -- and the
 * chunks of the final expectation sums -- are shared out among all CTAs, so a
 * large state's gate layers run on the whole GPU together with the other
 * states' (a CTA waits, with a bounded wait, until the previous pass of that
 * state has finished). States start as |0...0>. complex64 only. */
#define SV_BATCH_MAX_QUBITS 26
#define SV_BATCH_TILE_QUBITS 14
#define SV_BATCH_KEEP_STATES 1    /* flag: write every final state to d_states */
#define SV_BATCH_CHECK_WAIT 2     /* flag, diagnostic of device-side failure detection: every wait of the
                                     launch is for one more pass than the state will ever finish, bounded
                                     to about 0.1 s; sv_batch_results then returns SV_ERR_TIMEOUT */

typedef struct {
    int n_qubits;           /* 1..SV_BATCH_MAX_QUBITS */
    int gate_begin;         /* the state's gates: gates[gate_begin .. gate_begin + n_gates) */
    int n_gates;
    int pauli_begin;        /* its strings: n_strings rows of n_qubits codes (0=I,1=X,2=Y,3=Z) at
                               paulis[pauli_begin + s * n_qubits + q], code for qubit q */
    int n_strings;
    int out_begin;          /* its expectation values: out[out_begin .. out_begin + n_strings) */
    uint64_t state_offset;  /* amplitude offset of the state in d_states (2^n_qubits amplitudes) */
} sv_batch_item_t;

typedef struct sv_batch_ctx *sv_batch_t;

/* Create / destroy a batch engine bound to a cudaStream_t (NULL = legacy
 * default stream). Creation allocates nothing on the device; the first
 * launch allocates a program buffer, which grows as needed and is freed by
 * destroy. */
SV_API sv_status_t sv_batch_create(void *stream, sv_batch_t *out);
SV_API sv_status_t sv_batch_destroy(sv_batch_t b);

/* Compile the batch on the host (no GPU work): per state, greedy fusion into
 * blocks of at most fusion_width (1..4) qubits, exact structure analysis
 * (controls, diagonal, generalized permutation, dense), and passes of at most
 * 14 local qubits (sv_batch_compile_ex: tile_qubits). Each gate: 1..4
 * targets, at most 8 controls, all qubits distinct and < n_qubits,
 * targets + controls <= min(n_qubits, 14).
 * Errors: INVALID_ARGUMENT for any bad field; NOT_SUPPORTED for a fused block
 * the batch kernel cannot take. Replaces any previous program. */
SV_API sv_status_t sv_batch_compile(sv_batch_t b, const sv_batch_item_t *items, int n_items,
                                    const sv_gate_t *gates, int n_gates_total, const int *paulis,
                                    int fusion_width);

/* Compile options. window_qubits bounds the register windows: runs of ops
 * with at most 2 targets on at most that many local qubits applied to
 * amplitudes held in registers, one shared-memory round trip per run (0 = no
 * windows, else 2..4; tiles under 13 qubits use narrower windows so that every
 * thread keeps a group). keep_permutations changes the fusion pass (Sec.
 * II-B) only in which block a gate joins. tile_qubits is the number of local
 * qubits of a pass: a state of at most that many qubits stays in shared
 * memory for its whole circuit, a larger one is processed in passes over
 * 2^tile_qubits-amplitude tiles, and every gate's targets + controls must
 * not exceed min(n_qubits, tile_qubits). sv_batch_compile uses
 * window_qubits = 4, keep_permutations = 0, tile_qubits = 14. */
typedef struct {
    int fusion_width;       /* 1..4 */
    int window_qubits;      /* 0, 2, 3 or 4 */
    int keep_permutations;  /* 0 or 1: blocks of permutation gates (CNOT, X, ...) take no other gate, so
                               that they stay register exchanges instead of becoming dense products */
    int tile_qubits;        /* 10..SV_BATCH_TILE_QUBITS */
} sv_batch_options_t;

/* sv_batch_compile with explicit options; errors as sv_batch_compile, and
 * INVALID_ARGUMENT for options out of range or NULL. */
SV_API sv_status_t sv_batch_compile_ex(sv_batch_t b, const sv_batch_item_t *items, int n_items,
                                       const sv_gate_t *gates, int n_gates_total, const int *paulis,
                                       const sv_batch_options_t *options);

/* Sizes of the compiled program and the engine's launch count. Any pointer may be NULL. */
SV_API sv_status_t sv_batch_info(sv_batch_t b, int *n_items, int *n_stages, int *n_ops,
                                 uint64_t *state_amps, uint64_t *launches);

/* What the compiled program does, counted on the host (no GPU work): entry
 * [0] dense ops applied on their own (one pass over the tile each), [1]
 * diagonal ops, [2] permutation ops, [3] register windows, then the windows'
 * sub-ops: [4] 2x2 products, [5] of those, products fused with a CNOT-type
 * exchange before or after them, [6] 4x4 products, [7] exchanges and other
 * permutations on their own, [8] diagonals. Counts are per program (a stage
 * that runs over many tiles counts once). */
#define SV_BATCH_STATS 9
SV_API sv_status_t sv_batch_program_stats(sv_batch_t b, uint64_t counts[SV_BATCH_STATS]);

/* Upload the program and enqueue the one persistent kernel. d_states: device
 * memory of at least the largest state_offset + 2^n_qubits complex64
 * amplitudes, 16-byte aligned, caller-owned; states above 14 qubits always use
 * it, smaller ones only with SV_BATCH_KEEP_STATES. dtype must be SV_C64.
 * A program of no states launches nothing and accepts d_states = NULL.
 * Asynchronous. */
SV_API sv_status_t sv_batch_launch(sv_batch_t b, sv_dtype_t dtype, void *d_states, int flags);

/* Wait for the last launch and copy its expectation values (FP64, indexed by
 * out_begin + s) to host memory `out` of at least n_out doubles. Returns
 * SV_ERR_TIMEOUT if a CTA's bounded wait for another CTA's pass gave up (the
 * launch then stopped early and its results are not valid). The expectation
 * sums of a state above SV_BATCH_TILE_QUBITS qubits are formed per chunk of
 * its amplitudes and added in chunk order, so every value depends only on
 * that state's circuit and strings, never on the rest of the batch. */
SV_API sv_status_t sv_batch_results(sv_batch_t b, double *out, int n_out);

/* ---- State memory pool ----
 * A buddy allocator of state vectors inside one arena of device memory that
 * the caller allocated once and owns (Sec. II-A, relaxed memory model: the
 * library does not allocate state memory). A state of n qubits takes a block
 * of 2^n amplitudes, a power of two of bytes, so blocks are powers of two
 * aligned to their size and freeing merges buddies. Pure host bookkeeping:
 * no call touches the arena or calls CUDA; calls are thread-safe. A serving
 * loop admits a request when sv_pool_alloc finds its block (fragmentation
 * included) and returns the block when the request finishes, so no device
 * allocation happens per request. */
typedef struct sv_pool_ctx *sv_pool_t;

/* Pool over [d_base, d_base + bytes). d_base 256-byte aligned; min_block_bytes
 * a power of two >= 256 (smaller requests are rounded up to it). An arena that
 * is not a power of two is cut into maximal aligned power-of-two roots; bytes
 * beyond the last whole min block are not used. Errors: INVALID_ARGUMENT,
 * ALLOC (host memory). */
SV_API sv_status_t sv_pool_create(void *d_base, uint64_t bytes, uint64_t min_block_bytes, sv_pool_t *out);
SV_API sv_status_t sv_pool_destroy(sv_pool_t p);

/* *d_out = the lowest-addressed free block of the smallest power of two >=
 * bytes (and >= the minimum block). INSUFFICIENT_WORKSPACE when no free block
 * is large enough (nothing changes). */
SV_API sv_status_t sv_pool_alloc(sv_pool_t p, uint64_t bytes, void **d_out);

/* Return a block obtained from sv_pool_alloc. INVALID_ARGUMENT for a pointer
 * that is not an allocated block of this pool (nothing changes). */
SV_API sv_status_t sv_pool_free(sv_pool_t p, void *d_ptr);

/* Bytes in allocated blocks, the largest free block, and the usable capacity
 * (any pointer may be NULL). */
SV_API sv_status_t sv_pool_stats(sv_pool_t p, uint64_t *bytes_in_use, uint64_t *largest_free_block,
                                 uint64_t *capacity);

/* A static description of a status code. */
SV_API const char *sv_status_string(sv_status_t s);

#ifdef __cplusplus
}
#endif

#endif /* SV_GB300_SV_H */
