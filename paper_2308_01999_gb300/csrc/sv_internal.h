// sv_internal.h -- types shared by the host API and the kernels of libsv.so.
//
// Index geometry. For a gate with k targets and c controls on an n-qubit
// state, the 2^(n-k-c) amplitude groups are numbered g = 0, 1, ...; the first
// amplitude of group g is g with a zero bit inserted at every target and
// control position (in ascending order), with the control bits then set to
// their required values (Sec. II-C: each index bit is one qubit). Member j of
// the group adds bit t of j at target position t.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sv.h"

namespace svk {

constexpr int kMaxSpecial = SV_MAX_TARGETS + SV_MAX_CONTROLS;

// Sorted positions at which zero bits are inserted, plus the bits forced to 1.
struct GroupGeom {
    int ns;                 // number of inserted positions
    int pos[kMaxSpecial];   // ascending
    uint64_t cset;          // control bits whose required value is 1
};

// 1 << targets[t], targets ascending.
struct TargetOffs {
    uint64_t t[SV_MAX_TARGETS];
};

// Launch bookkeeping shared by every launch wrapper.
struct LaunchCtx {
    cudaStream_t stream;
    int num_sms;
    uint64_t *launches;     // incremented once per kernel launch
};

// ---- gate kernels (k_gate.cu) ----
// Dense 2^k x 2^k product on every group, k = 1..6. `mat` is row-major
// complex128 for targets in ascending order. `d_mat` is workspace for k >= 5.
cudaError_t launch_dense(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const GroupGeom &G,
                         const int *tpos, int k, const double *mat, void *d_mat);
// Diagonal d[j] on targets (any order; j's bit t is targets[t]) where controls hold, k = 0..6.
cudaError_t launch_diag(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const GroupGeom &Gctl,
                        const int *tpos, int k, const double *diag);
// Generalized permutation: out[j] = d[j] * in[perm[j]] per group, k = 1..4, targets ascending.
cudaError_t launch_perm(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const GroupGeom &G,
                        const int *tpos, int k, const int *perm, const double *d);

// Index-bit swap: bits a[k] <-> b[k] of every amplitude index (disjoint pairs, np <= 18).
cudaError_t launch_swap(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const int *a, const int *b, int np);

// psi <- exp(i theta P) psi, P given by its X|Y mask x, Z|Y mask z and Y count ny.
cudaError_t launch_pauli_rotation(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, uint64_t x, uint64_t z, int ny,
                                  double theta);

// ---- reductions (k_reduce.cu) ----
struct PauliPass {
    int S;              // strings in this pass (1..8)
    uint64_t x;         // common X|Y mask
    uint64_t z[8];      // Z|Y mask per string
    int use_im[8];      // take Im(w) instead of Re(w) (odd number of Y)
    double sign[8];     // +1 / -1 from i^{nY}
};
constexpr int kPauliMaxS = 8;
// Writes S doubles at d_out (device).
cudaError_t launch_pauli(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, const PauliPass &P,
                         double *d_partials, int max_partial_blocks, double *d_out);
// d_out[0] = sum over even parity of mask, d_out[1] = odd.
cudaError_t launch_parity(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, uint64_t mask,
                          double *d_partials, int max_partial_blocks, double *d_out);
cudaError_t launch_collapse(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, uint64_t mask,
                            int parity, double scale);
// d_out[q] = <Z_q> for q < n and d_out[n] = <psi|psi>, one pass (3 <= n <= 40).
cudaError_t launch_zall(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, double *d_partials,
                        int max_partial_blocks, double *d_out);
// Sampler: basis indices at which the cumulative probability first exceeds
// r * total, for each r. d_seg: workspace of at least 2^20 doubles; d_r / d_out:
// n_samples doubles / int64 (device). Segment size 2^max(12, n - 20).
cudaError_t launch_sample(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, const double *d_r, int n_samples,
                          double *d_seg, long long *d_out);
cudaError_t launch_set_basis(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, uint64_t index);

// ---- tensor-core fused apply (k_tc.cu) ----
// psi <- G psi for a 6-target block with G given as 64x64 complex128,
// targets ascending; prec = SV_PREC_TF32 or SV_PREC_SPLIT_BF16; c64 only.
// d_a: workspace for the staged operand (>= 64 KiB); d_err: device status word.
cudaError_t launch_tc6(const LaunchCtx &L, void *sv, int n, const int *tpos, const double *mat,
                       sv_precision_t prec, void *d_a, int *d_err);
bool tc6_supported(int n, const int *tpos);
// Bounded-wait diagnostic: a wait that nothing completes, limited to `cycles` clocks.
cudaError_t launch_wait_probe(const LaunchCtx &L, int *d_err, long long cycles);

// ---- batched small states (k_batch.cu, sv_batch.cu) ----
// One persistent launch advances many independent states. Each state's gates
// are compiled into ops on local bit positions of a tile of 2^T amplitudes
// (T = min(n, the compile's tile size <= kBatchTileQubits)) and grouped into stages: a stage names T
// "local" qubits (lmask) and its ops act on local qubits only, so one pass
// over the state -- 2^(n-T) tiles, each gathered into shared memory once --
// applies all of them.
constexpr int kBatchTileQubits = 14;
constexpr int kBatchMinTileQubits = 10;   // smallest tile a compile option may ask for (2 amplitudes a thread)
constexpr int kBatchThreads = 512;
enum BatchOpKind { BOP_DENSE = 0, BOP_DIAG = 1, BOP_PERM = 2, BOP_WIN = 3 };
// A window (BOP_WIN) applies a run of small ops to amplitudes held in registers:
// its np <= kBatchWinQubits local positions p[] span 2^np amplitudes per thread,
// k is the number of sub-ops, and pool[mat ..] holds k two-entry headers
// (kind | b0 << 8 | b1 << 16 | nd << 24, control mask | control values << 8 |
// case << 16, matrix offset from pool[mat], 0) followed by their matrices.
constexpr int kBatchWinQubits = 4;
enum BatchSubKind { BSUB_DENSE1 = 0, BSUB_DENSE2 = 1, BSUB_DIAG = 2, BSUB_SWAP1 = 3 };
// The sub-op's case: the kernel jumps on it once, into code whose window bits
// (and, for plain swaps, whose control) are compile-time constants.
enum BatchWinCase {
    WC_DENSE1 = 0,     // + b: 2x2 on window bit b, no control
    WC_DENSE1C = 4,    // + b: 2x2 where (r & cm) == cv
    WC_DENSE2 = 8,     // + wc_pair(b0, b1): 4x4 on bits b0 < b1, no control
    WC_DENSE2C = 14,   // + wc_pair(b0, b1): 4x4 where (r & cm) == cv
    WC_SWAP1 = 20,     // + b: member l -> 1 - l times f[l], where (r & cm) == cv
    WC_XSWAP = 24,     // + b: members exchanged (factors exactly 1), no control
    WC_CXSWAP = 28,    // + (4 b + c) * 2 + v: members exchanged where window bit c == v (c != b)
    WC_DIAG = 60,      // diagonal, run-time bits and control
    WC_D1CX = 64,      // + ((s ? 12 : 0) + wc_opair(c, t)) * 2 + v: 2x2 on bit t (s = 0) or c (s = 1),
                       //   then members exchanged across bit t where bit c == v
    WC_CXD1 = 112,     // + ((s ? 12 : 0) + wc_opair(c, t)) * 2 + v: members exchanged across bit t where
                       //   bit c == v, then a 2x2 on bit t (s = 0) or c (s = 1)
};
// index of the pair b0 < b1 < 4 among 01 02 03 12 13 23
constexpr __host__ __device__ int wc_pair(int b0, int b1) { return b0 * (7 - b0) / 2 + (b1 - b0 - 1); }
// index of the ordered pair (c, t), c != t < 4
constexpr __host__ __device__ int wc_opair(int c, int t) { return c * 3 + (t > c ? t - 1 : t); }

struct BItem {
    uint64_t state_off;      // amplitude offset of the state
    int n, T;                // qubits, tile qubits
    int stage_begin, stage_end;
    int str_begin, n_str;    // Pauli strings
    int out_begin;
    int n_chunks;            // states above the tile size: expectation chunks
    uint32_t part_begin;     // their FP64 partial sums: parts[part_begin + chunk * n_str + s]
    uint32_t pad;
};

struct BStage {
    uint64_t lmask;          // the T local qubits
    int op_begin, op_end;
    int pool_begin, pool_count;   // the stage's matrices: pool[pool_begin .. pool_begin + pool_count)
    uint8_t lpos[16];        // the qubit at local position b (b < T), ascending
};
constexpr int kBatchStageMat = 4096;   // float2 entries of one stage staged in shared memory at once

struct BOp {
    uint8_t kind, k, np, nt;  // kind, targets, inserted positions, (unused)
    uint8_t t[4];             // local target positions (ascending for dense / perm)
    uint8_t p[12];            // local inserted positions, ascending (targets + controls; controls only for diag)
    uint32_t cval;            // local control bits that must be 1
    uint32_t mat;             // offset into the matrix pool (float2 units)
    uint32_t pad[2];
};

struct BStr {
    uint64_t x, z;           // X|Y and Z|Y masks
    int use_im;              // odd number of Y: take Im(w)
    float sign;              // from i^{nY}
};

// The persistent kernel's work list, taken in order from an atomic counter.
// A state of at most T qubits is one BT_STATE task (its whole
// circuit in shared memory). A larger state is either one BT_WHOLE task (one
// CTA runs every pass and the expectation sums, so the state stays warm in L2
// between its passes) or, when it holds more work than one CTA's share of the
// launch, split so that many CTAs share it: one BT_TILES task per range of
// tiles of each stage, and one BT_EXPECT task per chunk of its expectation
// sums. Both forms add the same per-chunk partial sums in the same order. A task may start only when `need`
// tile tasks of its state have finished (all of the previous stage, or all
// stages for BT_EXPECT); every task a task waits for comes earlier in the
// list, so the earliest unfinished task can always run.
enum BatchTaskKind { BT_STATE = 0, BT_TILES = 1, BT_EXPECT = 2, BT_WHOLE = 3 };
struct BTask {
    int kind, item;
    int stage;               // BT_TILES: absolute stage index
    uint32_t a, b;           // BT_TILES: tiles [a, b); BT_EXPECT: chunk a
    uint32_t need;           // finished tile tasks of the item required first
    uint32_t pad[2];
};

// Device pointers of one uploaded program.
struct BProg {
    const BItem *items;
    const BStage *stages;
    const BOp *ops;
    const float2 *pool;
    const BStr *strs;
    const BTask *tasks;
    int n_tasks;
    int keep_states;
    double *out;             // expectation values
    double *parts;           // per-chunk partial sums of the split states
    unsigned *tiles_done;    // per item: finished BT_TILES tasks
    unsigned *chunks_done;   // per item: finished BT_EXPECT tasks
    int *counter;            // next task
    int *status;             // 0, or the timeout code of a wait that gave up
    unsigned need_extra;     // diagnostic: added to every wait's target (0 in normal runs)
    long long wait_cycles;   // bound of each wait
};
constexpr int kBatchErrTimeout = 0x7c02;
constexpr long long kBatchWaitCycles = 4000000000LL;   // ~2 s of SM clock per wait

// split: the program holds split states (tile and expectation tasks)
cudaError_t launch_batch(const LaunchCtx &L, float2 *states, const BProg &P, bool split);

}  // namespace svk
