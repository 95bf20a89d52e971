// sv_fuse.h -- host gate fusion (Sec. II-B; max_fused_gate_size, Sec. II-D-1).
#pragma once

#include <complex>
#include <vector>

#include "sv.h"

namespace svf {

using cd = std::complex<double>;

// A run of the plan: either a fused block (dense matrix on `qubits`, bit j of
// the matrix index is qubits[j]) or one gate passed through unchanged because
// it acts on more qubits than the fusion width allows.
struct Item {
    bool passthrough = false;
    int gate = -1;               // index into the input gates (passthrough only)
    std::vector<int> qubits;     // fused block qubits
    std::vector<cd> m;           // 2^k x 2^k row-major, k = qubits.size()
    int n_gates = 0;             // gates absorbed
    bool diagonal = false;       // a block of diagonal gates only (its matrix is diagonal)
    bool perm_only = true;       // every absorbed gate is a generalized permutation
};

// Greedy fusion in program order. A gate joins the open block that needs the
// fewest new qubits among the blocks at or after the last block touching any
// of its qubits (so it only moves past blocks on disjoint qubits, with which it
// commutes), provided the block stays within `width` qubits; otherwise it opens
// a new block. Block matrices are composed in FP64.
//
// With diag_width > 0, diagonal gates (Sec. II-D-1, dense/diagonal fusion) go
// to separate diagonal blocks of at most diag_width qubits instead: since
// diagonal matrices commute, such a gate may join any diagonal block after the
// last non-diagonal item touching its qubits. Dense blocks then take only the
// other gates.
//
// With keep_permutations, a block that holds only generalized-permutation
// gates (CNOT, X, SWAP and the like) takes no other gate: an engine that
// applies permutations as register exchanges then keeps them free instead of
// paying a dense product for them (a later rotation opens or joins another
// block). Permutation gates may still join dense blocks.
sv_status_t fuse(const sv_gate_t *gates, int n_gates, int n_qubits, int width, std::vector<Item> &out,
                 int diag_width = 0, bool keep_permutations = false);

// psi <- G psi for a (controlled) k-qubit gate on an s-qubit vector (host, FP64);
// used to compose block matrices column by column.
void apply_small(cd *psi, int s, const int *targets, int k, const int *controls, const int *cvals, int c,
                 const cd *m);

}  // namespace svf
