// sv_fuse.cpp -- host gate fusion (Sec. II-B: fusing many small gate matrices
// into one multi-qubit matrix applied in one pass; the width limit is qsim's
// max_fused_gate_size, Sec. II-D-1).
//
// The paper gives the idea and the width option, not an algorithm; the one here
// is a greedy pass in program order that may move a gate earlier only past
// blocks that share no qubit with it (such gates commute, so the product is
// unchanged). Block matrices are composed in FP64 by applying each absorbed
// gate to every column of the block matrix.
#include "sv_fuse.h"

#include <algorithm>
#include <cstdint>

namespace svf {

void apply_small(cd *psi, int s, const int *targets, int k, const int *controls, const int *cvals, int c,
                 const cd *m) {
    const uint64_t N = 1ull << s, D = 1ull << k;
    uint64_t tmask = 0, cmask = 0, cwant = 0;
    for (int t = 0; t < k; ++t) tmask |= 1ull << targets[t];
    for (int t = 0; t < c; ++t) {
        cmask |= 1ull << controls[t];
        if (cvals[t]) cwant |= 1ull << controls[t];
    }
    uint64_t off[64];
    for (uint64_t j = 0; j < D; ++j) {
        uint64_t o = 0;
        for (int t = 0; t < k; ++t)
            if ((j >> t) & 1) o |= 1ull << targets[t];
        off[j] = o;
    }
    cd in[64];
    for (uint64_t b = 0; b < N; ++b) {
        if ((b & tmask) || (b & cmask) != cwant) continue;
        for (uint64_t l = 0; l < D; ++l) in[l] = psi[b | off[l]];
        for (uint64_t j = 0; j < D; ++j) {
            cd acc = 0;
            for (uint64_t l = 0; l < D; ++l) acc += m[j * D + l] * in[l];
            psi[b | off[j]] = acc;
        }
    }
}

namespace {

int local_index(const std::vector<int> &qs, int q) {
    for (size_t i = 0; i < qs.size(); ++i)
        if (qs[i] == q) return (int)i;
    return -1;
}

// Grow the block to include `extra` qubits (appended as higher index bits):
// B <- I (x) B.
void grow(Item &b, const std::vector<int> &extra) {
    if (extra.empty()) return;
    const int s = (int)b.qubits.size();
    const int s2 = s + (int)extra.size();
    const uint64_t d = 1ull << s, d2 = 1ull << s2;
    std::vector<cd> m2(d2 * d2, cd(0));
    for (uint64_t r = 0; r < d2; ++r)
        for (uint64_t c = 0; c < d2; ++c)
            if ((r >> s) == (c >> s)) m2[r * d2 + c] = b.m[(r & (d - 1)) * d + (c & (d - 1))];
    b.m.swap(m2);
    b.qubits.insert(b.qubits.end(), extra.begin(), extra.end());
}

// B <- G B, G the gate embedded in the block's basis. G mixes, within each
// group of block rows that differ only in the gate's target bits (and satisfy
// its controls), the rows base | off[l]; each new row is the sum over l of
// G[j][l] times row l, taken in ascending l -- the same sums, in the same order,
// as applying G to every column, but on contiguous rows.
void absorb(Item &b, const sv_gate_t &g) {
    std::vector<int> extra;
    for (int t = 0; t < g.n_targets + g.n_controls; ++t) {
        const int q = t < g.n_targets ? g.targets[t] : g.controls[t - g.n_targets];
        if (local_index(b.qubits, q) < 0) extra.push_back(q);
    }
    grow(b, extra);
    const int s = (int)b.qubits.size();
    const uint64_t d = 1ull << s, D = 1ull << g.n_targets;
    uint64_t tmask = 0, cmask = 0, cwant = 0;
    uint64_t off[64];
    for (uint64_t j = 0; j < D; ++j) off[j] = 0;
    for (int t = 0; t < g.n_targets; ++t) {
        const uint64_t bit = 1ull << local_index(b.qubits, g.targets[t]);
        tmask |= bit;
        for (uint64_t j = 0; j < D; ++j)
            if ((j >> t) & 1) off[j] |= bit;
    }
    for (int t = 0; t < g.n_controls; ++t) {
        const uint64_t bit = 1ull << local_index(b.qubits, g.controls[t]);
        cmask |= bit;
        if (g.control_values[t]) cwant |= bit;
    }
    std::vector<cd> gm(D * D), tmp(D * d);
    for (uint64_t i = 0; i < D * D; ++i) gm[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
    for (uint64_t base = 0; base < d; ++base) {
        if ((base & tmask) || (base & cmask) != cwant) continue;
        for (uint64_t j = 0; j < D; ++j) {
            cd *out = &tmp[j * d];
            for (uint64_t c = 0; c < d; ++c) out[c] = 0;
            for (uint64_t l = 0; l < D; ++l) {
                const cd m = gm[j * D + l];
                const cd *row = &b.m[(base | off[l]) * d];
                for (uint64_t c = 0; c < d; ++c) out[c] += m * row[c];
            }
        }
        for (uint64_t j = 0; j < D; ++j)
            std::copy(&tmp[j * d], &tmp[j * d] + d, &b.m[(base | off[j]) * d]);
    }
    ++b.n_gates;
}

}  // namespace

bool gate_is_diagonal(const sv_gate_t &g) {
    const int D = 1 << g.n_targets;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            if (r != c && (g.matrix[2 * (r * D + c)] != 0.0 || g.matrix[2 * (r * D + c) + 1] != 0.0)) return false;
    return true;
}

// one nonzero in every row and column
bool gate_is_permutation(const sv_gate_t &g) {
    const int D = 1 << g.n_targets;
    for (int r = 0; r < D; ++r) {
        int nz = 0;
        for (int c = 0; c < D; ++c) nz += g.matrix[2 * (r * D + c)] != 0.0 || g.matrix[2 * (r * D + c) + 1] != 0.0;
        if (nz != 1) return false;
    }
    for (int c = 0; c < D; ++c) {
        int nz = 0;
        for (int r = 0; r < D; ++r) nz += g.matrix[2 * (r * D + c)] != 0.0 || g.matrix[2 * (r * D + c) + 1] != 0.0;
        if (nz != 1) return false;
    }
    return true;
}

sv_status_t fuse(const sv_gate_t *gates, int n_gates, int n_qubits, int width, std::vector<Item> &out,
                 int diag_width, bool keep_permutations) {
    out.clear();
    if (width < 1 || width > SV_MAX_TARGETS || n_qubits < 1 || n_qubits > SV_MAX_QUBITS || n_gates < 0 ||
        diag_width < 0 || diag_width > SV_MAX_TARGETS)
        return SV_ERR_INVALID_ARGUMENT;
    std::vector<int> last(n_qubits, -1);      // latest item touching each qubit
    std::vector<int> last_nd(n_qubits, -1);   // latest non-diagonal item touching each qubit
    constexpr int kScan = 64;                 // blocks examined per gate
    auto new_block = [&](const std::vector<int> &Q, bool diag) {
        Item it;
        it.qubits = Q;
        it.diagonal = diag;
        const uint64_t d = 1ull << Q.size();
        it.m.assign(d * d, cd(0));
        for (uint64_t i = 0; i < d; ++i) it.m[i * d + i] = 1;
        out.push_back(std::move(it));
        return (int)out.size() - 1;
    };
    auto growth_of = [&](const Item &b, const std::vector<int> &Q) {
        int g = 0;
        for (int q : Q)
            if (local_index(b.qubits, q) < 0) ++g;
        return g;
    };
    for (int gi = 0; gi < n_gates; ++gi) {
        const sv_gate_t &g = gates[gi];
        const int nq = g.n_targets + g.n_controls;
        int L = -1, Lnd = -1;
        std::vector<int> Q(nq);
        for (int t = 0; t < nq; ++t) {
            Q[t] = t < g.n_targets ? g.targets[t] : g.controls[t - g.n_targets];
            L = std::max(L, last[Q[t]]);
            Lnd = std::max(Lnd, last_nd[Q[t]]);
        }
        if (diag_width > 0 && nq <= diag_width && gate_is_diagonal(g)) {
            // diagonal blocks after the last non-diagonal item on these qubits
            int best = -1, best_growth = 1 << 30;
            const int lo = std::max({Lnd + 1, 0, (int)out.size() - kScan});
            for (int j = (int)out.size() - 1; j >= lo; --j) {
                const Item &b = out[j];
                if (!b.diagonal) continue;
                const int gr = growth_of(b, Q);
                if ((int)b.qubits.size() + gr <= diag_width && gr < best_growth) {
                    best = j;
                    best_growth = gr;
                }
            }
            if (best < 0) best = new_block(Q, true);
            absorb(out[best], g);
            for (int q : Q) last[q] = std::max(last[q], best);
            continue;
        }
        if (nq > width) {
            Item it;
            it.passthrough = true;
            it.gate = gi;
            it.n_gates = 1;
            out.push_back(std::move(it));
            for (int q : Q) last[q] = last_nd[q] = (int)out.size() - 1;
            continue;
        }
        const bool perm = keep_permutations && gate_is_permutation(g);
        int best = -1, best_growth = 1 << 30;
        const int lo = std::max({L, 0, (int)out.size() - kScan});
        for (int j = (int)out.size() - 1; j >= lo; --j) {
            const Item &b = out[j];
            if (b.passthrough || b.diagonal) continue;
            if (keep_permutations && b.perm_only && b.n_gates > 0 && !perm) continue;
            const int gr = growth_of(b, Q);
            if ((int)b.qubits.size() + gr <= width && gr < best_growth) {
                best = j;
                best_growth = gr;
            }
        }
        if (best < 0) best = new_block(Q, false);
        absorb(out[best], g);
        out[best].perm_only = out[best].perm_only && perm;
        for (int q : Q) last[q] = last_nd[q] = best;
    }
    return SV_OK;
}

}  // namespace svf
