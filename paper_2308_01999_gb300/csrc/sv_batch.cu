// sv_batch.cu -- host side of the batched small-state engine (include/sv.h,
// "Batched small state vectors"): compile many independent circuits into one
// program and run it in one persistent launch (k_batch.cu).
//
// Per state: the gates are fused greedily into blocks of at most
// `fusion_width` qubits (Sec. II-B, the same pass as sv_apply_fused), every
// block goes through the exact structure analysis of sv_apply_matrix
// (controls extracted; diagonal / generalized-permutation / dense), and the
// resulting ops are grouped into stages of at most 14 local qubits with the
// same commutation-aware greedy rule (an op may join any stage at or after the
// last stage touching its qubits). Compilation is host-only; the program is
// uploaded and run by sv_batch_launch.
#include <algorithm>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "sv_classify.h"
#include "sv_fuse.h"
#include "sv_internal.h"

using cd = std::complex<double>;

struct sv_batch_ctx {
    cudaStream_t stream = nullptr;
    int device = -1;
    int num_sms = 0;
    // compiled program (host)
    std::vector<svk::BItem> items;
    std::vector<svk::BStage> stages;
    std::vector<svk::BOp> ops;
    std::vector<float2> pool;
    std::vector<svk::BStr> strs;
    std::vector<svk::BTask> tasks;
    uint32_t n_parts = 0;        // FP64 partial sums of the split states
    int n_out = 0;
    uint64_t state_amps = 0;     // amplitudes the states need in d_states
    bool compiled = false;
    // device copy
    char *dbuf = nullptr;
    size_t dbuf_bytes = 0;
    double *d_out = nullptr;
    int *d_status = nullptr;
    bool uploaded = false;       // the device copy holds the current program
    uint64_t launches = 0;
};

namespace {

using svc::Gate;

struct QOp {                     // an op in global qubit numbering
    int kind;
    std::vector<int> t, c, cv;   // targets (ascending for dense/perm), controls, values
    std::vector<cd> data;        // dense: D*D; diag: D; perm: factors (D) then destinations (D, as numbers)
    uint64_t qmask;
};

bool gate_ok(const sv_gate_t &g, int n, int tile_qubits) {
    if (g.n_targets < 1 || g.n_targets > 4 || g.n_controls < 0 || g.n_controls > 8 || !g.matrix ||
        g.n_targets + g.n_controls > std::min(n, tile_qubits))
        return false;
    uint64_t seen = 0;
    for (int i = 0; i < g.n_targets + g.n_controls; ++i) {
        const int q = i < g.n_targets ? g.targets[i] : g.controls[i - g.n_targets];
        if (q < 0 || q >= n || ((seen >> q) & 1u)) return false;
        seen |= 1ull << q;
    }
    for (int i = 0; i < g.n_controls; ++i)
        if (g.control_values[i] != 0 && g.control_values[i] != 1) return false;
    return true;
}

// exact structure analysis of one (fused) gate -> at most one op
// A dense two-target gate M (bit j of its index on target t[j]) that is a
// CNOT P between its targets (control bit c with value v, target bit 1 - c)
// times a 2x2 gate K on one target alone, M = P K or M = K P: the factors in
// the order they apply. Gate fusion (Sec. II-B) makes such blocks whenever a
// CNOT meets a one-qubit gate on only one of its qubits; as one 4x4 product
// they cost twice the arithmetic of K followed by an exchange. P is its own
// inverse, so K = P M or M P, which must have the form K (x) I up to 1e-12.
bool split_cx(const Gate &g, Gate &first, Gate &second) {
    if (g.t.size() != 2) return false;
    constexpr double kTol = 1e-12;
    const std::vector<cd> &M = g.m;
    for (int c = 0; c < 2; ++c)
        for (int v = 0; v < 2; ++v) {
            const int t = 1 - c;
            auto pidx = [&](int i) { return ((i >> c) & 1) == v ? (i ^ (1 << t)) : i; };
            for (int order = 0; order < 2; ++order) {
                cd N[16];
                for (int r = 0; r < 4; ++r)
                    for (int q = 0; q < 4; ++q) N[r * 4 + q] = order == 0 ? M[pidx(r) * 4 + q] : M[r * 4 + pidx(q)];
                for (int j = 0; j < 2; ++j) {           // K acts on target bit j
                    const int o = 1 - j;
                    cd B[4];
                    bool ok = true;
                    // rows in increasing order: a row with bit o set comes after its partner
                    for (int r = 0; r < 4 && ok; ++r)
                        for (int q = 0; q < 4 && ok; ++q) {
                            const cd x = N[r * 4 + q];
                            if (((r >> o) & 1) != ((q >> o) & 1)) {
                                ok = std::abs(x) <= kTol;
                            } else {
                                cd &b = B[((r >> j) & 1) * 2 + ((q >> j) & 1)];
                                if (((r >> o) & 1) == 0) b = x;
                                else ok = std::abs(x - b) <= kTol;
                            }
                        }
                    if (!ok) continue;
                    Gate K{{g.t[j]}, g.c, g.cv, {B[0], B[1], B[2], B[3]}};
                    Gate X{{g.t[t]}, g.c, g.cv, {cd(0), cd(1), cd(1), cd(0)}};
                    X.c.push_back(g.t[c]);
                    X.cv.push_back(v);
                    first = order == 0 ? K : X;
                    second = order == 0 ? X : K;
                    return true;
                }
            }
        }
    return false;
}

bool classify(Gate g, std::vector<QOp> &out, bool split) {
    svc::simplify_controls(g);
    const int k = (int)g.t.size();
    QOp op;
    op.c = g.c;
    op.cv = g.cv;
    if (k == 0) {
        if (g.m[0] == cd(1)) return true;            // identity
        op.kind = svk::BOP_DIAG;
        op.data = {g.m[0]};
    } else if (svc::is_diagonal(g)) {
        op.kind = svk::BOP_DIAG;
        op.t = g.t;
        const int D = 1 << k;
        for (int j = 0; j < D; ++j) op.data.push_back(g.m[j * D + j]);
    } else {
        svc::sort_targets(g);
        op.t = g.t;
        std::vector<int> perm;
        std::vector<cd> d;
        const int D = 1 << k;
        if (k > 4) return false;
        Gate f1, f2;
        if (svc::as_permutation(g, perm, d)) {
            // source member l = perm[j] goes to destination j with factor d[j]
            op.kind = svk::BOP_PERM;
            op.data.assign(2 * D, cd(0));
            for (int j = 0; j < D; ++j) {
                op.data[perm[j]] = d[j];
                op.data[D + perm[j]] = cd((double)j, 0);
            }
        } else if (split && split_cx(g, f1, f2)) {
            return classify(f1, out, split) && classify(f2, out, split);
        } else {
            op.kind = svk::BOP_DENSE;
            op.data = g.m;
        }
    }
    op.qmask = 0;
    for (int q : op.t) op.qmask |= 1ull << q;
    for (int q : op.c) op.qmask |= 1ull << q;
    out.push_back(std::move(op));
    return true;
}

int popc64(uint64_t x) { return __builtin_popcountll(x); }

// local position of global qubit q in a stage with local mask lmask
uint8_t local_pos(uint64_t lmask, int q) { return (uint8_t)popc64(lmask & ((1ull << q) - 1ull)); }

// one op in a stage with local mask lm
void emit_op(sv_batch_ctx *b, const QOp &qo, uint64_t lm) {
    svk::BOp op{};
    op.kind = (uint8_t)qo.kind;
    op.k = (uint8_t)qo.t.size();
    for (size_t i = 0; i < qo.t.size(); ++i) op.t[i] = local_pos(lm, qo.t[i]);
    std::vector<int> ins;
    if (qo.kind != svk::BOP_DIAG)
        for (int q : qo.t) ins.push_back(local_pos(lm, q));
    for (int q : qo.c) ins.push_back(local_pos(lm, q));
    std::sort(ins.begin(), ins.end());
    op.np = (uint8_t)ins.size();
    for (size_t i = 0; i < ins.size(); ++i) op.p[i] = (uint8_t)ins[i];
    op.cval = 0;
    for (size_t i = 0; i < qo.c.size(); ++i)
        if (qo.cv[i]) op.cval |= 1u << local_pos(lm, qo.c[i]);
    op.mat = (uint32_t)b->pool.size();
    const int D = 1 << op.k;
    for (size_t i = 0; i < qo.data.size(); ++i) {
        float2 v;
        if (qo.kind == svk::BOP_PERM && (int)i >= D) {
            const int dst = (int)qo.data[i].real();
            std::memcpy(&v.x, &dst, 4);
            v.y = 0.f;
        } else {
            v = make_float2((float)qo.data[i].real(), (float)qo.data[i].imag());
        }
        b->pool.push_back(v);
    }
    b->ops.push_back(op);
}

float2 bits_f2(uint32_t x, uint32_t y) {
    float2 v;
    std::memcpy(&v.x, &x, 4);
    std::memcpy(&v.y, &y, 4);
    return v;
}

// an op that a window can hold: at most 2 targets, all its qubits among <= w
bool windowable(const QOp &qo, int w) {
    if (popc64(qo.qmask) > w || qo.t.size() > 2) return false;
    return qo.kind == svk::BOP_DENSE || qo.kind == svk::BOP_DIAG || qo.kind == svk::BOP_PERM;
}

bool plain_dense1(const QOp &qo) { return qo.kind == svk::BOP_DENSE && qo.t.size() == 1 && qo.c.empty(); }
bool plain_cx(const QOp &qo) {
    return qo.kind == svk::BOP_PERM && qo.t.size() == 1 && qo.c.size() == 1 && qo.data[0] == cd(1, 0) &&
           qo.data[1] == cd(1, 0);
}

// A window item: an op, optionally fused with a plain controlled exchange that
// runs after it (or before it, cx_first).
struct WItemOp {
    int op, cx;
    bool cx_first;
};

// Pairs each plain controlled exchange (CNOT, control value 0 or 1) with an
// uncontrolled one-qubit dense op on one of its qubits: first the nearest
// earlier one, where the ops between them leave that op's qubit alone (the
// dense op moves forward to the exchange and writes its outputs straight into
// the exchanged registers); else the nearest later one under the same
// condition (the dense op moves back to the exchange and reads the exchanged
// registers). Returns the window's items in a valid order.
std::vector<WItemOp> pair_exchanges(const std::vector<QOp> &qops, const std::vector<int> &idx) {
    std::vector<WItemOp> it;
    for (int i : idx) it.push_back({i, -1, false});
    auto mask_of = [&](const WItemOp &w) { return qops[w.op].qmask | (w.cx >= 0 ? qops[w.cx].qmask : 0); };
    for (size_t j = 0; j < it.size(); ++j) {
        const QOp &cx = qops[it[j].op];
        if (it[j].cx >= 0 || !plain_cx(cx)) continue;
        bool paired = false;
        uint64_t between = 0;
        for (size_t i = j; i-- > 0;) {
            const QOp &o = qops[it[i].op];
            if (it[i].cx < 0 && plain_dense1(o) && (o.qmask & cx.qmask)) {
                if ((between & o.qmask) == 0) {            // the dense op moves forward to the exchange
                    it[j] = {it[i].op, it[j].op, false};
                    it.erase(it.begin() + (long)i);
                    --j;
                    paired = true;
                }
                break;
            }
            between |= mask_of(it[i]);
        }
        if (paired) continue;
        between = 0;
        for (size_t i = j + 1; i < it.size(); ++i) {
            const QOp &o = qops[it[i].op];
            if (it[i].cx < 0 && plain_dense1(o) && (o.qmask & cx.qmask)) {
                if ((between & o.qmask) == 0) {            // the dense op moves back to the exchange
                    it[j] = {it[i].op, it[j].op, true};
                    it.erase(it.begin() + (long)i);
                }
                break;
            }
            between |= mask_of(it[i]);
        }
    }
    return it;
}

// a window: the ops (at most 2 targets each, all on the local positions `wq`)
// applied one after another to 2^|wq| amplitudes held in registers
void emit_window(sv_batch_ctx *b, const std::vector<QOp> &qops, const std::vector<int> &idx_in, uint64_t wq,
                 uint64_t lm) {
    const std::vector<WItemOp> items = pair_exchanges(qops, idx_in);
    svk::BOp op{};
    op.kind = svk::BOP_WIN;
    op.k = (uint8_t)items.size();
    std::vector<int> wl;                    // window bit i <-> local position wl[i]
    for (int q = 0; q < 64; ++q)
        if ((wq >> q) & 1u) wl.push_back(local_pos(lm, q));
    std::sort(wl.begin(), wl.end());
    op.np = (uint8_t)wl.size();
    for (size_t i = 0; i < wl.size(); ++i) op.p[i] = (uint8_t)wl[i];
    op.cval = 0;
    op.mat = (uint32_t)b->pool.size();
    auto wbit = [&](int q) {
        const int l = local_pos(lm, q);
        return (int)(std::find(wl.begin(), wl.end(), l) - wl.begin());
    };
    const size_t hdr = b->pool.size();
    b->pool.resize(hdr + 2 * items.size());
    for (size_t s = 0; s < items.size(); ++s) {
        const QOp &qo = qops[items[s].op];
        uint32_t cm = 0, cv = 0;
        for (size_t i = 0; i < qo.c.size(); ++i) {
            cm |= 1u << wbit(qo.c[i]);
            if (qo.cv[i]) cv |= 1u << wbit(qo.c[i]);
        }
        const int k = (int)qo.t.size(), D = 1 << k;
        const int b0 = k > 0 ? wbit(qo.t[0]) : 0, b1 = k > 1 ? wbit(qo.t[1]) : 0;
        const uint32_t moff = (uint32_t)(b->pool.size() - hdr);
        uint32_t kind, wc;
        if (qo.kind == svk::BOP_DIAG) {
            kind = svk::BSUB_DIAG;
            wc = svk::WC_DIAG;
            for (int j = 0; j < D; ++j) b->pool.push_back(make_float2((float)qo.data[j].real(), (float)qo.data[j].imag()));
        } else if (qo.kind == svk::BOP_PERM && k == 1) {
            // the only non-diagonal one-target permutation: member l goes to 1 - l times f[l];
            // with both factors exactly 1 and at most one control it is a plain exchange
            kind = svk::BSUB_SWAP1;
            const bool plain = qo.data[0] == cd(1, 0) && qo.data[1] == cd(1, 0);
            if (plain && cm == 0) {
                wc = svk::WC_XSWAP + b0;
            } else if (plain && popc64(cm) == 1) {
                const int c = __builtin_ctz(cm);
                wc = svk::WC_CXSWAP + (4 * b0 + c) * 2 + ((cv >> c) & 1u);
            } else {
                wc = svk::WC_SWAP1 + b0;
            }
            for (int l = 0; l < 2; ++l) b->pool.push_back(make_float2((float)qo.data[l].real(), (float)qo.data[l].imag()));
        } else {
            kind = k == 1 ? svk::BSUB_DENSE1 : svk::BSUB_DENSE2;
            if (items[s].cx >= 0) {
                const QOp &cx = qops[items[s].cx];
                const int c = wbit(cx.c[0]), t = wbit(cx.t[0]);
                wc = (items[s].cx_first ? svk::WC_CXD1 : svk::WC_D1CX) +
                     (uint32_t)(((b0 == t ? 0 : 12) + svk::wc_opair(c, t)) * 2 + (cx.cv[0] ? 1 : 0));
            } else if (k == 1)
                wc = (cm ? svk::WC_DENSE1C : svk::WC_DENSE1) + b0;
            else
                wc = (cm ? svk::WC_DENSE2C : svk::WC_DENSE2) + svk::wc_pair(b0, b1);
            std::vector<cd> m(D * D, cd(0));
            if (qo.kind == svk::BOP_PERM) {
                for (int l = 0; l < D; ++l) m[(int)qo.data[D + l].real() * D + l] = qo.data[l];
            } else {
                m = qo.data;
            }
            for (int i = 0; i < D * D; ++i) b->pool.push_back(make_float2((float)m[i].real(), (float)m[i].imag()));
        }
        b->pool[hdr + 2 * s] =
            bits_f2(kind | (uint32_t)b0 << 8 | (uint32_t)b1 << 16 | (uint32_t)k << 24, cm | cv << 8 | wc << 16);
        b->pool[hdr + 2 * s + 1] = bits_f2(moff, 0);
    }
    b->ops.push_back(op);
}

// The ops of one stage, in order. With window_qubits >= 2, runs of small ops go
// into windows of at most that many qubits -- fewer when the tile is small, so
// that the 2^(T - w) amplitude groups still give every thread of the CTA work
// -- chosen by the same commutation-aware greedy rule as gate fusion: an op
// joins the window, at or after the last item touching its qubits, that grows
// least while staying within the width.
void emit_stage(sv_batch_ctx *b, const std::vector<QOp> &qops, const std::vector<int> &ids, uint64_t lm, int T,
                int window_qubits) {
    const int wmax = std::min(window_qubits, T - 9);
    if (wmax < 2) {
        for (int i : ids) emit_op(b, qops[i], lm);
        return;
    }
    struct WItem { bool win; uint64_t q; std::vector<int> ops; };
    std::vector<WItem> items;
    std::vector<int> last(64, -1);
    for (int i : ids) {
        const QOp &qo = qops[i];
        int L = -1;
        for (int q = 0; q < 64; ++q)
            if ((qo.qmask >> q) & 1u) L = std::max(L, last[q]);
        if (qo.qmask == 0) L = (int)items.size() - 1;   // a global phase stays in place
        int best = -1;
        if (windowable(qo, wmax)) {
            int best_growth = 1 << 30;
            for (int j = std::max(L, 0); j < (int)items.size(); ++j) {
                if (!items[j].win || items[j].ops.size() >= 64) continue;
                const int growth = popc64(qo.qmask & ~items[j].q);
                if (popc64(items[j].q | qo.qmask) <= wmax && growth < best_growth) {
                    best = j;
                    best_growth = growth;
                }
            }
            if (best < 0) {
                items.push_back({true, 0, {}});
                best = (int)items.size() - 1;
            }
        } else {
            items.push_back({false, 0, {}});
            best = (int)items.size() - 1;
        }
        items[best].q |= qo.qmask;
        items[best].ops.push_back(i);
        for (int q = 0; q < 64; ++q)
            if ((qo.qmask >> q) & 1u) last[q] = best;
    }
    for (const WItem &w : items) {
        // a window needs at least 2 qubits (the kernel instantiates 2..4) and 2 ops
        if (!w.win || w.ops.size() == 1 || popc64(w.q) < 2)
            for (int i : w.ops) emit_op(b, qops[i], lm);
        else
            emit_window(b, qops, w.ops, w.q, lm);
    }
}

}  // namespace

extern "C" {

SV_API sv_status_t sv_batch_create(void *stream, sv_batch_t *out) {
    if (!out) return SV_ERR_INVALID_ARGUMENT;
    sv_batch_ctx *b = new (std::nothrow) sv_batch_ctx();
    if (!b) return SV_ERR_ALLOC;
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    *out = b;
    return SV_OK;
}

SV_API sv_status_t sv_batch_destroy(sv_batch_t b) {
    if (!b) return SV_ERR_INVALID_ARGUMENT;
    if (b->dbuf) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->dbuf);
    }
    delete b;
    return SV_OK;
}

}  // extern "C"

namespace {

constexpr uint64_t kBatchTargetTasks = 4096;   // tile tasks aimed at per launch
constexpr double kBatchCtaShare = 152.0;       // a state holding more than 1/152 of the work is split
constexpr int kBatchChunkQubits = 17;          // one expectation chunk per 2^17 amplitudes

// The work list of a compiled program (see svk::BTask). A state above the tile
// size whose work (amplitudes x passes) exceeds one CTA's share of the launch
// (1/152 of the total, the SM count of the target GPU) is split: each of its
// stages into tasks of equal tile ranges (a power of two of tiles each), its
// expectation sums into n_chunks = min(128, 2^max(0, n - 17)) chunks; any
// other state is one task. Order: stage 0 tasks of every split state, then
// stage 1 of every split state, ..., then their expectation chunks, then the
// one-task states, largest first (as items are stored), which fill the tail.
// A task only waits for tasks earlier in the list.
void build_tasks(sv_batch_ctx *b) {
    const int ni = (int)b->items.size();
    // work of a state: amplitudes times passes (its circuit), the unit of a CTA's share
    auto work = [](const svk::BItem &it) {
        return (double)(it.stage_end - it.stage_begin + 1) * (double)(1ull << it.n);
    };
    double total = 0.0;
    for (const svk::BItem &it : b->items) total += work(it);
    const double share = total / kBatchCtaShare;
    std::vector<char> split(ni, 0);
    uint64_t passes = 0;
    for (int i = 0; i < ni; ++i) {
        svk::BItem &it = b->items[i];
        if (it.n <= it.T) continue;
        split[i] = work(it) > share;
        if (split[i]) passes += (uint64_t)(it.stage_end - it.stage_begin) << (it.n - it.T);
        if (it.n_str > 0) {
            it.n_chunks = 1 << std::min(7, std::max(0, it.n - kBatchChunkQubits));
            if (split[i]) {
                it.part_begin = b->n_parts;
                b->n_parts += (uint32_t)(it.n_chunks * it.n_str);
            }
        } else {
            it.n_chunks = 1;
        }
    }
    // split states: tasks sized so that they number a few thousand, while each
    // stage of a state is still split in at least min(tiles, 8) tasks
    uint32_t coarse = 1;
    while ((uint64_t)coarse * 2 * kBatchTargetTasks <= passes) coarse *= 2;
    std::vector<uint32_t> per_task(ni, 0), tasks_per_stage(ni, 0);
    int max_stages = 0;
    for (int i = 0; i < ni; ++i) {
        if (!split[i]) continue;
        const svk::BItem &it = b->items[i];
        const uint32_t ntiles = 1u << (it.n - it.T);
        per_task[i] = std::max(1u, std::min(ntiles / 8, coarse));
        tasks_per_stage[i] = ntiles / per_task[i];
        max_stages = std::max(max_stages, it.stage_end - it.stage_begin);
    }
    for (int sr = 0; sr < max_stages; ++sr)
        for (int i = 0; i < ni; ++i) {
            const svk::BItem &it = b->items[i];
            if (!split[i] || sr >= it.stage_end - it.stage_begin) continue;
            for (uint32_t k = 0; k < tasks_per_stage[i]; ++k)
                b->tasks.push_back({svk::BT_TILES, i, it.stage_begin + sr, k * per_task[i], (k + 1) * per_task[i],
                                    (uint32_t)sr * tasks_per_stage[i], {0, 0}});
        }
    for (int i = 0; i < ni; ++i) {
        if (!split[i]) continue;
        const svk::BItem &it = b->items[i];
        const uint32_t all = (uint32_t)(it.stage_end - it.stage_begin) * tasks_per_stage[i];
        for (int c = 0; c < (it.n_str > 0 ? it.n_chunks : 0); ++c)
            b->tasks.push_back({svk::BT_EXPECT, i, 0, (uint32_t)c, 0, all, {0, 0}});
    }
    // the rest, one CTA each, largest first (items are stored largest first)
    for (int i = 0; i < ni; ++i) {
        const svk::BItem &it = b->items[i];
        if (split[i]) continue;
        b->tasks.push_back({it.n <= it.T ? svk::BT_STATE : svk::BT_WHOLE, i, 0, 0, 0, 0, {0, 0}});
    }
}

}  // namespace

extern "C" {

SV_API sv_status_t sv_batch_compile(sv_batch_t b, const sv_batch_item_t *items, int n_items, const sv_gate_t *gates,
                                    int n_gates_total, const int *paulis, int fusion_width) {
    const sv_batch_options_t opt{fusion_width, svk::kBatchWinQubits, 0, svk::kBatchTileQubits};
    return sv_batch_compile_ex(b, items, n_items, gates, n_gates_total, paulis, &opt);
}

SV_API sv_status_t sv_batch_compile_ex(sv_batch_t b, const sv_batch_item_t *items, int n_items,
                                       const sv_gate_t *gates, int n_gates_total, const int *paulis,
                                       const sv_batch_options_t *options) {
    if (!options) return SV_ERR_INVALID_ARGUMENT;
    const int fusion_width = options->fusion_width, window_qubits = options->window_qubits;
    const int keep_perm = options->keep_permutations, tile_qubits = options->tile_qubits;
    if (!b || (!items && n_items > 0) || n_items < 0 || fusion_width < 1 || fusion_width > 4 ||
        (n_gates_total > 0 && !gates) || n_gates_total < 0 || window_qubits < 0 || window_qubits == 1 ||
        window_qubits > svk::kBatchWinQubits || (keep_perm != 0 && keep_perm != 1) ||
        tile_qubits < svk::kBatchMinTileQubits || tile_qubits > svk::kBatchTileQubits)
        return SV_ERR_INVALID_ARGUMENT;
    b->compiled = false;
    b->items.clear();
    b->stages.clear();
    b->ops.clear();
    b->pool.clear();
    b->strs.clear();
    b->tasks.clear();
    b->n_parts = 0;
    b->uploaded = false;
    b->d_out = nullptr;
    b->d_status = nullptr;
    b->n_out = 0;
    b->state_amps = 0;
    // largest states first: they take longest, so they start first
    std::vector<int> order(n_items);
    for (int i = 0; i < n_items; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return items[a].n_qubits > items[c].n_qubits; });
    for (int oi : order) {
        const sv_batch_item_t &it = items[oi];
        const int n = it.n_qubits;
        if (n < 1 || n > SV_BATCH_MAX_QUBITS || it.n_gates < 0 || it.gate_begin < 0 ||
            it.gate_begin + it.n_gates > n_gates_total || it.n_strings < 0 || it.out_begin < 0 ||
            (it.n_strings > 0 && (!paulis || it.pauli_begin < 0)))
            return SV_ERR_INVALID_ARGUMENT;
        for (int g = 0; g < it.n_gates; ++g)
            if (!gate_ok(gates[it.gate_begin + g], n, tile_qubits)) return SV_ERR_INVALID_ARGUMENT;
        b->n_out = std::max(b->n_out, it.out_begin + it.n_strings);
        b->state_amps = std::max<uint64_t>(b->state_amps, it.state_offset + (1ull << n));
        // fusion, then structure analysis
        std::vector<svf::Item> fused;
        sv_status_t s = svf::fuse(gates + it.gate_begin, it.n_gates, n, fusion_width, fused, 0, keep_perm != 0);
        if (s != SV_OK) return s;
        // split CNOT-times-one-qubit blocks only where register windows can
        // take the two parts together: without windows each part is a pass
        const int T = std::min(n, tile_qubits);
        const bool split = std::min(window_qubits, T - 9) >= 2;
        std::vector<QOp> qops;
        for (const svf::Item &f : fused) {
            Gate g;
            if (f.passthrough) {
                const sv_gate_t &sg = gates[it.gate_begin + f.gate];
                g.t.assign(sg.targets, sg.targets + sg.n_targets);
                g.c.assign(sg.controls, sg.controls + sg.n_controls);
                g.cv.assign(sg.control_values, sg.control_values + sg.n_controls);
                const int D = 1 << sg.n_targets;
                g.m.resize(D * D);
                for (int i = 0; i < D * D; ++i) g.m[i] = cd(sg.matrix[2 * i], sg.matrix[2 * i + 1]);
            } else {
                g.t = f.qubits;
                g.m = f.m;
            }
            if (!classify(g, qops, split)) return SV_ERR_NOT_SUPPORTED;
        }
        // stages of at most T local qubits
        struct St { uint64_t q; std::vector<int> ops; };
        std::vector<St> sts;
        std::vector<int> last(n, -1);
        for (int oi2 = 0; oi2 < (int)qops.size(); ++oi2) {
            const uint64_t qm = qops[oi2].qmask;
            int L = -1;
            for (int q = 0; q < n; ++q)
                if ((qm >> q) & 1u) L = std::max(L, last[q]);
            int best = -1, best_growth = 1 << 30;
            for (int j = std::max(L, 0); j < (int)sts.size(); ++j) {
                const int growth = popc64(qm & ~sts[j].q);
                if (popc64(sts[j].q | qm) <= T && growth < best_growth) {
                    best = j;
                    best_growth = growth;
                }
            }
            if (best < 0) {
                sts.push_back({0, {}});
                best = (int)sts.size() - 1;
            }
            sts[best].q |= qm;
            sts[best].ops.push_back(oi2);
            for (int q = 0; q < n; ++q)
                if ((qm >> q) & 1u) last[q] = best;
        }
        if (sts.empty()) sts.push_back({0, {}});
        svk::BItem bi{};
        bi.state_off = it.state_offset;
        bi.n = n;
        bi.T = T;
        bi.stage_begin = (int)b->stages.size();
        for (St &st : sts) {
            // fill the local set with the lowest remaining qubits (contiguous tile rows)
            uint64_t lm = st.q;
            for (int q = 0; q < n && popc64(lm) < T; ++q) lm |= 1ull << q;
            svk::BStage bs{};
            bs.lmask = lm;
            for (int q = 0, b2 = 0; q < n; ++q)
                if ((lm >> q) & 1u) bs.lpos[b2++] = (uint8_t)q;
            bs.op_begin = (int)b->ops.size();
            const size_t pool0 = b->pool.size(), ops0 = b->ops.size();
            // windows need the stage's matrices staged in shared memory; if they would
            // not fit, the stage is emitted again op by op
            emit_stage(b, qops, st.ops, lm, T, window_qubits);
            if ((int)(b->pool.size() - pool0) > svk::kBatchStageMat) {
                b->pool.resize(pool0);
                b->ops.resize(ops0);
                emit_stage(b, qops, st.ops, lm, T, 0);
            }
            bs.op_end = (int)b->ops.size();
            bs.pool_begin = bs.op_end > bs.op_begin ? (int)b->ops[bs.op_begin].mat : (int)b->pool.size();
            bs.pool_count = (int)b->pool.size() - bs.pool_begin;
            b->stages.push_back(bs);
        }
        bi.stage_end = (int)b->stages.size();
        // Pauli strings: codes paulis[pauli_begin + s * n + q] act on qubit q
        bi.str_begin = (int)b->strs.size();
        bi.n_str = it.n_strings;
        bi.out_begin = it.out_begin;
        for (int s = 0; s < it.n_strings; ++s) {
            uint64_t x = 0, z = 0;
            int ny = 0;
            for (int q = 0; q < n; ++q) {
                const int p = paulis[(size_t)it.pauli_begin + (size_t)s * n + q];
                if (p < 0 || p > 3) return SV_ERR_INVALID_ARGUMENT;
                if (p == SV_PAULI_X || p == SV_PAULI_Y) x |= 1ull << q;
                if (p == SV_PAULI_Z || p == SV_PAULI_Y) z |= 1ull << q;
                ny += p == SV_PAULI_Y;
            }
            const int r = ny & 3;   // i^{nY}: +Re, -Im, -Re, +Im
            b->strs.push_back({x, z, r & 1, (r == 1 || r == 2) ? -1.f : 1.f});
        }
        b->items.push_back(bi);
    }
    build_tasks(b);
    b->compiled = true;
    return SV_OK;
}

SV_API sv_status_t sv_batch_info(sv_batch_t b, int *n_items, int *n_stages, int *n_ops, uint64_t *state_amps,
                                 uint64_t *launches) {
    if (!b) return SV_ERR_INVALID_ARGUMENT;
    if (n_items) *n_items = (int)b->items.size();
    if (n_stages) *n_stages = (int)b->stages.size();
    if (n_ops) *n_ops = (int)b->ops.size();
    if (state_amps) *state_amps = b->state_amps;
    if (launches) *launches = b->launches;
    return SV_OK;
}

SV_API sv_status_t sv_batch_program_stats(sv_batch_t b, uint64_t counts[SV_BATCH_STATS]) {
    if (!b || !counts || !b->compiled) return SV_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < SV_BATCH_STATS; ++i) counts[i] = 0;
    for (const svk::BOp &op : b->ops) {
        if (op.kind != svk::BOP_WIN) {
            ++counts[op.kind == svk::BOP_DENSE ? 0 : op.kind == svk::BOP_DIAG ? 1 : 2];
            continue;
        }
        ++counts[3];
        for (int s = 0; s < op.k; ++s) {
            uint32_t hy;
            std::memcpy(&hy, &b->pool[op.mat + 2 * s].y, 4);
            const uint32_t wc = hy >> 16;
            if (wc < svk::WC_DENSE2 || wc >= svk::WC_D1CX) {
                ++counts[4];
                if (wc >= svk::WC_D1CX) ++counts[5];
            } else if (wc < svk::WC_SWAP1) {
                ++counts[6];
            } else if (wc < svk::WC_DIAG) {
                ++counts[7];
            } else {
                ++counts[8];
            }
        }
    }
    return SV_OK;
}

SV_API sv_status_t sv_batch_launch(sv_batch_t b, sv_dtype_t dtype, void *d_states, int flags) {
    if (!b || !b->compiled) return SV_ERR_INVALID_ARGUMENT;
    if (dtype != SV_C64) return SV_ERR_NOT_SUPPORTED;
    if (b->items.empty()) return SV_OK;   // nothing to run: d_states may be NULL
    if (!d_states || (reinterpret_cast<uintptr_t>(d_states) & 15u)) return SV_ERR_INVALID_ARGUMENT;
    if (b->device < 0) {
        if (cudaGetDevice(&b->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
            return SV_ERR_CUDA;
    }
    const size_t ni = b->items.size();
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_items = 0;
    const size_t o_stages = align(o_items + ni * sizeof(svk::BItem));
    const size_t o_ops = align(o_stages + b->stages.size() * sizeof(svk::BStage));
    const size_t o_pool = align(o_ops + b->ops.size() * sizeof(svk::BOp));
    const size_t o_strs = align(o_pool + b->pool.size() * sizeof(float2));
    const size_t o_tasks = align(o_strs + b->strs.size() * sizeof(svk::BStr));
    const size_t o_out = align(o_tasks + b->tasks.size() * sizeof(svk::BTask));
    const size_t o_parts = align(o_out + (size_t)b->n_out * sizeof(double));
    // zeroed at every launch: task counter, status word, per-item counters
    const size_t o_zero = align(o_parts + (size_t)b->n_parts * sizeof(double));
    const size_t zero_bytes = 256 + 2 * ni * sizeof(unsigned);
    const size_t total = o_zero + zero_bytes;
    if (total > b->dbuf_bytes) {
        if (b->dbuf) {
            cudaStreamSynchronize(b->stream);
            cudaFree(b->dbuf);
            b->dbuf = nullptr;
            b->dbuf_bytes = 0;
        }
        if (cudaMalloc(reinterpret_cast<void **>(&b->dbuf), total) != cudaSuccess) {
            cudaGetLastError();
            return SV_ERR_ALLOC;
        }
        b->dbuf_bytes = total;
        b->uploaded = false;
    }
    auto up = [&](size_t off, const void *src, size_t bytes) {
        return bytes == 0 ? cudaSuccess
                          : cudaMemcpyAsync(b->dbuf + off, src, bytes, cudaMemcpyHostToDevice, b->stream);
    };
    if (!b->uploaded) {
        if (up(o_items, b->items.data(), ni * sizeof(svk::BItem)) != cudaSuccess ||
            up(o_stages, b->stages.data(), b->stages.size() * sizeof(svk::BStage)) != cudaSuccess ||
            up(o_ops, b->ops.data(), b->ops.size() * sizeof(svk::BOp)) != cudaSuccess ||
            up(o_pool, b->pool.data(), b->pool.size() * sizeof(float2)) != cudaSuccess ||
            up(o_strs, b->strs.data(), b->strs.size() * sizeof(svk::BStr)) != cudaSuccess ||
            up(o_tasks, b->tasks.data(), b->tasks.size() * sizeof(svk::BTask)) != cudaSuccess)
            return SV_ERR_CUDA;
        b->uploaded = true;
    }
    if (cudaMemsetAsync(b->dbuf + o_zero, 0, zero_bytes, b->stream) != cudaSuccess) return SV_ERR_CUDA;
    b->d_out = reinterpret_cast<double *>(b->dbuf + o_out);
    b->d_status = reinterpret_cast<int *>(b->dbuf + o_zero + 128);
    svk::BProg P{};
    P.items = reinterpret_cast<const svk::BItem *>(b->dbuf + o_items);
    P.stages = reinterpret_cast<const svk::BStage *>(b->dbuf + o_stages);
    P.ops = reinterpret_cast<const svk::BOp *>(b->dbuf + o_ops);
    P.pool = reinterpret_cast<const float2 *>(b->dbuf + o_pool);
    P.strs = reinterpret_cast<const svk::BStr *>(b->dbuf + o_strs);
    P.tasks = reinterpret_cast<const svk::BTask *>(b->dbuf + o_tasks);
    P.n_tasks = (int)b->tasks.size();
    P.keep_states = (flags & SV_BATCH_KEEP_STATES) ? 1 : 0;
    P.out = b->d_out;
    P.parts = reinterpret_cast<double *>(b->dbuf + o_parts);
    P.counter = reinterpret_cast<int *>(b->dbuf + o_zero);
    P.status = b->d_status;
    P.tiles_done = reinterpret_cast<unsigned *>(b->dbuf + o_zero + 256);
    P.chunks_done = P.tiles_done + ni;
    P.need_extra = (flags & SV_BATCH_CHECK_WAIT) ? 1u : 0u;
    P.wait_cycles = (flags & SV_BATCH_CHECK_WAIT) ? 200000000LL : svk::kBatchWaitCycles;
    const svk::LaunchCtx L{b->stream, b->num_sms, &b->launches};
    bool split = false;
    for (const svk::BTask &t : b->tasks) split |= t.kind == svk::BT_TILES || t.kind == svk::BT_EXPECT;
    const cudaError_t e = svk::launch_batch(L, reinterpret_cast<float2 *>(d_states), P, split);
    return e == cudaSuccess ? SV_OK : SV_ERR_CUDA;
}

SV_API sv_status_t sv_batch_results(sv_batch_t b, double *out, int n_out) {
    if (!b || !b->compiled || (!out && n_out > 0) || n_out < b->n_out) return SV_ERR_INVALID_ARGUMENT;
    if (!b->d_status) {   // nothing launched since the last compile
        if (b->n_out > 0) return SV_ERR_INVALID_ARGUMENT;
        return cudaStreamSynchronize(b->stream) == cudaSuccess ? SV_OK : SV_ERR_CUDA;
    }
    int status = 0;
    if (b->n_out > 0 &&
        cudaMemcpyAsync(out, b->d_out, sizeof(double) * b->n_out, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return SV_ERR_CUDA;
    if (cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return SV_ERR_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SV_ERR_CUDA;
    return status == 0 ? SV_OK : SV_ERR_TIMEOUT;
}

}  // extern "C"
