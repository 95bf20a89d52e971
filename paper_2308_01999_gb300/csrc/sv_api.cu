// sv_api.cu -- the C ABI of libsv.so (declared in include/sv.h).
//
// Host side of every call: argument validation, the exact structure analysis of
// a gate matrix (Sec. II-D-1: diagonal and generalized-permutation gates get
// their own cheaper kernels), the workspace owned by the handle (Table I,
// "Resource management"), and dispatch to the kernels in k_gate.cu,
// k_reduce.cu and k_tc.cu. No arithmetic on the state happens on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "sv_classify.h"
#include "sv_fuse.h"
#include "sv_internal.h"

using cd = std::complex<double>;

struct sv_ctx {
    int n = 0;
    sv_dtype_t dt = SV_C64;
    void *sv = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    char *ws = nullptr;
    double *d_partials = nullptr;
    int max_partial_blocks = 0;
    double *d_results = nullptr;
    int max_results = 0;
    int *d_err = nullptr;
    char *d_mat = nullptr;
    size_t mat_bytes = 0;
    double *h_results = nullptr;   // pinned
    uint64_t launches = 0;
};

namespace {

constexpr size_t kPartialBytes = 1u << 20;
constexpr size_t kResultBytes = 64u << 10;
constexpr size_t kErrBytes = 256;
constexpr size_t kMatOffset = 2u << 20;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

svk::LaunchCtx lctx(sv_ctx *h) { return svk::LaunchCtx{h->stream, h->num_sms, &h->launches}; }

sv_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? SV_OK : SV_ERR_CUDA; }

// qubits (targets then controls) in range and pairwise distinct
bool valid_qubits(int n, const int *targets, int k, const int *controls, int c) {
    uint64_t seen = 0;
    for (int i = 0; i < k + c; ++i) {
        const int q = i < k ? targets[i] : controls[i - k];
        if (q < 0 || q >= n || ((seen >> q) & 1u)) return false;
        seen |= 1ull << q;
    }
    return true;
}

using svc::Gate;
using svc::simplify_controls;
using svc::sort_targets;

svk::GroupGeom make_geom(const std::vector<int> &inserted, const std::vector<int> &c, const std::vector<int> &cv) {
    svk::GroupGeom G{};
    std::vector<int> p = inserted;
    std::sort(p.begin(), p.end());
    G.ns = (int)p.size();
    for (int i = 0; i < G.ns; ++i) G.pos[i] = p[i];
    G.cset = 0;
    for (size_t i = 0; i < c.size(); ++i)
        if (cv[i]) G.cset |= 1ull << c[i];
    return G;
}

sv_status_t apply_gate(sv_ctx *h, Gate g, sv_precision_t prec) {
    simplify_controls(g);
    const int k = (int)g.t.size();
    const svk::LaunchCtx L = lctx(h);
    std::vector<double> buf;
    if (k == 0) {
        // a phase on the subspace where every control holds
        if (g.m[0] == cd(1)) return SV_OK;
        buf = {g.m[0].real(), g.m[0].imag()};
        const svk::GroupGeom G = make_geom(g.c, g.c, g.cv);
        return cuda_status(svk::launch_diag(L, h->dt, h->sv, h->n, G, nullptr, 0, buf.data()));
    }
    const int D = 1 << k;
    bool diag = true;
    for (int r = 0; r < D && diag; ++r)
        for (int c = 0; c < D && diag; ++c)
            if (r != c && g.m[r * D + c] != cd(0)) diag = false;
    if (diag) {
        buf.resize(2 * D);
        for (int j = 0; j < D; ++j) {
            buf[2 * j] = g.m[j * D + j].real();
            buf[2 * j + 1] = g.m[j * D + j].imag();
        }
        const svk::GroupGeom G = make_geom(g.c, g.c, g.cv);
        return cuda_status(svk::launch_diag(L, h->dt, h->sv, h->n, G, g.t.data(), k, buf.data()));
    }
    sort_targets(g);
    std::vector<int> ins = g.t;
    ins.insert(ins.end(), g.c.begin(), g.c.end());
    const svk::GroupGeom G = make_geom(ins, g.c, g.cv);
    if (k <= 4) {
        // generalized permutation: exactly one nonzero per row and per column
        std::vector<int> perm(D, -1), colcount(D, 0);
        bool ok = true;
        for (int r = 0; r < D && ok; ++r)
            for (int c = 0; c < D; ++c)
                if (g.m[r * D + c] != cd(0)) {
                    if (perm[r] >= 0) { ok = false; break; }
                    perm[r] = c;
                    ++colcount[c];
                }
        for (int j = 0; j < D && ok; ++j) ok = perm[j] >= 0 && colcount[j] == 1;
        if (ok) {
            buf.resize(2 * D);
            for (int j = 0; j < D; ++j) {
                buf[2 * j] = g.m[j * D + perm[j]].real();
                buf[2 * j + 1] = g.m[j * D + perm[j]].imag();
            }
            return cuda_status(svk::launch_perm(L, h->dt, h->sv, h->n, G, g.t.data(), k, perm.data(), buf.data()));
        }
    }
    buf.resize(2 * D * D);
    for (int i = 0; i < D * D; ++i) {
        buf[2 * i] = g.m[i].real();
        buf[2 * i + 1] = g.m[i].imag();
    }
    if (prec != SV_PREC_NATIVE && h->dt == SV_C64 && k >= 5 && g.c.empty()) {
        // tensor-core path works on 6 targets; a 5-target block gains one identity
        // qubit, the highest one not in the block (low qubits stay free, which keeps
        // consecutive columns on adjacent amplitudes)
        std::vector<int> t6 = g.t;
        std::vector<double> m6;
        if (k == 5) {
            int extra = -1;
            for (int q = h->n - 1; q >= 0 && extra < 0; --q)
                if (std::find(t6.begin(), t6.end(), q) == t6.end()) extra = q;
            if (extra < 0) return SV_ERR_INVALID_ARGUMENT;
            Gate g6;
            g6.t = g.t;
            g6.t.push_back(extra);
            g6.m.assign(64 * 64, cd(0));
            for (int r = 0; r < 64; ++r)
                for (int c = 0; c < 64; ++c)
                    if ((r >> 5) == (c >> 5)) g6.m[r * 64 + c] = g.m[(r & 31) * 32 + (c & 31)];
            sort_targets(g6);
            t6 = g6.t;
            m6.resize(2 * 64 * 64);
            for (int i = 0; i < 64 * 64; ++i) {
                m6[2 * i] = g6.m[i].real();
                m6[2 * i + 1] = g6.m[i].imag();
            }
        } else {
            m6 = buf;
        }
        if (!svk::tc6_supported(h->n, t6.data())) return SV_ERR_NOT_SUPPORTED;
        return cuda_status(svk::launch_tc6(L, h->sv, h->n, t6.data(), m6.data(), prec, h->d_mat, h->d_err));
    }
    return cuda_status(svk::launch_dense(L, h->dt, h->sv, h->n, G, g.t.data(), k, buf.data(), h->d_mat));
}

sv_status_t check_gate_args(const sv_ctx *h, const int *targets, int k, const int *controls, const int *cvals, int c,
                            const double *matrix) {
    if (!h || !targets || !matrix || k < 1 || k > SV_MAX_TARGETS || c < 0 || c > SV_MAX_CONTROLS ||
        (c > 0 && !controls) || k + c > h->n)
        return SV_ERR_INVALID_ARGUMENT;
    if (!valid_qubits(h->n, targets, k, controls, c)) return SV_ERR_INVALID_ARGUMENT;
    if (cvals)
        for (int i = 0; i < c; ++i)
            if (cvals[i] != 0 && cvals[i] != 1) return SV_ERR_INVALID_ARGUMENT;
    return SV_OK;
}

Gate make_gate(const int *targets, int k, const int *controls, const int *cvals, int c, const double *matrix,
               int adjoint) {
    Gate g;
    g.t.assign(targets, targets + k);
    if (c > 0) g.c.assign(controls, controls + c);
    for (int i = 0; i < c; ++i) g.cv.push_back(cvals ? cvals[i] : 1);
    const int D = 1 << k;
    g.m.resize(D * D);
    for (int r = 0; r < D; ++r)
        for (int col = 0; col < D; ++col) {
            const cd v(matrix[2 * (r * D + col)], matrix[2 * (r * D + col) + 1]);
            if (adjoint) g.m[col * D + r] = std::conj(v);
            else g.m[r * D + col] = v;
        }
    return g;
}

sv_status_t sync_results(sv_ctx *h, int count) {
    cudaError_t e = cudaMemcpyAsync(h->h_results, h->d_results, sizeof(double) * count, cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e != cudaSuccess) return SV_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(h->stream));
}

// Tensor-core blocks whose lowest target is below qubit 2 are the slow ones
// (measured on GB300 at 32 qubits, TF32 / split BF16: 10.4 / 11.2 ms per block for
// lowest target 3 or more, 12.7 / 13.6 ms at 2, 14.8 / 15.4 ms at 1 and about
// 16 ms at 0, where the register-staged kernel runs).
int slow_below(sv_precision_t) { return 2; }

// Qubit relabelling for a fused run (Sec. II-C, qubit reordering, applied on one
// GPU): qubits 0..low-1 are swapped with the `low` qubits that the fewest wide
// blocks use (moving only some of them rarely helps, a block then keeps another
// low target). Returns the pairs -- empty when the blocks it speeds up do not pay
// for the two extra passes -- and the map logical -> physical. Cost model from
// the measurements above: a slow block costs about 0.4-0.6 of a fast block more,
// the two swap passes (one permutation pass each way over the whole state) about
// 2 fast blocks, so at least 6 fewer slow blocks are needed.
void choose_layout(const std::vector<svf::Item> &items, int n, int low, std::vector<int> &pairs,
                   std::vector<int> &map) {
    map.resize(n);
    for (int q = 0; q < n; ++q) map[q] = q;
    pairs.clear();
    if (n < 2 * low + 6) return;
    std::vector<const std::vector<int> *> wide;
    std::vector<int> uses(n, 0);
    for (const svf::Item &it : items)
        if (!it.passthrough && !it.diagonal && it.qubits.size() >= 5) {
            wide.push_back(&it.qubits);
            for (int q : it.qubits) ++uses[q];
        }
    auto slow_count = [&](const std::vector<int> &m) {
        int c = 0;
        for (const std::vector<int> *qs : wide) {
            int lo = 1 << 30;
            for (int q : *qs) lo = std::min(lo, m[q]);
            c += lo < low;
        }
        return c;
    };
    std::vector<int> cand;
    for (int q = low; q < n; ++q) cand.push_back(q);
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
        return uses[a] != uses[b] ? uses[a] < uses[b] : a > b;
    });
    std::vector<int> m = map;
    std::vector<int> trial;
    for (int l = 0; l < low; ++l) {
        const int h = cand[l];
        std::swap(m[l], m[h]);
        trial.push_back(l);
        trial.push_back(h);
    }
    const int before = slow_count(map), after = slow_count(m);
    if (before - after >= 6) {
        map = m;
        pairs = trial;
    }
}

sv_status_t qubit_mask(const sv_ctx *h, const int *qubits, int m, uint64_t *mask) {
    if (!qubits || m < 1 || m > h->n) return SV_ERR_INVALID_ARGUMENT;
    uint64_t s = 0;
    for (int i = 0; i < m; ++i) {
        if (qubits[i] < 0 || qubits[i] >= h->n || ((s >> qubits[i]) & 1u)) return SV_ERR_INVALID_ARGUMENT;
        s |= 1ull << qubits[i];
    }
    *mask = s;
    return SV_OK;
}

}  // namespace

extern "C" {

const char *sv_status_string(sv_status_t s) {
    switch (s) {
    case SV_OK: return "SV_OK";
    case SV_ERR_INVALID_ARGUMENT: return "SV_ERR_INVALID_ARGUMENT";
    case SV_ERR_NOT_SUPPORTED: return "SV_ERR_NOT_SUPPORTED";
    case SV_ERR_INSUFFICIENT_WORKSPACE: return "SV_ERR_INSUFFICIENT_WORKSPACE";
    case SV_ERR_CUDA: return "SV_ERR_CUDA";
    case SV_ERR_TIMEOUT: return "SV_ERR_TIMEOUT";
    case SV_ERR_ALLOC: return "SV_ERR_ALLOC";
    }
    return "SV_ERR_UNKNOWN";
}

sv_status_t sv_create(int n_qubits, sv_dtype_t dtype, void *d_state, void *stream, sv_handle_t *out) {
    if (!out || !d_state || n_qubits < 1 || n_qubits > SV_MAX_QUBITS || (dtype != SV_C64 && dtype != SV_C128) ||
        (reinterpret_cast<uintptr_t>(d_state) & 15u))
        return SV_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    sv_ctx *h = new (std::nothrow) sv_ctx();
    if (!h) return SV_ERR_ALLOC;
    h->n = n_qubits;
    h->dt = dtype;
    h->sv = d_state;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return SV_ERR_CUDA;
    }
    if (cudaMalloc(reinterpret_cast<void **>(&h->ws), SV_WORKSPACE_BYTES) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return SV_ERR_ALLOC;
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&h->h_results), kResultBytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->ws);
        delete h;
        return SV_ERR_ALLOC;
    }
    h->d_partials = reinterpret_cast<double *>(h->ws);
    h->max_partial_blocks = (int)(kPartialBytes / (8 * sizeof(double)));
    h->d_results = reinterpret_cast<double *>(h->ws + kPartialBytes);
    h->max_results = (int)(kResultBytes / sizeof(double));
    h->d_err = reinterpret_cast<int *>(h->ws + kPartialBytes + kResultBytes);
    h->d_mat = h->ws + kMatOffset;
    h->mat_bytes = SV_WORKSPACE_BYTES - kMatOffset;
    if (cudaMemsetAsync(h->d_err, 0, kErrBytes, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaFreeHost(h->h_results);
        cudaFree(h->ws);
        delete h;
        return SV_ERR_CUDA;
    }
    *out = h;
    return SV_OK;
}

sv_status_t sv_destroy(sv_handle_t h) {
    if (!h) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    cudaFreeHost(h->h_results);
    cudaFree(h->ws);
    delete h;
    return SV_OK;
}

sv_status_t sv_set_stream(sv_handle_t h, void *stream) {
    if (!h) return SV_ERR_INVALID_ARGUMENT;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return SV_OK;
}

sv_status_t sv_set_state_pointer(sv_handle_t h, void *d_state) {
    if (!h || !d_state || (reinterpret_cast<uintptr_t>(d_state) & 15u)) return SV_ERR_INVALID_ARGUMENT;
    h->sv = d_state;
    return SV_OK;
}

sv_status_t sv_set_state(sv_handle_t h, int n_qubits, sv_dtype_t dtype, void *d_state) {
    if (!h || !d_state || n_qubits < 1 || n_qubits > SV_MAX_QUBITS || (dtype != SV_C64 && dtype != SV_C128) ||
        (reinterpret_cast<uintptr_t>(d_state) & 15u))
        return SV_ERR_INVALID_ARGUMENT;
    h->n = n_qubits;
    h->dt = dtype;
    h->sv = d_state;
    return SV_OK;
}

sv_status_t sv_set_basis_state(sv_handle_t h, uint64_t index) {
    if (!h || index >= (1ull << h->n)) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    return cuda_status(svk::launch_set_basis(lctx(h), h->dt, h->sv, h->n, index));
}

sv_status_t sv_copy_from_host(sv_handle_t h, const void *host) {
    if (!h || !host) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    const size_t bytes = (size_t(1) << h->n) * (h->dt == SV_C64 ? 8 : 16);
    if (cudaMemcpyAsync(h->sv, host, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return SV_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(h->stream));
}

sv_status_t sv_copy_to_host(sv_handle_t h, void *host) {
    if (!h || !host) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    const size_t bytes = (size_t(1) << h->n) * (h->dt == SV_C64 ? 8 : 16);
    if (cudaMemcpyAsync(host, h->sv, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return SV_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(h->stream));
}

sv_status_t sv_copy_from_host_async(sv_handle_t h, const void *host) {
    if (!h || !host) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    const size_t bytes = (size_t(1) << h->n) * (h->dt == SV_C64 ? 8 : 16);
    return cuda_status(cudaMemcpyAsync(h->sv, host, bytes, cudaMemcpyHostToDevice, h->stream));
}

sv_status_t sv_copy_to_host_async(sv_handle_t h, void *host) {
    if (!h || !host) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    const size_t bytes = (size_t(1) << h->n) * (h->dt == SV_C64 ? 8 : 16);
    return cuda_status(cudaMemcpyAsync(host, h->sv, bytes, cudaMemcpyDeviceToHost, h->stream));
}

sv_status_t sv_apply_matrix(sv_handle_t h, const int *targets, int n_targets, const int *controls,
                            const int *control_values, int n_controls, const double *matrix, int adjoint) {
    sv_status_t s = check_gate_args(h, targets, n_targets, controls, control_values, n_controls, matrix);
    if (s != SV_OK) return s;
    DeviceGuard dg(h->device);
    return apply_gate(h, make_gate(targets, n_targets, controls, control_values, n_controls, matrix, adjoint),
                      SV_PREC_NATIVE);
}

sv_status_t sv_swap_index_bits(sv_handle_t h, const int *bit_pairs, int n_pairs) {
    if (!h || !bit_pairs || n_pairs < 1 || n_pairs > 18) return SV_ERR_INVALID_ARGUMENT;
    int a[18], b[18];
    uint64_t seen = 0;
    for (int k = 0; k < n_pairs; ++k) {
        a[k] = bit_pairs[2 * k];
        b[k] = bit_pairs[2 * k + 1];
        if (a[k] < 0 || a[k] >= h->n || b[k] < 0 || b[k] >= h->n || a[k] == b[k] || ((seen >> a[k]) & 1u) ||
            ((seen >> b[k]) & 1u))
            return SV_ERR_INVALID_ARGUMENT;
        seen |= (1ull << a[k]) | (1ull << b[k]);
    }
    DeviceGuard dg(h->device);
    return cuda_status(svk::launch_swap(lctx(h), h->dt, h->sv, h->n, a, b, n_pairs));
}

sv_status_t sv_fuse_plan(const sv_gate_t *gates, int n_gates, int n_qubits, int max_fused_qubits, int max_blocks,
                         int *n_blocks_out, int *block_k, int *block_targets, double *block_matrices) {
    sv_fusion_options_t opt{max_fused_qubits, 0, SV_PREC_NATIVE};
    return sv_fuse_plan_ex(gates, n_gates, n_qubits, &opt, max_blocks, n_blocks_out, block_k, block_targets,
                           block_matrices);
}

sv_status_t sv_fuse_plan_ex(const sv_gate_t *gates, int n_gates, int n_qubits, const sv_fusion_options_t *opt,
                            int max_blocks, int *n_blocks_out, int *block_k, int *block_targets,
                            double *block_matrices) {
    if ((!gates && n_gates > 0) || n_gates < 0 || !n_blocks_out || !opt || n_qubits < 1 || n_qubits > SV_MAX_QUBITS)
        return SV_ERR_INVALID_ARGUMENT;
    const int max_fused_qubits = opt->max_fused_qubits;
    for (int i = 0; i < n_gates; ++i) {
        const sv_gate_t &g = gates[i];
        if (g.n_targets < 1 || g.n_targets > SV_MAX_TARGETS || g.n_controls < 0 || g.n_controls > SV_MAX_CONTROLS ||
            !g.matrix || g.n_targets + g.n_controls > n_qubits ||
            !valid_qubits(n_qubits, g.targets, g.n_targets, g.controls, g.n_controls))
            return SV_ERR_INVALID_ARGUMENT;
    }
    std::vector<svf::Item> items;
    sv_status_t s = svf::fuse(gates, n_gates, n_qubits, max_fused_qubits, items, opt->max_fused_diagonal_qubits);
    if (s != SV_OK) return s;
    *n_blocks_out = (int)items.size();
    if ((int)items.size() > max_blocks) return SV_ERR_INSUFFICIENT_WORKSPACE;
    for (size_t b = 0; b < items.size(); ++b) {
        const svf::Item &it = items[b];
        std::vector<int> qs;
        std::vector<cd> m;
        if (it.passthrough) {
            // a gate wider than the fusion width, written as its dense block
            const sv_gate_t &g = gates[it.gate];
            const int nq = g.n_targets + g.n_controls;
            if (nq > SV_MAX_TARGETS) return SV_ERR_NOT_SUPPORTED;
            for (int t = 0; t < nq; ++t) qs.push_back(t < g.n_targets ? g.targets[t] : g.controls[t - g.n_targets]);
            const uint64_t d = 1ull << nq;
            m.assign(d * d, cd(0));
            for (uint64_t i = 0; i < d; ++i) m[i * d + i] = 1;
            int lt[SV_MAX_TARGETS], lc[SV_MAX_CONTROLS], cv[SV_MAX_CONTROLS];
            for (int t = 0; t < g.n_targets; ++t) lt[t] = t;
            for (int t = 0; t < g.n_controls; ++t) {
                lc[t] = g.n_targets + t;
                cv[t] = g.control_values[t] ? 1 : 0;
            }
            const uint64_t D = 1ull << g.n_targets;
            std::vector<cd> gm(D * D);
            for (uint64_t i = 0; i < D * D; ++i) gm[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
            std::vector<cd> col(d);
            for (uint64_t c = 0; c < d; ++c) {
                for (uint64_t r = 0; r < d; ++r) col[r] = m[r * d + c];
                svf::apply_small(col.data(), nq, lt, g.n_targets, lc, cv, g.n_controls, gm.data());
                for (uint64_t r = 0; r < d; ++r) m[r * d + c] = col[r];
            }
        } else {
            qs = it.qubits;
            m = it.m;
        }
        const int k = (int)qs.size();
        if (block_k) block_k[b] = k;
        if (block_targets)
            for (int t = 0; t < SV_MAX_TARGETS; ++t) block_targets[b * SV_MAX_TARGETS + t] = t < k ? qs[t] : -1;
        if (block_matrices) {
            double *dst = block_matrices + b * 64 * 64 * 2;
            for (size_t i = 0; i < m.size(); ++i) {
                dst[2 * i] = m[i].real();
                dst[2 * i + 1] = m[i].imag();
            }
        }
    }
    return SV_OK;
}

sv_status_t sv_apply_fused(sv_handle_t h, const sv_gate_t *gates, int n_gates, int max_fused_qubits,
                           sv_precision_t prec, int *n_fused_out) {
    sv_fusion_options_t opt{max_fused_qubits, 0, prec};
    return sv_apply_fused_ex(h, gates, n_gates, &opt, n_fused_out);
}

sv_status_t sv_apply_fused_ex(sv_handle_t h, const sv_gate_t *gates, int n_gates, const sv_fusion_options_t *opt,
                              int *n_fused_out) {
    if (!h || !opt || (!gates && n_gates > 0) || n_gates < 0) return SV_ERR_INVALID_ARGUMENT;
    const int max_fused_qubits = opt->max_fused_qubits;
    const sv_precision_t prec = opt->precision;
    if (max_fused_qubits < 1 || max_fused_qubits > SV_MAX_TARGETS || opt->max_fused_diagonal_qubits < 0 ||
        opt->max_fused_diagonal_qubits > SV_MAX_TARGETS ||
        (prec != SV_PREC_NATIVE && prec != SV_PREC_TF32 && prec != SV_PREC_SPLIT_BF16))
        return SV_ERR_INVALID_ARGUMENT;
    if (prec != SV_PREC_NATIVE && h->dt != SV_C64) return SV_ERR_NOT_SUPPORTED;
    for (int i = 0; i < n_gates; ++i) {
        const sv_gate_t &g = gates[i];
        sv_status_t s = check_gate_args(h, g.targets, g.n_targets, g.controls, g.control_values, g.n_controls,
                                        g.matrix);
        if (s != SV_OK) return s;
    }
    std::vector<svf::Item> items;
    sv_status_t s = svf::fuse(gates, n_gates, h->n, max_fused_qubits, items, opt->max_fused_diagonal_qubits);
    if (s != SV_OK) return s;
    DeviceGuard dg(h->device);
    std::vector<int> pairs, map;
    if (prec != SV_PREC_NATIVE) choose_layout(items, h->n, slow_below(prec), pairs, map);
    else {
        map.resize(h->n);
        for (int q = 0; q < h->n; ++q) map[q] = q;
    }
    const int npairs = (int)pairs.size() / 2;
    if (npairs > 0) {
        s = sv_swap_index_bits(h, pairs.data(), npairs);
        if (s != SV_OK) return s;
    }
    for (const svf::Item &it : items) {
        if (it.passthrough) {
            const sv_gate_t &g = gates[it.gate];
            Gate gg = make_gate(g.targets, g.n_targets, g.controls, g.control_values, g.n_controls, g.matrix, 0);
            for (int &q : gg.t) q = map[q];
            for (int &q : gg.c) q = map[q];
            s = apply_gate(h, gg, prec);
        } else {
            Gate g;
            g.t = it.qubits;
            for (int &q : g.t) q = map[q];
            g.m = it.m;
            s = apply_gate(h, g, prec);
        }
        if (s != SV_OK) return s;
    }
    if (npairs > 0) {
        s = sv_swap_index_bits(h, pairs.data(), npairs);
        if (s != SV_OK) return s;
    }
    if (n_fused_out) *n_fused_out = (int)items.size();
    return SV_OK;
}

sv_status_t sv_expectation_pauli(sv_handle_t h, const int *paulis, const int *sites, int n_sites, int n_strings,
                                 double *out) {
    if (!h || !out || n_sites < 0 || n_strings < 0 || ((!paulis || !sites) && n_sites > 0 && n_strings > 0))
        return SV_ERR_INVALID_ARGUMENT;
    struct Str { uint64_t x, z; int ny; };
    std::vector<Str> strs(n_strings);
    for (int s = 0; s < n_strings; ++s) {
        uint64_t x = 0, z = 0, seen = 0;
        int ny = 0;
        for (int i = 0; i < n_sites; ++i) {
            const int p = paulis[(size_t)s * n_sites + i], q = sites[(size_t)s * n_sites + i];
            if (p < 0 || p > 3 || q < 0 || q >= h->n || ((seen >> q) & 1u)) return SV_ERR_INVALID_ARGUMENT;
            seen |= 1ull << q;
            if (p == SV_PAULI_X || p == SV_PAULI_Y) x |= 1ull << q;
            if (p == SV_PAULI_Z || p == SV_PAULI_Y) z |= 1ull << q;
            ny += p == SV_PAULI_Y;
        }
        strs[s] = {x, z, ny};
    }
    if (n_strings == 0) return SV_OK;
    DeviceGuard dg(h->device);
    // strings of identities and at most one Z: all of them from one <Z_q> pass
    bool single_z = h->n >= 3;
    for (int s = 0; s < n_strings && single_z; ++s) single_z = strs[s].x == 0 && __builtin_popcountll(strs[s].z) <= 1;
    if (single_z && n_strings >= 2) {
        if (svk::launch_zall(lctx(h), h->dt, h->sv, h->n, h->d_partials, h->max_partial_blocks, h->d_results) !=
            cudaSuccess)
            return SV_ERR_CUDA;
        sv_status_t st = sync_results(h, h->n + 1);
        if (st != SV_OK) return st;
        for (int s = 0; s < n_strings; ++s)
            out[s] = strs[s].z ? h->h_results[__builtin_ctzll(strs[s].z)] : h->h_results[h->n];
        return SV_OK;
    }
    // strings with the same X/Y mask share a pass over the state
    std::map<uint64_t, std::vector<int>> by_x;
    for (int s = 0; s < n_strings; ++s) by_x[strs[s].x].push_back(s);
    std::vector<int> slot_of;   // result slot -> string
    const svk::LaunchCtx L = lctx(h);
    auto flush = [&]() -> sv_status_t {
        if (slot_of.empty()) return SV_OK;
        sv_status_t st = sync_results(h, (int)slot_of.size());
        if (st != SV_OK) return st;
        for (size_t i = 0; i < slot_of.size(); ++i) out[slot_of[i]] = h->h_results[i];
        slot_of.clear();
        return SV_OK;
    };
    for (auto &kv : by_x) {
        const std::vector<int> &ids = kv.second;
        for (size_t b = 0; b < ids.size(); b += svk::kPauliMaxS) {
            if ((int)slot_of.size() + svk::kPauliMaxS > h->max_results) {
                sv_status_t st = flush();
                if (st != SV_OK) return st;
            }
            svk::PauliPass P{};
            P.S = (int)std::min<size_t>(svk::kPauliMaxS, ids.size() - b);
            P.x = kv.first;
            for (int i = 0; i < P.S; ++i) {
                const Str &st = strs[ids[b + i]];
                P.z[i] = st.z;
                // Re(i^{nY} s w): +Re w, -Im w, -Re w, +Im w for nY = 0, 1, 2, 3 (mod 4)
                const int r = st.ny & 3;
                P.use_im[i] = r & 1;
                P.sign[i] = (r == 1 || r == 2) ? -1.0 : 1.0;
            }
            cudaError_t e = svk::launch_pauli(L, h->dt, h->sv, h->n, P, h->d_partials, h->max_partial_blocks,
                                              h->d_results + slot_of.size());
            if (e != cudaSuccess) return SV_ERR_CUDA;
            for (int i = 0; i < P.S; ++i) slot_of.push_back(ids[b + i]);
        }
    }
    return flush();
}

sv_status_t sv_apply_pauli_rotation(sv_handle_t h, double theta, const int *paulis, const int *sites, int n_sites) {
    if (!h || n_sites < 0 || (n_sites > 0 && (!paulis || !sites)) || !std::isfinite(theta))
        return SV_ERR_INVALID_ARGUMENT;
    uint64_t x = 0, z = 0, seen = 0;
    int ny = 0;
    for (int i = 0; i < n_sites; ++i) {
        const int p = paulis[i], q = sites[i];
        if (p < 0 || p > 3 || q < 0 || q >= h->n || ((seen >> q) & 1u)) return SV_ERR_INVALID_ARGUMENT;
        seen |= 1ull << q;
        if (p == SV_PAULI_X || p == SV_PAULI_Y) x |= 1ull << q;
        if (p == SV_PAULI_Z || p == SV_PAULI_Y) z |= 1ull << q;
        ny += p == SV_PAULI_Y;
    }
    DeviceGuard dg(h->device);
    return cuda_status(svk::launch_pauli_rotation(lctx(h), h->dt, h->sv, h->n, x, z, ny & 3, theta));
}

sv_status_t sv_sample(sv_handle_t h, const double *randnums, int n_samples, int64_t *out) {
    if (!h || n_samples < 0 || (n_samples > 0 && (!randnums || !out))) return SV_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < n_samples; ++i)
        if (!(randnums[i] >= 0.0 && randnums[i] < 1.0)) return SV_ERR_INVALID_ARGUMENT;
    if (n_samples == 0) return SV_OK;
    DeviceGuard dg(h->device);
    // workspace: 2^20 segment sums (8 MiB), then chunks of random numbers and outcomes
    constexpr int kChunk = 1 << 18;
    double *d_seg = reinterpret_cast<double *>(h->d_mat);
    double *d_r = d_seg + (1 << 20);
    long long *d_o = reinterpret_cast<long long *>(d_r + kChunk);
    for (int b = 0; b < n_samples; b += kChunk) {
        const int m = std::min(kChunk, n_samples - b);
        if (cudaMemcpyAsync(d_r, randnums + b, sizeof(double) * m, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
            return SV_ERR_CUDA;
        if (svk::launch_sample(lctx(h), h->dt, h->sv, h->n, d_r, m, d_seg, d_o) != cudaSuccess) return SV_ERR_CUDA;
        if (cudaMemcpyAsync(out + b, d_o, sizeof(long long) * m, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return SV_ERR_CUDA;
    }
    return SV_OK;
}

sv_status_t sv_measure_probs(sv_handle_t h, const int *qubits, int n_qubits, double *p_even, double *p_odd) {
    if (!h || !p_even || !p_odd) return SV_ERR_INVALID_ARGUMENT;
    uint64_t mask = 0;
    sv_status_t s = qubit_mask(h, qubits, n_qubits, &mask);
    if (s != SV_OK) return s;
    DeviceGuard dg(h->device);
    if (svk::launch_parity(lctx(h), h->dt, h->sv, h->n, mask, h->d_partials, h->max_partial_blocks, h->d_results) !=
        cudaSuccess)
        return SV_ERR_CUDA;
    s = sync_results(h, 2);
    if (s != SV_OK) return s;
    *p_even = h->h_results[0];
    *p_odd = h->h_results[1];
    return SV_OK;
}

sv_status_t sv_collapse(sv_handle_t h, const int *qubits, int n_qubits, int parity, double prob) {
    if (!h || (parity != 0 && parity != 1) || !(prob > 0.0) || !std::isfinite(prob)) return SV_ERR_INVALID_ARGUMENT;
    uint64_t mask = 0;
    sv_status_t s = qubit_mask(h, qubits, n_qubits, &mask);
    if (s != SV_OK) return s;
    DeviceGuard dg(h->device);
    return cuda_status(svk::launch_collapse(lctx(h), h->dt, h->sv, h->n, mask, parity, 1.0 / std::sqrt(prob)));
}

sv_status_t sv_measure(sv_handle_t h, const int *qubits, int n_qubits, double randnum, int collapse,
                       int *parity_out) {
    if (!h || !parity_out || !(randnum >= 0.0 && randnum < 1.0)) return SV_ERR_INVALID_ARGUMENT;
    double p0 = 0, p1 = 0;
    sv_status_t s = sv_measure_probs(h, qubits, n_qubits, &p0, &p1);
    if (s != SV_OK) return s;
    const double tot = p0 + p1;
    if (!(tot > 0.0)) return SV_ERR_INVALID_ARGUMENT;
    const int parity = randnum < p0 / tot ? 0 : 1;
    *parity_out = parity;
    if (collapse) return sv_collapse(h, qubits, n_qubits, parity, parity == 0 ? p0 : p1);
    return SV_OK;
}

sv_status_t sv_norm2(sv_handle_t h, double *out) {
    if (!h || !out) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    if (svk::launch_parity(lctx(h), h->dt, h->sv, h->n, 0, h->d_partials, h->max_partial_blocks, h->d_results) !=
        cudaSuccess)
        return SV_ERR_CUDA;
    sv_status_t s = sync_results(h, 1);
    if (s != SV_OK) return s;
    *out = h->h_results[0];
    return SV_OK;
}

sv_status_t sv_check_device_status(sv_handle_t h) {
    if (!h) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    int flag = 0;
    if (cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return SV_ERR_CUDA;
    if (flag == 0) return SV_OK;
    if (cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return SV_ERR_CUDA;
    return SV_ERR_TIMEOUT;
}

sv_status_t sv_check_bounded_wait(sv_handle_t h, long long cycles) {
    if (!h || cycles < 1000 || cycles > 4000000000ll) return SV_ERR_INVALID_ARGUMENT;
    DeviceGuard dg(h->device);
    if (svk::launch_wait_probe(lctx(h), h->d_err, cycles) != cudaSuccess) return SV_ERR_CUDA;
    return sv_check_device_status(h);
}

sv_status_t sv_launch_count(sv_handle_t h, uint64_t *out) {
    if (!h || !out) return SV_ERR_INVALID_ARGUMENT;
    *out = h->launches;
    return SV_OK;
}

}  // extern "C"
