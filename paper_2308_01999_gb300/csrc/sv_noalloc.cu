// sv_noalloc.cu -- Pauli-string expectation values for callers that cannot
// allocate device memory.
//
// The handle-based entry points get their scratch space (per-block partial
// sums and results) from a workspace that sv_create allocates with cudaMalloc.
// Some callers cannot do that: a process whose device memory is already owned
// by another allocator (a framework's caching allocator or a pool sized to the
// whole GPU) would see the allocation fail or force that allocator to give
// memory back, and a latency-critical loop cannot afford cudaMalloc/cudaFree,
// which may synchronise the whole device. sv_expectation_pauli_noalloc serves
// them: its scratch is the file-scope array below, which every GPU that loads
// this library holds from module load until the process exits.
//
// Host code must not use the array's name as a device address (on the host it
// names a host-side stand-in). The device address is looked up once per device,
// with that device current, on the first call made there (cudaGetSymbolAddress),
// and cached.
//
// Every call shares the one array, and it keeps the contents of the last call.
// Nothing in it needs to start at zero: each block writes its partial sums
// before the finishing kernel reads them, and each result slot is written
// before it is copied out. Calls whose work overlaps on the GPU (other streams,
// other host threads) race on the array; the caller must order them.
//
// The kernels are the ones sv_expectation_pauli uses (k_reduce.cu), launched on
// the caller's stream with the scratch address in place of the workspace.
#include <mutex>

#include "sv_internal.h"

namespace {

constexpr int kPartialBlocks = 2048;                       // 2048 blocks x 8 doubles
constexpr int kMaxStrings = SV_NOALLOC_MAX_STRINGS;        // result slots
constexpr int kMaxDevices = 64;

// 2048 * 8 + 4096 doubles = 160 KiB per device
static __device__ __align__(256) double sv_noalloc_scratch[kPartialBlocks * 8 + kMaxStrings];

struct DeviceScratch {
    double *addr = nullptr;   // device address of sv_noalloc_scratch on this device
    int num_sms = 0;
    bool ready = false;
};

DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current.
sv_status_t setup(int dev, DeviceScratch *&out) {
    if (dev < 0 || dev >= kMaxDevices) return SV_ERR_NOT_SUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch &d = g_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, sv_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return SV_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            return SV_ERR_CUDA;
        }
        d.addr = static_cast<double *>(p);
        d.num_sms = sms;
        d.ready = true;
    }
    out = &d;
    return SV_OK;
}

// X/Y mask, Z/Y mask and Y count of string s; false for a bad code or site
bool string_masks(const int *paulis, const int *sites, int n_sites, int s, int n, uint64_t &x, uint64_t &z, int &ny) {
    x = z = 0;
    ny = 0;
    uint64_t seen = 0;
    for (int i = 0; i < n_sites; ++i) {
        const int p = paulis[(size_t)s * n_sites + i], q = sites[(size_t)s * n_sites + i];
        if (p < 0 || p > 3 || q < 0 || q >= n || ((seen >> q) & 1u)) return false;
        seen |= 1ull << q;
        if (p == SV_PAULI_X || p == SV_PAULI_Y) x |= 1ull << q;
        if (p == SV_PAULI_Z || p == SV_PAULI_Y) z |= 1ull << q;
        ny += p == SV_PAULI_Y;
    }
    return true;
}

}  // namespace

extern "C" SV_API sv_status_t sv_expectation_pauli_noalloc(int n_qubits, sv_dtype_t dtype, const void *d_state,
                                                           void *stream, const int *paulis, const int *sites,
                                                           int n_sites, int n_strings, double *out) {
    if (n_qubits < 1 || n_qubits > SV_MAX_QUBITS || (dtype != SV_C64 && dtype != SV_C128) || !d_state ||
        (reinterpret_cast<uintptr_t>(d_state) & 15u) || !out || n_sites < 0 || n_strings < 0 ||
        ((!paulis || !sites) && n_sites > 0 && n_strings > 0))
        return SV_ERR_INVALID_ARGUMENT;
    if (n_strings > kMaxStrings) return SV_ERR_INSUFFICIENT_WORKSPACE;
    for (int s = 0; s < n_strings; ++s) {
        uint64_t x, z;
        int ny;
        if (!string_masks(paulis, sites, n_sites, s, n_qubits, x, z, ny)) return SV_ERR_INVALID_ARGUMENT;
    }
    if (n_strings == 0) return SV_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SV_ERR_CUDA;
    DeviceScratch *ds = nullptr;
    sv_status_t st = setup(dev, ds);
    if (st != SV_OK) return st;
    double *partials = ds->addr;
    double *results = ds->addr + kPartialBlocks * 8;
    uint64_t launches = 0;
    const svk::LaunchCtx L{reinterpret_cast<cudaStream_t>(stream), ds->num_sms, &launches};
    // one pass per run of at most 8 consecutive strings that share an X/Y mask;
    // results land in string order
    int s = 0;
    while (s < n_strings) {
        svk::PauliPass P{};
        uint64_t x0, z;
        int ny;
        string_masks(paulis, sites, n_sites, s, n_qubits, x0, z, ny);
        P.x = x0;
        P.S = 0;
        while (s + P.S < n_strings && P.S < svk::kPauliMaxS) {
            uint64_t x;
            string_masks(paulis, sites, n_sites, s + P.S, n_qubits, x, z, ny);
            if (x != x0) break;
            const int r = ny & 3;   // i^{nY}: +Re, -Im, -Re, +Im
            P.z[P.S] = z;
            P.use_im[P.S] = r & 1;
            P.sign[P.S] = (r == 1 || r == 2) ? -1.0 : 1.0;
            ++P.S;
        }
        if (svk::launch_pauli(L, dtype, d_state, n_qubits, P, partials, kPartialBlocks, results + s) != cudaSuccess)
            return SV_ERR_CUDA;
        s += P.S;
    }
    if (cudaMemcpyAsync(out, results, sizeof(double) * n_strings, cudaMemcpyDeviceToHost, L.stream) != cudaSuccess)
        return SV_ERR_CUDA;
    return cudaStreamSynchronize(L.stream) == cudaSuccess ? SV_OK : SV_ERR_CUDA;
}
