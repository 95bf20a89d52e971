// k_reduce.cu -- reductions over the state vector: Pauli-string expectation
// values (Table I, "Expectation"), parity probabilities of a Z-product-basis
// measurement and its collapse (Table I, "Measurement"), and the norm.
//
// Pauli expectation. For P = prod of Paulis, with x = mask of X/Y sites,
// z = mask of Z/Y sites and nY = number of Y sites,
//   P|i> = i^{nY} (-1)^{popcount(i & z)} |i ^ x>,
//   <psi|P|psi> = sum_i i^{nY} (-1)^{popcount(i & z)} psi_i conj(psi_{i^x}),
// which is real because P is Hermitian. With w_i = psi_i conj(psi_{i^x}) the
// real part per term is +-Re(w_i) (nY even) or +-Im(w_i) (nY odd); the host
// folds i^{nY} into a per-string selector and sign. Strings with the same x
// share one pass: each pass reads every amplitude once, pairing unit i with
// unit i ^ x so that both partners come from the same two loads.
//
// Precision. Terms are formed in the state's precision. For complex64 each
// thread sums the terms of one loop iteration in FP32 (at most 8 per string:
// 4 work items x 2 amplitudes), so that partial carries a relative rounding
// error of at most 8 u (u = 2^-24) of the sum of its terms' magnitudes; the
// partials are accumulated per thread in FP32 with compensation (error about
// 2 u of the sum of magnitudes) and summed in FP64 across threads and blocks.
// Since sum_i |w_i| <= <psi|psi> and a pair's term carries a factor 2, the
// absolute error of a complex64 expectation value is at most about
// 1.2e-6 <psi|psi> (typically far less). complex128 uses FP64 throughout.
// Block partials are reduced by a second kernel in a fixed order, so results
// are bitwise reproducible for a given launch shape.
#include "sv_internal.h"

namespace svk {
namespace {

constexpr int kThreads = 256;
constexpr int kIlp = 4;     // work items loaded before any is consumed
constexpr int kRun = 1;     // loop iterations summed in FP32 before an FP64 add

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; static constexpr int V = 2; };
template <> struct CT<double> { using T = double2; static constexpr int V = 1; };

// V consecutive amplitudes starting at unit index u (16-byte load either way)
template <typename R>
__device__ __forceinline__ void load_unit(const typename CT<R>::T *sv, uint64_t u, typename CT<R>::T (&a)[CT<R>::V]) {
    if constexpr (CT<R>::V == 2) {
        const float4 f = reinterpret_cast<const float4 *>(sv)[u];
        a[0] = float2{f.x, f.y};
        a[1] = float2{f.z, f.w};
    } else {
        a[0] = sv[u];
    }
}

template <typename C>
__device__ __forceinline__ C mul_conj(const C &a, const C &b) {  // a * conj(b)
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}

__device__ __forceinline__ uint64_t insert_zero(uint64_t g, int b) {
    const uint64_t lo = g & ((1ull << b) - 1ull);
    return ((g ^ lo) << 1) | lo;
}

template <int S>
__device__ __forceinline__ void block_reduce_store(double (&v)[S], int nS, double *out) {
    __shared__ double red[kThreads / 32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double x = v[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][s] = x;
    }
    __syncthreads();
    if (threadIdx.x < nS) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += red[w][threadIdx.x];
        out[threadIdx.x] = acc;
    }
}

// partials[b * 8 + s] summed over b in a fixed order; out[s] = sign[s] * sum
__global__ void __launch_bounds__(kThreads)
k_finish(const double *__restrict__ partials, int nblocks, int S, PauliPass P, int use_sign, double *__restrict__ out) {
    __shared__ double red[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < S; ++s) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kThreads) x += partials[(size_t)b * 8 + s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) acc += red[w];
            out[s] = use_sign ? P.sign[s] * acc : acc;
        }
        __syncthreads();
    }
}

// Pauli pass kernel. Terms are enumerated once per unordered pair {i, i ^ x}:
// with w = psi_i conj(psi_{i^x}) the pair contributes
//   (-1)^{par(i & z)} [sel(w) + (-1)^{par(x & z)} sel(conj(w))]
//     = (-1)^{par(i & z)} sel(w) (1 + (-1)^{par(x & z) + use_im}),
// i.e. twice the first term or exactly zero; the host folds that factor (2 or
// 0, and 1 when x = 0, where every i is its own partner and w = |psi_i|^2) into
// the string's sign. Within a 16-byte unit the parities of the elements differ
// from the unit's by the low bit of z, and the partner unit's by par(x & z),
// so one 64-bit popcount per unit and string suffices.
// MODE 0: x = 0. MODE 1: x = 1 (complex64 only: partners share a unit).
// MODE 2: partners in units u and u ^ xu (pairs enumerated by inserting a zero
// at xu's highest bit). SM: strings per pass rounded up to 1, 2, 4 or 8.
struct PauliK {
    int S;
    uint64_t zu[kPauliMaxS];     // z without its low unit-index bits
    unsigned zl[kPauliMaxS];     // bit 0 of z (complex64: element parity inside a unit)
    int use_im[kPauliMaxS];
};

// acc += x with the rounding error of each addition carried in c (Neumaier):
// for complex64 the running sums stay in FP32 (GB300's FP64 rate is a small
// fraction of its FP32 rate) at the accuracy of an FP64 accumulator of FP32 terms
__device__ __forceinline__ void comp_add(float &acc, float &c, float x) {
    const float t = acc + x;
    c += fabsf(acc) >= fabsf(x) ? (acc - t) + x : (x - t) + acc;
    acc = t;
}

template <typename R, int MODE, int SM>
__global__ void __launch_bounds__(kThreads)
k_pauli(const typename CT<R>::T *__restrict__ sv, uint64_t n_work, int pair_bit, uint64_t xu, unsigned xl, PauliK P,
        double *__restrict__ partials) {
    using C = typename CT<R>::T;
    constexpr int V = CT<R>::V;
    R acc[SM], cmp[SM];
#pragma unroll
    for (int s = 0; s < SM; ++s) { acc[s] = R(0); cmp[s] = R(0); }
    const uint64_t stride = (uint64_t)gridDim.x * kThreads * kIlp;
    for (uint64_t w0 = (uint64_t)blockIdx.x * kThreads * kIlp + threadIdx.x; w0 < n_work; w0 += stride) {
        C A[kIlp][V], B[kIlp][V];
        uint64_t ua[kIlp];
#pragma unroll
        for (int q = 0; q < kIlp; ++q) {
            const uint64_t w = w0 + (uint64_t)q * kThreads;
            ua[q] = MODE == 2 ? insert_zero(w, pair_bit) : w;
            if (w < n_work) {
                load_unit<R>(sv, ua[q], A[q]);
                if constexpr (MODE == 2) load_unit<R>(sv, ua[q] ^ xu, B[q]);
            }
        }
        R run[SM];
#pragma unroll
        for (int s = 0; s < SM; ++s) run[s] = R(0);
#pragma unroll
        for (int q = 0; q < kIlp; ++q) {
            if (w0 + (uint64_t)q * kThreads >= n_work) continue;
            // terms of this work item: element e's value t[e] (re, im) and its parity offset
            C t[V];
            if constexpr (MODE == 0) {
#pragma unroll
                for (int e = 0; e < V; ++e) t[e] = C{A[q][e].x * A[q][e].x + A[q][e].y * A[q][e].y, R(0)};
            } else if constexpr (MODE == 1) {
                t[0] = mul_conj(A[q][0], A[q][V - 1]);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) t[e] = mul_conj(A[q][e], xl ? B[q][V - 1 - e] : B[q][e]);
            }
#pragma unroll
            for (int s = 0; s < SM; ++s) {
                if (s >= P.S) continue;
                const unsigned p0 = (unsigned)__popcll(ua[q] & P.zu[s]) & 1u;
#pragma unroll
                for (int e = 0; e < (MODE == 1 ? 1 : V); ++e) {
                    const R v = P.use_im[s] ? t[e].y : t[e].x;
                    run[s] += (p0 ^ ((unsigned)e & P.zl[s])) ? -v : v;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < SM; ++s) {
            if (s >= P.S) continue;
            if constexpr (sizeof(R) == 4) comp_add(acc[s], cmp[s], run[s]);
            else acc[s] += run[s];
        }
    }
    double tot[SM];
#pragma unroll
    for (int s = 0; s < SM; ++s) tot[s] = (double)acc[s] + (double)cmp[s];
    block_reduce_store<SM>(tot, P.S, partials + (size_t)blockIdx.x * 8);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_parity(const typename CT<R>::T *__restrict__ sv, uint64_t n_units, uint64_t mask, double *__restrict__ partials) {
    using C = typename CT<R>::T;
    constexpr int V = CT<R>::V;
    double tot[2] = {0.0, 0.0};
    R run[2] = {R(0), R(0)};
    const uint64_t stride = (uint64_t)gridDim.x * kThreads * kIlp;
    int iter = 0;
    for (uint64_t u0 = (uint64_t)blockIdx.x * kThreads * kIlp + threadIdx.x; u0 < n_units; u0 += stride) {
        C A[kIlp][V];
#pragma unroll
        for (int q = 0; q < kIlp; ++q)
            if (u0 + (uint64_t)q * kThreads < n_units) load_unit<R>(sv, u0 + (uint64_t)q * kThreads, A[q]);
#pragma unroll
        for (int q = 0; q < kIlp; ++q) {
            const uint64_t u = u0 + (uint64_t)q * kThreads;
            if (u >= n_units) continue;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const R p = A[q][e].x * A[q][e].x + A[q][e].y * A[q][e].y;
                if (__popcll((u * V + e) & mask) & 1) run[1] += p; else run[0] += p;
            }
        }
        if (++iter == kRun) {
            tot[0] += (double)run[0];
            tot[1] += (double)run[1];
            run[0] = run[1] = R(0);
            iter = 0;
        }
    }
    tot[0] += (double)run[0];
    tot[1] += (double)run[1];
    block_reduce_store<2>(tot, 2, partials + (size_t)blockIdx.x * 8);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_collapse(typename CT<R>::T *__restrict__ sv, uint64_t n_units, uint64_t mask, int parity, R scale) {
    using C = typename CT<R>::T;
    constexpr int V = CT<R>::V;
    const uint64_t u = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (u >= n_units) return;
    C A[V];
    load_unit<R>(sv, u, A);
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const bool keep = (int)(__popcll((u * V + e) & mask) & 1) == parity;
        A[e].x = keep ? A[e].x * scale : R(0);
        A[e].y = keep ? A[e].y * scale : R(0);
    }
    if constexpr (V == 2) {
        reinterpret_cast<float4 *>(sv)[u] = make_float4(A[0].x, A[0].y, A[1].x, A[1].y);
    } else {
        sv[u] = A[0];
    }
}

template <typename R>
__global__ void k_set_one(typename CT<R>::T *sv, uint64_t index) {
    sv[index] = typename CT<R>::T{R(1), R(0)};
}

inline int reduce_grid(const LaunchCtx &L, uint64_t work, int max_blocks) {
    uint64_t b = (work + (uint64_t)kThreads * kIlp - 1) / ((uint64_t)kThreads * kIlp);
    uint64_t cap = (uint64_t)L.num_sms * 8;
    if (cap > (uint64_t)max_blocks) cap = (uint64_t)max_blocks;
    if (b > cap) b = cap;
    return (int)(b == 0 ? 1 : b);
}

template <typename R, int MODE>
cudaError_t pauli_launch(const LaunchCtx &L, const typename CT<R>::T *sv, int grid, uint64_t n_work, int pair_bit,
                         uint64_t xu, unsigned xl, const PauliK &K, double *d_partials) {
    const int S = K.S;
    if (S <= 1) k_pauli<R, MODE, 1><<<grid, kThreads, 0, L.stream>>>(sv, n_work, pair_bit, xu, xl, K, d_partials);
    else if (S <= 2) k_pauli<R, MODE, 2><<<grid, kThreads, 0, L.stream>>>(sv, n_work, pair_bit, xu, xl, K, d_partials);
    else if (S <= 4) k_pauli<R, MODE, 4><<<grid, kThreads, 0, L.stream>>>(sv, n_work, pair_bit, xu, xl, K, d_partials);
    else k_pauli<R, MODE, 8><<<grid, kThreads, 0, L.stream>>>(sv, n_work, pair_bit, xu, xl, K, d_partials);
    ++*L.launches;
    return cudaGetLastError();
}

template <typename R>
cudaError_t pauli_t(const LaunchCtx &L, const void *sv, int n, const PauliPass &P, double *d_partials, int maxb,
                    double *d_out) {
    using C = typename CT<R>::T;
    constexpr int V = CT<R>::V;
    if (P.S < 1 || P.S > kPauliMaxS) return cudaErrorInvalidValue;
    const int vb = V == 2 ? 1 : 0;                   // log2 V
    const uint64_t n_units = (1ull << n) >> vb;
    const unsigned xl = (unsigned)(P.x & (V - 1));
    const uint64_t xu = P.x >> vb;
    const int mode = P.x == 0 ? 0 : (xu == 0 ? 1 : 2);
    PauliK K{};
    K.S = P.S;
    PauliPass Pf = P;                                 // signs with the pair factor folded in
    for (int s = 0; s < P.S; ++s) {
        K.zu[s] = P.z[s] >> vb;
        K.zl[s] = (unsigned)(P.z[s] & (V - 1));
        K.use_im[s] = P.use_im[s];
        const int pxz = __builtin_popcountll(P.x & P.z[s]) & 1;
        Pf.sign[s] = mode == 0 ? P.sign[s] : (pxz == (P.use_im[s] ? 1 : 0) ? 2.0 * P.sign[s] : 0.0);
    }
    const uint64_t n_work = mode == 2 ? n_units / 2 : n_units;
    // pairs {u, u ^ xu} are enumerated by inserting a zero at one set bit of xu;
    // any set bit works, and the highest keeps each warp's loads in 512-byte runs
    const int pair_bit = mode == 2 ? 63 - __builtin_clzll(xu) : -1;
    const int grid = reduce_grid(L, n_work, maxb);
    const C *s = reinterpret_cast<const C *>(sv);
    cudaError_t e;
    if (mode == 0) e = pauli_launch<R, 0>(L, s, grid, n_work, pair_bit, xu, xl, K, d_partials);
    else if (mode == 2) e = pauli_launch<R, 2>(L, s, grid, n_work, pair_bit, xu, xl, K, d_partials);
    else if constexpr (V == 2) e = pauli_launch<R, 1>(L, s, grid, n_work, pair_bit, xu, xl, K, d_partials);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    k_finish<<<1, kThreads, 0, L.stream>>>(d_partials, grid, P.S, Pf, 1, d_out);
    ++*L.launches;
    return cudaGetLastError();
}

template <typename R>
cudaError_t parity_t(const LaunchCtx &L, const void *sv, int n, uint64_t mask, double *d_partials, int maxb,
                     double *d_out) {
    using C = typename CT<R>::T;
    constexpr int V = CT<R>::V;
    const uint64_t n_units = (1ull << n) / V;
    const int grid = reduce_grid(L, n_units, maxb);
    k_parity<R><<<grid, kThreads, 0, L.stream>>>(reinterpret_cast<const C *>(sv), n_units, mask, d_partials);
    ++*L.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    PauliPass none{};
    k_finish<<<1, kThreads, 0, L.stream>>>(d_partials, grid, 2, none, 0, d_out);
    ++*L.launches;
    return cudaGetLastError();
}

template <typename R>
cudaError_t collapse_t(const LaunchCtx &L, void *sv, int n, uint64_t mask, int parity, double scale) {
    using C = typename CT<R>::T;
    constexpr int V = CT<R>::V;
    const uint64_t n_units = (1ull << n) / V;
    const uint64_t grid = (n_units + kThreads - 1) / kThreads;
    k_collapse<R><<<(unsigned)grid, kThreads, 0, L.stream>>>(reinterpret_cast<C *>(sv), n_units, mask, parity,
                                                             (R)scale);
    ++*L.launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sampler (Table I, "Sampler"): measurement outcomes without collapse. The
// state is cut into segments of 2^seg_log amplitudes; their probabilities are
// summed (FP32 runs of 16 terms, FP64 beyond, fixed order), the segment sums
// are scanned into a cumulative distribution by one block in a fixed order,
// and each sample -- one warp -- binary-searches the segment and scans it
// with warp prefix sums for the first index whose cumulative probability
// exceeds r * total.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_seg_sums(const typename CT<R>::T *__restrict__ sv, int seg_log, uint64_t n_seg, double *__restrict__ seg) {
    __shared__ double red[kThreads / 32];
    const uint64_t S = 1ull << seg_log;
    for (uint64_t g = blockIdx.x; g < n_seg; g += gridDim.x) {
        double acc = 0.0;
        R run = R(0);
        int cnt = 0;
        for (uint64_t i = threadIdx.x; i < S; i += kThreads) {
            const typename CT<R>::T a = sv[g * S + i];
            run += a.x * a.x + a.y * a.y;
            if (++cnt == 16) {
                acc += (double)run;
                run = R(0);
                cnt = 0;
            }
        }
        acc += (double)run;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            seg[g] = t;
        }
        __syncthreads();
    }
}

// inclusive scan of seg[0 .. n) in place, one block of 1024 threads, fixed order
__global__ void __launch_bounds__(1024) k_scan(double *__restrict__ seg, uint64_t n) {
    __shared__ double part[1024];
    const uint64_t per = (n + 1023) / 1024;
    const uint64_t b = threadIdx.x * per, e = (b + per < n) ? b + per : n;
    double run = 0.0;
    for (uint64_t i = b; i < e; ++i) {
        run += seg[i];
        seg[i] = run;
    }
    part[threadIdx.x] = run;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 1024; ++i) {
            const double v = part[i];
            part[i] = t;
            t += v;
        }
    }
    __syncthreads();
    const double off = part[threadIdx.x];
    for (uint64_t i = b; i < e; ++i) seg[i] += off;
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_sample(const typename CT<R>::T *__restrict__ sv, int seg_log, uint64_t n_seg, const double *__restrict__ seg,
         const double *__restrict__ rands, int n_samples, long long *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int sidx = (int)((blockIdx.x * (uint64_t)kThreads + threadIdx.x) >> 5);
    if (sidx >= n_samples) return;
    const double total = seg[n_seg - 1];
    const double target = rands[sidx] * total;
    uint64_t lo = 0, hi = n_seg - 1;            // first segment with cum > target
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (seg[mid] > target) hi = mid; else lo = mid + 1;
    }
    const double before = lo > 0 ? seg[lo - 1] : 0.0;
    const double want = target - before;
    const uint64_t S = 1ull << seg_log, base = lo * S;
    double running = 0.0;
    long long last_nz = (long long)base;
    for (uint64_t c = 0; c < S; c += 32) {
        const uint64_t i = base + c + lane;
        double p = 0.0;
        if (c + lane < S) {
            const typename CT<R>::T a = sv[i];
            p = (double)a.x * (double)a.x + (double)a.y * (double)a.y;
        }
        double inc = p;                         // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, running + inc > want && p > 0.0);
        if (hit) {
            if (lane == 0) out[sidx] = (long long)(base + c + (__ffs(hit) - 1));
            return;
        }
        const unsigned nz = __ballot_sync(0xffffffffu, p > 0.0);
        if (nz) last_nz = (long long)(base + c + (31 - __clz(nz)));
        running += __shfl_sync(0xffffffffu, inc, 31);
    }
    // rounding left the target past the segment's own sum: its last nonzero amplitude
    if (lane == 0) out[sidx] = last_nz;
}

template <typename R>
cudaError_t sample_t(const LaunchCtx &L, const void *sv, int n, const double *d_r, int ns, double *d_seg,
                     long long *d_out) {
    using C = typename CT<R>::T;
    int seg_log = n - 20 > 12 ? n - 20 : 12;
    if (seg_log > n) seg_log = n;
    const uint64_t n_seg = 1ull << (n - seg_log);
    uint64_t grid = n_seg;
    const uint64_t cap = (uint64_t)L.num_sms * 8;
    if (grid > cap) grid = cap;
    k_seg_sums<R><<<(unsigned)grid, kThreads, 0, L.stream>>>(reinterpret_cast<const C *>(sv), seg_log, n_seg, d_seg);
    ++*L.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan<<<1, 1024, 0, L.stream>>>(d_seg, n_seg);
    ++*L.launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t blocks = ((uint64_t)ns * 32 + kThreads - 1) / kThreads;
    k_sample<R><<<(unsigned)blocks, kThreads, 0, L.stream>>>(reinterpret_cast<const C *>(sv), seg_log, n_seg, d_seg,
                                                             d_r, ns, d_out);
    ++*L.launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// <Z_q> for every qubit in one pass: with p_i = |psi_i|^2 and S_q the sum of
// p_i over indices with bit q set, <Z_q> = sum_i p_i - 2 S_q. The state is cut
// into chunks of 8 amplitudes; block b owns the aligned chunk range
// [b 2^m, (b+1) 2^m) and thread t the chunks b 2^m + j 2^mt + t. So amplitude
// bits 0..2 vary inside a chunk (three partial sums), bits 3..3+mt-1 are the
// thread's (its whole total counts for them), bits 3+mt..3+m-1 follow the loop
// counter j (one partial sum each) and the bits above are fixed per block.
// FP32 over 16 chunks, FP64 beyond; partial rows [kZMax + 1] per block are
// summed in a fixed order by k_zall_finish.
// ---------------------------------------------------------------------------
constexpr int kZMax = 40;
constexpr int kZJ = 16;   // most loop-counter bits

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_zall(const typename CT<R>::T *__restrict__ sv, int n, int m, int mt, double *__restrict__ partials) {
    using C = typename CT<R>::T;
    __shared__ double row[kZMax + 1];
    const int mj = m - mt;
    const int t = threadIdx.x;
    const bool active = t < (1 << mt);
    const uint64_t c0 = (uint64_t)blockIdx.x << m;
    double dT = 0.0, dB[3] = {0.0, 0.0, 0.0}, dJ[kZJ];
    R fT = R(0), fB[3] = {R(0), R(0), R(0)}, fJ[kZJ];
#pragma unroll
    for (int q = 0; q < kZJ; ++q) { dJ[q] = 0.0; fJ[q] = R(0); }
    int cnt = 0;
    const uint64_t nj = 1ull << mj;
    for (uint64_t j = 0; active && j < nj; ++j) {
        const uint64_t c = c0 + (j << mt) + t;
        R p[8];
        if constexpr (sizeof(R) == 4) {
            const float4 *src = reinterpret_cast<const float4 *>(sv) + 4 * c;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float4 f = src[h];
                p[2 * h] = f.x * f.x + f.y * f.y;
                p[2 * h + 1] = f.z * f.z + f.w * f.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const C x = sv[8 * c + e];
                p[e] = x.x * x.x + x.y * x.y;
            }
        }
        const R tot = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
        fT += tot;
        fB[0] += (p[1] + p[3]) + (p[5] + p[7]);
        fB[1] += (p[2] + p[3]) + (p[6] + p[7]);
        fB[2] += (p[4] + p[5]) + (p[6] + p[7]);
#pragma unroll
        for (int q = 0; q < kZJ; ++q)
            if (q < mj && ((j >> q) & 1u)) fJ[q] += tot;
        if (++cnt == 16) {
            dT += (double)fT;
            fT = R(0);
#pragma unroll
            for (int q = 0; q < 3; ++q) { dB[q] += (double)fB[q]; fB[q] = R(0); }
#pragma unroll
            for (int q = 0; q < kZJ; ++q) { dJ[q] += (double)fJ[q]; fJ[q] = R(0); }
            cnt = 0;
        }
    }
    dT += (double)fT;
#pragma unroll
    for (int q = 0; q < 3; ++q) dB[q] += (double)fB[q];
#pragma unroll
    for (int q = 0; q < kZJ; ++q) dJ[q] += (double)fJ[q];
    // block sums in a fixed order, all values at once: value v = 0 total, 1..3 the
    // chunk bits, 4 .. 4+mt-1 the thread-index bits, then the loop-counter bits;
    // each warp reduces every value with shuffles, then thread v adds the warps'
    // results in warp order
    constexpr int kV = 4 + 8 + kZJ;
    __shared__ double wred[kThreads / 32][kV];
    const int nv = 4 + mt + mj;
    auto warp_put = [&](double x, int v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((t & 31) == 0) wred[t >> 5][v] = x;
    };
    warp_put(dT, 0);
#pragma unroll
    for (int q = 0; q < 3; ++q) warp_put(dB[q], 1 + q);
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if (b < mt) warp_put(((t >> b) & 1) ? dT : 0.0, 4 + b);
#pragma unroll
    for (int q = 0; q < kZJ; ++q)
        if (q < mj) warp_put(dJ[q], 4 + mt + q);
    __syncthreads();
    __shared__ double total_s;
    if (t < nv) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += wred[w][t];
        if (t == 0) total_s = acc;
        else row[t - 1] = acc;                 // qubit t - 1: chunk, thread and loop bits in order
    }
    __syncthreads();
    const double total = total_s;
    if (t == 0) {
        const uint64_t base = c0 << 3;
        for (int q = 3 + m; q < n; ++q) row[q] = ((base >> q) & 1u) ? total : 0.0;
        for (int q = n; q < kZMax; ++q) row[q] = 0.0;
        row[kZMax] = total;
    }
    __syncthreads();
    for (int q = t; q <= kZMax; q += kThreads) partials[(size_t)blockIdx.x * (kZMax + 1) + q] = row[q];
}

// out[q] = total - 2 S_q for q < n, out[n] = total; partials summed in block order
__global__ void __launch_bounds__(64) k_zall_finish(const double *__restrict__ partials, int nblocks, int n,
                                                    double *__restrict__ out) {
    const int q = threadIdx.x;
    if (q > kZMax) return;
    double a = 0.0, tt = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        a += partials[(size_t)b * (kZMax + 1) + q];
        tt += partials[(size_t)b * (kZMax + 1) + kZMax];
    }
    if (q < n) out[q] = tt - 2.0 * a;
    if (q == kZMax) out[n] = tt;
}

template <typename R>
cudaError_t zall_t(const LaunchCtx &L, const void *sv, int n, double *d_partials, int maxb, double *d_out) {
    using C = typename CT<R>::T;
    // m = log2(chunks per block): about 512 blocks (measured faster than 2048 at 28
    // qubits, where the single-block finish pass grows with the block count), at
    // least 2^min(n-3, 8) chunks each, at most kZJ loop bits
    int m = n - 3 - 9;
    const int lo = (n - 3) < 8 ? (n - 3) : 8;
    if (m < lo) m = lo;
    if (m > 8 + kZJ) m = 8 + kZJ;
    const int mt = m < 8 ? m : 8;
    const uint64_t blocks = 1ull << (n - 3 - m);
    if (blocks * (kZMax + 1) > (uint64_t)maxb * 8) return cudaErrorInvalidValue;
    k_zall<R><<<(unsigned)blocks, kThreads, 0, L.stream>>>(reinterpret_cast<const C *>(sv), n, m, mt, d_partials);
    ++*L.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_zall_finish<<<1, 64, 0, L.stream>>>(d_partials, (int)blocks, n, d_out);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pauli(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, const PauliPass &P,
                         double *d_partials, int max_partial_blocks, double *d_out) {
    if (n < 1) return cudaErrorInvalidValue;
    return dt == SV_C64 ? pauli_t<float>(L, sv, n, P, d_partials, max_partial_blocks, d_out)
                        : pauli_t<double>(L, sv, n, P, d_partials, max_partial_blocks, d_out);
}

cudaError_t launch_parity(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, uint64_t mask,
                          double *d_partials, int max_partial_blocks, double *d_out) {
    if (n < 1) return cudaErrorInvalidValue;
    return dt == SV_C64 ? parity_t<float>(L, sv, n, mask, d_partials, max_partial_blocks, d_out)
                        : parity_t<double>(L, sv, n, mask, d_partials, max_partial_blocks, d_out);
}

cudaError_t launch_collapse(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, uint64_t mask, int parity,
                            double scale) {
    if (n < 1) return cudaErrorInvalidValue;
    return dt == SV_C64 ? collapse_t<float>(L, sv, n, mask, parity, scale)
                        : collapse_t<double>(L, sv, n, mask, parity, scale);
}

cudaError_t launch_sample(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, const double *d_r, int n_samples,
                          double *d_seg, long long *d_out) {
    if (n < 1 || n_samples < 1) return cudaErrorInvalidValue;
    return dt == SV_C64 ? sample_t<float>(L, sv, n, d_r, n_samples, d_seg, d_out)
                        : sample_t<double>(L, sv, n, d_r, n_samples, d_seg, d_out);
}

cudaError_t launch_zall(const LaunchCtx &L, sv_dtype_t dt, const void *sv, int n, double *d_partials,
                        int max_partial_blocks, double *d_out) {
    if (n < 3 || n > kZMax) return cudaErrorInvalidValue;
    return dt == SV_C64 ? zall_t<float>(L, sv, n, d_partials, max_partial_blocks, d_out)
                        : zall_t<double>(L, sv, n, d_partials, max_partial_blocks, d_out);
}

cudaError_t launch_set_basis(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, uint64_t index) {
    const size_t bytes = (size_t(1) << n) * (dt == SV_C64 ? 8 : 16);
    cudaError_t e = cudaMemsetAsync(sv, 0, bytes, L.stream);
    if (e != cudaSuccess) return e;
    if (dt == SV_C64)
        k_set_one<float><<<1, 1, 0, L.stream>>>(reinterpret_cast<float2 *>(sv), index);
    else
        k_set_one<double><<<1, 1, 0, L.stream>>>(reinterpret_cast<double2 *>(sv), index);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace svk
