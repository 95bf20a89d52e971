// k_gate.cu -- gate application on CUDA cores (Table I, "Gate application";
// Sec. II-B: gate application is memory-bound for small k, so every kernel here
// is a single streaming pass that reads and writes each touched amplitude once).
//
// Kernel families, all in place:
//   k_dense      dense 2^k x 2^k product per group, k <= 4, group data in registers;
//   k_dense_blk  the same for k = 2..4 with two or more low targets, the low bits
//                staged through shared memory by warps;
//   k_dense5     dense product for k = 5 in complex64, one group per thread in
//                registers, the matrix broadcast from shared memory;
//   k_dense6     the same for k = 6, a group over a pair of lanes;
//   k_dense_smem dense product for any k <= 6, a tile of groups staged in shared memory
//                (complex128, and states of fewer than 16 groups; for k = 5, 6 the work
//                is ALU-bound on CUDA cores; the tensor-core path in k_tc.cu is the
//                fast one);
//   k_diag       diagonal matrix on the amplitudes where the controls hold;
//   k_perm       generalized permutation matrix (one nonzero per row/column).
//
// Vector access. A complex64 amplitude is 8 bytes; every access is 16 bytes wide
// where the index layout allows it:
//   PAIR   bit 0 is neither a target nor a control: groups g and g+1 start at
//          adjacent amplitudes, so one float4 holds member j of both groups;
//   T0     bit 0 is the lowest target: members 2m and 2m+1 of a group are
//          adjacent, so one float4 holds both;
//   SCALAR one amplitude per access (complex128: always 16 bytes; complex64 with a
//          control on bit 0: 8 bytes).
// Within a warp, consecutive threads take consecutive units, so for every member
// the warp reads one contiguous run (coalesced), also for high target qubits.
#include <cmath>
#include <type_traits>
#include <vector>

#include "sv_internal.h"

namespace svk {
namespace {

enum Mode { PAIR = 0, T0 = 1, SCALAR = 2 };
constexpr int kThreads = 256;

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

__device__ __forceinline__ float fmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return __fma_rn(a, b, c); }

// acc += m * v (complex)
template <typename C>
__device__ __forceinline__ void cmad(C &acc, const C &m, const C &v) {
    acc.x = fmac(m.x, v.x, acc.x);
    acc.x = fmac(-m.y, v.y, acc.x);
    acc.y = fmac(m.x, v.y, acc.y);
    acc.y = fmac(m.y, v.x, acc.y);
}

template <typename C>
__device__ __forceinline__ C cmul(const C &a, const C &b) {
    C r;
    r.x = fmac(a.x, b.x, -a.y * b.y);
    r.y = fmac(a.x, b.y, a.y * b.x);
    return r;
}

// Zero bits inserted at G.pos (ascending), then the control bits set.
__device__ __forceinline__ uint64_t insert_zeros(uint64_t g, const GroupGeom &G) {
#pragma unroll 1
    for (int i = 0; i < G.ns; ++i) {
        const uint64_t lo = g & ((1ull << G.pos[i]) - 1ull);
        g = ((g ^ lo) << 1) | lo;
    }
    return g | G.cset;
}

__device__ __forceinline__ float4 ld16(const float2 *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st16(float2 *p, const float4 &v) { *reinterpret_cast<float4 *>(p) = v; }

template <int K> struct Offs { uint64_t o[1 << K]; };
template <typename R, int K> struct MatK { typename CT<R>::T m[1 << (2 * K)]; };

// ---------------------------------------------------------------------------
// dense, k <= 4, registers
// ---------------------------------------------------------------------------
template <typename R, int K, int MODE, int U>
__global__ void __launch_bounds__(kThreads)
k_dense(typename CT<R>::T *__restrict__ sv, uint64_t n_units, GroupGeom G, Offs<K> O, MatK<R, K> M) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    constexpr int E = (MODE == PAIR) ? 2 : 1;
    const uint64_t u0 = (uint64_t)blockIdx.x * (kThreads * U) + threadIdx.x;
    C v[U][D][E];
    uint64_t base[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t unit = u0 + (uint64_t)u * kThreads;
        base[u] = insert_zeros(MODE == PAIR ? (unit << 1) : unit, G);
        if (unit < n_units) {
            if constexpr (MODE == PAIR) {
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const float4 f = ld16(reinterpret_cast<const float2 *>(sv) + base[u] + O.o[j]);
                    v[u][j][0] = C{f.x, f.y};
                    v[u][j][E - 1] = C{f.z, f.w};
                }
            } else if constexpr (MODE == T0) {
#pragma unroll
                for (int m = 0; m < D / 2; ++m) {
                    const float4 f = ld16(reinterpret_cast<const float2 *>(sv) + base[u] + O.o[2 * m]);
                    v[u][2 * m][0] = C{f.x, f.y};
                    v[u][2 * m + 1][0] = C{f.z, f.w};
                }
            } else {
#pragma unroll
                for (int j = 0; j < D; ++j) v[u][j][0] = sv[base[u] + O.o[j]];
            }
        }
    }
    if constexpr (MODE == T0 && K >= 3 && U > 1) {
        // the thread's U groups side by side in the innermost loop, as PAIR mode
        // does with its two: each matrix entry feeds U products (same sums in the
        // same order per group); a group past the end computes on zeros, unstored
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (u0 + (uint64_t)u * kThreads >= n_units)
#pragma unroll
                for (int l = 0; l < D; ++l) v[u][l][0] = C{0, 0};
#pragma unroll
        for (int j0 = 0; j0 < D; j0 += 2) {
            C w[2][U];
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                C acc[U];
#pragma unroll
                for (int u = 0; u < U; ++u) acc[u] = C{0, 0};
#pragma unroll
                for (int l = 0; l < D; ++l) {
                    const C m = M.m[(j0 + jj) * D + l];
#pragma unroll
                    for (int u = 0; u < U; ++u) cmad(acc[u], m, v[u][l][0]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) w[jj][u] = acc[u];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (u0 + (uint64_t)u * kThreads < n_units)
                    st16(reinterpret_cast<float2 *>(sv) + base[u] + O.o[j0],
                         make_float4(w[0][u].x, w[0][u].y, w[1][u].x, w[1][u].y));
        }
        return;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t unit = u0 + (uint64_t)u * kThreads;
        if (unit >= n_units) continue;
        if constexpr (K >= 3) {
            // each output row (two in T0 mode) is stored as soon as its sums are formed: only
            // the inputs stay live, which for k = 4 halves the registers a thread holds and
            // lets more blocks share an SM (same sums in the same order)
            constexpr int RW = (MODE == T0) ? 2 : 1;
#pragma unroll
            for (int j0 = 0; j0 < D; j0 += RW) {
                C w[RW][E];
#pragma unroll
                for (int jj = 0; jj < RW; ++jj) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        C acc{0, 0};
#pragma unroll
                        for (int l = 0; l < D; ++l) cmad(acc, M.m[(j0 + jj) * D + l], v[u][l][e]);
                        w[jj][e] = acc;
                    }
                }
                if constexpr (MODE == PAIR)
                    st16(reinterpret_cast<float2 *>(sv) + base[u] + O.o[j0],
                         make_float4(w[0][0].x, w[0][0].y, w[0][E - 1].x, w[0][E - 1].y));
                else if constexpr (MODE == T0)
                    st16(reinterpret_cast<float2 *>(sv) + base[u] + O.o[j0],
                         make_float4(w[0][0].x, w[0][0].y, w[RW - 1][0].x, w[RW - 1][0].y));
                else
                    sv[base[u] + O.o[j0]] = w[0][0];
            }
            continue;
        }
        C w[D][E];
#pragma unroll
        for (int j = 0; j < D; ++j) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                C acc{0, 0};
#pragma unroll
                for (int l = 0; l < D; ++l) cmad(acc, M.m[j * D + l], v[u][l][e]);
                w[j][e] = acc;
            }
        }
        if constexpr (MODE == PAIR) {
#pragma unroll
            for (int j = 0; j < D; ++j)
                st16(reinterpret_cast<float2 *>(sv) + base[u] + O.o[j],
                     make_float4(w[j][0].x, w[j][0].y, w[j][E - 1].x, w[j][E - 1].y));
        } else if constexpr (MODE == T0) {
#pragma unroll
            for (int m = 0; m < D / 2; ++m)
                st16(reinterpret_cast<float2 *>(sv) + base[u] + O.o[2 * m],
                     make_float4(w[2 * m][0].x, w[2 * m][0].y, w[2 * m + 1][0].x, w[2 * m + 1][0].y));
        } else {
#pragma unroll
            for (int j = 0; j < D; ++j) sv[base[u] + O.o[j]] = w[j][0];
        }
    }
}

// ---------------------------------------------------------------------------
// dense, k = 2..4, complex64, low targets: warp-staged super-groups
// ---------------------------------------------------------------------------
// With two or more low targets (qubit 1 among them), consecutive groups (or
// group pairs) start 32 bytes or more apart, so the thread-per-group access
// modes above touch only part of every sector per instruction. Here the low
// bits are taken as a block: with
// KLO targets below bit B = 5 + KLO, the 2^B amplitudes of bits 0 .. B-1 hold
// 32 whole groups' low members, contiguous in memory (2^B * 8 >= 512 bytes).
// A warp takes one super-group -- fixed values of every bit at or above B that
// is neither a high target nor a control, i.e. 2^(k-KLO) such blocks, one per
// high member -- loads it with consecutive float4 per lane (every instruction
// covers whole sectors), writes it to shared memory, lets each lane apply the
// gate to its own group there, and stores it back the same way. Shared memory
// is swizzled (amplitude a at a ^ ((a >> 4) & 15), linear over XOR) so that the
// lanes' group members fall on different banks whatever the target bits.
template <int KLO> struct LoOffs { uint32_t o[1 << KLO]; uint8_t pos[KLO]; };

__device__ __forceinline__ uint32_t swz(uint32_t a) { return a ^ ((a >> 4) & 15u); }

template <int K, int KLO>
__global__ void __launch_bounds__(kThreads)
k_dense_blk(float2 *__restrict__ sv, uint64_t n_sg, GroupGeom Ghi, LoOffs<KLO> Olo, Offs<K - KLO> Ohi,
            MatK<float, K> M) {
    constexpr int D = 1 << K, DLO = 1 << KLO;
    constexpr int B = 5 + KLO, BLK = 1 << B;   // amplitudes of one block: 32 groups' low members
    constexpr int NA = D * 32;                 // amplitudes of a super-group
    constexpr int PER = NA / 64;               // float4 per lane
    __shared__ float2 sm[kThreads / 32][NA];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *buf = sm[warp];
    const uint64_t sgi = (uint64_t)blockIdx.x * (kThreads / 32) + warp;
    if (sgi >= n_sg) return;                   // warp-uniform
    const uint64_t base = insert_zeros(sgi << B, Ghi);
    float4 v[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t a = 2u * (uint32_t)(lane + 32 * r);
        v[r] = ld16(sv + base + Ohi.o[a >> B] + (a & (BLK - 1)));
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t a = 2u * (uint32_t)(lane + 32 * r), s = swz(a);
        const float4 f = v[r];
        *reinterpret_cast<float4 *>(buf + (s & ~1u)) = (s & 1u) ? make_float4(f.z, f.w, f.x, f.y) : f;
    }
    __syncwarp();
    // this lane's group: zero bits inserted at the low target positions
    uint32_t glo = (uint32_t)lane;
#pragma unroll
    for (int i = 0; i < KLO; ++i) {
        const uint32_t lo = glo & ((1u << Olo.pos[i]) - 1u);
        glo = ((glo ^ lo) << 1) | lo;
    }
    float2 x[D];
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = buf[swz((uint32_t)(j >> KLO) * BLK + glo + Olo.o[j & (DLO - 1)])];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < D; ++l) cmad(acc, M.m[j * D + l], x[l]);
        buf[swz((uint32_t)(j >> KLO) * BLK + glo + Olo.o[j & (DLO - 1)])] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t a = 2u * (uint32_t)(lane + 32 * r), s = swz(a);
        const float4 f = *reinterpret_cast<const float4 *>(buf + (s & ~1u));
        st16(sv + base + Ohi.o[a >> B] + (a & (BLK - 1)), (s & 1u) ? make_float4(f.z, f.w, f.x, f.y) : f);
    }
}

// ---------------------------------------------------------------------------
// dense, any k <= 6, tile of 2048 amplitudes in shared memory, persistent grid
// ---------------------------------------------------------------------------
constexpr int kTile = 2048;

template <typename R, int K>
__global__ void __launch_bounds__(kThreads)
k_dense_smem(typename CT<R>::T *__restrict__ sv, uint64_t n_groups, GroupGeom G, Offs<K> O,
             const typename CT<R>::T *__restrict__ Mg) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    constexpr int GB = kTile / D;          // groups per tile (>= 32)
    constexpr int PER = kTile / kThreads;  // amplitudes per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Ms = reinterpret_cast<C *>(smem_raw);
    C *Ts = Ms + D * D;
    for (int i = threadIdx.x; i < D * D; i += kThreads) Ms[i] = Mg[i];
    const uint64_t n_tiles = (n_groups + GB - 1) / GB;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        uint64_t addr[PER];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = threadIdx.x + r * kThreads;
            const int j = idx / GB, g = idx % GB;
            const uint64_t gg = tile * GB + g;
            addr[r] = insert_zeros(gg, G) + O.o[j];
            if (gg < n_groups) Ts[idx] = sv[addr[r]];
        }
        __syncthreads();
        C out[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = threadIdx.x + r * kThreads;
            const int j = idx / GB, g = idx % GB;
            C acc{0, 0};
#pragma unroll 8
            for (int l = 0; l < D; ++l) cmad(acc, Ms[j * D + l], Ts[l * GB + g]);
            out[r] = acc;
        }
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = threadIdx.x + r * kThreads;
            if (tile * GB + (idx % GB) < n_groups) sv[addr[r]] = out[r];
        }
    }
}

// ---------------------------------------------------------------------------
// dense k = 5, complex64: compute-bound on CUDA cores (128 FMAs per amplitude
// against 16 bytes moved, above the FP32 : HBM ratio). Each thread holds one
// group's 32 amplitudes in registers and forms its outputs 8 at a time from
// the matrix in shared memory (16-byte broadcast loads, two entries of a row
// per load: one load per 8 FMAs), writing each output straight back to its
// amplitude -- all inputs are in registers by then and no other thread
// touches the group. With qubit 0 a target (PAIR0) members 2m and 2m + 1 are
// adjacent amplitudes and move as one 16-byte access.
// ---------------------------------------------------------------------------
template <bool PAIR0>
__global__ void __launch_bounds__(kThreads, 2)
k_dense5(float2 *__restrict__ sv, uint64_t n_groups, GroupGeom G, Offs<5> O, const float2 *__restrict__ Mg) {
    __shared__ __align__(16) float2 Ms[32 * 32];
    for (int i = threadIdx.x; i < 32 * 32; i += kThreads) Ms[i] = Mg[i];
    __syncthreads();
    const float4 *M4 = reinterpret_cast<const float4 *>(Ms);
    for (uint64_t g = (uint64_t)blockIdx.x * kThreads + threadIdx.x; g < n_groups;
         g += (uint64_t)gridDim.x * kThreads) {
        const uint64_t base = insert_zeros(g, G);
        float2 x[32];
        if constexpr (PAIR0) {
#pragma unroll
            for (int l = 0; l < 32; l += 2) {
                const float4 q = ld16(sv + base + O.o[l]);
                x[l] = make_float2(q.x, q.y);
                x[l + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int l = 0; l < 32; ++l) x[l] = sv[base + O.o[l]];
        }
        // the stores recompute their addresses from an opaque copy of the base,
        // so the 32 load addresses (64 registers) are not kept alive for them
        float2 *ps;
        asm volatile("mov.b64 %0, %1;" : "=l"(ps) : "l"(sv + base));
        // the batch loop stays rolled: unrolled, the kernel's 4096 FMAs per group
        // overflow the instruction cache (instruction-fetch stalls led the warp
        // states) and ran 20 % slower
#pragma unroll 1
        for (int j0 = 0; j0 < 32; j0 += 8) {
            float2 acc[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) acc[jj] = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < 32; l += 2) {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const float4 m2 = M4[((j0 + jj) * 32 + l) >> 1];
                    cmad(acc[jj], make_float2(m2.x, m2.y), x[l]);
                    cmad(acc[jj], make_float2(m2.z, m2.w), x[l + 1]);
                }
            }
            if constexpr (PAIR0) {
#pragma unroll
                for (int jj = 0; jj < 8; jj += 2)
                    st16(ps + O.o[j0 + jj], make_float4(acc[jj].x, acc[jj].y, acc[jj + 1].x, acc[jj + 1].y));
            } else {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) ps[O.o[j0 + jj]] = acc[jj];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// dense k = 6, complex64: as k_dense5, but a group's 64 amplitudes are split
// over the two lanes of a pair (h = lane & 1 holds the members whose top bit is
// h). Each lane forms partial sums of 8 outputs at a time over its 32 inputs,
// takes its partner's partials with one shuffle per value (the sum a + b is the
// same in both lanes) and stores half of them. The host uses it only when the
// group count is a multiple of 16, so every warp's pairs enter and leave the
// grid-stride loop together and the shuffles see the whole warp.
// ---------------------------------------------------------------------------
template <bool PAIR0>
__global__ void __launch_bounds__(kThreads, 2)
k_dense6(float2 *__restrict__ sv, uint64_t n_groups, GroupGeom G, Offs<6> O, const float2 *__restrict__ Mg) {
    // the two lanes of a pair read the two halves of a matrix row at once: with
    // the halves 17 (not 16) 16-byte units apart and rows 34 apart, the two
    // addresses fall on different banks and each broadcast load is one
    // shared-memory wavefront instead of two (unpadded: 1.12 against 1.33 TB/s)
    __shared__ __align__(16) float2 Ms[64 * 34 * 2];
    for (int i = threadIdx.x; i < 64 * 64; i += kThreads) {
        const int j = i >> 6, l = i & 63, hh = l >> 5, q2 = l & 31;
        Ms[(j * 34 + hh * 17 + (q2 >> 1)) * 2 + (q2 & 1)] = Mg[i];
    }
    __syncthreads();
    const int h = threadIdx.x & 1;
    const float4 *M4 = reinterpret_cast<const float4 *>(Ms) + h * 17;   // row j: M4[j * 34 + i / 2]
    for (uint64_t g = ((uint64_t)blockIdx.x * kThreads + threadIdx.x) >> 1; g < n_groups;
         g += ((uint64_t)gridDim.x * kThreads) >> 1) {
        const uint64_t base = insert_zeros(g, G);
        float2 x[32];
        if constexpr (PAIR0) {
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                const float4 q = ld16(sv + base + O.o[32 * h + i]);
                x[i] = make_float2(q.x, q.y);
                x[i + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = sv[base + O.o[32 * h + i]];
        }
        float2 *ps;
        asm volatile("mov.b64 %0, %1;" : "=l"(ps) : "l"(sv + base));
#pragma unroll 1
        for (int j0 = 0; j0 < 64; j0 += 8) {
            float2 acc[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) acc[jj] = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const float4 m2 = M4[(j0 + jj) * 34 + (i >> 1)];
                    cmad(acc[jj], make_float2(m2.x, m2.y), x[i]);
                    cmad(acc[jj], make_float2(m2.z, m2.w), x[i + 1]);
                }
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                acc[jj].x += __shfl_xor_sync(0xffffffffu, acc[jj].x, 1);
                acc[jj].y += __shfl_xor_sync(0xffffffffu, acc[jj].y, 1);
            }
            // lane h stores outputs j0 + 4h .. j0 + 4h + 3 (selected, not indexed,
            // so that acc stays in registers)
            float2 mine[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) mine[p] = h ? acc[4 + p] : acc[p];
            if constexpr (PAIR0) {
#pragma unroll
                for (int p = 0; p < 4; p += 2)
                    st16(ps + O.o[j0 + 4 * h + p], make_float4(mine[p].x, mine[p].y, mine[p + 1].x, mine[p + 1].y));
            } else {
#pragma unroll
                for (int p = 0; p < 4; ++p) ps[O.o[j0 + 4 * h + p]] = mine[p];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// diagonal on targets where the controls hold (k = 0 is a phase on a subspace)
// ---------------------------------------------------------------------------
template <typename R> struct DiagP {
    typename CT<R>::T d[1 << SV_MAX_TARGETS];
    int tpos[SV_MAX_TARGETS];
    int k;
};

template <typename C, typename P>
__device__ __forceinline__ C diag_scale(const C &a, uint64_t idx, const P &p) {
    int j = 0;
#pragma unroll 1
    for (int t = 0; t < p.k; ++t) j |= (int)((idx >> p.tpos[t]) & 1u) << t;
    return cmul(p.d[j], a);
}

template <typename R, int MODE, int U>
__global__ void __launch_bounds__(kThreads)
k_diag(typename CT<R>::T *__restrict__ sv, uint64_t n_units, GroupGeom G, DiagP<R> P) {
    using C = typename CT<R>::T;
    const uint64_t u0 = (uint64_t)blockIdx.x * (kThreads * U) + threadIdx.x;
    if constexpr (MODE == PAIR) {
        float4 f[U];
        uint64_t idx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t unit = u0 + (uint64_t)u * kThreads;
            idx[u] = insert_zeros(unit << 1, G);
            if (unit < n_units) f[u] = ld16(reinterpret_cast<const float2 *>(sv) + idx[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u0 + (uint64_t)u * kThreads >= n_units) continue;
            const C a = diag_scale(C{f[u].x, f[u].y}, idx[u], P);
            const C b = diag_scale(C{f[u].z, f[u].w}, idx[u] + 1, P);
            st16(reinterpret_cast<float2 *>(sv) + idx[u], make_float4(a.x, a.y, b.x, b.y));
        }
    } else {
        C a[U];
        uint64_t idx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t unit = u0 + (uint64_t)u * kThreads;
            idx[u] = insert_zeros(unit, G);
            if (unit < n_units) a[u] = sv[idx[u]];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u0 + (uint64_t)u * kThreads >= n_units) continue;
            sv[idx[u]] = diag_scale(a[u], idx[u], P);
        }
    }
}

// ---------------------------------------------------------------------------
// generalized permutation: out[j] = d[j] * in[perm[j]]; source l goes to
// destination pinv[l] with factor d[pinv[l]] (both precomputed on the host)
// ---------------------------------------------------------------------------
template <typename R, int K> struct PermP {
    typename CT<R>::T f[1 << K];   // factor applied to source member l
    uint64_t dst[1 << K];          // offset of the destination of source member l
    uint64_t src[1 << K];          // offset of source member l
};

template <typename R, int K, int MODE, int U>
__global__ void __launch_bounds__(kThreads)
k_perm(typename CT<R>::T *__restrict__ sv, uint64_t n_units, GroupGeom G, PermP<R, K> P) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    constexpr int E = (MODE == PAIR) ? 2 : 1;
    const uint64_t u0 = (uint64_t)blockIdx.x * (kThreads * U) + threadIdx.x;
    C v[U][D][E];
    uint64_t base[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t unit = u0 + (uint64_t)u * kThreads;
        base[u] = insert_zeros(MODE == PAIR ? (unit << 1) : unit, G);
        if (unit < n_units) {
#pragma unroll
            for (int l = 0; l < D; ++l) {
                if constexpr (MODE == PAIR) {
                    const float4 f = ld16(reinterpret_cast<const float2 *>(sv) + base[u] + P.src[l]);
                    v[u][l][0] = C{f.x, f.y};
                    v[u][l][E - 1] = C{f.z, f.w};
                } else {
                    v[u][l][0] = sv[base[u] + P.src[l]];
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (u0 + (uint64_t)u * kThreads >= n_units) continue;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const C a = cmul(P.f[l], v[u][l][0]);
            if constexpr (MODE == PAIR) {
                const C b = cmul(P.f[l], v[u][l][E - 1]);
                st16(reinterpret_cast<float2 *>(sv) + base[u] + P.dst[l], make_float4(a.x, a.y, b.x, b.y));
            } else {
                sv[base[u] + P.dst[l]] = a;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename C> C to_c(const double *z) { return C{(decltype(C{}.x))z[0], (decltype(C{}.x))z[1]}; }

inline unsigned grid_for(uint64_t units, int per_block) {
    const uint64_t b = (units + per_block - 1) / per_block;
    return (unsigned)(b == 0 ? 1 : b);
}

// bytes in flight per thread are kept near 64-128 B
template <typename R, int K, int MODE> constexpr int dense_u() {
    constexpr int unit_bytes = (MODE == PAIR ? 16 : (int)sizeof(typename CT<R>::T)) * (1 << K) / (MODE == T0 ? 2 : 1);
    return unit_bytes >= 128 ? 1 : (unit_bytes >= 64 ? 2 : 4);
}

template <typename R, int K, int MODE>
cudaError_t run_dense_reg(const LaunchCtx &L, void *sv, uint64_t n_units, const GroupGeom &G, const Offs<K> &O,
                          const MatK<R, K> &M) {
    constexpr int U = dense_u<R, K, MODE>();
    k_dense<R, K, MODE, U><<<grid_for(n_units, kThreads * U), kThreads, 0, L.stream>>>(
        reinterpret_cast<typename CT<R>::T *>(sv), n_units, G, O, M);
    ++*L.launches;
    return cudaGetLastError();
}

template <int K, int KLO>
cudaError_t run_dense_blk(const LaunchCtx &L, void *sv, uint64_t n_sg, const GroupGeom &Ghi, const LoOffs<KLO> &Olo,
                          const Offs<K - KLO> &Ohi, const MatK<float, K> &M) {
    k_dense_blk<K, KLO><<<grid_for(n_sg, kThreads / 32), kThreads, 0, L.stream>>>(reinterpret_cast<float2 *>(sv), n_sg,
                                                                                   Ghi, Olo, Ohi, M);
    ++*L.launches;
    return cudaGetLastError();
}

// The warp-staged kernel takes a dense gate on a complex64 state when qubit 1
// and a second target fall inside the block (k = 2, 3) or all targets fall
// inside the block or three below bit 5 (k = 4),
// every control sits at or above the block (bit B = 5 + the number of targets
// below B) and at least one super-group exists. `G` holds
// the sorted target and control positions; targets ascending in tpos.
template <int K>
bool try_dense_blk(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, const MatK<float, K> &M,
                   cudaError_t &e) {
    // k = 2, 3: qubit 1 and a second target inside the block; k = 4: all four
    // targets inside the block, or three below bit 5. There the thread-per-group
    // modes leave a warp's accesses spread thin (measured on the 28-qubit state:
    // (0,1,2,3) 6.4 against 4.4 TB/s); with fewer low targets PAIR / T0 mode is
    // faster, its two groups per thread sharing every matrix entry ((1,9,21,22)
    // 6.1 against 5.3, (0,1,9,20) 6.1 against 5.6, (3,4,9,14) 6.3 against 5.6,
    // (1,9,12) 7.1 against 6.7, (1,9) 7.0 against 6.8)
    int klo = 0;
    while (klo < K && tpos[klo] < 5 + klo) ++klo;   // B = 5 + klo with klo targets below B
    bool t1 = false;
    int lo5 = 0;
    for (int t = 0; t < K; ++t) {
        t1 |= tpos[t] == 1;
        lo5 += tpos[t] < 5;
    }
    if (K >= 4 ? !(klo == K || lo5 >= 3) : !(t1 && klo >= 2)) return false;
    const int B = 5 + klo;
    GroupGeom Ghi{};
    Ghi.cset = G.cset;
    for (int i = 0; i < G.ns; ++i) {
        if (G.pos[i] < B) {
            bool is_target = false;
            for (int t = 0; t < klo; ++t) is_target |= tpos[t] == G.pos[i];
            if (!is_target) return false;             // a control below the block
            continue;
        }
        Ghi.pos[Ghi.ns++] = G.pos[i];
    }
    if (B + Ghi.ns > n) return false;                 // fewer than one super-group
    const uint64_t n_sg = 1ull << (n - B - Ghi.ns);
    auto run = [&](auto klo_c) {
        constexpr int KL = decltype(klo_c)::value;
        LoOffs<KL> Olo;
        for (int j = 0; j < (1 << KL); ++j) {
            uint32_t o = 0;
            for (int t = 0; t < KL; ++t)
                if ((j >> t) & 1) o |= 1u << tpos[t];
            Olo.o[j] = o;
        }
        for (int t = 0; t < KL; ++t) Olo.pos[t] = (uint8_t)tpos[t];
        Offs<K - KL> Ohi;
        for (int h = 0; h < (1 << (K - KL)); ++h) {
            uint64_t o = 0;
            for (int t = 0; t < K - KL; ++t)
                if ((h >> t) & 1) o |= 1ull << tpos[KL + t];
            Ohi.o[h] = o;
        }
        return run_dense_blk<K, KL>(L, sv, n_sg, Ghi, Olo, Ohi, M);
    };
    switch (klo) {
    case 1: e = run(std::integral_constant<int, 1>{}); break;
    case 2: e = run(std::integral_constant<int, (K >= 2 ? 2 : 1)>{}); break;
    case 3: e = run(std::integral_constant<int, (K >= 3 ? 3 : 1)>{}); break;
    default: e = run(std::integral_constant<int, (K >= 4 ? 4 : 1)>{}); break;
    }
    return true;
}

template <typename R, int K>
cudaError_t dense_reg(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, const double *mat) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    Offs<K> O;
    for (int j = 0; j < D; ++j) {
        uint64_t o = 0;
        for (int t = 0; t < K; ++t)
            if ((j >> t) & 1) o |= 1ull << tpos[t];
        O.o[j] = o;
    }
    MatK<R, K> M;
    for (int i = 0; i < D * D; ++i) M.m[i] = to_c<C>(mat + 2 * i);
    const uint64_t n_groups = 1ull << (n - G.ns);
    const bool bit0_special = G.ns > 0 && G.pos[0] == 0;
    if constexpr (sizeof(R) == 4) {
        if constexpr (K >= 2) {
            // low targets: warp-staged super-groups (needs every control above the block)
            cudaError_t e;
            if (try_dense_blk<K>(L, sv, n, G, tpos, M, e)) return e;
        }
        if (!bit0_special && n_groups >= 2) return run_dense_reg<R, K, PAIR>(L, sv, n_groups / 2, G, O, M);
        if (tpos[0] == 0) return run_dense_reg<R, K, T0>(L, sv, n_groups, G, O, M);
    }
    return run_dense_reg<R, K, SCALAR>(L, sv, n_groups, G, O, M);
}

template <typename R, int K>
cudaError_t dense_smem(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, const double *mat,
                       void *d_mat) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    Offs<K> O;
    for (int j = 0; j < D; ++j) {
        uint64_t o = 0;
        for (int t = 0; t < K; ++t)
            if ((j >> t) & 1) o |= 1ull << tpos[t];
        O.o[j] = o;
    }
    std::vector<C> hm(D * D);
    for (int i = 0; i < D * D; ++i) hm[i] = to_c<C>(mat + 2 * i);
    cudaError_t e = cudaMemcpyAsync(d_mat, hm.data(), sizeof(C) * D * D, cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(C) * (D * D + kTile);
    auto kern = k_dense_smem<R, K>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    const uint64_t n_groups = 1ull << (n - G.ns);
    const uint64_t n_tiles = (n_groups + kTile / D - 1) / (kTile / D);
    uint64_t grid = (uint64_t)L.num_sms * (per_sm > 0 ? per_sm : 1);
    if (grid > n_tiles) grid = n_tiles;
    kern<<<(unsigned)grid, kThreads, smem, L.stream>>>(reinterpret_cast<C *>(sv), n_groups, G, O,
                                                       reinterpret_cast<const C *>(d_mat));
    ++*L.launches;
    return cudaGetLastError();
}

cudaError_t dense5_c64(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, const double *mat,
                       void *d_mat) {
    Offs<5> O;
    for (int j = 0; j < 32; ++j) {
        uint64_t o = 0;
        for (int t = 0; t < 5; ++t)
            if ((j >> t) & 1) o |= 1ull << tpos[t];
        O.o[j] = o;
    }
    std::vector<float2> hm(32 * 32);
    for (int i = 0; i < 32 * 32; ++i) hm[i] = to_c<float2>(mat + 2 * i);
    cudaError_t e = cudaMemcpyAsync(d_mat, hm.data(), sizeof(float2) * 32 * 32, cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) return e;
    // qubit 0 a target: tpos[0] == 0 (targets ascending), and the base of every
    // group is even, so member pairs are 16-byte aligned
    const bool pair0 = tpos[0] == 0;
    auto kern = pair0 ? k_dense5<true> : k_dense5<false>;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    const uint64_t n_groups = 1ull << (n - G.ns);
    uint64_t grid = (uint64_t)L.num_sms * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (n_groups + kThreads - 1) / kThreads;
    if (grid > need) grid = need;
    kern<<<(unsigned)grid, kThreads, 0, L.stream>>>(reinterpret_cast<float2 *>(sv), n_groups, G, O,
                                                    reinterpret_cast<const float2 *>(d_mat));
    ++*L.launches;
    return cudaGetLastError();
}

cudaError_t dense6_c64(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, const double *mat,
                       void *d_mat) {
    Offs<6> O;
    for (int j = 0; j < 64; ++j) {
        uint64_t o = 0;
        for (int t = 0; t < 6; ++t)
            if ((j >> t) & 1) o |= 1ull << tpos[t];
        O.o[j] = o;
    }
    std::vector<float2> hm(64 * 64);
    for (int i = 0; i < 64 * 64; ++i) hm[i] = to_c<float2>(mat + 2 * i);
    cudaError_t e = cudaMemcpyAsync(d_mat, hm.data(), sizeof(float2) * 64 * 64, cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) return e;
    const bool pair0 = tpos[0] == 0;
    auto kern = pair0 ? k_dense6<true> : k_dense6<false>;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    const uint64_t n_groups = 1ull << (n - G.ns);
    uint64_t grid = (uint64_t)L.num_sms * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (2 * n_groups + kThreads - 1) / kThreads;
    if (grid > need) grid = need;
    kern<<<(unsigned)grid, kThreads, 0, L.stream>>>(reinterpret_cast<float2 *>(sv), n_groups, G, O,
                                                    reinterpret_cast<const float2 *>(d_mat));
    ++*L.launches;
    return cudaGetLastError();
}

template <typename R>
cudaError_t dense_any(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, int k,
                      const double *mat, void *d_mat) {
    switch (k) {
    case 1: return dense_reg<R, 1>(L, sv, n, G, tpos, mat);
    case 2: return dense_reg<R, 2>(L, sv, n, G, tpos, mat);
    case 3: return dense_reg<R, 3>(L, sv, n, G, tpos, mat);
    case 4: return dense_reg<R, 4>(L, sv, n, G, tpos, mat);
    case 5:
        if constexpr (std::is_same<R, float>::value) return dense5_c64(L, sv, n, G, tpos, mat, d_mat);
        else return dense_smem<R, 5>(L, sv, n, G, tpos, mat, d_mat);
    case 6:
        // pairs of lanes per group: whole warps need a group count divisible by 16
        if constexpr (std::is_same<R, float>::value)
            if (n - G.ns >= 4) return dense6_c64(L, sv, n, G, tpos, mat, d_mat);
        return dense_smem<R, 6>(L, sv, n, G, tpos, mat, d_mat);
    default: return cudaErrorInvalidValue;
    }
}

template <typename R>
cudaError_t diag_any(const LaunchCtx &L, void *sv, int n, const GroupGeom &Gc, const int *tpos, int k,
                     const double *diag) {
    using C = typename CT<R>::T;
    DiagP<R> P;
    P.k = k;
    for (int t = 0; t < SV_MAX_TARGETS; ++t) P.tpos[t] = t < k ? tpos[t] : 0;
    for (int j = 0; j < (1 << SV_MAX_TARGETS); ++j) P.d[j] = j < (1 << k) ? to_c<C>(diag + 2 * j) : C{1, 0};
    const uint64_t n_amps = 1ull << (n - Gc.ns);
    const bool bit0_ctl = Gc.ns > 0 && Gc.pos[0] == 0;
    constexpr int U = 4;
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        if (!bit0_ctl && n_amps >= 2) {
            k_diag<R, PAIR, U><<<grid_for(n_amps / 2, kThreads * U), kThreads, 0, L.stream>>>(
                reinterpret_cast<C *>(sv), n_amps / 2, Gc, P);
            done = true;
        }
    }
    if (!done)
        k_diag<R, SCALAR, U><<<grid_for(n_amps, kThreads * U), kThreads, 0, L.stream>>>(
            reinterpret_cast<C *>(sv), n_amps, Gc, P);
    ++*L.launches;
    return cudaGetLastError();
}

template <typename R, int K>
cudaError_t perm_k(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, const int *perm,
                   const double *d) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    auto off = [&](int j) {
        uint64_t o = 0;
        for (int t = 0; t < K; ++t)
            if ((j >> t) & 1) o |= 1ull << tpos[t];
        return o;
    };
    PermP<R, K> P;
    for (int j = 0; j < D; ++j) {
        const int l = perm[j];           // out[j] = d[j] * in[l]
        P.src[l] = off(l);
        P.dst[l] = off(j);
        P.f[l] = to_c<C>(d + 2 * j);
    }
    const uint64_t n_groups = 1ull << (n - G.ns);
    const bool bit0_special = G.ns > 0 && G.pos[0] == 0;
    constexpr int U = (K <= 2) ? 2 : 1;
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        if (!bit0_special && n_groups >= 2) {
            k_perm<R, K, PAIR, U><<<grid_for(n_groups / 2, kThreads * U), kThreads, 0, L.stream>>>(
                reinterpret_cast<C *>(sv), n_groups / 2, G, P);
            done = true;
        }
    }
    if (!done)
        k_perm<R, K, SCALAR, U><<<grid_for(n_groups, kThreads * U), kThreads, 0, L.stream>>>(
            reinterpret_cast<C *>(sv), n_groups, G, P);
    ++*L.launches;
    return cudaGetLastError();
}

template <typename R>
cudaError_t perm_any(const LaunchCtx &L, void *sv, int n, const GroupGeom &G, const int *tpos, int k, const int *perm,
                     const double *d) {
    switch (k) {
    case 1: return perm_k<R, 1>(L, sv, n, G, tpos, perm, d);
    case 2: return perm_k<R, 2>(L, sv, n, G, tpos, perm, d);
    case 3: return perm_k<R, 3>(L, sv, n, G, tpos, perm, d);
    case 4: return perm_k<R, 4>(L, sv, n, G, tpos, perm, d);
    default: return cudaErrorInvalidValue;
    }
}


// ---------------------------------------------------------------------------
// index-bit swap (Table I, "Index bit swap"): exchange bits a_k <-> b_k of
// every index for disjoint pairs, i.e. relabel qubits. The map is an
// involution, so each pair of amplitudes is swapped once, by the thread of the
// smaller index; amplitudes whose swapped bits agree stay.
// ---------------------------------------------------------------------------
struct SwapP {
    int np;
    int a[18], b[18];
};

__device__ __forceinline__ uint64_t swap_bits(uint64_t i, const SwapP &P) {
#pragma unroll 1
    for (int k = 0; k < P.np; ++k) {
        const uint64_t d = ((i >> P.a[k]) ^ (i >> P.b[k])) & 1u;
        i ^= (d << P.a[k]) | (d << P.b[k]);
    }
    return i;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads) k_swap(typename CT<R>::T *__restrict__ sv, uint64_t n_units, SwapP P) {
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t u = (uint64_t)blockIdx.x * kThreads + threadIdx.x; u < n_units; u += stride) {
        if constexpr (MODE == PAIR) {
            const uint64_t i = u << 1, j = swap_bits(i, P);     // bit 0 is not swapped: i+1 -> j+1
            if (j <= i) continue;
            float2 *p = reinterpret_cast<float2 *>(sv);
            const float4 x = ld16(p + i), y = ld16(p + j);
            st16(p + i, y);
            st16(p + j, x);
        } else {
            const uint64_t i = u, j = swap_bits(i, P);
            if (j <= i) continue;
            const typename CT<R>::T x = sv[i], y = sv[j];
            sv[i] = y;
            sv[j] = x;
        }
    }
}

template <typename R>
cudaError_t swap_t(const LaunchCtx &L, void *sv, int n, const int *a, const int *b, int np) {
    using C = typename CT<R>::T;
    SwapP P{};
    P.np = np;
    bool bit0 = false;
    for (int k = 0; k < np; ++k) {
        P.a[k] = a[k];
        P.b[k] = b[k];
        bit0 |= a[k] == 0 || b[k] == 0;
    }
    uint64_t units = 1ull << n;
    const bool pair = sizeof(R) == 4 && !bit0 && n >= 1;
    if (pair) units >>= 1;
    uint64_t grid = (units + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)L.num_sms * 16;
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    if constexpr (sizeof(R) == 4) {
        if (pair) {
            k_swap<R, PAIR><<<(unsigned)grid, kThreads, 0, L.stream>>>(reinterpret_cast<C *>(sv), units, P);
            ++*L.launches;
            return cudaGetLastError();
        }
    }
    k_swap<R, SCALAR><<<(unsigned)grid, kThreads, 0, L.stream>>>(reinterpret_cast<C *>(sv), units, P);
    ++*L.launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pauli rotation (Table I, "Pauli rotation"): psi <- exp(i theta P) psi
// = cos(theta) psi + i sin(theta) P psi, with P|k> = i^{nY} (-1)^{popcount(k & z)} |k ^ x>.
// Output amplitude j takes its P-term from source k = j ^ x; unit pairs
// (u, u ^ x) are read once and written once, as in the expectation kernel.
// ---------------------------------------------------------------------------
template <typename R> struct RotP {
    uint64_t x, z;
    int ny;
    R c, s;
};

template <typename C>
__device__ __forceinline__ C rot90(const C &a, int m) {   // a * i^m
    C r;
    r.x = (m == 0) ? a.x : (m == 1) ? -a.y : (m == 2) ? -a.x : a.y;
    r.y = (m == 0) ? a.y : (m == 1) ? a.x : (m == 2) ? -a.y : -a.x;
    return r;
}

template <typename R, typename C>
__device__ __forceinline__ C rot_out(const C &self, const C &src, uint64_t k, const RotP<R> &P) {
    const int m = (P.ny + 1 + 2 * (int)(__popcll(k & P.z) & 1)) & 3;
    const C t = rot90(src, m);
    C o;
    o.x = fmac(P.c, self.x, P.s * t.x);
    o.y = fmac(P.c, self.y, P.s * t.y);
    return o;
}

template <typename R, int V>
__global__ void __launch_bounds__(kThreads)
k_pauli_rot(typename CT<R>::T *__restrict__ sv, uint64_t n_work, int pair_bit, uint64_t xu, unsigned xl, RotP<R> P) {
    using C = typename CT<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t w = (uint64_t)blockIdx.x * kThreads + threadIdx.x; w < n_work; w += stride) {
        uint64_t ua = w;
        if (pair_bit >= 0) {
            const uint64_t lo = w & ((1ull << pair_bit) - 1ull);
            ua = ((w ^ lo) << 1) | lo;
        }
        const uint64_t ub = ua ^ xu;
        C A[V], B[V], NA[V], NB[V];
        if constexpr (V == 2) {
            const float4 f = ld16(reinterpret_cast<const float2 *>(sv) + 2 * ua);
            A[0] = C{f.x, f.y};
            A[V - 1] = C{f.z, f.w};
            if (pair_bit >= 0) {
                const float4 g = ld16(reinterpret_cast<const float2 *>(sv) + 2 * ub);
                B[0] = C{g.x, g.y};
                B[V - 1] = C{g.z, g.w};
            }
        } else {
            A[0] = sv[ua];
            if (pair_bit >= 0) B[0] = sv[ub];
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const uint64_t ja = ua * V + e;
            if (pair_bit < 0) {
                NA[e] = rot_out(A[e], xl ? A[V - 1 - e] : A[e], ja ^ P.x, P);
            } else {
                NA[e] = rot_out(A[e], xl ? B[V - 1 - e] : B[e], ja ^ P.x, P);
                NB[e] = rot_out(B[e], xl ? A[V - 1 - e] : A[e], (ub * V + e) ^ P.x, P);
            }
        }
        if constexpr (V == 2) {
            st16(reinterpret_cast<float2 *>(sv) + 2 * ua, make_float4(NA[0].x, NA[0].y, NA[V - 1].x, NA[V - 1].y));
            if (pair_bit >= 0)
                st16(reinterpret_cast<float2 *>(sv) + 2 * ub, make_float4(NB[0].x, NB[0].y, NB[V - 1].x, NB[V - 1].y));
        } else {
            sv[ua] = NA[0];
            if (pair_bit >= 0) sv[ub] = NB[0];
        }
    }
}

template <typename R>
cudaError_t pauli_rot_t(const LaunchCtx &L, void *sv, int n, uint64_t x, uint64_t z, int ny, double theta) {
    using C = typename CT<R>::T;
    constexpr int V = sizeof(R) == 4 ? 2 : 1;
    const int vb = V == 2 ? 1 : 0;
    if (n < 1) return cudaErrorInvalidValue;
    RotP<R> P{x, z, ny, (R)cos(theta), (R)sin(theta)};
    const uint64_t n_units = (1ull << n) >> vb;
    const unsigned xl = (unsigned)(x & (uint64_t)(V - 1));
    const uint64_t xu = x >> vb;
    int pair_bit = -1;
    uint64_t n_work = n_units;
    if (xu != 0) {
        // pairs {u, u ^ xu}: a zero inserted at xu's highest set bit (any set bit
        // enumerates each pair once; the highest keeps warp accesses contiguous)
        pair_bit = 63 - __builtin_clzll(xu);
        n_work = n_units / 2;
    }
    uint64_t grid = (n_work + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)L.num_sms * 16;
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    k_pauli_rot<R, V><<<(unsigned)grid, kThreads, 0, L.stream>>>(reinterpret_cast<C *>(sv), n_work, pair_bit, xu, xl, P);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dense(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const GroupGeom &G, const int *tpos,
                         int k, const double *mat, void *d_mat) {
    return dt == SV_C64 ? dense_any<float>(L, sv, n, G, tpos, k, mat, d_mat)
                        : dense_any<double>(L, sv, n, G, tpos, k, mat, d_mat);
}

cudaError_t launch_diag(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const GroupGeom &Gctl, const int *tpos,
                        int k, const double *diag) {
    return dt == SV_C64 ? diag_any<float>(L, sv, n, Gctl, tpos, k, diag)
                        : diag_any<double>(L, sv, n, Gctl, tpos, k, diag);
}

cudaError_t launch_perm(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const GroupGeom &G, const int *tpos,
                        int k, const int *perm, const double *d) {
    return dt == SV_C64 ? perm_any<float>(L, sv, n, G, tpos, k, perm, d)
                        : perm_any<double>(L, sv, n, G, tpos, k, perm, d);
}

cudaError_t launch_swap(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, const int *a, const int *b, int np) {
    if (np < 1 || np > 18) return cudaErrorInvalidValue;
    return dt == SV_C64 ? swap_t<float>(L, sv, n, a, b, np) : swap_t<double>(L, sv, n, a, b, np);
}

cudaError_t launch_pauli_rotation(const LaunchCtx &L, sv_dtype_t dt, void *sv, int n, uint64_t x, uint64_t z, int ny,
                                  double theta) {
    return dt == SV_C64 ? pauli_rot_t<float>(L, sv, n, x, z, ny, theta) : pauli_rot_t<double>(L, sv, n, x, z, ny, theta);
}

}  // namespace svk
