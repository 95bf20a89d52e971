// k_batch.cu -- many small state vectors advanced in one persistent launch.
//
// Gate application (Table I) and gate fusion (Sec. II-B) on a batch of
// independent states of up to 20 qubits. A CTA takes the next state from a
// work counter (states are ordered largest first) and runs its whole program:
//   * a state of T <= 14 qubits lives in shared memory (128 KiB at 14 qubits)
//     for its entire circuit, starts as |0...0> there, and never touches HBM
//     unless the caller asks for the final amplitudes;
//   * a larger state is processed stage by stage: each stage names 14 local
//     qubits that hold all of its ops; the state's 2^(n-14) tiles (the
//     amplitudes that share the non-local bits) are gathered into shared
//     memory one at a time, every op of the stage is applied there, and the
//     tile is written back. The first stage generates |0...0> instead of
//     loading. Tile gathers use two 128-entry deposit tables (local bit
//     pattern -> amplitude offset).
// Ops (compiled on the host, exact structure analysis as in sv_apply_matrix):
// dense k <= 4 (matrix staged in shared memory per op, one thread per group),
// diagonal (phases on the subspace where the controls hold) and generalized
// permutation; runs of such ops with at most 2 targets on at most 4 local
// qubits form register windows (op_window): each thread holds the 2^w
// amplitudes of one group in registers, applies the whole run there through
// one jump per sub-op into code with constant register indices, and writes
// them back once. Pauli expectations are then reduced from shared memory (or
// from the state in L2 / HBM) with FP32 runs of at most 8 terms per thread
// and FP64 beyond, block partials summed in a fixed order.
#include "sv_internal.h"

namespace svk {
namespace {

constexpr int kT = kBatchThreads;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}

// Shared-memory layout of the tile: amplitude a sits at a ^ ((a >> 4) & 15). A
// group's members differ in the op's target bits only, so without the swizzle
// the 32 lanes of a warp (consecutive groups) read member j of groups whose
// low four bits agree whenever the targets cover bits 0..3 -- all in one bank
// pair. Mixing bits 4..7 into the bank index spreads them; runs of consecutive
// amplitudes stay conflict free (each half-warp XORs one constant).
// The map is linear over XOR, and a group's base and its member offsets have
// disjoint bits, so sw(base | off) = sw(base) ^ sw(off): the offsets are
// swizzled once per op and every access costs one XOR.
__device__ __forceinline__ uint32_t sw(uint32_t a) { return a ^ ((a >> 4) & 15u); }
// the amplitude at a swizzled byte offset of the tile (one XOR per access)
__device__ __forceinline__ float2 &at8(float2 *tile, uint32_t byte_off) {
    return *reinterpret_cast<float2 *>(reinterpret_cast<char *>(tile) + byte_off);
}

// (unrolled over the twelve slots with constant indices, so that op.p stays in
// registers; the exit is uniform)
__device__ __forceinline__ uint32_t insert_zeros_local(uint32_t g, const BOp &op) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        if (i >= op.np) break;
        const uint32_t lo = g & ((1u << op.p[i]) - 1u);
        g = ((g ^ lo) << 1) | lo;
    }
    return g | op.cval;
}

template <int K>
__device__ __forceinline__ uint32_t member_off(int j, const BOp &op) {
    uint32_t o = 0;
#pragma unroll
    for (int t = 0; t < K; ++t)
        if ((j >> t) & 1) o |= 1u << op.t[t];
    return o;
}

// dense 2^K x 2^K product on every group of the tile (matrix in shared memory)
template <int K>
__device__ void op_dense(float2 *tile, const BOp &op, const float2 *msh, int T) {
    constexpr int D = 1 << K;
    constexpr bool kRegMat = K <= 2;      // small matrices live in registers
    const int ngroups = 1 << (T - op.np);
    uint32_t off[D];
#pragma unroll
    for (int j = 0; j < D; ++j) off[j] = sw(member_off<K>(j, op)) << 3;
    float2 mreg[kRegMat ? D * D : 1];
    if constexpr (kRegMat) {
#pragma unroll
        for (int i = 0; i < D * D; ++i) mreg[i] = msh[i];
    }
    for (int g = threadIdx.x; g < ngroups; g += kT) {
        const uint32_t base = sw(insert_zeros_local((uint32_t)g, op)) << 3;
        float2 v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = at8(tile, base ^ off[j]);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < D; ++l) {
                const float2 m = kRegMat ? mreg[j * D + l] : msh[j * D + l];
                acc.x = __fmaf_rn(m.x, v[l].x, acc.x);
                acc.x = __fmaf_rn(-m.y, v[l].y, acc.x);
                acc.y = __fmaf_rn(m.x, v[l].y, acc.y);
                acc.y = __fmaf_rn(m.y, v[l].x, acc.y);
            }
            at8(tile, base ^ off[j]) = acc;
        }
    }
}

// generalized permutation: source member l moves to destination dst[l] times f[l]
template <int K>
__device__ void op_perm(float2 *tile, const BOp &op, const float2 *msh, int T) {
    constexpr int D = 1 << K;
    const int ngroups = 1 << (T - op.np);
    uint32_t src[D], dst[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
        src[l] = sw(member_off<K>(l, op));
        dst[l] = sw(member_off<K>(__float_as_int(msh[D + l].x), op));
    }
    for (int g = threadIdx.x; g < ngroups; g += kT) {
        const uint32_t base = sw(insert_zeros_local((uint32_t)g, op));
        float2 v[D];
#pragma unroll
        for (int l = 0; l < D; ++l) v[l] = tile[base ^ src[l]];
#pragma unroll
        for (int l = 0; l < D; ++l) tile[base ^ dst[l]] = cmulf(msh[l], v[l]);
    }
}

// diagonal on the targets, on the amplitudes where the controls hold
__device__ void op_diag(float2 *tile, const BOp &op, const float2 *msh, int T) {
    const int namps = 1 << (T - op.np);
    for (int g = threadIdx.x; g < namps; g += kT) {
        const uint32_t a = insert_zeros_local((uint32_t)g, op);
        int j = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (t < op.k) j |= (int)((a >> op.t[t]) & 1u) << t;
        const uint32_t sa = sw(a);
        tile[sa] = cmulf(msh[j], tile[sa]);
    }
}

// ---- windows: a run of small ops on 2^W amplitudes held in registers ----
// Template arguments fix every register index; the host-computed case selects
// the instantiation. Run-time control conditions ((r & cm) == cv) are uniform
// across the CTA, so they only predicate; uncontrolled ops (CTRL false) and
// plain exchanges carry none.
// One 2x2 product on the pair (a, c) -> (o0, o1) = (m00 a + m01 c, m10 a + m11 c).
// Each output component is finished last with the input component whose
// register it takes over (x0 <- a.x, y0 <- a.y, x1 <- c.x, y1 <- c.y, or the
// exchanged assignment when SWAPPED), after every partial sum has been formed:
// each register dies exactly where its result is written, so the results
// need no copies back into the fixed registers of v[].
template <bool SWAPPED>
__device__ __forceinline__ void pair2x2(float2 &a, float2 &c, float2 m00, float2 m01, float2 m10, float2 m11) {
    if constexpr (!SWAPPED) {
        const float p0 = __fmaf_rn(m01.x, c.x, __fmaf_rn(-m00.y, a.y, -m01.y * c.y));   // o0.x without a.x
        const float p1 = __fmaf_rn(m01.x, c.y, __fmaf_rn(m00.y, a.x, m01.y * c.x));     // o0.y without a.y
        const float p2 = __fmaf_rn(m10.x, a.x, __fmaf_rn(-m10.y, a.y, -m11.y * c.y));   // o1.x without c.x
        const float p3 = __fmaf_rn(m10.x, a.y, __fmaf_rn(m10.y, a.x, m11.y * c.x));     // o1.y without c.y
        a.y = __fmaf_rn(m00.x, a.y, p1);
        c.x = __fmaf_rn(m11.x, c.x, p2);
        c.y = __fmaf_rn(m11.x, c.y, p3);
        a.x = __fmaf_rn(m00.x, a.x, p0);
    } else {   // o1 into a's registers, o0 into c's
        const float p0 = __fmaf_rn(m00.x, a.x, __fmaf_rn(-m00.y, a.y, -m01.y * c.y));   // o0.x without c.x
        const float p1 = __fmaf_rn(m00.x, a.y, __fmaf_rn(m00.y, a.x, m01.y * c.x));     // o0.y without c.y
        const float p2 = __fmaf_rn(m11.x, c.x, __fmaf_rn(-m10.y, a.y, -m11.y * c.y));   // o1.x without a.x
        const float p3 = __fmaf_rn(m11.x, c.y, __fmaf_rn(m10.y, a.x, m11.y * c.x));     // o1.y without a.y
        c.y = __fmaf_rn(m01.x, c.y, p1);
        a.x = __fmaf_rn(m10.x, a.x, p2);
        a.y = __fmaf_rn(m10.x, a.y, p3);
        c.x = __fmaf_rn(m01.x, c.x, p0);
    }
}

template <int W, int B, bool CTRL>
__device__ __forceinline__ void win_dense1(float2 (&v)[1 << W], const float2 *m, uint32_t cm, uint32_t cv) {
    if constexpr (B < W) {
        const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            if (CTRL && ((uint32_t)r & cm) != cv) continue;
            pair2x2<false>(v[r], v[r | (1 << B)], m00, m01, m10, m11);
        }
    }
}

template <int W, int B>
__device__ __forceinline__ void win_swap1(float2 (&v)[1 << W], const float2 *m, uint32_t cm, uint32_t cv) {
    if constexpr (B < W) {
        const float2 f0 = m[0], f1 = m[1];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            if (((uint32_t)r & cm) != cv) continue;
            const float2 a = v[r], c = v[r | (1 << B)];
            v[r] = cmulf(f1, c);
            v[r | (1 << B)] = cmulf(f0, a);
        }
    }
}

// a 2x2 on bit B followed by the exchange across bit T where bit C == CV
// (B is C or T): the products are written straight into the exchanged registers
template <int W, int B, int C, int T, int CV>
__device__ __forceinline__ void win_dense1_cx(float2 (&v)[1 << W], const float2 *m) {
    if constexpr (B < W && C < W && T < W && B == T) {
        // the exchange stays within each pair: its outputs trade registers
        const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            if (((r >> C) & 1) == CV)
                pair2x2<true>(v[r], v[r | (1 << B)], m00, m01, m10, m11);
            else
                pair2x2<false>(v[r], v[r | (1 << B)], m00, m01, m10, m11);
        }
    } else if constexpr (B < W && C < W && T < W) {
        const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
        float2 o[1 << W];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            const float2 a = v[r], c = v[r | (1 << B)];
            o[r] = make_float2(__fmaf_rn(m00.x, a.x, __fmaf_rn(-m00.y, a.y, __fmaf_rn(m01.x, c.x, -m01.y * c.y))),
                               __fmaf_rn(m00.x, a.y, __fmaf_rn(m00.y, a.x, __fmaf_rn(m01.x, c.y, m01.y * c.x))));
            o[r | (1 << B)] =
                make_float2(__fmaf_rn(m10.x, a.x, __fmaf_rn(-m10.y, a.y, __fmaf_rn(m11.x, c.x, -m11.y * c.y))),
                            __fmaf_rn(m10.x, a.y, __fmaf_rn(m10.y, a.x, __fmaf_rn(m11.x, c.y, m11.y * c.x))));
        }
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) v[((r >> C) & 1) == CV ? (r ^ (1 << T)) : r] = o[r];
    }
}

// the exchange across bit T where bit C == CV, then a 2x2 on bit B (B is C or
// T): the 2x2 reads the exchanged registers
template <int W, int B, int C, int T, int CV>
__device__ __forceinline__ void win_cx_dense1(float2 (&v)[1 << W], const float2 *m) {
    if constexpr (B < W && C < W && T < W && B == T) {
        // the exchange stays within each pair: where it applies, the pair's two
        // inputs trade places, which is the matrix with its columns exchanged
        const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            if (((r >> C) & 1) == CV)
                pair2x2<false>(v[r], v[r | (1 << B)], m01, m00, m11, m10);
            else
                pair2x2<false>(v[r], v[r | (1 << B)], m00, m01, m10, m11);
        }
    } else if constexpr (B < W && C < W && T < W) {
        const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
        float2 x[1 << W];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) x[r] = v[((r >> C) & 1) == CV ? (r ^ (1 << T)) : r];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            pair2x2<false>(x[r], x[r | (1 << B)], m00, m01, m10, m11);
        }
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) v[r] = x[r];
    }
}

// members exchanged across bit B (C < 0) or where window bit C equals CV: a
// renaming of registers, no arithmetic, but moves where the cases rejoin
template <int W, int B, int C, int CV>
__device__ __forceinline__ void win_xswap(float2 (&v)[1 << W]) {
    if constexpr (B < W && C < W) {
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            if constexpr (C >= 0) {
                if (((r >> C) & 1) != CV) continue;
            }
            const float2 a = v[r];
            v[r] = v[r | (1 << B)];
            v[r | (1 << B)] = a;
        }
    }
}

template <int W, int B0, int B1, bool CTRL>
__device__ __forceinline__ void win_dense2(float2 (&v)[1 << W], const float2 *m, uint32_t cm, uint32_t cv) {
    if constexpr (B0 < B1 && B1 < W) {
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & ((1 << B0) | (1 << B1))) continue;
            if (CTRL && ((uint32_t)r & cm) != cv) continue;
            const int o[4] = {r, r | (1 << B0), r | (1 << B1), r | (1 << B0) | (1 << B1)};
            float2 a[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) a[l] = v[o[l]];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const float2 x = m[4 * j + l];
                    acc.x = __fmaf_rn(x.x, a[l].x, acc.x);
                    acc.x = __fmaf_rn(-x.y, a[l].y, acc.x);
                    acc.y = __fmaf_rn(x.x, a[l].y, acc.y);
                    acc.y = __fmaf_rn(x.y, a[l].x, acc.y);
                }
                v[o[j]] = acc;
            }
        }
    }
}

template <int W>
__device__ __forceinline__ void win_diag(float2 (&v)[1 << W], const float2 *m, int nd, int b0, int b1, uint32_t cm,
                                         uint32_t cv) {
#pragma unroll
    for (int r = 0; r < (1 << W); ++r) {
        if (((uint32_t)r & cm) != cv) continue;
        const int j = nd == 0 ? 0 : nd == 1 ? ((r >> b0) & 1) : (((r >> b0) & 1) | (((r >> b1) & 1) << 1));
        v[r] = cmulf(m[j], v[r]);
    }
}

// the window's groups: zero bits inserted at its W positions
template <int W>
__device__ __forceinline__ uint32_t insert_zeros_win(uint32_t g, const BOp &op) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint32_t lo = g & ((1u << op.p[i]) - 1u);
        g = ((g ^ lo) << 1) | lo;
    }
    return g;
}

#define SV_WC_BIT(B)                                                              \
    case WC_DENSE1 + B: win_dense1<W, B, false>(v, m, cm, cv); break;            \
    case WC_DENSE1C + B: win_dense1<W, B, true>(v, m, cm, cv); break;            \
    case WC_SWAP1 + B: win_swap1<W, B>(v, m, cm, cv); break;                     \
    case WC_XSWAP + B: win_xswap<W, B, -1, 0>(v); break;
#define SV_WC_PAIR(B0, B1)                                                        \
    case WC_DENSE2 + wc_pair(B0, B1): win_dense2<W, B0, B1, false>(v, m, cm, cv); break; \
    case WC_DENSE2C + wc_pair(B0, B1): win_dense2<W, B0, B1, true>(v, m, cm, cv); break;
#define SV_WC_D1CX(C, T)                                                                             \
    case WC_D1CX + wc_opair(C, T) * 2: win_dense1_cx<W, T, C, T, 0>(v, m); break;                   \
    case WC_D1CX + wc_opair(C, T) * 2 + 1: win_dense1_cx<W, T, C, T, 1>(v, m); break;               \
    case WC_D1CX + (12 + wc_opair(C, T)) * 2: win_dense1_cx<W, C, C, T, 0>(v, m); break;            \
    case WC_D1CX + (12 + wc_opair(C, T)) * 2 + 1: win_dense1_cx<W, C, C, T, 1>(v, m); break;
#define SV_WC_CXD1(C, T)                                                                             \
    case WC_CXD1 + wc_opair(C, T) * 2: win_cx_dense1<W, T, C, T, 0>(v, m); break;                   \
    case WC_CXD1 + wc_opair(C, T) * 2 + 1: win_cx_dense1<W, T, C, T, 1>(v, m); break;               \
    case WC_CXD1 + (12 + wc_opair(C, T)) * 2: win_cx_dense1<W, C, C, T, 0>(v, m); break;            \
    case WC_CXD1 + (12 + wc_opair(C, T)) * 2 + 1: win_cx_dense1<W, C, C, T, 1>(v, m); break;
#define SV_WC_CX(B, C)                                                            \
    case WC_CXSWAP + (4 * B + C) * 2: win_xswap<W, B, C, 0>(v); break;           \
    case WC_CXSWAP + (4 * B + C) * 2 + 1: win_xswap<W, B, C, 1>(v); break;

template <int W>
__device__ void op_window(float2 *tile, const BOp &op, const float2 *blk, int T) {
    constexpr int D = 1 << W;
    const int ngroups = 1 << (T - W);
    const int nsub = op.k;
    // swizzled byte offsets of the members: XOR prefixes of the per-bit ones
    uint32_t off[D];
    off[0] = 0;
#pragma unroll
    for (int j = 1; j < D; ++j) {
        const int t = 31 - __clz(j);
        off[j] = off[j ^ (1 << t)] ^ (sw(1u << op.p[t]) << 3);
    }
    for (int g = threadIdx.x; g < ngroups; g += kT) {
        const uint32_t base = sw(insert_zeros_win<W>((uint32_t)g, op)) << 3;
        float2 v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = at8(tile, base ^ off[j]);
        for (int s = 0; s < nsub; ++s) {
            const float2 h0 = blk[2 * s], h1 = blk[2 * s + 1];
            const uint32_t hy = __float_as_uint(h0.y);
            const uint32_t cm = hy & 0xff, cv = (hy >> 8) & 0xff;
            const float2 *m = blk + __float_as_uint(h1.x);
            switch (hy >> 16) {
                SV_WC_BIT(0) SV_WC_BIT(1) SV_WC_BIT(2) SV_WC_BIT(3)
                SV_WC_PAIR(0, 1) SV_WC_PAIR(0, 2) SV_WC_PAIR(0, 3) SV_WC_PAIR(1, 2) SV_WC_PAIR(1, 3) SV_WC_PAIR(2, 3)
                SV_WC_CX(0, 1) SV_WC_CX(0, 2) SV_WC_CX(0, 3) SV_WC_CX(1, 0) SV_WC_CX(1, 2) SV_WC_CX(1, 3)
                SV_WC_CX(2, 0) SV_WC_CX(2, 1) SV_WC_CX(2, 3) SV_WC_CX(3, 0) SV_WC_CX(3, 1) SV_WC_CX(3, 2)
                SV_WC_D1CX(0, 1) SV_WC_D1CX(0, 2) SV_WC_D1CX(0, 3) SV_WC_D1CX(1, 0) SV_WC_D1CX(1, 2) SV_WC_D1CX(1, 3)
                SV_WC_D1CX(2, 0) SV_WC_D1CX(2, 1) SV_WC_D1CX(2, 3) SV_WC_D1CX(3, 0) SV_WC_D1CX(3, 1) SV_WC_D1CX(3, 2)
                SV_WC_CXD1(0, 1) SV_WC_CXD1(0, 2) SV_WC_CXD1(0, 3) SV_WC_CXD1(1, 0) SV_WC_CXD1(1, 2) SV_WC_CXD1(1, 3)
                SV_WC_CXD1(2, 0) SV_WC_CXD1(2, 1) SV_WC_CXD1(2, 3) SV_WC_CXD1(3, 0) SV_WC_CXD1(3, 1) SV_WC_CXD1(3, 2)
            default: {
                const uint32_t hx = __float_as_uint(h0.x);
                win_diag<W>(v, m, hx >> 24, (hx >> 8) & 0xff, (hx >> 16) & 0xff, cm, cv);
            }
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) at8(tile, base ^ off[j]) = v[j];
    }
}

#undef SV_WC_BIT
#undef SV_WC_PAIR
#undef SV_WC_CX
#undef SV_WC_D1CX
#undef SV_WC_CXD1

__device__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kT / 32; ++w) t += red[w];
    return t;
}

// Shared state of one CTA (besides the dynamic tile and stage-matrix area).
struct BSmem {
    float2 msh[2 * 256];                 // one op's matrix when the stage's do not fit
    uint32_t lo_tab[128], hi_tab[128];   // local bits 0..6 / 7..13 -> amplitude bits
    double red[kT / 32];
    int task;
    int go;
};

// Deposit tables of a stage (threads 0..255: local bits 0..6 and 7..13 of a
// tile index -> amplitude bits) and its matrices in shared memory.
__device__ bool stage_setup(const BStage &S, int T, const float2 *__restrict__ pool, float2 *smat, BSmem &sh) {
    if (threadIdx.x < 256) {
        const int hi = threadIdx.x >> 7, v = threadIdx.x & 127;
        uint32_t a = 0;
#pragma unroll
        for (int b = 0; b < 7; ++b)
            if (7 * hi + b < T && ((v >> b) & 1)) a |= 1u << S.lpos[7 * hi + b];
        (hi ? sh.hi_tab : sh.lo_tab)[v] = a;
    }
    const bool staged = S.pool_count <= kBatchStageMat;
    if (staged)
        for (int i = threadIdx.x; i < S.pool_count; i += kT) smat[i] = pool[S.pool_begin + i];
    __syncthreads();
    return staged;
}

// Every op of a stage on the tile in shared memory.
__device__ __forceinline__ void stage_ops(float2 *tile, const BStage &S, const BOp *__restrict__ ops, const float2 *__restrict__ pool,
                          const float2 *smat, bool staged, BSmem &sh, int T) {
    for (int o = S.op_begin; o < S.op_end; ++o) {
        const BOp op = ops[o];
        const float2 *m;
        if (staged) {
            m = smat + (op.mat - S.pool_begin);
            __syncthreads();   // the previous op is done with the tile
        } else {
            const int D = 1 << op.k;
            const int nm = op.kind == BOP_DENSE ? D * D : (op.kind == BOP_PERM ? 2 * D : D);
            __syncthreads();   // previous op done with the tile and msh
            for (int i = threadIdx.x; i < nm; i += kT) sh.msh[i] = pool[op.mat + i];
            __syncthreads();
            m = sh.msh;
        }
        if (op.kind == BOP_WIN) {
            // windows only occur in stages whose matrices are staged
            switch (op.np) {
            case 2: op_window<2>(tile, op, m, T); break;
            case 3: op_window<3>(tile, op, m, T); break;
            default: op_window<4>(tile, op, m, T); break;
            }
        } else if (op.kind == BOP_DENSE) {
            switch (op.k) {
            case 1: op_dense<1>(tile, op, m, T); break;
            case 2: op_dense<2>(tile, op, m, T); break;
            case 3: op_dense<3>(tile, op, m, T); break;
            default: op_dense<4>(tile, op, m, T); break;
            }
        } else if (op.kind == BOP_PERM) {
            switch (op.k) {
            case 1: op_perm<1>(tile, op, m, T); break;
            case 2: op_perm<2>(tile, op, m, T); break;
            case 3: op_perm<3>(tile, op, m, T); break;
            default: op_perm<4>(tile, op, m, T); break;
            }
        } else {
            op_diag(tile, op, m, T);
        }
    }
    __syncthreads();
}

// Sum over pairs g in [g_lo, g_hi) of one Pauli string's terms, from the tile
// (in_tile) or from the state in global memory (CG: read at L2, never L1, when
// other CTAs wrote it). Terms i and i ^ x come from the same pair of loads:
// w_i = psi_i conj(psi_{i^x}), w_{i^x} = conj(w_i); pairs are enumerated by
// inserting a zero at the highest bit of x (any set bit would do; the highest
// keeps a warp's loads contiguous). kU pairs per iteration, all loads issued
// before any use; the FP32 run of at most 8 terms goes into the FP64 sum after
// every fourth pair. Returns this thread's FP64 partial.
template <bool CG>
__device__ __forceinline__ double pauli_terms(const float2 *tile, const float2 *sv, bool in_tile, const BStr &P,
                                              uint32_t g_lo, uint32_t g_hi) {
    const uint32_t x = (uint32_t)P.x, z = (uint32_t)P.z;
    double acc = 0.0;
    float run = 0.f;
    const int pb = x ? 31 - __clz(x) : 0;
    constexpr int kU = 4;
    for (uint32_t g0 = g_lo + threadIdx.x; g0 < g_hi; g0 += kU * kT) {
        float2 a[kU], b[kU];
        uint32_t ii[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t g = g0 + (uint32_t)u * kT;
            ii[u] = x ? (((g >> pb) << (pb + 1)) | (g & ((1u << pb) - 1u))) : g;
            if (g < g_hi) {
                const uint32_t j = ii[u] ^ x;
                if constexpr (CG) {
                    a[u] = __ldcg(sv + ii[u]);
                    b[u] = x ? __ldcg(sv + j) : a[u];
                } else {
                    a[u] = in_tile ? tile[sw(ii[u])] : sv[ii[u]];
                    b[u] = x ? (in_tile ? tile[sw(j)] : sv[j]) : a[u];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (g0 + (uint32_t)u * kT >= g_hi) continue;
            const uint32_t i = ii[u], j = i ^ x;
            const float re = a[u].x * b[u].x + a[u].y * b[u].y, im = a[u].y * b[u].x - a[u].x * b[u].y;
            const float ti = P.use_im ? im : re;
            run += (__popc(i & z) & 1) ? -ti : ti;
            if (x) {
                const float tj = P.use_im ? -im : re;
                run += (__popc(j & z) & 1) ? -tj : tj;
            }
            if ((u & 3) == 3) {
                acc += (double)run;
                run = 0.f;
            }
        }
        acc += (double)run;
        run = 0.f;
    }
    return acc;
}

// Thread 0 waits (bounded) until `need` tile tasks of the item have finished;
// then every thread may read what they wrote. False when the wait gave up or
// another CTA had already given up.
__device__ bool wait_tiles(const BProg &P, int item, unsigned need, BSmem &sh) {
    if (threadIdx.x == 0) {
        int go = 1;
        volatile unsigned *done = P.tiles_done + item;
        volatile int *status = P.status;
        const long long t0 = clock64();
        need += P.need_extra;
        while (*done < need) {
            if (*status != 0) {
                go = 0;
                break;
            }
            if (clock64() - t0 > P.wait_cycles) {
                atomicExch(P.status, kBatchErrTimeout);
                go = 0;
                break;
            }
            __nanosleep(256);
        }
        __threadfence();
        sh.go = go;
    }
    __syncthreads();
    return sh.go != 0;
}

// The tile task is complete: publish its writes, then count it.
__device__ void finish_tiles(const BProg &P, int item) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(P.tiles_done + item, 1u);
    }
}

// Tiles [a, b) of one stage of a state above the tile size.
__device__ __noinline__ void task_tiles(float2 *tile, float2 *smat, BSmem &sh, float2 *states, const BProg &P,
                                        const BTask &tk) {
    const BItem it = P.items[tk.item];
    float2 *sv = states + it.state_off;
    const int n = it.n, T = it.T, L = 1 << T;
    const BStage S = P.stages[tk.stage];
    const bool staged = stage_setup(S, T, P.pool, smat, sh);
    const uint32_t other = (uint32_t)(~S.lmask & ((1ull << n) - 1ull));
    const bool first = tk.stage == it.stage_begin;
    for (uint32_t ti = tk.a; ti < tk.b; ++ti) {
        uint32_t tbase = 0;
        {
            uint32_t rem = other, src = ti;
            while (rem) {
                const uint32_t low = rem & (0u - rem);
                if (src & 1u) tbase |= low;
                src >>= 1;
                rem ^= low;
            }
        }
        __syncthreads();   // the previous tile has been written back
        if (first) {
            for (int l = threadIdx.x; l < L; l += kT)
                tile[sw(l)] = make_float2((tbase | sh.lo_tab[l & 127] | sh.hi_tab[l >> 7]) == 0u ? 1.f : 0.f, 0.f);
        } else {
            // eight gathers in flight per thread before the shared-memory writes
            for (int l0 = threadIdx.x; l0 < L; l0 += 8 * kT) {
                float2 t8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int l = l0 + u * kT;
                    if (l < L) t8[u] = __ldcg(sv + (tbase | sh.lo_tab[l & 127] | sh.hi_tab[l >> 7]));
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int l = l0 + u * kT;
                    if (l < L) tile[sw(l)] = t8[u];
                }
            }
        }
        stage_ops(tile, S, P.ops, P.pool, smat, staged, sh, T);
        for (int l = threadIdx.x; l < L; l += kT) sv[tbase | sh.lo_tab[l & 127] | sh.hi_tab[l >> 7]] = tile[sw(l)];
    }
}

// One chunk of the expectation sums of a state above the tile size; the CTA
// that finishes the state's last chunk adds the partials in chunk order.
__device__ __noinline__ void task_expect(BSmem &sh, float2 *states, const BProg &P, const BTask &tk) {
    const BItem it = P.items[tk.item];
    const float2 *sv = states + it.state_off;
    const int n = it.n;
    const uint32_t c = tk.a, nch = (uint32_t)it.n_chunks;
    for (int s = 0; s < it.n_str; ++s) {
        const BStr Ps = P.strs[it.str_begin + s];
        const uint32_t npairs = Ps.x ? (1u << n) / 2 : (1u << n);
        const uint32_t per = npairs / nch;
        const double tot = block_sum(pauli_terms<true>(nullptr, sv, false, Ps, c * per, (c + 1) * per), sh.red);
        if (threadIdx.x == 0) P.parts[it.part_begin + c * it.n_str + s] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(P.chunks_done + tk.item, 1u);
        if (prev + 1 == nch) {
            // every other chunk's partials were published before its count
            __threadfence();
            for (int s = 0; s < it.n_str; ++s) {
                double t = 0.0;
                for (uint32_t k = 0; k < nch; ++k) t += __ldcg(P.parts + it.part_begin + k * it.n_str + s);
                P.out[it.out_begin + s] = (double)P.strs[it.str_begin + s].sign * t;
            }
        }
    }
}

// One state run by one CTA (BT_STATE / BT_WHOLE). A state of T <= 14 qubits
// lives in the tile for its whole circuit; a larger one is processed stage by
// stage, each of its 2^(n-T) tiles gathered, updated and written back. Then
// the expectation values: from the tile (n == T) or, chunk by chunk in the
// order the split form adds its partials, from the state in global memory.
__device__ __forceinline__ void run_state(float2 *tile, float2 *smat, BSmem &sh, float2 *states, const BProg &P,
                                          const BItem &it) {
    float2 *sv = states + it.state_off;
    const int n = it.n, T = it.T, L = 1 << T;
    const uint32_t ntiles = 1u << (n - T);
    for (int st = it.stage_begin; st < it.stage_end; ++st) {
        const BStage S = P.stages[st];
        __syncthreads();
        const bool staged = stage_setup(S, T, P.pool, smat, sh);
        const uint32_t other = (uint32_t)(~S.lmask & ((1ull << n) - 1ull));
        for (uint32_t ti = 0; ti < ntiles; ++ti) {
            uint32_t tbase = 0;
            {
                uint32_t rem = other, src = ti;
                while (rem) {
                    const uint32_t low = rem & (0u - rem);
                    if (src & 1u) tbase |= low;
                    src >>= 1;
                    rem ^= low;
                }
            }
            if (st == it.stage_begin) {
                for (int l = threadIdx.x; l < L; l += kT)
                    tile[sw(l)] = make_float2((tbase | sh.lo_tab[l & 127] | sh.hi_tab[l >> 7]) == 0u ? 1.f : 0.f, 0.f);
            } else {
                // eight gathers in flight per thread before the shared-memory writes
                for (int l0 = threadIdx.x; l0 < L; l0 += 8 * kT) {
                    float2 t8[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int l = l0 + u * kT;
                        if (l < L) t8[u] = sv[tbase | sh.lo_tab[l & 127] | sh.hi_tab[l >> 7]];
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int l = l0 + u * kT;
                        if (l < L) tile[sw(l)] = t8[u];
                    }
                }
            }
            stage_ops(tile, S, P.ops, P.pool, smat, staged, sh, T);
            if (n > T || P.keep_states)
                for (int l = threadIdx.x; l < L; l += kT) sv[tbase | sh.lo_tab[l & 127] | sh.hi_tab[l >> 7]] = tile[sw(l)];
            __syncthreads();
        }
    }
    const uint32_t nch = n == T ? 1u : (uint32_t)it.n_chunks;
    for (int s = 0; s < it.n_str; ++s) {
        const BStr Ps = P.strs[it.str_begin + s];
        const uint32_t npairs = Ps.x ? (1u << n) / 2 : (1u << n);
        const uint32_t per = npairs / nch;
        double t = 0.0;
        for (uint32_t c = 0; c < nch; ++c) {
            t += block_sum(pauli_terms<false>(tile, sv, n == T, Ps, c * per, (c + 1) * per), sh.red);
        }
        if (threadIdx.x == 0) P.out[it.out_begin + s] = (double)Ps.sign * t;
    }
}

// SPLIT = false: every task is a one-CTA state (the program has no split
// states), so the work list is just the states, largest first. SPLIT = true:
// the full work list with split states' tile and expectation tasks.
template <bool SPLIT>
__global__ void __launch_bounds__(kT, 1) k_batch(float2 *__restrict__ states, const BProg P) {
    extern __shared__ float2 tile[];                 // 2^kBatchTileQubits amplitudes, then the stage's matrices
    float2 *smat = tile + (1 << kBatchTileQubits);   // kBatchStageMat entries
    __shared__ BSmem sh;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            if constexpr (SPLIT) sh.task = *(volatile int *)P.status != 0 ? P.n_tasks : atomicAdd(P.counter, 1);
            else sh.task = atomicAdd(P.counter, 1);
        }
        __syncthreads();
        const int ti_ = sh.task;
        if (ti_ >= P.n_tasks) break;
        if constexpr (!SPLIT) {
            const BItem it = P.items[P.tasks[ti_].item];
            run_state(tile, smat, sh, states, P, it);
            continue;
        }
        const BTask tk = P.tasks[ti_];
        if constexpr (SPLIT) {
            if (tk.kind == BT_TILES) {
                if (!wait_tiles(P, tk.item, tk.need, sh)) continue;
                task_tiles(tile, smat, sh, states, P, tk);
                finish_tiles(P, tk.item);
                continue;
            }
            if (tk.kind == BT_EXPECT) {
                if (!wait_tiles(P, tk.item, tk.need, sh)) continue;
                task_expect(sh, states, P, tk);
                continue;
            }
        }
        const BItem it = P.items[tk.item];
        run_state(tile, smat, sh, states, P, it);
    }
}

}  // namespace

cudaError_t launch_batch(const LaunchCtx &L, float2 *states, const BProg &P, bool split) {
    const int smem = (int)sizeof(float2) * ((1 << kBatchTileQubits) + kBatchStageMat);
    auto kern = split ? k_batch<true> : k_batch<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int grid = L.num_sms;
    if (grid > P.n_tasks) grid = P.n_tasks;
    if (grid < 1) grid = 1;
    kern<<<grid, kT, smem, L.stream>>>(states, P);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace svk
