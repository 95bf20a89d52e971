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
// permutation. Pauli expectations are then reduced from shared memory (or
// from the state in L2 / HBM) with FP32 sums of at most 16 terms per thread
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
__device__ __forceinline__ uint32_t sw(uint32_t a) { return a ^ ((a >> 4) & 15u); }

__device__ __forceinline__ uint32_t insert_zeros_local(uint32_t g, const BOp &op) {
#pragma unroll 1
    for (int i = 0; i < op.np; ++i) {
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
    for (int j = 0; j < D; ++j) off[j] = member_off<K>(j, op);
    float2 mreg[kRegMat ? D * D : 1];
    if constexpr (kRegMat) {
#pragma unroll
        for (int i = 0; i < D * D; ++i) mreg[i] = msh[i];
    }
    for (int g = threadIdx.x; g < ngroups; g += kT) {
        const uint32_t base = insert_zeros_local((uint32_t)g, op);
        float2 v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = tile[sw(base | off[j])];
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
            tile[sw(base | off[j])] = acc;
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
        src[l] = member_off<K>(l, op);
        dst[l] = member_off<K>(__float_as_int(msh[D + l].x), op);
    }
    for (int g = threadIdx.x; g < ngroups; g += kT) {
        const uint32_t base = insert_zeros_local((uint32_t)g, op);
        float2 v[D];
#pragma unroll
        for (int l = 0; l < D; ++l) v[l] = tile[sw(base | src[l])];
#pragma unroll
        for (int l = 0; l < D; ++l) tile[sw(base | dst[l])] = cmulf(msh[l], v[l]);
    }
}

// diagonal on the targets, on the amplitudes where the controls hold
__device__ void op_diag(float2 *tile, const BOp &op, const float2 *msh, int T) {
    const int namps = 1 << (T - op.np);
    for (int g = threadIdx.x; g < namps; g += kT) {
        const uint32_t a = insert_zeros_local((uint32_t)g, op);
        int j = 0;
        for (int t = 0; t < op.k; ++t) j |= (int)((a >> op.t[t]) & 1u) << t;
        tile[sw(a)] = cmulf(msh[j], tile[sw(a)]);
    }
}

// ---- windows: a run of small ops on 2^W amplitudes held in registers ----
// Template arguments fix every register index; the run-time target bits select
// the instantiation. Control conditions ((r & cm) == cv) are uniform across the
// CTA, so they only predicate.
template <int W, int B>
__device__ __forceinline__ void win_dense1(float2 (&v)[1 << W], const float2 *m, uint32_t cm, uint32_t cv) {
    if constexpr (B < W) {
        const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & (1 << B)) continue;
            if (((uint32_t)r & cm) != cv) continue;
            const float2 a = v[r], c = v[r | (1 << B)];
            v[r] = make_float2(__fmaf_rn(m00.x, a.x, __fmaf_rn(-m00.y, a.y, __fmaf_rn(m01.x, c.x, -m01.y * c.y))),
                               __fmaf_rn(m00.x, a.y, __fmaf_rn(m00.y, a.x, __fmaf_rn(m01.x, c.y, m01.y * c.x))));
            v[r | (1 << B)] =
                make_float2(__fmaf_rn(m10.x, a.x, __fmaf_rn(-m10.y, a.y, __fmaf_rn(m11.x, c.x, -m11.y * c.y))),
                            __fmaf_rn(m10.x, a.y, __fmaf_rn(m10.y, a.x, __fmaf_rn(m11.x, c.y, m11.y * c.x))));
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

template <int W, int B0, int B1>
__device__ __forceinline__ void win_dense2(float2 (&v)[1 << W], const float2 *m, uint32_t cm, uint32_t cv) {
    if constexpr (B0 < B1 && B1 < W) {
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) {
            if (r & ((1 << B0) | (1 << B1))) continue;
            if (((uint32_t)r & cm) != cv) continue;
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

template <int W>
__device__ void op_window(float2 *tile, const BOp &op, const float2 *blk, int T) {
    constexpr int D = 1 << W;
    const int ngroups = 1 << (T - W);
    const int nsub = op.k;
    uint32_t off[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        uint32_t o = 0;
#pragma unroll
        for (int t = 0; t < W; ++t)
            if ((j >> t) & 1) o |= 1u << op.p[t];
        off[j] = o;
    }
    for (int g = threadIdx.x; g < ngroups; g += kT) {
        const uint32_t base = insert_zeros_local((uint32_t)g, op);
        float2 v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = tile[sw(base | off[j])];
        for (int s = 0; s < nsub; ++s) {
            const float2 h0 = blk[2 * s], h1 = blk[2 * s + 1];
            const uint32_t hx = __float_as_uint(h0.x), hy = __float_as_uint(h0.y);
            const int kind = hx & 0xff, b0 = (hx >> 8) & 0xff, b1 = (hx >> 16) & 0xff, nd = hx >> 24;
            const uint32_t cm = hy & 0xff, cv = (hy >> 8) & 0xff;
            const float2 *m = blk + __float_as_uint(h1.x);
            if (kind == BSUB_DENSE1) {
                switch (b0) {
                case 0: win_dense1<W, 0>(v, m, cm, cv); break;
                case 1: win_dense1<W, 1>(v, m, cm, cv); break;
                case 2: win_dense1<W, 2>(v, m, cm, cv); break;
                default: win_dense1<W, 3>(v, m, cm, cv); break;
                }
            } else if (kind == BSUB_DENSE2) {
                switch (b0 * 4 + b1) {
                case 1: win_dense2<W, 0, 1>(v, m, cm, cv); break;
                case 2: win_dense2<W, 0, 2>(v, m, cm, cv); break;
                case 3: win_dense2<W, 0, 3>(v, m, cm, cv); break;
                case 6: win_dense2<W, 1, 2>(v, m, cm, cv); break;
                case 7: win_dense2<W, 1, 3>(v, m, cm, cv); break;
                default: win_dense2<W, 2, 3>(v, m, cm, cv); break;
                }
            } else if (kind == BSUB_SWAP1) {
                switch (b0) {
                case 0: win_swap1<W, 0>(v, m, cm, cv); break;
                case 1: win_swap1<W, 1>(v, m, cm, cv); break;
                case 2: win_swap1<W, 2>(v, m, cm, cv); break;
                default: win_swap1<W, 3>(v, m, cm, cv); break;
                }
            } else {
                win_diag<W>(v, m, nd, b0, b1, cm, cv);
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) tile[sw(base | off[j])] = v[j];
    }
}

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

__global__ void __launch_bounds__(kT, 1)
k_batch(float2 *__restrict__ states, const BItem *__restrict__ items, int n_items, const BStage *__restrict__ stages,
        const BOp *__restrict__ ops, const float2 *__restrict__ pool, const BStr *__restrict__ strs,
        double *__restrict__ out, int *__restrict__ counter, int keep_states) {
    extern __shared__ float2 tile[];                 // 2^kBatchTileQubits amplitudes, then the stage's matrices
    float2 *smat = tile + (1 << kBatchTileQubits);   // kBatchStageMat entries
    __shared__ float2 msh[2 * 256];                  // one op's matrix when the stage's do not fit
    __shared__ uint32_t lo_tab[128], hi_tab[128];    // local bits 0..6 / 7..13 -> amplitude bits
    __shared__ double red[kT / 32];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int ii = s_item;
        if (ii >= n_items) break;
        const BItem it = items[ii];
        float2 *sv = states + it.state_off;
        const int n = it.n, T = it.T, L = 1 << T;
        const uint32_t ntiles = 1u << (n - T);
        for (int st = it.stage_begin; st < it.stage_end; ++st) {
            const BStage S = stages[st];
            __syncthreads();
            if (threadIdx.x < 256) {
                const int hi = threadIdx.x >> 7, v = threadIdx.x & 127;
                uint32_t a = 0;
                int b = 0;
                for (int q = 0; q < n; ++q) {
                    if (!((S.lmask >> q) & 1u)) continue;
                    if (b >= 7 * hi && b < 7 * hi + 7 && ((v >> (b - 7 * hi)) & 1)) a |= 1u << q;
                    ++b;
                }
                (hi ? hi_tab : lo_tab)[v] = a;
            }
            const uint32_t other = (uint32_t)(~S.lmask & ((1ull << n) - 1ull));
            // the stage's matrices stay in shared memory for all of its tiles
            const bool staged = S.pool_count <= kBatchStageMat;
            if (staged)
                for (int i = threadIdx.x; i < S.pool_count; i += kT) smat[i] = pool[S.pool_begin + i];
            __syncthreads();
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
                        tile[sw(l)] = make_float2((tbase | lo_tab[l & 127] | hi_tab[l >> 7]) == 0u ? 1.f : 0.f, 0.f);
                } else {
                    for (int l = threadIdx.x; l < L; l += kT) tile[sw(l)] = sv[tbase | lo_tab[l & 127] | hi_tab[l >> 7]];
                }
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
                        for (int i = threadIdx.x; i < nm; i += kT) msh[i] = pool[op.mat + i];
                        __syncthreads();
                        m = msh;
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
                if (n > T || keep_states)
                    for (int l = threadIdx.x; l < L; l += kT) sv[tbase | lo_tab[l & 127] | hi_tab[l >> 7]] = tile[sw(l)];
                __syncthreads();
            }
        }
        // Pauli expectations: the tile (n == T) or the state in global memory
        const uint32_t N = 1u << n;
        for (int s = 0; s < it.n_str; ++s) {
            const BStr P = strs[it.str_begin + s];
            const uint32_t x = (uint32_t)P.x, z = (uint32_t)P.z;
            double acc = 0.0;
            float run = 0.f;
            int cnt = 0;
            // terms i and i ^ x come from the same pair of loads: w_i = psi_i conj(psi_{i^x}),
            // w_{i^x} = conj(w_i); pairs are enumerated by inserting a zero at the highest
            // bit of x (any set bit would do; the highest keeps a warp's loads contiguous)
            const int pb = x ? 31 - __clz(x) : 0;
            const uint32_t npairs = x ? N / 2 : N;
            for (uint32_t g = threadIdx.x; g < npairs; g += kT) {
                const uint32_t i = x ? (((g >> pb) << (pb + 1)) | (g & ((1u << pb) - 1u))) : g;
                const uint32_t j = i ^ x;
                const float2 a = n == T ? tile[sw(i)] : sv[i];
                const float2 b = x ? (n == T ? tile[sw(j)] : sv[j]) : a;
                const float re = a.x * b.x + a.y * b.y, im = a.y * b.x - a.x * b.y;
                const float ti = P.use_im ? im : re;
                run += (__popc(i & z) & 1) ? -ti : ti;
                if (x) {
                    const float tj = P.use_im ? -im : re;
                    run += (__popc(j & z) & 1) ? -tj : tj;
                }
                if (++cnt == 8) {
                    acc += (double)run;
                    run = 0.f;
                    cnt = 0;
                }
            }
            acc += (double)run;
            const double tot = block_sum(acc, red);
            if (threadIdx.x == 0) out[it.out_begin + s] = (double)P.sign * tot;
        }
    }
}

}  // namespace

cudaError_t launch_batch(const LaunchCtx &L, float2 *states, const BItem *items, int n_items, const BStage *stages,
                         const BOp *ops, const float2 *pool, const BStr *strs, double *out, int *counter,
                         int keep_states) {
    const int smem = (int)sizeof(float2) * ((1 << kBatchTileQubits) + kBatchStageMat);
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counter, 0, sizeof(int), L.stream);
    if (e != cudaSuccess) return e;
    int grid = L.num_sms;
    if (grid > n_items) grid = n_items;
    if (grid < 1) grid = 1;
    k_batch<<<grid, kT, smem, L.stream>>>(states, items, n_items, stages, ops, pool, strs, out, counter, keep_states);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace svk
