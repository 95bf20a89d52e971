// k_tc.cu -- fused 6-qubit gate application on the 5th-generation tensor cores
// (tcgen05, TMEM accumulators). Sec. II-B: gate fusion turns many small
// memory-bound gates into one 2^k x 2^k product; beyond k = 5 (complex64) the
// product is compute-bound on CUDA cores, so here it runs on the tensor cores.
//
// View the state as 64 x 2^(n-6): column c holds the 64 members of group c (the
// amplitudes whose non-target bits spell c); one fused gate G is the same
// product for every column. Two kernels:
//   k_tc6_raw (every state of 7 qubits or more): the state tile itself is the
//     MN-major B operand and the contraction runs over the 64 members
//     (described at the kernel); with qubit 0 a target the tile's member pairs
//     are rearranged into member rows in shared memory;
//   k_tc6 (a 6-qubit state, one column): with x_c the 128 reals of column c (re, im
//     interleaved: K index 2j + e for member j),
//       out_c = A x_c,  A[2j+e][2l+f] = the real 2x2 block [[Re, -Im], [Im, Re]] of G[j][l],
//     i.e. the real GEMM D(128 x N) = A(128 x 128) * B(128 x N) with B's
//     columns the state columns, staged through registers into the K-major
//     128-byte-swizzled layout.
//
// Precision: TF32 (operands rounded to nearest TF32, FP32 accumulation) or
// split BF16 (x = hi + lo with hi, lo BF16; A*B ~ Ahi*Bhi + Ahi*Blo + Alo*Bhi,
// three MMAs into one FP32 accumulator).
//
// k_tc6 structure (one persistent CTA per SM, 544 threads):
//   warps 0-7   producers: read a tile of 128 columns x 64 members from HBM in
//               address order (16-byte loads, each warp load one contiguous
//               512-byte run, whatever the target positions), round or split,
//               and scatter it to shared memory in the canonical K-major
//               128-byte-swizzled operand layout; two tile buffers;
//   warp 16     MMA issuer: one thread issues tcgen05.mma (M = N = 128) into one
//               of two TMEM accumulators and commits to mbarriers;
//   warps 8-15  epilogue: tcgen05.ld of the accumulator rows (warp w reads TMEM
//               lanes 32*(w%4)..+31, columns of one half of the tile), stage
//               them in shared memory and store runs of 16 members of one
//               column (qubit 0 being a target, members 2m and 2m + 1 are
//               adjacent amplitudes).
// Addresses: a tile starts at a multiple of 128 columns, so the amplitude
// offset of column t*128 + i is col_base(t*128) | pd[i], with the deposit table
// pd[] computed once per CTA.
// A (the gate) is staged once per CTA from a host-built image of its swizzled
// shared-memory layout. Every mbarrier wait is bounded by a clock budget; on
// expiry the kernel records an error code in the device status word, drains
// its own MMAs (again bounded), frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include <cstring>
#include <vector>

#include "sv_internal.h"

namespace svk {
namespace {

constexpr int kNT = 128;              // columns per tile (MMA N)
constexpr int kProdWarps = 8;         // warps 0..7
constexpr int kEpiWarps = 8;          // warps 8..15: two per TMEM lane quarter, one per column half
constexpr int kMmaWarp = kProdWarps + kEpiWarps;
constexpr int kThreadsTC = (kMmaWarp + 1) * 32;
constexpr int kProd = kProdWarps * 32;
constexpr int kEpi = kEpiWarps * 32;
constexpr int kAImg = 64 * 1024;      // bytes of the A image (either precision)
constexpr int kBStage = 64 * 1024;    // bytes of one B tile (either precision)
constexpr int kTmemCols = 2 * kNT;    // two accumulators
constexpr int kStgPitch = 17;         // floats per staged accumulator row (16 columns + 1 against bank conflicts)
constexpr int kEpiStage = kEpiWarps * 32 * kStgPitch * 4;   // bytes of epilogue staging
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz
constexpr int kErrTimeout = 0x7c01;

enum Prec { TF32 = 1, BF16 = 2 };

// Control block in dynamic shared memory after the operand area and the
// epilogue staging; the producer's tile tables in static shared memory.
struct TcCtl {
    unsigned long long full[2], empty[2], acc_full[2], acc_empty[2], done;
    uint16_t pd[kNT];   // column offset i in a tile -> amplitude offset (the 7 lowest non-target
                        // positions are below 13, so the offset fits 16 bits)
    unsigned tmem_base;
    int abort;
};
struct TcTab {
    // A tile's 8192 amplitudes in address order: index a (13 bits) deposited into
    // the 13 tile bit positions (the 6 targets and the 7 lowest other bits).
    uint64_t adr_lo[128], adr_hi[64];   // a's bits 0..6 / 7..12 -> amplitude offset
    uint16_t ij_lo[128], ij_hi[64];     // the same bits -> column i | member j << 7
};
constexpr int kErrSmemAlign = 0x7c02;

// dynamic shared memory of k_tc6: operands, staging, control
__host__ __device__ constexpr int tc_stage_off() { return kAImg + 2 * kBStage; }
__host__ __device__ constexpr int tc_ctl_off() { return tc_stage_off() + kEpiStage; }
__host__ __device__ constexpr int tc_smem_bytes() { return tc_ctl_off() + (int)sizeof(TcCtl); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false on timeout or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int *abort_flag, int *d_err,
                                          long long budget = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_try(a, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) {
            *abort_flag = 1;
            atomicExch(d_err, kErrTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start address, leading byte offset
// (unused for swizzled K-major, set to 16 B), stride byte offset 1024 B (eight
// 128-byte rows), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// Instruction descriptor: D = F32, A/B format (TF32 = 2, BF16 = 1), both K-major,
// N = 128 (bits 17-22 hold N >> 3), M = 128 (bits 24-28 hold M >> 4).
template <int P> __host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | ((P == TF32 ? 2u : 1u) << 7) | ((P == TF32 ? 2u : 1u) << 10) | ((uint32_t)(kNT >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

template <int P>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (P == TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc<P>()), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc<P>()), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// (hi, lo) BF16 pairs of (a, b), packed with a in the low half
__device__ __forceinline__ void split_bf16(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

struct TcGeom {
    int pos[6];          // target positions, ascending
    uint64_t off[64];    // member offsets
    uint64_t n_cols;     // 2^(n-6)
    uint64_t n_tiles;
};

__device__ __forceinline__ uint64_t col_base(uint64_t c, const TcGeom &G) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint64_t lo = c & ((1ull << G.pos[i]) - 1ull);
        c = ((c ^ lo) << 1) | lo;
    }
    return c;
}

// byte offset of the 16-byte chunk `chunk` (0..7 within the 128-byte row) of
// row r in K-block kb of an operand with `rows` rows (128-byte swizzle)
__device__ __forceinline__ uint32_t sw128(int kb, int r, int chunk) {
    return (uint32_t)(kb * (kNT * 128) + (r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4));
}

template <int P>
__global__ void __launch_bounds__(kThreadsTC, 1)
k_tc6(float2 *__restrict__ sv, TcGeom G, const uint4 *__restrict__ a_img, int *__restrict__ d_err) {
    // The operand area starts the dynamic shared memory and must be 1024-byte
    // aligned (128-byte swizzle atoms). Checked, uniformly for all threads, before
    // any barrier or TMEM allocation: a misplaced window records an error and
    // returns.
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    if (smem_u32(smem_dyn) & 1023u) {
        if (threadIdx.x == 0) atomicExch(d_err, kErrSmemAlign);
        return;
    }
    TcCtl &S = *reinterpret_cast<TcCtl *>(smem_dyn + tc_ctl_off());
    __shared__ TcTab T;
    unsigned char *sA = smem_dyn;
    unsigned char *sB0 = smem_dyn + kAImg;     // stage s at sB0 + s * kBStage
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort_flag = &S.abort;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&S.full[i]), kProd);
            mbar_init(smem_u32(&S.empty[i]), 1);
            mbar_init(smem_u32(&S.acc_full[i]), 1);
            mbar_init(smem_u32(&S.acc_empty[i]), kEpi);
        }
        mbar_init(smem_u32(&S.done), 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // A tile starts at a multiple of kNT columns, so col_base(t*kNT + i) = col_base(t*kNT) | pd[i]
    if (threadIdx.x < kNT) S.pd[threadIdx.x] = (uint16_t)col_base((uint64_t)threadIdx.x, G);
    if (threadIdx.x >= kNT && threadIdx.x < kNT + 192) {
        // tile bit b (0..12) in ascending position: either target tj (member bit tj)
        // or the k-th lowest non-target (column bit k); positions >= n only occur
        // for states under 13 qubits and land in columns >= n_cols (never loaded)
        const int e = threadIdx.x - kNT;
        const bool hi = e >= 128;
        const int v = hi ? e - 128 : e;
        uint64_t adr = 0;
        uint32_t ij = 0;
        int b = 0, tj = 0, k = 0;
        for (int p = 0; b < 13; ++p) {
            const bool is_t = tj < 6 && G.pos[tj] == p;
            if (!is_t && k >= 7) continue;
            const int vb = hi ? b - 7 : b;
            if (vb >= 0 && vb < (hi ? 6 : 7) && ((v >> vb) & 1)) {
                adr |= 1ull << p;
                ij |= is_t ? (1u << (7 + tj)) : (1u << k);
            }
            if (is_t) ++tj; else ++k;
            ++b;
        }
        if (hi) { T.adr_hi[v] = adr; T.ij_hi[v] = (uint16_t)ij; }
        else { T.adr_lo[v] = adr; T.ij_lo[v] = (uint16_t)ij; }
    }
    // A image -> shared memory (plain copy; the host built the swizzled layout)
    for (int i = threadIdx.x; i < kAImg / 16; i += kThreadsTC) reinterpret_cast<uint4 *>(sA)[i] = a_img[i];
    fence_proxy_async();
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const uint64_t ntl = G.n_tiles;

    if (warp < kProdWarps) {
        // ---------------- producers ----------------
            // Each thread loads 16 pairs of adjacent amplitudes of the tile in address
            // order (lane-consecutive 16-byte loads: every warp load is one contiguous
            // 512-byte run), then scatters each amplitude to its (column, member) slot
            // of the K-major swizzled operand, rounded to TF32 or split into BF16.
            int i = 0;
            for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
                const int s = i & 1, u = i >> 1;
                if (u >= 1 && !mbar_wait(smem_u32(&S.empty[s]), (u - 1) & 1, abort_flag, d_err)) break;
                const uint64_t tb = col_base(t * kNT, G);
                const uint64_t tcol = t * kNT;
                float4 v[16];
    #pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int a = 2 * ((int)threadIdx.x + kProd * r);
                    const int ij = T.ij_lo[a & 127] | T.ij_hi[a >> 7];
                    v[r] = (tcol + (ij & 127) < G.n_cols)
                               ? *reinterpret_cast<const float4 *>(sv + (tb | T.adr_lo[a & 127] | T.adr_hi[a >> 7]))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                unsigned char *sb = sB0 + s * kBStage;
    #pragma unroll
                for (int r = 0; r < 16; ++r) {
    #pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int a = 2 * ((int)threadIdx.x + kProd * r) + h;
                        const int ij = T.ij_lo[a & 127] | T.ij_hi[a >> 7];
                        const int col = ij & 127, j = ij >> 7;
                        const float re = h ? v[r].z : v[r].x, im = h ? v[r].w : v[r].y;
                        if constexpr (P == TF32) {
                            // K = 2j, 2j+1: K-block j/16, chunk (j%16)/2, 8-byte half j%2
                            *reinterpret_cast<uint2 *>(sb + sw128(j >> 4, col, (j & 15) >> 1) + (j & 1) * 8) =
                                make_uint2(to_tf32(re), to_tf32(im));
                        } else {
                            // K = 2j, 2j+1: K-block j/32, chunk (j%32)/4, 4-byte quarter j%4
                            uint32_t hi, lo;
                            split_bf16(re, im, hi, lo);
                            const uint32_t o = sw128(j >> 5, col, (j & 31) >> 2) + (j & 3) * 4;
                            *reinterpret_cast<uint32_t *>(sb + o) = hi;
                            *reinterpret_cast<uint32_t *>(sb + kBStage / 2 + o) = lo;
                        }
                    }
                }
                fence_proxy_async();
                mbar_arrive(smem_u32(&S.full[s]));
            }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t a_addr = smem_u32(sA);
            int i = 0;
            for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
                const int s = i & 1, a = i & 1, u = i >> 1;
                if (!mbar_wait(smem_u32(&S.full[s]), u & 1, abort_flag, d_err)) break;
                if (u >= 1 && !mbar_wait(smem_u32(&S.acc_empty[a]), (u - 1) & 1, abort_flag, d_err)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a * kNT);
                const uint32_t b_addr = smem_u32(sB0) + (uint32_t)(s * kBStage);
                if constexpr (P == TF32) {
                    // K = 128 in 16 steps of 8 (32 bytes); 4 steps per 128-byte K-block
#pragma unroll
                    for (int ks = 0; ks < 16; ++ks) {
                        const uint32_t off = (uint32_t)((ks >> 2) * (kNT * 128) + (ks & 3) * 32);
                        mma<P>(d_tmem, sdesc(a_addr + off), sdesc(b_addr + off), ks > 0);
                    }
                } else {
                    // K = 128 in 8 steps of 16 (32 bytes); Ahi*Bhi + Ahi*Blo + Alo*Bhi
                    const uint32_t a_lo = a_addr + kAImg / 2, b_lo = b_addr + kBStage / 2;
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const uint32_t off = (uint32_t)((ks >> 2) * (kNT * 128) + (ks & 3) * 32);
                        mma<P>(d_tmem, sdesc(a_addr + off), sdesc(b_addr + off), ks > 0);
                        mma<P>(d_tmem, sdesc(a_addr + off), sdesc(b_lo + off), 1);
                        mma<P>(d_tmem, sdesc(a_lo + off), sdesc(b_addr + off), 1);
                    }
                }
                mma_commit(smem_u32(&S.empty[s]));
                mma_commit(smem_u32(&S.acc_full[a]));
            }
            // drain: every MMA issued above has completed once `done` flips; if it
            // does not within the bound, the failure is recorded like any other wait
            mma_commit(smem_u32(&S.done));
            const long long t0 = clock64();
            bool drained;
            while (!(drained = mbar_try(smem_u32(&S.done), 0)) && clock64() - t0 < kWaitCycles) {
            }
            if (!drained) {
                *abort_flag = 1;
                atomicExch(d_err, kErrTimeout);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        // Each warp reads 16 accumulator columns of its 32 TMEM lanes (16 members
        // x re/im) at a time, stages them in shared memory, and stores them back
        // so that every store instruction writes contiguous runs: 16 consecutive
        // members of one column (qubit 0 is a target, so members 2m and 2m + 1
        // are adjacent amplitudes). Lane-per-row stores that scatter over 16 rows
        // run at a fraction of HBM bandwidth when the rows are far apart.
        const int ew = warp - kProdWarps;
        const int sub = warp & 3;                   // TMEM lanes 32*sub .. 32*sub+31: members 16*sub .. +15
        const int half = ew >> 2;                   // columns 64*half .. 64*half+63 of the tile
        float *stg = reinterpret_cast<float *>(smem_dyn + tc_stage_off()) + ew * 32 * kStgPitch;
        const int jj = lane & 15;                   // member 16*sub + jj
        const uint64_t offj = G.off[16 * sub + jj];
        int i = 0;
        for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
            const int a = i & 1, u = i >> 1;
            if (!mbar_wait(smem_u32(&S.acc_full[a]), u & 1, abort_flag, d_err)) break;
            tc_fence_after();
            const uint64_t tb = col_base(t * kNT, G);
            const uint64_t tcol = t * kNT;
#pragma unroll 1
            for (int cc = 0; cc < 4; ++cc) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(a * kNT + half * 64 + cc * 16), v);
#pragma unroll
                for (int c = 0; c < 16; ++c) stg[lane * kStgPitch + c] = v[c];
                __syncwarp();
                const int c0 = half * 64 + cc * 16;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int col = 2 * r + (lane >> 4);
                    const float re = stg[(2 * jj) * kStgPitch + col];
                    const float im = stg[(2 * jj + 1) * kStgPitch + col];
                    const int ci = c0 + col;
                    if (tcol + ci < G.n_cols) sv[(tb | S.pd[ci]) + offj] = make_float2(re, im);
                }
                __syncwarp();
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&S.acc_empty[a]));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------- raw-operand variant (TF32 or split BF16) ----------------
// The same product written with the member index as the contraction:
//   D(128 x 256) = A(128 x 64) * B(64 x 256),  B[l][2i + f] = component f of
//   amplitude (member l, column i),  A row m = 32q + r: member j = 16q + r % 16,
//   Re G[j][.] for r < 16 and Im G[j][.] for r >= 16,
// so D holds (Re G) x and (Im G) x for the re and im parts of x, and
//   out_j = (Re G x_re - Im G x_im, Re G x_im + Im G x_re)
// combines two rows that sit 16 TMEM lanes apart in the same warp's quarter.
// B in shared memory is the state itself, MN-major (columns contiguous): a stage
// is 64 atoms of 1 KiB, atom (a, g) = columns-floats 32a .. 32a+31 of members
// 8g .. 8g+7 at a * 8192 + g * 1024, each in the 128-byte swizzle with 32-byte
// atomicity (the swizzle tf32 MMA takes for MN-major operands; with the plain
// 128-byte swizzle it produced no result on GB300). Each 16-byte chunk is two
// adjacent amplitudes of one member. Roles (15 warps): 2 copy warps issue
// cp.async.cg (no registers, no L1 allocation) and let the copies arrive on the
// stage's `landed` barrier, so they never wait for data; 4 convert warps prepare
// the landed stage in place -- TF32: round to nearest (the tensor core drops the
// low 13 bits, which measured as a norm drift of -3.5e-4 per gate unrounded);
// split BF16: each warp turns one 1 KiB atom into a 512-byte hi atom and a
// 512-byte lo atom (x = hi + lo, both BF16, 64-byte swizzle) in the same 1 KiB;
// one thread issues the MMAs (TF32: 8 of K = 8; BF16: Ahi Bhi + Ahi Blo + Alo Bhi
// for 4 steps of K = 16); 8 epilogue warps combine, write the tile's result into
// the stage it came from and store it back in runs of columns. Three stages
// rotate. With qubit 0 free a 16-byte chunk is two adjacent amplitudes (columns
// 2p, 2p + 1) of one member; with qubit 0 a target (T0) it is members 2m, 2m + 1
// of one column: the copies land columns 2p and 2p + 1 in rows 2m and 2m + 1 of
// pair p, the convert stage trades the rows' 8-byte halves (TF32: in the same
// pass as the rounding; BF16: by one shuffle before the split), and the epilogue
// trades them back (one shuffle between the lanes of rows j and j ^ 1) before
// the result is stored in memory order.
constexpr int kNT3 = 128;                     // columns per tile (MMA N = 2 * kNT3 reals)
constexpr int kStages3 = 3;
constexpr int kA3 = 128 * 64 * 4;             // A image: 128 rows x 64 tf32 (or BF16 hi + lo), K-major
constexpr int kB3 = 64 * 2 * kNT3 * 4;        // one stage: 64 members x 256 floats
constexpr int kCopyWarps3 = 2;                // warps 0-1: cp.async issue
constexpr int kRoundWarps3 = 4;               // warps 2-5: TF32 rounding / BF16 split in place
constexpr int kProdWarps3 = kCopyWarps3 + kRoundWarps3;
constexpr int kEpiWarps3 = 8;                 // warps 6-13
constexpr int kMmaWarp3 = kProdWarps3 + kEpiWarps3;
constexpr int kThreads3 = (kMmaWarp3 + 1) * 32;
constexpr int kTmemCols3 = 2 * 2 * kNT3;      // two accumulators of 256 columns

struct TcCtl3 {
    unsigned long long landed[kStages3], full[kStages3], empty[kStages3], acc_full[2], acc_empty[2], done;
    unsigned tmem_base;
    int abort;
};
constexpr int kGuard3 = 2048;              // unused bytes after the last stage
constexpr int kSmem3 = kA3 + kStages3 * kB3 + kGuard3 + (int)sizeof(TcCtl3);
static_assert(kSmem3 <= 227 * 1024, "dynamic shared memory of the raw-operand kernel exceeds the per-block limit");

// byte offset of the 16-byte chunk holding floats 4c .. 4c+3 of member row l
// (c = amplitude pair, 0..63) in a stage: atom (c / 8, l / 8); inside it rows of
// 128 bytes (32 floats of one member) whose four 32-byte units are permuted by
// the row index mod 4
__device__ __forceinline__ uint32_t mn_chunk(int l, int c) {
    return (uint32_t)((c >> 3) * 8192 + (l >> 3) * 1024 + (l & 7) * 128 + ((((c & 7) >> 1) ^ (l & 3)) << 5) +
                      ((c & 1) << 4));
}

// MN-major operand descriptor: column atoms 8192 bytes apart (leading offset),
// 8-row member groups `sbo` bytes apart, swizzle `mode` (1: 128 bytes with
// 32-byte atomicity, 4: 64 bytes). Either reading of the two offsets stays
// inside the stage and its guard.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t addr, uint32_t sbo, uint32_t mode) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(8192u >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= 1ull << 46;
    d |= (uint64_t)mode << 61;
    return d;
}

// D = F32, A = B = TF32 (2) or BF16 (1), A K-major, B MN-major (bit 16), N = 256, M = 128
template <int P>
__host__ __device__ constexpr uint32_t idesc3() {
    return (1u << 4) | ((P == TF32 ? 2u : 1u) << 7) | ((P == TF32 ? 2u : 1u) << 10) | (1u << 16) |
           ((uint32_t)((2 * kNT3) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// split BF16: one warp turns the 1 KiB atom at `atom` (8 rows x 32 floats, 128-byte
// swizzle with 32-byte atomicity) into hi / lo atoms of 8 rows x 32 BF16 (64-byte
// swizzle: 16-byte chunk c of row r at r * 64 + ((c ^ (r / 2 % 4)) << 4)) at atom
// and atom + 512. Every lane reads its 32 bytes before any lane writes.
template <bool T0 = false>
__device__ __forceinline__ void split_atom(uint32_t atom, int lane) {
    const int r = lane >> 2, u = lane & 3;          // row, physical 32-byte unit
    const int lu = u ^ (r & 3);                     // logical unit: floats 8 lu .. 8 lu + 7
    float x[8];
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
                 : "r"(atom + (uint32_t)(r * 128 + u * 32)));
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "r"(atom + (uint32_t)(r * 128 + u * 32 + 16)));
    if constexpr (T0) {
        // rows 2m, 2m + 1 landed as member pairs of columns 2p, 2p + 1 (qubit 0 a
        // target): trade 8-byte halves with the lane holding the same columns of
        // the other row (lane ^ 5), so each row holds its own member of both columns
        const bool even = (r & 1) == 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float *c = x + 4 * h;
            const float s0 = __shfl_xor_sync(0xffffffffu, even ? c[2] : c[0], 5);
            const float s1 = __shfl_xor_sync(0xffffffffu, even ? c[3] : c[1], 5);
            if (even) {
                c[2] = s0;
                c[3] = s1;
            } else {
                c[0] = s0;
                c[1] = s1;
            }
        }
    }
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) split_bf16(x[2 * k], x[2 * k + 1], hi[k], lo[k]);
    __syncwarp();
    const uint32_t o = (uint32_t)(r * 64 + ((lu ^ ((r >> 1) & 3)) << 4));
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(atom + o), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]),
                 "r"(hi[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(atom + 512u + o), "r"(lo[0]), "r"(lo[1]), "r"(lo[2]),
                 "r"(lo[3])
                 : "memory");
    __syncwarp();
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// Which chunk of the tile each copy (and store) moves is set by the host
// (RawMap): with qubit 0 free a chunk is amplitudes (2p, 2p + 1) of member row l
// (2 x 6 index bits: the member's bits sit at the target positions, the pair's at
// non-target positions 1..6); with qubit 0 a target (T0) it is members 2m, 2m + 1
// of one column c (5 member-pair bits at target positions 1..5, 7 column bits at
// the non-target positions), landed in row 2m + (c & 1) of pair c / 2 and turned
// into member rows by the convert stage. The index bits are ordered by the
// address position they set (the three lowest lane bits chosen among the low
// ones so that eight consecutive lanes hit eight different 16-byte bank groups
// of shared memory); the five first vary across the lanes of a warp, the next
// one across the two copy warps, the rest across a thread's copies.
// Both the amplitude address and the operand offset (mn_chunk is linear over
// XOR) are OR / XOR of per-bit contributions, so a thread combines one
// per-thread and one per-copy table entry.
struct RawMap {
    uint64_t cthr_addr[64], cit_addr[64];   // copy: amplitude offset, thread part / copy part
    uint32_t cthr_sm[64], cit_sm[64];       // copy: operand byte offset in a stage
    uint32_t cthr_col[64], cit_col[64];     // copy: first column of the chunk (ragged tiles)
    uint64_t sl_addr[32], sr_addr[16];      // store: lane part / iteration part (one epilogue warp)
    uint32_t sl_sm[32], sr_sm[16];
    uint32_t sl_col[32], sr_col[16];
};

// Copy and store orders: PLAIN and IL are fixed orders for qubit 0 free (PLAIN:
// each instruction 32 consecutive amplitude pairs of one member; IL, lowest
// target t0 = 1..3: groups of g = 2^(t0-1) lanes alternate between members l and
// l ^ 1, lg = log2 g), MAPPED the table order of RawMap (qubit 0 free), T0 the
// table order with qubit 0 a target.
enum RawMode { RAW_PLAIN = 0, RAW_IL = 1, RAW_MAPPED = 2, RAW_T0 = 3 };

template <int P, int MODE>
__global__ void __launch_bounds__(kThreads3, 1)
k_tc6_raw(float2 *__restrict__ sv, const TcGeom G, const RawMap R, const uint4 *__restrict__ a_img,
          int *__restrict__ d_err, int lg) {
    constexpr bool T0 = MODE == RAW_T0, TABLE = MODE == RAW_MAPPED || MODE == RAW_T0, IL = MODE == RAW_IL;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    if (smem_u32(smem_dyn) & 1023u) {
        if (threadIdx.x == 0) atomicExch(d_err, kErrSmemAlign);
        return;
    }
    TcCtl3 &S = *reinterpret_cast<TcCtl3 *>(smem_dyn + kA3 + kStages3 * kB3 + kGuard3);
    unsigned char *sA = smem_dyn;
    const uint32_t sB0 = smem_u32(smem_dyn + kA3);     // stage s at sB0 + s * kB3
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort_flag = &S.abort;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages3; ++i) {
            mbar_init(smem_u32(&S.landed[i]), kCopyWarps3 * 32);
            mbar_init(smem_u32(&S.full[i]), kRoundWarps3 * 32);
            mbar_init(smem_u32(&S.empty[i]), kEpiWarps3 * 32);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&S.acc_full[i]), 1);
            mbar_init(smem_u32(&S.acc_empty[i]), kEpiWarps3 * 32);
        }
        mbar_init(smem_u32(&S.done), 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < kA3 / 16; i += kThreads3) reinterpret_cast<uint4 *>(sA)[i] = a_img[i];
    fence_proxy_async();
    if (warp == kMmaWarp3) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols3)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const uint64_t ntl = G.n_tiles;

    if (warp < kCopyWarps3) {
        // ---------------- copy ----------------
        // The copies signal `landed` themselves (cp.async.mbarrier.arrive), so these
        // threads never wait for data.
        const int tid = threadIdx.x;
        int i = 0;
        if constexpr (TABLE) {
            // chunk k of thread t is chunk index cthr[t] ^ cit[k] of the tile (RawMap)
            const uint64_t ta = R.cthr_addr[tid];
            const uint32_t tsm = R.cthr_sm[tid], tcol = R.cthr_col[tid];
            const bool full = G.n_cols >= (uint64_t)kNT3;
            for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
                const int s = i % kStages3, u = i / kStages3;
                if (u >= 1 && !mbar_wait(smem_u32(&S.empty[s]), (u - 1) & 1, abort_flag, d_err)) break;
                const uint64_t tb = col_base(t * kNT3, G) | ta;
                const uint32_t sb = sB0 + (uint32_t)(s * kB3);
                if (full) {
#pragma unroll 16
                    for (int k = 0; k < 64; ++k) cp_async16(sb + (tsm ^ R.cit_sm[k]), sv + (tb | R.cit_addr[k]), 16u);
                } else {
                    for (int k = 0; k < 64; ++k) {
                        const bool ok = (uint64_t)(tcol | R.cit_col[k]) < G.n_cols;
                        cp_async16(sb + (tsm ^ R.cit_sm[k]), ok ? sv + (tb | R.cit_addr[k]) : sv, ok ? 16u : 0u);
                    }
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.landed[s]))
                             : "memory");
            }
        } else {
            // thread c takes amplitude pair c of all 64 members (a warp load is 32
            // consecutive pairs of one member: 512 contiguous bytes once the lowest target
            // is 6 or more); with IL, thread t takes pairs c' and c' + 32
            // (c' = t % g + (t / 2g) g) of the members with bit 0 = (t / g) % 2
            const int g = 1 << lg;
            const int c0 = IL ? (tid & (g - 1)) + ((tid >> (lg + 1)) << lg) : tid;
            const uint64_t pc0 = col_base((uint64_t)(2 * c0), G);
            const uint64_t pc1 = col_base((uint64_t)(2 * (c0 + 32)), G);
            const bool ok0 = (uint64_t)(2 * c0) < G.n_cols, ok1 = (uint64_t)(2 * (c0 + 32)) < G.n_cols;
            const int mb = IL ? (tid >> lg) & 1 : 0;
            const uint64_t offb = IL ? G.off[mb] : 0;
            for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
                const int s = i % kStages3, u = i / kStages3;
                if (u >= 1 && !mbar_wait(smem_u32(&S.empty[s]), (u - 1) & 1, abort_flag, d_err)) break;
                const uint64_t tb = col_base(t * kNT3, G);
                const uint32_t sb = sB0 + (uint32_t)(s * kB3);
                if constexpr (IL) {
                    const uint64_t b0 = tb | pc0 | offb, b1 = tb | pc1 | offb;
#pragma unroll 8
                    for (int m = 0; m < 32; ++m) {
                        const int l = 2 * m + mb;
                        const uint64_t om = G.off[2 * m];
                        cp_async16(sb + mn_chunk(l, c0), ok0 ? sv + (b0 | om) : sv, ok0 ? 16u : 0u);
                        cp_async16(sb + mn_chunk(l, c0 + 32), ok1 ? sv + (b1 | om) : sv, ok1 ? 16u : 0u);
                    }
                } else {
                    const uint64_t b0 = tb | pc0;
#pragma unroll 16
                    for (int l = 0; l < 64; ++l)
                        cp_async16(sb + mn_chunk(l, c0), ok0 ? sv + (b0 | G.off[l]) : sv, ok0 ? 16u : 0u);
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.landed[s]))
                             : "memory");
            }
        }
        // every copy this thread issued has landed before the CTA may exit
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp < kProdWarps3) {
        // ---------------- convert: TF32 rounding or BF16 split, in place ----------------
        // TF32: the tensor core reads a TF32 operand as the float's top 19 bits; adding
        // half of their last place (0x1000) to the bit pattern first makes that
        // truncation a rounding to nearest, ties away from zero (what cvt.rna.tf32.f32
        // computes), for one integer add per value.
        const int rt = threadIdx.x - kCopyWarps3 * 32;   // 0..127: pair rt & 63, members 2r + rt / 64
        const int rw = rt >> 5;                          // convert warp 0..3: BF16 atoms 16 rw .. 16 rw + 15
        int i = 0;
        for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
            const int s = i % kStages3;
            if (!mbar_wait(smem_u32(&S.landed[s]), (i / kStages3) & 1, abort_flag, d_err)) break;
            const uint32_t sb = sB0 + (uint32_t)(s * kB3);
            if constexpr (P == TF32 && T0) {
                // rows 2m, 2m + 1 hold members (2m, 2m + 1) of columns 2p and 2p + 1:
                // trade the 8-byte halves so that each row holds its own member
#pragma unroll 4
                for (int m = 16 * (rt >> 6); m < 16 * (rt >> 6) + 16; ++m) {
                    const uint32_t a0 = sb + mn_chunk(2 * m, rt & 63), a1 = sb + mn_chunk(2 * m + 1, rt & 63);
                    uint32_t x0, y0, z0, w0, x1, y1, z1, w1;
                    asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];" : "=r"(x0), "=r"(y0), "=r"(z0), "=r"(w0) : "r"(a0));
                    asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];" : "=r"(x1), "=r"(y1), "=r"(z1), "=r"(w1) : "r"(a1));
                    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a0), "r"(x0 + 0x1000u), "r"(y0 + 0x1000u),
                                 "r"(x1 + 0x1000u), "r"(y1 + 0x1000u)
                                 : "memory");
                    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a1), "r"(z0 + 0x1000u), "r"(w0 + 0x1000u),
                                 "r"(z1 + 0x1000u), "r"(w1 + 0x1000u)
                                 : "memory");
                }
            } else if constexpr (P == TF32) {
#pragma unroll 8
                for (int r = 0; r < 32; ++r) {
                    const uint32_t a = sb + mn_chunk(2 * r + (rt >> 6), rt & 63);
                    uint32_t x, y, z, w;
                    asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];" : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(a));
                    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(x + 0x1000u), "r"(y + 0x1000u),
                                 "r"(z + 0x1000u), "r"(w + 0x1000u)
                                 : "memory");
                }
            } else {
#pragma unroll 4
                for (int k = 0; k < 16; ++k) split_atom<T0>(sb + (uint32_t)((16 * rw + k) * 1024), lane);
            }
            fence_proxy_async();
            mbar_arrive(smem_u32(&S.full[s]));
        }
    } else if (warp == kMmaWarp3) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t a_addr = smem_u32(sA);
            int i = 0;
            for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
                const int s = i % kStages3, a = i & 1;
                if (!mbar_wait(smem_u32(&S.full[s]), (i / kStages3) & 1, abort_flag, d_err)) break;
                if (i >= 2 && !mbar_wait(smem_u32(&S.acc_empty[a]), ((i >> 1) - 1) & 1, abort_flag, d_err)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a * 2 * kNT3);
                const uint32_t b_addr = sB0 + (uint32_t)(s * kB3);
                if constexpr (P == TF32) {
                    // K = 64 members in 8 steps of 8: A K-block ks / 4 (16 KB apart), 32 bytes
                    // per step within its rows; B member group ks (1024 bytes apart)
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const uint64_t ad = sdesc(a_addr + (uint32_t)((ks >> 2) * 16384 + (ks & 3) * 32));
                        const uint64_t bd = sdesc_mn(b_addr + (uint32_t)(ks * 1024), 512u, 1u);
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                            "l"(ad), "l"(bd), "r"(idesc3<TF32>()), "r"(ks)
                            : "memory");
                    }
                } else {
                    // K = 64 members in 4 steps of 16 (A: 32 bytes per step within its 128-byte
                    // rows, lo image 16 KB on; B: member groups 2 ks, 2 ks + 1, lo atoms 512
                    // bytes on): Ahi Bhi + Ahi Blo + Alo Bhi
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ah = sdesc(a_addr + (uint32_t)(ks * 32));
                        const uint64_t al = sdesc(a_addr + 16384u + (uint32_t)(ks * 32));
                        const uint64_t bh = sdesc_mn(b_addr + (uint32_t)(ks * 2048), 1024u, 4u);
                        const uint64_t bl = sdesc_mn(b_addr + (uint32_t)(ks * 2048 + 512), 1024u, 4u);
                        const uint64_t av[3] = {ah, ah, al}, bv[3] = {bh, bl, bh};
#pragma unroll
                        for (int x = 0; x < 3; ++x)
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                                "l"(av[x]), "l"(bv[x]), "r"(idesc3<BF16>()), "r"(ks + x)
                                : "memory");
                    }
                }
                mma_commit(smem_u32(&S.acc_full[a]));
            }
            mma_commit(smem_u32(&S.done));
            const long long t0 = clock64();
            bool drained;
            while (!(drained = mbar_try(smem_u32(&S.done), 0)) && clock64() - t0 < kWaitCycles) {
            }
            if (!drained) {
                *abort_flag = 1;
                atomicExch(d_err, kErrTimeout);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        // warp: TMEM lane quarter q (members 16q .. 16q + 15, Re rows then Im rows),
        // column half hh (amplitudes 64 hh .. 64 hh + 63 of the tile)
        const int ew = warp - kProdWarps3;
        const int q = warp & 3, hh = ew >> 2;
        const int e = lane >> 4, j = 16 * q + (lane & 15);
        // TABLE: this warp's 512 chunks (rows 16q .. 16q+15, pairs 32hh .. 32hh+31) in the
        // order of RawMap; otherwise each lane stores pair cst (PLAIN) or, with IL, member
        // bit lb and pairs 32 hh + pl and 32 hh + 16 + pl
        const uint64_t wa = TABLE ? G.off[16 * q] | col_base((uint64_t)(64 * hh), G) | R.sl_addr[lane] : 0;
        const uint32_t wsm = TABLE ? mn_chunk(16 * q, 32 * hh) ^ R.sl_sm[lane] : 0;
        const uint32_t wcol = TABLE ? (uint32_t)(64 * hh) | R.sl_col[lane] : 0;
        const int cst = 32 * hh + lane;
        const uint64_t pst = col_base((uint64_t)(2 * cst), G);
        const bool okst = (uint64_t)(2 * cst) < G.n_cols;
        const int lb = (lane >> lg) & 1, pl = (lane & ((1 << lg) - 1)) + ((lane >> (lg + 1)) << lg);
        const uint64_t pst0 = IL ? col_base((uint64_t)(2 * (32 * hh + pl)), G) : 0;
        const uint64_t pst1 = IL ? col_base((uint64_t)(2 * (32 * hh + 16 + pl)), G) : 0;
        int i = 0;
        for (uint64_t t = blockIdx.x; t < ntl; t += gridDim.x, ++i) {
            const int s = i % kStages3, a = i & 1;
            if (!mbar_wait(smem_u32(&S.acc_full[a]), (i >> 1) & 1, abort_flag, d_err)) break;
            tc_fence_after();
            const uint32_t sb = sB0 + (uint32_t)(s * kB3);
            const uint64_t tb = col_base(t * kNT3, G);
#pragma unroll 1
            for (int cc = 0; cc < 4; ++cc) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 2 * kNT3 + hh * kNT3 + cc * 32), v);
                // v[2u + f] = row product for amplitude 64 hh + 16 cc + u, component f. Of each
                // four amplitudes 4g .. 4g+3 the Re lane finishes the first two, the Im lane
                // the last two; each sends the partner the four products it needs.
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    float r[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        r[k] = __shfl_xor_sync(0xffffffffu, e ? v[8 * g + k] : v[8 * g + 4 + k], 16);
                    float4 o;
                    if (e == 0) {
                        o = make_float4(v[8 * g] - r[1], v[8 * g + 1] + r[0], v[8 * g + 2] - r[3], v[8 * g + 3] + r[2]);
                    } else {
                        o = make_float4(r[0] - v[8 * g + 5], r[1] + v[8 * g + 4], r[2] - v[8 * g + 7],
                                        r[3] + v[8 * g + 6]);
                    }
                    if constexpr (T0) {
                        // back to memory order: member rows j, j ^ 1 (lanes lane, lane ^ 1)
                        // trade halves, so the even row holds members (j, j + 1) of column 2c
                        // and the odd row those of column 2c + 1
                        const bool even = (lane & 1) == 0;
                        const float s0 = __shfl_xor_sync(0xffffffffu, even ? o.z : o.x, 1);
                        const float s1 = __shfl_xor_sync(0xffffffffu, even ? o.w : o.y, 1);
                        o = even ? make_float4(o.x, o.y, s0, s1) : make_float4(s0, s1, o.z, o.w);
                    }
                    // amplitude pair c of the tile, staged as one 16-byte chunk (conflict free:
                    // the 16 rows of an instruction fall in four 32-byte bank groups)
                    const int c = 32 * hh + 8 * cc + 2 * g + e;
                    asm volatile("st.shared.v4.f32 [%0], {%1,%2,%3,%4};" ::"r"(sb + mn_chunk(j, c)), "f"(o.x),
                                 "f"(o.y), "f"(o.z), "f"(o.w)
                                 : "memory");
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&S.acc_empty[a]));
            __syncwarp();
            // store: chunk r of this lane is wsm ^ sr_sm[r] of the stage, in address order
            // across the lanes (runs as long as the target positions allow)
#pragma unroll 4
            for (int r = 0; r < 16; ++r) {
                float4 o;
                if constexpr (TABLE) {
                    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                                 : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
                                 : "r"(sb + (wsm ^ R.sr_sm[r])));
                    if ((uint64_t)(wcol | R.sr_col[r]) < G.n_cols)
                        *reinterpret_cast<float4 *>(sv + (tb | wa | R.sr_addr[r])) = o;
                } else {
                    const int l = IL ? 16 * q + 2 * (r >> 1) + lb : 16 * q + r;
                    const int c = IL ? 32 * hh + 16 * (r & 1) + pl : cst;
                    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                                 : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
                                 : "r"(sb + mn_chunk(l, c)));
                    if constexpr (IL) {
                        if ((uint64_t)(2 * c) < G.n_cols)
                            *reinterpret_cast<float4 *>(sv + (tb | (r & 1 ? pst1 : pst0) | G.off[l])) = o;
                    } else {
                        if (okst) *reinterpret_cast<float4 *>(sv + (tb | pst | G.off[l])) = o;
                    }
                }
            }
            mbar_arrive(smem_u32(&S.empty[s]));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp3)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols3) : "memory");
}

// Diagnostic of the bounded wait: one thread waits on an mbarrier whose phase
// never completes (nothing arrives), with a budget of `cycles` clock ticks, so
// the wait must give up and record kErrTimeout in the status word.
__global__ void k_wait_probe(int *d_err, long long cycles) {
    __shared__ unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    abort_flag = 0;
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(smem_u32(&bar), 0, &abort_flag, d_err, cycles);
}

// ---------------- host: operand image of A ----------------
uint32_t host_tf32(float x) {
    // round to nearest (ties away from zero) to a 10-bit mantissa, as cvt.rna.tf32.f32
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u & 0xffffe000u;
    u += 0x1000u;
    return u & 0xffffe000u;
}

uint16_t host_bf16(float x) {
    // round to nearest even
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

float bf16_to_float(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

size_t host_sw128(int kb, int r, int chunk) {
    return (size_t)kb * (128 * 128) + (size_t)(r >> 3) * 1024 + (size_t)(r & 7) * 128 + (size_t)((chunk ^ (r & 7)) << 4);
}

// A[2j+e][2l+f] from G (64x64 complex, row-major, interleaved doubles)
double a_real(const double *g, int m, int k) {
    const int j = m >> 1, e = m & 1, l = k >> 1, f = k & 1;
    const double re = g[2 * (j * 64 + l)], im = g[2 * (j * 64 + l) + 1];
    if (e == 0) return f == 0 ? re : -im;
    return f == 0 ? im : re;
}

std::vector<unsigned char> build_a_image(const double *g, sv_precision_t prec) {
    std::vector<unsigned char> img(kAImg, 0);
    for (int m = 0; m < 128; ++m)
        for (int k = 0; k < 128; ++k) {
            const float x = (float)a_real(g, m, k);
            if (prec == SV_PREC_TF32) {
                const uint32_t w = host_tf32(x);
                std::memcpy(&img[host_sw128(k >> 5, m, (k & 31) >> 2) + (k & 3) * 4], &w, 4);
            } else {
                const uint16_t hi = host_bf16(x);
                const uint16_t lo = host_bf16(x - bf16_to_float(hi));
                const size_t o = host_sw128(k >> 6, m, (k & 63) >> 3) + (k & 7) * 2;
                std::memcpy(&img[o], &hi, 2);
                std::memcpy(&img[kAImg / 2 + o], &lo, 2);
            }
        }
    return img;
}

// A image of the raw-operand variant: row m = 32q + r holds Re G[16q + r % 16][.]
// (r < 16) or Im G[16q + r % 16][.] (r >= 16). TF32: K = 64 members in two
// 128-byte K-blocks. Split BF16: hi and lo images (16 KB each) of one 128-byte
// K-block each.
std::vector<unsigned char> build_a_image3(const double *g, sv_precision_t prec) {
    std::vector<unsigned char> img(kA3, 0);
    for (int m = 0; m < 128; ++m) {
        const int j = 16 * (m >> 5) + (m & 15), part = (m >> 4) & 1;
        for (int k = 0; k < 64; ++k) {
            const float x = (float)g[2 * (j * 64 + k) + part];
            if (prec == SV_PREC_TF32) {
                const uint32_t w = host_tf32(x);
                std::memcpy(&img[host_sw128(k >> 5, m, (k & 31) >> 2) + (k & 3) * 4], &w, 4);
            } else {
                const uint16_t hi = host_bf16(x);
                const uint16_t lo = host_bf16(x - bf16_to_float(hi));
                const size_t o = host_sw128(0, m, k >> 3) + (k & 7) * 2;
                std::memcpy(&img[o], &hi, 2);
                std::memcpy(&img[16384 + o], &lo, 2);
            }
        }
    }
    return img;
}

template <int P, int MODE>
cudaError_t run_tc_raw(const LaunchCtx &L, float2 *sv, const TcGeom &G, const RawMap &R, const uint4 *d_a,
                       int *d_err, int lg) {
    cudaError_t e = cudaFuncSetAttribute(k_tc6_raw<P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem3);
    if (e != cudaSuccess) return e;
    uint64_t grid = (uint64_t)L.num_sms;
    if (grid > G.n_tiles) grid = G.n_tiles;
    k_tc6_raw<P, MODE><<<(unsigned)grid, kThreads3, kSmem3, L.stream>>>(sv, G, R, d_a, d_err, lg);
    ++*L.launches;
    return cudaGetLastError();
}

// operand byte offset of row l, amplitude pair c in a stage (the host twin of mn_chunk)
uint32_t host_mn_chunk(int l, int c) {
    return (uint32_t)((c >> 3) * 8192 + (l >> 3) * 1024 + (l & 7) * 128 + ((((c & 7) >> 1) ^ (l & 3)) << 5) +
                      ((c & 1) << 4));
}

// The address-ordered chunk mapping of the raw-operand kernel for targets tpos on
// an n-qubit state (see RawMap). Each index bit of a chunk has an amplitude
// address bit, an operand offset and a column contribution; the bits are sorted
// by address bit and dealt out to lanes first.
RawMap build_raw_map(int n, const int *tpos, bool t0) {
    std::vector<int> npos;                       // non-target positions, ascending; past n for tiny states
    for (int q = 0, t = 0; (int)npos.size() < 8; ++q) {
        if (t < 6 && q == tpos[t]) {
            ++t;
            continue;
        }
        npos.push_back(q);
    }
    struct Bit { int apos; uint64_t addr; uint32_t sm; uint32_t col; };
    auto member_bit = [&](int i) {      // member index bit i (row bit i with qubit 0 free)
        return Bit{tpos[i], 1ull << tpos[i], host_mn_chunk(1 << i, 0), 0u};
    };
    std::vector<Bit> copy, store;
    if (!t0) {
        for (int i = 0; i < 6; ++i)     // pair bit i: column bit i + 1
            copy.push_back(Bit{npos[i + 1], 1ull << npos[i + 1], host_mn_chunk(0, 1 << i), 2u << i});
        for (int i = 0; i < 6; ++i) copy.push_back(member_bit(i));
        for (int i = 0; i < 5; ++i)
            store.push_back(Bit{npos[i + 1], 1ull << npos[i + 1], host_mn_chunk(0, 1 << i), 2u << i});
        for (int i = 0; i < 4; ++i) store.push_back(member_bit(i));
    } else {
        // member-pair bit i (member bit i + 1, row bit i + 1); column bit 0 selects the
        // row of the pair, column bit i >= 1 is pair bit i - 1
        auto pair_bit = [&](int i) {
            return Bit{tpos[i + 1], 1ull << tpos[i + 1], host_mn_chunk(2 << i, 0), 0u};
        };
        auto col_bit = [&](int i) {
            return Bit{npos[i], 1ull << npos[i], i == 0 ? host_mn_chunk(1, 0) : host_mn_chunk(0, 1 << (i - 1)), 1u << i};
        };
        for (int i = 0; i < 5; ++i) copy.push_back(pair_bit(i));
        for (int i = 0; i < 7; ++i) copy.push_back(col_bit(i));
        for (int i = 0; i < 3; ++i) store.push_back(pair_bit(i));
        for (int i = 0; i < 6; ++i) store.push_back(col_bit(i));
    }
    // Address order, except that lanes 0-2 (the eight lanes of one shared-memory
    // wavefront of 16-byte accesses) take the lowest bits whose operand offsets
    // fall in independent 16-byte bank groups, so that those accesses never
    // conflict; the other bits follow in address order.
    auto order = [](std::vector<Bit> &bits) {
        std::sort(bits.begin(), bits.end(), [](const Bit &a, const Bit &b) { return a.apos < b.apos; });
        std::vector<Bit> out;
        std::vector<char> used(bits.size(), 0);
        uint32_t span = 1;                        // bank groups reachable: bit set of a subspace of GF(2)^3
        for (size_t i = 0; i < bits.size() && out.size() < 3; ++i) {
            const uint32_t g = (bits[i].sm >> 4) & 7u;
            if ((span >> g) & 1u) continue;       // g is 0 or already in the span
            uint32_t next = span;
            for (uint32_t v = 0; v < 8; ++v)
                if ((span >> v) & 1u) next |= 1u << (v ^ g);
            span = next;
            out.push_back(bits[i]);
            used[i] = 1;
        }
        for (size_t i = 0; i < bits.size(); ++i)
            if (!used[i]) out.push_back(bits[i]);
        bits = out;
    };
    if (!t0 && tpos[0] >= 3) {
        // qubits 0-2 free: pair bits across the lanes (each instruction 32 consecutive
        // amplitude pairs of one member), member bits across a thread's copies -- the
        // order that measured fastest there (10.8 ms per 32-qubit block against 11.4
        // in address order); the bits are already in that order
    } else {
        order(copy);
        order(store);
    }
    RawMap R{};
    auto fill = [](const std::vector<Bit> &bits, int first, int count, uint64_t *addr, uint32_t *sm, uint32_t *col) {
        for (int v = 0; v < (1 << count); ++v) {
            uint64_t a = 0;
            uint32_t m = 0, c = 0;
            for (int b = 0; b < count; ++b)
                if ((v >> b) & 1) {
                    a |= bits[first + b].addr;
                    m ^= bits[first + b].sm;
                    c |= bits[first + b].col;
                }
            addr[v] = a;
            sm[v] = m;
            col[v] = c;
        }
    };
    fill(copy, 0, 6, R.cthr_addr, R.cthr_sm, R.cthr_col);
    fill(copy, 6, 6, R.cit_addr, R.cit_sm, R.cit_col);
    fill(store, 0, 5, R.sl_addr, R.sl_sm, R.sl_col);
    fill(store, 5, 4, R.sr_addr, R.sr_sm, R.sr_col);
    (void)n;
    return R;
}

template <int P>
cudaError_t run_tc(const LaunchCtx &L, float2 *sv, const TcGeom &G, const uint4 *d_a, int *d_err) {
    auto kern = k_tc6<P>;
    const int smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    uint64_t grid = (uint64_t)L.num_sms;
    if (grid > G.n_tiles) grid = G.n_tiles;
    kern<<<(unsigned)grid, kThreadsTC, smem, L.stream>>>(sv, G, d_a, d_err);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace

bool tc6_supported(int n, const int *tpos) {
    if (n < 6 || n > SV_MAX_QUBITS) return false;
    for (int i = 0; i < 6; ++i)
        if (tpos[i] < 0 || tpos[i] >= n || (i > 0 && tpos[i] <= tpos[i - 1])) return false;
    return true;
}

cudaError_t launch_tc6(const LaunchCtx &L, void *sv, int n, const int *tpos, const double *mat, sv_precision_t prec,
                       void *d_a, int *d_err) {
    if (!tc6_supported(n, tpos) || (prec != SV_PREC_TF32 && prec != SV_PREC_SPLIT_BF16)) return cudaErrorInvalidValue;
    TcGeom G{};
    for (int i = 0; i < 6; ++i) G.pos[i] = tpos[i];
    for (int j = 0; j < 64; ++j) {
        uint64_t o = 0;
        for (int t = 0; t < 6; ++t)
            if ((j >> t) & 1) o |= 1ull << tpos[t];
        G.off[j] = o;
    }
    G.n_cols = 1ull << (n - 6);
    G.n_tiles = (G.n_cols + kNT - 1) / kNT;
    float2 *s = reinterpret_cast<float2 *>(sv);
    const uint4 *a = reinterpret_cast<const uint4 *>(d_a);
    // Every state of 7 qubits or more (a tile then holds whole amplitude pairs or
    // member pairs): the raw-operand kernel; a 6-qubit state: the register-staged one.
    if (n >= 7) {
        const std::vector<unsigned char> img = build_a_image3(mat, prec);
        cudaError_t e = cudaMemcpyAsync(d_a, img.data(), img.size(), cudaMemcpyHostToDevice, L.stream);
        if (e != cudaSuccess) return e;
        // The copy and store order by target positions (TF32, 32-qubit state, one block):
        // qubit 0 a target -> RawMap order (14.2-16.1 ms, against 15.8-16.7 for the
        // register-staged kernel); lowest target 1 or 2 with a second target below 6
        // -> RawMap order ((1..6) 13.9 ms, (2..7) 11.7, against 16.8 and 13.3 in IL order);
        // otherwise the fixed orders (lowest target 3 or more: 10.4-10.8 ms; the table
        // loop's extra instructions per copy cost the copy warps about 13 % there).
        const bool t0 = tpos[0] == 0;
        const bool mapped = !t0 && tpos[0] <= 2 && tpos[1] < 6;
        const RawMap R = t0 || mapped ? build_raw_map(n, tpos, t0) : RawMap{};
        const bool tf = prec == SV_PREC_TF32;
        if (t0) return tf ? run_tc_raw<TF32, RAW_T0>(L, s, G, R, a, d_err, 0) : run_tc_raw<BF16, RAW_T0>(L, s, G, R, a, d_err, 0);
        if (mapped)
            return tf ? run_tc_raw<TF32, RAW_MAPPED>(L, s, G, R, a, d_err, 0)
                      : run_tc_raw<BF16, RAW_MAPPED>(L, s, G, R, a, d_err, 0);
        if (tpos[0] <= 3) {
            const int lg = tpos[0] - 1;
            return tf ? run_tc_raw<TF32, RAW_IL>(L, s, G, R, a, d_err, lg) : run_tc_raw<BF16, RAW_IL>(L, s, G, R, a, d_err, lg);
        }
        return tf ? run_tc_raw<TF32, RAW_PLAIN>(L, s, G, R, a, d_err, 0) : run_tc_raw<BF16, RAW_PLAIN>(L, s, G, R, a, d_err, 0);
    }
    const std::vector<unsigned char> img = build_a_image(mat, prec);
    cudaError_t e = cudaMemcpyAsync(d_a, img.data(), img.size(), cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) return e;
    // a 6-qubit state (one column): the register-staged kernel
    return prec == SV_PREC_TF32 ? run_tc<TF32>(L, s, G, a, d_err) : run_tc<BF16>(L, s, G, a, d_err);
}

cudaError_t launch_wait_probe(const LaunchCtx &L, int *d_err, long long cycles) {
    k_wait_probe<<<1, 32, 0, L.stream>>>(d_err, cycles);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace svk
