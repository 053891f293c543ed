// Small-space projection on the tensor cores (tcgen05, TMA): the dense part of the exact small
// space of the sign function (Sec. 2, Fig. 1) for a batch of right-hand sides,
//
//   C = V^+ X            (N x k, contraction over the 12 V complex numbers of a vector),
//   X_perp = X - V C,    Y_s = V diag(s) C,
//
// with V the N FP32 eigenvectors of Q of one bank and X the k FP32 vectors of a batch.  Both
// products are real GEMMs on the interleaved (re, im) floats:
//   Re C = V . X and Im C = V . (J X), J (a, b) = (b, -a)          (rows of [X; J X] as operand B);
//   X_perp and Y_s from the K = 2N columns (Re V_i, Im V_i) of each complex position against the
//   4k coefficient rows of (-C, s C) arranged for the complex product.
// FP32 accuracy on the TF32 tensor cores by the three-term split a = a_hi + a_lo (a_hi = tf32(a),
// a_lo = tf32(a - a_hi)): a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, relative error ~2^-21 per
// product, FP32 accumulation in tensor memory (TMEM), FP64 sums of the per-CTA partials.
//
// Data path, one warp-specialised block per SM: a producer warp brings raw FP32 tiles of V and X into
// shared memory by TMA (cp.async.bulk.tensor, this GPU's memory, no multicast) through a multi-stage
// mbarrier pipeline; eight warps split each tile into the hi/lo operand tiles (128-byte swizzled,
// K-major: one 128-byte row of 32 floats per matrix row); one thread issues tcgen05.mma (kind::tf32,
// M = 128, cta_group::1) into TMEM accumulators, which the eight warps read back with tcgen05.ld.
// Every wait on a barrier is bounded (about a second); a wait that runs out records the timeout in
// g_tc_timeouts and makes every role of the block stop; the block then waits (bounded) for the copies
// and MMAs it started and frees its TMEM before it returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "ovl_internal.h"

namespace ovl {
namespace {

constexpr int KT = 32;            // floats per K-tile row: one 128-byte swizzle span
constexpr int ROW_BYTES = KT * 4;  // 128
constexpr long long kTcWaitCycles = 2000000000LL;  // about one second at the SM clock

__device__ int g_tc_timeouts;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of bar for at most about a second; false (and the flag set) if it did not complete.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!bar_try_wait(bar, parity))
        if (clock64() - t0 > kTcWaitCycles) {
            atomicExch(&g_tc_timeouts, 1);
            return false;
        }
    return true;
}

// 2-D tiled TMA load of the box at (x, y) (x innermost, in elements) into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// 1-D bulk copy (addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation by one full warp; the base address is written to shared memory at slot.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: K-major operand with the 128-byte swizzle, 128-byte rows, groups of
// 8 rows 1024 bytes apart (stride byte offset); the leading byte offset is unused for this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (16 B; not used with the swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version of tcgen05
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on bar once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// hi = tf32(x), lo = tf32(x - hi) for the four floats of a 16-byte chunk.
__device__ __forceinline__ void split4(float4 v, float4& hi, float4& lo) {
    hi = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
    lo = make_float4(tf32_round(v.x - hi.x), tf32_round(v.y - hi.y), tf32_round(v.z - hi.z), tf32_round(v.w - hi.w));
}

// Columns of the TMEM accumulator: a power of two >= 32 covering n (at most 512, all of TMEM).
__host__ __device__ constexpr uint32_t tmem_cols(int n) {
    return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : n <= 256 ? 256u : 512u;
}

// One arrival on bar (no transaction bytes).
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Wait of one role of a warp-specialised block: phase `parity` of bar, for at most about a second, and
// no longer once another role has given up (abort set).  false: the wait ran out (recorded in
// g_tc_timeouts, abort set) or the block is aborting.
__device__ __forceinline__ bool role_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
    const long long t0 = clock64();
    int spins = 0;
    while (!bar_try_wait(bar, parity)) {
        if ((++spins & 31) == 0 && *abort) return false;
        if (clock64() - t0 > kTcWaitCycles) {
            atomicExch(&g_tc_timeouts, 1);
            *abort = 1;
            return false;
        }
    }
    return true;
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- C = V^+ X: split over the contraction ------------------------------------------------
//
// Grid (nchunk, ceil(na / 128)), 192 threads in three roles that hand tiles over through mbarriers:
//   warp 0   TMA producer: K-tile i of this block (32 floats of every row) into raw stage i % S,
//            V rows [128 my, 128 my + 128) (rows beyond na arrive as zeros) and the KP rows of X;
//   warp 1   MMA issuer (and TMEM owner): D = V [X; J X]^T, M = 128, N = 2 KP, three TF32 products
//            per K-step, into the accumulator set of the tile's group of G K-tiles;
//   warps 2-9  split each raw tile into the hi/lo operand tiles (the 128-byte swizzle keeps every
//            16-byte chunk at its offset, J X too, rows KP..2KP-1), and add each completed group's
//            accumulators into FP32 registers; at the end they write partial[cx][i][j] = (Re, Im).
// Barriers: full[s] (TMA bytes), empty[s] (the eight transform warps), opfull[b] (transform warps),
// opempty[b] (MMA commit), accempty[set] (transform warps, once a group's sums are read).
template <int KP>
struct VdotLayout {
    static constexpr int S = 6;
    static constexpr int RAW_V = 128 * ROW_BYTES;
    static constexpr int RAW_X = KP * ROW_BYTES;
    static constexpr int RAW = RAW_V + RAW_X;
    static constexpr int OPA = 128 * ROW_BYTES;
    static constexpr int OPB = 2 * KP * ROW_BYTES;
    static constexpr int OP = 2 * OPA + 2 * OPB;
    static constexpr int BYTES = S * RAW + 2 * OP + 512 + 1024;  // + barriers and flags + alignment slack
};

// Warp 0 TMA, warp 1 MMA and TMEM, warps 2-9 transform (two warps per scheduler hide each other's
// shared-memory and conversion latency); warps w and w + 4 share TMEM lanes 32 (w % 4) .. and split the
// accumulator columns.
constexpr int WS_THREADS = 320;
constexpr int NXW = 8;                 // transform warps
constexpr int NXT = NXW * 32;          // transform threads

template <int KP>
__global__ void __launch_bounds__(WS_THREADS, 1)
    vdot_tc_k(const __grid_constant__ CUtensorMap tV, const __grid_constant__ CUtensorMap tX, int na, int nb, int ktiles,
              int tpc, double2* __restrict__ partial) {
    using L = VdotLayout<KP>;
    static_assert(KP % 8 == 0 && KP >= 8 && KP <= 32, "KP");
    constexpr int S = L::S, G = 4;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* raw = base;
    unsigned char* op = base + S * L::RAW;
    uint64_t* bars = (uint64_t*)(op + 2 * L::OP);  // full[S], empty[S], opfull[2], opempty[2], accempty[2]
    int* flags = (int*)(bars + 2 * S + 6);        // abort, issued, consumed, committed
    uint32_t* tslot = (uint32_t*)(flags + 4);
    volatile int* abort_flag = flags;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cx = blockIdx.x, row0 = blockIdx.y * 128;
    const int t0 = cx * tpc;
    const int nt = min(tpc, ktiles - t0);
    if (nt <= 0) {  // no K-tiles left for this block: its partial rows are zero
        for (int q = tid; q < 128 * nb; q += WS_THREADS) {
            const int i = row0 + q / nb, j = q % nb;
            if (i < na) partial[((long long)cx * na + i) * nb + j] = make_double2(0.0, 0.0);
        }
        return;
    }
    const uint32_t full0 = su32(bars), empty0 = full0 + 8 * S, opfull0 = empty0 + 8 * S, opempty0 = opfull0 + 16,
                   accempty0 = opempty0 + 16;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(full0 + 8 * s, 1);
            bar_init(empty0 + 8 * s, NXW);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(opfull0 + 8 * b, NXW);
            bar_init(opempty0 + 8 * b, 1);
            bar_init(accempty0 + 8 * b, NXW);
        }
        flags[0] = 0;
        flags[1] = flags[2] = flags[3] = 0;
        bar_fence_init();
    }
    // two accumulator sets (groups alternate), each {hi x hi: 2 KP columns | hi x lo + lo x hi: 2 KP}
    constexpr uint32_t NCOL = tmem_cols(8 * KP);
    if (warp == 1) tmem_alloc(su32(tslot), NCOL);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t IDESC = tf32_idesc(128, 2 * KP);
    if (warp == 0) {
        if (lane == 0) {  // producer
            int i = 0;
            for (; i < nt; ++i) {
                const int s = i % S;
                if (i >= S && !role_wait(empty0 + 8 * s, ((i - S) / S) & 1, abort_flag)) break;
                const uint32_t dst = su32(raw + s * L::RAW), bar = full0 + 8 * s;
                bar_expect_tx(bar, (uint32_t)L::RAW);
                tma_load_2d(dst, &tV, (t0 + i) * KT, row0, bar);
                tma_load_2d(dst + L::RAW_V, &tX, (t0 + i) * KT, 0, bar);
            }
            flags[1] = i;
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int i = 0;
            for (; i < nt; ++i) {
                const int b = i & 1, g = i / G, set = g & 1;
                if (!role_wait(opfull0 + 8 * b, (i >> 1) & 1, abort_flag)) break;
                if (i % G == 0 && g >= 2 && !role_wait(accempty0 + 8 * set, ((g - 2) >> 1) & 1, abort_flag)) break;
                tc_fence_after();
                unsigned char* ob = op + b * L::OP;
                const uint32_t a_hi = su32(ob), a_lo = a_hi + L::OPA, b_hi = a_hi + 2 * L::OPA, b_lo = b_hi + L::OPB;
                const uint32_t big = tmem + set * 4 * KP, small = big + 2 * KP;
#pragma unroll
                for (int ks = 0; ks < KT / 8; ++ks) {
                    const uint32_t o = ks * 32;  // 8 TF32 of K: 32 bytes along the swizzled row
                    const uint32_t more = (i % G > 0 || ks > 0) ? 1u : 0u;
                    mma_tf32(big, sw128_desc(a_hi + o), sw128_desc(b_hi + o), IDESC, more);
                    mma_tf32(small, sw128_desc(a_hi + o), sw128_desc(b_lo + o), IDESC, more);
                    mma_tf32(small, sw128_desc(a_lo + o), sw128_desc(b_hi + o), IDESC, 1u);
                }
                mma_commit(opempty0 + 8 * b);
            }
            flags[3] = i;
        }
    } else {  // warps 2-9: transform and promotion
        const int t = tid - 64;
        // Warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31; of the two warps on a quarter, the first
        // keeps the real parts (columns j), the second the imaginary parts (KP + j).
        const int half = (warp - 2) >> 2;
        const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        float acc[KP];
#pragma unroll
        for (int q = 0; q < KP; ++q) acc[q] = 0.f;
        // The tensor core rounds its accumulation steps toward zero, a bias that grows with the steps
        // summed in one accumulator: each group of G K-tiles has fresh accumulators, added here into
        // FP32 registers with round-to-nearest.
        auto promote = [&](int set) {
#pragma unroll
            for (int c0 = 0; c0 < KP; c0 += 8) {
                float v[8], w[8];
                tmem_ld8(tlane + set * 4 * KP + half * KP + c0, v);
                tmem_ld8(tlane + set * 4 * KP + 2 * KP + half * KP + c0, w);
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[c0 + q] += v[q] + w[q];
            }
        };
        constexpr int XC = KP * ROW_BYTES / 16;  // 16-byte chunks of the X tile
        int promoted = 0, i = 0;
        bool ok = true;
        for (; i < nt; ++i) {
            const int s = i % S, b = i & 1;
            if (!role_wait(full0 + 8 * s, (i / S) & 1, abort_flag)) {
                ok = false;
                break;
            }
            if (i >= 2) {
                if (!role_wait(opempty0 + 8 * b, ((i - 2) >> 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                if ((i - 2) % G == G - 1) {  // tile i - 2 completed its group
                    const int set = ((i - 2) / G) & 1;
                    tc_fence_after();
                    promote(set);
                    ++promoted;
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) bar_arrive(accempty0 + 8 * set);
                }
            }
            const float4* rv = (const float4*)(raw + s * L::RAW);
            const float4* rx = (const float4*)(raw + s * L::RAW + L::RAW_V);
            unsigned char* ob = op + b * L::OP;
            float4* ah = (float4*)ob;
            float4* al = (float4*)(ob + L::OPA);
            float4* bh = (float4*)(ob + 2 * L::OPA);
            float4* bl = (float4*)(ob + 2 * L::OPA + L::OPB);
#pragma unroll 4
            for (int c = t; c < L::RAW_V / 16; c += NXT) {
                float4 h, l;
                split4(rv[c], h, l);
                ah[c] = h;
                al[c] = l;
            }
            for (int c = t; c < XC; c += NXT) {
                const float4 v = rx[c];
                float4 h, l;
                split4(v, h, l);
                bh[c] = h;
                bl[c] = l;
                split4(make_float4(v.y, -v.x, v.w, -v.z), h, l);  // J x: (re, im) -> (im, -re)
                bh[XC + c] = h;
                bl[XC + c] = l;
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                bar_arrive(empty0 + 8 * s);
                bar_arrive(opfull0 + 8 * b);
            }
        }
        if (t == 0) flags[2] = i;
        if (ok && role_wait(opempty0 + 8 * ((nt - 1) & 1), ((nt - 1) >> 1) & 1, abort_flag)) {
            tc_fence_after();
            const int ngroups = (nt + G - 1) / G;  // at most the last two are not added yet
            for (int gi = promoted; gi < ngroups; ++gi) promote(gi & 1);
            const int m = row0 + (warp & 3) * 32 + lane;
            double* pd = (double*)partial;
            if (m < na) {
#pragma unroll
                for (int j = 0; j < KP; ++j)
                    if (j < nb) pd[2 * (((long long)cx * na + m) * nb + j) + half] = (double)acc[j];
            }
        }
    }
    __syncthreads();
    if (*abort_flag && tid == 0) {  // before the block exits: copies and MMAs it started must be done
        for (int i = flags[2]; i < flags[1]; ++i) bar_wait(full0 + 8 * (i % S), (i / S) & 1);
        const int c = flags[3];
        if (c > 0) bar_wait(opempty0 + 8 * ((c - 1) & 1), ((c - 1) >> 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_free(tmem, NCOL);
    }
}

// C[q] = sum over chunks of partial[chunk][q], in chunk order (deterministic).
__global__ void tc_sum_partials_k(const double2* __restrict__ partial, int nchunk, int nq, double2* __restrict__ C) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nchunk; ++k) {
        const double2 v = partial[(long long)k * nq + q];
        re += v.x;
        im += v.y;
    }
    C[q] = make_double2(re, im);
}

// ---- X_perp = X - V C and Y_s = V diag(s) C ----------------------------------------------------
//
// Per output tile of 128 complex positions p (one TMEM lane each) and per K-tile of 16 eigenvectors
// (K = 32: Re V_i, Im V_i), D[p][n] += A[p][q] B[n][q] with A[p][2i + c] = component c of V_i at p and
// the 4 KP coefficient rows of B (n = j: Re of -V C_j; KP + j: Im; 2 KP + j, 3 KP + j: Re and Im of
// V s C_j).  The raw V tile (16 rows of 256 floats, TMA, no swizzle) is transposed by the thread pass
// into the swizzled K-major A rows and split into hi/lo; the coefficient rows come pre-split from
// apply_prep_k as one contiguous image per K-tile (1-D bulk copy into the same stage) and are read
// by the tensor core in place.  A block walks its output tiles (blockIdx.x, + gridDim.x, ...) and all
// their K-tiles as one pipelined sequence of steps; after the last K-tile of a tile the epilogue
// reads the accumulator and writes X_perp and Y_s while the next tiles' copies are in flight.
template <int KP>
struct ApplyLayout {
    static constexpr int S = KP <= 16 ? 5 : (KP <= 24 ? 4 : 3);
    static constexpr int RAW_V = 16 * 256 * 4;        // 16 eigenvectors x 128 complex positions
    static constexpr int BIMG = 2 * 4 * KP * ROW_BYTES;  // hi and lo images of the 4 KP coefficient rows
    static constexpr int RAW = RAW_V + BIMG;
    static constexpr int OPA = 128 * ROW_BYTES;
    static constexpr int OP = 2 * OPA;
    static constexpr int BYTES = S * RAW + 2 * OP + 512 + 1024;
};

// Coefficient images: img[kt][hi, lo][row n < 4 KP][32 floats], rows in the 128-byte swizzled order of
// the operand tile (16-byte chunk c of row n stored at chunk c ^ (n % 8)).
__global__ void apply_prep_k(const double2* __restrict__ C, int ldc, const double* __restrict__ sg, int na, int nb,
                             int KP, int nkt, float4* __restrict__ img) {
    const long long total = (long long)nkt * 4 * KP * 8;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int jc = (int)(idx % 8);
        const int r = (int)((idx / 8) % (4 * KP));
        const int kt = (int)(idx / (8LL * 4 * KP));
        const int g = r / KP, j = r % KP;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = 4 * jc + e, i = 16 * kt + q / 2, c = q & 1;
            double x = 0.0;
            if (i < na && j < nb) {
                const double2 cij = C[(long long)i * ldc + j];
                const double sgn = sg[i];
                if (g == 0) x = c == 0 ? -cij.x : cij.y;                // Re of -V C: -Re C, +Im C
                else if (g == 1) x = c == 0 ? -cij.y : -cij.x;          // Im of -V C
                else if (g == 2) x = c == 0 ? sgn * cij.x : -sgn * cij.y;  // Re of V s C
                else x = c == 0 ? sgn * cij.y : sgn * cij.x;            // Im of V s C
            }
            v[e] = (float)x;
        }
        float4 h, l;
        split4(make_float4(v[0], v[1], v[2], v[3]), h, l);
        const long long at = (long long)kt * (2 * 4 * KP * 8) + (long long)r * 8 + (jc ^ (r & 7));
        img[at] = h;
        img[at + 4 * KP * 8] = l;
    }
}

template <int KP>
__global__ void __launch_bounds__(WS_THREADS, 1)
    apply_tc_k(const __grid_constant__ CUtensorMap tV, const unsigned char* __restrict__ bimg, int nkt,
               const float2* __restrict__ X, float2* __restrict__ Xp, float2* __restrict__ Ys, long long n, int nb,
               int mtiles) {
    // Roles as in vdot_tc_k: warp 0 TMA (the raw V tile and, by a 1-D bulk copy, the K-tile's
    // coefficient image), warp 1 MMA issue and TMEM, warps 2-9 the transposing split of V and the
    // epilogue.  Steps u run over this block's output tiles (blockIdx.x, + gridDim.x, ...) and their
    // K-tiles; the MMAs read the coefficient image in the raw stage, so a stage is released by the MMA
    // commit.  Output tiles alternate between two accumulator sets, each {hi x hi: 4 KP | small: 4 KP};
    // the epilogue of tile q runs after the first K-tile of tile q + 1 has been handed to the MMAs.
    using L = ApplyLayout<KP>;
    static_assert(KP % 8 == 0 && KP >= 8 && KP <= 32, "KP");
    constexpr int S = L::S;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* raw = base;
    unsigned char* op = base + S * L::RAW;
    uint64_t* bars = (uint64_t*)(op + 2 * L::OP);  // full[S], empty[S], opfull[2], opempty[2], accfull[2], accempty[2]
    int* flags = (int*)(bars + 2 * S + 8);        // abort, issued, consumed, committed
    uint32_t* tslot = (uint32_t*)(flags + 4);
    volatile int* abort_flag = flags;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nmt = mtiles > (int)blockIdx.x ? (mtiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const int nsteps = nmt * nkt;
    if (nsteps == 0) return;
    const uint32_t full0 = su32(bars), empty0 = full0 + 8 * S, opfull0 = empty0 + 8 * S, opempty0 = opfull0 + 16,
                   accfull0 = opempty0 + 16, accempty0 = accfull0 + 16;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(full0 + 8 * s, 1);
            bar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(opfull0 + 8 * b, NXW);
            bar_init(opempty0 + 8 * b, 1);
            bar_init(accfull0 + 8 * b, 1);
            bar_init(accempty0 + 8 * b, NXW);
        }
        flags[0] = 0;
        flags[1] = flags[2] = flags[3] = 0;
        bar_fence_init();
    }
    constexpr uint32_t NCOL = tmem_cols(16 * KP);
    if (warp == 1) tmem_alloc(su32(tslot), NCOL);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t IDESC = tf32_idesc(128, 4 * KP);
    if (warp == 0) {
        if (lane == 0) {  // producer
            int u = 0;
            for (; u < nsteps; ++u) {
                const int s = u % S, kt = u % nkt, mt = (int)blockIdx.x + (u / nkt) * (int)gridDim.x;
                if (u >= S && !role_wait(empty0 + 8 * s, ((u - S) / S) & 1, abort_flag)) break;
                const uint32_t dst = su32(raw + s * L::RAW), bar = full0 + 8 * s;
                bar_expect_tx(bar, (uint32_t)L::RAW);
                tma_load_2d(dst, &tV, mt * 256, kt * 16, bar);
                bulk_load(dst + L::RAW_V, bimg + (size_t)kt * L::BIMG, (uint32_t)L::BIMG, bar);
            }
            flags[1] = u;
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int u = 0;
            for (; u < nsteps; ++u) {
                const int s = u % S, b = u & 1, kt = u % nkt, q = u / nkt, ts = q & 1;
                if (!role_wait(opfull0 + 8 * b, (u >> 1) & 1, abort_flag)) break;
                if (kt == 0 && q >= 2 && !role_wait(accempty0 + 8 * ts, ((q - 2) >> 1) & 1, abort_flag)) break;
                tc_fence_after();
                const uint32_t a_hi = su32(op + b * L::OP), a_lo = a_hi + L::OPA;
                const uint32_t b_hi = su32(raw + s * L::RAW + L::RAW_V), b_lo = b_hi + L::BIMG / 2;
                const uint32_t big = tmem + ts * 8 * KP, small = big + 4 * KP;
#pragma unroll
                for (int ks = 0; ks < KT / 8; ++ks) {
                    const uint32_t o = ks * 32;
                    const uint32_t more = (kt > 0 || ks > 0) ? 1u : 0u;
                    mma_tf32(big, sw128_desc(a_hi + o), sw128_desc(b_hi + o), IDESC, more);
                    mma_tf32(small, sw128_desc(a_hi + o), sw128_desc(b_lo + o), IDESC, more);
                    mma_tf32(small, sw128_desc(a_lo + o), sw128_desc(b_hi + o), IDESC, 1u);
                }
                mma_commit(opempty0 + 8 * b);  // the operand buffer is free
                mma_commit(empty0 + 8 * s);    // the raw stage (and its coefficient image) is free
                if (kt == nkt - 1) mma_commit(accfull0 + 8 * ts);
            }
            flags[3] = u;
        }
    } else {  // warps 2-9: transposing split and epilogue
        const int t = tid - 64;
        const int q4 = warp & 3;  // TMEM lanes 32 q4 .. 32 q4 + 31
        const uint32_t tlane = tmem + ((uint32_t)(q4 * 32) << 16);
        auto epilogue = [&](int q) -> bool {  // output tile q of this block
            const int ts = q & 1;
            if (!role_wait(accfull0 + 8 * ts, (q >> 1) & 1, abort_flag)) return false;
            tc_fence_after();
            const int mt = (int)blockIdx.x + q * (int)gridDim.x;
            const long long pos = (long long)mt * 128 + q4 * 32 + lane;
            const uint32_t tl = tlane + ts * 8 * KP;
#pragma unroll 1
            for (int j0 = 8 * ((warp - 2) >> 2); j0 < KP; j0 += 16) {  // the quarter's two warps alternate
                float r1[8], i1[8], r2[8], i2[8], w[8];
                tmem_ld8(tl + j0, r1);
                tmem_ld8(tl + KP + j0, i1);
                tmem_ld8(tl + 2 * KP + j0, r2);
                tmem_ld8(tl + 3 * KP + j0, i2);
                tmem_ld8(tl + 4 * KP + j0, w);
#pragma unroll
                for (int e = 0; e < 8; ++e) r1[e] += w[e];
                tmem_ld8(tl + 5 * KP + j0, w);
#pragma unroll
                for (int e = 0; e < 8; ++e) i1[e] += w[e];
                tmem_ld8(tl + 6 * KP + j0, w);
#pragma unroll
                for (int e = 0; e < 8; ++e) r2[e] += w[e];
                tmem_ld8(tl + 7 * KP + j0, w);
#pragma unroll
                for (int e = 0; e < 8; ++e) i2[e] += w[e];
                if (pos < n) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int j = j0 + e;
                        if (j < nb) {
                            const long long o = (long long)j * n + pos;
                            const float2 x = X[o];
                            Xp[o] = make_float2(x.x + r1[e], x.y + i1[e]);
                            Ys[o] = make_float2(r2[e], i2[e]);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(accempty0 + 8 * ts);
            return true;
        };
        int u = 0;
        bool ok = true;
        for (; u < nsteps && ok; ++u) {
            const int s = u % S, b = u & 1, kt = u % nkt, q = u / nkt;
            if (!role_wait(full0 + 8 * s, (u / S) & 1, abort_flag)) break;
            if (u >= 2 && !role_wait(opempty0 + 8 * b, ((u - 2) >> 1) & 1, abort_flag)) break;
            // thread t builds half a row of A
            const float2* rv = (const float2*)(raw + s * L::RAW);
            float4* ah = (float4*)(op + b * L::OP);
            float4* al = (float4*)(op + b * L::OP + L::OPA);
            const int p = t & 127, jh = (t >> 7) * 4;  // row p, chunks jh .. jh + 3
#pragma unroll
            for (int jc = jh; jc < jh + 4; ++jc) {
                const float2 v0 = rv[(2 * jc) * 128 + p], v1 = rv[(2 * jc + 1) * 128 + p];
                float4 h, l;
                split4(make_float4(v0.x, v0.y, v1.x, v1.y), h, l);
                const int at = p * 8 + (jc ^ (p & 7));
                ah[at] = h;
                al[at] = l;
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) bar_arrive(opfull0 + 8 * b);
            if (kt == 0 && q >= 1) ok = epilogue(q - 1);
        }
        if (t == 0) flags[2] = u;
        if (ok && u == nsteps) epilogue(nmt - 1);
    }
    __syncthreads();
    if (*abort_flag && tid == 0) {  // before the block exits: copies and MMAs it started must be done
        for (int u = flags[2]; u < flags[1]; ++u) bar_wait(full0 + 8 * (u % S), (u / S) & 1);
        const int c = flags[3];
        if (c > 0) bar_wait(opempty0 + 8 * ((c - 1) & 1), ((c - 1) >> 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_free(tmem, NCOL);
    }
}

}  // namespace
}  // namespace ovl

// ---- host side ------------------------------------------------------------------------------

namespace ovl {
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point query (no link to libcuda).
EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D FP32 tensor map over rows of `inner` floats, `outer` rows `stride` bytes apart; elements outside
// the tensor read as zero.
bool map_2d(CUtensorMap* m, const void* base, unsigned long long inner, unsigned long long outer,
            unsigned long long stride, unsigned box_inner, unsigned box_outer, bool swizzle128) {
    EncodeTiledFn f = encode_tiled();
    if (!f) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {stride};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int kTcBlocks = 152;  // one block per SM (the shared-memory footprint allows one)

template <int KP>
cudaError_t vdot_tc(const void* V, int na, const void* X, int nb, long long n, double2* d_C, double2* d_partial,
                    long long partial_cap, cudaStream_t s) {
    using L = VdotLayout<KP>;
    const unsigned long long Lf = 2ULL * n;  // floats per vector
    CUtensorMap tV, tX;
    if (!map_2d(&tV, V, Lf, (unsigned long long)na, Lf * 4, KT, 128, true) ||
        !map_2d(&tX, X, Lf, (unsigned long long)nb, Lf * 4, KT, KP, true))
        return cudaErrorInvalidValue;
    const int ktiles = (int)((Lf + KT - 1) / KT);
    const int mtiles = (na + 127) / 128;
    long long nchunk = std::max(1, kTcBlocks / mtiles);
    const long long cap = partial_cap / ((long long)na * nb);
    if (nchunk > cap) nchunk = std::max(1LL, cap);
    const int tpc = (int)((ktiles + nchunk - 1) / nchunk);
    nchunk = (ktiles + tpc - 1) / tpc;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(vdot_tc_k<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    vdot_tc_k<KP><<<dim3((unsigned)nchunk, mtiles), WS_THREADS, L::BYTES, s>>>(tV, tX, na, nb, ktiles, tpc, d_partial);
    count_launch();
    const int nq = na * nb;
    tc_sum_partials_k<<<(nq + 255) / 256, 256, 0, s>>>(d_partial, (int)nchunk, nq, d_C);
    count_launch();
    return cudaGetLastError();
}

template <int KP>
cudaError_t apply_tc(const void* V, int na, const double* d_signs, const double2* d_C, const void* X, int nb, void* Xp,
                     void* Ys, long long n, void* d_img, cudaStream_t s) {
    using L = ApplyLayout<KP>;
    const unsigned long long Lf = 2ULL * n;
    CUtensorMap tV;
    if (!map_2d(&tV, V, Lf, (unsigned long long)na, Lf * 4, 256, 16, false)) return cudaErrorInvalidValue;
    const int nkt = (na + 15) / 16;
    const long long nimg = (long long)nkt * 4 * KP * 8;
    apply_prep_k<<<(unsigned)std::min<long long>((nimg + 255) / 256, 1024), 256, 0, s>>>(d_C, nb, d_signs, na, nb, KP, nkt,
                                                                                        (float4*)d_img);
    count_launch();
    const int mtiles = (int)((n + 127) / 128);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(apply_tc_k<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    apply_tc_k<KP><<<std::min(mtiles, kTcBlocks), WS_THREADS, L::BYTES, s>>>(
        tV, (const unsigned char*)d_img, nkt, (const float2*)X, (float2*)Xp, (float2*)Ys, n, nb, mtiles);
    count_launch();
    return cudaGetLastError();
}

template <int KP>
cudaError_t project_group(const void* V, int na, const double* d_signs, const void* X, int nb, void* Xp, void* Ys,
                          long long n, double2* d_C, double2* d_partial, long long partial_cap, void* d_img,
                          cudaStream_t s) {
    cudaError_t e = vdot_tc<KP>(V, na, X, nb, n, d_C, d_partial, partial_cap, s);
    if (e != cudaSuccess) return e;
    return apply_tc<KP>(V, na, d_signs, d_C, X, nb, Xp, Ys, n, d_img, s);
}

}  // namespace

size_t tc_project_image_bytes(int na) {
    // coefficient images of the widest group (32 right-hand sides): per K-tile 2 x 4 x 32 rows of 128 B
    return (size_t)((na + 15) / 16) * ApplyLayout<32>::BIMG;
}

bool tc_project_available() { return encode_tiled() != nullptr; }

int take_tc_timeouts() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc_timeouts, &zero, sizeof(int));
    }
    return v;
}

cudaError_t small_space_project_tc(const void* V, int na, const double* d_signs, const void* X, int nb, void* Xp,
                                   void* Ys, long long n, double2* d_C, double2* d_partial, long long partial_cap,
                                   void* d_img, cudaStream_t s) {
    if (na < 1 || na > kTcMaxBank || nb < 1) return cudaErrorInvalidValue;
    const size_t vb = sizeof(float2) * (size_t)n;
    for (int j0 = 0; j0 < nb; j0 += 32) {
        const int nj = std::min(32, nb - j0);
        const char* Xj = (const char*)X + vb * j0;
        char* Pj = (char*)Xp + vb * j0;
        char* Yj = (char*)Ys + vb * j0;
        cudaError_t e;
        if (nj <= 8) e = project_group<8>(V, na, d_signs, Xj, nj, Pj, Yj, n, d_C, d_partial, partial_cap, d_img, s);
        else if (nj <= 16) e = project_group<16>(V, na, d_signs, Xj, nj, Pj, Yj, n, d_C, d_partial, partial_cap, d_img, s);
        else if (nj <= 24) e = project_group<24>(V, na, d_signs, Xj, nj, Pj, Yj, n, d_C, d_partial, partial_cap, d_img, s);
        else e = project_group<32>(V, na, d_signs, Xj, nj, Pj, Yj, n, d_C, d_partial, partial_cap, d_img, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ovl
