// Split tensor-core product K_y V on tcgen05 (sm_103a), for t in {16, 32} (kernel template).
//
// Arithmetic. Each kernel entry k (generated in float32 registers, never stored to
// global memory) is split as k = hi + lo with hi = rn(k), lo = rn(k - hi) in a 16-bit
// format; the block V is split the same way once per call. The contraction is
//   out = K_hi V_hi + K_hi V_lo + K_lo V_hi   (float32 accumulation in tensor memory).
// V_hi and V_lo are stacked as one B operand of 2t columns, so K_hi [V_hi V_lo] is a single
// MMA of N = 2t (A read once) and K_lo V_hi a second MMA of N = t over the first half of the
// same B tile; their three t-column results are summed in float32 when the accumulators drain.
// Two formats:
//   kFmtBF16: bfloat16 halves (8 significant bits each, about 16 bits per factor);
//   kFmtF16:  float16 halves (11 bits each, about 22 bits per factor) on values scaled
//             by exact powers of two into float16 range: entries as k * 2^15 / s^2
//             (the exponent offset replaces log2 s^2), each column of V by 2^e_c so that
//             its largest magnitude is at most 2^15; the epilogue multiplies by
//             s^2 2^-15 2^-e_c. Entries below 2^-18 s^2 lose relative precision in their
//             lo half but keep an absolute error below 2^-40 s^2.
//
// CTA structure (one CTA per SM: 22 warps, ~190 KB shared memory):
//   warps 0-15  generate the 128 x 64 entry tile of each column chunk in registers. Two ways
//               to hand it to the MMA, chosen by D at compile time:
//               - A in tensor memory (D <= 4): each thread computes one row x 16 columns and
//                 stores the hi/lo halves with tcgen05.st (lane = row, two 16-bit entries per
//                 32-bit column); the entry tile never touches shared memory;
//               - A in shared memory (D > 4): each thread computes 2 rows x 8 columns, which
//                 halves its x_j loads, and stores the halves in the K-major no-swizzle layout;
//   warp 16     producer: TMA (cp.async.bulk.tensor) of the transposed prescaled x_j tile and
//               of the pre-split V_hi / V_lo tiles into a shared-memory ring;
//   warp 17     allocates tensor memory (two float32 accumulators of 128 lanes x 32 columns,
//               plus the entry stages when A lives there) and one elected thread issues the
//               tcgen05.mma instructions (M=128, N=t, K=16, three per K step) and commits them
//               to the ring's "empty" barriers;
//   warps 18-21 drain: every kGroup chunks the MMA switches accumulator and these warps move
//               the finished one into float32 registers (round-to-nearest adds), so no
//               tensor-core accumulation chain is longer than kGroup * 12 MMAs; they also run
//               the epilogue (registers -> HBM).
// Accumulation chains are kept short because the tensor pipe's float32 accumulation rounds
// less carefully than an IEEE add: measured, its error grew linearly with the chain length
// (1.8e-5 at N=4099, 6.6e-4 at N=500000 for one chain per CTA), and ~1e-6 with drains.
// A CTA owns 128 output rows and a range of 64-column chunks; when the grid splits the
// column range, each CTA writes float32 partial sums that a second kernel reduces in a
// fixed order.
//
// The service warps (producer, MMA, drain) back off with nanosleep while they poll, so the
// generation warps keep the issue slots. Every wait on an mbarrier is bounded by a cycle budget: a wait that runs out records
// an error code in a device word, raises a CTA-wide abort flag, and all roles leave their
// loops; the producer then waits (bounded) for its own copies in flight, the MMA thread
// for its own MMAs, and the TMEM accumulator is freed before the CTA exits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "lgp_internal.cuh"

namespace lgp {

constexpr int kFmtBF16 = 0;
constexpr int kFmtF16 = 1;

namespace tc {

// pipeline depth: 6 stages with A in tensor memory (10 KB of shared memory each), 4 with A in
// shared memory (43 KB each)
template <bool ATMEM> struct Depth { static constexpr int value = 4; };
constexpr int kMaxStages = 6;
constexpr int kBM = 128;          // rows per CTA (MMA M)
constexpr int kBK = 64;           // columns j per chunk (4 MMA K steps)
constexpr int kGenWarps = 16;
constexpr int kProducerWarp = 16;
constexpr int kMmaWarp = 17;
constexpr int kDrainWarp0 = 18;
constexpr int kThreads = 704;     // 16 generation warps + producer + MMA + 4 drain warps
constexpr int kGroup = 2;         // chunks accumulated in tensor memory between drains
constexpr int kAccCols = 128;     // tensor-memory columns per accumulator buffer: [hi*[Vh Vl] (2t) | lo*Vh (t)]
constexpr int kAStageCols = 64;   // tensor-memory columns per entry stage (hi 32 + lo 32)
constexpr int kACol0 = 2 * kAccCols;
template <bool ATMEM> struct TmemCols { static constexpr int value = ATMEM ? 512 : 256; };
constexpr long long kDrainBudget = 2000000000LL;

// error codes written to the device error word on a timeout
constexpr int kErrWaitFull = 0x10, kErrWaitEmpty = 0x20, kErrWaitReady = 0x40, kErrWaitAcc = 0x80;

// Shared-memory stage: [A hi | A lo] (only when A lives in shared memory) [V hi | V lo] [x tile].
template <int T, int DP, bool ATMEM>
struct TcLayout {
    static constexpr int kStages = Depth<ATMEM>::value;
    static constexpr int kA = ATMEM ? 0 : kBM * kBK * 2;  // one 16-bit half of the entry tile
    static constexpr int kB = T * kBK * 2;                // one 16-bit half of the V tile (stacked: 2 kB)
    static constexpr int kX = kBK * DP * 4;               // prescaled x_j tile, transposed: [DP][64] floats
    static constexpr int kStage = 2 * kA + 2 * kB + kX;
    static constexpr int kBar = kStages * kStage;      // barriers after the ring
    // + barriers/flags, alignment slack, and a guard band after the ring so that no
    // descriptor-addressed read of the last stage can leave the CTA's allocation
    static constexpr int kBytes = kBar + 256 + 1024 + 4096;
};

// A from shared memory (descriptor) instead of tensor memory.
__device__ __forceinline__ void mma_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity. Returns false on timeout or abort.
static __device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget, volatile int *abort_flag,
                                              int *err, int code, int sleep_ns = 0) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (sleep_ns) __nanosleep(sleep_ns);
        if (clock64() - t0 > budget) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8 rows x 16 bytes;
// lbo = byte distance between core matrices adjacent along K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, swizzle mode 0 (none)
}

// Instruction descriptor: kind::f16, A = B = bf16 or f16 (K-major), D = f32, M = 128, N = T.
template <int NCOLS, int FMT>
__device__ __forceinline__ uint32_t instr_desc() {
    constexpr uint32_t ab = FMT == kFmtBF16 ? 1u : 0u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(NCOLS >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

// D (tensor memory) += A (tensor memory) x B (shared-memory descriptor); acc = 0 overwrites D.
__device__ __forceinline__ void mma_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Eight 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[N]);

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Round two floats to a packed pair (first in the low half) and read the pair back as floats.
template <int FMT>
__device__ __forceinline__ uint32_t pack2(float first, float second) {
    if (FMT == kFmtBF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(first, second);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(first, second);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

template <int FMT>
__device__ __forceinline__ void unpack2(uint32_t u, float &a, float &b) {
    if (FMT == kFmtBF16) {
        a = __uint_as_float(u << 16);
        b = __uint_as_float(u & 0xFFFF0000u);
    } else {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&u));
        a = f.x;
        b = f.y;
    }
}

// Two kernel entries at once on packed float32x2 arithmetic (same roundings as the scalar
// form in lgp_internal.cuh: FFMA2 performs two independent FFMAs).
template <int KIND> struct Entry2;

// acc0(ls2) is where the squared-distance accumulation starts, k(acc, ls2) turns the accumulated
// value into the entry. RBF folds the outputscale exponent into the accumulation
// (acc = rh2 - log2 s^2, k = 2^-acc); Matern-5/2 needs rh = sqrt(rh2) and uses
// k = e + e * (rh + rh2/3), e = 2^(log2 s^2 - rh log2 e).
template <> struct Entry2<LGP_RBF> {
    static __device__ __forceinline__ float2 acc0(float2 ls2) { return make_float2(-ls2.x, -ls2.y); }
    static __device__ __forceinline__ float2 k(float2 acc, float2 ls2) {
        (void)ls2;
        return make_float2(ex2_approx(-acc.x), ex2_approx(-acc.y));
    }
};

template <> struct Entry2<LGP_MATERN52> {
    static __device__ __forceinline__ float2 acc0(float2 ls2) { (void)ls2; return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ float2 k(float2 rh2, float2 ls2) {
        const float2 rh = make_float2(sqrt_approx(rh2.x), sqrt_approx(rh2.y));
        const float2 arg = __ffma2_rn(rh, make_float2(-kLog2e, -kLog2e), ls2);
        const float2 e = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
        const float2 q = __ffma2_rn(rh2, make_float2(1.0f / 3.0f, 1.0f / 3.0f), rh);
        return __ffma2_rn(e, q, e);
    }
};

// Matern-1/2 on x = log2(e) x / l: k = 2^(log2 s^2 - rh).
template <> struct Entry2<LGP_MATERN12> {
    static __device__ __forceinline__ float2 acc0(float2 ls2) { (void)ls2; return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ float2 k(float2 rh2, float2 ls2) {
        const float2 rh = make_float2(sqrt_approx(rh2.x), sqrt_approx(rh2.y));
        const float2 arg = __ffma2_rn(rh, make_float2(-1.0f, -1.0f), ls2);
        return make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
    }
};

// Matern-3/2 on x = sqrt3 x / l: k = e + e rh, e = 2^(log2 s^2 - rh log2 e).
template <> struct Entry2<LGP_MATERN32> {
    static __device__ __forceinline__ float2 acc0(float2 ls2) { (void)ls2; return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ float2 k(float2 rh2, float2 ls2) {
        const float2 rh = make_float2(sqrt_approx(rh2.x), sqrt_approx(rh2.y));
        const float2 arg = __ffma2_rn(rh, make_float2(-kLog2e, -kLog2e), ls2);
        const float2 e = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
        return __ffma2_rn(e, rh, e);
    }
};

struct TcArgs {
    const float *Xs;     // prescaled x [Np, DP] (row-major; each generation thread reads its own rows)
    const float *V;      // user V [N, ldv] (for the sigma^2 V term)
    float *out;          // [N, ldo] or nullptr in split mode
    float *partial;      // [S, Np, T] in split mode
    const int *skip;
    int *err;
    int64_t N, Np, ldv, ldo;
    int chunks_per_split;
    int total_chunks;
    float log2s2;            // exponent offset of the entries: log2 s^2 (bf16) or 15 (f16)
    float noise;
    const float *col_scale;  // [T] epilogue multiplier per column (f16 mode), or nullptr
    long long budget;
};

template <int KIND, int D, int T, int FMT>
__global__ void __launch_bounds__(kThreads, 1)
    mv_tc_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_v,
                 const TcArgs a) {
    constexpr int DP = D <= 4 ? 4 : 8;
    constexpr bool ATMEM = D <= 4;
    using L = TcLayout<T, DP, ATMEM>;
    constexpr int kStages = L::kStages;
    constexpr int kTmemCols = TmemCols<ATMEM>::value;
    extern __shared__ uint8_t smem_raw[];
    if (a.skip && *a.skip) return;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBar);
    // bars: full[4], ready[4], empty[4], acc_full[2], acc_empty[2], fin
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L::kBar + 192);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::kBar + 200);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * kBM;
    const int c_begin = blockIdx.y * a.chunks_per_split;
    const int c_end = min(a.total_chunks, c_begin + a.chunks_per_split);
    const int n_it = c_end - c_begin;

    auto bar_full = [&](int s) { return smem_u32(&bars[s]); };
    auto bar_ready = [&](int s) { return smem_u32(&bars[kStages + s]); };
    auto bar_empty = [&](int s) { return smem_u32(&bars[2 * kStages + s]); };
    auto bar_acc_full = [&](int b) { return smem_u32(&bars[3 * kStages + b]); };
    auto bar_acc_empty = [&](int b) { return smem_u32(&bars[3 * kStages + 2 + b]); };
    const uint32_t bar_fin = smem_u32(&bars[3 * kStages + 4]);
    const int n_groups = (n_it + kGroup - 1) / kGroup;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_ready(s), kGenWarps);
            mbar_init(bar_empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_acc_full(b), 1);
            mbar_init(bar_acc_empty(b), 4);
        }
        mbar_init(bar_fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_acc = *tmem_slot;

    if (warp == kProducerWarp) {
        // ------------------------------------------------------------ producer (TMA)
        int last_it[kStages];
        for (int s = 0; s < kStages; ++s) last_it[s] = -1;
        if (lane == 0) {
            for (int it = 0; it < n_it; ++it) {
                const int s = it % kStages;
                if (it >= kStages &&
                    !mbar_wait(bar_empty(s), ((it / kStages) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitEmpty, 64))
                    break;
                uint8_t *st = smem + s * L::kStage;
                const int q = c_begin + it;
                mbar_arrive_expect_tx(bar_full(s), (uint32_t)(2 * L::kB + L::kX));
                tma_load_2d(smem_u32(st + 2 * L::kA + 2 * L::kB), &tm_x, q * kBK, 0, bar_full(s));
                tma_load_2d(smem_u32(st + 2 * L::kA), &tm_v, 0, q * 2 * T, bar_full(s));
                last_it[s] = it;
            }
            if (*abort_flag) {
                // drain the copies this thread issued
                for (int s = 0; s < kStages; ++s) {
                    if (last_it[s] < 0) continue;
                    volatile int no_abort = 0;
                    mbar_wait(bar_full(s), (last_it[s] / kStages) & 1, kDrainBudget, &no_abort, a.err, 0);
                }
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc2 = instr_desc<2 * T, FMT>();  // K_hi x [V_hi V_lo]
            const uint32_t idesc1 = instr_desc<T, FMT>();      // K_lo x V_hi
            bool issued = false;
            for (int it = 0; it < n_it; ++it) {
                const int s = it % kStages;
                const int g = it / kGroup;
                const int buf = g & 1;
                const bool group_start = (it % kGroup) == 0;
                const bool group_end = (it % kGroup) == kGroup - 1 || it == n_it - 1;
                // the drain warps must have read this buffer's previous group (g - 2)
                if (group_start && g >= 2 &&
                    !mbar_wait(bar_acc_empty(buf), ((g >> 1) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitAcc, 32))
                    break;
                if (!mbar_wait(bar_ready(s), (it / kStages) & 1, a.budget, abort_flag, a.err, kErrWaitReady, 32)) break;
                tc_fence_after();
                const uint32_t acc = tmem_acc + (uint32_t)(buf * kAccCols);
                const uint32_t st = smem_u32(smem + s * L::kStage);
                const uint32_t b_v = st + 2 * L::kA;  // stacked [V_hi; V_lo]: 2t B rows
                // A in tensor memory: hi at columns [a_col, a_col + 32), lo at +32, K step ks reads 8
                // columns (16 entries) of each. A in shared memory: core matrix (row group rg, k group
                // kg) at (kg * 16 + rg) * 128 bytes.
                const uint32_t a_col = tmem_acc + (uint32_t)(kACol0 + s * kAStageCols);
#pragma unroll
                for (int ks = 0; ks < kBK / 16; ++ks) {
                    // B: core matrix (stacked column group cg in 0..2t/8, k group kg) at
                    // (kg * 2t/8 + cg) * 128 bytes; the first t/8 groups are V_hi
                    const uint64_t dbv = smem_desc(b_v + ks * 2 * (2 * T) * 16, 2 * T * 16, 128);
                    const uint32_t acc_lo = acc + 2 * T;
                    const uint32_t first = (group_start && ks == 0) ? 0u : 1u;
                    if constexpr (ATMEM) {
                        const uint32_t ah = a_col + 8 * ks, al = a_col + 32 + 8 * ks;
                        mma_ts(acc, ah, dbv, idesc2, first);
                        mma_ts(acc_lo, al, dbv, idesc1, first);
                    } else {
                        const uint64_t dah = smem_desc(st + ks * 4096, 2048, 128);
                        const uint64_t dal = smem_desc(st + L::kA + ks * 4096, 2048, 128);
                        mma_ss(acc, dah, dbv, idesc2, first);
                        mma_ss(acc_lo, dal, dbv, idesc1, first);
                    }
                }
                mma_commit(bar_empty(s));
                if (group_end) mma_commit(bar_acc_full(buf));
                issued = true;
            }
            if (issued) {
                // every MMA this thread issued has completed before the CTA frees tensor memory
                mma_commit(bar_fin);
                volatile int no_abort = 0;
                mbar_wait(bar_fin, 0, kDrainBudget, &no_abort, a.err, 0);
            }
        }
    } else if (warp < kGenWarps) {
        if constexpr (ATMEM) {
        // ------------------------------------------------------------ generation (warps 0-15)
        const int quarter = warp & 3;  // tensor-memory lanes (= rows) 32*quarter .. +31
        const int cgrp = warp >> 2;    // columns 16*cgrp .. 16*cgrp + 15 of every chunk
        const float2 m1 = make_float2(-1.0f, -1.0f);
        const float2 ls2 = make_float2(a.log2s2, a.log2s2);
        const float2 acc_init = Entry2<KIND>::acc0(ls2);
        // this thread's row of the prescaled x, each coordinate duplicated into both halves of a
        // float2 (row0 + 127 < Np because Np % 256 == 0)
        float2 xi2[D];
        {
            const float *xr = a.Xs + (row0 + 32 * quarter + lane) * DP;
#pragma unroll
            for (int d = 0; d < D; ++d) xi2[d] = make_float2(xr[d], xr[d]);
        }
        const uint32_t lane_addr = tmem_acc + ((uint32_t)(32 * quarter) << 16);
        for (int it = 0; it < n_it; ++it) {
            const int s = it % kStages;
            const bool got = mbar_wait(bar_full(s), (it / kStages) & 1, a.budget, abort_flag, a.err, kErrWaitFull);
            if (!__all_sync(0xffffffffu, got)) break;
            const float *xs = reinterpret_cast<const float *>(smem + s * L::kStage + 2 * L::kA + 2 * L::kB);  // [DP][64]
            uint32_t h[8], l[8];
#pragma unroll
            for (int jq = 0; jq < 4; ++jq) {
                // columns j = 16*cgrp + 4*jq + {0,1} (pair 0) and {2,3} (pair 1), every coordinate
                float2 xj2[D][2];
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float4 q = *reinterpret_cast<const float4 *>(xs + d * kBK + 16 * cgrp + 4 * jq);
                    xj2[d][0] = make_float2(q.x, q.y);
                    xj2[d][1] = make_float2(q.z, q.w);
                }
#pragma unroll
                for (int jp = 0; jp < 2; ++jp) {
                    float2 dd = __ffma2_rn(xj2[0][jp], m1, xi2[0]);
                    float2 r2 = __ffma2_rn(dd, dd, acc_init);
#pragma unroll
                    for (int d = 1; d < D; ++d) {
                        dd = __ffma2_rn(xj2[d][jp], m1, xi2[d]);
                        r2 = __ffma2_rn(dd, dd, r2);
                    }
                    const float2 kv = Entry2<KIND>::k(r2, ls2);
                    const uint32_t hw = pack2<FMT>(kv.x, kv.y);
                    float h0, h1;
                    unpack2<FMT>(hw, h0, h1);
                    const float2 lo = __ffma2_rn(make_float2(h0, h1), m1, kv);
                    h[2 * jq + jp] = hw;
                    l[2 * jq + jp] = pack2<FMT>(lo.x, lo.y);
                }
            }
            // 16 entries = 8 columns of this row's lane in the stage's hi and lo regions
            const uint32_t col = (uint32_t)(kACol0 + s * kAStageCols + 8 * cgrp);
            tmem_st8(lane_addr + col, h);
            tmem_st8(lane_addr + col + 32, l);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_ready(s));
        }
        } else {
        // ------------------------------------------------------------ generation (warps 0-15)
        const int kg = warp & 7;    // this warp's 8-column group of every chunk
        const int half = warp >> 3; // rows 64*half .. 64*half + 63
        const float2 m1 = make_float2(-1.0f, -1.0f);
        const float2 ls2 = make_float2(a.log2s2, a.log2s2);
        const float2 acc_init = Entry2<KIND>::acc0(ls2);
        // this thread's 2 rows of the prescaled x, each coordinate duplicated into both halves
        // of a float2 (row0 + 127 < Np because Np % 256 == 0)
        float2 xi2[2][D];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float *xr = a.Xs + (row0 + 64 * half + 32 * r + lane) * DP;
#pragma unroll
            for (int d = 0; d < D; ++d) xi2[r][d] = make_float2(xr[d], xr[d]);
        }
        for (int it = 0; it < n_it; ++it) {
            const int s = it % kStages;
            const bool got = mbar_wait(bar_full(s), (it / kStages) & 1, a.budget, abort_flag, a.err, kErrWaitFull);
            if (!__all_sync(0xffffffffu, got)) break;
            uint8_t *st = smem + s * L::kStage;
            const float *xs = reinterpret_cast<const float *>(st + 2 * L::kA + 2 * L::kB);  // [DP][64]
            float k[2][8];
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
                // columns j = 8*kg + 4*jh + {0,1} (pair 0) and {2,3} (pair 1), every coordinate
                float2 xj2[D][2];
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float4 q = *reinterpret_cast<const float4 *>(xs + d * kBK + 8 * kg + 4 * jh);
                    xj2[d][0] = make_float2(q.x, q.y);
                    xj2[d][1] = make_float2(q.z, q.w);
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
#pragma unroll
                    for (int jp = 0; jp < 2; ++jp) {
                        float2 dd = __ffma2_rn(xj2[0][jp], m1, xi2[r][0]);
                        float2 r2 = __ffma2_rn(dd, dd, acc_init);
#pragma unroll
                        for (int d = 1; d < D; ++d) {
                            dd = __ffma2_rn(xj2[d][jp], m1, xi2[r][d]);
                            r2 = __ffma2_rn(dd, dd, r2);
                        }
                        const float2 kv = Entry2<KIND>::k(r2, ls2);
                        k[r][4 * jh + 2 * jp] = kv.x;
                        k[r][4 * jh + 2 * jp + 1] = kv.y;
                    }
                }
            }
            uint8_t *ahi = st;
            uint8_t *alo = st + L::kA;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    h[u] = pack2<FMT>(k[r][2 * u], k[r][2 * u + 1]);
                    float h0, h1;
                    unpack2<FMT>(h[u], h0, h1);
                    const float2 lo = __ffma2_rn(make_float2(h0, h1), m1, make_float2(k[r][2 * u], k[r][2 * u + 1]));
                    l[u] = pack2<FMT>(lo.x, lo.y);
                }
                const int rg = 8 * half + 4 * r + (lane >> 3);
                const int off = (kg * 16 + rg) * 128 + (lane & 7) * 16;
                *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4 *>(alo + off) = make_uint4(l[0], l[1], l[2], l[3]);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_ready(s));
        }
        }
    } else if (warp >= kDrainWarp0) {
        // ------------------------------------------------------------ drain + epilogue (warps 18-21)
        const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
        float sum[T];
#pragma unroll
        for (int c = 0; c < T; ++c) sum[c] = 0.0f;
        bool ok = true;
        for (int g = 0; g < n_groups; ++g) {
            const int buf = g & 1;
            const bool got = mbar_wait(bar_acc_full(buf), (g >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitAcc, 128);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t base = tmem_acc + (uint32_t)(buf * kAccCols) + ((uint32_t)(32 * quarter) << 16);
            // blocks: K_hi V_hi at +0, K_hi V_lo at +t, K_lo V_hi at +2t (one at a time: registers)
#pragma unroll
            for (int blk = 0; blk < 3; ++blk) {
                uint32_t v[T];
                tmem_ld<T>(base + (uint32_t)(blk * T), v);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < T; ++c) sum[c] += __uint_as_float(v[c]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_acc_empty(buf));
        }
        if (ok && !*abort_flag) {
            const int64_t i = row0 + 32 * quarter + lane;
            if (a.col_scale) {
#pragma unroll
                for (int c = 0; c < T; ++c) sum[c] *= a.col_scale[c];
            }
            if (i < a.N) {
                if (a.partial) {
                    float4 *dst = reinterpret_cast<float4 *>(a.partial + ((int64_t)blockIdx.y * a.Np + i) * T);
#pragma unroll
                    for (int c = 0; c < T; c += 4) dst[c / 4] = make_float4(sum[c], sum[c + 1], sum[c + 2], sum[c + 3]);
                } else {
                    const float *vi = a.V + i * a.ldv;
                    float *oi = a.out + i * a.ldo;
#pragma unroll
                    for (int c = 0; c < T; ++c) oi[c] = fmaf(a.noise, vi[c], sum[c]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_acc), "n"(kTmemCols)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace lgp
