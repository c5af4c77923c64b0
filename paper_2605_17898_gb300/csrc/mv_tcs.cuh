// Symmetric split tensor-core product K_y V on tcgen05 (sm_103a), for t in {16, 32}.
//
// K is symmetric, so the upper triangle of 128 x 128 tiles (I <= J) holds every entry. Each
// tile's entries are generated once, split into 16-bit hi/lo halves exactly as in mv_tc.cuh and
// stored to shared memory in the K-major no-swizzle layout; the MMA then reads that one copy
// twice:
//   out_I += K_IJ [V_J]     A = the tile read K-major (M = i, K = j),
//   out_J += K_IJ^T [V_I]   A = the same bytes read MN-major (M = j, K = i), I != J only,
// so each entry costs half the generation work of the row-by-row product. The contraction per
// direction is the same three-product split (K_hi [V_hi V_lo] as one N = 2t MMA, K_lo V_hi as an
// N = t MMA) into float32 accumulators in tensor memory, drained after every tile (K = 128).
//
// Work split: the nb (nb + 1) / 2 tiles of the triangle, numbered row by row, are cut into one
// contiguous range per CTA (persistent grid of min(SMs, tiles) CTAs, equal tile counts to within
// one). A CTA's range crosses a few tile rows; within one row, out_I accumulates in the drain
// warps' registers and is added to HBM when the row ends, while out_J is added after every
// tile. Both additions are float32 adds onto out, which the V-splitting kernel initialised to
// sigma^2 V: the drain writes the 128 x t block to a swizzled shared-memory tile and one thread
// hands it to the TMA unit as a bulk tensor reduce-add (cp.reduce.async.bulk.tensor), so the
// drain warps release the accumulator after their tensor-memory reads alone. (Outputs whose rows
// are not 16-byte aligned take per-thread red.global.add instead.) The order of the additions
// across CTAs is not fixed, so the result can differ between runs in the last bits.
//
// CTA structure (one CTA per SM: 22 warps, ~205 KB shared memory, all 512 tensor-memory columns):
//   warps 0-15  generation: each thread computes 2 rows x 16 columns of the tile (two 8-column
//               passes) and stores the hi/lo halves;
//   warp 16     producer: TMA of x_J (transposed, two 64-column boxes) and V_J [hi; lo] per
//               tile into a 2-stage ring, and of V_I once per tile row into a 2-slot buffer;
//   warp 17     tensor-memory allocation and the MMA issuer (16 or 32 MMAs per tile);
//   warps 18-21 drain: tensor memory -> registers -> staging tile -> TMA reduce-add.
// Accumulators: two buffers of [out_I (128 columns) | out_J (128 columns)].
// Waits are bounded and abort the CTA as in mv_tc.cuh.
#pragma once

#include "mv_tc.cuh"

namespace lgp {
namespace tcs {

using tc::fence_async_smem;
using tc::kDrainBudget;
using tc::kDrainWarp0;
using tc::kErrWaitAcc;
using tc::kErrWaitEmpty;
using tc::kErrWaitFull;
using tc::kErrWaitReady;
using tc::kGenWarps;
using tc::kMmaWarp;
using tc::kProducerWarp;
using tc::kThreads;
using tc::mbar_arrive;
using tc::mbar_arrive_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::mma_ss;
using tc::smem_desc;
using tc::smem_u32;
using tc::tc_fence_after;
using tc::tc_fence_before;
using tc::tma_load_2d;
using tc::tmem_ld;
using tc::tmem_wait_ld;

constexpr int kTile = 128;          // tile rows = tile columns = MMA M
constexpr int kStages = 2;
constexpr int kTmemCols = 512;      // 2 buffers x [out_I 128 | out_J 128]
constexpr int kErrWaitVi = 0x100;

template <int T, int DP>
struct TcsLayout {
    static constexpr int kA = kTile * kTile * 2;  // one 16-bit half of the entry tile
    static constexpr int kB = T * kTile * 2;      // one 16-bit half of a 128-row V tile (stacked: 2 kB)
    static constexpr int kX = kTile * DP * 4;     // x_J, transposed: two [DP][64] boxes
    static constexpr int kStage = 2 * kA + 2 * kB + kX;
    static constexpr int kVi = kStages * kStage;  // V_I slots, 2 x 2 kB
    static constexpr int kStaging = kVi + 2 * 2 * kB;  // 128 x t float32 block for the TMA reduce
    static constexpr int kBar = kStaging + kTile * T * 4;
    static constexpr int kBytes = kBar + 256 + 1024 + 4096;
};

// Instruction descriptor with A read MN-major (bit 15), B K-major, M = 128, N = NCOLS.
template <int NCOLS, int FMT>
__device__ __forceinline__ uint32_t instr_desc_amn() {
    return tc::instr_desc<NCOLS, FMT>() | (1u << 15);
}

// Tile number -> (I, J) in the row-by-row numbering of the upper triangle; first tile of row I
// is I nb - I (I - 1) / 2.
struct TileWalk {
    int nb, I, J;
    __device__ __forceinline__ static int64_t row_start(int64_t I, int64_t nb) { return I * nb - I * (I - 1) / 2; }
    __device__ __forceinline__ void init(int64_t t0, int nb_) {
        nb = nb_;
        int lo = 0, hi = nb - 1;  // largest I with row_start(I) <= t0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_start(mid, nb) <= t0) lo = mid;
            else hi = mid - 1;
        }
        I = lo;
        J = I + (int)(t0 - row_start(I, nb));
    }
    __device__ __forceinline__ void next() {
        if (++J == nb) {
            ++I;
            J = I;
        }
    }
};

struct TcsArgs {
    const float *Xs;         // prescaled x [Np, DP] row-major (x_I rows for the generation threads)
    float *out;              // [N, ldo], holds sigma^2 V on entry
    const int *skip;
    int *err;
    int64_t N, Np, ldo;
    int nb;                  // Np / 128
    int64_t tiles;           // nb (nb + 1) / 2
    float log2s2;            // exponent offset of the entries: log2 s^2 (bf16) or 15 (f16)
    const float *col_scale;  // [T] multiplier per column (f16 mode), or nullptr
    int add_mode;            // kAddTma (tm_out is valid), kAddVec4 or kAddScalar
    long long budget;
};

// How the drain adds its blocks onto out: TMA bulk tensor reduce (out 16-byte aligned with a row
// stride that is a multiple of 16 bytes), red.global.add.v4.f32 (16-byte aligned rows), or one
// red.global.add.f32 per element.
constexpr int kAddTma = 2, kAddVec4 = 1, kAddScalar = 0;

// Byte offset of 16-byte chunk c of row r in the staging tile, in the TMA swizzle pattern of a
// T-float row (T = 32: 128-byte swizzle, chunk ^= r mod 8; T = 16: 64-byte swizzle, chunk ^=
// (r / 2) mod 4), which spreads a warp's 32 rows over all banks.
template <int T>
__device__ __forceinline__ uint32_t staging_off(int r, int c) {
    if constexpr (T == 32) return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
    else return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}

__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap *map, int c0, int c1, uint32_t src) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// barrier 1 among the 4 drain warps
__device__ __forceinline__ void drain_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// barrier 1 among the 4 drain warps that also returns the AND of `v` over them, so that all four
// leave their loop together (none is left waiting at a later barrier)
__device__ __forceinline__ bool drain_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 1, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void red_add4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ void red_add1(float *p, float a) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(a) : "memory");
}

// out[0..n) += s[0..n) * scale[0..n) (scale may be null)
template <int NV>
__device__ __forceinline__ void red_row(float *dst, const float (&s)[NV], const float *scale, int vec4) {
#pragma unroll
    for (int c = 0; c < NV; c += 4) {
        float4 m = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
        if (scale) m = make_float4(scale[c], scale[c + 1], scale[c + 2], scale[c + 3]);
        const float v0 = s[c] * m.x, v1 = s[c + 1] * m.y, v2 = s[c + 2] * m.z, v3 = s[c + 3] * m.w;
        if (vec4) {
            red_add4(dst + c, v0, v1, v2, v3);
        } else {
            red_add1(dst + c, v0);
            red_add1(dst + c + 1, v1);
            red_add1(dst + c + 2, v2);
            red_add1(dst + c + 3, v3);
        }
    }
}

template <int KIND, int D, int T, int FMT>
__global__ void __launch_bounds__(kThreads, 1)
    mv_tcs_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_v,
                  const __grid_constant__ CUtensorMap tm_out, const TcsArgs a) {
    constexpr int DP = D <= 4 ? 4 : 8;
    using L = TcsLayout<T, DP>;
    extern __shared__ uint8_t smem_raw[];
    if (a.skip && *a.skip) return;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L::kBar + 192);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::kBar + 200);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t t0 = (int64_t)blockIdx.x * a.tiles / gridDim.x;
    const int64_t t1 = (int64_t)(blockIdx.x + 1) * a.tiles / gridDim.x;
    const int n_it = (int)(t1 - t0);

    // bars: full[2], ready[2], empty[2], acc_full[2], acc_empty[2], vi_full[2], vi_empty[2], fin
    auto bar_full = [&](int s) { return smem_u32(&bars[s]); };
    auto bar_ready = [&](int s) { return smem_u32(&bars[2 + s]); };
    auto bar_empty = [&](int s) { return smem_u32(&bars[4 + s]); };
    auto bar_acc_full = [&](int b) { return smem_u32(&bars[6 + b]); };
    auto bar_acc_empty = [&](int b) { return smem_u32(&bars[8 + b]); };
    auto bar_vi_full = [&](int b) { return smem_u32(&bars[10 + b]); };
    auto bar_vi_empty = [&](int b) { return smem_u32(&bars[12 + b]); };
    const uint32_t bar_fin = smem_u32(&bars[14]);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_ready(s), kGenWarps);
            mbar_init(bar_empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_acc_full(b), 1);
            mbar_init(bar_acc_empty(b), 4);
            mbar_init(bar_vi_full(b), 1);
            mbar_init(bar_vi_empty(b), 1);
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

    TileWalk w;
    w.init(t0, a.nb);

    if (warp == kProducerWarp) {
        // ------------------------------------------------------------ producer (TMA)
        if (lane == 0) {
            int last_it[kStages] = {-1, -1};
            int last_sg[2] = {-1, -1};
            int sg = -1;
            for (int it = 0; it < n_it; ++it, w.next()) {
                if (it == 0 || w.J == w.I) {
                    // new tile row: V_I [hi; lo] (two 64-row chunks) into slot sg & 1
                    ++sg;
                    const int b = sg & 1;
                    if (sg >= 2 && !mbar_wait(bar_vi_empty(b), ((sg >> 1) - 1) & 1, a.budget, abort_flag, a.err,
                                              kErrWaitVi, 64))
                        break;
                    const uint32_t dst = smem_u32(smem + L::kVi + b * 2 * L::kB);
                    mbar_arrive_expect_tx(bar_vi_full(b), (uint32_t)(2 * L::kB));
                    tma_load_2d(dst, &tm_v, 0, (2 * w.I) * 2 * T, bar_vi_full(b));
                    tma_load_2d(dst + L::kB, &tm_v, 0, (2 * w.I + 1) * 2 * T, bar_vi_full(b));
                    last_sg[b] = sg;
                }
                const int s = it % kStages;
                if (it >= kStages &&
                    !mbar_wait(bar_empty(s), ((it / kStages) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitEmpty, 64))
                    break;
                uint8_t *st = smem + s * L::kStage;
                mbar_arrive_expect_tx(bar_full(s), (uint32_t)(2 * L::kB + L::kX));
                const uint32_t xdst = smem_u32(st + 2 * L::kA + 2 * L::kB);
                tma_load_2d(xdst, &tm_x, w.J * kTile, 0, bar_full(s));
                tma_load_2d(xdst + L::kX / 2, &tm_x, w.J * kTile + 64, 0, bar_full(s));
                const uint32_t vdst = smem_u32(st + 2 * L::kA);
                tma_load_2d(vdst, &tm_v, 0, (2 * w.J) * 2 * T, bar_full(s));
                tma_load_2d(vdst + L::kB, &tm_v, 0, (2 * w.J + 1) * 2 * T, bar_full(s));
                last_it[s] = it;
            }
            if (*abort_flag) {
                // drain the copies this thread issued
                volatile int no_abort = 0;
                for (int s = 0; s < kStages; ++s)
                    if (last_it[s] >= 0)
                        mbar_wait(bar_full(s), (last_it[s] / kStages) & 1, kDrainBudget, &no_abort, a.err, 0);
                for (int b = 0; b < 2; ++b)
                    if (last_sg[b] >= 0)
                        mbar_wait(bar_vi_full(b), (last_sg[b] >> 1) & 1, kDrainBudget, &no_abort, a.err, 0);
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc2 = tc::instr_desc<2 * T, FMT>();  // K_hi x [V_hi V_lo]
            const uint32_t idesc1 = tc::instr_desc<T, FMT>();      // K_lo x V_hi
            const uint32_t idesc2t = instr_desc_amn<2 * T, FMT>();
            const uint32_t idesc1t = instr_desc_amn<T, FMT>();
            bool issued = false;
            int sg = -1;
            for (int it = 0; it < n_it; ++it) {
                const bool seg_first = it == 0 || w.J == w.I;
                const bool diag = w.J == w.I;
                const int I = w.I;
                w.next();
                const bool seg_last = it == n_it - 1 || w.I != I;
                if (seg_first) ++sg;
                const int s = it % kStages;
                const int buf = it & 1;
                if (it >= 2 &&
                    !mbar_wait(bar_acc_empty(buf), ((it >> 1) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitAcc, 32))
                    break;
                if (seg_first &&
                    !mbar_wait(bar_vi_full(sg & 1), (sg >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitVi, 32))
                    break;
                if (!mbar_wait(bar_ready(s), (it / kStages) & 1, a.budget, abort_flag, a.err, kErrWaitReady, 32)) break;
                tc_fence_after();
                const uint32_t acc_i = tmem_acc + (uint32_t)(buf * 256);
                const uint32_t acc_j = acc_i + 128;
                const uint32_t st = smem_u32(smem + s * L::kStage);
                const uint32_t b_vj = st + 2 * L::kA;
                const uint32_t b_vi = smem_u32(smem + L::kVi + (sg & 1) * 2 * L::kB);
                // A core matrix (row group rg of i, column group kg of j) at (kg * 16 + rg) * 128 bytes.
                // K-major read (K = j): step ks covers kg = 2ks, 2ks+1: start + ks * 4096, K-group stride
                // 2048, row-group stride 128. MN-major read (M = j, K = i): step ks covers rg = 2ks, 2ks+1:
                // start + ks * 256, K-group (rg) stride 128, M-group (kg) stride 2048.
                // B (V tile, 128 rows): core matrix (column group cg of the stacked 2t, row group kg) at
                // (kg * 2t/8 + cg) * 128 bytes.
#pragma unroll
                for (int ks = 0; ks < kTile / 16; ++ks) {
                    const uint32_t first = ks == 0 ? 0u : 1u;
                    const uint64_t dbv = smem_desc(b_vj + ks * 2 * (2 * T) * 16, 2 * T * 16, 128);
                    mma_ss(acc_i, smem_desc(st + ks * 4096, 2048, 128), dbv, idesc2, first);
                    mma_ss(acc_i + 2 * T, smem_desc(st + L::kA + ks * 4096, 2048, 128), dbv, idesc1, first);
                }
                if (!diag) {
#pragma unroll
                    for (int ks = 0; ks < kTile / 16; ++ks) {
                        const uint32_t first = ks == 0 ? 0u : 1u;
                        const uint64_t dbv = smem_desc(b_vi + ks * 2 * (2 * T) * 16, 2 * T * 16, 128);
                        mma_ss(acc_j, smem_desc(st + ks * 256, 128, 2048), dbv, idesc2t, first);
                        mma_ss(acc_j + 2 * T, smem_desc(st + L::kA + ks * 256, 128, 2048), dbv, idesc1t, first);
                    }
                }
                mma_commit(bar_empty(s));
                mma_commit(bar_acc_full(buf));
                if (seg_last) mma_commit(bar_vi_empty(sg & 1));
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
        // ------------------------------------------------------------ generation (warps 0-15)
        const int kg0 = warp & 7;    // column groups kg0 and kg0 + 8 of every tile
        const int half = warp >> 3;  // rows 64*half .. 64*half + 63
        const float2 m1 = make_float2(-1.0f, -1.0f);
        const float2 ls2 = make_float2(a.log2s2, a.log2s2);
        const float2 acc_init = tc::Entry2<KIND>::acc0(ls2);
        float2 xi2[2][D];
        for (int it = 0; it < n_it; ++it, w.next()) {
            if (it == 0 || w.J == w.I) {
                // this thread's 2 rows of tile row I, each coordinate duplicated into both halves of
                // a float2 (rows < Np because Np % 128 == 0)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float *xr = a.Xs + ((int64_t)w.I * kTile + 64 * half + 32 * r + lane) * DP;
#pragma unroll
                    for (int d = 0; d < D; ++d) xi2[r][d] = make_float2(xr[d], xr[d]);
                }
            }
            const int s = it % kStages;
            const bool got = mbar_wait(bar_full(s), (it / kStages) & 1, a.budget, abort_flag, a.err, kErrWaitFull);
            if (!__all_sync(0xffffffffu, got)) break;
            uint8_t *st = smem + s * L::kStage;
            // the two 64-column passes: unrolled when D is small (short bodies), kept as a loop for
            // larger D (measured faster, smaller code)
            constexpr int kPassUnroll = D <= 4 ? 2 : 1;
#pragma unroll kPassUnroll
            for (int p = 0; p < 2; ++p) {
                const int kg = kg0 + 8 * p;
                const float *xs = reinterpret_cast<const float *>(st + 2 * L::kA + 2 * L::kB + p * (L::kX / 2));
                float k[2][8];
#pragma unroll
                for (int jh = 0; jh < 2; ++jh) {
                    // columns j = 8*kg + 4*jh + {0,1} (pair 0) and {2,3} (pair 1): the squared
                    // distances of 2 rows x 4 columns accumulate one coordinate at a time
                    float2 r2[2][2];
#pragma unroll
                    for (int r = 0; r < 2; ++r) r2[r][0] = r2[r][1] = acc_init;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const float4 q = *reinterpret_cast<const float4 *>(xs + d * 64 + 8 * kg0 + 4 * jh);
                        const float2 xa = make_float2(q.x, q.y), xb = make_float2(q.z, q.w);
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const float2 da = __ffma2_rn(xa, m1, xi2[r][d]);
                            const float2 db = __ffma2_rn(xb, m1, xi2[r][d]);
                            r2[r][0] = __ffma2_rn(da, da, r2[r][0]);
                            r2[r][1] = __ffma2_rn(db, db, r2[r][1]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
#pragma unroll
                        for (int jp = 0; jp < 2; ++jp) {
                            const float2 kv = tc::Entry2<KIND>::k(r2[r][jp], ls2);
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
                        h[u] = tc::pack2<FMT>(k[r][2 * u], k[r][2 * u + 1]);
                        float h0, h1;
                        tc::unpack2<FMT>(h[u], h0, h1);
                        const float2 lo =
                            __ffma2_rn(make_float2(h0, h1), m1, make_float2(k[r][2 * u], k[r][2 * u + 1]));
                        l[u] = tc::pack2<FMT>(lo.x, lo.y);
                    }
                    const int rg = 8 * half + 4 * r + (lane >> 3);
                    const int off = (kg * 16 + rg) * 128 + (lane & 7) * 16;
                    *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(alo + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_ready(s));
        }
    } else if (warp >= kDrainWarp0) {
        // ------------------------------------------------------------ drain (warps 18-21)
        const int quarter = warp & 3;       // tensor-memory lanes 32*quarter .. +31
        const int row = 32 * quarter + lane;  // this thread's row of the 128-row block
        const bool leader = threadIdx.x == kDrainWarp0 * 32;
        uint8_t *staging = smem + L::kStaging;
        const uint32_t staging_u32 = smem_u32(staging);
        float sum_i[T];
#pragma unroll
        for (int c = 0; c < T; ++c) sum_i[c] = 0.0f;
        // hands the staged block to the TMA unit (tile rows r0 .. r0 + 127 of out; rows >= N are clipped
        // by the tensor map, and a block that starts at or after row N holds only padding rows)
        auto flush_staged = [&](int r0) {
            fence_async_smem();
            drain_bar();
            if (leader && r0 < a.N) {
                tma_reduce_add_2d(&tm_out, 0, r0, staging_u32);
                bulk_commit();
            }
        };
        // the staging tile may be rewritten once the previous reduce has read it
        auto staging_free = [&]() {
            if (leader) bulk_wait_read_all();
            drain_bar();
        };
        for (int it = 0; it < n_it; ++it) {
            const bool diag = w.J == w.I;
            const int I = w.I, J = w.J;
            w.next();
            const bool seg_last = it == n_it - 1 || w.I != I;
            const int buf = it & 1;
            const bool got = mbar_wait(bar_acc_full(buf), (it >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitAcc, 128);
            if (!drain_all(got)) break;
            tc_fence_after();
            const uint32_t base = tmem_acc + (uint32_t)(buf * 256) + ((uint32_t)(32 * quarter) << 16);
            // blocks of each accumulator: K_hi V_hi at +0, K_hi V_lo at +t, K_lo V_hi at +2t; 8 columns
            // of the three blocks per round (three loads, one wait)
#pragma unroll
            for (int g = 0; g < T / 8; ++g) {
                uint32_t v0[8], v1[8], v2[8];
                tmem_ld<8>(base + (uint32_t)(8 * g), v0);
                tmem_ld<8>(base + (uint32_t)(T + 8 * g), v1);
                tmem_ld<8>(base + (uint32_t)(2 * T + 8 * g), v2);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    sum_i[8 * g + c] += (__uint_as_float(v0[c]) + __uint_as_float(v1[c])) + __uint_as_float(v2[c]);
            }
            const bool tma = a.add_mode == kAddTma;
            if (!diag) {
                if (tma) staging_free();
                const int64_t j = (int64_t)J * kTile + row;
#pragma unroll
                for (int g = 0; g < T / 8; ++g) {
                    uint32_t v0[8], v1[8], v2[8];
                    tmem_ld<8>(base + 128 + (uint32_t)(8 * g), v0);
                    tmem_ld<8>(base + 128 + (uint32_t)(T + 8 * g), v1);
                    tmem_ld<8>(base + 128 + (uint32_t)(2 * T + 8 * g), v2);
                    tmem_wait_ld();
                    float sj[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        sj[c] = (__uint_as_float(v0[c]) + __uint_as_float(v1[c])) + __uint_as_float(v2[c]);
                        if (a.col_scale) sj[c] *= a.col_scale[8 * g + c];
                    }
                    if (tma) {
                        *reinterpret_cast<float4 *>(staging + staging_off<T>(row, 2 * g)) =
                            make_float4(sj[0], sj[1], sj[2], sj[3]);
                        *reinterpret_cast<float4 *>(staging + staging_off<T>(row, 2 * g + 1)) =
                            make_float4(sj[4], sj[5], sj[6], sj[7]);
                    } else if (j < a.N) {
                        red_row<8>(a.out + j * a.ldo + 8 * g, sj, nullptr, a.add_mode == kAddVec4);
                    }
                }
            }
            // the accumulator is free once this warp's tensor-memory reads are done
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_acc_empty(buf));
            if (!diag && tma) flush_staged(J * kTile);
            if (seg_last) {
                if (a.col_scale) {
#pragma unroll
                    for (int c = 0; c < T; ++c) sum_i[c] *= a.col_scale[c];
                }
                if (tma) {
                    staging_free();
#pragma unroll
                    for (int c = 0; c < T / 4; ++c)
                        *reinterpret_cast<float4 *>(staging + staging_off<T>(row, c)) =
                            make_float4(sum_i[4 * c], sum_i[4 * c + 1], sum_i[4 * c + 2], sum_i[4 * c + 3]);
                    flush_staged(I * kTile);
                } else {
                    const int64_t i = (int64_t)I * kTile + row;
                    if (i < a.N) red_row<T>(a.out + i * a.ldo, sum_i, nullptr, a.add_mode == kAddVec4);
                }
#pragma unroll
                for (int c = 0; c < T; ++c) sum_i[c] = 0.0f;
            }
        }
        // every reduce this CTA issued has completed before it exits
        if (leader) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_acc), "n"(kTmemCols)
                     : "memory");
    }
}

}  // namespace tcs
}  // namespace lgp
