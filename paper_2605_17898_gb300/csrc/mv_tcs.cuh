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
// Work split (tile_walk.cuh): the nb (nb + 1) / 2 tiles of the triangle, numbered row by row within
// column bands of W tiles, are cut into one contiguous range per CTA and band (persistent grid of
// min(SMs, tiles) CTAs, equal tile counts to within one per band). W keeps a band's column-side
// operands within a share of L2, so that every CTA sweeping the same band reuses them; at the
// sizes where they fit L2 whole (N up to about 157000 at t = 32, 262000 at t = 16) there is one
// band. A CTA's range crosses a few tile rows; within one row segment, out_I accumulates in the
// drain warps' registers and is added to HBM when the segment ends, while out_J is added after
// every tile. Both additions are float32 adds onto out, which the V-splitting kernel initialised to
// sigma^2 V: the drain writes the 128 x t block to a swizzled shared-memory tile and one thread
// hands it to the TMA unit as a bulk tensor reduce-add (cp.reduce.async.bulk.tensor), so the
// drain warps release the accumulator after their tensor-memory reads alone. (Outputs whose rows
// are not 16-byte aligned take per-thread red.global.add instead.) The order of the additions
// across CTAs is not fixed, so the result can differ between runs in the last bits.
//
// Two forms of the squared distance, one kernel template (DOT):
//
// Difference form (DOT = false; every kernel and D). CTA: one per SM, 22 warps, ~226 KB shared
// memory, all 512 tensor-memory columns:
//   warps 0-15  generation: each thread computes 2 rows x 16 columns of the tile (two 8-column
//               passes, r^2 from 2D float32 operations on a transposed x_J tile) and stores the
//               hi/lo halves;
//   warp 16     producer: TMA of x_J (transposed, two 64-column boxes) and V_J [hi; lo] per
//               tile into a 2-stage ring, and of V_I once per tile row into a 2-slot buffer;
//   warp 17     tensor-memory allocation and the MMA issuer (16 or 32 MMAs per tile);
//   warps 18-21 drain: tensor memory -> registers -> staging tile -> TMA reduce-add.
// Accumulators: two buffers of [out_I (128 columns) | out_J (128 columns)].
//
// Dot form (DOT = true; RBF, Matern-3/2, Matern-5/2 at any D, when the data's spread allows):
// r^2 = a_i + a_j - 2 u_i . u_j for the box-centred coordinates u, as one 128 x 128 tensor-core Gram
// tile per tile whose float16 hi/lo operand rows also carry the squared norms a (built once per X by
// mv_tc.cu), so the tensor core returns -r^2 and an entry costs the kernel value and the split. CTA: 24 warps:
//   warps 0-15  generation from the Gram tile (one row x 32 columns per thread);
//   warp 16     producer (lane 0: V_J ring and the tile-row slot [V_I | U_I]; lane 1: U_J ring);
//   warp 17     tensor-memory allocation and the out_I MMAs;  warp 22  the out_J MMAs;
//   warp 23     the Gram MMAs (two buffers, issued as soon as the generation has read one);
//   warps 18-21 drain, as above.
// Both instances are launched; a device word (max |u|^2, written by the operand kernel) makes
// exactly one of them work.
// Waits are bounded and abort the CTA as in mv_tc.cuh.
#pragma once

#include <type_traits>

#include "mv_tc.cuh"
#include "tile_walk.cuh"

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
constexpr int kTmemCols = 512;      // 2 accumulator buffers (+ the Gram tile in the dot form)
constexpr int kErrWaitVi = 0x100;
constexpr int kErrWaitGram = 0x200;
// The dot form issues its MMAs from three warps: one thread issues a tcgen05.mma about every 100
// cycles (measured), while the tensor pipe finishes an M = 128, N <= 64, K = 16 product in about
// 50, so a single issuer leaves it half idle; and the Gram tile that the generation warps wait for
// must not queue behind a contraction's issue. Warp 17 issues the out_I products, warp 22 the
// out_J products, warp 23 the Gram tiles.
constexpr int kMmaWarpJ = 22;
constexpr int kGramWarp = 23;
constexpr int kDotThreads = 768;

// Difference form: a 2-stage ring of [entry tile hi | lo | V_J hi; lo | x_J], two V_I slots.
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
    // tensor-memory columns: accumulator buffer stride, out_J block inside a buffer, and the block
    // that K_lo V_hi accumulates into (its own third block here)
    static constexpr int kAccStride = 256;
    static constexpr int kAccJ = 128;
    static constexpr bool kMerged = false;
    static constexpr int kLoCol = 2 * T;
    static constexpr int kAccBufs = 2;
};

// Dot form: the operands that the copies bring in live in rings of their own, so that no copy
// waits on the entry tiles. Two entry buffers [hi | lo], a V_J ring (released by the contraction),
// a U_J ring (the B-role Gram operand, released by the Gram MMA), one tile-row slot [V_I hi; lo |
// U_I], the staging tile. Tensor memory: two accumulator buffers of 128 columns, [out_I | out_J],
// then two 128 x 128 float32 Gram tiles. At t = 32 each direction has 2t = 64 columns: K_lo V_hi
// accumulates into the K_hi V_lo block (both are the small split corrections, summed in float32
// by the tensor pipe instead of by the drain); at t = 16 the three t-column blocks fit in 64.
template <int T, int DP>
struct TcdLayout {
    static constexpr int kA = kTile * kTile * 2;
    static constexpr int kB = T * kTile * 2;
    static constexpr int kKg = 32;                 // Gram operand width (16-bit values per row)
    static constexpr int kU = kTile * kKg * 2;
    static constexpr int kK = 0;                   // entry buffers: 2 x [hi | lo]
    static constexpr int kV = 4 * kA;              // V_J ring: 2 x [hi; lo]
    static constexpr int kUr = kV + 4 * kB;        // U_J ring: 2 slots
    static constexpr int kVi = kUr + 2 * kU;       // tile-row slot: V_I [hi; lo], then U_I
    static constexpr int kStaging = kVi + 2 * kB + kU;
    static constexpr int kBar = kStaging + kTile * T * 4;
    static constexpr int kBytes = kBar + 256 + 1024 + 4096;
    static constexpr int kAccStride = 128;
    static constexpr int kAccJ = 64;
    static constexpr bool kMerged = T == 32;
    static constexpr int kLoCol = kMerged ? T : 2 * T;
    static constexpr int kAccBufs = 2;
    static constexpr int kGramCol = 256;
};

// Instruction descriptor with A read MN-major (bit 15), B K-major, M = 128, N = NCOLS.
template <int NCOLS, int FMT>
__device__ __forceinline__ uint32_t instr_desc_amn() {
    return tc::instr_desc<NCOLS, FMT>() | (1u << 15);
}

struct TcsArgs {
    const float *Xs;         // prescaled x [Np, DP] row-major (x_I rows for the generation threads)
    float *out;              // [N, ldo], holds sigma^2 V on entry
    const int *skip;
    int *err;
    int64_t N, Np, ldo;
    int nb;                  // Np / 128
    int64_t tiles;           // nb (nb + 1) / 2
    int band;                // column-band width of the tile order, in tiles (tile_walk.cuh)
    float log2s2;            // exponent offset of the entries: log2 s^2 (bf16) or 15 (f16)
    const float *col_scale;  // [T] multiplier per column (f16 mode), or nullptr
    int add_mode;            // kAddTma (tm_out is valid), kAddVec4 or kAddScalar
    long long budget;
    // Distance form. gate (device word, float bits) holds the largest squared norm of the centred
    // prescaled rows; with gate set, the dot-form kernel runs only when *gate <= gate_lim and the
    // difference-form kernel only otherwise (both are launched; the other returns at once).
    const unsigned int *gate;
    float gate_lim;
    int dot;                 // host side: launch the dot-form instance
    const float *arow;       // dot form: a_i, the squared norm of centred row i, [Np]
    const uint8_t *ua;       // dot form: A-role Gram operand, kU bytes per 128-row tile
    const uint8_t *ub;       // dot form: B-role Gram operand
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
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing on bar
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
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

// Entries from the dot-form Gram value g = -|u_i - u_j|^2 (tensor memory; the operand rows carry both
// squared norms, mv_tc.cu): RBF k = 2^(g + ls2). The Matern forms take |g| as the squared distance:
// near r = 0, where rounding can make g slightly positive, their entries are smooth in r^2
// (k = s^2 (1 - rh^2 / 6 + ...) for Matern-5/2, s^2 (1 - rh^2 / 2 + ...) for Matern-3/2), so |g| and a
// clamp give the same entry up to that rounding; measured, the absolute value makes the Matern-5/2
// product 3% faster than a clamp. (The Matern forms are those of Entry2 in mv_tc.cuh.)
template <int KIND> struct DotEntry2;
template <> struct DotEntry2<LGP_RBF> {
    static __device__ __forceinline__ float2 k(float2 g, float ls2) {
        const float2 arg = __fadd2_rn(g, make_float2(ls2, ls2));
        return make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
    }
};
template <> struct DotEntry2<LGP_MATERN52> {
    // k = e + e (rh + rh^2 / 3), e = 2^(ls2 - rh log2 e), rh = sqrt|g|; rh^2 / 3 taken as -g / 3, which
    // needs no absolute value (a rounding-positive g near r = 0 only perturbs q by that rounding)
    static __device__ __forceinline__ float2 k(float2 g, float ls2) {
        const float2 rh = make_float2(sqrt_approx(fabsf(g.x)), sqrt_approx(fabsf(g.y)));
        const float2 arg = __ffma2_rn(rh, make_float2(-kLog2e, -kLog2e), make_float2(ls2, ls2));
        const float2 e = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
        const float2 q = __ffma2_rn(g, make_float2(-1.0f / 3.0f, -1.0f / 3.0f), rh);
        return __ffma2_rn(e, q, e);
    }
};
template <> struct DotEntry2<LGP_MATERN32> {
    static __device__ __forceinline__ float2 k(float2 g, float ls2) {
        return tc::Entry2<LGP_MATERN32>::k(make_float2(fabsf(g.x), fabsf(g.y)), make_float2(ls2, ls2));
    }
};
// Matern-1/2 has no dot form (its entries are not smooth in r^2 at 0); this stub is never launched.
template <> struct DotEntry2<LGP_MATERN12> {
    static __device__ __forceinline__ float2 k(float2 g, float ls2) { (void)ls2; return g; }
};

// hi/lo split of two entries for the MMA, lo = k - hi (exact in float32), then both packed.
// float16: hi = k with its float32 significand cut to 11 bits by clearing the low bits, so that
//   |lo| < one unit of hi's last place. Cutting instead of rounding costs one bit of lo's range (hi + lo
//   keeps 21 significant bits, against 22) and takes the split off the FMA pipe: two bitwise ANDs and
//   one subtraction per pair. (Measured against the rounding split below: 1% faster on Matern-5/2, 4%
//   on the RBF product, the same product error.) Entries below float16's normal range keep an absolute
//   error below 2^-40 s^2, as with rounding.
// bfloat16, whose 16-bit budget has no bit to spare: hi = k rounded to 8 bits by Veltkamp's splitting
//   (t = 65537 k, hi = t - (t - k)). Entries stay below 2^16 in magnitude, so t cannot overflow.
template <int FMT>
__device__ __forceinline__ void split_pair(float2 k, uint32_t &h, uint32_t &l) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    float2 hi;
    if constexpr (FMT == kFmtF16) {
        hi = make_float2(__uint_as_float(__float_as_uint(k.x) & 0xFFFFE000u),
                         __uint_as_float(__float_as_uint(k.y) & 0xFFFFE000u));
    } else {
        const float2 t = __fmul2_rn(k, make_float2(65537.0f, 65537.0f));
        const float2 u = __ffma2_rn(k, m1, t);  // t - k
        hi = __ffma2_rn(u, m1, t);              // t - (t - k)
    }
    const float2 lo = __ffma2_rn(hi, m1, k);
    h = tc::pack2<FMT>(hi.x, hi.y);
    l = tc::pack2<FMT>(lo.x, lo.y);
}

// The dot form's MMA-issue loops over K steps stay rolled (#pragma unroll 1): one issue costs ~100
// cycles whatever the loop overhead, and the unrolled issue code competes for the instruction cache
// with the generation warps (measured: the dot-form product is ~25% faster rolled). The difference
// form's single issuer runs both directions and stays unrolled (rolled, it measured ~6% slower).
// The dot form's three issuers poll their barriers without a back-off sleep (measured ~0.5% faster
// than a 32 ns sleep between polls).
//
// The dot-form generation reads nothing of the tile order. The single-band instance steps its walk
// there all the same: a version without that step (and with the segment flag kept per thread)
// allocated its registers differently and measured 2.99 against 2.94 ms at N = 100000, t = 32. The
// banded instance leaves the step out, which saves it spills.
template <bool STEP, class Walk>
__device__ __forceinline__ void step_unread(Walk &w, const TileOrder &o) {
    if constexpr (STEP) w.next(o);
}

// DOT selects the dot form of the squared distance (D is then 4 or 8, the padded width DP). BANDED
// selects the banded tile order (tile_walk.cuh); the instance without it walks the single-band
// order in fewer registers.
template <int KIND, int D, int T, int FMT, bool DOT = false, bool BANDED = false>
__global__ void __launch_bounds__(DOT ? kDotThreads : kThreads, 1)
    mv_tcs_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_v,
                  const __grid_constant__ CUtensorMap tm_out, const TcsArgs a) {
    constexpr int DP = D <= 4 ? 4 : 8;
    using L = std::conditional_t<DOT, TcdLayout<T, DP>, TcsLayout<T, DP>>;
    extern __shared__ uint8_t smem_raw[];
    if (a.skip && *a.skip) return;
    if (a.gate && (__uint_as_float(*a.gate) <= a.gate_lim) != DOT) return;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L::kBar + 240);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::kBar + 248);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    using Walk = std::conditional_t<BANDED, TileWalk, RowWalk>;
    const TileOrder ord = tile_order(a.nb, BANDED ? a.band : a.nb, (int)blockIdx.x, (int)gridDim.x);
    const int n_it = (int)Walk::count(ord);

    // bars: full[2], ready[2], empty[2], acc_full[2], acc_empty[2], vi_full[2], vi_empty[2], fin
    auto bar_full = [&](int s) { return smem_u32(&bars[s]); };
    auto bar_ready = [&](int s) { return smem_u32(&bars[2 + s]); };
    auto bar_empty = [&](int s) { return smem_u32(&bars[4 + s]); };
    auto bar_acc_full = [&](int b) { return smem_u32(&bars[6 + b]); };
    auto bar_acc_empty = [&](int b) { return smem_u32(&bars[8 + b]); };
    constexpr int NB = L::kAccBufs;  // accumulator buffers (2)
    auto bar_vi_full = [&](int b) { return smem_u32(&bars[10 + b]); };
    auto bar_vi_empty = [&](int b) { return smem_u32(&bars[12 + b]); };
    const uint32_t bar_fin = smem_u32(&bars[14]);
    const uint32_t bar_fin_j = smem_u32(&bars[21]);  // dot form: the out_J issuer's final commit
    const uint32_t bar_fin_g = smem_u32(&bars[22]);  // dot form: the Gram issuer's final commit
    // dot form: generation warps have read Gram buffer b (16 arrivals)
    auto bar_gram_empty = [&](int b) { return smem_u32(&bars[23 + b]); };
    // dot form: the entry buffer / V_J slot, the accumulators and the tile-row slot are released
    // by both MMA issuers
    constexpr uint32_t kIssuers = DOT ? 2 : 1;
    // dot form: Gram tile buffer b in tensor memory written (gram_full), the U_J ring
    auto bar_gram_full = [&](int b) { return smem_u32(&bars[15 + b]); };
    auto bar_u_full = [&](int b) { return smem_u32(&bars[17 + b]); };
    auto bar_u_empty = [&](int b) { return smem_u32(&bars[19 + b]); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_ready(s), kGenWarps);
            mbar_init(bar_empty(s), kIssuers);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_acc_full(b), kIssuers);
            mbar_init(bar_acc_empty(b), 4);
            mbar_init(bar_vi_full(b), 1);
            mbar_init(bar_vi_empty(b), kIssuers);
        }
        mbar_init(bar_fin, 1);
        mbar_init(bar_fin_j, 1);
        mbar_init(bar_fin_g, 1);
        mbar_init(bar_gram_empty(0), kGenWarps);
        mbar_init(bar_gram_empty(1), kGenWarps);
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_gram_full(b), 1);
            mbar_init(bar_u_full(b), 1);
            mbar_init(bar_u_empty(b), 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    // the per-column epilogue factors (float16 halves), read by the drain from shared memory
    float *col_scale = reinterpret_cast<float *>(smem + L::kBar + 256);
    if (a.col_scale && threadIdx.x < T) col_scale[threadIdx.x] = a.col_scale[threadIdx.x];
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

    Walk w;
    w.init(ord);

    if (warp == kProducerWarp) {
        if constexpr (DOT) {
            // -------------------------------------------------------- producer, dot form
            // lane 0: the tile-row slot (V_I, U_I) and the V_J ring, released by the contraction;
            // lane 1: the U_J ring, released by the Gram MMA, so it runs a tile ahead
            if (lane == 0) {
                int last_v[2] = {-1, -1};
                int last_sg = -1;
                int sg = -1;
                for (int it = 0; it < n_it; ++it, w.next(ord)) {
                    if (w.starts_segment(it)) {
                        ++sg;
                        if (sg >= 1 &&
                            !mbar_wait(bar_vi_empty(0), (sg - 1) & 1, a.budget, abort_flag, a.err, kErrWaitVi, 64))
                            break;
                        const uint32_t dst = smem_u32(smem + L::kVi);
                        mbar_arrive_expect_tx(bar_vi_full(0), (uint32_t)(2 * L::kB + L::kU));
                        tma_load_2d(dst, &tm_v, 0, (2 * w.I) * 2 * T, bar_vi_full(0));
                        tma_load_2d(dst + L::kB, &tm_v, 0, (2 * w.I + 1) * 2 * T, bar_vi_full(0));
                        bulk_load(dst + 2 * L::kB, a.ua + (int64_t)w.I * L::kU, (uint32_t)L::kU, bar_vi_full(0));
                        last_sg = sg;
                    }
                    const int s = it & 1;
                    if (it >= 2 &&
                        !mbar_wait(bar_empty(s), ((it >> 1) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitEmpty, 64))
                        break;
                    const uint32_t vdst = smem_u32(smem + L::kV + s * 2 * L::kB);
                    mbar_arrive_expect_tx(bar_full(s), (uint32_t)(2 * L::kB));
                    tma_load_2d(vdst, &tm_v, 0, (2 * w.J) * 2 * T, bar_full(s));
                    tma_load_2d(vdst + L::kB, &tm_v, 0, (2 * w.J + 1) * 2 * T, bar_full(s));
                    last_v[s] = it;
                }
                if (*abort_flag) {
                    volatile int no_abort = 0;
                    for (int s = 0; s < 2; ++s)
                        if (last_v[s] >= 0) mbar_wait(bar_full(s), (last_v[s] >> 1) & 1, kDrainBudget, &no_abort, a.err, 0);
                    if (last_sg >= 0) mbar_wait(bar_vi_full(0), last_sg & 1, kDrainBudget, &no_abort, a.err, 0);
                }
            } else if (lane == 1) {
                int last_u[2] = {-1, -1};
                for (int it = 0; it < n_it; ++it, w.next(ord)) {
                    const int s = it & 1;
                    if (it >= 2 &&
                        !mbar_wait(bar_u_empty(s), ((it >> 1) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitEmpty, 64))
                        break;
                    mbar_arrive_expect_tx(bar_u_full(s), (uint32_t)L::kU);
                    bulk_load(smem_u32(smem + L::kUr + s * L::kU), a.ub + (int64_t)w.J * L::kU, (uint32_t)L::kU,
                              bar_u_full(s));
                    last_u[s] = it;
                }
                if (*abort_flag) {
                    volatile int no_abort = 0;
                    for (int s = 0; s < 2; ++s)
                        if (last_u[s] >= 0) mbar_wait(bar_u_full(s), (last_u[s] >> 1) & 1, kDrainBudget, &no_abort, a.err, 0);
                }
            }
        } else {
            // ------------------------------------------------------------ producer (TMA)
            if (lane == 0) {
                int last_it[kStages] = {-1, -1};
                int last_sg[2] = {-1, -1};
                int sg = -1;
                for (int it = 0; it < n_it; ++it, w.next(ord)) {
                    if (w.starts_segment(it)) {
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
        }
    } else if (warp == kMmaWarp) {
        if constexpr (DOT) {
            // -------------------------------------------------------- MMA issuer (out_I), dot form
            if (lane == 0) {
                const uint32_t idesc2 = tc::instr_desc<2 * T, FMT>();  // K_hi x [V_hi V_lo]
                const uint32_t idesc1 = tc::instr_desc<T, FMT>();      // K_lo x V_hi
                // K_lo V_hi starts its own block (first K step) or adds onto K_hi V_lo (merged)
                const uint32_t lo_first = L::kMerged ? 1u : 0u;
                bool issued = false;
                for (int it = 0; it < n_it; ++it) {
                    const int s = it & 1;
                    const int buf = it % NB;
                    if (it >= NB &&
                        !mbar_wait(bar_acc_empty(buf), ((it / NB) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitAcc))
                        break;
                    if (!mbar_wait(bar_full(s), (it >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitFull)) break;
                    if (!mbar_wait(bar_ready(s), (it >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitReady)) break;
                    tc_fence_after();
                    const uint32_t acc_i = tmem_acc + (uint32_t)(buf * L::kAccStride);
                    const uint32_t ka = smem_u32(smem + L::kK + s * 2 * L::kA);
                    const uint32_t b_vj = smem_u32(smem + L::kV + s * 2 * L::kB);
                    // descriptors as in the difference form (entry buffer ka in place of the stage)
#pragma unroll 1
                    for (int ks = 0; ks < kTile / 16; ++ks) {
                        const uint32_t first = ks == 0 ? 0u : 1u;
                        const uint64_t dbv = smem_desc(b_vj + ks * 2 * (2 * T) * 16, 2 * T * 16, 128);
                        mma_ss(acc_i, smem_desc(ka + ks * 4096, 2048, 128), dbv, idesc2, first);
                        mma_ss(acc_i + L::kLoCol, smem_desc(ka + L::kA + ks * 4096, 2048, 128), dbv, idesc1,
                               first | lo_first);
                    }
                    mma_commit(bar_empty(s));  // V_J slot and entry buffer s (with the out_J issuer)
                    mma_commit(bar_acc_full(buf));
                    issued = true;
                }
                if (issued) {
                    // every MMA this thread issued has completed before the CTA frees tensor memory
                    mma_commit(bar_fin);
                    volatile int no_abort = 0;
                    mbar_wait(bar_fin, 0, kDrainBudget, &no_abort, a.err, 0);
                }
            }
        } else {
            // ------------------------------------------------------------ MMA issuer
            if (lane == 0) {
                const uint32_t idesc2 = tc::instr_desc<2 * T, FMT>();  // K_hi x [V_hi V_lo]
                const uint32_t idesc1 = tc::instr_desc<T, FMT>();      // K_lo x V_hi
                const uint32_t idesc2t = instr_desc_amn<2 * T, FMT>();
                const uint32_t idesc1t = instr_desc_amn<T, FMT>();
                bool issued = false;
                int sg = -1;
                for (int it = 0; it < n_it; ++it) {
                    const bool seg_first = w.starts_segment(it);
                    const bool diag = w.J == w.I;
                    const int I = w.I;
                    w.next(ord);
                    const bool seg_last = it == n_it - 1 || w.segment_changed(I);
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
        }
    } else if (warp < kGenWarps) {
        if constexpr (DOT) {
            // ------------------------------------------------------------ generation, dot form (warps 0-15)
            // Warp w reads tensor-memory lanes 32 (w % 4) .. +31 (its rows i of the tile) and Gram
            // columns 32 (w / 4) .. +31 (j): 32 entries per thread.
            const int q = warp & 3, cb = warp >> 2;
            const int rloc = 32 * q + lane;
            const uint32_t taddr = tmem_acc + ((uint32_t)(32 * q) << 16) + (uint32_t)(L::kGramCol + 32 * cb);
            const float ls2 = a.log2s2;
            for (int it = 0; it < n_it; ++it, step_unread<!BANDED>(w, ord)) {
                // Gram tile it (buffer it & 1), and entry buffer it & 1 released by both issuers'
                // products of tile it - 2
                bool got = mbar_wait(bar_gram_full(it & 1), (it >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitGram);
                if (it >= 2 && got)
                    got = mbar_wait(bar_empty(it & 1), ((it >> 1) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitEmpty);
                if (!__all_sync(0xffffffffu, got)) break;
                tc_fence_after();
                uint32_t g[32];
                tmem_ld<32>(taddr + (uint32_t)((it & 1) * kTile), g);
                tmem_wait_ld();
                // the Gram buffer may be rewritten once every generation warp holds its part
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_gram_empty(it & 1));
                const int s = it & 1;
                uint8_t *st = smem + L::kK + s * 2 * L::kA;  // entry buffer s: [hi | lo]
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float2 dv = make_float2(__uint_as_float(g[8 * u + 2 * v]), __uint_as_float(g[8 * u + 2 * v + 1]));
                        split_pair<FMT>(DotEntry2<KIND>::k(dv, ls2), h[v], l[v]);
                    }
                    // columns j = 32 cb + 8 u .. +7 of row rloc: one 16-byte row of core matrix (rg, kg)
                    const int off = ((4 * cb + u) * 16 + (rloc >> 3)) * 128 + (rloc & 7) * 16;
                    *reinterpret_cast<uint4 *>(st + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(st + L::kA + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_ready(s));
            }
        } else {
            // ------------------------------------------------------------ generation (warps 0-15)
            const int kg0 = warp & 7;    // column groups kg0 and kg0 + 8 of every tile
            const int half = warp >> 3;  // rows 64*half .. 64*half + 63
            const float2 m1 = make_float2(-1.0f, -1.0f);
            const float2 ls2 = make_float2(a.log2s2, a.log2s2);
            const float2 acc_init = tc::Entry2<KIND>::acc0(ls2);
            float2 xi2[2][D];
            for (int it = 0; it < n_it; ++it, w.next(ord)) {
                if (w.starts_segment(it)) {
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
        }
    } else if (warp == kMmaWarpJ) {
        if constexpr (DOT) {
            // -------------------------------------------------------- MMA issuer (out_J), dot form
            if (lane == 0) {
                const uint32_t idesc2t = instr_desc_amn<2 * T, FMT>();  // K_hi^T x [V_hi V_lo]
                const uint32_t idesc1t = instr_desc_amn<T, FMT>();      // K_lo^T x V_hi
                const uint32_t lo_first = L::kMerged ? 1u : 0u;
                bool issued = false;
                int sg = -1;
                for (int it = 0; it < n_it; ++it) {
                    const bool seg_first = w.starts_segment(it);
                    const bool diag = w.J == w.I;
                    const int I = w.I;
                    w.next(ord);
                    const bool seg_last = it == n_it - 1 || w.segment_changed(I);
                    if (seg_first) ++sg;
                    const int s = it & 1;
                    const int buf = it % NB;
                    if (it >= NB &&
                        !mbar_wait(bar_acc_empty(buf), ((it / NB) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitAcc))
                        break;
                    if (seg_first && !mbar_wait(bar_vi_full(0), sg & 1, a.budget, abort_flag, a.err, kErrWaitVi)) break;
                    if (!mbar_wait(bar_ready(s), (it >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitReady)) break;
                    tc_fence_after();
                    if (!diag) {
                        const uint32_t acc_j = tmem_acc + (uint32_t)(buf * L::kAccStride + L::kAccJ);
                        const uint32_t ka = smem_u32(smem + L::kK + s * 2 * L::kA);
                        const uint32_t b_vi = smem_u32(smem + L::kVi);
#pragma unroll 1
                        for (int ks = 0; ks < kTile / 16; ++ks) {
                            const uint32_t first = ks == 0 ? 0u : 1u;
                            const uint64_t dbv = smem_desc(b_vi + ks * 2 * (2 * T) * 16, 2 * T * 16, 128);
                            mma_ss(acc_j, smem_desc(ka + ks * 256, 128, 2048), dbv, idesc2t, first);
                            mma_ss(acc_j + L::kLoCol, smem_desc(ka + L::kA + ks * 256, 128, 2048), dbv, idesc1t,
                                   first | lo_first);
                        }
                    }
                    // (a commit with nothing outstanding arrives at once: diagonal tiles)
                    mma_commit(bar_empty(s));
                    mma_commit(bar_acc_full(buf));
                    if (seg_last) mma_commit(bar_vi_empty(0));
                    issued = true;
                }
                if (issued) {
                    mma_commit(bar_fin_j);
                    volatile int no_abort = 0;
                    mbar_wait(bar_fin_j, 0, kDrainBudget, &no_abort, a.err, 0);
                }
            }
        }
    } else if (warp == kGramWarp) {
        if constexpr (DOT) {
            // -------------------------------------------------------- MMA issuer (Gram tiles), dot form
            // Gram tile k into tensor-memory buffer k & 1 (A = the tile-row operand U_I, B = U_J from
            // the ring) as soon as the generation warps have read Gram tile k - 2 out of that buffer.
            if (lane == 0) {
                const uint32_t idg = tc::instr_desc<kTile, kFmtF16>();  // M = N = 128, float16
                bool issued = false;
                int sg = -1;
                for (int k = 0; k < n_it; ++k) {
                    const bool seg_first = w.starts_segment(k);
                    const int I = w.I;
                    w.next(ord);
                    const bool seg_last = k == n_it - 1 || w.segment_changed(I);
                    if (seg_first) ++sg;
                    const int b = k & 1;  // Gram buffer and U_J ring slot
                    if (k >= 2 &&
                        !mbar_wait(bar_gram_empty(b), ((k >> 1) - 1) & 1, a.budget, abort_flag, a.err, kErrWaitGram))
                        break;
                    if (!mbar_wait(bar_u_full(b), (k >> 1) & 1, a.budget, abort_flag, a.err, kErrWaitFull)) break;
                    if (seg_first && !mbar_wait(bar_vi_full(0), sg & 1, a.budget, abort_flag, a.err, kErrWaitVi)) break;
                    tc_fence_after();
                    const uint32_t ua = smem_u32(smem + L::kVi + 2 * L::kB);
                    const uint32_t ub = smem_u32(smem + L::kUr + b * L::kU);
                    const uint32_t dg = tmem_acc + (uint32_t)(L::kGramCol + b * kTile);
#pragma unroll
                    for (int ks = 0; ks < L::kKg / 16; ++ks)
                        mma_ss(dg, smem_desc(ua + ks * 4096, 2048, 128), smem_desc(ub + ks * 4096, 2048, 128), idg,
                               ks == 0 ? 0u : 1u);
                    mma_commit(bar_u_empty(b));
                    mma_commit(bar_gram_full(b));
                    if (seg_last) mma_commit(bar_vi_empty(0));  // U_I of this row
                    issued = true;
                }
                if (issued) {
                    mma_commit(bar_fin_g);
                    volatile int no_abort = 0;
                    mbar_wait(bar_fin_g, 0, kDrainBudget, &no_abort, a.err, 0);
                }
            }
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
            w.next(ord);
            const bool seg_last = it == n_it - 1 || w.segment_changed(I);
            const int buf = it % NB;
            const bool got = mbar_wait(bar_acc_full(buf), (it / NB) & 1, a.budget, abort_flag, a.err, kErrWaitAcc, 128);
            if (!drain_all(got)) break;
            tc_fence_after();
            const uint32_t base = tmem_acc + (uint32_t)(buf * L::kAccStride) + ((uint32_t)(32 * quarter) << 16);
            // blocks of each accumulator: K_hi V_hi at +0, K_hi V_lo at +t, K_lo V_hi at +2t (or, merged,
            // added onto the +t block by the tensor pipe); GW columns of each block per round, one wait
            // per round (16 for two blocks of out_I, else 8: out_J's rounds also hold the staged values)
            constexpr int GW = L::kMerged ? 16 : 8;
            constexpr int GWJ = 8;
#pragma unroll
            for (int g = 0; g < T / GW; ++g) {
                uint32_t v0[GW], v1[GW], v2[GW];
                tmem_ld<GW>(base + (uint32_t)(GW * g), v0);
                tmem_ld<GW>(base + (uint32_t)(T + GW * g), v1);
                if constexpr (!L::kMerged) tmem_ld<GW>(base + (uint32_t)(2 * T + GW * g), v2);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < GW; ++c) {
                    float v = __uint_as_float(v0[c]) + __uint_as_float(v1[c]);
                    if constexpr (!L::kMerged) v += __uint_as_float(v2[c]);
                    sum_i[GW * g + c] += v;
                }
            }
            const bool tma = a.add_mode == kAddTma;
            if (!diag) {
                if (tma) staging_free();
                const int64_t j = (int64_t)J * kTile + row;
#pragma unroll
                for (int g = 0; g < T / GWJ; ++g) {
                    uint32_t v0[GWJ], v1[GWJ], v2[GWJ];
                    tmem_ld<GWJ>(base + L::kAccJ + (uint32_t)(GWJ * g), v0);
                    tmem_ld<GWJ>(base + L::kAccJ + (uint32_t)(T + GWJ * g), v1);
                    if constexpr (!L::kMerged) tmem_ld<GWJ>(base + L::kAccJ + (uint32_t)(2 * T + GWJ * g), v2);
                    tmem_wait_ld();
                    float sj[GWJ];
#pragma unroll
                    for (int c = 0; c < GWJ; ++c) {
                        sj[c] = __uint_as_float(v0[c]) + __uint_as_float(v1[c]);
                        if constexpr (!L::kMerged) sj[c] += __uint_as_float(v2[c]);
                        if (a.col_scale) sj[c] *= col_scale[GWJ * g + c];
                    }
                    if (tma) {
#pragma unroll
                        for (int q = 0; q < GWJ / 4; ++q)
                            *reinterpret_cast<float4 *>(staging + staging_off<T>(row, (GWJ / 4) * g + q)) =
                                make_float4(sj[4 * q], sj[4 * q + 1], sj[4 * q + 2], sj[4 * q + 3]);
                    } else if (j < a.N) {
                        red_row<GWJ>(a.out + j * a.ldo + GWJ * g, sj, nullptr, a.add_mode == kAddVec4);
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
                    for (int c = 0; c < T; ++c) sum_i[c] *= col_scale[c];
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
