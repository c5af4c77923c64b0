// Host side of the split tensor-core product: V splitting, tensor maps, grid shape, launch.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "mv_tc_inst.cuh"
#include "mv_tcs_inst.cuh"

namespace lgp {

namespace {

using tc::kBK;
using tc::kBM;

// Per-column largest |V| as float bits (non-negative floats order like their bit patterns). Thread
// (row r, column c) of a block of 256 (T divides 256) scans rows r, r + rows-per-grid, ...; the block
// reduces its columns in shared memory and adds one atomicMax per column.
__global__ void __launch_bounds__(256) col_absmax_kernel(const float *__restrict__ V, int64_t ldv, int64_t N, int T,
                                                         unsigned int *__restrict__ vmax, const int *skip) {
    if (skip && *skip) return;
    __shared__ unsigned int red[256];
    const int c = threadIdx.x % T;
    unsigned int m = 0;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x / T) + threadIdx.x / T; j < N;
         j += (int64_t)gridDim.x * (blockDim.x / T))
        m = max(m, __float_as_uint(fabsf(V[j * ldv + c])));
    red[threadIdx.x] = m;
    __syncthreads();
    if ((int)threadIdx.x < T) {
        for (int k = threadIdx.x + T; k < (int)blockDim.x; k += T) m = max(m, red[k]);
        atomicMax(vmax + c, m);
    }
}

// Power-of-two exponent e_c with max_c * 2^e_c < 2^15 (clamped to keep the epilogue factor normal).
__device__ __forceinline__ int col_exponent(unsigned int maxbits) {
    const float m = __uint_as_float(maxbits);
    if (!(m > 0.0f) || !isfinite(m)) return 0;
    int ex;
    frexpf(m, &ex);  // m = f * 2^ex, f in [0.5, 1): m < 2^ex
    return min(60, max(-60, 15 - ex));
}

// V -> stacked [V_hi; V_lo] in the tile order the MMA reads: B row c' = c (hi) or t + c (lo);
// element (j, c') of chunk q = j / 64 sits at q*64*2t + ((j%64)/8 * 2t/8 + c'/8) * 64 + (c'%8) * 8 + j%8;
// rows j >= N are zero. One thread per (8-row group, column): its 8 hi and 8 lo values are contiguous
// in that order and go out as one 16-byte store each; the warp's loads of a row are contiguous.
// FMT f16: V is first scaled per column by 2^e_c and col_scale[c] = s^2 2^-15 2^-e_c is written.
// With out_init set, also out_init[j, c] = noise * V[j, c] for j < N (the symmetric product adds
// onto it).
template <int T, int FMT>
__global__ void split_v_kernel(const float *__restrict__ V, int64_t ldv, int64_t N, int64_t Np,
                               uint16_t *__restrict__ vs,
                               const unsigned int *__restrict__ vmax, float *__restrict__ col_scale, float s2,
                               float *__restrict__ out_init, int64_t ldo, float noise, const int *skip) {
    if (skip && *skip) return;
    const int64_t total = (Np / 8) * T;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / T;  // rows 8g .. 8g + 7
        const int c = (int)(e - g * T);
        int ec = 0;
        if (FMT == kFmtF16) {
            ec = col_exponent(vmax[c]);
            if (g == 0) col_scale[c] = ldexpf(s2, -15 - ec);
        }
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t j = 8 * g + k;
            float v = j < N ? V[j * ldv + c] : 0.0f;
            if (out_init && j < N) out_init[j * ldo + c] = noise * v;
            uint16_t h, l;
            if (FMT == kFmtBF16) {
                const __nv_bfloat16 hb = __float2bfloat16_rn(v);
                const __nv_bfloat16 lb = __float2bfloat16_rn(v - __bfloat162float(hb));
                h = *reinterpret_cast<const uint16_t *>(&hb);
                l = *reinterpret_cast<const uint16_t *>(&lb);
            } else {
                v = ldexpf(v, ec);
                const __half hh = __float2half_rn(v);
                const __half lh = __float2half_rn(v - __half2float(hh));
                h = *reinterpret_cast<const uint16_t *>(&hh);
                l = *reinterpret_cast<const uint16_t *>(&lh);
            }
            if (k & 1) {
                hw[k >> 1] |= (uint32_t)h << 16;
                lw[k >> 1] |= (uint32_t)l << 16;
            } else {
                hw[k >> 1] = h;
                lw[k >> 1] = l;
            }
        }
        const int64_t q = (8 * g) / kBK;
        const int jj = (int)(8 * g - q * kBK);  // multiple of 8
        const int64_t chunk = q * kBK * 2 * T + (int64_t)(jj >> 3) * (2 * T / 8) * 64 + (c & 7) * 8;
        *reinterpret_cast<uint4 *>(vs + chunk + (int64_t)(c >> 3) * 64) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(vs + chunk + (int64_t)((T + c) >> 3) * 64) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// XsT[d, j] = Xs[j, d]: the transposed prescaled X the tensor-core product stages by TMA.
__global__ void transpose_x_kernel(const float *__restrict__ Xs, int64_t Np, int dpad, float *__restrict__ XsT,
                                   const int *skip) {
    if (skip && *skip) return;
    const int64_t total = Np * dpad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(e / Np);
        const int64_t j = e - (int64_t)d * Np;
        XsT[e] = Xs[j * dpad + d];
    }
}

// Monotone map of a float onto unsigned integers (and back), so that atomicMax orders floats.
__device__ __forceinline__ unsigned int ord_of(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of_ord(unsigned int o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// Dot-form distance, step 1: bounding box of the prescaled rows i < N. words[d] = ord(max x_d),
// words[8 + d] = ord(max -x_d); the words start at zero (below every ordered float).
__global__ void dot_bbox_kernel(const float *__restrict__ Xs, int64_t N, int dpad, unsigned int *__restrict__ words,
                                const int *skip) {
    if (skip && *skip) return;
    unsigned int hi[8], lo[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) hi[d] = lo[d] = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            if (d < dpad) {
                const float x = Xs[i * dpad + d];
                hi[d] = max(hi[d], ord_of(x));
                lo[d] = max(lo[d], ord_of(-x));
            }
        }
    }
    // warp, then block, then one global atomic per word and block
    __shared__ unsigned int blk[16];
    if (threadIdx.x < 16) blk[threadIdx.x] = 0u;
    __syncthreads();
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const unsigned int h = __reduce_max_sync(0xffffffffu, hi[d]);
        const unsigned int l = __reduce_max_sync(0xffffffffu, lo[d]);
        if ((threadIdx.x & 31) == 0 && d < dpad) {
            atomicMax(blk + d, h);
            atomicMax(blk + 8 + d, l);
        }
    }
    __syncthreads();
    if (threadIdx.x < 16 && (threadIdx.x & 7) < dpad) atomicMax(words + threadIdx.x, blk[threadIdx.x]);
}

// Dot-form distance, step 2: per row j, the centred coordinates u = x - c (c the box centre)
// split as u = h + m (h = f16(u), m = f16(u - h)), the squared norm a_j = sum_d (h^2 + 2 h m)
// (what the Gram products below give for <u_j, u_j> without the m m term) in float32 and in three
// float16 parts, and the two Gram operand rows, K-major, in the tile layout the MMA reads
// (element (r, k) of 128-row tile q at q kU + ((k / 8) 16 + r / 8) 128 + (r % 8) 16 + (k % 8) 2),
// 32 values per row:
//   A role:  [h | m | h | 1 1 1 | -a_h -a_m -a_l | 0 ...]
//   B role:  [2h | 2h | 2m | -a_h -a_m -a_l | 1 1 1 | 0 ...]
// so that A_i . B_j = 2 (h_i h_j + m_i h_j + h_i m_j) - a_j - a_i = -|u_i - u_j|^2 to about 22 bits: the
// tensor core hands the generation the negated squared distance itself.
// words[16] collects max a_j over rows j < N (float bits, a_j >= 0).
template <int DP>
__global__ void dot_operands_kernel(const float *__restrict__ Xs, int64_t N, int64_t Np,
                                    unsigned int *__restrict__ words, float *__restrict__ arow,
                                    uint4 *__restrict__ ua, uint4 *__restrict__ ub, const int *skip) {
    if (skip && *skip) return;
    constexpr int KG = 32;
    static_assert(3 * DP + 6 <= KG, "Gram operand row too short");
    constexpr int kTileBytes = 128 * KG * 2;
    float c[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) c[d] = 0.5f * (float_of_ord(words[d]) - float_of_ord(words[8 + d]));
    unsigned int amax = 0u;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < Np; j += (int64_t)gridDim.x * blockDim.x) {
        __half h[DP], m[DP];
        double a = 0.0;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const float u = Xs[j * DP + d] - c[d];
            h[d] = __float2half_rn(u);
            const float hf = __half2float(h[d]);
            m[d] = __float2half_rn(u - hf);
            const double hd = hf, md = __half2float(m[d]);
            a += hd * hd + 2.0 * hd * md;
        }
        const float a32 = (float)a;
        const __half ah = __float2half_rn(a32);
        const float r1 = a32 - __half2float(ah);
        const __half am = __float2half_rn(r1);
        const __half al = __float2half_rn(r1 - __half2float(am));
        __half ra[KG], rb[KG];
        const __half zero = __float2half_rn(0.0f), one = __float2half_rn(1.0f);
#pragma unroll
        for (int k = 0; k < KG; ++k) ra[k] = rb[k] = zero;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const __half h2 = __hadd(h[d], h[d]), m2 = __hadd(m[d], m[d]);
            ra[d] = h[d];
            ra[DP + d] = m[d];
            ra[2 * DP + d] = h[d];
            rb[d] = h2;
            rb[DP + d] = h2;
            rb[2 * DP + d] = m2;
        }
        ra[3 * DP] = ra[3 * DP + 1] = ra[3 * DP + 2] = one;
        ra[3 * DP + 3] = __hneg(ah);
        ra[3 * DP + 4] = __hneg(am);
        ra[3 * DP + 5] = __hneg(al);
        rb[3 * DP] = __hneg(ah);
        rb[3 * DP + 1] = __hneg(am);
        rb[3 * DP + 2] = __hneg(al);
        rb[3 * DP + 3] = rb[3 * DP + 4] = rb[3 * DP + 5] = one;
        arow[j] = a32;
        const int64_t q = j / 128;
        const int r = (int)(j - q * 128);
#pragma unroll
        for (int kg = 0; kg < KG / 8; ++kg) {
            const int64_t off = (q * kTileBytes + (int64_t)((kg * 16 + (r >> 3)) * 128 + (r & 7) * 16)) / 16;
            ua[off] = *reinterpret_cast<const uint4 *>(ra + 8 * kg);
            ub[off] = *reinterpret_cast<const uint4 *>(rb + 8 * kg);
        }
        if (j < N) amax = max(amax, __float_as_uint(a32));
    }
    amax = __reduce_max_sync(0xffffffffu, amax);
    if ((threadIdx.x & 31) == 0) atomicMax(words + 16, amax);
}

__global__ void tc_reduce_kernel(const float *__restrict__ partial, int S, int64_t Np, int64_t N, int t,
                                 const float *__restrict__ V, int64_t ldv, float *__restrict__ out, int64_t ldo,
                                 float noise, const int *skip) {
    if (skip && *skip) return;
    const int64_t total = N * t;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / t;
        const int c = (int)(e - i * t);
        float s = 0.0f;
        for (int k = 0; k < S; ++k) s += partial[((int64_t)k * Np + i) * t + c];
        out[i * ldo + c] = fmaf(noise, V[i * ldv + c], s);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            (void)cudaGetLastError();
    }
    return fn;
}

// 2-D row-major map: `rows` rows of `cols` elements, box of box_cols x box_rows.
bool make_map(CUtensorMap *m, CUtensorMapDataType dt, int elem_bytes, const void *base, uint64_t cols, uint64_t rows,
              uint32_t box_cols, uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * (uint64_t)elem_bytes};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D map over a row-strided float32 matrix (rows x cols, row stride in bytes), box of
// box_cols x box_rows, shared-memory side swizzled as given.
bool make_map_strided(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t row_stride_bytes,
                      uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {row_stride_bytes};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcGrid {
    int rb, S, cps, total;
};

// Wave efficiency of s column splits: work items over whole waves of one-CTA-per-SM, with a
// mild preference for fewer splits.
double split_efficiency(int rb, int total, int s, int num_sms) {
    const int cps = (total + s - 1) / s;
    const int real_s = (total + cps - 1) / cps;
    const long long ctas = (long long)rb * real_s;
    const long long waves = (ctas + num_sms - 1) / num_sms;
    return (double)ctas / (double)(waves * num_sms) - 0.002 * s;
}

int max_splits(int total) { return std::max(1, std::min(32, total / 8)); }

TcGrid grid_for_splits(int64_t Np, int s) {
    TcGrid g;
    g.rb = (int)(Np / kBM);
    g.total = (int)(Np / kBK);
    s = std::max(1, std::min(s, max_splits(g.total)));
    g.cps = (g.total + s - 1) / s;
    g.S = (g.total + g.cps - 1) / g.cps;
    return g;
}

// Column splits chosen by wave efficiency (the autotuner may override with a measured choice).
TcGrid tc_grid(int64_t Np, int num_sms, int forced_splits = 0) {
    if (forced_splits > 0) return grid_for_splits(Np, forced_splits);
    const int rb = (int)(Np / kBM), total = (int)(Np / kBK);
    int best_s = 1;
    double best_eff = -1.0;
    for (int s = 1; s <= max_splits(total); ++s) {
        const double eff = split_efficiency(rb, total, s, num_sms);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best_s = s;
        }
    }
    return grid_for_splits(Np, best_s);
}

}  // namespace

bool tc_supported(int t) { return (t == 16 || t == 32) && encode_fn() != nullptr; }

// V_hi, V_lo [Np, t] 16-bit each, per-column max bits [64] and epilogue scales [64], the
// transposed prescaled X [8, Np] float32, then the dot-form distance data of the symmetric
// product: 32 words (bounding box, largest squared norm), a [Np] float32 and the A- and B-role
// Gram operands (up to 64 bytes per row each).
int64_t tc_vsplit_bytes(int64_t Np, int t) {
    return 2 * Np * t * 2 + 2 * 64 * 4 + 8 * Np * 4 + 32 * 4 + Np * 4 + 2 * Np * 64;
}

// LGP_TC_BANDS=1 lets the dot-form symmetric product walk its tiles in column bands (tile_walk.cuh).
// Measured at N = 500000, t = 32: the one-band order (every CTA on its own rows across all columns)
// read 80.6 GB and wrote 34.0 GB of DRAM per product, against about 0.26 GB of operands, and took
// 65.6 ms; the banded order moved 0.96 GB and took 68.2 ms (its walk costs registers in a kernel at
// its register limit). So the default keeps the single band.
bool tcs_bands_enabled() {
    const char *env = std::getenv("LGP_TC_BANDS");
    return env && std::strcmp(env, "1") == 0;
}

// Column-band width in 128-column tiles: a band's column-side operands (the split V rows, 4t bytes
// each; the B-role Gram operand, 64; and the rows of out its reductions add onto, 4t) take at most
// 48 MiB, about a third of the 129 MB L2, so that they stay cached while all CTAs sweep the band.
int tcs_band_tiles(int t) {
    const int64_t bytes_per_tile = (int64_t)tcs::kTile * (8 * t + 64);
    return (int)std::max<int64_t>(1, (48ll << 20) / bytes_per_tile);
}

int64_t tc_dot_gate_offset(int64_t Np, int t) { return 2 * Np * t * 2 + 2 * 64 * 4 + 8 * Np * 4 + 16 * 4; }

// Squared-norm limits of the dot form, per kernel: with a = max_j |u_j|^2 the rounding error of
// a_i + a_j - 2 u_i . u_j is about 4 a 2^-24, and an entry moves by at most |dk / dr^2| times that
// (ln 2 s^2 for the RBF on its prescaled coordinates, s^2 / 6 for Matern-5/2, s^2 / 2 for
// Matern-3/2). The limits hold that bound near 1.6e-5 s^2; data that spread wider take the
// difference form.
float dot_gate_limit(int kind) {
    switch (kind) {
        case LGP_RBF: return 97.0f;
        case LGP_MATERN52: return 403.0f;
        case LGP_MATERN32: return 134.0f;
    }
    return -1.0f;
}

// The dot form serves D >= 2. At D = 1 every point sits on one axis, so pairs of close points at
// the far ends of the box, where the Gram terms cancel most, are common: a NumPy model of the
// form's roundings gives Matern-5/2 column errors of 1.2e-5 at 90% of the limit, above the 1e-5
// product gate (D = 2: at most 3.9e-6, as at D = 3). LGP_DISTANCE=diff keeps the symmetric product
// on the difference form.
bool dot_form_allowed(int kind, int D) {
    if (dot_gate_limit(kind) <= 0.0f || D < 2) return false;
    const char *env = std::getenv("LGP_DISTANCE");
    return !(env && std::strcmp(env, "diff") == 0);
}

int64_t mv_tc_partial_floats(int64_t Np, int t, int num_sms, int forced_splits) {
    if (forced_splits == kTcSymmetric) return 0;
    const TcGrid g = tc_grid(Np, num_sms, forced_splits);
    return g.S > 1 ? (int64_t)g.S * Np * t : 0;
}

int64_t mv_tc_partial_floats(int64_t Np, int t, int num_sms) { return mv_tc_partial_floats(Np, t, num_sms, 0); }

bool tc_symmetric_ok(int64_t Np) { return Np / tcs::kTile >= 8; }

void tc_split_candidates(int64_t Np, int num_sms, int *cand, int *n) {
    const int rb = (int)(Np / kBM), total = (int)(Np / kBK);
    *n = 0;
    if (tc_symmetric_ok(Np)) cand[(*n)++] = kTcSymmetric;
    // the three most wave-efficient split counts, best first
    for (int k = 0; k < 3; ++k) {
        int best_s = 0;
        double best_eff = -1e9;
        for (int s = 1; s <= max_splits(total); ++s) {
            bool taken = false;
            for (int q = 0; q < *n; ++q) taken |= cand[q] == grid_for_splits(Np, s).S;
            if (taken) continue;
            const double eff = split_efficiency(rb, total, s, num_sms);
            if (eff > best_eff + 1e-9) {
                best_eff = eff;
                best_s = s;
            }
        }
        if (best_s == 0) break;
        cand[(*n)++] = grid_for_splits(Np, best_s).S;
        if (*n == 4) break;
    }
}

int mv_tc_launches(int64_t Np, int t, int num_sms, int fmt, int forced_splits, int kind, int D, bool operands_ready,
                   int dist_form) {
    // split V (+ column maxima for F16), transpose X unless ready, the product, the split reduction
    int n = 2 + (operands_ready ? 0 : 1) + (mv_tc_partial_floats(Np, t, num_sms, forced_splits) > 0 ? 1 : 0) +
            (fmt == kFmtF16 ? 1 : 0);
    if (forced_splits == kTcSymmetric && dot_form_allowed(kind, D))
        n += (operands_ready ? 0 : 2) + (dist_form < 0 ? 1 : 0);  // operand kernels, the second instance
    return n;
}

namespace {

cudaError_t launch_dot_operands(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, int t, void *vsplit,
                                const int *skip, cudaStream_t st) {
    unsigned int *words = (unsigned int *)((uint8_t *)vsplit + tc_dot_gate_offset(Np, t) - 16 * 4);
    float *arow = (float *)(words + 32);
    uint8_t *ua = (uint8_t *)(arow + Np);
    uint8_t *ub = ua + Np * 64;
    cudaError_t e = cudaMemsetAsync(words, 0, 32 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int bb = (int)std::min<int64_t>((N + 255) / 256, 1024);
    dot_bbox_kernel<<<bb, 256, 0, st>>>(Xs, N, kp.dpad, words, skip);
    const int ob = (int)std::min<int64_t>((Np + 255) / 256, 4096);
    if (kp.dpad <= 4)
        dot_operands_kernel<4><<<ob, 256, 0, st>>>(Xs, N, Np, words, arow, (uint4 *)ua, (uint4 *)ub, skip);
    else
        dot_operands_kernel<8><<<ob, 256, 0, st>>>(Xs, N, Np, words, arow, (uint4 *)ua, (uint4 *)ub, skip);
    return cudaGetLastError();
}

void launch_transpose_x(const KernelParams &kp, const float *Xs, int64_t Np, void *vsplit, int t, const int *skip,
                        cudaStream_t st) {
    float *XsT = (float *)((uint8_t *)vsplit + 2 * Np * t * 2 + 2 * 64 * 4);
    transpose_x_kernel<<<(int)std::min<int64_t>((Np * kp.dpad + 255) / 256, 4096), 256, 0, st>>>(Xs, Np, kp.dpad,
                                                                                              XsT, skip);
}

}  // namespace

cudaError_t launch_tc_operands(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, int t, void *vsplit,
                               bool dot, cudaStream_t st) {
    launch_transpose_x(kp, Xs, Np, vsplit, t, nullptr, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !dot) return e;
    return launch_dot_operands(kp, Xs, N, Np, t, vsplit, nullptr, st);
}

cudaError_t launch_mv_tc(const KernelParams &kp, const float *Xs, int64_t N, int64_t Np, const float *V, int64_t ldv,
                         float *out, int64_t ldo, int t, int fmt, void *vsplit, float *partial, int64_t partial_cap,
                         const int *skip, int *err_flag, long long wait_budget, int num_sms, cudaStream_t st,
                         int forced_splits, bool operands_ready, int dist_form, cudaEvent_t ev_begin,
                         cudaEvent_t ev_end) {
    auto mark = [&](cudaEvent_t ev) {
        if (ev) cudaEventRecord(ev, st);
    };
    if (!(t == 16 || t == 32) || Np % 256 != 0) return cudaErrorInvalidValue;
    uint16_t *vs = (uint16_t *)vsplit;  // stacked [V_hi; V_lo], 2 * Np * t entries
    unsigned int *vmax = (unsigned int *)(vs + 2 * Np * t);
    float *col_scale = (float *)(vmax + 64);
    float *XsT = col_scale + 64;
    const int blocks = (int)std::min<int64_t>((Np / 8 * t + 255) / 256, 8192);  // split_v: (8-row group, column)
    const bool symmetric = forced_splits == kTcSymmetric;
    float *out_init = symmetric ? out : nullptr;
    cudaError_t e;
    if (fmt == kFmtF16) {
        e = cudaMemsetAsync(vmax, 0, 64 * sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
        const int mb = (int)std::max<int64_t>(1, std::min<int64_t>((N * t + 255) / 256, 4 * num_sms));
        col_absmax_kernel<<<mb, (256 / t) * t, 0, st>>>(V, ldv, N, t, vmax, skip);
        if (t == 16)
            split_v_kernel<16, kFmtF16><<<blocks, 256, 0, st>>>(V, ldv, N, Np, vs, vmax, col_scale, kp.s2, out_init,
                                                              ldo, kp.noise, skip);
        else
            split_v_kernel<32, kFmtF16><<<blocks, 256, 0, st>>>(V, ldv, N, Np, vs, vmax, col_scale, kp.s2, out_init,
                                                              ldo, kp.noise, skip);
    } else {
        if (t == 16)
            split_v_kernel<16, kFmtBF16><<<blocks, 256, 0, st>>>(V, ldv, N, Np, vs, vmax, col_scale, kp.s2, out_init,
                                                              ldo, kp.noise, skip);
        else
            split_v_kernel<32, kFmtBF16><<<blocks, 256, 0, st>>>(V, ldv, N, Np, vs, vmax, col_scale, kp.s2, out_init,
                                                              ldo, kp.noise, skip);
    }
    if (!operands_ready) launch_transpose_x(kp, Xs, Np, vsplit, t, skip, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    const CUtensorMapDataType vt = fmt == kFmtF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (symmetric) {
        CUtensorMap mx, mv;
        if (!make_map(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, XsT, (uint64_t)Np, (uint64_t)kp.dpad, 64u,
                      (uint32_t)kp.dpad) ||
            !make_map(&mv, vt, 2, vs, 64, (uint64_t)(Np * 2 * t / 64), 64, (uint32_t)(2 * t)))
            return cudaErrorInvalidValue;
        tcs::TcsArgs a;
        a.Xs = Xs;
        a.out = out;
        a.skip = skip;
        a.err = err_flag;
        a.N = N;
        a.Np = Np;
        a.ldo = ldo;
        a.nb = (int)(Np / tcs::kTile);
        a.tiles = (int64_t)a.nb * (a.nb + 1) / 2;
        a.band = tcs_bands_enabled() ? tcs_band_tiles(t) : a.nb;
        a.log2s2 = fmt == kFmtF16 ? 15.0f : kp.log2_s2;
        a.col_scale = fmt == kFmtF16 ? col_scale : nullptr;
        // the drain's blocks go to out by TMA reduce when out's rows are 16-byte aligned
        CUtensorMap mo;
        memset(&mo, 0, sizeof mo);
        const bool aligned = (uintptr_t)out % 16 == 0 && ldo % 4 == 0;
        a.add_mode = aligned ? tcs::kAddTma : tcs::kAddScalar;
        if (aligned && !make_map_strided(&mo, out, (uint64_t)t, (uint64_t)N, (uint64_t)ldo * 4, (uint32_t)t,
                                         (uint32_t)tcs::kTile,
                                         t == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B))
            a.add_mode = tcs::kAddVec4;
        a.budget = wait_budget;
        a.gate = nullptr;
        a.gate_lim = 0.0f;
        a.dot = 0;
        a.arow = nullptr;
        a.ua = a.ub = nullptr;
        const dim3 grid((unsigned)std::min<int64_t>(num_sms, a.tiles), 1, 1);
        auto launch = [&]() {
            return fmt == kFmtF16 ? tcs::dispatch_f16(kp.kind, kp.D, t, grid, mx, mv, mo, a, st)
                                  : tcs::dispatch_bf16(kp.kind, kp.D, t, grid, mx, mv, mo, a, st);
        };
        if (!dot_form_allowed(kp.kind, kp.D)) {
            mark(ev_begin);
            e = launch();
            mark(ev_end);
            return e;
        }
        // dot form: operands (unless the caller built them for this X), then the instance of the known
        // distance form, or both instances, of which the gate word lets exactly one work
        if (!operands_ready && (e = launch_dot_operands(kp, Xs, N, Np, t, vsplit, skip, st)) != cudaSuccess)
            return e;
        unsigned int *words = (unsigned int *)(XsT + 8 * Np);
        float *arow = (float *)(words + 32);
        uint8_t *ua = (uint8_t *)(arow + Np);
        uint8_t *ub = ua + Np * 64;
        a.gate = words + 16;
        a.gate_lim = dot_gate_limit(kp.kind);
        a.arow = arow;
        a.ua = ua;
        a.ub = ub;
        mark(ev_begin);
        if (dist_form != 0) {
            a.dot = 1;
            if ((e = launch()) != cudaSuccess) return e;
        }
        if (dist_form != 1) {
            a.dot = 0;
            if ((e = launch()) != cudaSuccess) return e;
        }
        mark(ev_end);
        return cudaSuccess;
    }
    const TcGrid g = tc_grid(Np, num_sms, forced_splits);
    if (g.S > 1 && (partial == nullptr || (int64_t)g.S * Np * t > partial_cap)) return cudaErrorInvalidValue;
    CUtensorMap mx, mv;
    if (!make_map(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, XsT, (uint64_t)Np, (uint64_t)kp.dpad, (uint32_t)kBK,
                  (uint32_t)kp.dpad) ||
        !make_map(&mv, vt, 2, vs, 64, (uint64_t)(Np * 2 * t / 64), 64, (uint32_t)(2 * t)))
        return cudaErrorInvalidValue;
    tc::TcArgs a;
    a.Xs = Xs;
    a.V = V;
    a.out = g.S > 1 ? nullptr : out;
    a.partial = g.S > 1 ? partial : nullptr;
    a.skip = skip;
    a.err = err_flag;
    a.N = N;
    a.Np = Np;
    a.ldv = ldv;
    a.ldo = ldo;
    a.chunks_per_split = g.cps;
    a.total_chunks = g.total;
    a.log2s2 = fmt == kFmtF16 ? 15.0f : kp.log2_s2;
    a.noise = kp.noise;
    a.col_scale = fmt == kFmtF16 ? col_scale : nullptr;
    a.budget = wait_budget;
    const dim3 grid((unsigned)g.rb, (unsigned)g.S, 1);
    mark(ev_begin);
    e = fmt == kFmtF16 ? tc::dispatch_f16(kp.kind, kp.D, t, grid, mx, mv, a, st)
                       : tc::dispatch_bf16(kp.kind, kp.D, t, grid, mx, mv, a, st);
    mark(ev_end);
    if (e != cudaSuccess || g.S == 1) return e;
    const int rblocks = (int)std::min<int64_t>((N * t + 255) / 256, 4096);
    tc_reduce_kernel<<<rblocks, 256, 0, st>>>(partial, g.S, Np, N, t, V, ldv, out, ldo, kp.noise, skip);
    return cudaGetLastError();
}

}  // namespace lgp
