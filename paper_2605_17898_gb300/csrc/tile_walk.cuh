// Order in which the symmetric-tile product visits the upper triangle of 128 x 128 tiles (I <= J),
// and each CTA's share of it. Plain integer arithmetic, compiled for the device and, in the tests,
// for the host.
//
// The triangle is cut into column bands of W tiles: band b holds the columns J in [b W, min(nb, (b+1) W))
// and, for every row I below the band's end, the tiles J >= I of those columns. Within a band the tiles
// are numbered row by row, and each band is cut into one contiguous range per CTA (equal counts to
// within one). A CTA walks its range of band 0, then of band 1, and so on, so that all CTAs work in the
// same band at the same time and the column-side operands of that band (V_J, the Gram operand U_J,
// the rows of out that the out_J reductions add onto) stay in L2 while it is swept. With W >= nb there
// is one band and the order is the plain row-by-row numbering of the whole triangle.
//
// A segment is a run of consecutive tiles of one CTA in one band and one row I. The row-side operands
// (V_I, U_I, x_I) are loaded once per segment and out_I is added onto out when the segment ends.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define LGP_TW_FN __host__ __device__ __forceinline__
#else
#define LGP_TW_FN inline
#endif

namespace lgp {
namespace tcs {

// The order's parameters, the same for every thread of a launch: tiles per side, band width, number of
// bands, this CTA and the number of CTAs.
struct TileOrder {
    int nb, W, nbands, cta, ncta;
};

LGP_TW_FN TileOrder tile_order(int nb, int W, int cta, int ncta) {
    TileOrder o;
    o.nb = nb;
    o.W = W < 1 ? 1 : (W > nb ? nb : W);
    o.nbands = (nb + o.W - 1) / o.W;
    o.cta = cta;
    o.ncta = ncta;
    return o;
}

// end of the columns of the band that starts at column c0
LGP_TW_FN int band_end(const TileOrder &o, int c0) { return o.nb - c0 < o.W ? o.nb : c0 + o.W; }

// tiles of the band with columns [c0, c1): c0 full rows above its diagonal block, then the block
LGP_TW_FN int64_t band_tiles(int c0, int c1) {
    const int64_t w = c1 - c0;
    return (int64_t)c0 * w + w * (w + 1) / 2;
}

// A CTA's position in the order. Kept small (the kernel's threads are at their register limit): the
// parameters come in with each call.
struct TileWalk {
    int I, J;    // the current tile
    int band;    // current band (nbands once the walk has passed its last tile)
    int left;    // tiles of this CTA's range in the band from the current one on
    bool first;  // the current tile starts a segment

    // this CTA's range in band `band` or, if that is empty, in the next band that gives it tiles; then
    // (I, J) of the range's first tile in the band's row-by-row numbering
    LGP_TW_FN void enter_band(const TileOrder &o) {
        first = true;
        for (; band < o.nbands; ++band) {
            const int c0 = band * o.W;
            const int c1 = band_end(o, c0);
            const int64_t T = band_tiles(c0, c1);
            const int64_t k = (int64_t)o.cta * T / o.ncta;
            const int64_t k_end = (int64_t)(o.cta + 1) * T / o.ncta;
            if (k == k_end) continue;
            left = (int)(k_end - k);
            const int64_t w = c1 - c0;
            const int64_t top = (int64_t)c0 * w;
            if (k < top) {
                I = (int)(k / w);
                J = c0 + (int)(k - (int64_t)I * w);
                return;
            }
            // diagonal block: row r (I = c0 + r) holds w - r tiles and starts at r w - r (r - 1) / 2
            const int64_t kk = k - top;
            int lo = 0, hi = (int)w - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int64_t)mid * w - (int64_t)mid * (mid - 1) / 2 <= kk) lo = mid;
                else hi = mid - 1;
            }
            I = c0 + lo;
            J = I + (int)(kk - ((int64_t)lo * w - (int64_t)lo * (lo - 1) / 2));
            return;
        }
        left = 0;
    }

    LGP_TW_FN void init(const TileOrder &o) {
        I = J = 0;
        band = 0;
        enter_band(o);
    }

    // whether tile `it` of the walk starts a segment; after next(), whether the tile just left ended one
    // (prev_I: its row)
    LGP_TW_FN bool starts_segment(int it) const {
        (void)it;
        return first;
    }
    LGP_TW_FN bool segment_changed(int prev_I) const {
        (void)prev_I;
        return first;
    }

    LGP_TW_FN void next(const TileOrder &o) {
        if (band >= o.nbands) return;
        if (--left == 0) {
            ++band;
            enter_band(o);
            return;
        }
        const int c0 = band * o.W;
        if (++J == band_end(o, c0)) {
            ++I;
            J = I > c0 ? I : c0;
            first = true;
        } else {
            first = false;
        }
    }

    // tiles that the CTA of `o` visits
    LGP_TW_FN static int64_t count(const TileOrder &o) {
        int64_t n = 0;
        for (int b = 0; b < o.nbands; ++b) {
            const int c0 = b * o.W;
            const int64_t T = band_tiles(c0, band_end(o, c0));
            n += (int64_t)(o.cta + 1) * T / o.ncta - (int64_t)o.cta * T / o.ncta;
        }
        return n;
    }
};

// The same order with a single band (the row-by-row numbering of the whole triangle, cut into one
// contiguous range per CTA), in fewer registers: a segment is then a tile row, so its start and end
// follow from (I, J) alone. The kernel instance that never needs a second band walks with this one.
struct RowWalk {
    int nb, I, J;

    LGP_TW_FN static int64_t row_start(int64_t I, int64_t nb) { return I * nb - I * (I - 1) / 2; }

    LGP_TW_FN void init(const TileOrder &o) {
        nb = o.nb;
        const int64_t t0 = (int64_t)o.cta * band_tiles(0, o.nb) / o.ncta;
        int lo = 0, hi = nb - 1;  // largest I with row_start(I) <= t0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_start(mid, nb) <= t0) lo = mid;
            else hi = mid - 1;
        }
        I = lo;
        J = I + (int)(t0 - row_start(I, nb));
    }

    LGP_TW_FN void next(const TileOrder &) {
        if (++J == nb) {
            ++I;
            J = I;
        }
    }

    LGP_TW_FN bool starts_segment(int it) const { return it == 0 || J == I; }
    LGP_TW_FN bool segment_changed(int prev_I) const { return I != prev_I; }

    LGP_TW_FN static int64_t count(const TileOrder &o) {
        const int64_t T = band_tiles(0, o.nb);
        return (int64_t)(o.cta + 1) * T / o.ncta - (int64_t)o.cta * T / o.ncta;
    }
};

}  // namespace tcs
}  // namespace lgp

#undef LGP_TW_FN
