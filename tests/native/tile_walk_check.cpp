// Host check of the symmetric product's tile order (csrc/tile_walk.cuh): every tile of the upper
// triangle is visited exactly once over all CTAs; segment starts fall exactly on a CTA's first tile, a
// band change or a row change; each CTA's count is what the kernel sizes its loops by; per band the
// CTAs' counts differ by at most one; and with one band the order is the plain row-by-row numbering
// of the triangle cut into contiguous ranges, walked in the same steps by the single-band walk.
// Usage: tile_walk_check nb W ncta; prints "ok <tiles> <bands>".
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "tile_walk.cuh"

using lgp::tcs::TileOrder;
using lgp::tcs::TileWalk;

static int fail(const char *what, int cta, long long it) {
    std::printf("FAIL %s (cta %d, step %lld)\n", what, cta, it);
    return 1;
}

int main(int argc, char **argv) {
    if (argc != 4) return 2;
    const int nb = std::atoi(argv[1]), W = std::atoi(argv[2]), ncta = std::atoi(argv[3]);
    const long long total = (long long)nb * (nb + 1) / 2;
    std::vector<unsigned char> seen((size_t)nb * nb, 0);
    const int Wc = W < 1 ? 1 : (W > nb ? nb : W);
    const int nbands = (nb + Wc - 1) / Wc;
    std::vector<long long> per_band((size_t)nbands * ncta, 0);
    long long visited = 0;
    for (int c = 0; c < ncta; ++c) {
        const TileOrder o = lgp::tcs::tile_order(nb, W, c, ncta);
        TileWalk w;
        w.init(o);
        const long long n = TileWalk::count(o);
        lgp::tcs::RowWalk rw;
        rw.init(o);
        if (Wc >= nb && n != lgp::tcs::RowWalk::count(o)) return fail("single-band walk count", c, 0);
        int prevI = -1, prevBand = -1;
        for (long long it = 0; it < n; ++it) {
            if (w.band >= nbands) return fail("walk ended early", c, it);
            const int I = w.I, J = w.J;
            if (I < 0 || J < I || J >= nb) return fail("tile outside the triangle", c, it);
            if (J < w.band * o.W || J >= lgp::tcs::band_end(o, w.band * o.W)) return fail("tile outside its band", c, it);
            if (seen[(size_t)I * nb + J]++) return fail("tile visited twice", c, it);
            const bool expect_first = it == 0 || w.band != prevBand || I != prevI;
            if (w.first != expect_first || w.starts_segment((int)it) != expect_first)
                return fail("segment start flag", c, it);
            per_band[(size_t)w.band * ncta + c] += 1;
            if (Wc >= nb) {
                // one band: the single-band walk takes the same steps
                if (rw.I != I || rw.J != J || rw.starts_segment((int)it) != expect_first)
                    return fail("single-band walk differs", c, it);
                rw.next(o);
                // after the step, both walks tell whether the tile just left ended its segment
                if (it + 1 < n) {
                    TileWalk ahead = w;
                    ahead.next(o);
                    if (rw.segment_changed(I) != ahead.segment_changed(I))
                        return fail("single-band walk: segment end", c, it);
                }
                // and the tile index is the row-by-row numbering of the whole triangle
                const long long idx = (long long)I * nb - (long long)I * (I - 1) / 2 + (J - I);
                const long long t0 = (long long)c * total / ncta;
                if (idx != t0 + it) return fail("one-band order differs from the row-by-row numbering", c, it);
            }
            prevI = I;
            prevBand = w.band;
            w.next(o);
        }
        if (w.band < nbands) return fail("walk longer than its count", c, n);
        if (!w.first) return fail("no segment end after the last tile", c, n);
        visited += n;
    }
    if (visited != total) return fail("tile count", -1, visited);
    for (int b = 0; b < nbands; ++b) {
        long long lo = per_band[(size_t)b * ncta], hi = lo;
        for (int c = 1; c < ncta; ++c) {
            const long long v = per_band[(size_t)b * ncta + c];
            lo = v < lo ? v : lo;
            hi = v > hi ? v : hi;
        }
        if (hi - lo > 1) return fail("band split uneven", -1, b);
    }
    std::printf("ok %lld %d\n", total, nbands);
    return 0;
}
