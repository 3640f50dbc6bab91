// sched.cpp -- work decomposition of the separable l3 contraction.
//
// The valid pairs lmin <= l1 <= l2 <= lmax become, per parity class pi,
// the region  i >= 0,  j - i >= lmin,  i + j + pi <= lmax  of the (i, j)
// plane (d = 2i + pi, s = 2j + pi).  It is covered by TILE_I x TILE_J
// blocks; a block's work is the number of l3 terms of its valid pairs,
// 2 l1 + 1 per pair over both parities of L (Sec. 3: the l3 sum of a pair
// runs over |l1 - l2| .. l1 + l2), so blocks far from the diagonal cost
// more.  The list is sorted by decreasing cost (longest-processing-time
// order) so that the heaviest blocks start first.
#include <algorithm>

#include "internal.h"

namespace cpl {

static inline long long pair_terms(int l1, int band) {
    // l3 terms of a pair with l1 <= l2 over both parities, l3 <= band
    (void)band;
    return 2LL * l1 + 1;
}

double tile_terms(const Tile &t, int lmax, int lmin, int band) {
    double sum = 0.0;
    for (int di = 0; di < TILE_I; ++di) {
        const int i = t.i0 + di;
        const int d = 2 * i + t.pi;
        for (int dj = 0; dj < TILE_J; ++dj) {
            const int j = t.j0 + dj;
            const int l1 = j - i, l2 = i + j + t.pi;
            if (l1 < lmin || l2 > lmax || l1 > l2) continue;
            if (band < 0) {
                sum += (double)pair_terms(l1, band);
            } else {
                const int hi = std::min(l1 + l2, band);
                if (hi >= d) sum += (double)(hi - d + 1);
            }
        }
    }
    return sum;
}

void tile_terms_split(const Tile &t, int lmax, int lmin, int cap, double *even, double *odd,
                      double *pairs) {
    // even l3 = 2k + pi, k in [i, min(j, (cap - pi)/2)];
    // odd  l3 = 2k + 1 - pi, k in [i + pi, min(j + pi - 1, (cap - 1 + pi)/2)]
    const int pi = t.pi;
    const int kce = (cap - pi) >> 1, kco = (cap - 1 + pi) >> 1;
    double e = 0.0, o = 0.0, np = 0.0;
    for (int di = 0; di < TILE_I; ++di) {
        const int i = t.i0 + di;
        for (int dj = 0; dj < TILE_J; ++dj) {
            const int j = t.j0 + dj;
            const int l1 = j - i, l2 = i + j + pi;
            if (l1 < lmin || l2 > lmax || l1 > l2) continue;
            np += 1.0;
            const int ne = std::min(j, kce) - i + 1;
            const int no = std::min(j + pi - 1, kco) - (i + pi) + 1;
            if (ne > 0) e += ne;
            if (no > 0) o += no;
        }
    }
    *even = e;
    *odd = o;
    *pairs = np;
}

void make_tiles(int lmax, int lmin, std::vector<Tile> &tiles) {
    tiles.clear();
    for (int pi = 0; pi < 2; ++pi) {
        const int imax = (lmax - lmin - pi) / 2;   // d = 2i + pi <= lmax - lmin
        if (lmax - lmin - pi < 0) continue;
        for (int i0 = 0; i0 <= imax; i0 += TILE_I) {
            // j from i0 + lmin (smallest l1 at the block's first row) up to lmax - pi - i0
            const int jlo = std::max(0, i0 + lmin - (TILE_J - 1));
            const int jhi = lmax - pi - i0;
            for (int j0 = (jlo / TILE_J) * TILE_J; j0 <= jhi; j0 += TILE_J) {
                Tile t;
                t.pi = (int16_t)pi;
                t.pad = 0;
                t.i0 = i0;
                t.j0 = j0;
                const double c = tile_terms(t, lmax, lmin, -1);
                if (c <= 0.0) continue;
                t.cost = (int32_t)std::min(c / 1024.0 + 1.0, 2.0e9);
                tiles.push_back(t);
            }
        }
    }
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const Tile &a, const Tile &b) { return a.cost > b.cost; });
}


}  // namespace cpl
