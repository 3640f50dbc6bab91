// sched.cpp -- work decomposition of the separable l3 contraction.
//
// The valid pairs lmin <= l1 <= l2 <= lmax become, per parity class pi,
// the region  i >= 0,  j - i >= lmin,  i + j + pi <= lmax  of the (i, j)
// plane (d = 2i + pi, s = 2j + pi).  It is covered by TILE_I x TILE_J
// blocks.  The plain kernels run every pair of a block over the block's
// whole k range (l3 = 2k + pi or 2k + 1 - pi, from the first row's
// smallest k to the last column's largest; a pair's own range, |l1 - l2|
// .. l1 + l2 (Sec. 3), is selected by zero operands), so a block's run time
// is set by that range, not by its count of valid terms: edge blocks with
// few valid pairs cost as much as full ones.  The list is sorted by this
// run-time model, largest first (longest-processing-time order), so that
// the longest blocks start first and the launch ends with short ones.
#include <algorithm>

#include "internal.h"

namespace cpl {

double tile_time(const Tile &t, int cap) {
    // k range of the block as the kernels run it (even and odd sweeps),
    // staged in chunks of 16 k, plus the epilogue (about a dozen k steps of
    // FP64 work per pair); in units of one k step of the block
    const int pi = t.pi;
    const int kce = (cap - pi) >> 1, kco = (cap - 1 + pi) >> 1;
    const int khi = std::max(std::min(t.j0 + TILE_J - 1, kce), std::min(t.j0 + TILE_J - 2 + pi, kco));
    const int span = std::max(khi - t.i0 + 1, 0);
    return (double)span + (double)((span + 15) / 16) + 12.0;
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

static bool tile_has_pairs(const Tile &t, int lmax, int lmin) {
    for (int di = 0; di < TILE_I; ++di)
        for (int dj = 0; dj < TILE_J; ++dj) {
            const int i = t.i0 + di, j = t.j0 + dj;
            const int l1 = j - i, l2 = i + j + t.pi;
            if (l1 >= lmin && l2 <= lmax && l1 <= l2) return true;
        }
    return false;
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
                if (!tile_has_pairs(t, lmax, lmin)) continue;
                t.cost = (int32_t)tile_time(t, 2 * lmax);
                tiles.push_back(t);
            }
        }
    }
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const Tile &a, const Tile &b) { return a.cost > b.cost; });
}


}  // namespace cpl
