// tiles.cuh -- the order in which the CTAs of the one-kernel Uzawa steps take their tiles.
#pragma once

namespace smg {

// Order in which the CTAs take the tiles: first the tiles whose u^{m-1/2} region meets a mid-line
// (their cells run the slower per-cell rows), column band then row band, then all others, so that
// the block scheduler hands the long tiles out first and fills in with short ones.
struct TileOrder {
    int cols, rows;   // tiles per row and per column
    int c0, nc;       // tile columns c0 .. c0 + nc - 1 meet the mid-line x = 1/2
    int r0, nr;       // tile rows r0 .. r0 + nr - 1 meet y = 1/2
    __device__ __forceinline__ void tile(int b, int& c, int& r) const {
        const int na = nc * rows;
        if (b < na) {
            c = c0 + b % nc;
            r = b / nc;
            return;
        }
        b -= na;
        const int nb = nr * (cols - nc);
        if (b < nb) {
            r = r0 + b % nr;
            const int cc = b / nr;
            c = cc < c0 ? cc : cc + nc;
            return;
        }
        b -= nb;
        const int cc = b % (cols - nc), rr = b / (cols - nc);
        c = cc < c0 ? cc : cc + nc;
        r = rr < r0 ? rr : rr + nr;
    }
};

// tiles of size `len` whose region [t len - 2, t len + len + 2) contains h: first and count
inline void mid_band(int h, int len, int tiles, int& first, int& count) {
    first = -1;
    count = 0;
    for (int t = 0; t < tiles; ++t)
        if (t * len - 2 <= h && h < t * len + len + 2) {
            if (first < 0) first = t;
            ++count;
        }
    if (first < 0) first = 0;
}

}  // namespace smg
