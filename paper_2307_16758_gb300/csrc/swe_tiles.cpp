// Host plan of the one-pass tile step.
//
// Tile b is the cells [b * tile, (b + 1) * tile) of the library's (Morton)
// order.  A tile lists each edge with both cells inside it once and each
// edge towards another tile (a crossing edge) from its own side, where it
// recomputes the far cell's face value; emax and xmax are the largest counts
// over the tiles, which size the tile's shared memory.  The kernel counts the
// same way and refuses a tile that would not fit.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "swe_mesh.h"
#include "swe_tiles.h"

int swe_build_tile_plan(const swe_mesh &m, int tile, TilePlan &out)
{
    if (tile < 32 || tile > 1024 || tile % 32) return -1;
    const int64_t n = m.n;
    out = TilePlan{};
    out.tile = tile;
    out.n_tiles = (n + tile - 1) / tile;
    for (int64_t b = 0; b < out.n_tiles; b++) {
        const int64_t s0 = b * tile, s1 = std::min<int64_t>(n, s0 + tile);
        int inside = 0, cross = 0;
        for (int64_t i = s0; i < s1; i++)
            for (int k = 0; k < 3; k++) {
                const int64_t j = m.nbr[3 * i + k];
                if (j < 0) continue;
                if (j >= s0 && j < s1) inside += j > i ? 1 : 0;
                else cross++;
            }
        out.emax = std::max(out.emax, inside);
        out.xmax = std::max(out.xmax, cross);
        out.n_cross += cross;
    }
    return 0;
}
