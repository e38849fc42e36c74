// Tile plan of the one-pass tile step (built on the host from the mesh).
#pragma once
#include <cstdint>
#include <vector>

struct swe_mesh;

struct TilePlan {
    int tile = 0;                     // cells per tile = threads per block
    int64_t n_tiles = 0;
    int emax = 0;                     // most edges inside one tile
    int xmax = 0;                     // most crossing edges of one tile
    int64_t n_cross = 0;              // crossing edges of all tiles
};

// Returns 0, or a negative value if the tile size is unsupported.
int swe_build_tile_plan(const swe_mesh &m, int tile, TilePlan &out);
