// Tile plan of the one-pass tile step (built on the host from the mesh).
#pragma once
#include <cstdint>
#include <vector>

struct swe_mesh;

// Per tile b (cells [b * tile, (b + 1) * tile) of the library's order):
//   inside edges: edges with both cells in the tile;
//   crossing edges: edges from a tile cell to a cell outside, in the order
//     the kernel lists them (cells ascending, then local edge k ascending);
//   halo: the outside cells the tile reads -- first the far cells of its
//     crossing edges (H1, distinct, in order of first use), then the other
//     outside neighbours of those (H2, distinct, ascending).
// The tile's plan words, words[hdr[b].x ..], are (all int32):
//   halo ids        [n_halo]         global cell ids, H1 then H2
//   H1 neighbours   [3 * n_h1]       per H1 cell and local edge k: -1 on the
//                                    domain boundary, else (slot << 3) |
//                                    (k' << 1) | 1 with slot the neighbour's
//                                    place (0 .. tile-1 a tile cell, tile +
//                                    q halo cell q) and k' its local edge
//   crossing far    [n_cross]        H1 index of each crossing edge's far cell
// padded to a multiple of 4 words; hdr[b] = (offset, n_halo, n_h1, n_cross).
struct TilePlan {
    int tile = 0;                     // cells per tile = threads per block
    int64_t n_tiles = 0;
    int emax = 0;                     // most inside edges of one tile
    int xmax = 0;                     // most crossing edges of one tile
    int hmax = 0;                     // most halo cells of one tile
    int h1max = 0;                    // most H1 cells of one tile
    int wmax = 0;                     // most plan words of one tile (a multiple of 4)
    std::vector<int32_t> hdr;         // [4 * n_tiles]
    std::vector<int32_t> words;
};

// Returns 0, or a negative value if the tile size is unsupported.
int swe_build_tile_plan(const swe_mesh &m, int tile, TilePlan &out);
