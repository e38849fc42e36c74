// Tile plan of the one-pass tile step (built on the host from the mesh).
#pragma once
#include <cstdint>
#include <vector>

struct swe_mesh;

// Tile b is the cells [b * tile, (b + 1) * tile) of the library's order.
// A tile works in a slot space: slots 0 .. tile-1 are its cells (a slot past
// the end of the mesh is unused), slots tile .. tile + n_halo - 1 its halo,
// the outside cells it reads: first the far cells of its crossing edges (H1,
// distinct, in order of first use), then the other outside neighbours of
// those (H2, distinct, ascending).
//
// The tile's plan words, words[hdr[8 b] ..], all int32:
//   halo ids     [n_halo]    global cell ids, H1 then H2
//   edges        [n_edges]   crossing edges first, then the edges inside the
//                            tile, each once: slot_i | k_i << 11 | slot_j << 13 |
//                            k_j << 24 | own_i << 26 | crossing << 27
//   local words  [3 * (tile + n_h1)] as int16 pairs: per slot (tile cells,
//                then H1 cells) and local edge k, (slot' << 3) | (k' << 1) |
//                own for a neighbour in slot' whose local edge is k', own = 1
//                when this cell is the edge's canonical left state; -1 - tag
//                on the domain boundary (the global words' encoding)
// padded to a multiple of 8 words.  hdr[8 b ..] = (offset, n_halo, n_h1,
// n_edges, n_cross, number of words, 0, 0).
struct TilePlan {
    int tile = 0;                     // cells per tile = threads per block
    int64_t n_tiles = 0;
    int hmax = 0;                     // most halo cells of one tile
    int h1max = 0;                    // most H1 cells of one tile
    int wmax = 0;                     // most plan words of one tile (a multiple of 8)
    std::vector<int32_t> hdr;         // [8 * n_tiles]
    std::vector<int32_t> words;
};

// Returns 0, or a negative value if the tile size is unsupported or a tile's
// slots do not fit the edge records.
int swe_build_tile_plan(const swe_mesh &m, int tile, TilePlan &out);
