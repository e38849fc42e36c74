// Tiling of the renumbered cells for the fused kernel (built on the host).
#pragma once
#include <cstdint>
#include <vector>

struct swe_mesh;

struct Tiling {
    int block = 0;                    // threads per block = largest tile + halo
    int n_tiles = 0;
    int max_edges = 0;
    std::vector<int32_t> tile_start;  // [n_tiles + 1]
    std::vector<int32_t> halo_ptr;    // [n_tiles + 1]
    std::vector<int32_t> halo_ids;    // halo cells of all tiles, sorted per tile
    std::vector<int32_t> edge_ptr;    // [n_tiles + 1]
    std::vector<uint32_t> edges;      // per tile, see FusedArgs
    std::vector<uint16_t> nbr_local;  // [3n], see FusedArgs
};

// Returns 0, or a negative value if the block size is unsupported.
int swe_build_tiling(const swe_mesh &m, int block, Tiling &out);
