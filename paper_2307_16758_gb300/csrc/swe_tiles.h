// Tiling of the renumbered cells for the fused kernel (built on the host).
#pragma once
#include <cstdint>
#include <vector>

struct swe_mesh;

struct Tiling {
    int tile = 0;
    int max_halo = 0;
    std::vector<int32_t> halo_ptr;    // [n_tiles + 1]
    std::vector<int32_t> halo_ids;    // halo cells of all tiles, sorted per tile
    std::vector<uint16_t> nbr_local;  // [3n], see FusedArgs
};

// Returns 0, or -1 if a slot does not fit in 12 bits (tile too large).
int swe_build_tiling(const swe_mesh &m, int tile, Tiling &out);
