// Host tiling for the fused kernel: per tile of consecutive (Morton-ordered)
// cells, the sorted list of halo cells (neighbours outside the tile) and, per
// cell edge, the neighbour's slot in the tile's shared-memory arrays.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "swe_mesh.h"
#include "swe_tiles.h"

int swe_build_tiling(const swe_mesh &m, int tile, Tiling &out)
{
    const int64_t n = m.n;
    const int64_t n_tiles = (n + tile - 1) / tile;
    out.tile = tile;
    out.halo_ptr.assign((size_t)(n_tiles + 1), 0);
    out.halo_ids.clear();
    out.nbr_local.assign((size_t)(3 * n), 0);
    out.max_halo = 0;
    std::vector<int32_t> halo;
    for (int64_t b = 0; b < n_tiles; b++) {
        const int64_t s = b * tile, e = std::min<int64_t>(n, s + tile);
        halo.clear();
        for (int64_t i = s; i < e; i++)
            for (int k = 0; k < 3; k++) {
                int32_t j = m.nbr[3 * i + k];
                if (j >= 0 && (j < s || j >= e)) halo.push_back(j);
            }
        std::sort(halo.begin(), halo.end());
        halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
        for (int64_t i = s; i < e; i++)
            for (int k = 0; k < 3; k++) {
                const int64_t ed = 3 * i + k;
                int32_t j = m.nbr[ed];
                if (j < 0) { out.nbr_local[ed] = (uint16_t)(0x8000 | m.btag[ed]); continue; }
                int32_t slot = (j >= s && j < e)
                                   ? (int32_t)(j - s)
                                   : tile + (int32_t)(std::lower_bound(halo.begin(), halo.end(), j) - halo.begin());
                if (slot >= 4096) return -1;
                out.nbr_local[ed] = (uint16_t)((slot << 3) | (m.nbr_edge[ed] << 1) | (m.owner[ed] ? 1 : 0));
            }
        out.halo_ids.insert(out.halo_ids.end(), halo.begin(), halo.end());
        out.halo_ptr[(size_t)(b + 1)] = (int32_t)out.halo_ids.size();
        out.max_halo = std::max(out.max_halo, (int)halo.size());
    }
    return 0;
}
