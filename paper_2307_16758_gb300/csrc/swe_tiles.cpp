// Host tiling for the fused kernel.
//
// Tiles are runs of consecutive (Morton-ordered) cells, grown greedily while
// the tile's cells plus its halo (neighbours outside the tile) fit in one
// block, so that each thread loads and reconstructs exactly one cell.  Slots:
// tile cells 0..nc-1, halo cells nc..nc+H-1 (sorted by id).  Per tile, the
// edge list names every interior edge with at least one side in the tile
// once, from a tile cell's side (i): slot_i | k_i | slot_j | k_j | i owns the
// edge | j is in the tile.  Boundary edges are not listed (each cell handles
// its own).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "swe_mesh.h"
#include "swe_tiles.h"

int swe_build_tiling(const swe_mesh &m, int block, Tiling &out)
{
    const int64_t n = m.n;
    if (block < 32 || block > 512) return -1;
    out.block = block;
    out.tile_start.clear();
    out.halo_ptr.assign(1, 0);
    out.edge_ptr.assign(1, 0);
    out.halo_ids.clear();
    out.edges.clear();
    out.nbr_local.assign((size_t)(3 * n), 0);
    out.max_edges = 0;
    std::vector<int64_t> tile_mark((size_t)n, -1), halo_mark((size_t)n, -1);
    std::vector<int32_t> cand, halo;
    int64_t i = 0, tile = 0;
    while (i < n) {
        const int64_t s = i;
        int nc = 0, H = 0;
        cand.clear();
        while (i < n) {
            // halo size if cell i joins: i leaves the halo, its outside neighbours join
            int dh = halo_mark[i] == tile ? -1 : 0;
            int32_t add[3];
            int na = 0;
            for (int k = 0; k < 3; k++) {
                int32_t j = m.nbr[3 * i + k];
                if (j < 0 || j == i || tile_mark[j] == tile || halo_mark[j] == tile) continue;
                bool dup = false;
                for (int q = 0; q < na; q++) dup = dup || add[q] == j;
                if (!dup) add[na++] = j;
            }
            dh += na;
            if (nc > 0 && nc + 1 + H + dh > block) break;
            tile_mark[i] = tile;
            if (halo_mark[i] == tile) halo_mark[i] = -1;
            for (int q = 0; q < na; q++) { halo_mark[add[q]] = tile; cand.push_back(add[q]); }
            H += dh;
            nc++;
            i++;
        }
        halo.clear();
        for (int32_t c : cand)
            if (halo_mark[c] == tile && tile_mark[c] != tile) halo.push_back(c);
        std::sort(halo.begin(), halo.end());
        halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
        if ((int)halo.size() != H || nc + H > block) return -2;   // bookkeeping check
        out.tile_start.push_back((int32_t)s);
        out.halo_ids.insert(out.halo_ids.end(), halo.begin(), halo.end());
        out.halo_ptr.push_back((int32_t)out.halo_ids.size());
        auto slot_of = [&](int32_t j) -> int {
            if (j >= s && j < s + nc) return (int)(j - s);
            return nc + (int)(std::lower_bound(halo.begin(), halo.end(), j) - halo.begin());
        };
        int ne = 0;
        const size_t e0 = out.edges.size();
        for (int64_t c = s; c < s + nc; c++)
            for (int k = 0; k < 3; k++) {
                const int64_t e = 3 * c + k;
                int32_t j = m.nbr[e];
                if (j < 0) { out.nbr_local[e] = (uint16_t)(0x8000 | m.btag[e]); continue; }
                const int sj = slot_of(j), si = (int)(c - s);
                out.nbr_local[e] = (uint16_t)((sj << 3) | (m.nbr_edge[e] << 1) | (m.owner[e] ? 1 : 0));
                const bool in_tile = sj < nc;
                if (in_tile && j < c) continue;          // listed once, from the lower slot
                uint32_t w = (uint32_t)si | ((uint32_t)k << 9) | ((uint32_t)sj << 11) |
                             ((uint32_t)m.nbr_edge[e] << 20) | ((uint32_t)(m.owner[e] ? 1 : 0) << 22) |
                             ((uint32_t)(in_tile ? 1 : 0) << 23);
                out.edges.push_back(w);
                ne++;
            }
        // order by (k_i, slot_i): neighbouring threads then touch neighbouring
        // shared-memory words (no bank conflicts on side i)
        std::sort(out.edges.begin() + e0, out.edges.end(), [](uint32_t x, uint32_t y) {
            const uint32_t kx = (x >> 9) & 3u, ky = (y >> 9) & 3u;
            return kx != ky ? kx < ky : (x & 511u) < (y & 511u);
        });
        out.edge_ptr.push_back((int32_t)out.edges.size());
        out.max_edges = std::max(out.max_edges, ne);
        tile++;
    }
    out.tile_start.push_back((int32_t)n);
    out.n_tiles = (int)tile;
    return 0;
}
