// Host plan of the one-pass tile step (see swe_tiles.h for the layout).
//
// Tile b is the cells [b * tile, (b + 1) * tile) of the library's (Morton)
// order.  The kernel lists each edge with both cells inside the tile once and
// each edge towards another tile (a crossing edge) from its own side; for a
// crossing edge it needs the far cell's face value, whose gradient needs the
// far cell's own neighbours.  The plan names those outside cells (the halo),
// so that their state and normals can be gathered into shared memory ahead
// of the tile, and gives the local place of each neighbour of a far cell.
// emax, xmax, hmax, h1max and wmax are the largest counts over the tiles and
// size the tile's shared memory; the kernel counts its edges the same way
// and refuses a tile that would not fit.
#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "swe_mesh.h"
#include "swe_tiles.h"

int swe_build_tile_plan(const swe_mesh &m, int tile, TilePlan &out)
{
    if (tile < 32 || tile > 1024 || (tile & (tile - 1))) return -1;     // a power of two: divides the array padding
    const int64_t n = m.n;
    out = TilePlan{};
    out.tile = tile;
    out.n_tiles = (n + tile - 1) / tile;
    out.hdr.assign((size_t)(4 * out.n_tiles), 0);
    std::vector<int32_t> h1, h2, far;
    std::unordered_map<int32_t, int> place;      // outside cell -> halo index
    for (int64_t b = 0; b < out.n_tiles; b++) {
        const int64_t s0 = b * tile, s1 = std::min<int64_t>(n, s0 + tile);
        auto inside = [&](int64_t j) { return j >= s0 && j < s1; };
        int n_in = 0;
        h1.clear(); h2.clear(); far.clear(); place.clear();
        for (int64_t i = s0; i < s1; i++)
            for (int k = 0; k < 3; k++) {
                const int32_t j = m.nbr[3 * i + k];
                if (j < 0) continue;
                if (inside(j)) { n_in += j > i ? 1 : 0; continue; }
                auto it = place.find(j);
                if (it == place.end()) {
                    it = place.emplace(j, (int)h1.size()).first;
                    h1.push_back(j);
                }
                far.push_back(it->second);
            }
        // H2: outside neighbours of H1 cells that are not H1 cells themselves
        for (int32_t j : h1)
            for (int k = 0; k < 3; k++) {
                const int32_t q = m.nbr[3 * (int64_t)j + k];
                if (q >= 0 && !inside(q) && !place.count(q)) { place.emplace(q, -1); h2.push_back(q); }
            }
        std::sort(h2.begin(), h2.end());
        const int nh1 = (int)h1.size();
        for (size_t q = 0; q < h2.size(); q++) place[h2[q]] = nh1 + (int)q;
        const int n_halo = nh1 + (int)h2.size(), n_cross = (int)far.size();
        if (tile + n_halo >= (1 << 28)) return -2;
        const size_t off = out.words.size();
        out.words.insert(out.words.end(), h1.begin(), h1.end());
        out.words.insert(out.words.end(), h2.begin(), h2.end());
        for (int32_t j : h1)
            for (int k = 0; k < 3; k++) {
                const int64_t e = 3 * (int64_t)j + k;
                const int32_t q = m.nbr[e];
                if (q < 0) { out.words.push_back(-1); continue; }
                const int slot = inside(q) ? (int)(q - s0) : tile + place[q];
                out.words.push_back((slot << 3) | (m.nbr_edge[e] << 1) | 1);
            }
        out.words.insert(out.words.end(), far.begin(), far.end());
        while (out.words.size() % 4) out.words.push_back(0);
        const int nw = (int)(out.words.size() - off);
        int32_t *h = &out.hdr[(size_t)(4 * b)];
        h[0] = (int32_t)off; h[1] = n_halo; h[2] = nh1; h[3] = n_cross;
        if (out.words.size() > (size_t)INT32_MAX) return -3;
        out.emax = std::max(out.emax, n_in);
        out.xmax = std::max(out.xmax, n_cross);
        out.hmax = std::max(out.hmax, n_halo);
        out.h1max = std::max(out.h1max, nh1);
        out.wmax = std::max(out.wmax, nw);
    }
    if (out.words.empty()) out.words.assign(4, 0);
    return 0;
}
