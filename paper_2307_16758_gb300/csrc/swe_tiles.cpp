// Host plan of the one-pass tile step (see swe_tiles.h for the layout).
//
// Everything about a tile that does not change from step to step is laid out
// here once: which outside cells it reads (its halo), where each neighbour
// of a tile or far cell sits in the tile's slot space, and the list of edges
// it solves -- each edge with both cells in the tile once, and each edge
// towards another tile (crossing) from the tile's side, whose far face value
// the tile recomputes from its halo.  The kernel then only indexes.
#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "swe_mesh.h"
#include "swe_tiles.h"

namespace {

// Local word of one edge of cell c (new id) in a tile that starts at s0,
// with `slot` mapping an outside cell to its slot.
template <typename F> int32_t local_word(const swe_mesh &m, int64_t c, int k, F slot)
{
    const int64_t e = 3 * c + k;
    const int32_t q = m.nbr[e];
    if (q < 0) return -1 - m.btag[e];
    return (slot(q) << 3) | (m.nbr_edge[e] << 1) | (m.owner[e] ? 1 : 0);
}

}  // namespace

int swe_build_tile_plan(const swe_mesh &m, int tile, TilePlan &out)
{
    if (tile < 32 || tile > 1024 || (tile & (tile - 1))) return -1;     // a power of two: divides the array padding
    const int64_t n = m.n;
    out = TilePlan{};
    out.tile = tile;
    out.n_tiles = (n + tile - 1) / tile;
    out.hdr.assign((size_t)(8 * out.n_tiles), 0);
    std::vector<int32_t> h1, h2, cross, inner;
    std::vector<int16_t> lw;
    std::unordered_map<int32_t, int> place;      // outside cell -> halo index
    for (int64_t b = 0; b < out.n_tiles; b++) {
        const int64_t s0 = b * tile, s1 = std::min<int64_t>(n, s0 + tile);
        auto inside = [&](int64_t j) { return j >= s0 && j < s1; };
        h1.clear(); h2.clear(); cross.clear(); inner.clear(); place.clear();
        // H1 in order of first use (cells ascending, then local edge)
        for (int64_t i = s0; i < s1; i++)
            for (int k = 0; k < 3; k++) {
                const int32_t j = m.nbr[3 * i + k];
                if (j >= 0 && !inside(j) && !place.count(j)) { place.emplace(j, (int)h1.size()); h1.push_back(j); }
            }
        for (int32_t j : h1)
            for (int k = 0; k < 3; k++) {
                const int32_t q = m.nbr[3 * (int64_t)j + k];
                if (q >= 0 && !inside(q) && !place.count(q)) { place.emplace(q, -1); h2.push_back(q); }
            }
        std::sort(h2.begin(), h2.end());
        const int nh1 = (int)h1.size();
        for (size_t q = 0; q < h2.size(); q++) place[h2[q]] = nh1 + (int)q;
        const int n_halo = nh1 + (int)h2.size();
        if (tile + n_halo > 2047) return -2;         // slots are 11-bit fields of the edge records
        auto slot = [&](int64_t q) -> int { return inside(q) ? (int)(q - s0) : tile + place[(int32_t)q]; };
        // edges: crossing ones first, then the ones inside the tile (from the lower slot)
        for (int64_t i = s0; i < s1; i++)
            for (int k = 0; k < 3; k++) {
                const int64_t e = 3 * i + k;
                const int32_t j = m.nbr[e];
                if (j < 0) continue;
                const bool cr = !inside(j);
                if (!cr && j < i) continue;
                const uint32_t r = (uint32_t)(i - s0) | ((uint32_t)k << 11) | ((uint32_t)slot(j) << 13) |
                                   ((uint32_t)m.nbr_edge[e] << 24) | ((uint32_t)(m.owner[e] ? 1 : 0) << 26) |
                                   ((uint32_t)(cr ? 1 : 0) << 27);
                (cr ? cross : inner).push_back((int32_t)r);
            }
        // local words of the tile's slots (unused slots past the mesh: boundary walls) and of H1
        lw.assign((size_t)(3 * (tile + nh1)), (int16_t)-1);
        for (int64_t i = s0; i < s1; i++)
            for (int k = 0; k < 3; k++) lw[(size_t)(3 * (i - s0) + k)] = (int16_t)local_word(m, i, k, slot);
        for (int q = 0; q < nh1; q++)
            for (int k = 0; k < 3; k++) lw[(size_t)(3 * (tile + q) + k)] = (int16_t)local_word(m, h1[q], k, slot);
        const size_t off = out.words.size();
        out.words.insert(out.words.end(), h1.begin(), h1.end());
        out.words.insert(out.words.end(), h2.begin(), h2.end());
        out.words.insert(out.words.end(), cross.begin(), cross.end());
        out.words.insert(out.words.end(), inner.begin(), inner.end());
        const size_t lw0 = out.words.size();
        out.words.resize(lw0 + (lw.size() + 1) / 2, 0);
        std::copy(lw.begin(), lw.end(), reinterpret_cast<int16_t *>(out.words.data() + lw0));
        while (out.words.size() % 8) out.words.push_back(0);
        const int nw = (int)(out.words.size() - off);
        int32_t *h = &out.hdr[(size_t)(8 * b)];
        h[0] = (int32_t)off; h[1] = n_halo; h[2] = nh1; h[3] = (int)(cross.size() + inner.size());
        h[4] = (int)cross.size(); h[5] = nw;
        if (out.words.size() > (size_t)INT32_MAX) return -3;
        out.hmax = std::max(out.hmax, n_halo);
        out.h1max = std::max(out.h1max, nh1);
        out.wmax = std::max(out.wmax, nw);
    }
    if (out.words.empty()) out.words.assign(8, 0);
    return 0;
}
