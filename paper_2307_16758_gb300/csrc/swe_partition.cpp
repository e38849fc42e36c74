// Host partitioning with two halo layers (see swe_partition.h).
//
// The mesh is already in Morton order, so contiguous ranges of cells are
// compact sub-domains.  For part p: halo1 = cells outside p adjacent to p;
// halo2 = cells outside p and halo1 adjacent to halo1 (the second layer that
// the MUSCL and WAF reconstructions of halo1 cells read, Sec. 6.4); boundary =
// owned cells that some other part holds in its halo (they are updated first
// and sent); interior = the other owned cells.
#include <algorithm>

#include "swe_mesh.h"
#include "swe_partition.h"

int swe_partition_build(const swe_mesh &m, int n_parts, swe_partition &out)
{
    const int64_t n = m.n;
    if (n_parts < 1 || n_parts > 1024 || n_parts > n) return -1;
    out = swe_partition{};
    out.n = n;
    out.n_parts = n_parts;
    out.start.resize(n_parts + 1);
    for (int p = 0; p <= n_parts; p++) out.start[p] = n * p / n_parts;
    out.halo1.assign(n_parts, {});
    out.halo2.assign(n_parts, {});
    out.boundary.assign(n_parts, {});
    out.interior.assign(n_parts, {});
    std::vector<uint8_t> needed((size_t)n, 0);   // cell is in some other part's halo
    std::vector<int64_t> mark((size_t)n, -1);     // mark[c] = p when c is already in p's halo
    for (int p = 0; p < n_parts; p++) {
        const int64_t a = out.start[p], b = out.start[p + 1];
        std::vector<int32_t> &h1 = out.halo1[p], &h2 = out.halo2[p];
        for (int64_t c = a; c < b; c++)
            for (int k = 0; k < 3; k++) {
                const int32_t j = m.nbr[3 * c + k];
                if (j >= 0 && (j < a || j >= b) && mark[j] != p) { mark[j] = p; h1.push_back(j); }
            }
        for (int32_t c : h1)
            for (int k = 0; k < 3; k++) {
                const int32_t j = m.nbr[3 * (int64_t)c + k];
                if (j >= 0 && (j < a || j >= b) && mark[j] != p) { mark[j] = p; h2.push_back(j); }
            }
        std::sort(h1.begin(), h1.end());
        std::sort(h2.begin(), h2.end());
        for (int32_t c : h1) needed[c] = 1;
        for (int32_t c : h2) needed[c] = 1;
    }
    out.recv_ptr.assign(1, 0);
    for (int p = 0; p < n_parts; p++) {
        for (int64_t c = out.start[p]; c < out.start[p + 1]; c++)
            (needed[c] ? out.boundary[p] : out.interior[p]).push_back((int32_t)c);
        out.boundary_all.insert(out.boundary_all.end(), out.boundary[p].begin(), out.boundary[p].end());
        out.interior_all.insert(out.interior_all.end(), out.interior[p].begin(), out.interior[p].end());
        out.recv_cell.insert(out.recv_cell.end(), out.halo1[p].begin(), out.halo1[p].end());
        out.recv_cell.insert(out.recv_cell.end(), out.halo2[p].begin(), out.halo2[p].end());
        out.recv_ptr.push_back((int64_t)out.recv_cell.size());
    }
    for (int p = 0; p < n_parts; p++)      // bookkeeping check: a part receives no cell it owns
        for (int64_t s = out.recv_ptr[p]; s < out.recv_ptr[p + 1]; s++)
            if (out.recv_cell[s] >= out.start[p] && out.recv_cell[s] < out.start[p + 1]) return -2;
    return 0;
}
