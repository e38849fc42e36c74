// Host-side mesh representation built by swe_mesh_create (cells renumbered).
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/swe.h"

struct swe_mesh {
    int64_t n = 0;
    std::vector<int32_t> perm;      // perm[new] = original id
    std::vector<int32_t> inv;       // inv[original] = new id
    std::vector<int32_t> tri;       // [n][3] oriented counter-clockwise (new order)
    std::vector<int32_t> nbr;       // [n][3] neighbour (new id) or -1
    std::vector<int32_t> nbr_edge;  // [n][3] local edge index in the neighbour or -1
    std::vector<int32_t> btag;      // [n][3] boundary tag or -1
    std::vector<uint8_t> owner;     // [n][3] 1 if this cell is the canonical left state of the edge
    std::vector<double> lnx, lny;   // [n][3] outward normal times length
    std::vector<double> len;        // [n][3] edge length
    std::vector<double> area, cx, cy, rin;
    std::vector<double> dx, dy;     // [n][3] centroid offsets to the neighbour
    double r_min = 0.0;
    double group_len[SWE_MAX_GROUPS] = {};   // total length of the INFLOW edges per group
};

// Packed neighbour word used on the device: interior edges carry
// (neighbour << 3) | (neighbour's local edge << 1) | owner; boundary edges
// carry -1 - tag.
inline int32_t swe_pack_nbr(const swe_mesh &m, int64_t i, int k)
{
    int64_t e = 3 * i + k;
    if (m.nbr[e] >= 0) return (m.nbr[e] << 3) | (m.nbr_edge[e] << 1) | (m.owner[e] ? 1 : 0);
    return -1 - m.btag[e];
}
