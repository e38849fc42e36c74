// Host partitioning of a renumbered mesh into sub-domains with two halo
// layers, for the boundary-first schedule (Sec. 6.4: each sub-domain updates
// the cells its neighbours need first, then its interior while the halo is
// exchanged).
#pragma once
#include <cstdint>
#include <vector>

struct swe_mesh;

struct swe_partition {
    int64_t n = 0;                      // cells of the mesh
    int n_parts = 0;
    std::vector<int64_t> start;         // [n_parts + 1]: part p owns cells [start[p], start[p+1])
    // per part, sorted by cell id:
    std::vector<std::vector<int32_t>> halo1;     // not owned, neighbour of an owned cell
    std::vector<std::vector<int32_t>> halo2;     // not owned nor in halo1, neighbour of a halo1 cell
    std::vector<std::vector<int32_t>> boundary;  // owned and in another part's halo1 or halo2
    std::vector<std::vector<int32_t>> interior;  // owned and in no other part's halo
    // all parts' boundary (then interior) cells, concatenated in part order
    std::vector<int32_t> boundary_all, interior_all;
    // halo exchange: part p receives halo1 then halo2, in that order, into
    // recv[recv_ptr[p] .. recv_ptr[p+1]); recv_cell lists the global cell of
    // every received slot (the cell's owner sends it)
    std::vector<int64_t> recv_ptr;
    std::vector<int32_t> recv_cell;
};

// Contiguous parts of equal size (within one cell) in the mesh's cell order.
// Returns 0, or a negative value for an unusable part count.
int swe_partition_build(const swe_mesh &m, int n_parts, swe_partition &out);
