/*
 * swe_tile_plan.h -- host-side inspection of the tile step's plan.
 *
 * The one-pass tile step (SWE_KERNEL_FUSED; the default for FP64) solves the
 * semi-discrete form of Sec. 6.1 tile by tile: a tile is `tile` consecutive
 * cells of the library's order, and every edge L_ij with a cell in the tile
 * is handled by that tile.  Which outside cells a tile reads and how its
 * edges are indexed does not change from step to step, so the library lays
 * it out once on the host, as a plan, and uploads it.  These two calls build
 * the same plan for a mesh and hand it to the caller, so that it can be
 * checked or sized without a GPU.  Both run on the host only and never touch
 * a device.
 *
 * Layout (int32 words).  Tile b covers the cells [b*tile, (b+1)*tile) and
 * numbers them slots 0 .. tile-1 (slots past the last cell are unused); its
 * halo takes the slots from `tile` on: first H1, the cells outside the tile
 * that share an edge with it (each once, in the order in which the tile's
 * cells, ascending, and their local edges 0..2 first reach them), then H2,
 * the cells outside the tile and H1 that share an edge with an H1 cell
 * (ascending).  hdr[8*b .. 8*b+7] = (offset of the tile's words, n_halo,
 * n_h1, n_edges, n_cross, number of words, 0, 0).  At words[offset]:
 *   n_halo   halo cell ids (new order), H1 then H2;
 *   n_edges  edge records, the n_cross edges towards other tiles first (one
 *            per local edge of a tile cell whose neighbour is outside), then
 *            each edge with both cells in the tile once, from the cell with
 *            the lower (new) id:
 *            slot_i | k_i << 11 | slot_j << 13 | k_j << 24 | own_i << 26 |
 *            crossing << 27, where slot_i (a tile cell) and slot_j are
 *            the edge's cells, k_i and k_j its local index in each, and
 *            own_i = 1 when cell i is the edge's left state: the cell with
 *            the lower id in the caller's (original) order, so that the
 *            renumbering does not change the orientation;
 *   then 3 * (tile + n_h1) int16 values, two per word, low half first: for
 *            each tile slot and then each H1 cell, and each local edge k,
 *            (slot' << 3) | (k' << 1) | own for a neighbour in slot' whose
 *            local edge is k' (own = 1 when this cell is the left state), or
 *            -1 - tag on the domain boundary (unused slots: -1, a wall);
 * padded with zeros to a multiple of 8 words.  Slots are 11-bit fields, so
 * tile + n_halo must not exceed 2047 for any tile.
 */
#ifndef SWE_TILE_PLAN_H
#define SWE_TILE_PLAN_H

#include "swe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Size of the plan of mesh m with `tile` cells per tile.  tile must be a
 * power of two within 32 .. 1024.  Outputs (any may be NULL): number of
 * tiles; the most halo cells, H1 cells and words of any one tile; the total
 * number of words.
 * Errors: SWE_ERR_ARG (NULL mesh, bad tile size, a tile whose slots exceed
 * the 11-bit fields: renumber the mesh or take a smaller tile),
 * SWE_ERR_NOMEM. */
int swe_tile_plan_info(const swe_mesh *m, int tile, int64_t *n_tiles, int32_t *hmax, int32_t *h1max,
                       int32_t *wmax, int64_t *n_words);

/* Copy the plan into caller-owned buffers: hdr[8 * n_tiles] and
 * words[n_words] (the sizes that swe_tile_plan_info gives; either pointer
 * may be NULL).  Errors as swe_tile_plan_info. */
int swe_tile_plan_export(const swe_mesh *m, int tile, int32_t *hdr, int32_t *words);

#ifdef __cplusplus
}
#endif

#endif /* SWE_TILE_PLAN_H */
