// Batched ensemble: the per-member table and the launcher (swe_ensemble.cu).
#pragma once
#include "swe_dev.h"

// One member of a batched ensemble: its step arguments for each phase of the
// launch pattern (steps taken mod 6: ping-pong buffer and CFL slot ring),
// its tile plan and its split-kernel scratch.
template <typename T> struct EnsEntry {
    StepArgs<T> a[6];
    TileArgs t;
    Vec4<T> *F, *U;
};

// Block b of a batched launch runs block blk[b].y of member blk[b].x.  One
// launch (two for the split kernels with a prep pass) advances every member
// by one step of the given phase.  hr2: the members use the second-order
// hydrostatic reconstruction (all or none of them).  room: the tile kernel's
// shared-memory room, the members' largest.
template <typename T>
cudaError_t launch_ensemble(int scheme, bool hr2, bool fused, const EnsEntry<T> *tab, const int2 *blk, int phase,
                            int grid, int block, const TileArgs &room, cudaStream_t s);
template <typename T> cudaError_t ensemble_prepare(int scheme, bool fused, size_t smem);
// The batched tile kernel (swe_tile.cu, beside the single-mesh one so that both run one compiled body).
template <typename T>
cudaError_t launch_tile_ensemble(int scheme, const EnsEntry<T> *tab, const int2 *blk, int phase, int n_total, int block,
                                 const TileArgs &room, cudaStream_t s);
template <typename T> cudaError_t tile_ensemble_prepare(int scheme, size_t smem);
template <typename T> int tile_ensemble_max_threads(int scheme);
// The largest block that every batched kernel of this configuration launches with.
template <typename T> int ensemble_max_threads(int scheme, bool hr2, bool fused);
