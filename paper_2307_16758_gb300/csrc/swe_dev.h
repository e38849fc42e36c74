// Device data layout and kernel launch interface (shared by the host API and
// the CUDA translation unit).  Cells are in the library's (renumbered) order;
// every per-cell array is structure-of-arrays except the small vector records.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/swe.h"

// 2- and 4-vectors of the compute type.  The 4-vector of doubles is 32-byte
// aligned so that one record is one 32-byte sector.
template <typename T> struct Vec2 { T x, y; };
template <> struct alignas(8) Vec2<float> { float x, y; };
template <> struct alignas(16) Vec2<double> { double x, y; };
template <typename T> struct Vec4 { T x, y, z, w; };
template <> struct alignas(16) Vec4<float> { float x, y, z, w; };
template <> struct alignas(32) Vec4<double> { double x, y, z, w; };

// Per-state scalars updated on the device.  smax[] is a ring of three slots
// holding the bit pattern of a non-negative wave speed in the compute type
// (float bits zero-extended in FP32, double bits in FP64; either way atomicMax
// on the integer is a max on the values): step k reads slot k%3, writes slot
// (k+1)%3 and clears slot (k+2)%3.
struct DevScalars {
    unsigned long long smax[3];
    double t;            // simulated time
    long long steps;     // steps taken
    double clipped;      // mass added by clipping negative depths
    double bnd_in;       // net mass that entered through the boundary
    int status;          // ST_* bits
    int pad;
};

// Status bits: a non-finite value, no wet cell for the CFL rule, a tile's edge
// list outgrew its plan, a bulk copy into shared memory did not complete.
enum { ST_NONFINITE = 1, ST_DRY = 2, ST_TILE = 4, ST_TIMEOUT = 8 };
enum { MODE_EULER = 0, MODE_STAGE = 1 };

template <typename T> struct DevMesh {
    int64_t n;
    const int32_t *nbr;        // [3n] packed neighbour words (see swe_mesh.h)
    const Vec2<T> *ln;         // [3n] outward normal times edge length
    const Vec2<T> *dd;         // [3n] centroid offset to the neighbour
    const T *z;                // [n] bed elevation
    const T *nman;             // [n] Manning coefficient (may be NULL)
    const double *area;        // [n] FP64 area (mass totals only)
};

template <typename T> struct StepArgs {
    DevMesh<T> m;
    const T *h, *hu, *hv;       // state in
    T *ho, *huo, *hvo;          // state out
    const Vec4<T> *F;           // MUSCL: face values [3n] (eta, u, v, z); WAF: centre values [n] (h, u, v, z);
                                //   written for wet cells only (a dry cell's are built from its h and z)
    const Vec4<T> *U;           // WAF: upwind means [3n] (h or eta, u, v, -), wet cells only
    DevScalars *sc;
    const double *dtv;          // replayed time step (NULL: CFL rule)
    double *dt_hist;            // ring of the last SWE_DT_HISTORY time steps
    int slot_cur, slot_next, slot_clear;
    int mode;                   // MODE_EULER or MODE_STAGE (first Heun stage or second without averaging)
    T cfl_rmin;                 // cfl * r_min (global CFL form) or cfl (local form)
    int cfl_local;              // 1: the published wave speed is s_i / r_i (local CFL form)
    T g, h_eps, r_eps;
    T beta;                     // MUSCL_EDGE slope-limiter parameter
    const int32_t *cells;       // boundary-first schedule: the flux launch covers these cells
    int n_list;                 //   (n_list of them) instead of 0..n-1
    int no_advance;             // 1: not the step's last flux launch (time is advanced by the last)
    int hr2;                    // 1: second-order hydrostatic reconstruction (linear bed, MUSCL)
    int waf_surface;            // 1: WAF ratios on the free surface instead of the depth
    int waf_limiter;
    T qlen[SWE_MAX_GROUPS];     // inflow discharge per unit length [m^2/s]
    T level[SWE_MAX_GROUPS];    // fixed free-surface levels [m]
};

// One-pass tile step (swe_tile.cu, plan built by swe_tiles.cpp, layout in
// swe_tiles.h): tile b is the cells [b * tile, min((b + 1) * tile, n)), one
// per thread; the maxima over the tiles size the block's shared memory.
struct TileArgs {
    int64_t n_tiles;
    const int32_t *plan_hdr;     // [8 n_tiles] per tile: plan-word offset, halo cells, H1 cells, edges,
                                 //   crossing edges, plan words
    const int32_t *plan_words;   // halo ids, edge records, local neighbour words
    int tile;
    int hmax, h1max, wmax;       // room for halo cells, H1 cells and plan words
    int grid;                    // blocks of the persistent launch (resident blocks on this GPU)
};

// Launchers (defined in swe_kernels.cu and swe_tile.cu).  All launches go to `stream`.
template <typename T>
cudaError_t launch_prep(int scheme, const StepArgs<T> &a, Vec4<T> *F, Vec4<T> *U, int block, cudaStream_t s);
template <typename T>
cudaError_t launch_flux(int scheme, const StepArgs<T> &a, int block, cudaStream_t s);
template <typename T>
cudaError_t launch_smax(const StepArgs<T> &a, int slot, int block, cudaStream_t s);
template <typename T>
cudaError_t launch_heun_avg(const StepArgs<T> &a, const T *h0, const T *hu0, const T *hv0,
                            int block, cudaStream_t s);
template <typename T>
cudaError_t launch_mass(const DevMesh<T> &m, const T *h, double *partials, int n_partials, double *out,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_scatter_in(int64_t n, const int32_t *perm, const double *src, T *h, T *hu, T *hv,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_gather_out(int64_t n, const int32_t *perm, const T *h, const T *hu, const T *hv,
                              double *dst, cudaStream_t s);
template <typename T>
cudaError_t launch_convert(int64_t n, const double *src, T *dst, cudaStream_t s);

// The tile step: one launch advances every tile.
template <typename T> cudaError_t launch_tile(int scheme, const StepArgs<T> &a, const TileArgs &t, cudaStream_t s);
template <typename T> size_t tile_smem_bytes(const TileArgs &t);
template <typename T> int tile_max_threads(int scheme);     // launch limit of the tile kernel (registers)
template <typename T> int tile_grid(int scheme, int tile, size_t smem);   // resident blocks (persistent grid)
template <typename T> cudaError_t tile_prepare(int scheme, size_t smem);   // shared-memory attribute, once

// Boundary-first schedule: flux over a list of cells (a.cells, a.n_list), and
// the halo of every part packed (SoA, [3][n]) from the new state.
template <typename T> cudaError_t launch_flux_list(int scheme, const StepArgs<T> &a, int block, cudaStream_t s);
template <typename T>
cudaError_t launch_pack_halo(int64_t n, const int32_t *cells, const T *h, const T *hu, const T *hv, T *buf,
                             cudaStream_t s);
template <typename T> int split_max_threads(int scheme, bool hr2);     // launch limit of the flux kernels

int mass_partials_needed(int64_t n);
