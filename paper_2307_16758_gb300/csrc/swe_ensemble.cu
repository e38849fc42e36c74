// Batched ensemble kernels: one launch advances every member of an ensemble
// of independent meshes by one explicit step.  The grid is the concatenation
// of the members' grids; a block reads its member and its block index within
// the member from a per-block table (one 8-byte load, no search and no
// barrier) and runs the same per-mesh device code as the single-mesh
// kernels, with that member's arguments (its own buffers, CFL slots and time
// step).
#include <cuda_runtime.h>

#include "swe_ensemble.h"
#include "swe_device.cuh"
#include "swe_split.cuh"

namespace {
using namespace swe_dev;

// Register caps as for the single-mesh kernels (swe_kernels.cu): FP32 MUSCL
// prep at 40, the FP32 flux kernels at 32 (WAF at 48).  SCHEME
// FLUX_MUSCL_HR2 is the LSQ MUSCL scheme with the second-order hydrostatic
// reconstruction (its prep reconstructs h as well: 48 registers).
template <typename T, int SCHEME>
__global__ void __maxnreg__((sizeof(T) != 4 ? 255 : SCHEME == SWE_SCHEME_MUSCL ? 40 : SCHEME == FLUX_MUSCL_HR2 ? 48 : 255))
    k_prep_ens(const EnsEntry<T> *__restrict__ tab, const int2 *__restrict__ blk, int phase)
{
    const int2 b = blk[blockIdx.x];
    const EnsEntry<T> &e = tab[b.x];
    const StepArgs<T> &a = e.a[phase];
    const int i = b.y * (int)blockDim.x + (int)threadIdx.x;
    if (i >= a.m.n) return;
    if (SCHEME == FLUX_MUSCL_HR2) prep_muscl_cell<T, 4>(a, i, e.F);
    else if (SCHEME == SWE_SCHEME_MUSCL) prep_muscl_cell(a, i, e.F);
    else if (SCHEME == SWE_SCHEME_MUSCL_EDGE) prep_muscl_edge_cell(a, i, e.F);
    else prep_waf_cell(a, i, e.F, e.U);
}

template <typename T, int SCHEME>
__global__ void __maxnreg__((sizeof(T) != 4 ? 255 : SCHEME == SWE_SCHEME_WAF ? 48 : 32))
    k_flux_ens(const EnsEntry<T> *__restrict__ tab, const int2 *__restrict__ blk, int phase)
{
    const int2 b = blk[blockIdx.x];
    flux_block<T, SCHEME>(tab[b.x].a[phase], b.y);
}

}  // namespace

template <typename T>
cudaError_t launch_ensemble(int scheme, bool hr2, bool fused, const EnsEntry<T> *tab, const int2 *blk, int phase,
                            int grid, int block, const TileArgs &room, cudaStream_t s)
{
    if (fused) return launch_tile_ensemble<T>(scheme, tab, blk, phase, grid, block, room, s);
    if (scheme == SWE_SCHEME_MUSCL && hr2) {
        k_prep_ens<T, FLUX_MUSCL_HR2><<<grid, block, 0, s>>>(tab, blk, phase);
        k_flux_ens<T, FLUX_MUSCL_HR2><<<grid, block, 0, s>>>(tab, blk, phase);
    } else if (scheme == SWE_SCHEME_MUSCL) {
        k_prep_ens<T, SWE_SCHEME_MUSCL><<<grid, block, 0, s>>>(tab, blk, phase);
        k_flux_ens<T, SWE_SCHEME_MUSCL><<<grid, block, 0, s>>>(tab, blk, phase);
    } else if (scheme == SWE_SCHEME_MUSCL_EDGE) {
        k_prep_ens<T, SWE_SCHEME_MUSCL_EDGE><<<grid, block, 0, s>>>(tab, blk, phase);
        k_flux_ens<T, SWE_SCHEME_MUSCL><<<grid, block, 0, s>>>(tab, blk, phase);
    } else if (scheme == SWE_SCHEME_WAF) {
        k_prep_ens<T, SWE_SCHEME_WAF><<<grid, block, 0, s>>>(tab, blk, phase);
        k_flux_ens<T, SWE_SCHEME_WAF><<<grid, block, 0, s>>>(tab, blk, phase);
    } else {
        k_flux_ens<T, SWE_SCHEME_HLLC><<<grid, block, 0, s>>>(tab, blk, phase);
    }
    return cudaGetLastError();
}

template <typename T> cudaError_t ensemble_prepare(int scheme, bool fused, size_t smem)
{
    return fused ? tile_ensemble_prepare<T>(scheme, smem) : cudaSuccess;
}

namespace {
template <typename K> int max_threads(K kern)
{
    cudaFuncAttributes fa{};
    return cudaFuncGetAttributes(&fa, kern) == cudaSuccess ? fa.maxThreadsPerBlock : 0;
}
template <typename T, int SCHEME, bool PREP> int split_ens_max_threads()
{
    const int f = max_threads(k_flux_ens<T, SCHEME>);
    if (!PREP) return f;
    const int p = max_threads(k_prep_ens<T, SCHEME>);
    return p < f ? p : f;
}
}  // namespace

template <typename T> int ensemble_max_threads(int scheme, bool hr2, bool fused)
{
    if (fused) return tile_ensemble_max_threads<T>(scheme);
    if (scheme == SWE_SCHEME_MUSCL && hr2) return split_ens_max_threads<T, FLUX_MUSCL_HR2, true>();
    if (scheme == SWE_SCHEME_MUSCL) return split_ens_max_threads<T, SWE_SCHEME_MUSCL, true>();
    if (scheme == SWE_SCHEME_MUSCL_EDGE) {
        const int p = max_threads(k_prep_ens<T, SWE_SCHEME_MUSCL_EDGE>), f = max_threads(k_flux_ens<T, SWE_SCHEME_MUSCL>);
        return p < f ? p : f;
    }
    if (scheme == SWE_SCHEME_WAF) return split_ens_max_threads<T, SWE_SCHEME_WAF, true>();
    return split_ens_max_threads<T, SWE_SCHEME_HLLC, false>();
}
template int ensemble_max_threads<float>(int, bool, bool);
template int ensemble_max_threads<double>(int, bool, bool);

template cudaError_t launch_ensemble<float>(int, bool, bool, const EnsEntry<float> *, const int2 *, int, int, int,
                                            const TileArgs &, cudaStream_t);
template cudaError_t launch_ensemble<double>(int, bool, bool, const EnsEntry<double> *, const int2 *, int, int, int,
                                             const TileArgs &, cudaStream_t);
template cudaError_t ensemble_prepare<float>(int, bool, size_t);
template cudaError_t ensemble_prepare<double>(int, bool, size_t);
