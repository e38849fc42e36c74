// One-pass tile step of the explicit finite-volume scheme (Sec. 6.1-6.2):
// one launch per time step; each block advances one tile of consecutive
// cells with the tile's face values and edge contributions in shared memory
// and every Riemann problem inside the tile solved once.  See swe_tile.cuh
// for the phases.
#include <cuda_runtime.h>

#include "swe_dev.h"
#include "swe_device.cuh"
#include "swe_ensemble.h"
#include "swe_tile.cuh"

namespace {
using namespace swe_dev;

template <typename T, int SCHEME>
__global__ void __maxnreg__((sizeof(T) == 4 ? 48 : 255))
    k_tile(StepArgs<T> a, TileArgs t)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    tile_step<T, SCHEME>(a, blockIdx.x, t.emax, t.xmax, smem_raw);
}

// Batched: block b runs tile blk[b].y of member blk[b].x.  The library's
// device code is compiled without floating-point contraction (every fused
// multiply-add is written out), so this kernel and the single-mesh one give
// a member the same bits as stepping it alone.
template <typename T, int SCHEME>
__global__ void __maxnreg__((sizeof(T) == 4 ? 48 : 255))
    k_tile_ens(const EnsEntry<T> *__restrict__ tab, const int2 *__restrict__ blk, int phase)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int2 b = blk[blockIdx.x];
    const EnsEntry<T> &e = tab[b.x];
    tile_step<T, SCHEME>(e.a[phase], b.y, e.t.emax, e.t.xmax, smem_raw);
}

template <typename T> auto tile_kernel(int scheme)
{
    return scheme == SWE_SCHEME_HLLC ? k_tile<T, SWE_SCHEME_HLLC> : k_tile<T, SWE_SCHEME_MUSCL>;
}

template <typename T> auto tile_ens_kernel(int scheme)
{
    return scheme == SWE_SCHEME_HLLC ? k_tile_ens<T, SWE_SCHEME_HLLC> : k_tile_ens<T, SWE_SCHEME_MUSCL>;
}

}  // namespace

template <typename T> size_t tile_smem_bytes(int tile, int emax, int xmax)
{
    return TileSmem<T>::bytes(tile, emax, xmax);
}

template <typename T> int tile_max_threads(int scheme)
{
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, tile_kernel<T>(scheme)) != cudaSuccess) return 0;
    return fa.maxThreadsPerBlock;
}

// Allow the tile kernel `smem` bytes of dynamic shared memory (called when a
// state is configured, outside any stream capture).
template <typename T> cudaError_t tile_prepare(int scheme, size_t smem)
{
    auto kern = tile_kernel<T>(scheme);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

template <typename T> cudaError_t launch_tile(int scheme, const StepArgs<T> &a, const TileArgs &t, cudaStream_t s)
{
    if (scheme != SWE_SCHEME_MUSCL && scheme != SWE_SCHEME_HLLC) return cudaErrorInvalidValue;
    const size_t smem = tile_smem_bytes<T>(t.tile, t.emax, t.xmax);
    tile_kernel<T>(scheme)<<<(unsigned)t.n_tiles, t.tile, smem, s>>>(a, t);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tile_ensemble(int scheme, const EnsEntry<T> *tab, const int2 *blk, int phase, int grid, int block,
                                 size_t smem, cudaStream_t s)
{
    if (scheme != SWE_SCHEME_MUSCL && scheme != SWE_SCHEME_HLLC) return cudaErrorInvalidValue;
    tile_ens_kernel<T>(scheme)<<<grid, block, smem, s>>>(tab, blk, phase);
    return cudaGetLastError();
}

template <typename T> cudaError_t tile_ensemble_prepare(int scheme, size_t smem)
{
    auto kern = tile_ens_kernel<T>(scheme);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

template <typename T> int tile_ensemble_max_threads(int scheme)
{
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, tile_ens_kernel<T>(scheme)) != cudaSuccess) return 0;
    return fa.maxThreadsPerBlock;
}

template cudaError_t launch_tile_ensemble<float>(int, const EnsEntry<float> *, const int2 *, int, int, int, size_t,
                                                 cudaStream_t);
template cudaError_t launch_tile_ensemble<double>(int, const EnsEntry<double> *, const int2 *, int, int, int, size_t,
                                                  cudaStream_t);
template cudaError_t tile_ensemble_prepare<float>(int, size_t);
template cudaError_t tile_ensemble_prepare<double>(int, size_t);
template int tile_ensemble_max_threads<float>(int);
template int tile_ensemble_max_threads<double>(int);
template size_t tile_smem_bytes<float>(int, int, int);
template size_t tile_smem_bytes<double>(int, int, int);
template int tile_max_threads<float>(int);
template int tile_max_threads<double>(int);
template cudaError_t tile_prepare<float>(int, size_t);
template cudaError_t tile_prepare<double>(int, size_t);
template cudaError_t launch_tile<float>(int, const StepArgs<float> &, const TileArgs &, cudaStream_t);
template cudaError_t launch_tile<double>(int, const StepArgs<double> &, const TileArgs &, cudaStream_t);
