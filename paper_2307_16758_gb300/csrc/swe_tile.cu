// One-pass tile step of the explicit finite-volume scheme (Sec. 6.1-6.2):
// one persistent launch per time step; each block advances tiles of
// consecutive cells with the tile's face values and edge contributions in shared memory
// and every Riemann problem inside the tile solved once.  See swe_tile.cuh
// for the phases.
#include <cuda_runtime.h>

#include "swe_dev.h"
#include "swe_device.cuh"
#include "swe_ensemble.h"
#include "swe_tile.cuh"

namespace {
using namespace swe_dev;

// Shared-memory room of a launch.
__host__ __device__ inline TileDims dims_of(const TileArgs &t)
{
    return TileDims{t.tile, t.hmax, t.h1max, t.wmax};
}

// Tiles of one mesh: g is the tile index.
template <typename T> struct OneMesh {
    const StepArgs<T> &a;
    const TileArgs &t;
    __device__ const StepArgs<T> &args(int64_t) const { return a; }
    __device__ const TileArgs &targs(int64_t) const { return t; }
    __device__ int64_t tile(int64_t g) const { return g; }
};

// Tiles of an ensemble: global tile g is tile blk[g].y of member blk[g].x.
template <typename T> struct Members {
    const EnsEntry<T> *tab;
    const int2 *blk;
    int phase;
    __device__ const StepArgs<T> &args(int64_t g) const { return tab[blk[g].x].a[phase]; }
    __device__ const TileArgs &targs(int64_t g) const { return tab[blk[g].x].t; }
    __device__ int64_t tile(int64_t g) const { return blk[g].y; }
};

// FP32 register cap: the pipeline's shared memory, not registers, bounds the
// blocks per SM, so the tile code runs without spills.
template <typename T, int SCHEME>
__global__ void __maxnreg__((sizeof(T) == 4 ? 96 : 255)) k_tile(StepArgs<T> a, TileArgs t)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    tile_loop<T, SCHEME>(OneMesh<T>{a, t}, t.n_tiles, dims_of(t), smem_raw);
}

// Batched: the library's device code is compiled without floating-point
// contraction (every fused multiply-add is written out), so this kernel and
// the single-mesh one give a member the same bits as stepping it alone.
// d: the members' largest room.
template <typename T, int SCHEME>
__global__ void __maxnreg__((sizeof(T) == 4 ? 96 : 255))
    k_tile_ens(const EnsEntry<T> *__restrict__ tab, const int2 *__restrict__ blk, int64_t n_total, int phase,
               TileDims d)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    tile_loop<T, SCHEME>(Members<T>{tab, blk, phase}, n_total, d, smem_raw);
}

template <typename T> auto tile_kernel(int scheme)
{
    return scheme == SWE_SCHEME_HLLC ? k_tile<T, SWE_SCHEME_HLLC> : k_tile<T, SWE_SCHEME_MUSCL>;
}

template <typename T> auto tile_ens_kernel(int scheme)
{
    return scheme == SWE_SCHEME_HLLC ? k_tile_ens<T, SWE_SCHEME_HLLC> : k_tile_ens<T, SWE_SCHEME_MUSCL>;
}

// Resident blocks of a persistent launch: blocks per SM at this block size
// and shared memory, times the SMs.
template <typename K> int persistent_grid(K kern, int block, size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem) != cudaSuccess) return 0;
    return per_sm * sms;
}

// Let kernel `kern` launch with as much dynamic shared memory as the device
// allows a block beside the kernel's static shared memory (`smem` bytes are
// needed).  The limit is a property of the kernel on the current device,
// shared by every state: it is set to that maximum, never to one state's own
// need, so that configuring a state with a smaller tile plan cannot lower
// what another state launches with.  Called when a state or an ensemble is
// configured, outside any capture.
template <typename K> cudaError_t allow_dynamic_smem(K kern, size_t smem)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (smem > room) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

}  // namespace

template <typename T> size_t tile_smem_bytes(const TileArgs &t)
{
    return TileSmem<T>::bytes(dims_of(t));
}

template <typename T> int tile_max_threads(int scheme)
{
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, tile_kernel<T>(scheme)) != cudaSuccess) return 0;
    return fa.maxThreadsPerBlock;
}

template <typename T> cudaError_t tile_prepare(int scheme, size_t smem)
{
    return allow_dynamic_smem(tile_kernel<T>(scheme), smem);
}

template <typename T> cudaError_t launch_tile(int scheme, const StepArgs<T> &a, const TileArgs &t, cudaStream_t s)
{
    if (scheme != SWE_SCHEME_MUSCL && scheme != SWE_SCHEME_HLLC) return cudaErrorInvalidValue;
    const size_t smem = tile_smem_bytes<T>(t);
    const int64_t grid = t.grid < t.n_tiles ? t.grid : t.n_tiles;
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    tile_kernel<T>(scheme)<<<(unsigned)grid, t.tile, smem, s>>>(a, t);
    return cudaGetLastError();
}

template <typename T> int tile_grid(int scheme, int tile, size_t smem)
{
    return persistent_grid(tile_kernel<T>(scheme), tile, smem);
}

template <typename T>
cudaError_t launch_tile_ensemble(int scheme, const EnsEntry<T> *tab, const int2 *blk, int phase, int n_total, int block,
                                 const TileArgs &room, cudaStream_t s)
{
    if (scheme != SWE_SCHEME_MUSCL && scheme != SWE_SCHEME_HLLC) return cudaErrorInvalidValue;
    const size_t smem = tile_smem_bytes<T>(room);
    int grid = persistent_grid(tile_ens_kernel<T>(scheme), block, smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if (grid > n_total) grid = n_total;
    tile_ens_kernel<T>(scheme)<<<grid, block, smem, s>>>(tab, blk, (int64_t)n_total, phase, dims_of(room));
    return cudaGetLastError();
}

template <typename T> cudaError_t tile_ensemble_prepare(int scheme, size_t smem)
{
    return allow_dynamic_smem(tile_ens_kernel<T>(scheme), smem);
}

template <typename T> int tile_ensemble_max_threads(int scheme)
{
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, tile_ens_kernel<T>(scheme)) != cudaSuccess) return 0;
    return fa.maxThreadsPerBlock;
}

template cudaError_t launch_tile_ensemble<float>(int, const EnsEntry<float> *, const int2 *, int, int, int,
                                                 const TileArgs &, cudaStream_t);
template cudaError_t launch_tile_ensemble<double>(int, const EnsEntry<double> *, const int2 *, int, int, int,
                                                  const TileArgs &, cudaStream_t);
template int tile_grid<float>(int, int, size_t);
template int tile_grid<double>(int, int, size_t);
template cudaError_t tile_ensemble_prepare<float>(int, size_t);
template cudaError_t tile_ensemble_prepare<double>(int, size_t);
template int tile_ensemble_max_threads<float>(int);
template int tile_ensemble_max_threads<double>(int);
template size_t tile_smem_bytes<float>(const TileArgs &);
template size_t tile_smem_bytes<double>(const TileArgs &);
template int tile_max_threads<float>(int);
template int tile_max_threads<double>(int);
template cudaError_t tile_prepare<float>(int, size_t);
template cudaError_t tile_prepare<double>(int, size_t);
template cudaError_t launch_tile<float>(int, const StepArgs<float> &, const TileArgs &, cudaStream_t);
template cudaError_t launch_tile<double>(int, const StepArgs<double> &, const TileArgs &, cudaStream_t);
