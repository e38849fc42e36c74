// Fused tile kernel: one launch per time step does the whole second-order
// step (MUSCL face values or WAF upwind data, edge fluxes, update, friction
// and the wave-speed reduction) for a tile of consecutive (Morton-ordered)
// cells, so face values never go to HBM and every Riemann problem inside a
// tile is solved once.
//
// A block holds a tile (nc cells, slots 0..nc-1) and its halo (H cells,
// slots nc..nc+H-1), nc + H <= blockDim.x, so each thread owns one slot:
//   phase 0: the slot's state -> primitives in shared memory;
//   phase 1: the slot's face values (MUSCL) or upwind means (WAF): tile cells
//            read their neighbours from shared memory, halo cells gather
//            theirs from global memory;
//   phase 2: the tile's edge list, one thread per edge: hydrostatic
//            reconstruction and Riemann flux once per edge, contributions to
//            both sides written to shared memory;
//   phase 3: each tile cell adds its three contributions in edge order
//            (boundary edges computed here) and updates.
// The per-edge and per-cell arithmetic is the same device code as the split
// kernels (swe_device.cuh), so both give the same bits.
#include <cuda_runtime.h>

#include "swe_dev.h"
#include "swe_device.cuh"
#include "swe_fused.cuh"

namespace {
using namespace swe_dev;

template <typename T, int SCHEME>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_fused(StepArgs<T> a, FusedArgs f)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    fused_tile<T, SCHEME>(a, f, blockIdx.x, smem_raw);
}

}  // namespace

template <typename T> int fused_max_threads(int scheme)
{
    cudaFuncAttributes fa{};
    cudaError_t e = scheme == SWE_SCHEME_WAF ? cudaFuncGetAttributes(&fa, k_fused<T, SWE_SCHEME_WAF>)
                                             : cudaFuncGetAttributes(&fa, k_fused<T, SWE_SCHEME_MUSCL>);
    return e == cudaSuccess ? fa.maxThreadsPerBlock : 0;
}

// Allow the kernel the dynamic shared memory of a block of `block` threads
// (called once when a state is set up, outside any stream capture).
template <typename T> cudaError_t fused_prepare(int scheme, int block)
{
    const int smem = (int)fused_smem_bytes<T>(scheme, block);
    auto kern = scheme == SWE_SCHEME_WAF ? k_fused<T, SWE_SCHEME_WAF> : k_fused<T, SWE_SCHEME_MUSCL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

template <typename T> size_t fused_smem_bytes(int scheme, int block)
{
    (void)scheme;
    return (size_t)block * (4 * sizeof(Vec4<T>) + 9 * sizeof(T));
}

template <typename T>
cudaError_t launch_fused(int scheme, const StepArgs<T> &a, const FusedArgs &f, cudaStream_t s)
{
    const size_t smem = fused_smem_bytes<T>(scheme, f.block);
    if (scheme == SWE_SCHEME_MUSCL) {
        k_fused<T, SWE_SCHEME_MUSCL><<<f.n_tiles, f.block, smem, s>>>(a, f);
    } else if (scheme == SWE_SCHEME_WAF) {
        k_fused<T, SWE_SCHEME_WAF><<<f.n_tiles, f.block, smem, s>>>(a, f);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_fused<float>(int, const StepArgs<float> &, const FusedArgs &, cudaStream_t);
template cudaError_t launch_fused<double>(int, const StepArgs<double> &, const FusedArgs &, cudaStream_t);
template size_t fused_smem_bytes<float>(int, int);
template size_t fused_smem_bytes<double>(int, int);
template int fused_max_threads<float>(int);
template cudaError_t fused_prepare<float>(int, int);
template cudaError_t fused_prepare<double>(int, int);
template int fused_max_threads<double>(int);
