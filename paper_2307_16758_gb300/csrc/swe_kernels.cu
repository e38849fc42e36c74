// CUDA kernels of the explicit finite-volume shallow-water step (sm_103a).
//
// One time step (Sec. 6.1 of Delmas & Soulaimani, arXiv 2307.16758):
//   prep  : per cell, the values each cell shows at the midpoints of its three
//           edges -- MUSCL: least-squares gradients of (eta, u, v) limited
//           with Barth-Jespersen; WAF: the cell's primitives and, per edge,
//           the mean of its two other neighbours (the upwind data of Sec. 6.2.2).
//   flux  : per cell, for its three edges: hydrostatic reconstruction, the
//           HLLC (Sec. 6.2.1) or WAF (Sec. 6.2.2) flux in the canonical edge
//           frame, boundary fluxes (Sec. 6.1), the explicit Euler update,
//           depth clipping, point-implicit Manning friction, and the wave
//           speed of the new state reduced (warp shuffle, then one atomicMax
//           per block) for the next CFL time step.
// The first-order HLLC path needs no prep: it gathers the neighbour state.
//
// Both sides of an interior edge evaluate the same canonical flux (left
// state = the cell with the lower original id, normal pointing from left to
// right) from the same inputs, so the mass flux is bitwise antisymmetric.
#include <cuda_runtime.h>

#include <algorithm>

#include "swe_dev.h"
#include "swe_device.cuh"
#include "swe_split.cuh"

namespace {
using namespace swe_dev;

// ---------------------------------------------------------------------------
// prep kernels
// ---------------------------------------------------------------------------

// MUSCL face values: unweighted least squares over the face neighbours, then
// Barth-Jespersen limiting at the three edge midpoints.  Zero gradient if the
// cell or a neighbour is dry or the 2x2 system is singular.  NQ = 4 also
// reconstructs h (second-order hydrostatic reconstruction).  FP32 register
// caps: 40 (twelve of the default 128-thread blocks per SM) and 48 for
// NQ = 4 (ten).
template <typename T, int NQ = 3>
__global__ void __maxnreg__((sizeof(T) == 4 ? (NQ == 3 ? 40 : 48) : 255)) k_prep_muscl(StepArgs<T> a, Vec4<T> *F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.m.n) prep_muscl_cell<T, NQ>(a, i, F);
}

// The paper's MUSCL (Sec. 6.2.3): edge-upwind slopes, beta-limited.
template <typename T>
__global__ void k_prep_muscl_edge(StepArgs<T> a, Vec4<T> *F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.m.n) prep_muscl_edge_cell(a, i, F);
}

template <typename T>
__global__ void k_prep_waf(StepArgs<T> a, Vec4<T> *P, Vec4<T> *U)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.m.n) prep_waf_cell(a, i, P, U);
}

// Register cap of the FP32 flux kernels.  They wait on memory more than they
// compute, so resident warps pay more than spills cost: 32 registers fit
// eight 256-thread blocks per SM (every warp slot), 40 six, 48 five.  On the
// 13M river the LSQ MUSCL flux kernel runs 0.281 ms at 32 (about 90 bytes of
// spills), 0.303 at 40, 0.326 at 48 (none); HLLC 0.238, 0.257, 0.290; with
// the second-order hydrostatic reconstruction 0.283 at 32, 0.297 at 40.  WAF
// keeps 48: its limiter state spills (0.394 ms at 48, 0.454 at 40, 0.493 at
// 32).  The FP64 instances are bound by the FP64 units and left to the
// compiler.
template <typename T, int SCHEME> constexpr int flux_maxnreg()
{
    return sizeof(T) != 4 ? 255 : (SCHEME == SWE_SCHEME_WAF ? 48 : 32);
}

template <typename T, int SCHEME>
__global__ void __maxnreg__((flux_maxnreg<T, SCHEME>())) k_flux(StepArgs<T> a)
{
    flux_block<T, SCHEME>(a, blockIdx.x);
}

template <typename T, int SCHEME>
__global__ void __maxnreg__((flux_maxnreg<T, SCHEME>())) k_flux_list(StepArgs<T> a)
{
    flux_block<T, SCHEME, true>(a, blockIdx.x);
}

// Halo of the boundary-first schedule: the new state of the listed cells,
// packed as [h..., hu..., hv...] (what each part would receive).
template <typename T>
__global__ void k_pack_halo(int64_t n, const int32_t *cells, const T *h, const T *hu, const T *hv, T *buf)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) {
        const int32_t c = cells[s];
        buf[s] = h[c]; buf[n + s] = hu[c]; buf[2 * n + s] = hv[c];
    }
}

// Wave speed of the current state into slot `slot` (CFL rule of Sec. 6.1).
template <typename T>
__global__ void k_smax(StepArgs<T> a, int slot)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T s = T(0);
    if (i < a.m.n) {
        T h = a.h[i];
        if (h > a.h_eps) s = cfl_speed(a, i, wave_speed(a.g, h, a.hu[i], a.hv[i]));
    }
    block_publish<T>(s, T(0), T(0), a.sc, slot, true, 1.0);
}

// Heun: U^{n+1} = (U^n + U2) / 2 with U2 = E(E(U^n)); then the wave speed.
template <typename T>
__global__ void k_heun_avg(StepArgs<T> a, const T *h0, const T *hu0, const T *hv0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T s = T(0);
    if (i < a.m.n) {
        T h = T(0.5) * (h0[i] + a.h[i]), hu = T(0.5) * (hu0[i] + a.hu[i]), hv = T(0.5) * (hv0[i] + a.hv[i]);
        a.ho[i] = h; a.huo[i] = hu; a.hvo[i] = hv;
        if (h > a.h_eps) s = cfl_speed(a, i, wave_speed(a.g, h, hu, hv));
    }
    block_publish<T>(s, T(0), T(0), a.sc, a.slot_next, true, 1.0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool dry;
        T dt = step_dt(a, &dry);
        a.dt_hist[a.sc->steps % SWE_DT_HISTORY] = (double)dt;
        a.sc->t += (double)dt;
        a.sc->steps += 1;
        a.sc->smax[a.slot_clear] = 0ULL;
    }
}

// Mass: per-block FP64 compensated partial sums (value and lost low-order
// part) in a fixed tree order, then one block merges the partials in a fixed
// order (deterministic; the total is within a few ulp of the exact sum).
constexpr int MASS_BLOCK = 256;
constexpr int MASS_ITEMS = 8;

// Compensated (Neumaier) summation: (s, c) holds the sum s and the lost
// low-order part c; the total is s + c.
struct Comp { double s, c; };

__device__ __forceinline__ void comp_add(Comp &a, double x)
{
    const double t = __dadd_rn(a.s, x);
    a.c += fabs(a.s) >= fabs(x) ? __dadd_rn(__dsub_rn(a.s, t), x) : __dadd_rn(__dsub_rn(x, t), a.s);
    a.s = t;
}

__device__ __forceinline__ void comp_merge(Comp &a, const Comp &b)
{
    comp_add(a, b.s);
    a.c += b.c;
}

// Fixed-order tree over the block's (s, c) pairs; thread 0 ends with the total.
__device__ __forceinline__ Comp block_comp_sum(Comp v)
{
    __shared__ double ss[MASS_BLOCK], sc[MASS_BLOCK];
    ss[threadIdx.x] = v.s; sc[threadIdx.x] = v.c;
    __syncthreads();
    for (int o = MASS_BLOCK / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            Comp a{ss[threadIdx.x], sc[threadIdx.x]};
            comp_merge(a, Comp{ss[threadIdx.x + o], sc[threadIdx.x + o]});
            ss[threadIdx.x] = a.s; sc[threadIdx.x] = a.c;
        }
        __syncthreads();
    }
    return Comp{ss[0], sc[0]};
}

template <typename T>
__global__ void __launch_bounds__(MASS_BLOCK) k_mass_partial(DevMesh<T> m, const T *h, double *partials)
{
    const int64_t base = (int64_t)blockIdx.x * MASS_BLOCK * MASS_ITEMS;
    Comp v{0.0, 0.0};
    for (int q = 0; q < MASS_ITEMS; q++) {
        int64_t i = base + (int64_t)q * MASS_BLOCK + threadIdx.x;
        if (i < m.n) comp_add(v, __dmul_rn(m.area[i], (double)h[i]));
    }
    const Comp t = block_comp_sum(v);
    if (threadIdx.x == 0) { partials[2 * blockIdx.x] = t.s; partials[2 * blockIdx.x + 1] = t.c; }
}

__global__ void __launch_bounds__(MASS_BLOCK) k_mass_final(const double *partials, int n, double *out)
{
    Comp v{0.0, 0.0};
    for (int q = threadIdx.x; q < n; q += MASS_BLOCK) comp_merge(v, Comp{partials[2 * q], partials[2 * q + 1]});
    const Comp t = block_comp_sum(v);
    if (threadIdx.x == 0) out[0] = t.s + t.c;
}

// Original-order FP64 host layout <-> renumbered device state.
template <typename T>
__global__ void k_scatter_in(int64_t n, const int32_t *perm, const double *src, T *h, T *hu, T *hv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    h[i] = (T)src[o]; hu[i] = (T)src[n + o]; hv[i] = (T)src[2 * n + o];
}

template <typename T>
__global__ void k_gather_out(int64_t n, const int32_t *perm, const T *h, const T *hu, const T *hv, double *dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    dst[o] = (double)h[i]; dst[n + o] = (double)hu[i]; dst[2 * n + o] = (double)hv[i];
}

template <typename T>
__global__ void k_convert(int64_t n, const double *src, T *dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)src[i];
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

namespace {
template <typename K> int max_threads(K kern)
{
    cudaFuncAttributes fa{};
    return cudaFuncGetAttributes(&fa, kern) == cudaSuccess ? fa.maxThreadsPerBlock : 0;
}
template <typename T, int SCHEME> int flux_max_threads()
{
    const int a = max_threads(k_flux<T, SCHEME>), b = max_threads(k_flux_list<T, SCHEME>);
    return a < b ? a : b;
}
}  // namespace

// The largest block that the flux kernels (plain and list-driven) launch with.
template <typename T> int split_max_threads(int scheme, bool hr2)
{
    if (scheme == SWE_SCHEME_MUSCL && hr2) return flux_max_threads<T, FLUX_MUSCL_HR2>();
    if (scheme == SWE_SCHEME_MUSCL || scheme == SWE_SCHEME_MUSCL_EDGE) return flux_max_threads<T, SWE_SCHEME_MUSCL>();
    if (scheme == SWE_SCHEME_WAF) return flux_max_threads<T, SWE_SCHEME_WAF>();
    return flux_max_threads<T, SWE_SCHEME_HLLC>();
}
template int split_max_threads<float>(int, bool);
template int split_max_threads<double>(int, bool);

int mass_partials_needed(int64_t n) { return (int)((n + MASS_BLOCK * MASS_ITEMS - 1) / (MASS_BLOCK * MASS_ITEMS)); }

template <typename T>
cudaError_t launch_prep(int scheme, const StepArgs<T> &a, Vec4<T> *F, Vec4<T> *U, int block, cudaStream_t s)
{
    if (scheme == SWE_SCHEME_MUSCL && a.hr2) k_prep_muscl<T, 4><<<grid_for(a.m.n, block), block, 0, s>>>(a, F);
    else if (scheme == SWE_SCHEME_MUSCL) k_prep_muscl<T><<<grid_for(a.m.n, block), block, 0, s>>>(a, F);
    else if (scheme == SWE_SCHEME_MUSCL_EDGE) k_prep_muscl_edge<T><<<grid_for(a.m.n, block), block, 0, s>>>(a, F);
    else if (scheme == SWE_SCHEME_WAF) k_prep_waf<T><<<grid_for(a.m.n, block), block, 0, s>>>(a, F, U);
    return cudaGetLastError();
}

template <typename T, int SCHEME> cudaError_t launch_flux_s(const StepArgs<T> &a, int block, cudaStream_t s)
{
    k_flux<T, SCHEME><<<grid_for(a.m.n, block), block, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flux(int scheme, const StepArgs<T> &a, int block, cudaStream_t s)
{
    // the paper's MUSCL differs only in prep: its flux kernel is the MUSCL one
    if (scheme == SWE_SCHEME_MUSCL && a.hr2) return launch_flux_s<T, FLUX_MUSCL_HR2>(a, block, s);
    if (scheme == SWE_SCHEME_MUSCL || scheme == SWE_SCHEME_MUSCL_EDGE) return launch_flux_s<T, SWE_SCHEME_MUSCL>(a, block, s);
    if (scheme == SWE_SCHEME_WAF) return launch_flux_s<T, SWE_SCHEME_WAF>(a, block, s);
    return launch_flux_s<T, SWE_SCHEME_HLLC>(a, block, s);
}

template <typename T>
cudaError_t launch_flux_list(int scheme, const StepArgs<T> &a, int block, cudaStream_t s)
{
    if (a.n_list <= 0) return cudaSuccess;
    const unsigned grid = grid_for(a.n_list, block);
    if (scheme == SWE_SCHEME_MUSCL && a.hr2)
        k_flux_list<T, FLUX_MUSCL_HR2><<<grid, block, 0, s>>>(a);
    else if (scheme == SWE_SCHEME_MUSCL || scheme == SWE_SCHEME_MUSCL_EDGE)
        k_flux_list<T, SWE_SCHEME_MUSCL><<<grid, block, 0, s>>>(a);
    else if (scheme == SWE_SCHEME_WAF)
        k_flux_list<T, SWE_SCHEME_WAF><<<grid, block, 0, s>>>(a);
    else
        k_flux_list<T, SWE_SCHEME_HLLC><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack_halo(int64_t n, const int32_t *cells, const T *h, const T *hu, const T *hv, T *buf,
                             cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_pack_halo<T><<<grid_for(n, 256), 256, 0, s>>>(n, cells, h, hu, hv, buf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smax(const StepArgs<T> &a, int slot, int block, cudaStream_t s)
{
    k_smax<T><<<grid_for(a.m.n, block), block, 0, s>>>(a, slot);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_heun_avg(const StepArgs<T> &a, const T *h0, const T *hu0, const T *hv0, int block,
                            cudaStream_t s)
{
    k_heun_avg<T><<<grid_for(a.m.n, block), block, 0, s>>>(a, h0, hu0, hv0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mass(const DevMesh<T> &m, const T *h, double *partials, int n_partials, double *out,
                        cudaStream_t s)
{
    k_mass_partial<T><<<n_partials, MASS_BLOCK, 0, s>>>(m, h, partials);
    k_mass_final<<<1, MASS_BLOCK, 0, s>>>(partials, n_partials, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_in(int64_t n, const int32_t *perm, const double *src, T *h, T *hu, T *hv,
                              cudaStream_t s)
{
    k_scatter_in<T><<<grid_for(n, 256), 256, 0, s>>>(n, perm, src, h, hu, hv);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_out(int64_t n, const int32_t *perm, const T *h, const T *hu, const T *hv,
                              double *dst, cudaStream_t s)
{
    k_gather_out<T><<<grid_for(n, 256), 256, 0, s>>>(n, perm, h, hu, hv, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert(int64_t n, const double *src, T *dst, cudaStream_t s)
{
    k_convert<T><<<grid_for(n, 256), 256, 0, s>>>(n, src, dst);
    return cudaGetLastError();
}

#define SWE_INSTANTIATE(T)                                                                                 \
    template cudaError_t launch_prep<T>(int, const StepArgs<T> &, Vec4<T> *, Vec4<T> *, int, cudaStream_t); \
    template cudaError_t launch_flux<T>(int, const StepArgs<T> &, int, cudaStream_t);                      \
    template cudaError_t launch_flux_list<T>(int, const StepArgs<T> &, int, cudaStream_t);                 \
    template cudaError_t launch_pack_halo<T>(int64_t, const int32_t *, const T *, const T *, const T *, T *, \
                                             cudaStream_t);                                                \
    template cudaError_t launch_smax<T>(const StepArgs<T> &, int, int, cudaStream_t);                      \
    template cudaError_t launch_heun_avg<T>(const StepArgs<T> &, const T *, const T *, const T *, int,     \
                                            cudaStream_t);                                                 \
    template cudaError_t launch_mass<T>(const DevMesh<T> &, const T *, double *, int, double *,           \
                                        cudaStream_t);                                                     \
    template cudaError_t launch_scatter_in<T>(int64_t, const int32_t *, const double *, T *, T *, T *,     \
                                              cudaStream_t);                                               \
    template cudaError_t launch_gather_out<T>(int64_t, const int32_t *, const T *, const T *, const T *,   \
                                              double *, cudaStream_t);                                     \
    template cudaError_t launch_convert<T>(int64_t, const double *, T *, cudaStream_t);

SWE_INSTANTIATE(float)
SWE_INSTANTIATE(double)
