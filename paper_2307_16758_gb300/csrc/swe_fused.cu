// Fused tile kernel: one launch per time step does the whole second-order
// step (MUSCL face values or WAF upwind data, edge fluxes, update, friction
// and the wave-speed reduction) for a tile of consecutive (Morton-ordered)
// cells, so the face values never go to HBM.
//
//   phase 0: primitives of the tile's cells (coalesced) and of its halo
//            cells (gathered) into shared memory;
//   phase 1: face values (MUSCL) or upwind means (WAF) of the tile's cells,
//            from shared memory, and of the halo cells, from global memory
//            (their own neighbours may lie outside the tile);
//   phase 2: per cell, the fluxes of its three edges from shared memory and
//            the update -- the same device code as the split kernels.
// Each cell reads its state, bed, Manning n, normals, centroid offsets and
// tile-local neighbour slots once and writes its state once.
#include <cuda_runtime.h>

#include "swe_dev.h"
#include "swe_device.cuh"

namespace {
using namespace swe_dev;

template <typename T> struct SmemSrc {
    const Vec4<T> *Fs;      // MUSCL: [3*slots] face values; WAF: [3*slots] upwind means
    const Vec4<T> *Ps;      // WAF: [slots] centre values (h, u, v, z)
    int t;
    __device__ Vec4<T> own_face(int k) const { return Fs[3 * t + k]; }
    __device__ Vec4<T> nbr_face(const Nb &b) const { return Fs[3 * b.idx + b.kj]; }
    __device__ Vec4<T> nbr_centre(const Nb &b) const { return Ps[b.idx]; }
    __device__ Vec4<T> own_up(int k) const { return Fs[3 * t + k]; }
    __device__ Vec4<T> nbr_up(const Nb &b) const { return Fs[3 * b.idx + b.kj]; }
    __device__ Vec4<T> nbr_state(const Nb &) const { return Vec4<T>{}; }
};

// Upwind means of WAF for the three edges of a cell from its neighbours'
// (h, u, v); a missing neighbour stands in with the cell itself.
template <typename T>
__device__ __forceinline__ void waf_upwind(const T qh[3], const T qu[3], const T qv[3], Vec4<T> U[3])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        U[k].x = (qh[k1] + qh[k2]) / T(2);
        U[k].y = (qu[k1] + qu[k2]) / T(2);
        U[k].z = (qv[k1] + qv[k2]) / T(2);
        U[k].w = T(0);
    }
}

template <typename T, int SCHEME>
__global__ void k_fused(StepArgs<T> a, FusedArgs f)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    Vec4<T> *Ps = reinterpret_cast<Vec4<T> *>(smem_raw);          // [slots]
    Vec4<T> *Fs = Ps + f.slots;                                     // [3*slots]
    const int TC = f.tile;
    const int t = threadIdx.x;
    const int64_t start = (int64_t)blockIdx.x * TC;
    const int nt = (int)min((int64_t)TC, a.m.n - start);
    const int hp0 = f.halo_ptr[blockIdx.x];
    const int H = f.halo_ptr[blockIdx.x + 1] - hp0;
    const int64_t i = start + t;
    const bool valid = t < nt;
    const T h_eps = a.h_eps;
    bool dry;
    const T dt = block_dt(a, &dry);

    // ---- phase 0: primitives into shared memory ----
    // MUSCL: Ps = (eta, u, v, h); WAF: Ps = (h, u, v, z)
    T hi = T(0), hui = T(0), hvi = T(0), zi = T(0);
    if (valid) {
        hi = a.h[i]; hui = a.hu[i]; hvi = a.hv[i]; zi = a.m.z[i];
        T u, v;
        primitives(hi, hui, hvi, h_eps, u, v);
        Vec4<T> p;
        if (SCHEME == SWE_SCHEME_MUSCL) { p.x = hi + zi; p.y = u; p.z = v; p.w = hi; }
        else { p.x = hi; p.y = u; p.z = v; p.w = zi; }
        Ps[t] = p;
    }
    for (int q = t; q < H; q += blockDim.x) {
        const int g = f.halo_ids[hp0 + q];
        const T hg = a.h[g], zg = a.m.z[g];
        T u, v;
        primitives(hg, a.hu[g], a.hv[g], h_eps, u, v);
        Vec4<T> p;
        if (SCHEME == SWE_SCHEME_MUSCL) { p.x = hg + zg; p.y = u; p.z = v; p.w = hg; }
        else { p.x = hg; p.y = u; p.z = v; p.w = zg; }
        Ps[TC + q] = p;
    }
    __syncthreads();

    // ---- phase 1: face values / upwind means ----
    Nb nb[3];
    Vec2<T> ln[3], dd[3];
    if (valid) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            nb[k] = decode_local(f.nbr_local[3 * i + k]);
            ln[k] = a.m.ln[3 * i + k];
            dd[k] = a.m.dd[3 * i + k];
        }
        const Vec4<T> pi = Ps[t];
        if (SCHEME == SWE_SCHEME_MUSCL) {
            T qi[3] = {pi.x, pi.y, pi.z};
            T qn[3][3];
            bool has[3];
            bool ok = pi.w > h_eps;
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                has[k] = nb[k].interior;
                if (has[k]) {
                    const Vec4<T> pj = Ps[nb[k].idx];
                    ok = ok && pj.w > h_eps;
                    qn[k][0] = pj.x; qn[k][1] = pj.y; qn[k][2] = pj.z;
                    cnt++;
                } else {
                    qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
                }
            }
            Vec4<T> fv[3];
            muscl_faces(qi, zi, ok, cnt, qn, has, ln, dd, fv);
#pragma unroll
            for (int k = 0; k < 3; k++) Fs[3 * t + k] = fv[k];
        } else {
            T qh[3], qu[3], qv[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const Vec4<T> pj = nb[k].interior ? Ps[nb[k].idx] : pi;
                qh[k] = pj.x; qu[k] = pj.y; qv[k] = pj.z;
            }
            Vec4<T> U[3];
            waf_upwind(qh, qu, qv, U);
#pragma unroll
            for (int k = 0; k < 3; k++) Fs[3 * t + k] = U[k];
        }
    }
    for (int q = t; q < H; q += blockDim.x) {
        const int64_t g = f.halo_ids[hp0 + q];
        const Vec4<T> pg = Ps[TC + q];
        Vec4<T> out[3];
        if (SCHEME == SWE_SCHEME_MUSCL) {
            T qi[3] = {pg.x, pg.y, pg.z};
            T qn[3][3];
            bool has[3];
            bool ok = pg.w > h_eps;
            int cnt = 0;
            Vec2<T> lg[3], dg[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int w = a.m.nbr[3 * g + k];
                lg[k] = a.m.ln[3 * g + k];
                dg[k] = a.m.dd[3 * g + k];
                has[k] = w >= 0;
                if (has[k]) {
                    const int j = w >> 3;
                    T hj = a.h[j], uj, vj;
                    primitives(hj, a.hu[j], a.hv[j], h_eps, uj, vj);
                    ok = ok && hj > h_eps;
                    qn[k][0] = hj + a.m.z[j]; qn[k][1] = uj; qn[k][2] = vj;
                    cnt++;
                } else {
                    qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
                }
            }
            muscl_faces(qi, a.m.z[g], ok, cnt, qn, has, lg, dg, out);
        } else {
            T qh[3], qu[3], qv[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int w = a.m.nbr[3 * g + k];
                if (w >= 0) {
                    const int j = w >> 3;
                    qh[k] = a.h[j];
                    primitives(qh[k], a.hu[j], a.hv[j], h_eps, qu[k], qv[k]);
                } else {
                    qh[k] = pg.x; qu[k] = pg.y; qv[k] = pg.z;
                }
            }
            waf_upwind(qh, qu, qv, out);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) Fs[3 * (TC + q) + k] = out[k];
    }
    __syncthreads();

    // ---- phase 2: fluxes and update ----
    CellOut<T> o;
    o.smax = T(0); o.clip = T(0); o.bsum = T(0);
    if (valid) {
        const T nm = a.m.nman ? a.m.nman[i] : T(0);
        SmemSrc<T> src{Fs, Ps, t};
        o = cell_update<T, SCHEME>(a, dt, hi, hui, hvi, zi, nm, nb, ln, dd, src);
        a.ho[i] = o.h; a.huo[i] = o.hu; a.hvo[i] = o.hv;
        if (!(dfinite(o.h) && dfinite(o.hu) && dfinite(o.hv))) atomicOr(&a.sc->status, ST_NONFINITE);
    }
    step_epilogue<T>(a, dt, dry, o.smax, o.clip, o.bsum);
}

}  // namespace

template <typename T> int fused_max_threads(int scheme)
{
    cudaFuncAttributes fa{};
    cudaError_t e = scheme == SWE_SCHEME_WAF ? cudaFuncGetAttributes(&fa, k_fused<T, SWE_SCHEME_WAF>)
                                             : cudaFuncGetAttributes(&fa, k_fused<T, SWE_SCHEME_MUSCL>);
    return e == cudaSuccess ? fa.maxThreadsPerBlock : 0;
}

template <typename T> size_t fused_smem_bytes(int scheme, int slots)
{
    (void)scheme;
    return (size_t)slots * 4 * sizeof(Vec4<T>);
}

template <typename T>
cudaError_t launch_fused(int scheme, const StepArgs<T> &a, const FusedArgs &f, cudaStream_t s)
{
    const size_t smem = fused_smem_bytes<T>(scheme, f.slots);
    const unsigned grid = (unsigned)((a.m.n + f.tile - 1) / f.tile);
    if (scheme == SWE_SCHEME_MUSCL) {
        cudaFuncSetAttribute(k_fused<T, SWE_SCHEME_MUSCL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fused<T, SWE_SCHEME_MUSCL><<<grid, f.tile, smem, s>>>(a, f);
    } else if (scheme == SWE_SCHEME_WAF) {
        cudaFuncSetAttribute(k_fused<T, SWE_SCHEME_WAF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fused<T, SWE_SCHEME_WAF><<<grid, f.tile, smem, s>>>(a, f);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_fused<float>(int, const StepArgs<float> &, const FusedArgs &, cudaStream_t);
template cudaError_t launch_fused<double>(int, const StepArgs<double> &, const FusedArgs &, cudaStream_t);
template size_t fused_smem_bytes<float>(int, int);
template int fused_max_threads<float>(int);
template int fused_max_threads<double>(int);
template size_t fused_smem_bytes<double>(int, int);
