// Per-cell device code of the split kernels (prep and flux), shared by the
// single-mesh kernels (swe_kernels.cu) and the batched ensemble kernels
// (swe_ensemble.cu).
#pragma once
#include "swe_device.cuh"

namespace swe_dev {

template <typename T>
__device__ __forceinline__ void prep_muscl_cell(const StepArgs<T> &a, int i, Vec4<T> *F)
{
    const T h_eps = a.h_eps;
    T hi = a.h[i], zi = a.m.z[i];
    T ui, vi;
    primitives(hi, a.hu[i], a.hv[i], h_eps, ui, vi);
    T qi[3] = {hi + zi, ui, vi};
    Vec2<T> ln[3], dd[3];
    T qn[3][3];
    bool has[3];
    bool ok = hi > h_eps;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int w = a.m.nbr[3 * i + k];
        ln[k] = a.m.ln[3 * i + k];
        dd[k] = a.m.dd[3 * i + k];
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
    Vec4<T> f[3];
    muscl_faces(qi, zi, ok, cnt, qn, has, ln, dd, f);
#pragma unroll
    for (int k = 0; k < 3; k++) F[3 * i + k] = f[k];
}

// WAF: centre primitives P[i] = (h, u, v, z) and, per edge k, the mean of
// (h, u, v) over the neighbours across edges k+1 and k+2 (a missing neighbour
// stands in with the cell itself).
template <typename T>
__device__ __forceinline__ void prep_waf_cell(const StepArgs<T> &a, int i, Vec4<T> *P, Vec4<T> *U)
{
    T hi = a.h[i], ui, vi;
    primitives(hi, a.hu[i], a.hv[i], a.h_eps, ui, vi);
    T qh[3], qu[3], qv[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int nb = a.m.nbr[3 * i + k];
        if (nb >= 0) {
            int j = nb >> 3;
            qh[k] = a.h[j];
            primitives(qh[k], a.hu[j], a.hv[j], a.h_eps, qu[k], qv[k]);
        } else {
            qh[k] = hi; qu[k] = ui; qv[k] = vi;
        }
    }
    Vec4<T> p;
    p.x = hi; p.y = ui; p.z = vi; p.w = a.m.z[i];
    P[i] = p;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        Vec4<T> u;
        u.x = (qh[k1] + qh[k2]) / T(2);
        u.y = (qu[k1] + qu[k2]) / T(2);
        u.z = (qv[k1] + qv[k2]) / T(2);
        u.w = T(0);
        U[3 * i + k] = u;
    }
}

// ---------------------------------------------------------------------------
// flux + update kernel (split path): neighbours through global memory
// ---------------------------------------------------------------------------
template <typename T> struct GlobalSrc {
    const StepArgs<T> &a;
    int i;
    __device__ Vec4<T> own_face(int k) const { return a.F[3 * i + k]; }
    __device__ Vec4<T> nbr_face(const Nb &b) const { return a.F[3 * b.idx + b.kj]; }
    __device__ Vec4<T> nbr_centre(const Nb &b) const { return a.F[b.idx]; }
    __device__ Vec4<T> own_up(int k) const { return a.U[3 * i + k]; }
    __device__ Vec4<T> nbr_up(const Nb &b) const { return a.U[3 * b.idx + b.kj]; }
    __device__ Vec4<T> nbr_state(const Nb &b) const
    {
        Vec4<T> q;
        q.x = a.h[b.idx]; q.y = a.hu[b.idx]; q.z = a.hv[b.idx]; q.w = a.m.z[b.idx];
        return q;
    }
};

// Shared memory of one warp in the flux kernel (see flux_block).
template <typename T, int SCHEME> struct WarpSmem {
    static constexpr int kItems = 96;
    Vec4<T> *S;      // [3][32] face side data (ef, uf, vf, z)
    Vec4<T> *U;      // [3][32] WAF upwind means
    Vec2<T> *LN;     // [3][32] scaled normals
    T *HC;           // [32]    cell-centre depth
    T *DL;           // [3][32] WAF centroid distances
    T *C;            // [9][32] contributions (component c, edge k) at C[(3c+k)*32 + lane]
    uint32_t *item;  // [96]    queued edges: lane_i | k_i << 5 | lane_j << 7 | k_j << 12 | own << 14 | in_warp << 15
    int32_t *item_j; // [96]    neighbour cell of each queued edge

    __host__ __device__ static constexpr size_t bytes()
    {
        return 3 * 32 * sizeof(Vec4<T>) * (SCHEME == SWE_SCHEME_WAF ? 2 : 1) + 3 * 32 * sizeof(Vec2<T>) +
               32 * sizeof(T) * (1 + 9 + (SCHEME == SWE_SCHEME_WAF ? 3 : 0)) + kItems * 8;
    }
    __device__ WarpSmem(unsigned char *base)
    {
        S = reinterpret_cast<Vec4<T> *>(base);
        U = S + 96;                                   // used by WAF only
        LN = reinterpret_cast<Vec2<T> *>(S + (SCHEME == SWE_SCHEME_WAF ? 192 : 96));
        HC = reinterpret_cast<T *>(LN + 96);
        DL = HC + 32;
        C = DL + (SCHEME == SWE_SCHEME_WAF ? 96 : 0);
        item = reinterpret_cast<uint32_t *>(C + 9 * 32);
        item_j = reinterpret_cast<int32_t *>(item + kItems);
    }
};

template <typename T, int SCHEME> __host__ __device__ constexpr size_t flux_smem_per_warp()
{
    return (WarpSmem<T, SCHEME>::bytes() + 31) & ~size_t(31);
}

// Flux kernel body for one block of cells.  Each warp handles 32 consecutive
// cells: the Riemann problem of an edge whose two cells are in the warp is
// solved once (by a queue of the warp's edges, compacted with ballots), the
// other edges once per side; each cell then adds its three contributions in
// edge order.  The arithmetic is the shared per-edge code, so the result is
// the same as evaluating every edge from both cells.
template <typename T, int SCHEME>
__device__ __forceinline__ void flux_block(const StepArgs<T> &a, int block_index)
{
    extern __shared__ __align__(32) unsigned char flux_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem<T, SCHEME> ws(flux_smem + warp * flux_smem_per_warp<T, SCHEME>());
    const int i = block_index * blockDim.x + threadIdx.x;
    const int w0 = i - lane;
    const bool valid = i < a.m.n;
    const T h_eps = a.h_eps;
    bool dry;
    const T dt = block_dt(a, &dry);

    // own data into the warp's shared memory
    Nb nb[3];
    Vec2<T> ln[3];
    T hi = T(0), hui = T(0), hvi = T(0), zi = T(0);
    if (valid) {
        hi = a.h[i]; hui = a.hu[i]; hvi = a.hv[i]; zi = a.m.z[i];
        T ui, vi;
        primitives(hi, hui, hvi, h_eps, ui, vi);
        ws.HC[lane] = hi;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            nb[k] = decode_global(a.m.nbr[3 * i + k]);
            ln[k] = a.m.ln[3 * i + k];
            ws.LN[k * 32 + lane] = ln[k];
            Vec4<T> sd;
            if (SCHEME == SWE_SCHEME_MUSCL) {
                sd = a.F[3 * i + k];
            } else {
                sd.x = hi + zi; sd.y = ui; sd.z = vi; sd.w = zi;
            }
            ws.S[k * 32 + lane] = sd;
            if (SCHEME == SWE_SCHEME_WAF) {
                ws.U[k * 32 + lane] = a.U[3 * i + k];
                const Vec2<T> d = a.m.dd[3 * i + k];
                ws.DL[k * 32 + lane] = dsqrt(d.x * d.x + d.y * d.y);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) { nb[k].interior = false; nb[k].own = false; nb[k].idx = 0; nb[k].kj = 0; nb[k].tag = 0; }
    }
    // queue of the warp's edges: an edge inside the warp once (from its lower cell)
    int n_items = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int j = nb[k].idx;
        const bool in_warp = nb[k].interior && j >= w0 && j < w0 + 32;
        const bool pred = valid && nb[k].interior && !(in_warp && j < i);
        const unsigned mask = __ballot_sync(0xffffffffu, pred);
        if (pred) {
            const int pos = n_items + __popc(mask & ((1u << lane) - 1u));
            ws.item[pos] = (uint32_t)lane | ((uint32_t)k << 5) | ((uint32_t)(in_warp ? j - w0 : 0) << 7) |
                           ((uint32_t)nb[k].kj << 12) | ((uint32_t)(nb[k].own ? 1 : 0) << 14) |
                           ((uint32_t)(in_warp ? 1 : 0) << 15);
            ws.item_j[pos] = j;
        }
        n_items += __popc(mask);
    }
    __syncwarp();

    // solve the queued edges, 32 at a time
    for (int it = lane; it < n_items; it += 32) {
        const uint32_t w = ws.item[it];
        const int li = (int)(w & 31u), ki = (int)((w >> 5) & 3u);
        const int lj = (int)((w >> 7) & 31u), kj = (int)((w >> 12) & 3u);
        const bool own_i = (w >> 14) & 1u, in_warp = (w >> 15) & 1u;
        Side<T> Si, Sj;
        {
            const Vec4<T> sd = ws.S[ki * 32 + li];
            Si.ef = sd.x; Si.uf = sd.y; Si.vf = sd.z; Si.z = sd.w; Si.hc = ws.HC[li];
        }
        Vec4<T> Ui{}, Uj{};
        T dlen = T(0);
        if (in_warp) {
            const Vec4<T> sd = ws.S[kj * 32 + lj];
            Sj.ef = sd.x; Sj.uf = sd.y; Sj.vf = sd.z; Sj.z = sd.w; Sj.hc = ws.HC[lj];
            if (SCHEME == SWE_SCHEME_WAF) Uj = ws.U[kj * 32 + lj];
        } else {
            const int j = ws.item_j[it];
            Nb bj;
            bj.idx = j; bj.kj = kj;
            GlobalSrc<T> src{a, j};
            if (SCHEME == SWE_SCHEME_MUSCL) {
                const Vec4<T> f = src.nbr_face(bj);
                Sj.ef = f.x; Sj.uf = f.y; Sj.vf = f.z; Sj.z = f.w; Sj.hc = T(0);
            } else if (SCHEME == SWE_SCHEME_WAF) {
                const Vec4<T> pc = src.nbr_centre(bj);
                Sj.hc = pc.x; Sj.uf = pc.y; Sj.vf = pc.z; Sj.z = pc.w; Sj.ef = pc.x + pc.w;
                Uj = src.nbr_up(bj);
            } else {
                const Vec4<T> q = src.nbr_state(bj);
                Sj.hc = q.x; Sj.z = q.w; Sj.ef = q.x + q.w;
                primitives(q.x, q.y, q.z, h_eps, Sj.uf, Sj.vf);
            }
        }
        if (SCHEME == SWE_SCHEME_WAF) {
            Ui = ws.U[ki * 32 + li];
            dlen = ws.DL[ki * 32 + li];
        }
        const Vec2<T> l = ws.LN[ki * 32 + li];
        Contrib<T> ci, cj;
        interior_edge<T, SCHEME>(a, dt, Si, Sj, own_i, l.x, l.y, dlen, Ui, Uj, ci, in_warp ? &cj : nullptr);
        ws.C[(0 + ki) * 32 + li] = ci.c0; ws.C[(3 + ki) * 32 + li] = ci.c1; ws.C[(6 + ki) * 32 + li] = ci.c2;
        if (in_warp) {
            ws.C[(0 + kj) * 32 + lj] = cj.c0; ws.C[(3 + kj) * 32 + lj] = cj.c1; ws.C[(6 + kj) * 32 + lj] = cj.c2;
        }
    }
    __syncwarp();

    CellOut<T> o;
    o.smax = T(0); o.clip = T(0); o.bsum = T(0);
    if (valid) {
        T R0 = T(0), R1 = T(0), R2 = T(0), bs = T(0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Contrib<T> c;
            if (nb[k].interior) {
                c.c0 = ws.C[(0 + k) * 32 + lane]; c.c1 = ws.C[(3 + k) * 32 + lane]; c.c2 = ws.C[(6 + k) * 32 + lane];
            } else {
                const Vec4<T> sd = ws.S[k * 32 + lane];
                Side<T> s;
                s.ef = sd.x; s.uf = sd.y; s.vf = sd.z; s.z = sd.w; s.hc = hi;
                c = boundary_edge<T>(a, s, nb[k].tag, ln[k].x, ln[k].y, bs);
            }
            accumulate(k, c, R0, R1, R2);
        }
        const T nm = a.m.nman ? a.m.nman[i] : T(0);
        o = cell_finish<T>(a, dt, hi, hui, hvi, R0, R1, R2, ln, nm, bs);
        a.ho[i] = o.h; a.huo[i] = o.hu; a.hvo[i] = o.hv;
        if (!(dfinite(o.h) && dfinite(o.hu) && dfinite(o.hv))) atomicOr(&a.sc->status, ST_NONFINITE);
    }
    step_epilogue<T>(a, dt, dry, o.smax, o.clip, o.bsum, block_index == 0);
}

}  // namespace swe_dev
