// Device code of the fused tile kernel (one tile of a mesh), shared by the
// single-mesh kernel (swe_fused.cu) and the batched ensemble kernel
// (swe_ensemble.cu).  See swe_fused.cu for the phases.
#pragma once
#include "swe_device.cuh"

namespace swe_dev {

template <typename T> struct FusedSmem {
    Vec4<T> *Ps;      // [B]     MUSCL: (eta, u, v, h); WAF: (h, u, v, z)
    Vec4<T> *Fs;      // [3][B]  MUSCL: face values (eta, u, v, z); WAF: upwind means
    T *C0, *C1, *C2;  // [3][B]  edge contributions of tile cells

    __device__ FusedSmem(unsigned char *base, int B)
    {
        Ps = reinterpret_cast<Vec4<T> *>(base);
        Fs = Ps + B;
        C0 = reinterpret_cast<T *>(Fs + 3 * B);
        C1 = C0 + 3 * B;
        C2 = C1 + 3 * B;
    }
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
__device__ __forceinline__ Side<T> slot_side(const FusedSmem<T> &sm, int B, int slot, int k)
{
    Side<T> s;
    const Vec4<T> p = sm.Ps[slot];
    if (SCHEME == SWE_SCHEME_MUSCL) {
        const Vec4<T> f = sm.Fs[k * B + slot];
        s.ef = f.x; s.uf = f.y; s.vf = f.z; s.z = f.w; s.hc = p.w; s.zc = f.w;   // first-order bed
    } else {
        s.hc = p.x; s.uf = p.y; s.vf = p.z; s.z = p.w; s.ef = p.x + p.w; s.zc = p.w;
    }
    return s;
}

template <typename T, int SCHEME>
__device__ __forceinline__ void fused_tile(const StepArgs<T> &a, const FusedArgs &f, int tile, unsigned char *smem_raw)
{
    const int B = blockDim.x;
    FusedSmem<T> sm(smem_raw, B);
    const int s0 = f.tile_start[tile], nc = f.tile_start[tile + 1] - s0;
    const int hp0 = f.halo_ptr[tile], H = f.halo_ptr[tile + 1] - hp0;
    const int ep0 = f.edge_ptr[tile], E = f.edge_ptr[tile + 1] - ep0;
    const int t = threadIdx.x;
    const T h_eps = a.h_eps;
    bool dry;
    const T dt = block_dt(a, &dry);

    // ---- phase 0: primitives of the slot's cell ----
    const bool is_cell = t < nc, is_halo = !is_cell && t < nc + H;
    const int cell = is_cell ? s0 + t : (is_halo ? f.halo_ids[hp0 + t - nc] : 0);
    T hi = T(0), hui = T(0), hvi = T(0), zi = T(0);
    if (is_cell || is_halo) {
        hi = a.h[cell]; hui = a.hu[cell]; hvi = a.hv[cell]; zi = a.m.z[cell];
        T u, v;
        primitives(hi, hui, hvi, h_eps, u, v);
        Vec4<T> p;
        if (SCHEME == SWE_SCHEME_MUSCL) { p.x = hi + zi; p.y = u; p.z = v; p.w = hi; }
        else { p.x = hi; p.y = u; p.z = v; p.w = zi; }
        sm.Ps[t] = p;
    }
    __syncthreads();

    // ---- phase 1: face values / upwind means ----
    Nb nb[3];
    Vec2<T> ln[3];
    if (is_cell) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            nb[k] = decode_local(f.nbr_local[3 * cell + k]);
            ln[k] = a.m.ln[3 * cell + k];
        }
        const Vec4<T> pi = sm.Ps[t];
        if (SCHEME == SWE_SCHEME_MUSCL) {
            T qi[3] = {pi.x, pi.y, pi.z};
            T qn[3][3], ox[3], oy[3];
            Vec2<T> dd[3];
            bool has[3];
            bool ok = pi.w > h_eps;
            int cnt = 0;
            midpoint_offsets(ln, ox, oy);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                has[k] = nb[k].interior;
                if (has[k]) {
                    const Vec4<T> pj = sm.Ps[nb[k].idx];
                    ok = ok && pj.w > h_eps;
                    qn[k][0] = pj.x; qn[k][1] = pj.y; qn[k][2] = pj.z;
                    // global index of the neighbour's slot: a tile cell or a halo cell
                    const int jg = nb[k].idx < nc ? s0 + nb[k].idx : f.halo_ids[hp0 + nb[k].idx - nc];
                    dd[k] = centroid_offset(a.m.ln, ox[k], oy[k], jg, nb[k].kj);
                    cnt++;
                } else {
                    qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
                    dd[k].x = T(0); dd[k].y = T(0);
                }
            }
            Vec4<T> fv[3];
            muscl_faces(qi, zi, ok, cnt, qn, has, ox, oy, dd, fv);
#pragma unroll
            for (int k = 0; k < 3; k++) sm.Fs[k * B + t] = fv[k];
        } else {
            T qh[3], qu[3], qv[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const Vec4<T> pj = nb[k].interior ? sm.Ps[nb[k].idx] : pi;
                qh[k] = pj.x; qu[k] = pj.y; qv[k] = pj.z;
            }
            Vec4<T> U[3];
            waf_upwind(qh, qu, qv, U);
#pragma unroll
            for (int k = 0; k < 3; k++) sm.Fs[k * B + t] = U[k];
        }
    } else if (is_halo) {
        const Vec4<T> pg = sm.Ps[t];
        Vec4<T> out[3];
        if (SCHEME == SWE_SCHEME_MUSCL) {
            T qi[3] = {pg.x, pg.y, pg.z};
            T qn[3][3], ox[3], oy[3];
            bool has[3];
            bool ok = pg.w > h_eps;
            int cnt = 0;
            Vec2<T> lg[3], dg[3];
#pragma unroll
            for (int k = 0; k < 3; k++) lg[k] = a.m.ln[3 * cell + k];
            midpoint_offsets(lg, ox, oy);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int w = a.m.nbr[3 * cell + k];
                has[k] = w >= 0;
                if (has[k]) {
                    const int j = w >> 3;
                    T hj = a.h[j], uj, vj;
                    primitives(hj, a.hu[j], a.hv[j], h_eps, uj, vj);
                    ok = ok && hj > h_eps;
                    qn[k][0] = hj + a.m.z[j]; qn[k][1] = uj; qn[k][2] = vj;
                    dg[k] = centroid_offset(a.m.ln, ox[k], oy[k], j, (w >> 1) & 3);
                    cnt++;
                } else {
                    qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
                    dg[k].x = T(0); dg[k].y = T(0);
                }
            }
            muscl_faces(qi, zi, ok, cnt, qn, has, ox, oy, dg, out);
        } else {
            T qh[3], qu[3], qv[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int w = a.m.nbr[3 * cell + k];
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
        for (int k = 0; k < 3; k++) sm.Fs[k * B + t] = out[k];
    }
    __syncthreads();

    // ---- phase 2: one thread per edge of the tile ----
    for (int e = t; e < E; e += B) {
        const uint32_t w = f.edges[ep0 + e];
        const int si = (int)(w & 511u), ki = (int)((w >> 9) & 3u);
        const int sj = (int)((w >> 11) & 511u), kj = (int)((w >> 20) & 3u);
        const bool own_i = (w >> 22) & 1u, jin = (w >> 23) & 1u;
        const Side<T> Si = slot_side<T, SCHEME>(sm, B, si, ki);
        const Side<T> Sj = slot_side<T, SCHEME>(sm, B, sj, kj);
        const int ei = 3 * (s0 + si) + ki;
        const Vec2<T> l = a.m.ln[ei];           // just read by the tile's thread: an L1 hit
        Vec4<T> Ui{}, Uj{};
        T dlen = T(0);
        if (SCHEME == SWE_SCHEME_WAF) {
            Ui = sm.Fs[ki * B + si];
            Uj = sm.Fs[kj * B + sj];
            const Vec2<T> d = a.m.dd[ei];
            dlen = dsqrt(fma_rn(d.x, d.x, mul_rn(d.y, d.y)));
        }
        Contrib<T> ci, cj;
        interior_edge<T, SCHEME>(a, dt, Si, Sj, own_i, l.x, l.y, dlen, Ui, Uj, ci, jin ? &cj : nullptr);
        sm.C0[ki * B + si] = ci.c0; sm.C1[ki * B + si] = ci.c1; sm.C2[ki * B + si] = ci.c2;
        if (jin) { sm.C0[kj * B + sj] = cj.c0; sm.C1[kj * B + sj] = cj.c1; sm.C2[kj * B + sj] = cj.c2; }
    }
    __syncthreads();

    // ---- phase 3: sums in edge order, update ----
    CellOut<T> o;
    o.smax = T(0); o.clip = T(0); o.bsum = T(0);
    if (is_cell) {
        T R0 = T(0), R1 = T(0), R2 = T(0), bs = T(0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Contrib<T> c;
            if (nb[k].interior) {
                c.c0 = sm.C0[k * B + t]; c.c1 = sm.C1[k * B + t]; c.c2 = sm.C2[k * B + t];
            } else {
                const Side<T> s = slot_side<T, SCHEME>(sm, B, t, k);
                c = boundary_edge<T>(a, s, nb[k].tag, ln[k].x, ln[k].y, bs);
            }
            accumulate(k, c, R0, R1, R2);
        }
        const T nm = a.m.nman ? a.m.nman[cell] : T(0);
        o = cell_finish<T>(a, dt, hi, hui, hvi, R0, R1, R2, ln, nm, bs);
        a.ho[cell] = o.h; a.huo[cell] = o.hu; a.hvo[cell] = o.hv;
        if (!(dfinite(o.h) && dfinite(o.hu) && dfinite(o.hv))) atomicOr(&a.sc->status, ST_NONFINITE);
    }
    step_epilogue<T>(a, dt, dry, o.smax, o.clip, o.bsum, tile == 0);
}


}  // namespace swe_dev
