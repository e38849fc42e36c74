// Per-cell device code of the split kernels (prep and flux), shared by the
// single-mesh kernels (swe_kernels.cu) and the batched ensemble kernels
// (swe_ensemble.cu).
#pragma once
#include "swe_device.cuh"

namespace swe_dev {

// The face values of a dry cell (h <= h_eps): its centre values (eta, 0, 0, z)
// on all three edges, for every MUSCL variant.  The prep kernels store no
// face values for dry cells; readers take them from the cell's h and z.
template <typename T>
__device__ __forceinline__ Vec4<T> dry_face(T h, T z)
{
    Vec4<T> f;
    f.x = h + z; f.y = T(0); f.z = T(0); f.w = z;
    return f;
}

// MUSCL face values of cell i (least squares + Barth-Jespersen): f[k] =
// (eta, u, v, z) at the midpoint of edge k.  NQ = 4: also the limited
// gradient of h, for the face bed of the second-order hydrostatic
// reconstruction (R16); f[k].w is then the face bed.
template <typename T, int NQ = 3>
__device__ __forceinline__ void muscl_cell_faces(const StepArgs<T> &a, int64_t i, Vec4<T> f[3])
{
    const T h_eps = a.h_eps;
    T hi = a.h[i], zi = a.m.z[i];
    if (hi <= h_eps) {
        // a dry cell has a zero gradient and zero velocity: its three face
        // values are its centre values, as muscl_faces gives them; the
        // neighbours and the geometry are not needed
#pragma unroll
        for (int k = 0; k < 3; k++) f[k] = dry_face(hi, zi);
        return;
    }
    T ui, vi;
    primitives(hi, a.hu[i], a.hv[i], h_eps, ui, vi);
    T qi[NQ];
    qi[0] = hi + zi; qi[1] = ui; qi[2] = vi;
    if (NQ == 4) qi[NQ - 1] = hi;
    Vec2<T> ln[3], dd[3];
    T qn[3][NQ], ox[3], oy[3];
    bool has[3];
    bool ok = hi > h_eps;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) ln[k] = a.m.ln[3 * i + k];
    midpoint_offsets(ln, ox, oy);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int w = a.m.nbr[3 * i + k];
        has[k] = w >= 0;
        if (has[k]) {
            const int j = w >> 3;
            T hj = a.h[j], uj, vj;
            primitives(hj, a.hu[j], a.hv[j], h_eps, uj, vj);
            ok = ok && hj > h_eps;
            qn[k][0] = hj + a.m.z[j]; qn[k][1] = uj; qn[k][2] = vj;
            if (NQ == 4) qn[k][NQ - 1] = hj;
            dd[k] = centroid_offset(a.m.ln, ox[k], oy[k], j, (w >> 1) & 3);
            cnt++;
        } else {
#pragma unroll
            for (int s = 0; s < NQ; s++) qn[k][s] = qi[s];
            dd[k].x = T(0); dd[k].y = T(0);
        }
    }
    muscl_faces<T, NQ>(qi, zi, ok, cnt, qn, has, ox, oy, dd, f);
}

template <typename T, int NQ = 3>
__device__ __forceinline__ void prep_muscl_cell(const StepArgs<T> &a, int i, Vec4<T> *F)
{
    if (a.h[i] <= a.h_eps) return;                      // dry: faces implied (dry_face)
    Vec4<T> f[3];
    muscl_cell_faces<T, NQ>(a, i, f);
#pragma unroll
    for (int k = 0; k < 3; k++) F[3 * i + k] = f[k];
}

// The limited slope of the paper's MUSCL (Sec. 6.2.3) from the slope "up"
// behind the cell and the slope "dn" towards the other side of the edge
// (beta = 1 MINBEE, 2 SUPERBEE); zero when dn is zero.
template <typename T>
__device__ __forceinline__ T beta_limit(T beta, T up, T dn)
{
    if (dn > T(0)) return dmax(T(0), dmax(dmin(mul_rn(beta, up), dn), dmin(up, mul_rn(beta, dn))));
    if (dn < T(0)) return dmin(T(0), dmin(dmax(mul_rn(beta, up), dn), dmax(up, mul_rn(beta, dn))));
    return T(0);
}

// Prep of the paper's MUSCL (Sec. 6.2.3) for cell i: for each edge k towards
// the neighbour O, the slope of (eta, u, v) along the edge is the limited
// combination of the slope behind the cell, (U_i - U_upw) / |c_i - x_upw|
// with U_upw the mean over the cell's two other neighbours at the mean of
// their centroids, and the slope towards O, (U_O - U_i) / |c_O - c_i|; the
// face value is U_i + |m_k - c_i| * slope.  The paper writes the two sides of
// an edge apart (U~_L = U_L + |x_RL - x_L| dU_L, U~_R = U_R - |x_R - x_RL| dU_R);
// since the limiter satisfies lim(a, b) = -lim(-b, -a), the right side's
// formula is this one seen from R, so each cell reconstructs its own faces
// and the flux kernel is the MUSCL one.  A missing neighbour stands in with
// the cell; slopes are zero next to a dry cell and on boundary edges.
template <typename T>
__device__ __forceinline__ void prep_muscl_edge_cell(const StepArgs<T> &a, int i, Vec4<T> *F)
{
    const T h_eps = a.h_eps;
    const T hi = a.h[i], zi = a.m.z[i];
    if (hi <= h_eps) return;                            // dry: zero slopes, faces implied (dry_face)
    T ui, vi;
    primitives(hi, a.hu[i], a.hv[i], h_eps, ui, vi);
    const T qi[3] = {hi + zi, ui, vi};
    Vec2<T> ln[3], dd[3];
    T qn[3][3], ox[3], oy[3];
    bool has[3], wet[3];
#pragma unroll
    for (int k = 0; k < 3; k++) ln[k] = a.m.ln[3 * i + k];
    midpoint_offsets(ln, ox, oy);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int w = a.m.nbr[3 * i + k];
        has[k] = w >= 0;
        if (has[k]) {
            const int j = w >> 3;
            T hj = a.h[j], uj, vj;
            primitives(hj, a.hu[j], a.hv[j], h_eps, uj, vj);
            wet[k] = hj > h_eps;
            qn[k][0] = hj + a.m.z[j]; qn[k][1] = uj; qn[k][2] = vj;
            dd[k] = centroid_offset(a.m.ln, ox[k], oy[k], j, (w >> 1) & 3);
        } else {
            wet[k] = true;
            qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
            dd[k].x = T(0); dd[k].y = T(0);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        Vec4<T> f;
        f.x = qi[0]; f.y = qi[1]; f.z = qi[2]; f.w = zi;
        if (has[k]) {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            const T ux = mul_rn(dd[k1].x + dd[k2].x, T(0.5)), uy = mul_rn(dd[k1].y + dd[k2].y, T(0.5));
            const T d_up = dsqrt(fma_rn(ux, ux, mul_rn(uy, uy)));
            const T d_o = dsqrt(fma_rn(dd[k].x, dd[k].x, mul_rn(dd[k].y, dd[k].y)));
            const T d_m = dsqrt(fma_rn(ox[k], ox[k], mul_rn(oy[k], oy[k])));
            if (wet[k] && wet[k1] && wet[k2]) {
                T r[3];
#pragma unroll
                for (int s = 0; s < 3; s++) {
                    const T up = d_up > T(0) ? ddiv(qi[s] - mul_rn(qn[k1][s] + qn[k2][s], T(0.5)), d_up) : T(0);
                    const T dn = ddiv(qn[k][s] - qi[s], d_o);
                    r[s] = fma_rn(d_m, beta_limit(a.beta, up, dn), qi[s]);
                }
                f.x = r[0]; f.y = r[1]; f.z = r[2];
            }
        }
        F[3 * i + k] = f;
    }
}

// WAF: centre primitives P[i] = (h, u, v, z) and, per edge k, the mean of
// (q, u, v) over the neighbours across edges k+1 and k+2 (a missing neighbour
// stands in with the cell itself); q is the depth h, or the free surface
// eta = h + z when the ratios are taken on it.
template <typename T>
__device__ __forceinline__ void prep_waf_cell(const StepArgs<T> &a, int i, Vec4<T> *P, Vec4<T> *U)
{
    // A dry cell stores nothing: its primitives are (h, 0, 0, z), which the
    // flux kernel builds from h and z, and its upwind means are never used:
    // every Riemann problem it takes part in has a dry side, where the WAF
    // weights are A = 1 whatever the ratios (R18).
    if (a.h[i] <= a.h_eps) return;
    T hi = a.h[i], ui, vi;
    const T zi = a.m.z[i];
    primitives(hi, a.hu[i], a.hv[i], a.h_eps, ui, vi);
    T qh[3], qu[3], qv[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int nb = a.m.nbr[3 * i + k];
        if (nb >= 0) {
            int j = nb >> 3;
            const T hj = a.h[j];
            primitives(hj, a.hu[j], a.hv[j], a.h_eps, qu[k], qv[k]);
            qh[k] = a.waf_surface ? hj + a.m.z[j] : hj;
        } else {
            qh[k] = a.waf_surface ? hi + zi : hi; qu[k] = ui; qv[k] = vi;
        }
    }
    Vec4<T> p;
    p.x = hi; p.y = ui; p.z = vi; p.w = zi;
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
    T hi, zi;                                           // the cell's depth and bed
    __device__ Vec4<T> own_face(int k) const { return hi <= a.h_eps ? dry_face(hi, zi) : a.F[3 * i + k]; }
    // The neighbour's face value: stored if it is wet, else dry_face(h_j, z_j).
    __device__ Vec4<T> nbr_face(const Nb &b) const
    {
        const T hj = a.h[b.idx];
        return hj <= a.h_eps ? dry_face(hj, a.m.z[b.idx]) : a.F[3 * b.idx + b.kj];
    }
    // WAF: the neighbour's primitives (h, u, v, z), stored if it is wet
    __device__ Vec4<T> nbr_centre(const Nb &b) const
    {
        const T hj = a.h[b.idx];
        if (hj > a.h_eps) return a.F[b.idx];
        Vec4<T> p;
        p.x = hj; p.y = T(0); p.z = T(0); p.w = a.m.z[b.idx];
        return p;
    }
    __device__ Vec4<T> own_up(int k) const { return a.U[3 * i + k]; }
    __device__ Vec4<T> nbr_up(const Nb &b) const { return a.U[3 * b.idx + b.kj]; }
    __device__ Vec4<T> nbr_state(const Nb &b) const
    {
        Vec4<T> q;
        q.x = a.h[b.idx]; q.y = a.hu[b.idx]; q.z = a.hv[b.idx]; q.w = a.m.z[b.idx];
        return q;
    }
};

// Flux kernel body for one block of cells: each cell evaluates its three
// edges (hydrostatic reconstruction, canonical Riemann flux), adds the
// contributions in edge order and updates.
// With LIST, thread t of the launch updates cell a.cells[t] (boundary-first
// schedule); otherwise cell t.
template <typename T, int SCHEME, bool LIST = false>
__device__ __forceinline__ void flux_block(const StepArgs<T> &a, int block_index)
{
    const int t = block_index * blockDim.x + threadIdx.x;
    const int i = LIST ? (t < a.n_list ? a.cells[t] : -1) : t;
    bool dry;
    const T dt = block_dt(a, &dry);
    CellOut<T> o;
    o.smax = T(0); o.clip = T(0); o.bsum = T(0);
    if (LIST ? i >= 0 : i < a.m.n) {
        Nb nb[3];
        Vec2<T> ln[3], dd[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            nb[k] = decode_global(a.m.nbr[3 * i + k]);
            ln[k] = a.m.ln[3 * i + k];
            if (SCHEME == SWE_SCHEME_WAF) dd[k] = a.m.dd[3 * i + k];
        }
        const T nm = a.m.nman ? a.m.nman[i] : T(0);
        const T hi = a.h[i], zi = a.m.z[i];
        GlobalSrc<T> src{a, i, hi, zi};
        o = cell_update<T, SCHEME>(a, dt, hi, a.hu[i], a.hv[i], zi, nm, nb, ln, dd, src);
        a.ho[i] = o.h; a.huo[i] = o.hu; a.hvo[i] = o.hv;
        if (!(dfinite(o.h) && dfinite(o.hu) && dfinite(o.hv))) atomicOr(&a.sc->status, ST_NONFINITE);
    }
    step_epilogue<T>(a, dt, dry, o.smax, o.clip, o.bsum, block_index == 0 && !(LIST && a.no_advance));
}

}  // namespace swe_dev
