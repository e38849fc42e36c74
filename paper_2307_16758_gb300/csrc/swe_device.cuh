// Device functions shared by the split kernels (swe_kernels.cu), the tile
// step (swe_tile.cu) and the batched ensemble (swe_ensemble.cu): the Riemann
// solver of Sec. 6.2, the MUSCL face values, WAF helpers and the block
// reductions.  Every kernel inlines the same code, so a cell gets the same
// bits whichever kernel computes it.
#pragma once
#include <cuda_runtime.h>

#include "swe_dev.h"

namespace swe_dev {

// Square root and division.  FP64 keeps IEEE-rounded sqrt and division (the
// FP64 path is compared with the oracle to 1e-12).  The FP32 path uses the
// hardware approximations (MUFU.RSQ / MUFU.RCP based, about 2 ulp), which is
// far inside its error budget and keeps every exact-zero and symmetry
// property, since equal inputs still give equal outputs.
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double ddiv(double a, double b) { return a / b; }
__device__ __forceinline__ float ddiv(float a, float b) { return __fdividef(a, b); }
template <typename T> __device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T dmin(T a, T b) { return a < b ? a : b; }
// h^(4/3) of the Manning term: FP64 h * cbrt(h); FP32 the fast exp2/log2 form.
__device__ __forceinline__ float dpow43(float x) { return __powf(x, 4.0f / 3.0f); }
__device__ __forceinline__ double dpow43(double x) { return x * cbrt(x); }
__device__ __forceinline__ bool dfinite(float x) { return isfinite(x); }
__device__ __forceinline__ bool dfinite(double x) { return isfinite(x); }

// Products and sums that the compiler must not fuse, so that an edge's
// contribution and a cell's sum of contributions have the same bits whether
// the edge is evaluated by the cell (split kernels) or once per edge (tile step).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
// A fused multiply-add written out (a*b + c, one rounding): the compiler's own
// contraction choices can differ between kernels that inline the same code.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------------------
// Riemann problem in the rotated frame.  Inputs are the reconstructed depths
// h*_L, h*_R (after the hydrostatic reconstruction) and the normal (u) and
// tangential (v) velocities of both sides.  Outputs: the mass flux M, the
// tangential momentum flux Tt and, for each side s, D_s = F_2 - G_2(U*_s),
// the normal-momentum flux minus that side's physical flux.  In the star
// region of HLL (Sec. 6.2.1),
//   F - G_L = S_L (S_R dU - dG) / (S_R - S_L),  F - G_R = S_R (S_L dU - dG) / (S_R - S_L),
// which is the printed star flux rearranged so that equal states give an
// exact zero (well-balancing).
// ---------------------------------------------------------------------------
template <typename T> struct Flux { T M, Tt, DL2, DR2; };

template <typename T> struct WafIn {
    T dtdx;            // dt / |c_R - c_L|
    T hupL, hupR;      // upwind mean depth of each side
    T vupL, vupR;      // upwind mean tangential velocity of each side
    T hcL, hcR;        // the ratios' cell values (depth or free surface)
    bool dry_cell;     // a cell on either side is dry (h <= h_eps)
};

template <typename T>
__device__ __forceinline__ T waf_ratio(T r_eps, T upw, T qL, T qR)
{
    T loc = qR - qL;
    T sc = dmax(dmax(fabs(qL), fabs(qR)), T(1));
    if (fabs(loc) <= r_eps * sc) return T(0);
    return ddiv(upw, loc);
}

// A(r, c) of Sec. 6.2.2: SUPERBEE's branch table, its phi = 1 / phi = 0
// variants, and 1 - (1 - |c|) phi(r) for MINBEE and van Leer.
template <typename T>
__device__ __forceinline__ T waf_A(int lim, T r, T c)
{
    T ac = fabs(c);
    if (lim == SWE_WAF_PHI1) return ac;
    if (lim == SWE_WAF_PHI0) return T(1);
    if (lim == SWE_WAF_MINBEE) return T(1) - (T(1) - ac) * (r <= T(0) ? T(0) : dmin(r, T(1)));
    if (lim == SWE_WAF_VANLEER) return T(1) - (T(1) - ac) * (r <= T(0) ? T(0) : ddiv(T(2) * r, T(1) + r));
    if (r <= T(0)) return T(1);
    if (r <= T(0.5)) return T(1) - T(2) * (T(1) - ac) * r;
    if (r <= T(1)) return ac;
    if (r <= T(2)) return T(1) - (T(1) - ac) * r;
    return T(2) * ac - T(1);
}

template <typename T, bool WAF>
__device__ __forceinline__ Flux<T> riemann(T hsL, T uL, T vL, T hsR, T uR, T vR, T g, T h_eps,
                                           const WafIn<T> &w, int lim, T r_eps)
{
    Flux<T> f;
    const T half = T(0.5), hg = half * g;
    T GL1 = hsL * uL, GL2 = fma_rn(GL1, uL, hg * hsL * hsL);
    T GR1 = hsR * uR, GR2 = fma_rn(GR1, uR, hg * hsR * hsR);
    T dG1 = GR1 - GL1, dG2 = GR2 - GL2;
    T dU1 = hsR - hsL, dU2 = dG1;              // the momentum jump is the mass-flux jump
    bool dryL = hsL <= h_eps, dryR = hsR <= h_eps;
    if (dryL && dryR) {                    // both sides dry: zero numerical flux
        f.M = T(0); f.Tt = T(0); f.DL2 = -GL2; f.DR2 = -GR2;
        return f;
    }
    if ((!WAF || lim != SWE_WAF_PHI1) && hsL == hsR && uL == uR && vL == vR) {
        // equal states (a lake at rest, or any uniform flow): whichever wave
        // pattern the speeds give, dU = dG = 0, so the HLL flux is G(U) and
        // the HLLC tangential flux is M v; the solver below would return the
        // same values (up to the sign of a zero), so its speeds are skipped.
        // WAF too: its weighted sums of G_L, F_HLL and G_R are all G(U), and
        // the shear wave's local change of v is zero, so its ratio is 0 and
        // A = 1 (every limiter but phi = 1, which keeps A = |c|): the
        // tangential weights are exactly 1 and 0, and the flux is M v.
        f.M = GL1 + T(0); f.Tt = f.M * vL; f.DL2 = T(0); f.DR2 = T(0);
        return f;
    }
    T aL = dsqrt(g * hsL), aR = dsqrt(g * hsR);
    T SL, SR;
    if (dryL) {                            // dry-bed wave speeds
        SL = uR - T(2) * aR; SR = uR + aR;
    } else if (dryR) {
        SL = uL - aL; SR = uL + T(2) * aL;
    } else {
        T h0 = (hsL + hsR) / T(2) - ddiv((uR - uL) * (hsL + hsR), T(4) * (aR + aL));
        T hs;
        if (h0 <= dmin(hsL, hsR)) {        // two rarefactions
            T br = dmax((aR + aL) / T(2) + (uL - uR) / T(4), T(0));
            hs = ddiv(br * br, g);
        } else {                           // two shocks
            T gL = dsqrt(ddiv(g * (h0 + hsL), T(2) * h0 * hsL));
            T gR = dsqrt(ddiv(g * (h0 + hsR), T(2) * h0 * hsR));
            hs = ddiv(hsL * gL + hsR * gR + uL - uR, gL + gR);
        }
        T pL = hs > hsL ? ddiv(dsqrt(hs * (hs + hsL) / T(2)), hsL) : T(1);
        T pR = hs > hsR ? ddiv(dsqrt(hs * (hs + hsR) / T(2)), hsR) : T(1);
        SL = uL - aL * pL;
        SR = uR + aR * pR;
    }
    const T qR = hsR * (uR - SR), qL = hsL * (uL - SL);
    T num = fma_rn(SL, qR, -(SR * qL));
    T den = qR - qL;
    T Ss = den != T(0) ? ddiv(num, den) : T(0);
    // HLL (three branches) as differences to G_L and G_R
    T hL1, hL2, hR2;
    bool rightgoing = SL >= T(0), leftgoing = !rightgoing && SR <= T(0);
    if (rightgoing) {
        hL1 = T(0); hL2 = T(0); hR2 = -dG2;
    } else if (leftgoing) {
        hL1 = dG1; hL2 = dG2; hR2 = T(0);
    } else {
        const T iw = ddiv(T(1), SR - SL);
        hL1 = SL * fma_rn(SR, dU1, -dG1) * iw;
        hL2 = SL * fma_rn(SR, dU2, -dG2) * iw;
        hR2 = SR * fma_rn(SL, dU2, -dG2) * iw;
    }
    if (!WAF) {
        f.M = leftgoing ? GR1 : GL1 + hL1;
        f.Tt = f.M * (Ss >= T(0) ? vL : vR);      // HLLC: upwind tangential velocity
        f.DL2 = hL2; f.DR2 = hR2;
    } else {
        T cL = SL * w.dtdx, cR = SR * w.dtdx, cs = Ss * w.dtdx;
        T rL = waf_ratio(r_eps, SL >= T(0) ? w.hcL - w.hupL : w.hupR - w.hcR, w.hcL, w.hcR);
        T rR = waf_ratio(r_eps, SR >= T(0) ? w.hcL - w.hupL : w.hupR - w.hcR, w.hcL, w.hcR);
        T rs = waf_ratio(r_eps, Ss >= T(0) ? vL - w.vupL : w.vupR - vR, vL, vR);
        T sgL = cL >= T(0) ? T(1) : T(-1), sgR = cR >= T(0) ? T(1) : T(-1), sgs = cs >= T(0) ? T(1) : T(-1);
        T AL = waf_A(lim, rL, cL), AR = waf_A(lim, rR, cR), As = waf_A(lim, rs, cs);
        // no wet star region (a dry side: a dry cell or a dry reconstructed
        // depth; or the vacuum condition): the weights of Sec. 6.2.2 do not
        // apply, A = 1 gives the HLLC flux
        if (dryL || dryR || w.dry_cell || uR - uL >= T(2) * (aL + aR)) { AL = T(1); AR = T(1); As = T(1); }
        T wL = (T(1) + sgL * AL) / T(2);
        T wLR = (sgR * AR - sgL * AL) / T(2);
        T wR = (T(1) - sgR * AR) / T(2);
        T wLs = (T(1) + sgs * As) / T(2), wRs = (T(1) - sgs * As) / T(2);
        // weighted average of G_L, F_HLL and G_R, as differences to G_L and G_R
        T DL1 = wLR * hL1 + wR * dG1;
        f.DL2 = wLR * hL2 + wR * dG2;
        f.DR2 = -wL * dG2 + wLR * hR2;
        f.M = GL1 + DL1;
        f.Tt = (wLs * vL + wRs * vR) * f.M;
    }
    return f;
}


// Offsets from the centroid to the three edge midpoints, from the scaled
// outward normals: with e_k = (-ln_k.y, ln_k.x) the edge vectors,
// m_0 - c = (e_2 - e_1)/6, m_1 - c = (e_0 - e_2)/6, m_2 - c = (e_1 - e_0)/6.
template <typename T>
__device__ __forceinline__ void midpoint_offsets(const Vec2<T> ln[3], T ox[3], T oy[3])
{
    // products rounded on their own (mul_rn): the offsets feed differences
    // that the compiler could otherwise fuse differently in each kernel
    const T s = T(1) / T(6);
    ox[0] = mul_rn(ln[1].y - ln[2].y, s); oy[0] = mul_rn(ln[2].x - ln[1].x, s);
    ox[1] = mul_rn(ln[2].y - ln[0].y, s); oy[1] = mul_rn(ln[0].x - ln[2].x, s);
    ox[2] = mul_rn(ln[0].y - ln[1].y, s); oy[2] = mul_rn(ln[1].x - ln[0].x, s);
}

// Centroid offset c_j - c_i across edge k of cell i, where j is the
// neighbour and k_j its local index of the shared edge:
// c_j - c_i = (m - c_i) - (m - c_j) with m the edge midpoint, the second term
// the midpoint offset of j's edge k_j from j's scaled normals.  (oxi, oyi) is
// the midpoint offset of cell i's edge k.  The centroid offsets are thus
// derived from the normals that the kernels read anyway, not stored.
// a1, a2: the neighbour's scaled normals of its edges k_j + 1 and k_j + 2.
template <typename T>
__device__ __forceinline__ Vec2<T> centroid_offset_from(T oxi, T oyi, const Vec2<T> &a1, const Vec2<T> &a2)
{
    const T s = T(1) / T(6);
    Vec2<T> d;
    d.x = oxi - mul_rn(a1.y - a2.y, s);
    d.y = oyi - mul_rn(a2.x - a1.x, s);
    return d;
}

template <typename T>
__device__ __forceinline__ Vec2<T> centroid_offset(const Vec2<T> *ln, T oxi, T oyi, int j, int kj)
{
    const int k1 = kj == 2 ? 0 : kj + 1, k2 = kj == 0 ? 2 : kj - 1;
    return centroid_offset_from(oxi, oyi, ln[3 * j + k1], ln[3 * j + k2]);
}

// Wave speed sqrt(g h) + |u| of a wet cell (the CFL rule of Sec. 6.1): one
// expression wherever it is evaluated (after an update, after set_state, in
// Heun's average), so a run resumed from a saved state takes the same steps.
template <typename T>
__device__ __forceinline__ T wave_speed(T g, T h, T hu, T hv)
{
    const T u = ddiv(hu, h), v = ddiv(hv, h);
    return dsqrt(g * h) + dsqrt(fma_rn(u, u, mul_rn(v, v)));
}

template <typename T>
__device__ __forceinline__ void primitives(T h, T hu, T hv, T h_eps, T &u, T &v)
{
    bool wet = h > h_eps;
    u = wet ? ddiv(hu, h) : T(0);
    v = wet ? ddiv(hv, h) : T(0);
}

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = dmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Max of s and sums of c1, c2 over the block (in the compute type; a warp
// whose values are all zero skips its sum); thread 0 publishes them: the
// max into the CFL slot (atomicMax on the bits of the non-negative double),
// the sums into the FP64 diagnostics, scaled by wsum.
// Wave speeds as ordered integers: the bits of a non-negative float or double
// compare like the values, so atomicMax on them is a max on the speeds.
__device__ __forceinline__ unsigned long long speed_bits(float s) { return (unsigned long long)__float_as_uint(s); }
__device__ __forceinline__ unsigned long long speed_bits(double s)
{
    return (unsigned long long)__double_as_longlong(s);
}
__device__ __forceinline__ float speed_from_bits(unsigned long long b, float) { return __uint_as_float((unsigned)b); }
__device__ __forceinline__ double speed_from_bits(unsigned long long b, double)
{
    return __longlong_as_double((long long)b);
}

template <typename T>
__device__ __forceinline__ void block_publish(T s, T c1, T c2, DevScalars *sc, int slot_next,
                                              bool want_max, double wsum)
{
    __shared__ T sh_s[32], sh_c1[32], sh_c2[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    s = warp_max(s);
    if (__any_sync(0xffffffffu, c1 != T(0))) c1 = warp_sum(c1);
    if (__any_sync(0xffffffffu, c2 != T(0))) c2 = warp_sum(c2);
    if (lane == 0) { sh_s[wid] = s; sh_c1[wid] = c1; sh_c2[wid] = c2; }
    __syncthreads();
    if (wid == 0) {
        s = lane < nw ? sh_s[lane] : T(0);
        c1 = lane < nw ? sh_c1[lane] : T(0);
        c2 = lane < nw ? sh_c2[lane] : T(0);
        s = warp_max(s);
        if (__any_sync(0xffffffffu, c1 != T(0))) c1 = warp_sum(c1);
        if (__any_sync(0xffffffffu, c2 != T(0))) c2 = warp_sum(c2);
        if (lane == 0) {
            if (want_max && s > T(0)) atomicMax(&sc->smax[slot_next], speed_bits(s));
            if (c1 != T(0)) atomicAdd(&sc->clipped, wsum * (double)c1);
            if (c2 != T(0)) atomicAdd(&sc->bnd_in, wsum * (double)c2);
        }
    }
}

// The CFL time step of Sec. 6.1 from the current wave-speed slot, or the
// replayed time step.
template <typename T>
__device__ __forceinline__ T step_dt(const StepArgs<T> &a, bool *dry)
{
    if (a.dtv) { *dry = false; return (T)a.dtv[0]; }
    const T sm = speed_from_bits(a.sc->smax[a.slot_cur], T(0));
    *dry = !(sm > T(0));
    if (*dry) return T(0);
    return ddiv(a.cfl_rmin, sm);
}

// The time step for a block.  From the CFL slot every thread evaluates it
// itself (one broadcast load and a division, no barrier); a replayed time
// step (FP64 in memory) is converted by one thread and shared.
template <typename T>
__device__ __forceinline__ T block_dt(const StepArgs<T> &a, bool *dry)
{
    if (!a.dtv) return step_dt(a, dry);
    __shared__ T sh_dt;
    if (threadIdx.x == 0) {
        bool d;
        sh_dt = step_dt(a, &d);
    }
    __syncthreads();
    *dry = false;
    return sh_dt;
}

// MUSCL face values of one cell (least squares + Barth-Jespersen, zero
// gradient next to a dry cell or for a singular 2x2 system).  qi = own
// (eta, u, v); qn[k] = neighbour k's (eta, u, v) where has[k]; ok = the cell
// and all its neighbours are wet; cnt = number of neighbours.  F[k] =
// (eta, u, v, z) at the midpoint of edge k.
template <typename T, int NQ = 3>
__device__ __forceinline__ void muscl_faces(const T qi[NQ], T zi, bool ok, int cnt, const T qn[3][NQ],
                                            const bool has[3], const T ox[3], const T oy[3],
                                            const Vec2<T> dd[3], Vec4<T> F[3])
{
    // NQ = 3: (eta, u, v).  NQ = 4 adds h (second-order hydrostatic
    // reconstruction, R16): the face bed is then z_i + (grad eta - grad h).(m_k - c_i).
    T gx[NQ], gy[NQ];
#pragma unroll
    for (int s = 0; s < NQ; s++) { gx[s] = T(0); gy[s] = T(0); }
    // Every product below is either fused explicitly (fma_rn) or rounded on
    // its own (mul_rn), so all kernels that inline this give the same bits.
    // When every neighbour holds the cell's own values (a lake at rest, a
    // uniform flow) the least-squares right-hand sides are exact zeros and the
    // limited gradient is +0: the solve is skipped, with the same bits.
    bool flat = true;
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int s = 0; s < NQ; s++) flat = flat && qn[k][s] == qi[s];
    if (ok && cnt >= 2 && !flat) {
        T Mxx = T(0), Mxy = T(0), Myy = T(0);
        T bx[NQ], by[NQ];
#pragma unroll
        for (int s = 0; s < NQ; s++) { bx[s] = T(0); by[s] = T(0); }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (!has[k]) continue;
            T dx = dd[k].x, dy = dd[k].y;
            Mxx = fma_rn(dx, dx, Mxx); Mxy = fma_rn(dx, dy, Mxy); Myy = fma_rn(dy, dy, Myy);
#pragma unroll
            for (int s = 0; s < NQ; s++) {
                T dq = qn[k][s] - qi[s];
                bx[s] = fma_rn(dx, dq, bx[s]); by[s] = fma_rn(dy, dq, by[s]);
            }
        }
        T det = fma_rn(Mxx, Myy, -mul_rn(Mxy, Mxy)), tr = Mxx + Myy;
        if (det > mul_rn(mul_rn(T(1e-12), tr), tr)) {
#pragma unroll
            for (int s = 0; s < NQ; s++) {
                T px = ddiv(fma_rn(Myy, bx[s], -mul_rn(Mxy, by[s])), det);
                T py = ddiv(fma_rn(Mxx, by[s], -mul_rn(Mxy, bx[s])), det);
                T qmin = qi[s], qmax = qi[s];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if (!has[k]) continue;
                    qmin = dmin(qmin, qn[k][s]);
                    qmax = dmax(qmax, qn[k][s]);
                }
                T phi = T(1);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    T d = fma_rn(px, ox[k], mul_rn(py, oy[k]));
                    T ph = T(1);
                    if (d > T(0)) ph = ddiv(qmax - qi[s], d);
                    else if (d < T(0)) ph = ddiv(qmin - qi[s], d);
                    phi = dmin(phi, ph);
                }
                gx[s] = mul_rn(phi, px); gy[s] = mul_rn(phi, py);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        F[k].x = qi[0] + fma_rn(gx[0], ox[k], mul_rn(gy[0], oy[k]));
        F[k].y = qi[1] + fma_rn(gx[1], ox[k], mul_rn(gy[1], oy[k]));
        F[k].z = qi[2] + fma_rn(gx[2], ox[k], mul_rn(gy[2], oy[k]));
        F[k].w = NQ == 4 ? zi + fma_rn(gx[0] - gx[NQ - 1], ox[k], mul_rn(gy[0] - gy[NQ - 1], oy[k])) : zi;
    }
}

// A decoded neighbour word: interior edge (index into the caller's arrays,
// the neighbour's local edge, owner flag) or boundary tag.
struct Nb {
    bool interior, own;
    int idx, kj, tag;
};

__device__ __forceinline__ Nb decode_global(int w)
{
    Nb b;
    b.interior = w >= 0;
    b.idx = w >> 3; b.kj = (w >> 1) & 3; b.own = w & 1;
    b.tag = -1 - w;
    return b;
}

__device__ __forceinline__ Nb decode_local(unsigned w)
{
    Nb b;
    b.interior = !(w & 0x8000u);
    b.idx = (int)(w >> 3); b.kj = (int)((w >> 1) & 3u); b.own = w & 1u;
    b.tag = (int)(w & 0x7fffu);
    return b;
}

template <typename T> struct CellOut { T h, hu, hv, smax, clip, bsum; };


// Edge length and unit normal from the scaled normal (FP32: one rsqrt).
__device__ __forceinline__ void unit_normal(float lx, float ly, float &L, float &nx, float &ny)
{
    const float l2 = fma_rn(lx, lx, mul_rn(ly, ly));
    const float ri = rsqrtf(l2);
    L = l2 * ri; nx = lx * ri; ny = ly * ri;
}
__device__ __forceinline__ void unit_normal(double lx, double ly, double &L, double &nx, double &ny)
{
    L = sqrt(fma_rn(lx, lx, mul_rn(ly, ly)));
    nx = lx / L; ny = ly / L;
}

// The edge length alone (the same bits as unit_normal's L in FP32).
__device__ __forceinline__ float edge_length(float lx, float ly)
{
    const float l2 = fma_rn(lx, lx, mul_rn(ly, ly));
    return l2 * rsqrtf(l2);
}
__device__ __forceinline__ double edge_length(double lx, double ly) { return sqrt(fma_rn(lx, lx, mul_rn(ly, ly))); }

// Contribution of one edge to its cell's flux sum: L * (M, P n - Tt t) with t = (-n_y, n_x).
template <typename T> struct Contrib { T c0, c1, c2; };

template <typename T>
__device__ __forceinline__ Contrib<T> contribution(T L, T sM, T P, T Tt, T nx, T ny)
{
    Contrib<T> c;
    c.c0 = mul_rn(L, sM);
    c.c1 = mul_rn(L, fma_rn(P, nx, -mul_rn(Tt, ny)));
    c.c2 = mul_rn(L, fma_rn(P, ny, mul_rn(Tt, nx)));
    return c;
}

// One side of an edge: the free surface and velocities at the edge midpoint,
// the cell's bed and its cell-centre depth.
// z is the bed at the face (the cell bed, or with the second-order
// reconstruction the linear bed at the midpoint); zc is the cell bed.
template <typename T> struct Side { T ef, uf, vf, z, hc, zc; };

// Flux-template id of the LSQ MUSCL scheme with the second-order hydrostatic
// reconstruction (R16).  It is not a public scheme value: the flux kernels
// are instantiated for it so that the first-order path carries no test.
constexpr int FLUX_MUSCL_HR2 = 0x10 | SWE_SCHEME_MUSCL;

// Schemes whose flux kernel reads reconstructed face values.
__host__ __device__ constexpr bool face_scheme(int s) { return s == SWE_SCHEME_MUSCL || s == FLUX_MUSCL_HR2; }

// The cell's own pressure term of a face (the hydrostatic correction).  First
// order (Sec. 6.2.3 HR, R6): g/2 (h_f^2 - h_c^2).  Second-order
// reconstruction (R16): that plus the centred bed source of the face,
// g/2 (h_f + h_c)(eta_f - eta_c) on a wet face and g/2 (h_f + h_c)(z_f - eta_c)
// on a dry one, so that a lake at rest gives an exact zero.
template <typename T, bool HR2>
__device__ __forceinline__ T own_pressure(const StepArgs<T> &a, T hf, const Side<T> &s)
{
    const T half = T(0.5);
    if (!HR2) return half * a.g * (hf - s.hc) * (hf + s.hc);
    return mul_rn(mul_rn(mul_rn(half, a.g), hf + s.hc), (hf > T(0) ? s.ef : s.z) - (s.hc + s.zc));
}

// Interior edge seen from side i (scaled outward normal (lx, ly) of i):
// hydrostatic reconstruction, canonical-orientation Riemann flux, and the
// contribution to i -- and, if cj is given, to j (normal -n).
template <typename T, int SCHEME>
__device__ __forceinline__ void interior_edge(const StepArgs<T> &a, T dt, const Side<T> &si, const Side<T> &sj,
                                              bool own_i, T lx, T ly, T dlen, const Vec4<T> &Ui,
                                              const Vec4<T> &Uj, Contrib<T> &ci, Contrib<T> *cj)
{
    const T g = a.g, h_eps = a.h_eps, half = T(0.5);
    T L, nx, ny;
    unit_normal(lx, ly, L, nx, ny);
    // canonical orientation: side A is the owner of the edge
    const T cnx = own_i ? nx : -nx, cny = own_i ? ny : -ny;
    const Side<T> &A = own_i ? si : sj;
    const Side<T> &B = own_i ? sj : si;
    const T zf = dmax(si.z, sj.z);
    const T hsA = dmax(A.ef - zf, T(0)), hsB = dmax(B.ef - zf, T(0));
    const T unA = fma_rn(A.uf, cnx, mul_rn(A.vf, cny)), vtA = fma_rn(A.vf, cnx, -mul_rn(A.uf, cny));
    const T unB = fma_rn(B.uf, cnx, mul_rn(B.vf, cny)), vtB = fma_rn(B.vf, cnx, -mul_rn(B.uf, cny));
    Flux<T> fl;
    if (SCHEME == SWE_SCHEME_WAF) {
        WafIn<T> wi;
        wi.dtdx = ddiv(dt, dlen);
        const Vec4<T> &UA = own_i ? Ui : Uj;
        const Vec4<T> &UB = own_i ? Uj : Ui;
        wi.hupL = UA.x; wi.hupR = UB.x;
        wi.vupL = -UA.y * cny + UA.z * cnx;
        wi.vupR = -UB.y * cny + UB.z * cnx;
        // the ratios' cell values: depth, or free surface (eta = h + z)
        wi.hcL = a.waf_surface ? A.hc + A.zc : A.hc;
        wi.hcR = a.waf_surface ? B.hc + B.zc : B.hc;
        wi.dry_cell = A.hc <= h_eps || B.hc <= h_eps;
        fl = riemann<T, true>(hsA, unA, vtA, hsB, unB, vtB, g, h_eps, wi, a.waf_limiter, a.r_eps);
    } else {
        WafIn<T> wi{};
        fl = riemann<T, false>(hsA, unA, vtA, hsB, unB, vtB, g, h_eps, wi, 0, a.r_eps);
    }
    const T PA = fma_rn(hsA * unA, unA, fl.DL2), PB = fma_rn(hsB * unB, unB, fl.DR2);
    const T hfi = dmax(si.ef - si.z, T(0));
    const T Pi = (own_i ? PA : PB) + own_pressure<T, SCHEME == FLUX_MUSCL_HR2>(a, hfi, si);
    const T sMi = own_i ? fl.M : -fl.M;
    ci = contribution(L, sMi, Pi, fl.Tt, nx, ny);
    if (cj) {
        const T hfj = dmax(sj.ef - sj.z, T(0));
        const T Pj = (own_i ? PB : PA) + own_pressure<T, SCHEME == FLUX_MUSCL_HR2>(a, hfj, sj);
        const T sMj = own_i ? -fl.M : fl.M;
        *cj = contribution(L, sMj, Pj, fl.Tt, -nx, -ny);
    }
}

// Boundary edge of cell i (outward normal, Sec. 6.1): wall, open, inflow,
// fixed level.  bs receives the mass that leaves, -L*M.
template <typename T, bool HR2 = false>
__device__ __forceinline__ Contrib<T> boundary_edge(const StepArgs<T> &a, const Side<T> &si, int tag, T lx, T ly,
                                                    T &bs)
{
    const T g = a.g, h_eps = a.h_eps, half = T(0.5);
    T L, nx, ny;
    unit_normal(lx, ly, L, nx, ny);
    const T hf = dmax(si.ef - si.z, T(0));
    const T hyd = own_pressure<T, HR2>(a, hf, si);
    const int kind = tag & 3, grp = tag >> 2;
    const T un = si.uf * nx + si.vf * ny, vt = -si.uf * ny + si.vf * nx;
    T M, P, Tt;
    if (kind == SWE_WALL) {
        M = T(0); P = hyd; Tt = T(0);
    } else if (kind == SWE_OPEN) {
        M = hf * un; P = hf * un * un + hyd; Tt = M * vt;
    } else if (kind == SWE_INFLOW) {
        const T q = a.qlen[grp];
        M = -q; P = (hf > h_eps ? ddiv(q * q, hf) : T(0)) + hyd; Tt = T(0);
    } else {
        const T hg = dmax(a.level[grp] - si.z, T(0));
        WafIn<T> wi{};
        Flux<T> fl = riemann<T, false>(hf, un, vt, hg, un, vt, g, h_eps, wi, 0, a.r_eps);
        M = fl.M; P = hf * un * un + fl.DL2 + hyd; Tt = fl.Tt;
    }
    bs -= L * M;
    return contribution(L, M, P, Tt, nx, ny);
}

// 1 / r of a triangle from its scaled normals: the perimeter over twice the
// area (r = 2A / P, the CFL length of Sec. 6.1).
template <typename T>
__device__ __forceinline__ T inv_inradius(const Vec2<T> ln[3])
{
    const T per = edge_length(ln[0].x, ln[0].y) + edge_length(ln[1].x, ln[1].y) + edge_length(ln[2].x, ln[2].y);
    return ddiv(per, ln[0].x * ln[1].y - ln[0].y * ln[1].x);
}

// The CFL quantity that cell i publishes for its wave speed s: s itself in the
// global form, s / r_i in the local form (normals read here).
template <typename T>
__device__ __forceinline__ T cfl_speed(const StepArgs<T> &a, int64_t i, T s)
{
    if (!a.cfl_local || !(s > T(0))) return s;
    Vec2<T> ln[3];
#pragma unroll
    for (int k = 0; k < 3; k++) ln[k] = a.m.ln[3 * i + k];
    return mul_rn(s, inv_inradius(ln));
}

// Add contribution k (k = 0, 1, 2 in this order) to the cell's sum.
template <typename T>
__device__ __forceinline__ void accumulate(int k, const Contrib<T> &c, T &R0, T &R1, T &R2)
{
    if (k == 0) { R0 = c.c0; R1 = c.c1; R2 = c.c2; }
    else { R0 = add_rn(R0, c.c0); R1 = add_rn(R1, c.c1); R2 = add_rn(R2, c.c2); }
}

// Explicit Euler update, clipping, point-implicit Manning friction and the
// wave speed of the new state.  Area from the scaled normals: |e_0 x e_1|/2.
template <typename T>
__device__ __forceinline__ CellOut<T> cell_finish(const StepArgs<T> &a, T dt, T hi, T hui, T hvi, T R0, T R1, T R2,
                                                  const Vec2<T> ln[3], T nm, T bs)
{
    const T g = a.g, h_eps = a.h_eps, half = T(0.5);
    CellOut<T> o;
    const T area = half * (ln[0].x * ln[1].y - ln[0].y * ln[1].x);
    const T r = ddiv(dt, area);
    T hn = fma_rn(-r, R0, hi), hun = fma_rn(-r, R1, hui), hvn = fma_rn(-r, R2, hvi);
    o.clip = T(0);
    if (hn < T(0)) { o.clip = -hn * area; hn = T(0); }
    if (hn <= h_eps) {
        hun = T(0); hvn = T(0);
    } else if (nm > T(0)) {
        const T sp = ddiv(dsqrt(fma_rn(hun, hun, mul_rn(hvn, hvn))), hn);
        const T fr = T(1) + ddiv(dt * g * nm * nm * sp, dpow43(hn));
        hun = ddiv(hun, fr); hvn = ddiv(hvn, fr);
    }
    o.h = hn; o.hu = hun; o.hv = hvn;
    o.smax = T(0);
    if (hn > h_eps) {
        o.smax = wave_speed(g, hn, hun, hvn);
        if (a.cfl_local) o.smax = mul_rn(o.smax, inv_inradius(ln));
    }
    o.bsum = bs * dt;
    return o;
}

// Edge fluxes and update of one cell, all three edges evaluated by the cell
// (split kernels).  Data of the cell and of its neighbours come through `src`:
//   MUSCL: own_face(k), nbr_face(nb) -> (eta, u, v, z) at the edge midpoint
//   WAF  : nbr_centre(nb) -> (h, u, v, z); own_up(k), nbr_up(nb) -> upwind means
//   HLLC : nbr_state(nb) -> (h, hu, hv, z)
template <typename T, int SCHEME, typename Src>
__device__ __forceinline__ CellOut<T> cell_update(const StepArgs<T> &a, T dt, T hi, T hui, T hvi, T zi, T nm,
                                                  const Nb nb[3], const Vec2<T> ln[3], const Vec2<T> dd[3],
                                                  const Src &src)
{
    const T h_eps = a.h_eps;
    T ui, vi;
    primitives(hi, hui, hvi, h_eps, ui, vi);
    T R0 = T(0), R1 = T(0), R2 = T(0), bs = T(0);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        Side<T> si;
        si.z = zi; si.hc = hi; si.zc = zi;
        if (face_scheme(SCHEME)) {
            const Vec4<T> f = src.own_face(k);
            si.ef = f.x; si.uf = f.y; si.vf = f.z;
            if (SCHEME == FLUX_MUSCL_HR2) si.z = f.w;          // the face bed (R16)
        } else {
            si.ef = hi + zi; si.uf = ui; si.vf = vi;
        }
        Contrib<T> c;
        if (nb[k].interior) {
            Side<T> sj;
            Vec4<T> Ui{}, Uj{};
            T dlen = T(0);
            if (face_scheme(SCHEME)) {
                const Vec4<T> f = src.nbr_face(nb[k]);
                sj.ef = f.x; sj.uf = f.y; sj.vf = f.z; sj.z = f.w; sj.hc = T(0); sj.zc = f.w;
            } else if (SCHEME == SWE_SCHEME_WAF) {
                const Vec4<T> p = src.nbr_centre(nb[k]);
                sj.hc = p.x; sj.uf = p.y; sj.vf = p.z; sj.z = p.w; sj.ef = p.x + p.w; sj.zc = p.w;
                // a dry side's upwind means are not stored (and not needed: R18)
                if (hi > h_eps) Ui = src.own_up(k);
                if (p.x > h_eps) Uj = src.nbr_up(nb[k]);
                dlen = dsqrt(fma_rn(dd[k].x, dd[k].x, mul_rn(dd[k].y, dd[k].y)));
            } else {
                const Vec4<T> q = src.nbr_state(nb[k]);
                sj.hc = q.x; sj.z = q.w; sj.ef = q.x + q.w; sj.zc = q.w;
                primitives(q.x, q.y, q.z, h_eps, sj.uf, sj.vf);
            }
            interior_edge<T, SCHEME>(a, dt, si, sj, nb[k].own, ln[k].x, ln[k].y, dlen, Ui, Uj, c, nullptr);
        } else {
            c = boundary_edge<T, SCHEME == FLUX_MUSCL_HR2>(a, si, nb[k].tag, ln[k].x, ln[k].y, bs);
        }
        accumulate(k, c, R0, R1, R2);
    }
    return cell_finish<T>(a, dt, hi, hui, hvi, R0, R1, R2, ln, nm, bs);
}

// Step epilogue: publish the block's wave speed and diagnostics; block 0
// advances time and the step count and clears the stale CFL slot.
template <typename T>
__device__ __forceinline__ void step_epilogue(const StepArgs<T> &a, T dt, bool dry, T smax, T clip, T bsum,
                                              bool first_block)
{
    const bool euler = a.mode == MODE_EULER;
    block_publish<T>(smax, clip, bsum, a.sc, a.slot_next, euler, euler ? 1.0 : 0.5);
    if (first_block && threadIdx.x == 0) {
        if (dry) atomicOr(&a.sc->status, ST_DRY);
        if (euler) {
            a.dt_hist[a.sc->steps % SWE_DT_HISTORY] = (double)dt;
            a.sc->t += (double)dt;
            a.sc->steps += 1;
            a.sc->smax[a.slot_clear] = 0ULL;
        }
    }
}

}  // namespace swe_dev
