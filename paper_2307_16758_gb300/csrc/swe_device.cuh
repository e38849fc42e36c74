// Device functions shared by the split kernels (swe_kernels.cu) and the fused
// tile kernel (swe_fused.cu): the Riemann solver of Sec. 5.2, the MUSCL face
// values, WAF helpers and the block reductions.  Both kernels inline the same
// code, so a cell gets the same bits whichever kernel computes it.
#pragma once
#include <cuda_runtime.h>

#include "swe_dev.h"

namespace swe_dev {

template <typename T> __device__ __forceinline__ T dsqrt(T x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T dmin(T a, T b) { return a < b ? a : b; }
__device__ __forceinline__ float dcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double dcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ bool dfinite(float x) { return isfinite(x); }
__device__ __forceinline__ bool dfinite(double x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// Riemann problem in the rotated frame.  Inputs are the reconstructed depths
// h*_L, h*_R (after the hydrostatic reconstruction) and the normal (u) and
// tangential (v) velocities of both sides.  Outputs: the mass flux M, the
// tangential momentum flux Tt and, for each side s, D_s = F_2 - G_2(U*_s),
// the normal-momentum flux minus that side's physical flux.  In the star
// region of HLL (Sec. 5.2.1),
//   F - G_L = S_L (S_R dU - dG) / (S_R - S_L),  F - G_R = S_R (S_L dU - dG) / (S_R - S_L),
// which is the printed star flux rearranged so that equal states give an
// exact zero (well-balancing).
// ---------------------------------------------------------------------------
template <typename T> struct Flux { T M, Tt, DL2, DR2; };

template <typename T> struct WafIn {
    T dtdx;            // dt / |c_R - c_L|
    T hupL, hupR;      // upwind mean depth of each side
    T vupL, vupR;      // upwind mean tangential velocity of each side
    T hcL, hcR;        // cell-centre depths
};

template <typename T>
__device__ __forceinline__ T waf_ratio(T r_eps, T upw, T qL, T qR)
{
    T loc = qR - qL;
    T sc = dmax(dmax(fabs(qL), fabs(qR)), T(1));
    if (fabs(loc) <= r_eps * sc) return T(0);
    return upw / loc;
}

// A(r, c) of Sec. 5.2.2 (SUPERBEE), or its phi = 1 / phi = 0 variants.
template <typename T>
__device__ __forceinline__ T waf_A(int lim, T r, T c)
{
    T ac = fabs(c);
    if (lim == SWE_WAF_PHI1) return ac;
    if (lim == SWE_WAF_PHI0) return T(1);
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
    const T half = T(0.5);
    T GL1 = hsL * uL, GL2 = hsL * uL * uL + half * g * hsL * hsL;
    T GR1 = hsR * uR, GR2 = hsR * uR * uR + half * g * hsR * hsR;
    T dU1 = hsR - hsL, dU2 = hsR * uR - hsL * uL;
    T dG1 = GR1 - GL1, dG2 = GR2 - GL2;
    bool dryL = hsL <= h_eps, dryR = hsR <= h_eps;
    if (dryL && dryR) {                    // both sides dry: zero numerical flux
        f.M = T(0); f.Tt = T(0); f.DL2 = -GL2; f.DR2 = -GR2;
        return f;
    }
    T aL = dsqrt(g * hsL), aR = dsqrt(g * hsR);
    T SL, SR;
    if (dryL) {                            // dry-bed wave speeds
        SL = uR - T(2) * aR; SR = uR + aR;
    } else if (dryR) {
        SL = uL - aL; SR = uL + T(2) * aL;
    } else {
        T h0 = (hsL + hsR) / T(2) - (uR - uL) * (hsL + hsR) / (T(4) * (aR + aL));
        T hs;
        if (h0 <= dmin(hsL, hsR)) {        // two rarefactions
            T br = dmax((aR + aL) / T(2) + (uL - uR) / T(4), T(0));
            hs = br * br / g;
        } else {                           // two shocks
            T gL = dsqrt(g * (h0 + hsL) / (T(2) * h0 * hsL));
            T gR = dsqrt(g * (h0 + hsR) / (T(2) * h0 * hsR));
            hs = (hsL * gL + hsR * gR + uL - uR) / (gL + gR);
        }
        T pL = hs > hsL ? dsqrt(hs * (hs + hsL) / T(2)) / hsL : T(1);
        T pR = hs > hsR ? dsqrt(hs * (hs + hsR) / T(2)) / hsR : T(1);
        SL = uL - aL * pL;
        SR = uR + aR * pR;
    }
    T num = SL * hsR * (uR - SR) - SR * hsL * (uL - SL);
    T den = hsR * (uR - SR) - hsL * (uL - SL);
    T Ss = den != T(0) ? num / den : T(0);
    // HLL (three branches) as differences to G_L and G_R
    T hL1, hL2, hR2;
    bool rightgoing = SL >= T(0), leftgoing = !rightgoing && SR <= T(0);
    if (rightgoing) {
        hL1 = T(0); hL2 = T(0); hR2 = -dG2;
    } else if (leftgoing) {
        hL1 = dG1; hL2 = dG2; hR2 = T(0);
    } else {
        T wd = SR - SL;
        hL1 = SL * (SR * dU1 - dG1) / wd;
        hL2 = SL * (SR * dU2 - dG2) / wd;
        hR2 = SR * (SL * dU2 - dG2) / wd;
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
    const T s = T(1) / T(6);
    ox[0] = (-ln[2].y + ln[1].y) * s; oy[0] = (ln[2].x - ln[1].x) * s;
    ox[1] = (-ln[0].y + ln[2].y) * s; oy[1] = (ln[0].x - ln[2].x) * s;
    ox[2] = (-ln[1].y + ln[0].y) * s; oy[2] = (ln[1].x - ln[0].x) * s;
}

template <typename T>
__device__ __forceinline__ void primitives(T h, T hu, T hv, T h_eps, T &u, T &v)
{
    bool wet = h > h_eps;
    u = wet ? hu / h : T(0);
    v = wet ? hv / h : T(0);
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
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Max of s, sums of c1 and c2 over the block; thread 0 publishes them.
template <typename T>
__device__ __forceinline__ void block_publish(T s, double c1, double c2, DevScalars *sc, int slot_next,
                                              bool want_max, double wsum)
{
    __shared__ double sh_s[32], sh_c1[32], sh_c2[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double sd = (double)warp_max(s);
    c1 = warp_sum(c1);
    c2 = warp_sum(c2);
    if (lane == 0) { sh_s[wid] = sd; sh_c1[wid] = c1; sh_c2[wid] = c2; }
    __syncthreads();
    if (wid == 0) {
        sd = lane < nw ? sh_s[lane] : 0.0;
        c1 = lane < nw ? sh_c1[lane] : 0.0;
        c2 = lane < nw ? sh_c2[lane] : 0.0;
        sd = warp_max(sd);
        c1 = warp_sum(c1);
        c2 = warp_sum(c2);
        if (lane == 0) {
            if (want_max && sd > 0.0) atomicMax(&sc->smax[slot_next], (unsigned long long)__double_as_longlong(sd));
            if (c1 != 0.0) atomicAdd(&sc->clipped, wsum * c1);
            if (c2 != 0.0) atomicAdd(&sc->bnd_in, wsum * c2);
        }
    }
}

template <typename T>
__device__ __forceinline__ T step_dt(const StepArgs<T> &a, bool *dry)
{
    if (a.dtv) { *dry = false; return (T)a.dtv[0]; }
    double sm = __longlong_as_double((long long)a.sc->smax[a.slot_cur]);
    *dry = !(sm > 0.0);
    if (*dry) return T(0);
    return (T)a.cfl_rmin / (T)sm;
}


}  // namespace swe_dev
