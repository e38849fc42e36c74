// Device code of the one-pass tile step (one tile of a mesh), shared by the
// single-mesh kernel (swe_tile.cu) and the batched ensemble kernel
// (swe_ensemble.cu).
//
// A tile is a run of B consecutive (Morton-ordered) cells, one per thread.
// One launch per time step advances every tile:
//   A  each thread loads its cell (state, bed, neighbour words, scaled
//      normals) into shared memory and counts the edges it lists: every edge
//      with both cells in the tile once (from its lower slot) and every edge
//      towards another tile (a crossing edge) from the tile's side; a
//      block-wide scan places them, crossing edges first;
//   B  MUSCL face values of the tile's cells from shared memory (least
//      squares + Barth-Jespersen, the MUSCL idea of Sec. 6.2.3); a cell with
//      a neighbour outside the tile gathers that neighbour from global memory;
//   C  one thread per listed edge: for a crossing edge the face value of the
//      far cell is recomputed from global memory (its gradient needs its own
//      neighbours), then the hydrostatic reconstruction and the
//      canonical-orientation Riemann flux (Sec. 6.2.1); the contribution to
//      each tile cell on the edge goes to shared memory;
//   D  each cell adds its three contributions in edge order (boundary edges
//      of the domain evaluated here), updates, clips, applies friction and
//      publishes its wave speed.
// Face values never leave the chip, and every edge inside a tile is solved
// once.  The per-edge and per-cell arithmetic is the split kernels' device
// code, so a cell gets the same bits whichever path advances it.
#pragma once
#include "swe_device.cuh"
#include "swe_split.cuh"

namespace swe_dev {

// Edge records.  Inside the tile: slot_i | k_i << 10 | slot_j << 12 |
// k_j << 22 | own_i << 24.  Crossing: slot_i | k_i << 10 | k_j << 12 |
// own_i << 14, with the far cell's id in a second word.
__device__ __forceinline__ uint32_t tile_edge(int si, int ki, int sj, int kj, bool own)
{
    return (uint32_t)si | ((uint32_t)ki << 10) | ((uint32_t)sj << 12) | ((uint32_t)kj << 22) | ((uint32_t)own << 24);
}
__device__ __forceinline__ uint32_t cross_edge(int si, int ki, int kj, bool own)
{
    return (uint32_t)si | ((uint32_t)ki << 10) | ((uint32_t)kj << 12) | ((uint32_t)own << 14);
}

// Shared-memory layout of a tile of B cells with room for emax edges inside
// the tile and xmax crossing edges.  Per-face arrays are slot-major
// ([slot * 3 + k]) so that neighbouring threads touch neighbouring words.
template <typename T> struct TileSmem {
    Vec4<T> *P;          // [B]     (eta, u, v, h) at the cell centre
    Vec2<T> *Ln;         // [B][3]  scaled outward normals
    T *Z;                // [B]     bed
    T *Fe, *Fu, *Fv;     // [B][3]  face values (eta, u, v) at the edge midpoints
    T *C0, *C1, *C2;     // [B][3]  edge contributions
    uint32_t *IE;        // [emax]  edges inside the tile
    uint32_t *XE;        // [xmax]  crossing edges
    int32_t *XJ;         // [xmax]  far cell of each crossing edge
    int *scan;           // [33]    per-warp sums of the block scan, then the totals

    static __host__ __device__ size_t bytes(int B, int emax, int xmax)
    {
        return (size_t)B * sizeof(Vec4<T>) + 3 * (size_t)B * sizeof(Vec2<T>) + (size_t)B * sizeof(T) +
               6 * 3 * (size_t)B * sizeof(T) + (size_t)emax * sizeof(uint32_t) + 2 * (size_t)xmax * sizeof(uint32_t) +
               40 * sizeof(int);
    }

    __device__ TileSmem(unsigned char *base, int B, int emax, int xmax)
    {
        P = reinterpret_cast<Vec4<T> *>(base);
        Ln = reinterpret_cast<Vec2<T> *>(P + B);
        Z = reinterpret_cast<T *>(Ln + 3 * B);
        Fe = Z + B; Fu = Fe + 3 * B; Fv = Fu + 3 * B;
        C0 = Fv + 3 * B; C1 = C0 + 3 * B; C2 = C1 + 3 * B;
        IE = reinterpret_cast<uint32_t *>(C2 + 3 * B);
        XE = IE + emax;
        XJ = reinterpret_cast<int32_t *>(XE + xmax);
        scan = XJ + xmax;
    }
};

// Exclusive scan of v over the block (two 16-bit counters packed in one int);
// returns the thread's offset and leaves the block total in *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *sh, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;          // inclusive prefix of the warp sums
        if (lane == nw - 1) sh[32] = s;
    }
    __syncthreads();
    *total = sh[32];
    return x - v + (wid > 0 ? sh[wid - 1] : 0);
}

// One tile (tile index b, cells s0 .. s0 + nc - 1 of the mesh of `a`).
// SCHEME: SWE_SCHEME_MUSCL or SWE_SCHEME_HLLC.  A tile whose edge lists
// would not fit (emax, xmax) raises ST_TILE in the status word and leaves
// its cells' new state unwritten.
template <typename T, int SCHEME>
__device__ __forceinline__ void tile_step(const StepArgs<T> &a, int b, int emax, int xmax, unsigned char *smem_raw)
{
    constexpr bool MUSCL = SCHEME == SWE_SCHEME_MUSCL;
    const int B = blockDim.x, t = threadIdx.x;
    TileSmem<T> sm(smem_raw, B, emax, xmax);
    const int64_t s0 = (int64_t)b * B;
    const int nc = (int)(a.m.n - s0 < (int64_t)B ? a.m.n - s0 : (int64_t)B);
    const bool valid = t < nc;
    const int64_t i = s0 + t;
    const T h_eps = a.h_eps;
    bool dry;
    const T dt = block_dt(a, &dry);

    // ---- A: the cell, its primitives and its edges ----
    T hi = T(0), hui = T(0), hvi = T(0), zi = T(0), ui = T(0), vi = T(0), nm = T(0);
    int w[3] = {-1, -1, -1};
    if (valid) {
        hi = a.h[i]; hui = a.hu[i]; hvi = a.hv[i]; zi = a.m.z[i];
        nm = a.m.nman ? a.m.nman[i] : T(0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            w[k] = a.m.nbr[3 * i + k];
            sm.Ln[3 * t + k] = a.m.ln[3 * i + k];
        }
        primitives(hi, hui, hvi, h_eps, ui, vi);
    }
    {
        Vec4<T> p;
        p.x = hi + zi; p.y = ui; p.z = vi; p.w = hi;
        sm.P[t] = p;
        sm.Z[t] = zi;
    }
    // edges inside the tile this thread lists (low 16 bits), crossing edges (high 16 bits)
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (w[k] < 0) continue;
        const int64_t sj = (int64_t)(w[k] >> 3) - s0;
        if (sj >= 0 && sj < nc) cnt += sj > t ? 1 : 0;
        else cnt += 1 << 16;
    }
    int total;
    const int base = block_exclusive_scan(cnt, sm.scan, &total);     // (its barriers publish P, Z, Ln)
    const int n_in = total & 0xffff, n_cross = total >> 16;
    if (n_in > emax || n_cross > xmax) {
        if (t == 0) atomicOr(&a.sc->status, ST_TILE);
        return;                                                       // uniform over the block
    }

    // ---- B: face values and the edge lists ----
    if (valid) {
        int pe = base & 0xffff, px = base >> 16;
        bool inside = true;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (w[k] < 0) continue;
            const int j = w[k] >> 3, kj = (w[k] >> 1) & 3;
            const int64_t sj = (int64_t)j - s0;
            const bool own = w[k] & 1;
            if (sj >= 0 && sj < nc) {
                if (sj > t) sm.IE[pe++] = tile_edge(t, k, (int)sj, kj, own);
            } else {
                sm.XE[px] = cross_edge(t, k, kj, own);
                sm.XJ[px] = j;
                px++;
                inside = false;
            }
        }
        T fe[3], fu[3], fv[3];
        if (!MUSCL || hi <= h_eps) {
            // first order, or a dry cell (zero gradient, zero velocity): the
            // face values are the centre values
#pragma unroll
            for (int k = 0; k < 3; k++) { fe[k] = hi + zi; fu[k] = ui; fv[k] = vi; }
        } else {
            T qi[3] = {hi + zi, ui, vi};
            T qn[3][3], ox[3], oy[3];
            Vec2<T> ln[3], dd[3];
            bool has[3];
            bool ok = true;
            int cnt_n = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) ln[k] = sm.Ln[3 * t + k];
            midpoint_offsets(ln, ox, oy);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                has[k] = w[k] >= 0;
                if (has[k]) {
                    const int j = w[k] >> 3, kj = (w[k] >> 1) & 3;
                    const int k1 = kj == 2 ? 0 : kj + 1, k2 = kj == 0 ? 2 : kj - 1;
                    const int64_t sj = (int64_t)j - s0;
                    T hj, ej, uj, vj;
                    Vec2<T> a1, a2;
                    if (inside || (sj >= 0 && sj < nc)) {
                        const Vec4<T> pj = sm.P[sj];
                        ej = pj.x; uj = pj.y; vj = pj.z; hj = pj.w;
                        a1 = sm.Ln[3 * sj + k1]; a2 = sm.Ln[3 * sj + k2];
                    } else {
                        hj = a.h[j];
                        primitives(hj, a.hu[j], a.hv[j], h_eps, uj, vj);
                        ej = hj + a.m.z[j];
                        a1 = a.m.ln[3 * (int64_t)j + k1]; a2 = a.m.ln[3 * (int64_t)j + k2];
                    }
                    ok = ok && hj > h_eps;
                    qn[k][0] = ej; qn[k][1] = uj; qn[k][2] = vj;
                    dd[k] = centroid_offset_from(ox[k], oy[k], a1, a2);
                    cnt_n++;
                } else {
                    qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
                    dd[k].x = T(0); dd[k].y = T(0);
                }
            }
            Vec4<T> f[3];
            muscl_faces<T, 3>(qi, zi, ok, cnt_n, qn, has, ox, oy, dd, f);
#pragma unroll
            for (int k = 0; k < 3; k++) { fe[k] = f[k].x; fu[k] = f[k].y; fv[k] = f[k].z; }
        }
#pragma unroll
        for (int k = 0; k < 3; k++) { sm.Fe[3 * t + k] = fe[k]; sm.Fu[3 * t + k] = fu[k]; sm.Fv[3 * t + k] = fv[k]; }
    }
    __syncthreads();

    // ---- C: one thread per listed edge, crossing edges first ----
    const int n_edges = n_cross + n_in;
    for (int e = t; e < n_edges; e += B) {
        int si, ki, kj, far = 0;
        bool own, cross = e < n_cross;
        Side<T> Sj;
        if (cross) {
            const uint32_t r = sm.XE[e];
            si = (int)(r & 1023u); ki = (int)((r >> 10) & 3u); kj = (int)((r >> 12) & 3u); own = (r >> 14) & 1u;
            const int j = sm.XJ[e];
            Vec4<T> f;
            if (MUSCL) {
                Vec4<T> fj[3];
                muscl_cell_faces<T, 3>(a, j, fj);           // the far cell's face values, recomputed
                f = kj == 0 ? fj[0] : (kj == 1 ? fj[1] : fj[2]);
            } else {
                const T hj = a.h[j], zj = a.m.z[j];
                T uj, vj;
                primitives(hj, a.hu[j], a.hv[j], h_eps, uj, vj);
                f.x = hj + zj; f.y = uj; f.z = vj; f.w = zj;
            }
            Sj.ef = f.x; Sj.uf = f.y; Sj.vf = f.z; Sj.z = f.w; Sj.zc = f.w; Sj.hc = T(0);
        } else {
            const uint32_t r = sm.IE[e - n_cross];
            si = (int)(r & 1023u); ki = (int)((r >> 10) & 3u); far = (int)((r >> 12) & 1023u);
            kj = (int)((r >> 22) & 3u); own = (r >> 24) & 1u;
            Sj.ef = sm.Fe[3 * far + kj]; Sj.uf = sm.Fu[3 * far + kj]; Sj.vf = sm.Fv[3 * far + kj];
            Sj.z = sm.Z[far]; Sj.zc = Sj.z; Sj.hc = sm.P[far].w;
        }
        Side<T> Si;
        Si.ef = sm.Fe[3 * si + ki]; Si.uf = sm.Fu[3 * si + ki]; Si.vf = sm.Fv[3 * si + ki];
        Si.z = sm.Z[si]; Si.zc = Si.z; Si.hc = sm.P[si].w;
        const Vec2<T> l = sm.Ln[3 * si + ki];
        const Vec4<T> none{};
        Contrib<T> ci, cj;
        interior_edge<T, MUSCL ? SWE_SCHEME_MUSCL : SWE_SCHEME_HLLC>(a, dt, Si, Sj, own, l.x, l.y, T(0), none, none,
                                                                    ci, cross ? nullptr : &cj);
        sm.C0[3 * si + ki] = ci.c0; sm.C1[3 * si + ki] = ci.c1; sm.C2[3 * si + ki] = ci.c2;
        if (!cross) { sm.C0[3 * far + kj] = cj.c0; sm.C1[3 * far + kj] = cj.c1; sm.C2[3 * far + kj] = cj.c2; }
    }
    __syncthreads();

    // ---- D: sums in edge order, update ----
    CellOut<T> o;
    o.smax = T(0); o.clip = T(0); o.bsum = T(0);
    if (valid) {
        Vec2<T> ln[3];
#pragma unroll
        for (int k = 0; k < 3; k++) ln[k] = sm.Ln[3 * t + k];
        T R0 = T(0), R1 = T(0), R2 = T(0), bs = T(0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Contrib<T> c;
            if (w[k] >= 0) {
                c.c0 = sm.C0[3 * t + k]; c.c1 = sm.C1[3 * t + k]; c.c2 = sm.C2[3 * t + k];
            } else {
                Side<T> s;
                s.ef = sm.Fe[3 * t + k]; s.uf = sm.Fu[3 * t + k]; s.vf = sm.Fv[3 * t + k];
                s.z = zi; s.zc = zi; s.hc = hi;
                c = boundary_edge<T>(a, s, -1 - w[k], ln[k].x, ln[k].y, bs);
            }
            accumulate(k, c, R0, R1, R2);
        }
        o = cell_finish<T>(a, dt, hi, hui, hvi, R0, R1, R2, ln, nm, bs);
        a.ho[i] = o.h; a.huo[i] = o.hu; a.hvo[i] = o.hv;
        if (!(dfinite(o.h) && dfinite(o.hu) && dfinite(o.hv))) atomicOr(&a.sc->status, ST_NONFINITE);
    }
    step_epilogue<T>(a, dt, dry, o.smax, o.clip, o.bsum, b == 0);
}

}  // namespace swe_dev
