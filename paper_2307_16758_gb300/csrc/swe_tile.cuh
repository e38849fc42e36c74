// Device code of the one-pass tile step, shared by the single-mesh kernel
// and the batched ensemble kernel (both in swe_tile.cu).
//
// A tile is a run of B consecutive (Morton-ordered) cells, one per thread.
// The kernel is persistent: each block loops over tiles through a pipeline
// of shared-memory stages.  A stage receives a tile's contiguous per-cell
// arrays (scaled normals, state, bed, Manning n, neighbour words) and its
// plan (see swe_tiles.h) by bulk asynchronous copies (cp.async.bulk on an
// mbarrier); the state and normals of the tile's halo -- the outside cells
// it reads: the far cells of its crossing edges (H1) and their other
// neighbours (H2) -- are gathered into the stage by cp.async one tile ahead.
// Every phase of a tile then reads shared memory only:
//   A  primitives of the tile and halo cells; each thread counts the edges
//      it lists: every edge with both cells in the tile once (from its lower
//      slot) and every edge towards another tile (a crossing edge) from the
//      tile's side; a block-wide scan places them, crossing edges first;
//   B  MUSCL face values (least squares + Barth-Jespersen, the MUSCL idea of
//      Sec. 6.2.3) of the tile's cells and of the H1 cells;
//   C  one thread per listed edge: hydrostatic reconstruction and the
//      canonical-orientation Riemann flux (Sec. 6.2.1); the contribution to
//      each tile cell on the edge goes to shared memory;
//   D  each cell adds its three contributions in edge order (boundary edges
//      of the domain evaluated here), updates, clips, applies friction and
//      publishes its wave speed.
// Face values never leave the chip, every edge inside a tile is solved once,
// and the per-edge and per-cell arithmetic is the split kernels' device code,
// so a cell gets the same bits whichever path advances it.
#pragma once
#include "swe_async.cuh"
#include "swe_device.cuh"
#include "swe_split.cuh"

namespace swe_dev {

// Stages of the tile pipeline (tiles in flight per block).
constexpr int kTileStages = 2;
// Polls of an mbarrier before a block gives up on a copy (ST_TIMEOUT).
constexpr uint32_t kWaitPolls = 1u << 22;

// Edge records.  Inside the tile: slot_i | k_i << 10 | slot_j << 12 |
// k_j << 22 | own_i << 24.  Crossing: slot_i | k_i << 10 | k_j << 12 |
// own_i << 14 (the far cell follows from the plan).
__device__ __forceinline__ uint32_t tile_edge(int si, int ki, int sj, int kj, bool own)
{
    return (uint32_t)si | ((uint32_t)ki << 10) | ((uint32_t)sj << 12) | ((uint32_t)kj << 22) | ((uint32_t)own << 24);
}
__device__ __forceinline__ uint32_t cross_edge(int si, int ki, int kj, bool own)
{
    return (uint32_t)si | ((uint32_t)ki << 10) | ((uint32_t)kj << 12) | ((uint32_t)own << 14);
}

// Room a block reserves per stage: B cells, hmax halo cells, wmax plan words.
struct TileDims {
    int B, emax, xmax, hmax, h1max, wmax;
};

// One stage: a tile's inputs.  Every array starts on a 32-byte boundary when
// B is a power of two of at least 32, hmax a multiple of 4 and wmax of 8.
template <typename T> struct TileStage {
    Vec2<T> *ln;         // [3B]      scaled outward normals
    T *h, *hu, *hv, *z;  // [B]
    T *nm;               // [B]       Manning n (friction only)
    int32_t *nbr;        // [3B]      packed neighbour words
    int32_t *hdr;        // [8]       plan header: offset, halo cells, H1 cells, crossing edges
    Vec4<T> *hs;         // [hmax]    halo state (h, hu, hv, z), gathered
    Vec2<T> *hl;         // [3 hmax]  halo scaled normals, gathered
    int32_t *words;      // [wmax]    plan words

    static __host__ __device__ size_t bytes(const TileDims &d)
    {
        return 3 * (size_t)d.B * sizeof(Vec2<T>) + 5 * (size_t)d.B * sizeof(T) + 3 * (size_t)d.B * 4 + 32 +
               (size_t)d.hmax * (sizeof(Vec4<T>) + 3 * sizeof(Vec2<T>)) + (size_t)d.wmax * 4;
    }

    __device__ void place(unsigned char *base, const TileDims &d)
    {
        const int B = d.B;
        ln = reinterpret_cast<Vec2<T> *>(base);
        h = reinterpret_cast<T *>(ln + 3 * B);
        hu = h + B; hv = hu + B; z = hv + B; nm = z + B;
        nbr = reinterpret_cast<int32_t *>(nm + B);
        hdr = nbr + 3 * B;
        hs = reinterpret_cast<Vec4<T> *>(hdr + 8);
        hl = reinterpret_cast<Vec2<T> *>(hs + d.hmax);
        words = reinterpret_cast<int32_t *>(hl + 3 * d.hmax);
    }
};

// Shared memory of a block: the stages and their mbarriers, then the
// working arrays of the tile being computed.  Per-face arrays are
// slot-major ([slot * 3 + k]) so that neighbouring threads touch
// neighbouring words.  Addresses are recomputed from the base on use.
template <typename T> struct TileSmem {
    unsigned char *base;
    TileDims d;
    Vec4<T> *P;          // [B]       (eta, u, v, h) of the tile's cells
    Vec4<T> *HP;         // [hmax]    (eta, u, v, h) of the halo cells
    T *Fe, *Fu, *Fv;     // [B][3]    face values (eta, u, v) at the edge midpoints
    T *C0, *C1, *C2;     // [B][3]    edge contributions
    T *Ge, *Gu, *Gv;     // [h1max][3] face values of the H1 cells
    uint32_t *IE;        // [emax]    edges inside the tile
    uint32_t *XE;        // [xmax]    crossing edges
    int *scan;           // [40]      block scan

    static __host__ __device__ size_t bytes(const TileDims &d)
    {
        return kTileStages * TileStage<T>::bytes(d) + 64 + ((size_t)d.B + d.hmax) * sizeof(Vec4<T>) +
               (6 * 3 * (size_t)d.B + 3 * 3 * (size_t)d.h1max) * sizeof(T) + ((size_t)d.emax + d.xmax) * 4 + 40 * 4;
    }

    __device__ TileSmem(unsigned char *base_, const TileDims &d_) : base(base_), d(d_)
    {
        unsigned char *p = base + kTileStages * TileStage<T>::bytes(d) + 64;
        P = reinterpret_cast<Vec4<T> *>(p);
        HP = P + d.B;
        Fe = reinterpret_cast<T *>(HP + d.hmax); Fu = Fe + 3 * d.B; Fv = Fu + 3 * d.B;
        C0 = Fv + 3 * d.B; C1 = C0 + 3 * d.B; C2 = C1 + 3 * d.B;
        Ge = C2 + 3 * d.B; Gu = Ge + 3 * d.h1max; Gv = Gu + 3 * d.h1max;
        IE = reinterpret_cast<uint32_t *>(Gv + 3 * d.h1max);
        XE = IE + d.emax;
        scan = reinterpret_cast<int *>(XE + d.xmax);
    }

    __device__ TileStage<T> stage(int s) const
    {
        TileStage<T> st;
        st.place(base + s * TileStage<T>::bytes(d), d);
        return st;
    }
    __device__ uint64_t *bar(int s) const
    {
        return reinterpret_cast<uint64_t *>(base + kTileStages * TileStage<T>::bytes(d)) + s;
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

// Thread 0: start the bulk copies of tile b (of the mesh of `a`, plan `ta`)
// into a stage; hdr is the tile's plan header (offset, halo, H1, crossing).
// The per-cell arrays are allocated to a whole number of tiles, so a full
// tile is copied even at the end of the mesh.
template <typename T>
__device__ __forceinline__ void tile_issue(const StepArgs<T> &a, const TileArgs &ta, int64_t b, int4 hdr,
                                           const TileStage<T> &st, uint64_t *bar)
{
    const int B = blockDim.x;
    const int64_t s0 = b * B;
    const uint32_t fb = (uint32_t)(B * sizeof(T));
    const bool fric = a.m.nman != nullptr;
    const uint32_t nw = (uint32_t)((hdr.y + 3 * hdr.z + hdr.w + 3) & ~3);
    mbar_arrive_expect(bar, 3 * (uint32_t)B * (uint32_t)sizeof(Vec2<T>) + (fric ? 5 : 4) * fb + 12 * (uint32_t)B + 16 +
                                4 * nw);
    bulk_load(st.ln, a.m.ln + 3 * s0, 3 * (uint32_t)B * (uint32_t)sizeof(Vec2<T>), bar);
    bulk_load(st.h, a.h + s0, fb, bar);
    bulk_load(st.hu, a.hu + s0, fb, bar);
    bulk_load(st.hv, a.hv + s0, fb, bar);
    bulk_load(st.z, a.m.z + s0, fb, bar);
    if (fric) bulk_load(st.nm, a.m.nman + s0, fb, bar);
    bulk_load(st.nbr, a.m.nbr + 3 * s0, 12 * (uint32_t)B, bar);
    bulk_load(st.hdr, ta.plan_hdr + 4 * b, 16, bar);
    if (nw) bulk_load(st.words, ta.plan_words + hdr.x, 4 * nw, bar);
}

// All threads: gather the state and normals of the stage's halo cells
// (H1 only for first-order HLLC) with cp.async, one commit group per thread.
template <typename T, bool H2>
__device__ __forceinline__ void tile_gather(const StepArgs<T> &a, const TileStage<T> &st)
{
    const int nh = H2 ? st.hdr[1] : st.hdr[2];
    for (int q = threadIdx.x; q < nh; q += blockDim.x) {
        const int64_t id = st.words[q];
        cp_async<sizeof(T)>(&st.hs[q].x, a.h + id);
        cp_async<sizeof(T)>(&st.hs[q].y, a.hu + id);
        cp_async<sizeof(T)>(&st.hs[q].z, a.hv + id);
        cp_async<sizeof(T)>(&st.hs[q].w, a.m.z + id);
#pragma unroll
        for (int k = 0; k < 3; k++) cp_async<sizeof(Vec2<T>)>(&st.hl[3 * q + k], a.m.ln + 3 * id + k);
    }
    cp_async_commit();
}


// Primitives (eta, u, v, h) of a cell from (h, hu, hv, z).
template <typename T> __device__ __forceinline__ Vec4<T> prim4(T h, T hu, T hv, T z, T h_eps)
{
    Vec4<T> p;
    T u, v;
    primitives(h, hu, hv, h_eps, u, v);
    p.x = h + z; p.y = u; p.z = v; p.w = h;
    return p;
}

// MUSCL face values of a wet cell from its primitives pi, bed zi, scaled
// normals ln and, per local edge k, whether it has a neighbour, the
// neighbour's primitives pn[k] and the neighbour's scaled normals of its
// edges k' + 1 and k' + 2 (k' its local index of the shared edge).  The
// arithmetic of prep_muscl_cell / muscl_cell_faces, operand for operand.
template <typename T>
__device__ __forceinline__ void faces_from(const Vec4<T> &pi, T zi, const Vec2<T> ln[3], const bool has[3],
                                           const Vec4<T> pn[3], const Vec2<T> a1[3], const Vec2<T> a2[3], T h_eps,
                                           T fe[3], T fu[3], T fv[3])
{
    T qi[3] = {pi.x, pi.y, pi.z};
    T qn[3][3], ox[3], oy[3];
    Vec2<T> dd[3];
    bool ok = pi.w > h_eps;
    int cnt = 0;
    midpoint_offsets(ln, ox, oy);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (has[k]) {
            ok = ok && pn[k].w > h_eps;
            qn[k][0] = pn[k].x; qn[k][1] = pn[k].y; qn[k][2] = pn[k].z;
            dd[k] = centroid_offset_from(ox[k], oy[k], a1[k], a2[k]);
            cnt++;
        } else {
            qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
            dd[k].x = T(0); dd[k].y = T(0);
        }
    }
    Vec4<T> f[3];
    muscl_faces<T, 3>(qi, zi, ok, cnt, qn, has, ox, oy, dd, f);
#pragma unroll
    for (int k = 0; k < 3; k++) { fe[k] = f[k].x; fu[k] = f[k].y; fv[k] = f[k].z; }
}

// One tile (index b, cells s0 .. s0 + nc - 1 of the mesh of `a`) whose inputs
// and halo are in stage `st`.  SCHEME: SWE_SCHEME_MUSCL or SWE_SCHEME_HLLC.
// Returns the tile's wave speed, clipped mass and boundary mass in o; false
// (block uniform) if its edge lists do not fit the room reserved.
template <typename T, int SCHEME>
__device__ __forceinline__ bool tile_compute(const StepArgs<T> &a, int64_t b, const TileSmem<T> &sm,
                                             const TileStage<T> &st, T dt, CellOut<T> &o)
{
    constexpr bool MUSCL = SCHEME == SWE_SCHEME_MUSCL;
    const int B = blockDim.x, t = threadIdx.x;
    const int64_t s0 = b * B;
    const int nc = (int)(a.m.n - s0 < (int64_t)B ? a.m.n - s0 : (int64_t)B);
    const bool valid = t < nc;
    const int64_t i = s0 + t;
    const T h_eps = a.h_eps;
    const int n_halo = st.hdr[1], n_h1 = st.hdr[2];
    const int32_t *h1nb = st.words + n_halo;           // [3 * n_h1]
    const int32_t *xfar = h1nb + 3 * n_h1;             // [n_cross]

    // ---- A: primitives and the edge counts ----
    T hi = T(0), hui = T(0), hvi = T(0), zi = T(0);
    int w[3] = {-1, -1, -1};
    if (valid) {
        hi = st.h[t]; hui = st.hu[t]; hvi = st.hv[t]; zi = st.z[t];
#pragma unroll
        for (int k = 0; k < 3; k++) w[k] = st.nbr[3 * t + k];
    }
    const Vec4<T> pi = prim4(hi, hui, hvi, zi, h_eps);
    sm.P[t] = pi;
    const int n_prim = MUSCL ? n_halo : n_h1;
    for (int q = t; q < (n_prim < sm.d.hmax ? n_prim : sm.d.hmax); q += B) {
        const Vec4<T> hq = st.hs[q];
        sm.HP[q] = prim4(hq.x, hq.y, hq.z, hq.w, h_eps);
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
    const int base = block_exclusive_scan(cnt, sm.scan, &total);     // (its barriers publish P, HP)
    const int n_in = total & 0xffff, n_cross = total >> 16;
    if (n_in > sm.d.emax || n_cross > sm.d.xmax || n_cross != st.hdr[3] || n_halo > sm.d.hmax || n_h1 > sm.d.h1max)
        return false;                                                 // uniform over the block

    // ---- B: face values and the edge lists ----
    if (valid) {
        int pe = base & 0xffff, px = base >> 16;
        int xk[3] = {-1, -1, -1};                      // crossing index of each local edge
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
                xk[k] = px++;
            }
        }
        T fe[3], fu[3], fv[3];
        if (!MUSCL || hi <= h_eps) {
            // first order, or a dry cell (zero gradient, zero velocity): the
            // face values are the centre values
#pragma unroll
            for (int k = 0; k < 3; k++) { fe[k] = pi.x; fu[k] = pi.y; fv[k] = pi.z; }
        } else {
            Vec2<T> ln[3], a1[3], a2[3];
            Vec4<T> pn[3];
            bool has[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                ln[k] = st.ln[3 * t + k];
                has[k] = w[k] >= 0;
                if (has[k]) {
                    const int kj = (w[k] >> 1) & 3;
                    const int k1 = kj == 2 ? 0 : kj + 1, k2 = kj == 0 ? 2 : kj - 1;
                    if (xk[k] < 0) {
                        const int sj = (w[k] >> 3) - (int)s0;
                        pn[k] = sm.P[sj]; a1[k] = st.ln[3 * sj + k1]; a2[k] = st.ln[3 * sj + k2];
                    } else {
                        const int q = xfar[xk[k]];
                        pn[k] = sm.HP[q]; a1[k] = st.hl[3 * q + k1]; a2[k] = st.hl[3 * q + k2];
                    }
                } else {
                    pn[k] = pi; a1[k] = ln[k]; a2[k] = ln[k];
                }
            }
            faces_from(pi, zi, ln, has, pn, a1, a2, h_eps, fe, fu, fv);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) { sm.Fe[3 * t + k] = fe[k]; sm.Fu[3 * t + k] = fu[k]; sm.Fv[3 * t + k] = fv[k]; }
    }
    // face values of the H1 cells (the far sides of the crossing edges)
    if (MUSCL) {
        for (int q = t; q < n_h1; q += B) {
            const Vec4<T> pq = sm.HP[q];
            const T zq = st.hs[q].w;
            T fe[3], fu[3], fv[3];
            if (pq.w <= h_eps) {
#pragma unroll
                for (int k = 0; k < 3; k++) { fe[k] = pq.x; fu[k] = pq.y; fv[k] = pq.z; }
            } else {
                Vec2<T> ln[3], a1[3], a2[3];
                Vec4<T> pn[3];
                bool has[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    ln[k] = st.hl[3 * q + k];
                    const int wq = h1nb[3 * q + k];
                    has[k] = wq >= 0;
                    if (has[k]) {
                        const int slot = wq >> 3, kj = (wq >> 1) & 3;
                        const int k1 = kj == 2 ? 0 : kj + 1, k2 = kj == 0 ? 2 : kj - 1;
                        if (slot < B) {
                            pn[k] = sm.P[slot]; a1[k] = st.ln[3 * slot + k1]; a2[k] = st.ln[3 * slot + k2];
                        } else {
                            const int r = slot - B;
                            pn[k] = sm.HP[r]; a1[k] = st.hl[3 * r + k1]; a2[k] = st.hl[3 * r + k2];
                        }
                    } else {
                        pn[k] = pq; a1[k] = ln[k]; a2[k] = ln[k];
                    }
                }
                faces_from(pq, zq, ln, has, pn, a1, a2, h_eps, fe, fu, fv);
            }
#pragma unroll
            for (int k = 0; k < 3; k++) { sm.Ge[3 * q + k] = fe[k]; sm.Gu[3 * q + k] = fu[k]; sm.Gv[3 * q + k] = fv[k]; }
        }
    }
    __syncthreads();


    // ---- C: one thread per listed edge, crossing edges first ----
    const int n_edges = n_cross + n_in;
    for (int e = t; e < n_edges; e += B) {
        int si, ki, kj, far;
        bool own, cross = e < n_cross;
        Side<T> Sj;
        if (cross) {
            const uint32_t r = sm.XE[e];
            si = (int)(r & 1023u); ki = (int)((r >> 10) & 3u); kj = (int)((r >> 12) & 3u); own = (r >> 14) & 1u;
            far = xfar[e];
            if (MUSCL) {
                Sj.ef = sm.Ge[3 * far + kj]; Sj.uf = sm.Gu[3 * far + kj]; Sj.vf = sm.Gv[3 * far + kj];
            } else {
                const Vec4<T> pf = sm.HP[far];
                Sj.ef = pf.x; Sj.uf = pf.y; Sj.vf = pf.z;
            }
            Sj.z = st.hs[far].w; Sj.zc = Sj.z; Sj.hc = T(0);
        } else {
            const uint32_t r = sm.IE[e - n_cross];
            si = (int)(r & 1023u); ki = (int)((r >> 10) & 3u); far = (int)((r >> 12) & 1023u);
            kj = (int)((r >> 22) & 3u); own = (r >> 24) & 1u;
            Sj.ef = sm.Fe[3 * far + kj]; Sj.uf = sm.Fu[3 * far + kj]; Sj.vf = sm.Fv[3 * far + kj];
            Sj.z = st.z[far]; Sj.zc = Sj.z; Sj.hc = sm.P[far].w;
        }
        Side<T> Si;
        Si.ef = sm.Fe[3 * si + ki]; Si.uf = sm.Fu[3 * si + ki]; Si.vf = sm.Fv[3 * si + ki];
        Si.z = st.z[si]; Si.zc = Si.z; Si.hc = sm.P[si].w;
        const Vec2<T> l = st.ln[3 * si + ki];
        const Vec4<T> none{};
        Contrib<T> ci, cj;
        interior_edge<T, MUSCL ? SWE_SCHEME_MUSCL : SWE_SCHEME_HLLC>(a, dt, Si, Sj, own, l.x, l.y, T(0), none, none,
                                                                    ci, cross ? nullptr : &cj);
        sm.C0[3 * si + ki] = ci.c0; sm.C1[3 * si + ki] = ci.c1; sm.C2[3 * si + ki] = ci.c2;
        if (!cross) { sm.C0[3 * far + kj] = cj.c0; sm.C1[3 * far + kj] = cj.c1; sm.C2[3 * far + kj] = cj.c2; }
    }
    __syncthreads();

    // ---- D: sums in edge order, update ----
    o.smax = T(0); o.clip = T(0); o.bsum = T(0);
    if (valid) {
        Vec2<T> ln[3];
#pragma unroll
        for (int k = 0; k < 3; k++) ln[k] = st.ln[3 * t + k];
        T R0 = T(0), R1 = T(0), R2 = T(0), bs = T(0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Contrib<T> c;
            if (w[k] >= 0) {
                c.c0 = sm.C0[3 * t + k]; c.c1 = sm.C1[3 * t + k]; c.c2 = sm.C2[3 * t + k];
            } else {
                Side<T> sd;
                sd.ef = sm.Fe[3 * t + k]; sd.uf = sm.Fu[3 * t + k]; sd.vf = sm.Fv[3 * t + k];
                sd.z = zi; sd.zc = zi; sd.hc = hi;
                c = boundary_edge<T>(a, sd, -1 - w[k], ln[k].x, ln[k].y, bs);
            }
            accumulate(k, c, R0, R1, R2);
        }
        const T nm = a.m.nman ? st.nm[t] : T(0);
        o = cell_finish<T>(a, dt, hi, hui, hvi, R0, R1, R2, ln, nm, bs);
        a.ho[i] = o.h; a.huo[i] = o.hu; a.hvo[i] = o.hv;
        if (!(dfinite(o.h) && dfinite(o.hu) && dfinite(o.hv))) atomicOr(&a.sc->status, ST_NONFINITE);
    }
    return true;
}

// Plan header of tile b (read by thread 0 ahead of its bulk copies).
__device__ __forceinline__ int4 tile_hdr(const TileArgs &ta, int64_t b)
{
    return *reinterpret_cast<const int4 *>(ta.plan_hdr + 4 * b);
}

// The persistent loop of a block over global tile indices g = blockIdx.x,
// blockIdx.x + gridDim.x, ... < n_total.  src.args(g) and src.targs(g) are
// the tile's step arguments and plan, src.tile(g) its index within its mesh;
// d sizes the shared memory (the largest over the meshes).  Stage k %
// kTileStages holds the block's k-th tile: its bulk copies start when the
// (k - kTileStages)-th tile is done, its halo gathers when the (k - 1)-th
// tile begins.
template <typename T, int SCHEME, typename Src>
__device__ __forceinline__ void tile_loop(const Src &src, int64_t n_total, const TileDims &d, unsigned char *smem_raw)
{
    constexpr int S = kTileStages;
    constexpr bool H2 = SCHEME == SWE_SCHEME_MUSCL;
    const int t = threadIdx.x;
    const int64_t G = gridDim.x, g0 = blockIdx.x;
    TileSmem<T> sm(smem_raw, d);
    if (t == 0) {
        for (int s = 0; s < S; s++) mbar_init(sm.bar(s));
        mbar_init_fence();
    }
    __syncthreads();
    if (t == 0)
        for (int s = 0; s < S; s++) {
            const int64_t g = g0 + s * G;
            if (g < n_total) {
                const int64_t b = src.tile(g);
                tile_issue<T>(src.args(g), src.targs(g), b, tile_hdr(src.targs(g), b), sm.stage(s), sm.bar(s));
            }
        }
    // the first tile's halo
    if (g0 < n_total) {
        const bool ok = mbar_wait(sm.bar(0), 0, kWaitPolls);
        if (!__syncthreads_and(ok)) {
            if (t == 0) atomicOr(&src.args(g0).sc->status, ST_TIMEOUT);
            return;
        }
        tile_gather<T, H2>(src.args(g0), sm.stage(0));
    }
    for (int64_t k = 0;; k++) {
        const int64_t g = g0 + k * G;
        if (g >= n_total) break;
        const int s = (int)(k % S);
        // this tile's halo has landed; the next tile's inputs are wanted for its halo gathers
        cp_async_wait_all();
        const int64_t gn = g + G;
        const bool ok = gn >= n_total || mbar_wait(sm.bar((int)((k + 1) % S)), (uint32_t)(((k + 1) / S) & 1), kWaitPolls);
        if (!__syncthreads_and(ok)) {
            if (t == 0) {
                atomicOr(&src.args(g).sc->status, ST_TIMEOUT);
                for (int64_t q = k + 1; q < k + S && g0 + q * G < n_total; q++)
                    mbar_wait(sm.bar((int)(q % S)), (uint32_t)((q / S) & 1), kWaitPolls);
            }
            cp_async_wait_all();
            return;
        }
        if (gn < n_total) tile_gather<T, H2>(src.args(gn), sm.stage((int)((k + 1) % S)));
        int4 hn = make_int4(0, 0, 0, 0);
        const int64_t gf = g + S * G;
        if (t == 0 && gf < n_total) hn = tile_hdr(src.targs(gf), src.tile(gf));   // ahead of its use below
        const StepArgs<T> &a = src.args(g);
        const int64_t b = src.tile(g);
        bool dry;
        const T dt = block_dt(a, &dry);
        CellOut<T> o;
        if (tile_compute<T, SCHEME>(a, b, sm, sm.stage(s), dt, o)) {
            step_epilogue<T>(a, dt, dry, o.smax, o.clip, o.bsum, b == 0);
        } else if (t == 0) {
            atomicOr(&a.sc->status, ST_TILE);
        }
        __syncthreads();                    // stage s and the working arrays are free again
        if (t == 0 && gf < n_total) {
            async_proxy_fence();
            tile_issue<T>(src.args(gf), src.targs(gf), src.tile(gf), hn, sm.stage(s), sm.bar(s));
        }
    }
    cp_async_wait_all();
}

}  // namespace swe_dev
