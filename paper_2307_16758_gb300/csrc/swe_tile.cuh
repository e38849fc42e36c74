// Device code of the one-pass tile step, shared by the single-mesh kernel
// and the batched ensemble kernel (both in swe_tile.cu).
//
// A tile is a run of B consecutive (Morton-ordered) cells, one per thread,
// worked in a slot space: slots 0 .. B-1 are the tile's cells, slots B ..
// B + n_halo - 1 its halo, the outside cells it reads (the far cells of its
// crossing edges, H1, then their other outside neighbours, H2); the host
// plan (swe_tiles.h) gives every neighbour's slot and the tile's edge list.
// The kernel is persistent: each block loops over tiles through a pipeline
// of shared-memory stages.  A stage receives a tile's contiguous per-cell
// arrays (scaled normals, state, bed, Manning n) and its plan by bulk
// asynchronous copies (cp.async.bulk on an mbarrier); the state, bed and
// normals of its halo cells are gathered into the same arrays by cp.async
// one tile ahead.  Every phase of a tile then reads shared memory only:
//   A  primitives of every slot;
//   B  MUSCL face values (least squares + Barth-Jespersen, the MUSCL idea of
//      Sec. 6.2.3) of the tile's cells and of the H1 cells;
//   C  one thread per listed edge: hydrostatic reconstruction and the
//      canonical-orientation Riemann flux (Sec. 6.2.1); the contribution to
//      each tile cell on the edge goes to shared memory (every edge inside
//      the tile is solved once);
//   D  each cell adds its three contributions in edge order (boundary edges
//      of the domain evaluated here), updates, clips, applies friction and
//      publishes its wave speed.
// The per-edge and per-cell arithmetic is the split kernels' device code, so
// a cell gets the same bits whichever path advances it.
#pragma once
#include "swe_async.cuh"
#include "swe_device.cuh"
#include "swe_split.cuh"

namespace swe_dev {

// Stages of the tile pipeline (tiles in flight per block).
constexpr int kTileStages = 2;
// Polls of an mbarrier before a block gives up on a copy (ST_TIMEOUT).
constexpr uint32_t kWaitPolls = 1u << 22;

// Room a block reserves: B cells, hmax halo cells (a multiple of 8), h1max
// H1 cells, wmax plan words (a multiple of 8).
struct TileDims {
    int B, hmax, h1max, wmax;
};

// One stage: a tile's inputs.  Slot-indexed arrays hold the tile's cells
// (bulk copies) followed by its halo cells (gathers).
template <typename T> struct TileStage {
    Vec2<T> *ln;         // [3 (B + hmax)] scaled outward normals
    T *h, *hu, *hv, *z;  // [B + hmax]
    T *nm;               // [B]            Manning n (friction only)
    int32_t *hdr;        // [8]            plan header
    int32_t *words;      // [wmax]         plan words

    static __host__ __device__ size_t bytes(const TileDims &d)
    {
        const size_t S = (size_t)d.B + d.hmax;
        return 3 * S * sizeof(Vec2<T>) + 4 * S * sizeof(T) + (size_t)d.B * sizeof(T) + 32 + (size_t)d.wmax * 4;
    }

    __device__ void place(unsigned char *base, const TileDims &d)
    {
        const int S = d.B + d.hmax;
        ln = reinterpret_cast<Vec2<T> *>(base);
        h = reinterpret_cast<T *>(ln + 3 * S);
        hu = h + S; hv = hu + S; z = hv + S; nm = z + S;
        hdr = reinterpret_cast<int32_t *>(nm + d.B);
        words = hdr + 8;
    }
};

// Shared memory of a block: the stages and their mbarriers, then the
// working arrays of the tile being computed (slot-major per-face arrays:
// [slot * 3 + k]).  Addresses are recomputed from the base on use.
template <typename T> struct TileSmem {
    unsigned char *base;
    TileDims d;
    Vec4<T> *P;          // [B + hmax]       (eta, u, v, h) of every slot
    T *Fe, *Fu, *Fv;     // [B + h1max][3]   face values (eta, u, v) at the edge midpoints
    T *C0, *C1, *C2;     // [B][3]           edge contributions

    static __host__ __device__ size_t bytes(const TileDims &d)
    {
        return kTileStages * TileStage<T>::bytes(d) + 64 + ((size_t)d.B + d.hmax) * sizeof(Vec4<T>) +
               (3 * 3 * ((size_t)d.B + d.h1max) + 3 * 3 * (size_t)d.B) * sizeof(T);
    }

    __device__ TileSmem(unsigned char *base_, const TileDims &d_) : base(base_), d(d_)
    {
        unsigned char *p = base + kTileStages * TileStage<T>::bytes(d) + 64;
        P = reinterpret_cast<Vec4<T> *>(p);
        Fe = reinterpret_cast<T *>(P + d.B + d.hmax);
        Fu = Fe + 3 * (d.B + d.h1max); Fv = Fu + 3 * (d.B + d.h1max);
        C0 = Fv + 3 * (d.B + d.h1max); C1 = C0 + 3 * d.B; C2 = C1 + 3 * d.B;
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

// Plan header of tile b: offset, halo cells, H1 cells, edges, crossing edges,
// plan words (read by thread 0 ahead of the tile's bulk copies).
struct TileHdr {
    int off, n_halo, n_h1, n_edges, n_cross, n_words;
};

__device__ __forceinline__ TileHdr tile_hdr(const TileArgs &ta, int64_t b)
{
    const int4 x = *reinterpret_cast<const int4 *>(ta.plan_hdr + 8 * b);
    const int4 y = *reinterpret_cast<const int4 *>(ta.plan_hdr + 8 * b + 4);
    return TileHdr{x.x, x.y, x.z, x.w, y.x, y.y};
}

// Thread 0: start the bulk copies of tile b (of the mesh of `a`, plan `ta`)
// into a stage.  The per-cell arrays are allocated to a whole number of
// tiles, so a full tile is copied even at the end of the mesh.
template <typename T>
__device__ __forceinline__ void tile_issue(const StepArgs<T> &a, const TileArgs &ta, int64_t b, const TileHdr &hd,
                                           const TileStage<T> &st, uint64_t *bar)
{
    const int B = blockDim.x;
    const int64_t s0 = b * B;
    const uint32_t fb = (uint32_t)(B * sizeof(T)), lb = 3 * (uint32_t)B * (uint32_t)sizeof(Vec2<T>);
    const bool fric = a.m.nman != nullptr;
    mbar_arrive_expect(bar, lb + (fric ? 5 : 4) * fb + 32 + 4 * (uint32_t)hd.n_words);
    bulk_load(st.ln, a.m.ln + 3 * s0, lb, bar);
    bulk_load(st.h, a.h + s0, fb, bar);
    bulk_load(st.hu, a.hu + s0, fb, bar);
    bulk_load(st.hv, a.hv + s0, fb, bar);
    bulk_load(st.z, a.m.z + s0, fb, bar);
    if (fric) bulk_load(st.nm, a.m.nman + s0, fb, bar);
    bulk_load(st.hdr, ta.plan_hdr + 8 * b, 32, bar);
    bulk_load(st.words, ta.plan_words + hd.off, 4 * (uint32_t)hd.n_words, bar);
}

// All threads: gather the state, bed and normals of the stage's halo cells
// into their slots (H1 only for first-order HLLC) with cp.async, one commit
// group per thread.
template <typename T, bool H2>
__device__ __forceinline__ void tile_gather(const StepArgs<T> &a, const TileStage<T> &st)
{
    const int B = blockDim.x, nh = H2 ? st.hdr[1] : st.hdr[2];
    for (int q = threadIdx.x; q < nh; q += B) {
        const int64_t id = st.words[q];
        const int s = B + q;
        cp_async<sizeof(T)>(st.h + s, a.h + id);
        cp_async<sizeof(T)>(st.hu + s, a.hu + id);
        cp_async<sizeof(T)>(st.hv + s, a.hv + id);
        cp_async<sizeof(T)>(st.z + s, a.m.z + id);
#pragma unroll
        for (int k = 0; k < 3; k++) cp_async<sizeof(Vec2<T>)>(st.ln + 3 * s + k, a.m.ln + 3 * id + k);
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


// MUSCL face values of slot q (a tile cell or an H1 cell) from the
// primitives and normals of its neighbours' slots (lw: its three local
// words).  The arithmetic of muscl_cell_faces, operand for operand.
template <typename T>
__device__ __forceinline__ void slot_faces(const TileSmem<T> &sm, const TileStage<T> &st, int q, const int lw[3],
                                           T h_eps, T fe[3], T fu[3], T fv[3])
{
    const Vec4<T> pi = sm.P[q];
    if (pi.w <= h_eps) {
        // a dry cell: zero gradient and zero velocity, the centre values
#pragma unroll
        for (int k = 0; k < 3; k++) { fe[k] = pi.x; fu[k] = pi.y; fv[k] = pi.z; }
        return;
    }
    Vec2<T> ln[3], dd[3];
    T qi[3] = {pi.x, pi.y, pi.z};
    T qn[3][3], ox[3], oy[3];
    bool has[3];
    bool ok = true;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) ln[k] = st.ln[3 * q + k];
    midpoint_offsets(ln, ox, oy);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        has[k] = lw[k] >= 0;
        if (has[k]) {
            const int sj = lw[k] >> 3, kj = (lw[k] >> 1) & 3;
            const int k1 = kj == 2 ? 0 : kj + 1, k2 = kj == 0 ? 2 : kj - 1;
            const Vec4<T> pj = sm.P[sj];
            ok = ok && pj.w > h_eps;
            qn[k][0] = pj.x; qn[k][1] = pj.y; qn[k][2] = pj.z;
            dd[k] = centroid_offset_from(ox[k], oy[k], st.ln[3 * sj + k1], st.ln[3 * sj + k2]);
            cnt++;
        } else {
            qn[k][0] = qi[0]; qn[k][1] = qi[1]; qn[k][2] = qi[2];
            dd[k].x = T(0); dd[k].y = T(0);
        }
    }
    Vec4<T> f[3];
    muscl_faces<T, 3>(qi, st.z[q], ok, cnt, qn, has, ox, oy, dd, f);
#pragma unroll
    for (int k = 0; k < 3; k++) { fe[k] = f[k].x; fu[k] = f[k].y; fv[k] = f[k].z; }
}

// One tile (index b, cells s0 .. s0 + nc - 1 of the mesh of `a`) whose inputs
// and halo are in stage `st`.  SCHEME: SWE_SCHEME_MUSCL or SWE_SCHEME_HLLC.
// Returns the wave speed, clipped mass and boundary mass of the thread's
// cell in o; false (block uniform) if the tile's plan outgrows the room.
template <typename T, int SCHEME>
__device__ __forceinline__ bool tile_compute(const StepArgs<T> &a, int64_t b, const TileSmem<T> &sm,
                                             const TileStage<T> &st, T dt, CellOut<T> &o)
{
    constexpr bool MUSCL = SCHEME == SWE_SCHEME_MUSCL;
    const int B = blockDim.x, t = threadIdx.x;
    const int64_t s0 = b * B;
    const int nc = (int)(a.m.n - s0 < (int64_t)B ? a.m.n - s0 : (int64_t)B);
    const bool valid = t < nc;
    const T h_eps = a.h_eps;
    const int n_halo = st.hdr[1], n_h1 = st.hdr[2], n_edges = st.hdr[3];
    if (n_halo > sm.d.hmax || n_h1 > sm.d.h1max || st.hdr[5] > sm.d.wmax) return false;   // uniform over the block
    const uint32_t *edges = reinterpret_cast<const uint32_t *>(st.words + n_halo);
    const int16_t *lwords = reinterpret_cast<const int16_t *>(st.words + n_halo + n_edges);

    // ---- A: primitives of every slot ----
    const int n_slots = B + (MUSCL ? n_halo : n_h1);
    for (int q = t; q < n_slots; q += B)
        if (q < nc || q >= B) sm.P[q] = prim4(st.h[q], st.hu[q], st.hv[q], st.z[q], h_eps);
    __syncthreads();

    // ---- B: face values of the tile's cells and of the H1 cells ----
    for (int q = t; q < B + n_h1; q += B) {
        if (q >= nc && q < B) continue;
        T fe[3], fu[3], fv[3];
        if (MUSCL) {
            const int lw[3] = {lwords[3 * q], lwords[3 * q + 1], lwords[3 * q + 2]};
            slot_faces(sm, st, q, lw, h_eps, fe, fu, fv);
        } else {
            const Vec4<T> pi = sm.P[q];
#pragma unroll
            for (int k = 0; k < 3; k++) { fe[k] = pi.x; fu[k] = pi.y; fv[k] = pi.z; }
        }
#pragma unroll
        for (int k = 0; k < 3; k++) { sm.Fe[3 * q + k] = fe[k]; sm.Fu[3 * q + k] = fu[k]; sm.Fv[3 * q + k] = fv[k]; }
    }
    __syncthreads();

    // ---- C: one thread per listed edge, crossing edges first ----
    for (int e = t; e < n_edges; e += B) {
        const uint32_t r = edges[e];
        const int si = (int)(r & 2047u), ki = (int)((r >> 11) & 3u), sj = (int)((r >> 13) & 2047u);
        const int kj = (int)((r >> 24) & 3u);
        const bool own = (r >> 26) & 1u, cross = (r >> 27) & 1u;
        Side<T> Si, Sj;
        Si.ef = sm.Fe[3 * si + ki]; Si.uf = sm.Fu[3 * si + ki]; Si.vf = sm.Fv[3 * si + ki];
        Si.z = st.z[si]; Si.zc = Si.z; Si.hc = st.h[si];
        Sj.ef = sm.Fe[3 * sj + kj]; Sj.uf = sm.Fu[3 * sj + kj]; Sj.vf = sm.Fv[3 * sj + kj];
        Sj.z = st.z[sj]; Sj.zc = Sj.z; Sj.hc = st.h[sj];
        const Vec2<T> l = st.ln[3 * si + ki];
        const Vec4<T> none{};
        Contrib<T> ci, cj;
        interior_edge<T, MUSCL ? SWE_SCHEME_MUSCL : SWE_SCHEME_HLLC>(a, dt, Si, Sj, own, l.x, l.y, T(0), none, none,
                                                                    ci, cross ? nullptr : &cj);
        sm.C0[3 * si + ki] = ci.c0; sm.C1[3 * si + ki] = ci.c1; sm.C2[3 * si + ki] = ci.c2;
        if (!cross) { sm.C0[3 * sj + kj] = cj.c0; sm.C1[3 * sj + kj] = cj.c1; sm.C2[3 * sj + kj] = cj.c2; }
    }
    __syncthreads();

    // ---- D: sums in edge order, update ----
    o.smax = T(0); o.clip = T(0); o.bsum = T(0);
    if (valid) {
        const int64_t i = s0 + t;
        const T hi = st.h[t], hui = st.hu[t], hvi = st.hv[t], zi = st.z[t];
        Vec2<T> ln[3];
        T R0 = T(0), R1 = T(0), R2 = T(0), bs = T(0);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            ln[k] = st.ln[3 * t + k];
            const int w = lwords[3 * t + k];
            Contrib<T> c;
            if (w >= 0) {
                c.c0 = sm.C0[3 * t + k]; c.c1 = sm.C1[3 * t + k]; c.c2 = sm.C2[3 * t + k];
            } else {
                Side<T> sd;
                sd.ef = sm.Fe[3 * t + k]; sd.uf = sm.Fu[3 * t + k]; sd.vf = sm.Fv[3 * t + k];
                sd.z = zi; sd.zc = zi; sd.hc = hi;
                c = boundary_edge<T>(a, sd, -1 - w, ln[k].x, ln[k].y, bs);
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
            if (t == 0) {
                atomicOr(&src.args(g0).sc->status, ST_TIMEOUT);
                for (int s = 1; s < S && g0 + s * G < n_total; s++) mbar_wait(sm.bar(s), 0, kWaitPolls);
            }
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
            return;
        }
        if (gn < n_total) tile_gather<T, H2>(src.args(gn), sm.stage((int)((k + 1) % S)));
        TileHdr hn{};
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
