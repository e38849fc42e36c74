// C ABI of the shallow-water library: handles, device memory, launches.
// Every numerical step runs in the CUDA kernels of swe_kernels.cu; this file
// only validates arguments, moves data and orders the launches on a stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "swe_dev.h"
#include "swe_ensemble.h"
#include "swe_mesh.h"
#include "swe_partition.h"
#include "swe_tiles.h"
#include "../../include/swe_tile_plan.h"

int swe_mesh_build_host(const double *xy, int64_t n_nodes, const int32_t *tri, int64_t n,
                        const int32_t *bnd, const int32_t *bnd_tag, int64_t n_bnd,
                        const int32_t *cut, int64_t n_cut, int reorder, swe_mesh **out);

static thread_local std::string g_err;
void swe_set_error(const std::string &msg) { g_err = msg; }

namespace {
std::mutex g_alloc_mu;
swe_alloc_fn g_alloc = nullptr;
swe_free_fn g_free = nullptr;
void *g_ctx = nullptr;
// Blocks that came from an installed allocator, with the free function and
// context to return them to (the pair may have been replaced since).
std::unordered_map<void *, std::pair<swe_free_fn, void *>> g_owner;
}  // namespace

// Device memory through the allocator installed by swe_set_allocator, else
// cudaMalloc (also used by the arithmetic-peak probe).
void *dev_alloc(size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    swe_alloc_fn alloc;
    swe_free_fn free_fn;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        alloc = g_alloc; free_fn = g_free; ctx = g_ctx;
    }
    if (alloc) {
        void *p = alloc(bytes, (void *)s, ctx);
        if (p) {
            std::lock_guard<std::mutex> lk(g_alloc_mu);
            g_owner[p] = {free_fn, ctx};
        }
        return p;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    return p;
}

// Returns a block to whichever allocator gave it out.
void dev_free(void *p, cudaStream_t s)
{
    if (!p) return;
    swe_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        auto it = g_owner.find(p);
        if (it != g_owner.end()) {
            free_fn = it->second.first; ctx = it->second.second;
            g_owner.erase(it);
        }
    }
    if (free_fn) free_fn(p, (void *)s, ctx);
    else cudaFree(p);
}

namespace {

// Message for a non-zero return of swe_build_tile_plan.
std::string tile_plan_error(int rc)
{
    if (rc == -1) return "the tile size must be a power of two within 32 .. 1024";
    if (rc == -2) return "a tile and its halo exceed the plan's 2047 slots: renumber the mesh (Morton or RCM) or take a smaller tile";
    return "the tile plan exceeds 2^31 words";
}

#define CK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            swe_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));    \
            return SWE_ERR_CUDA;                                                  \
        }                                                                         \
    } while (0)

struct Alloc {
    std::vector<std::pair<void *, size_t>> blocks;
    int64_t bytes = 0;
};

// Largest tile of the tile step; per-cell arrays are allocated to a multiple
// of it so that every tile, the last one included, is copied whole.
constexpr int64_t kTilePad = 1024;

template <typename T> struct StateT {
    swe_params p{};
    int64_t n = 0;
    double r_min = 0.0;
    cudaStream_t stream = nullptr;
    Alloc mem;
    // mesh on the device
    int32_t *nbr = nullptr, *perm = nullptr;
    Vec2<T> *ln = nullptr, *dd = nullptr;
    T *z = nullptr, *nman = nullptr;
    double *area = nullptr;
    // state: ping-pong buffers plus the Heun stage buffer
    T *h[3] = {}, *hu[3] = {}, *hv[3] = {};
    int cur = 0;
    // scratch: face values / centre values and upwind means
    Vec4<T> *F = nullptr, *U = nullptr;
    DevScalars *sc = nullptr;
    double *mass_part = nullptr, *mass_out = nullptr, *staging = nullptr;
    int n_part = 0;
    double *dtbuf = nullptr;
    int dtbuf_len = 0;
    double *dt_hist = nullptr;
    // tracing: CUDA events around every launch while profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> ev_used;
    // one-pass tile step
    bool fused = false;
    TileArgs ta{};
    // boundary-first schedule (swe_set_partition)
    bool sched = false;
    int32_t *d_bnd = nullptr, *d_int = nullptr, *d_recv = nullptr;
    int64_t n_bnd = 0, n_int = 0, n_recv = 0;
    std::vector<int64_t> recv_ptr;
    T *halo_buf = nullptr;
    cudaStream_t halo_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // CUDA graphs of kGraphSteps CFL steps, keyed by (steps launched mod 6, cfl):
    // the launch pattern (ping-pong buffer, CFL slot ring) repeats every 6 steps
    static constexpr int kGraphSteps = 24;
    std::map<std::pair<int, double>, cudaGraphExec_t> graphs;
    cudaStream_t cap_stream = nullptr;
    bool use_graphs = true;
    // Threads per block of the split prep kernels, apart from the flux
    // kernel's: prep is bound by memory latency and runs best in short blocks
    // (FP32 MUSCL on a 13M-cell river: 128 threads 0.227 ms, 256 0.234, 512
    // 0.248); the autotuner may pick another.
    int prep_bl = 128;
    int64_t k = 0;            // steps launched (selects the smax slots)
    bool smax_valid = false;
    T qlen[SWE_MAX_GROUPS] = {}, level[SWE_MAX_GROUPS] = {};

    // Device array of `count` elements, zero-filled (on the state's stream).
    template <typename P> P *alloc(size_t count)
    {
        size_t b = count * sizeof(P);
        void *ptr = dev_alloc(b, stream);
        if (ptr) {
            mem.blocks.push_back({ptr, b});
            mem.bytes += (int64_t)((b + 255) & ~size_t(255));
            if (cudaMemsetAsync(ptr, 0, b, stream) != cudaSuccess) return nullptr;
        }
        return (P *)ptr;
    }
    ~StateT()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (halo_stream) { cudaStreamSynchronize(halo_stream); cudaStreamDestroy(halo_stream); }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (auto &e : ev_used) { cudaEventDestroy(std::get<1>(e)); cudaEventDestroy(std::get<2>(e)); }
        for (auto e : ev_pool) cudaEventDestroy(e);
        for (auto &b : mem.blocks) dev_free(b.first, stream);
    }

    cudaEvent_t take_event()
    {
        if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    // Launch f (returning cudaError_t), bracketed by events when profiling.
    template <typename F> cudaError_t traced(int kind, F &&f)
    {
        if (!prof) return f();
        cudaEvent_t a = take_event(), b = take_event();
        cudaEventRecord(a, stream);
        cudaError_t e = f();
        cudaEventRecord(b, stream);
        ev_used.emplace_back(kind, a, b);
        return e;
    }

    void release(void *ptr)
    {
        if (!ptr) return;
        for (auto it = mem.blocks.begin(); it != mem.blocks.end(); ++it)
            if (it->first == ptr) {
                dev_free(it->first, stream);
                mem.bytes -= (int64_t)((it->second + 255) & ~size_t(255));
                mem.blocks.erase(it);
                return;
            }
    }

    void clear_graphs()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
    }

    // Tile steps need a scheme and options that the tile kernel implements.
    bool tile_capable() const
    {
        return (p.scheme == SWE_SCHEME_MUSCL || p.scheme == SWE_SCHEME_HLLC) && p.hr_order == 1;
    }

    // Select the split kernels or the one-pass tile step with `block` threads
    // (cells per tile; the tile plan is built from the mesh); allocates what
    // that path needs.
    int configure(bool want_fused, int block, const swe_mesh *m)
    {
        if (want_fused && sched) {
            swe_set_error("the boundary-first schedule runs the split kernels (clear the partition first)");
            return SWE_ERR_ARG;
        }
        if (want_fused && !tile_capable()) {
            swe_set_error("the tile step runs LSQ MUSCL or first-order HLLC with the first-order hydrostatic "
                          "reconstruction (WAF, the paper's MUSCL and hr_order 2 run the split kernels)");
            return SWE_ERR_ARG;
        }
        const int lim = want_fused ? tile_max_threads<T>(p.scheme) : split_max_threads<T>(p.scheme, p.hr_order == 2);
        if (lim <= 0) { swe_set_error("cannot query the kernels (no usable GPU?)"); return SWE_ERR_CUDA; }
        if (block <= 0 || block % 32 || block > lim) {
            swe_set_error("block of " + std::to_string(block) + " threads is not a multiple of 32 within the kernel's limit of " +
                          std::to_string(lim));
            return SWE_ERR_ARG;
        }
        CK(cudaStreamSynchronize(stream));
        clear_graphs();
        if (!want_fused) {
            if ((p.scheme == SWE_SCHEME_MUSCL || p.scheme == SWE_SCHEME_MUSCL_EDGE) && !F) F = alloc<Vec4<T>>(3 * n);
            if (p.scheme == SWE_SCHEME_WAF && !F) { F = alloc<Vec4<T>>(n); U = alloc<Vec4<T>>(3 * n); }
            if (p.scheme != SWE_SCHEME_HLLC && (!F || (p.scheme == SWE_SCHEME_WAF && !U))) {
                swe_set_error("device allocation failed");
                return SWE_ERR_NOMEM;
            }
        }
        if (want_fused) {
            if (!m || m->n != n) { swe_set_error("the tile step needs the state's mesh"); return SWE_ERR_ARG; }
            TilePlan tp;
            if (const int rc = swe_build_tile_plan(*m, block, tp)) { swe_set_error(tile_plan_error(rc)); return SWE_ERR_ARG; }
            TileArgs t{};
            t.tile = block;
            t.n_tiles = tp.n_tiles;
            t.hmax = (std::max(tp.hmax, 1) + 7) & ~7;          // stage alignment (see TileStage)
            t.h1max = std::max(tp.h1max, 1);
            t.wmax = (std::max(tp.wmax, 8) + 7) & ~7;
            const size_t smem = tile_smem_bytes<T>(t);
            if (smem > 227 * 1024) {
                swe_set_error("tile needs more shared memory than a block has");
                return SWE_ERR_ARG;
            }
            CK(tile_prepare<T>(p.scheme, smem));
            t.grid = tile_grid<T>(p.scheme, block, smem);
            if (t.grid <= 0) { swe_set_error("the tile kernel cannot be resident with this tile size"); return SWE_ERR_ARG; }
            release((void *)ta.plan_hdr);
            release((void *)ta.plan_words);
            int32_t *hdr = alloc<int32_t>(tp.hdr.size());
            int32_t *words = alloc<int32_t>(tp.words.size());
            if (!hdr || !words) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
            CK(cudaMemcpy(hdr, tp.hdr.data(), sizeof(int32_t) * tp.hdr.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(words, tp.words.data(), sizeof(int32_t) * tp.words.size(), cudaMemcpyHostToDevice));
            t.plan_hdr = hdr;
            t.plan_words = words;
            ta = t;
            p.kernel = SWE_KERNEL_FUSED;
        } else {
            p.kernel = SWE_KERNEL_SPLIT;
        }
        fused = want_fused;
        p.block = block;
        return SWE_OK;
    }

    // Copy of the evolving data (state, scalars, dt history) for trial runs.
    struct Snapshot {
        T *h = nullptr, *hu = nullptr, *hv = nullptr;
        DevScalars *sc = nullptr;
        double *hist = nullptr;
        int64_t k = 0;
        int cur = 0;
        bool smax_valid = false;
    };

    int snapshot(Snapshot &sn)
    {
        if (!sn.h) {
            sn.h = alloc<T>(n); sn.hu = alloc<T>(n); sn.hv = alloc<T>(n);
            sn.sc = alloc<DevScalars>(1); sn.hist = alloc<double>(SWE_DT_HISTORY);
            if (!sn.h || !sn.hu || !sn.hv || !sn.sc || !sn.hist) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
        }
        CK(cudaMemcpyAsync(sn.h, h[cur], sizeof(T) * n, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(sn.hu, hu[cur], sizeof(T) * n, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(sn.hv, hv[cur], sizeof(T) * n, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(sn.sc, sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(sn.hist, dt_hist, sizeof(double) * SWE_DT_HISTORY, cudaMemcpyDeviceToDevice, stream));
        sn.k = k; sn.cur = cur; sn.smax_valid = smax_valid;
        return SWE_OK;
    }

    int restore(const Snapshot &sn)
    {
        k = sn.k; cur = sn.cur; smax_valid = sn.smax_valid;
        CK(cudaMemcpyAsync(h[cur], sn.h, sizeof(T) * n, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(hu[cur], sn.hu, sizeof(T) * n, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(hv[cur], sn.hv, sizeof(T) * n, cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(sc, sn.sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(dt_hist, sn.hist, sizeof(double) * SWE_DT_HISTORY, cudaMemcpyDeviceToDevice, stream));
        return SWE_OK;
    }

    void drop(Snapshot &sn)
    {
        cudaStreamSynchronize(stream);
        release(sn.h); release(sn.hu); release(sn.hv); release(sn.sc); release(sn.hist);
        sn = Snapshot{};
    }

    // Step arguments for phase p = (steps taken) mod 6 of the launch pattern.
    StepArgs<T> args_for_phase(int ph, double cfl)
    {
        const int64_t k0 = k;
        k = ph;
        StepArgs<T> a = args(ph & 1, (ph & 1) ^ 1);
        k = k0;
        a.cfl_rmin = cfl_factor(cfl);
        return a;
    }

    DevMesh<T> dmesh() const
    {
        DevMesh<T> m;
        m.n = n; m.nbr = nbr; m.ln = ln; m.dd = dd; m.z = z; m.nman = nman; m.area = area;
        return m;
    }

    // Numerator of the CFL time step: cfl * r_min in the global form (the
    // published speed is max s_i), cfl in the local form (max s_i / r_i).
    T cfl_factor(double cfl) const { return (T)(p.cfl_mode == SWE_CFL_LOCAL ? cfl : cfl * r_min); }

    StepArgs<T> args(int in, int out) const
    {
        StepArgs<T> a{};
        a.m = dmesh();
        a.h = h[in]; a.hu = hu[in]; a.hv = hv[in];
        a.ho = h[out]; a.huo = hu[out]; a.hvo = hv[out];
        a.F = F; a.U = U; a.sc = sc;
        a.dtv = nullptr;
        a.dt_hist = dt_hist;
        a.slot_cur = (int)(k % 3); a.slot_next = (int)((k + 1) % 3); a.slot_clear = (int)((k + 2) % 3);
        a.mode = MODE_EULER;
        a.cfl_local = p.cfl_mode == SWE_CFL_LOCAL;
        a.g = (T)p.g; a.h_eps = (T)p.h_eps; a.r_eps = (T)p.r_eps;
        a.beta = (T)p.muscl_beta;
        a.hr2 = p.hr_order == 2;
        a.waf_surface = p.waf_ratio == SWE_WAF_RATIO_SURFACE;
        a.waf_limiter = p.waf_limiter;
        for (int q = 0; q < SWE_MAX_GROUPS; q++) { a.qlen[q] = qlen[q]; a.level[q] = level[q]; }
        return a;
    }

    int block() const { return fused ? ta.tile : (p.block > 0 ? p.block : 256); }

    cudaError_t launch_step_kernels(const StepArgs<T> &a, int bl)
    {
        if (fused) return traced(SWE_K_FUSED, [&] { return launch_tile<T>(p.scheme, a, ta, stream); });
        if (p.scheme != SWE_SCHEME_HLLC) {
            cudaError_t e = traced(SWE_K_PREP, [&] { return launch_prep<T>(p.scheme, a, F, U, prep_bl, stream); });
            if (e != cudaSuccess) return e;
        }
        if (!sched) return traced(SWE_K_FLUX, [&] { return launch_flux<T>(p.scheme, a, bl, stream); });
        // boundary-first schedule (Sec. 6.4): first the cells that other parts
        // hold in their halos, then, while their new state is packed into the
        // halo buffers on a second stream, the interior
        StepArgs<T> b = a;
        b.cells = d_bnd; b.n_list = (int)n_bnd; b.no_advance = n_int > 0;
        cudaError_t e = traced(SWE_K_FLUX, [&] { return launch_flux_list<T>(p.scheme, b, bl, stream); });
        if (e == cudaSuccess) e = cudaEventRecord(ev_fork, stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(halo_stream, ev_fork, 0);
        if (e == cudaSuccess) e = launch_pack_halo<T>(n_recv, d_recv, a.ho, a.huo, a.hvo, halo_buf, halo_stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev_join, halo_stream);
        StepArgs<T> c = a;
        c.cells = d_int; c.n_list = (int)n_int; c.no_advance = 0;
        if (e == cudaSuccess) e = traced(SWE_K_FLUX, [&] { return launch_flux_list<T>(p.scheme, c, bl, stream); });
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_join, 0);
        return e;
    }

    // Boundary-first schedule over a partition of the mesh (NULL: plain).
    int set_partition(const swe_partition *part)
    {
        CK(cudaStreamSynchronize(stream));
        clear_graphs();
        for (void *q : {(void *)d_bnd, (void *)d_int, (void *)d_recv, (void *)halo_buf}) release(q);
        d_bnd = d_int = d_recv = nullptr;
        halo_buf = nullptr;
        sched = false;
        recv_ptr.clear();
        if (!part) return SWE_OK;
        if (part->n != n) { swe_set_error("swe_set_partition: the partition is of another mesh"); return SWE_ERR_ARG; }
        if (fused || p.time_scheme != SWE_EULER) {
            swe_set_error("swe_set_partition: the boundary-first schedule runs the split kernels with Euler steps");
            return SWE_ERR_ARG;
        }
        n_bnd = (int64_t)part->boundary_all.size();
        n_int = (int64_t)part->interior_all.size();
        n_recv = (int64_t)part->recv_cell.size();
        d_bnd = alloc<int32_t>(std::max<int64_t>(n_bnd, 1));
        d_int = alloc<int32_t>(std::max<int64_t>(n_int, 1));
        d_recv = alloc<int32_t>(std::max<int64_t>(n_recv, 1));
        halo_buf = alloc<T>(std::max<int64_t>(3 * n_recv, 1));
        if (!d_bnd || !d_int || !d_recv || !halo_buf) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
        CK(cudaMemcpy(d_bnd, part->boundary_all.data(), sizeof(int32_t) * n_bnd, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_int, part->interior_all.data(), sizeof(int32_t) * n_int, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_recv, part->recv_cell.data(), sizeof(int32_t) * n_recv, cudaMemcpyHostToDevice));
        CK(cudaMemset(halo_buf, 0, sizeof(T) * std::max<int64_t>(3 * n_recv, 1)));
        if (!halo_stream) CK(cudaStreamCreateWithFlags(&halo_stream, cudaStreamNonBlocking));
        if (!ev_fork) CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        if (!ev_join) CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        recv_ptr = part->recv_ptr;
        sched = true;
        return SWE_OK;
    }

    // The packed halo of part q after the last step, as FP64 host arrays.
    int halo_get(int q, double *ho, double *huo, double *hvo)
    {
        if (!sched || q < 0 || q + 1 >= (int)recv_ptr.size()) { swe_set_error("swe_halo_get: no such part"); return SWE_ERR_ARG; }
        CK(cudaStreamSynchronize(stream));
        const int64_t a = recv_ptr[q], len = recv_ptr[q + 1] - a;
        std::vector<T> tmp((size_t)std::max<int64_t>(len, 1));
        double *dst[3] = {ho, huo, hvo};
        for (int f = 0; f < 3; f++) {
            if (!dst[f] || len == 0) continue;
            CK(cudaMemcpy(tmp.data(), halo_buf + f * n_recv + a, sizeof(T) * len, cudaMemcpyDeviceToHost));
            for (int64_t s = 0; s < len; s++) dst[f][s] = (double)tmp[s];
        }
        return SWE_OK;
    }

    int init_smax()
    {
        CK(cudaMemsetAsync(sc->smax, 0, sizeof(sc->smax), stream));
        StepArgs<T> a = args(cur, cur);
        CK(traced(SWE_K_SMAX, [&] { return launch_smax<T>(a, (int)(k % 3), block(), stream); }));
        smax_valid = true;
        return SWE_OK;
    }

    // One explicit step (Euler, or Heun's two stages and the average).
    int one_step(double cfl, const double *dt_dev)
    {
        const int nxt = cur ^ 1;
        StepArgs<T> a = args(cur, nxt);
        a.cfl_rmin = cfl_factor(cfl);
        a.dtv = dt_dev;
        const int bl = block();
        if (p.time_scheme == SWE_EULER) {
            CK(launch_step_kernels(a, bl));
        } else {
            StepArgs<T> s1 = args(cur, 2);
            s1.cfl_rmin = a.cfl_rmin; s1.dtv = dt_dev; s1.mode = MODE_STAGE;
            CK(launch_step_kernels(s1, bl));
            StepArgs<T> s2 = args(2, nxt);
            s2.cfl_rmin = a.cfl_rmin; s2.dtv = dt_dev; s2.mode = MODE_STAGE;
            CK(launch_step_kernels(s2, bl));
            StepArgs<T> av = args(nxt, nxt);
            av.cfl_rmin = a.cfl_rmin; av.dtv = dt_dev;
            CK(traced(SWE_K_HEUN_AVG, [&] { return launch_heun_avg<T>(av, h[cur], hu[cur], hv[cur], bl, stream); }));
        }
        cur = nxt;
        k++;
        return SWE_OK;
    }

    // kGraphSteps CFL steps through a cached CUDA graph (captured on a private
    // stream on first use, launched on the state's stream).
    int graph_steps(double cfl)
    {
        const std::pair<int, double> key((int)(k % 6), cfl);
        auto it = graphs.find(key);
        if (it == graphs.end()) {
            if (!cap_stream) CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
            const cudaStream_t user = stream;
            const int64_t k0 = k;
            const int cur0 = cur;
            stream = cap_stream;
            cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
            int rc = SWE_OK;
            for (int q = 0; q < kGraphSteps && rc == SWE_OK && e == cudaSuccess; q++) rc = one_step(cfl, nullptr);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cap_stream, &g);
            stream = user;
            k = k0;
            cur = cur0;
            if (e != cudaSuccess || e2 != cudaSuccess || rc != SWE_OK) {
                if (g) cudaGraphDestroy(g);
                swe_set_error("CUDA graph capture failed");
                return rc != SWE_OK ? rc : SWE_ERR_CUDA;
            }
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            CK(e);
            it = graphs.emplace(key, ex).first;
        }
        CK(cudaGraphLaunch(it->second, stream));
        k += kGraphSteps;
        cur = (cur + kGraphSteps) & 1;
        return SWE_OK;
    }

    int read_scalars(DevScalars &out)
    {
        CK(cudaMemcpyAsync(&out, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        return SWE_OK;
    }

    int status()
    {
        DevScalars s;
        int rc = read_scalars(s);
        if (rc) return rc;
        if (s.status & ST_NONFINITE) { swe_set_error("a non-finite depth or discharge was produced"); return SWE_ERR_NONFINITE; }
        if (s.status & ST_DRY) { swe_set_error("CFL rule: no wet cell"); return SWE_ERR_DRY; }
        if (s.status & ST_TILE) { swe_set_error("a tile's edge list exceeded its plan (internal error)"); return SWE_ERR_CUDA; }
        if (s.status & ST_TIMEOUT) { swe_set_error("a bulk copy into shared memory did not complete in time"); return SWE_ERR_TIMEOUT; }
        return SWE_OK;
    }
};

// ---- autotuner --------------------------------------------------------------

struct Candidate { bool fused; int block; };

template <typename T> std::vector<Candidate> candidates(const StateT<T> &S, const swe_mesh *m)
{
    std::vector<Candidate> c;
    const int ls = split_max_threads<T>(S.p.scheme, S.p.hr_order == 2);
    for (int b : {128, 256, 512})
        if (b <= ls) c.push_back({false, b});
    if (S.tile_capable() && m && !S.sched) {
        const int lf = tile_max_threads<T>(S.p.scheme);
        for (int b : {128, 256, 512})
            if (b <= lf) c.push_back({true, b});
    }
    return c;
}

// Time `trials` CFL steps of every candidate kernel configuration on copies
// of the current state, keep the fastest; the state is left as it was.
template <typename T>
int autotune(StateT<T> &S, const swe_mesh *m, int trials, double cfl, int &best_kernel, int &best_block,
             double &best_ms)
{
    if (trials < 1 || !(cfl > 0)) { swe_set_error("swe_autotune: bad argument"); return SWE_ERR_ARG; }
    if (m && m->n != S.n) { swe_set_error("swe_autotune: mesh does not match the state"); return SWE_ERR_ARG; }
    if (!S.smax_valid) { int rc = S.init_smax(); if (rc) return rc; }
    typename StateT<T>::Snapshot sn;
    int rc = S.snapshot(sn);
    if (rc) return rc;
    const bool fused0 = S.fused;
    const int block0 = S.block();
    best_ms = 1e30;
    Candidate best{fused0, block0};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (const Candidate &c : candidates(S, m)) {
        if (S.configure(c.fused, c.block, m) != SWE_OK) continue;
        rc = S.one_step(cfl, nullptr);                      // warm-up
        if (rc == SWE_OK) rc = S.restore(sn);
        if (rc == SWE_OK) rc = (cudaEventRecord(e0, S.stream) == cudaSuccess) ? SWE_OK : SWE_ERR_CUDA;
        for (int q = 0; q < trials && rc == SWE_OK; q++) rc = S.one_step(cfl, nullptr);
        float ms = 0.f;
        if (rc == SWE_OK && cudaEventRecord(e1, S.stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            if (ms / trials < best_ms) { best_ms = ms / trials; best = c; }
        }
        int rr = S.restore(sn);
        if (rc == SWE_OK) rc = rr;
        if (rc != SWE_OK) break;
    }
    // the split kernels' prep block, with the chosen kernel and block
    int rc2 = S.configure(best.fused, best.block, m);
    if (rc == SWE_OK && rc2 == SWE_OK && !best.fused && S.p.scheme != SWE_SCHEME_HLLC) {
        const int pb0 = S.prep_bl;
        int best_pb = pb0;
        double best_pms = 1e30;
        for (int pb : {64, 128, 256}) {
            S.prep_bl = pb;
            rc = S.one_step(cfl, nullptr);                  // warm-up
            if (rc == SWE_OK) rc = S.restore(sn);
            if (rc == SWE_OK) rc = (cudaEventRecord(e0, S.stream) == cudaSuccess) ? SWE_OK : SWE_ERR_CUDA;
            for (int q = 0; q < trials && rc == SWE_OK; q++) rc = S.one_step(cfl, nullptr);
            float ms = 0.f;
            if (rc == SWE_OK && cudaEventRecord(e1, S.stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / trials < best_pms) {
                best_pms = ms / trials;
                best_pb = pb;
            }
            int rr = S.restore(sn);
            if (rc == SWE_OK) rc = rr;
            if (rc != SWE_OK) break;
        }
        S.prep_bl = rc == SWE_OK ? best_pb : pb0;
        if (rc == SWE_OK && best_pms < best_ms) best_ms = best_pms;
        S.clear_graphs();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc2 == SWE_OK) rc2 = S.restore(sn);
    S.drop(sn);
    if (rc != SWE_OK) return rc;
    if (rc2 != SWE_OK) return rc2;
    best_kernel = best.fused ? SWE_KERNEL_FUSED : SWE_KERNEL_SPLIT;
    best_block = best.block;
    return SWE_OK;
}

// ---- ensemble -----------------------------------------------------------------

template <typename T> struct EnsembleT {
    std::vector<StateT<T> *> mem;
    cudaStream_t stream = nullptr;
    int scheme = 0;
    double cfl = -1.0;                 // CFL number baked into the table
    bool built_fused = false;
    int built_block = 0;
    EnsEntry<T> *d_tab = nullptr;
    int2 *d_blk = nullptr;        // per block of the batched grid: (member, block within the member)
    size_t tab_cap = 0, blk_cap = 0;
    int grid = 0;
    size_t smem = 0;              // the tile kernel's dynamic shared memory
    TileArgs room{};              // its shared-memory room (the members' largest)
    // CUDA graphs of kGraphSteps batched steps, keyed by the starting step
    // phase (steps taken mod 6); captured on a private stream, dropped when
    // the table is rebuilt
    static constexpr int kGraphSteps = 24;
    std::map<int, cudaGraphExec_t> graphs;
    cudaStream_t cap_stream = nullptr;

    ~EnsembleT()
    {
        if (stream) cudaStreamSynchronize(stream);
        clear_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        dev_free(d_tab, stream);
        dev_free(d_blk, stream);
    }

    void clear_graphs()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
    }

    cudaError_t launch_one(int phase, cudaStream_t s)
    {
        return launch_ensemble<T>(scheme, mem[0]->p.hr_order == 2, built_fused, d_tab, d_blk, phase, grid, built_block,
                                  room, s);
    }

    // kGraphSteps batched steps through a cached CUDA graph.
    int graph_steps()
    {
        const int ph0 = (int)(mem[0]->k % 6);
        auto it = graphs.find(ph0);
        if (it == graphs.end()) {
            if (!cap_stream) CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
            cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
            for (int q = 0; q < kGraphSteps && e == cudaSuccess; q++) e = launch_one((ph0 + q) % 6, cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cap_stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                swe_set_error("CUDA graph capture failed");
                return SWE_ERR_CUDA;
            }
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            CK(e);
            it = graphs.emplace(ph0, ex).first;
        }
        CK(cudaGraphLaunch(it->second, stream));
        for (StateT<T> *s : mem) { s->k += kGraphSteps; s->cur = (s->cur + kGraphSteps) & 1; }
        return SWE_OK;
    }

    int check_uniform()
    {
        StateT<T> &s0 = *mem[0];
        for (StateT<T> *s : mem) {
            if (s->sched) {
                swe_set_error("ensemble members run without a boundary-first schedule");
                return SWE_ERR_ARG;
            }
            if (s->p.scheme != s0.p.scheme || s->p.hr_order != s0.p.hr_order || s->p.time_scheme != SWE_EULER ||
                s->fused != s0.fused ||
                s->block() != s0.block() || s->stream != s0.stream || (s->k % 6) != (s0.k % 6)) {
                swe_set_error("ensemble members need the same scheme and reconstruction order, Euler steps, kernel, block, stream and step phase");
                return SWE_ERR_ARG;
            }
        }
        return SWE_OK;
    }

    int build(double cfl_)
    {
        int rc = check_uniform();
        if (rc) return rc;
        const size_t nm = mem.size();
        std::vector<EnsEntry<T>> h(nm);
        std::vector<int> begin(nm + 1, 0);
        const bool fused = mem[0]->fused;
        size_t smem_max = 0;
        const int block = mem[0]->block();
        TileArgs room_{};
        room_.tile = block;
        const int lim = ensemble_max_threads<T>(mem[0]->p.scheme, mem[0]->p.hr_order == 2, fused);
        if (block > lim) {
            swe_set_error("block of " + std::to_string(block) + " threads exceeds the batched kernels' limit of " +
                          std::to_string(lim));
            return lim > 0 ? SWE_ERR_ARG : SWE_ERR_CUDA;
        }
        for (size_t m = 0; m < nm; m++) {
            StateT<T> &s = *mem[m];
            for (int ph = 0; ph < 6; ph++) h[m].a[ph] = s.args_for_phase(ph, cfl_);
            h[m].t = s.ta;
            h[m].F = s.F;
            h[m].U = s.U;
            const int64_t blocks = fused ? s.ta.n_tiles : (s.n + block - 1) / block;
            if ((int64_t)begin[m] + blocks > INT32_MAX) { swe_set_error("ensemble too large"); return SWE_ERR_ARG; }
            begin[m + 1] = begin[m] + (int)blocks;
            if (fused) {
                room_.hmax = std::max(room_.hmax, s.ta.hmax); room_.h1max = std::max(room_.h1max, s.ta.h1max);
                room_.wmax = std::max(room_.wmax, s.ta.wmax);
            }
        }
        const size_t nb = (size_t)begin[nm];
        std::vector<int2> blk(nb);
        for (size_t m = 0; m < nm; m++)
            for (int b = begin[m]; b < begin[m + 1]; b++) blk[b] = make_int2((int)m, b - begin[m]);
        if (fused) smem_max = tile_smem_bytes<T>(room_);
        if (smem_max > 227 * 1024) { swe_set_error("tile needs more shared memory than a block has"); return SWE_ERR_ARG; }
        if (tab_cap < nm) {
            dev_free(d_tab, stream);
            d_tab = (EnsEntry<T> *)dev_alloc(sizeof(EnsEntry<T>) * nm, stream);
            if (!d_tab) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
            tab_cap = nm;
        }
        if (blk_cap < nb) {
            dev_free(d_blk, stream);
            d_blk = (int2 *)dev_alloc(sizeof(int2) * nb, stream);
            if (!d_blk) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
            blk_cap = nb;
        }
        CK(cudaMemcpyAsync(d_tab, h.data(), sizeof(EnsEntry<T>) * nm, cudaMemcpyHostToDevice, stream));
        CK(cudaMemcpyAsync(d_blk, blk.data(), sizeof(int2) * nb, cudaMemcpyHostToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        CK(ensemble_prepare<T>(mem[0]->p.scheme, fused, smem_max));
        clear_graphs();
        grid = begin[nm];
        smem = smem_max;
        room = room_;
        cfl = cfl_;
        built_fused = fused;
        built_block = block;
        return SWE_OK;
    }

    int step(int n, double cfl_)
    {
        if (n < 0 || !(cfl_ > 0.0)) { swe_set_error("swe_ensemble_step: bad argument"); return SWE_ERR_ARG; }
        // members stepped on their own in between must still share the step phase
        int rc = check_uniform();
        if (rc) return rc;
        if (cfl_ != cfl || built_fused != mem[0]->fused || built_block != mem[0]->block()) {
            rc = build(cfl_);
            if (rc) return rc;
        }
        for (StateT<T> *s : mem)
            if (!s->smax_valid) { rc = s->init_smax(); if (rc) return rc; }
        int left = n;
        while (left >= kGraphSteps) {
            rc = graph_steps();
            if (rc) return rc;
            left -= kGraphSteps;
        }
        for (; left > 0; left--) {
            CK(launch_one((int)(mem[0]->k % 6), stream));
            for (StateT<T> *s : mem) { s->k++; s->cur ^= 1; }
        }
        return SWE_OK;
    }

    int sync()
    {
        CK(cudaStreamSynchronize(stream));
        for (StateT<T> *s : mem) {
            int rc = s->status();
            if (rc) return rc;
        }
        return SWE_OK;
    }

    int autotune(const swe_mesh *const *meshes, int trials, double cfl_, int &best_kernel, int &best_block,
                 double &best_ms)
    {
        if (trials < 1 || !(cfl_ > 0)) { swe_set_error("swe_ensemble_autotune: bad argument"); return SWE_ERR_ARG; }
        const size_t nm = mem.size();
        for (size_t m = 0; m < nm; m++)
            if (meshes && (!meshes[m] || meshes[m]->n != mem[m]->n)) {
                swe_set_error("swe_ensemble_autotune: meshes do not match the members");
                return SWE_ERR_ARG;
            }
        for (StateT<T> *s : mem)
            if (!s->smax_valid) { int rc = s->init_smax(); if (rc) return rc; }
        std::vector<typename StateT<T>::Snapshot> sn(nm);
        for (size_t m = 0; m < nm; m++) { int rc = mem[m]->snapshot(sn[m]); if (rc) return rc; }
        const Candidate start{mem[0]->fused, mem[0]->block()};
        Candidate best = start;
        best_ms = 1e30;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        int rc = SWE_OK;
        for (const Candidate &c : candidates(*mem[0], meshes ? meshes[0] : nullptr)) {
            bool ok = true;
            for (size_t m = 0; m < nm && ok; m++) ok = mem[m]->configure(c.fused, c.block, meshes ? meshes[m] : nullptr) == SWE_OK;
            if (!ok || build(cfl_) != SWE_OK) continue;
            rc = step(1, cfl_);
            for (size_t m = 0; m < nm && rc == SWE_OK; m++) rc = mem[m]->restore(sn[m]);
            if (rc == SWE_OK) rc = cudaEventRecord(e0, stream) == cudaSuccess ? SWE_OK : SWE_ERR_CUDA;
            if (rc == SWE_OK) rc = step(trials, cfl_);
            float ms = 0.f;
            if (rc == SWE_OK && cudaEventRecord(e1, stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / trials < best_ms) {
                best_ms = ms / trials;
                best = c;
            }
            for (size_t m = 0; m < nm; m++) { int rr = mem[m]->restore(sn[m]); if (rc == SWE_OK) rc = rr; }
            if (rc != SWE_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int rc2 = SWE_OK;
        for (size_t m = 0; m < nm && rc2 == SWE_OK; m++) rc2 = mem[m]->configure(best.fused, best.block, meshes ? meshes[m] : nullptr);
        for (size_t m = 0; m < nm && rc2 == SWE_OK; m++) rc2 = mem[m]->restore(sn[m]);
        for (size_t m = 0; m < nm; m++) mem[m]->drop(sn[m]);
        if (rc2 == SWE_OK) rc2 = build(cfl_);
        if (rc != SWE_OK) return rc;
        if (rc2 != SWE_OK) return rc2;
        best_kernel = best.fused ? SWE_KERNEL_FUSED : SWE_KERNEL_SPLIT;
        best_block = best.block;
        return SWE_OK;
    }
};

bool valid_params(const swe_params *p)
{
    return p && p->scheme >= 0 && p->scheme <= 3 && (p->precision == SWE_FP64 || p->precision == SWE_FP32) &&
           (p->time_scheme == SWE_EULER || p->time_scheme == SWE_HEUN) && p->waf_limiter >= 0 &&
           p->waf_limiter <= SWE_WAF_VANLEER && p->g > 0 && p->h_eps > 0 && p->r_eps >= 0 && p->kernel >= 0 &&
           p->kernel <= 2 && p->block >= 0 && p->block <= 1024 && (p->block % 32) == 0 &&
           (p->cfl_mode == SWE_CFL_GLOBAL || p->cfl_mode == SWE_CFL_LOCAL) &&
           (p->scheme != SWE_SCHEME_MUSCL_EDGE || (p->muscl_beta >= 1.0 && p->muscl_beta <= 2.0)) &&
           (p->scheme != SWE_SCHEME_MUSCL_EDGE || p->kernel != SWE_KERNEL_FUSED) &&
           (p->hr_order == 1 || (p->hr_order == 2 && p->scheme == SWE_SCHEME_MUSCL && p->kernel != SWE_KERNEL_FUSED)) &&
           (p->waf_ratio == SWE_WAF_RATIO_DEPTH || p->waf_ratio == SWE_WAF_RATIO_SURFACE);
}

template <typename T>
int state_init(StateT<T> &s, const swe_mesh *m, const double *h, const double *hu, const double *hv,
               const double *z, const double *nman, const swe_bc_values *bc)
{
    const int64_t n = m->n;
    s.n = n;
    s.r_min = m->r_min;
    std::vector<int32_t> nbr((size_t)(3 * n));
    std::vector<Vec2<T>> ln((size_t)(3 * n)), dd((size_t)(3 * n));
    std::vector<T> zt((size_t)n), nt((size_t)n);
    bool friction = false;
    for (int64_t i = 0; i < n; i++) {
        int32_t o = m->perm[i];
        zt[i] = (T)z[o];
        nt[i] = nman ? (T)nman[o] : T(0);
        friction = friction || (nman && nman[o] > 0.0);
        for (int k = 0; k < 3; k++) {
            int64_t e = 3 * i + k;
            nbr[e] = swe_pack_nbr(*m, i, k);
            ln[e].x = (T)m->lnx[e]; ln[e].y = (T)m->lny[e];
            dd[e].x = (T)m->dx[e]; dd[e].y = (T)m->dy[e];
        }
    }
    if (bc) {
        for (int g = 0; g < bc->n_inflow && g < SWE_MAX_GROUPS; g++)
            s.qlen[g] = m->group_len[g] > 0.0 ? (T)(bc->inflow_q[g] / m->group_len[g]) : T(0);
        for (int g = 0; g < bc->n_level && g < SWE_MAX_GROUPS; g++) s.level[g] = (T)bc->level[g];
    }
    // per-cell arrays the tile step copies by whole tiles: allocated (and
    // zero-filled) to a multiple of the largest tile
    const int64_t np = (n + kTilePad - 1) / kTilePad * kTilePad;
    s.nbr = s.template alloc<int32_t>(3 * np);
    s.perm = s.template alloc<int32_t>(n);
    s.ln = s.template alloc<Vec2<T>>(3 * np);
    if (s.p.scheme == SWE_SCHEME_WAF) s.dd = s.template alloc<Vec2<T>>(3 * n);   // WAF's centroid distance
    s.z = s.template alloc<T>(np);
    if (friction) s.nman = s.template alloc<T>(np);
    s.area = s.template alloc<double>(n);
    const int nbuf = s.p.time_scheme == SWE_HEUN ? 3 : 2;
    for (int b = 0; b < nbuf; b++) {
        s.h[b] = s.template alloc<T>(np); s.hu[b] = s.template alloc<T>(np); s.hv[b] = s.template alloc<T>(np);
    }
    s.sc = s.template alloc<DevScalars>(1);
    s.n_part = mass_partials_needed(n);
    s.mass_part = s.template alloc<double>(2 * s.n_part);   // (sum, compensation) per block
    s.mass_out = s.template alloc<double>(1);
    s.staging = s.template alloc<double>(3 * n);
    s.dt_hist = s.template alloc<double>(SWE_DT_HISTORY);
    for (auto &b : s.mem.blocks)
        if (!b.first) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
    if (!s.nbr || !s.staging) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
    cudaStream_t st = s.stream;
    CK(cudaMemcpyAsync(s.nbr, nbr.data(), sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.perm, m->perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.ln, ln.data(), sizeof(Vec2<T>) * 3 * n, cudaMemcpyHostToDevice, st));
    if (s.dd) CK(cudaMemcpyAsync(s.dd, dd.data(), sizeof(Vec2<T>) * 3 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.z, zt.data(), sizeof(T) * n, cudaMemcpyHostToDevice, st));
    if (s.nman) CK(cudaMemcpyAsync(s.nman, nt.data(), sizeof(T) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.area, m->area.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(s.sc, 0, sizeof(DevScalars), st));
    {
        // kernel choice (SWE_KERNEL_AUTO): the one-pass tile step, in tiles of
        // 128 cells, for FP64, whose time is FP64 arithmetic and which gains
        // from solving each edge once (13M river, MUSCL: 11.5 against 13.1 ms
        // per step; HLLC: 9.7 against 13.2); the split kernels for FP32, whose
        // time is memory traffic and instruction issue at high occupancy
        const bool want_fused = s.p.kernel == SWE_KERNEL_FUSED ||
                                (s.p.kernel == SWE_KERNEL_AUTO && s.tile_capable() && std::is_same<T, double>::value);
        const int bl = s.p.block > 0 ? s.p.block : (want_fused && std::is_same<T, double>::value ? 128 : 256);
        int rc = s.configure(want_fused, bl, m);
        if (rc) return rc;
    }
    // initial state through the same path as swe_set_state
    CK(cudaMemcpyAsync(s.staging, h, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.staging + n, hu, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.staging + 2 * n, hv, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CK(launch_scatter_in<T>(n, s.perm, s.staging, s.h[0], s.hu[0], s.hv[0], st));
    CK(cudaStreamSynchronize(st));   // host vectors above go out of scope
    return s.init_smax();
}

}  // namespace

struct swe_state {
    int precision = SWE_FP64;
    std::unique_ptr<StateT<float>> f;
    std::unique_ptr<StateT<double>> d;
};

#define DISPATCH(st, expr)                 \
    ((st)->precision == SWE_FP32 ? [&](auto &S) { return expr; }(*(st)->f) : [&](auto &S) { return expr; }(*(st)->d))

extern "C" {

const char *swe_last_error(void) { return g_err.c_str(); }

int swe_params_default(swe_params *p, int scheme, int precision)
{
    if (!p || scheme < 0 || scheme > 3 || (precision != SWE_FP64 && precision != SWE_FP32)) {
        swe_set_error("swe_params_default: bad argument");
        return SWE_ERR_ARG;
    }
    std::memset(p, 0, sizeof(*p));
    p->scheme = scheme;
    p->precision = precision;
    p->time_scheme = SWE_EULER;
    p->waf_limiter = SWE_WAF_SUPERBEE;
    p->g = 9.81;
    p->h_eps = precision == SWE_FP64 ? 1e-6 : 1e-4;
    p->r_eps = precision == SWE_FP64 ? 1e-12 : 1e-6;
    p->kernel = SWE_KERNEL_AUTO;
    p->block = 0;
    p->cfl_mode = SWE_CFL_GLOBAL;
    p->muscl_beta = 2.0;
    p->hr_order = 1;
    p->waf_ratio = SWE_WAF_RATIO_SURFACE;
    return SWE_OK;
}

int swe_set_allocator(swe_alloc_fn alloc, swe_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        swe_set_error("swe_set_allocator: give both functions or neither");
        return SWE_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc; g_free = free_fn; g_ctx = ctx;
    return SWE_OK;
}

int swe_mesh_create(const double *node_xy, int64_t n_nodes, const int32_t *tri, int64_t n_tri,
                    const int32_t *bnd_edges, const int32_t *bnd_tag, int64_t n_bnd,
                    const int32_t *cut_edges, int64_t n_cut, int reorder, swe_mesh **out)
{
    if (out) *out = nullptr;
    try {
        return swe_mesh_build_host(node_xy, n_nodes, tri, n_tri, bnd_edges, bnd_tag, n_bnd, cut_edges, n_cut,
                                   reorder, out);
    } catch (const std::bad_alloc &) {
        swe_set_error("swe_mesh_create: out of host memory");
        return SWE_ERR_NOMEM;
    }
}

int swe_mesh_destroy(swe_mesh *m)
{
    delete m;
    return SWE_OK;
}

int swe_mesh_info(const swe_mesh *m, int64_t *n_cells, double *r_min)
{
    if (!m) { swe_set_error("swe_mesh_info: NULL mesh"); return SWE_ERR_ARG; }
    if (n_cells) *n_cells = m->n;
    if (r_min) *r_min = m->r_min;
    return SWE_OK;
}

int swe_mesh_export(const swe_mesh *m, int32_t *perm, int32_t *tri, int32_t *nbr, int32_t *nbr_edge,
                    int32_t *btag, double *lnx, double *lny, double *area, double *cx, double *cy,
                    double *rin, double *dx, double *dy)
{
    if (!m) { swe_set_error("swe_mesh_export: NULL mesh"); return SWE_ERR_ARG; }
    const size_t n = (size_t)m->n;
    auto cp = [](auto *dst, const auto &src) { if (dst) std::memcpy(dst, src.data(), src.size() * sizeof(src[0])); };
    cp(perm, m->perm); cp(tri, m->tri); cp(nbr, m->nbr); cp(nbr_edge, m->nbr_edge); cp(btag, m->btag);
    cp(lnx, m->lnx); cp(lny, m->lny); cp(area, m->area); cp(cx, m->cx); cp(cy, m->cy); cp(rin, m->rin);
    cp(dx, m->dx); cp(dy, m->dy);
    (void)n;
    return SWE_OK;
}

int swe_state_init(const swe_mesh *m, const swe_params *p, const double *h, const double *hu,
                   const double *hv, const double *z, const double *manning_n, const swe_bc_values *bc,
                   void *stream, swe_state **out)
{
    if (out) *out = nullptr;
    if (!m || !out || !h || !hu || !hv || !z || !valid_params(p)) {
        swe_set_error("swe_state_init: bad argument");
        return SWE_ERR_ARG;
    }
    if (bc && ((bc->n_inflow > 0 && !bc->inflow_q) || (bc->n_level > 0 && !bc->level) || bc->n_inflow < 0 ||
               bc->n_level < 0 || bc->n_inflow > SWE_MAX_GROUPS || bc->n_level > SWE_MAX_GROUPS)) {
        swe_set_error("swe_state_init: bad boundary values");
        return SWE_ERR_ARG;
    }
    auto *s = new swe_state();
    s->precision = p->precision;
    int rc;
    try {
        if (p->precision == SWE_FP32) {
            s->f.reset(new StateT<float>());
            s->f->p = *p; s->f->stream = (cudaStream_t)stream;
            rc = state_init<float>(*s->f, m, h, hu, hv, z, manning_n, bc);
        } else {
            s->d.reset(new StateT<double>());
            s->d->p = *p; s->d->stream = (cudaStream_t)stream;
            rc = state_init<double>(*s->d, m, h, hu, hv, z, manning_n, bc);
        }
    } catch (const std::bad_alloc &) {
        rc = SWE_ERR_NOMEM;
        swe_set_error("swe_state_init: out of host memory");
    }
    if (rc != SWE_OK) { delete s; return rc; }
    *out = s;
    return SWE_OK;
}

int swe_state_destroy(swe_state *s)
{
    if (!s) return SWE_OK;
    cudaStream_t st = s->precision == SWE_FP32 ? s->f->stream : s->d->stream;
    cudaStreamSynchronize(st);
    delete s;
    return SWE_OK;
}

int swe_set_stream(swe_state *s, void *stream)
{
    if (!s) { swe_set_error("swe_set_stream: NULL state"); return SWE_ERR_ARG; }
    return DISPATCH(s, (S.stream = (cudaStream_t)stream, SWE_OK));
}

int swe_set_state(swe_state *s, const double *h, const double *hu, const double *hv)
{
    if (!s || !h || !hu || !hv) { swe_set_error("swe_set_state: bad argument"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        const int64_t n = S.n;
        CK(cudaMemcpyAsync(S.staging, h, sizeof(double) * n, cudaMemcpyHostToDevice, S.stream));
        CK(cudaMemcpyAsync(S.staging + n, hu, sizeof(double) * n, cudaMemcpyHostToDevice, S.stream));
        CK(cudaMemcpyAsync(S.staging + 2 * n, hv, sizeof(double) * n, cudaMemcpyHostToDevice, S.stream));
        CK(launch_scatter_in(n, S.perm, S.staging, S.h[S.cur], S.hu[S.cur], S.hv[S.cur], S.stream));
        CK(cudaMemsetAsync(&S.sc->status, 0, sizeof(int), S.stream));
        return S.init_smax();
    })());
}

int swe_step(swe_state *s, int n_steps, double cfl)
{
    if (!s || n_steps < 0 || !(cfl > 0.0) || !std::isfinite(cfl)) {
        swe_set_error("swe_step: bad argument");
        return SWE_ERR_ARG;
    }
    return DISPATCH(s, ([&]() -> int {
        if (!S.smax_valid) { int rc = S.init_smax(); if (rc) return rc; }
        int left = n_steps;
        while (left > 0) {
            int rc;
            if (S.use_graphs && !S.prof && left >= S.kGraphSteps) {
                rc = S.graph_steps(cfl);
                left -= S.kGraphSteps;
            } else {
                rc = S.one_step(cfl, nullptr);
                left -= 1;
            }
            if (rc) return rc;
        }
        return SWE_OK;
    })());
}

int swe_step_dt(swe_state *s, const double *dt, int n_steps)
{
    if (!s || n_steps < 0 || (n_steps > 0 && !dt)) { swe_set_error("swe_step_dt: bad argument"); return SWE_ERR_ARG; }
    for (int q = 0; q < n_steps; q++)
        if (!(dt[q] >= 0.0) || !std::isfinite(dt[q])) { swe_set_error("swe_step_dt: bad time step"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        if (n_steps == 0) return SWE_OK;
        if (S.dtbuf_len < n_steps) {
            CK(cudaStreamSynchronize(S.stream));
            for (auto it = S.mem.blocks.begin(); it != S.mem.blocks.end(); ++it)
                if (it->first == S.dtbuf) { dev_free(it->first, S.stream); S.mem.bytes -= (int64_t)((it->second + 255) & ~size_t(255)); S.mem.blocks.erase(it); break; }
            S.dtbuf = S.template alloc<double>((size_t)std::max(n_steps, 64));
            if (!S.dtbuf) { swe_set_error("device allocation failed"); return SWE_ERR_NOMEM; }
            S.dtbuf_len = std::max(n_steps, 64);
        }
        CK(cudaMemcpyAsync(S.dtbuf, dt, sizeof(double) * n_steps, cudaMemcpyHostToDevice, S.stream));
        if (!S.smax_valid) { int rc = S.init_smax(); if (rc) return rc; }
        for (int q = 0; q < n_steps; q++) {
            int rc = S.one_step(1.0, S.dtbuf + q);
            if (rc) return rc;
        }
        // the replayed sequence must stay readable until the kernels ran
        CK(cudaStreamSynchronize(S.stream));
        return SWE_OK;
    })());
}

int swe_sync(swe_state *s)
{
    if (!s) { swe_set_error("swe_sync: NULL state"); return SWE_ERR_ARG; }
    return DISPATCH(s, S.status());
}

int swe_get_state(swe_state *s, double *h, double *hu, double *hv)
{
    if (!s || !h || !hu || !hv) { swe_set_error("swe_get_state: bad argument"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        const int64_t n = S.n;
        CK(launch_gather_out(n, S.perm, S.h[S.cur], S.hu[S.cur], S.hv[S.cur], S.staging, S.stream));
        CK(cudaMemcpyAsync(h, S.staging, sizeof(double) * n, cudaMemcpyDeviceToHost, S.stream));
        CK(cudaMemcpyAsync(hu, S.staging + n, sizeof(double) * n, cudaMemcpyDeviceToHost, S.stream));
        CK(cudaMemcpyAsync(hv, S.staging + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, S.stream));
        return S.status();
    })());
}

int swe_mass(swe_state *s, double *mass, double *clipped_mass, double *boundary_net_inflow)
{
    if (!s) { swe_set_error("swe_mass: NULL state"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        double m = 0.0;
        CK(launch_mass(S.dmesh(), S.h[S.cur], S.mass_part, S.n_part, S.mass_out, S.stream));
        CK(cudaMemcpyAsync(&m, S.mass_out, sizeof(double), cudaMemcpyDeviceToHost, S.stream));
        DevScalars d;
        int rc = S.read_scalars(d);
        if (rc) return rc;
        if (mass) *mass = m;
        if (clipped_mass) *clipped_mass = d.clipped;
        if (boundary_net_inflow) *boundary_net_inflow = d.bnd_in;
        return S.status();
    })());
}

int swe_time(swe_state *s, double *t, int64_t *steps)
{
    if (!s) { swe_set_error("swe_time: NULL state"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        DevScalars d;
        int rc = S.read_scalars(d);
        if (rc) return rc;
        if (t) *t = d.t;
        if (steps) *steps = d.steps;
        return S.status();
    })());
}

int swe_flags(swe_state *s, int *flags)
{
    if (!s || !flags) { swe_set_error("swe_flags: bad argument"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        DevScalars d;
        int rc = S.read_scalars(d);
        if (rc) return rc;
        *flags = (d.clipped > 0.0 ? SWE_FLAG_CLIPPED : 0) | ((d.status & ST_NONFINITE) ? SWE_FLAG_NONFINITE : 0) |
                 ((d.status & ST_DRY) ? SWE_FLAG_DRY : 0);
        return SWE_OK;
    })());
}

int swe_state_info(const swe_state *s, int64_t *device_bytes, int *kernel, int *block)
{
    if (!s) { swe_set_error("swe_state_info: NULL state"); return SWE_ERR_ARG; }
    auto *ms = const_cast<swe_state *>(s);
    return DISPATCH(ms, ([&]() -> int {
        if (device_bytes) *device_bytes = S.mem.bytes;
        if (kernel) *kernel = S.fused ? SWE_KERNEL_FUSED : SWE_KERNEL_SPLIT;
        if (block) *block = S.block();
        return SWE_OK;
    })());
}

int swe_profile_begin(swe_state *s)
{
    if (!s) { swe_set_error("swe_profile_begin: NULL state"); return SWE_ERR_ARG; }
    return DISPATCH(s, (S.prof = true, SWE_OK));
}

int swe_profile_end(swe_state *s, double *kernel_ms, int64_t *launches)
{
    if (!s) { swe_set_error("swe_profile_end: NULL state"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        CK(cudaStreamSynchronize(S.stream));
        double ms[SWE_K_COUNT] = {};
        int64_t cnt[SWE_K_COUNT] = {};
        for (auto &e : S.ev_used) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, std::get<1>(e), std::get<2>(e)));
            ms[std::get<0>(e)] += t;
            cnt[std::get<0>(e)]++;
            S.ev_pool.push_back(std::get<1>(e));
            S.ev_pool.push_back(std::get<2>(e));
        }
        S.ev_used.clear();
        S.prof = false;
        for (int q = 0; q < SWE_K_COUNT; q++) {
            if (kernel_ms) kernel_ms[q] = ms[q];
            if (launches) launches[q] = cnt[q];
        }
        return SWE_OK;
    })());
}

int swe_dt_history(swe_state *s, double *dt, int n)
{
    if (!s || n < 0 || n > SWE_DT_HISTORY || (n > 0 && !dt)) { swe_set_error("swe_dt_history: bad argument"); return SWE_ERR_ARG; }
    return DISPATCH(s, ([&]() -> int {
        DevScalars d;
        int rc = S.read_scalars(d);
        if (rc) return rc;
        if (n > d.steps) { swe_set_error("swe_dt_history: fewer steps taken"); return SWE_ERR_ARG; }
        std::vector<double> ring(SWE_DT_HISTORY);
        CK(cudaMemcpy(ring.data(), S.dt_hist, sizeof(double) * SWE_DT_HISTORY, cudaMemcpyDeviceToHost));
        for (int q = 0; q < n; q++) {
            long long idx = d.steps - n + q;
            dt[q] = ring[(size_t)(idx % SWE_DT_HISTORY)];
        }
        return SWE_OK;
    })());
}

struct swe_ensemble {
    int precision = SWE_FP64;
    std::unique_ptr<EnsembleT<float>> f;
    std::unique_ptr<EnsembleT<double>> d;
};

int swe_ensemble_create(swe_state *const *members, int n_members, swe_ensemble **out)
{
    if (out) *out = nullptr;
    if (!members || n_members < 1 || !out) { swe_set_error("swe_ensemble_create: bad argument"); return SWE_ERR_ARG; }
    for (int m = 0; m < n_members; m++)
        if (!members[m] || members[m]->precision != members[0]->precision) {
            swe_set_error("swe_ensemble_create: members must exist and share the precision");
            return SWE_ERR_ARG;
        }
    {
        // a state listed twice would be stepped twice per step, both times from the same old state
        std::vector<const swe_state *> seen(members, members + n_members);
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
            swe_set_error("swe_ensemble_create: a state is listed more than once");
            return SWE_ERR_ARG;
        }
    }
    auto *e = new swe_ensemble();
    e->precision = members[0]->precision;
    auto fill = [&](auto &E, auto getter) -> int {
        for (int m = 0; m < n_members; m++) E.mem.push_back(getter(members[m]));
        E.stream = E.mem[0]->stream;
        E.scheme = E.mem[0]->p.scheme;
        return E.check_uniform();
    };
    int rc;
    if (e->precision == SWE_FP32) {
        e->f.reset(new EnsembleT<float>());
        rc = fill(*e->f, [](swe_state *s) { return s->f.get(); });
    } else {
        e->d.reset(new EnsembleT<double>());
        rc = fill(*e->d, [](swe_state *s) { return s->d.get(); });
    }
    if (rc) { delete e; return rc; }
    *out = e;
    return SWE_OK;
}

int swe_ensemble_destroy(swe_ensemble *e)
{
    delete e;
    return SWE_OK;
}

int swe_ensemble_step(swe_ensemble *e, int n_steps, double cfl)
{
    if (!e) { swe_set_error("swe_ensemble_step: NULL ensemble"); return SWE_ERR_ARG; }
    return e->precision == SWE_FP32 ? e->f->step(n_steps, cfl) : e->d->step(n_steps, cfl);
}

int swe_ensemble_sync(swe_ensemble *e)
{
    if (!e) { swe_set_error("swe_ensemble_sync: NULL ensemble"); return SWE_ERR_ARG; }
    return e->precision == SWE_FP32 ? e->f->sync() : e->d->sync();
}

int swe_ensemble_autotune(swe_ensemble *e, const swe_mesh *const *meshes, int trial_steps, double cfl,
                          int *kernel, int *block, double *ms_per_step)
{
    if (!e) { swe_set_error("swe_ensemble_autotune: NULL ensemble"); return SWE_ERR_ARG; }
    int k = 0, b = 0;
    double ms = 0.0;
    int rc = e->precision == SWE_FP32 ? e->f->autotune(meshes, trial_steps, cfl, k, b, ms)
                                      : e->d->autotune(meshes, trial_steps, cfl, k, b, ms);
    if (rc == SWE_OK) {
        if (kernel) *kernel = k;
        if (block) *block = b;
        if (ms_per_step) *ms_per_step = ms;
    }
    return rc;
}

int swe_autotune(swe_state *s, const swe_mesh *m, int trial_steps, double cfl, int *kernel, int *block,
                 double *ms_per_step)
{
    if (!s) { swe_set_error("swe_autotune: NULL state"); return SWE_ERR_ARG; }
    int k = 0, b = 0;
    double ms = 0.0;
    int rc = s->precision == SWE_FP32 ? autotune(*s->f, m, trial_steps, cfl, k, b, ms)
                                      : autotune(*s->d, m, trial_steps, cfl, k, b, ms);
    if (rc == SWE_OK) {
        if (kernel) *kernel = k;
        if (block) *block = b;
        if (ms_per_step) *ms_per_step = ms;
    }
    return rc;
}

// ---- partitions and the boundary-first schedule ---------------------------

int swe_partition_create(const swe_mesh *m, int n_parts, swe_partition **out)
{
    if (out) *out = nullptr;
    if (!m || !out || n_parts < 1) {
        swe_set_error("swe_partition_create: bad argument");
        return SWE_ERR_ARG;
    }
    auto *p = new (std::nothrow) swe_partition();
    if (!p) { swe_set_error("host allocation failed"); return SWE_ERR_NOMEM; }
    if (swe_partition_build(*m, n_parts, *p) != 0) {
        delete p;
        swe_set_error("swe_partition_create: the part count must be within 1 .. min(1024, cells)");
        return SWE_ERR_ARG;
    }
    *out = p;
    return SWE_OK;
}

int swe_partition_destroy(swe_partition *p)
{
    delete p;
    return SWE_OK;
}

int swe_partition_info(const swe_partition *p, int part, int64_t *owned_begin, int64_t *owned_end,
                       int64_t *n_halo1, int64_t *n_halo2, int64_t *n_boundary)
{
    if (!p || part < 0 || part >= p->n_parts) { swe_set_error("swe_partition_info: bad argument"); return SWE_ERR_ARG; }
    if (owned_begin) *owned_begin = p->start[part];
    if (owned_end) *owned_end = p->start[part + 1];
    if (n_halo1) *n_halo1 = (int64_t)p->halo1[part].size();
    if (n_halo2) *n_halo2 = (int64_t)p->halo2[part].size();
    if (n_boundary) *n_boundary = (int64_t)p->boundary[part].size();
    return SWE_OK;
}

int swe_partition_export(const swe_partition *p, int part, int32_t *halo1, int32_t *halo2, int32_t *boundary)
{
    if (!p || part < 0 || part >= p->n_parts) { swe_set_error("swe_partition_export: bad argument"); return SWE_ERR_ARG; }
    if (halo1) std::copy(p->halo1[part].begin(), p->halo1[part].end(), halo1);
    if (halo2) std::copy(p->halo2[part].begin(), p->halo2[part].end(), halo2);
    if (boundary) std::copy(p->boundary[part].begin(), p->boundary[part].end(), boundary);
    return SWE_OK;
}

int swe_set_partition(swe_state *s, const swe_partition *part)
{
    if (!s) { swe_set_error("swe_set_partition: bad argument"); return SWE_ERR_ARG; }
    return DISPATCH(s, S.set_partition(part));
}

int swe_halo_get(swe_state *s, int part, double *h, double *hu, double *hv)
{
    if (!s) { swe_set_error("swe_halo_get: bad argument"); return SWE_ERR_ARG; }
    return DISPATCH(s, S.halo_get(part, h, hu, hv));
}

// ---- the tile step's plan, host side ---------------------------------------

int swe_tile_plan_info(const swe_mesh *m, int tile, int64_t *n_tiles, int32_t *hmax, int32_t *h1max,
                       int32_t *wmax, int64_t *n_words)
{
    if (!m) { swe_set_error("swe_tile_plan_info: bad argument"); return SWE_ERR_ARG; }
    TilePlan tp;
    try {
        if (const int rc = swe_build_tile_plan(*m, tile, tp)) { swe_set_error(tile_plan_error(rc)); return SWE_ERR_ARG; }
    } catch (const std::bad_alloc &) {
        swe_set_error("host allocation failed");
        return SWE_ERR_NOMEM;
    }
    if (n_tiles) *n_tiles = tp.n_tiles;
    if (hmax) *hmax = tp.hmax;
    if (h1max) *h1max = tp.h1max;
    if (wmax) *wmax = tp.wmax;
    if (n_words) *n_words = (int64_t)tp.words.size();
    return SWE_OK;
}

int swe_tile_plan_export(const swe_mesh *m, int tile, int32_t *hdr, int32_t *words)
{
    if (!m) { swe_set_error("swe_tile_plan_export: bad argument"); return SWE_ERR_ARG; }
    TilePlan tp;
    try {
        if (const int rc = swe_build_tile_plan(*m, tile, tp)) { swe_set_error(tile_plan_error(rc)); return SWE_ERR_ARG; }
    } catch (const std::bad_alloc &) {
        swe_set_error("host allocation failed");
        return SWE_ERR_NOMEM;
    }
    if (hdr) std::copy(tp.hdr.begin(), tp.hdr.end(), hdr);
    if (words) std::copy(tp.words.begin(), tp.words.end(), words);
    return SWE_OK;
}


}  // extern "C"
