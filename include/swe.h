/*
 * swe.h -- C ABI of the GB300 shallow-water finite-volume library.
 *
 * The library advances the 2D shallow-water equations (h, hu, hv) on an
 * unstructured triangle mesh with bathymetry by explicit finite-volume steps
 * (Delmas & Soulaimani, arXiv 2307.16758, Sec. 6.1: the semi-discrete form
 * |Omega_i| dU_i/dt = -sum_j L_ij T^-1 G~(T U_i, T U_j) + sources, explicit
 * Euler in time, CFL time step with the inscribed radius).  Fluxes are HLLC
 * (Sec. 6.2.1), HLLC on MUSCL states (least-squares gradients with a
 * Barth-Jespersen limiter) or WAF (Sec. 6.2.2), with a well-balanced
 * hydrostatic reconstruction, wet/dry handling and Manning friction.  Every
 * step runs in CUDA kernels for sm_103a; the host side only builds the mesh,
 * copies inputs and outputs, and launches.
 *
 * Conventions
 *  - Every function returns SWE_OK (0) or a negative SWE_ERR_* code and never
 *    aborts; swe_last_error() gives a message for the calling thread.
 *  - Host arrays are caller-owned and are copied; outputs go into
 *    caller-allocated buffers.  Per-cell arrays use the caller's (original)
 *    cell order: the library renumbers cells internally and undoes the
 *    permutation on output.
 *  - Cell ids are int32 (fewer than 2^28 cells per mesh).
 *  - Boundary tags: tag = kind + 4*group with kind SWE_WALL, SWE_OPEN
 *    (transmissive), SWE_INFLOW (group selects the discharge) or SWE_LEVEL
 *    (group selects the free-surface level); 0 <= group < SWE_MAX_GROUPS.
 *  - Device work is asynchronous on the state's stream.  Errors detected on
 *    the device (a non-finite value, no wet cell for the CFL rule) are
 *    returned by the next call that synchronises (swe_sync, swe_get_state,
 *    swe_mass, swe_time).
 */
#ifndef SWE_H
#define SWE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SWE_OK = 0,
    SWE_ERR_ARG = -1,        /* bad argument (NULL, size, enum, range) */
    SWE_ERR_MESH = -2,       /* invalid mesh (degenerate, non-manifold, bad tags) */
    SWE_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    SWE_ERR_DRY = -4,        /* CFL rule: no wet cell, no time step defined */
    SWE_ERR_NONFINITE = -5,  /* a non-finite depth or discharge was produced */
    SWE_ERR_TIMEOUT = -6,    /* a bounded device wait (a bulk copy into shared memory) gave up */
    SWE_ERR_NOMEM = -7       /* host or device allocation failed */
};

enum { SWE_WALL = 0, SWE_OPEN = 1, SWE_INFLOW = 2, SWE_LEVEL = 3 };
enum { SWE_REORDER_NONE = 0, SWE_REORDER_MORTON = 1, SWE_REORDER_RCM = 2 };
/* HLLC first order (Sec. 6.2.1); MUSCL-HLLC with least-squares gradients and
 * a Barth-Jespersen limiter; WAF-HLLC (Sec. 6.2.2); MUSCL_EDGE: the paper's
 * MUSCL (Sec. 6.2.3), slopes along each edge from the upwind means of the
 * two other neighbours, limited with parameter beta (split kernels only). */
enum { SWE_SCHEME_HLLC = 0, SWE_SCHEME_MUSCL = 1, SWE_SCHEME_WAF = 2, SWE_SCHEME_MUSCL_EDGE = 3 };
enum { SWE_FP64 = 0, SWE_FP32 = 1 };
enum { SWE_EULER = 0, SWE_HEUN = 1 };
/* WAF limiter A(r, c) = 1 - (1 - |c|) phi(r) (Sec. 6.2.2): SUPERBEE (the
 * paper's choice), phi = 1 (no limiting), phi = 0 (the HLLC flux), and two
 * other classical limiters: MINBEE phi = max(0, min(1, r)) and van Leer
 * phi = (r + |r|)/(1 + |r|).  Whatever the limiter, an edge whose Riemann
 * problem has no wet star region (a dry side: a dry cell or a dry
 * reconstructed depth; or two rarefactions that open a dry gap:
 * u_R - u_L >= 2(a_L + a_R)) takes A = 1, its HLLC flux. */
enum { SWE_WAF_SUPERBEE = 0, SWE_WAF_PHI1 = 1, SWE_WAF_PHI0 = 2, SWE_WAF_MINBEE = 3, SWE_WAF_VANLEER = 4 };
/* Quantity of the WAF ratios r_L, r_R (Sec. 6.2.2 takes the depth of the
 * Riemann problem): SURFACE (default) the free surface eta = h + z, whose
 * differences are those of the hydrostatically reconstructed depths
 * h* = eta - z_f of each edge; DEPTH the cell depth h (over a steep bed it
 * varies with the bathymetry at rest, and WAF-SUPERBEE grows spurious speeds
 * on river-like beds).  The two are equal on a flat bed. */
enum { SWE_WAF_RATIO_DEPTH = 0, SWE_WAF_RATIO_SURFACE = 1 };
enum { SWE_KERNEL_AUTO = 0, SWE_KERNEL_SPLIT = 1, SWE_KERNEL_FUSED = 2 };
/* CFL rule (Sec. 6.1, d = inscribed radius r): GLOBAL dt = CFL min_i r_i /
 * max_wet s_i as printed; LOCAL dt = CFL min over wet cells of r_i / s_i. */
enum { SWE_CFL_GLOBAL = 0, SWE_CFL_LOCAL = 1 };
#define SWE_MAX_GROUPS 16

typedef struct swe_mesh swe_mesh;
typedef struct swe_state swe_state;
typedef struct swe_ensemble swe_ensemble;
typedef struct swe_partition swe_partition;

/* Solver options.  Fill with swe_params_default, then override. */
typedef struct {
    int scheme;       /* SWE_SCHEME_*; HLLC first order, MUSCL-HLLC or WAF-HLLC */
    int precision;    /* SWE_FP64, or SWE_FP32 (FP32 state and fluxes; mass and time in FP64) */
    int time_scheme;  /* SWE_EULER (Sec. 6.1) or SWE_HEUN (two Euler stages averaged) */
    int waf_limiter;  /* SWE_WAF_* (Sec. 6.2.2; SUPERBEE is the paper's choice) */
    double g;         /* gravity [m/s^2] */
    double h_eps;     /* depth below which a cell counts as dry [m] */
    double r_eps;     /* WAF: relative size of a local change treated as zero */
    int kernel;       /* SWE_KERNEL_SPLIT: prep + flux kernels (face values in scratch);
                         SWE_KERNEL_FUSED: the one-pass tile step (LSQ MUSCL or HLLC, hr_order 1);
                         SWE_KERNEL_AUTO: the tile step in FP64 where it applies, else split */
    int block;        /* threads per block of the flux kernel, or cells per tile of the tile step
                         (a power of two, 32 .. 1024); 0: 256, or 128 for FP64 tiles (the split prep
                         kernels use 128 unless swe_autotune picks another) */
    int cfl_mode;     /* SWE_CFL_GLOBAL (default) or SWE_CFL_LOCAL */
    double muscl_beta; /* SWE_SCHEME_MUSCL_EDGE limiter, 1 (MINBEE) .. 2 (SUPERBEE, default) */
    int hr_order;     /* hydrostatic reconstruction: 1 on the cell bed (default); 2 (SWE_SCHEME_MUSCL,
                         split kernels) second order, with the linear bed that the reconstructed
                         eta and h imply in each cell -- the paper's future work (Sec. 7) */
    int waf_ratio;    /* SWE_WAF_RATIO_* (used by SWE_SCHEME_WAF only) */
} swe_params;

/* Values of the boundary groups (copied at init). */
typedef struct {
    int n_inflow;
    const double *inflow_q;   /* [n_inflow] discharge in m^3/s, spread per unit length over the group's edges */
    int n_level;
    const double *level;      /* [n_level] free-surface level in m */
} swe_bc_values;

const char *swe_last_error(void);

/* Defaults: g = 9.81, h_eps = 1e-6 (FP64) or 1e-4 (FP32),
 * r_eps = 1e-12 (FP64) or 1e-6 (FP32), Euler, SUPERBEE, automatic kernel,
 * global CFL form, muscl_beta = 2, hr_order = 1, waf_ratio = SWE_WAF_RATIO_SURFACE. */
int swe_params_default(swe_params *p, int scheme, int precision);

/* Device memory: by default cudaMalloc/cudaFree.  A host program (for example
 * the Python binding, which routes to PyTorch's caching allocator) may install
 * its own pair (both or neither; NULL, NULL restores the default); ctx is
 * passed back unchanged.  Global to the library.  Every block goes back to
 * the allocator that gave it out, so the pair may be replaced while states
 * exist; the old pair must stay callable until their memory is freed. */
typedef void *(*swe_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*swe_free_fn)(void *ptr, void *stream, void *ctx);
int swe_set_allocator(swe_alloc_fn alloc, swe_free_fn free_fn, void *ctx);

/* ---- Mesh (host only) -------------------------------------------------- */

/* Build a mesh (Sec. 6.1 notation: cells Omega_i, sides L_ij, normals n_ij).
 *  node_xy[n_nodes][2] FP64 coordinates; tri[n_tri][3] node ids (any
 *  orientation; the library orients counter-clockwise);
 *  bnd_edges[n_bnd][2] node pairs on the boundary with bnd_tag[n_bnd]
 *  (unlisted boundary edges are walls); cut_edges[n_cut][2] interior edges
 *  that act as walls on both sides (may be NULL when n_cut = 0);
 *  reorder: SWE_REORDER_NONE, _MORTON (centroid Z-order) or _RCM.
 * Errors: SWE_ERR_ARG, SWE_ERR_MESH (degenerate triangle, edge shared by more
 * than two cells, folded mesh, listed edge not on the boundary). */
int swe_mesh_create(const double *node_xy, int64_t n_nodes,
                    const int32_t *tri, int64_t n_tri,
                    const int32_t *bnd_edges, const int32_t *bnd_tag, int64_t n_bnd,
                    const int32_t *cut_edges, int64_t n_cut,
                    int reorder, swe_mesh **out);
int swe_mesh_destroy(swe_mesh *m);
/* Number of cells and the smallest inscribed radius (CFL rule, Sec. 6.1). */
int swe_mesh_info(const swe_mesh *m, int64_t *n_cells, double *r_min);

/* Export the builder's arrays in the library's (new) cell order; any pointer
 * may be NULL.  perm[new] = original id; tri[n][3] oriented; nbr[n][3]
 * neighbour (new id) or -1; nbr_edge[n][3] local edge index in the
 * neighbour or -1; btag[n][3] boundary tag or -1; lnx,lny[n][3] outward
 * normal times edge length; area, cx, cy, rin[n]; dx,dy[n][3] centroid
 * offset to the neighbour (0 on boundaries). */
int swe_mesh_export(const swe_mesh *m, int32_t *perm, int32_t *tri, int32_t *nbr,
                    int32_t *nbr_edge, int32_t *btag, double *lnx, double *lny,
                    double *area, double *cx, double *cy, double *rin,
                    double *dx, double *dy);

/* ---- State (device) ---------------------------------------------------- */

/* Allocate the device state for a mesh and upload it.  h, hu, hv, z and
 * manning_n are FP64 host arrays of n_cells in the original order (manning_n
 * may be NULL: no friction).  bc may be NULL.  stream is a cudaStream_t
 * (NULL: the legacy default stream).  The mesh may be destroyed afterwards. */
int swe_state_init(const swe_mesh *m, const swe_params *p,
                   const double *h, const double *hu, const double *hv,
                   const double *z, const double *manning_n,
                   const swe_bc_values *bc, void *stream, swe_state **out);
int swe_state_destroy(swe_state *s);
int swe_set_stream(swe_state *s, void *stream);
/* Replace the conserved variables from FP64 host arrays (original order);
 * time, step count and mass diagnostics are kept. */
int swe_set_state(swe_state *s, const double *h, const double *hu, const double *hv);

/* Advance n_steps explicit steps with the CFL rule dt = cfl * r_min / max_wet(sqrt(g h)+|u|)
 * (Sec. 6.1).  Asynchronous: returns once the work is enqueued. */
int swe_step(swe_state *s, int n_steps, double cfl);
/* Advance with a given time-step sequence dt[n_steps] (host array). */
int swe_step_dt(swe_state *s, const double *dt, int n_steps);
/* Wait for the stream and return the device status (SWE_OK or an error). */
int swe_sync(swe_state *s);

/* Copy the conserved variables U = (h, hu, hv) of Sec. 6.1 (cell averages of
 * the finite-volume form) to FP64 host arrays in the original order. */
int swe_get_state(swe_state *s, double *h, double *hu, double *hv);
/* Mass budget of the continuity equation (Sec. 6.1: integrated over the
 * cells, sum |Omega_i| h_i changes only through the boundary fluxes):
 * the sum of area*h in FP64 (deterministic, compensated), the mass added by
 * clipping negative depths and the net mass that entered through the
 * boundary since init (m^3).  Any output pointer may be NULL. */
int swe_mass(swe_state *s, double *mass, double *clipped_mass, double *boundary_net_inflow);
/* Simulated time, the FP64 sum of the explicit Euler steps' dt (Sec. 6.1),
 * and the number of steps. */
int swe_time(swe_state *s, double *t, int64_t *steps);
/* Flags of the state since init (waits for the stream): SWE_FLAG_CLIPPED
 * when a negative depth was clipped to zero at least once (the wet/dry
 * treatment of Sec. 6.2.3 keeps h >= 0; the mass added is in swe_mass) --
 * a warning, not an error; SWE_FLAG_NONFINITE and SWE_FLAG_DRY when the
 * device saw a non-finite value or no wet cell for the CFL rule (those also
 * make the next synchronising call return an error). */
enum { SWE_FLAG_CLIPPED = 1, SWE_FLAG_NONFINITE = 2, SWE_FLAG_DRY = 4 };
int swe_flags(swe_state *s, int *flags);
/* Device bytes held by the state and the kernel configuration in use. */
int swe_state_info(const swe_state *s, int64_t *device_bytes, int *kernel, int *block);

/* ---- Tracing ----------------------------------------------------------- */

/* Kernel kinds reported by swe_profile_end. */
enum { SWE_K_PREP = 0, SWE_K_FLUX = 1, SWE_K_HEUN_AVG = 2, SWE_K_SMAX = 3, SWE_K_FUSED = 4,
       SWE_K_ENSEMBLE = 5, SWE_K_COUNT = 8 };
#define SWE_DT_HISTORY 4096

/* While profiling, every kernel launched by swe_step / swe_step_dt is
 * bracketed by CUDA events on the state's stream (and CUDA graphs are not
 * used).  swe_profile_end waits for the stream and returns, per kernel kind,
 * the summed device time in ms and the number of launches (arrays of
 * SWE_K_COUNT; either may be NULL). */
int swe_profile_begin(swe_state *s);
int swe_profile_end(swe_state *s, double *kernel_ms, int64_t *launches);
/* The last n time steps taken (oldest first), n <= min(steps taken, SWE_DT_HISTORY). */
int swe_dt_history(swe_state *s, double *dt, int n);

/* ---- Arithmetic peak ------------------------------------------------------ */

/* Not in the paper.  Fused multiply-adds per second of this GPU in FP32 or
 * FP64 (precision SWE_FP32 / SWE_FP64), measured by one launch of
 * 8 x 256 threads per SM, each running 8 independent FMA chains `iters`
 * times (1 .. 2^20; about 65536 for FP32 and 2048 for FP64 give a few ms),
 * timed with CUDA events on `stream` (a cudaStream_t, may be NULL) after one
 * shorter warm-up launch.  *flops_per_s counts an FMA as two operations.
 * It is the denominator of the arithmetic roofline of the FP64 path.  Uses a
 * small device buffer from the allocator; blocks until the launch ends.
 * Errors: SWE_ERR_ARG, SWE_ERR_NOMEM, SWE_ERR_CUDA. */
int swe_fma_peak(int precision, int iters, void *stream, double *flops_per_s);

/* Not in the paper.  A self-check of the bounded waits that every in-kernel
 * wait of this library uses (the tile step's waits for its bulk copies into
 * shared memory): one block of 128 threads waits on an mbarrier whose phase
 * completes only if `arrive` is nonzero (one thread arrives).  With arrive = 0
 * nothing completes it: the wait gives up after `polls` polls (1 .. 2^22), the
 * kernel records that and returns, and the context stays usable -- the way a
 * tile step that loses a copy reports SWE_ERR_TIMEOUT instead of hanging.
 * *timed_out = 1 if the wait gave up, 0 if the phase completed.  Uses a small
 * device buffer from the allocator; blocks until the launch ends.
 * Errors: SWE_ERR_ARG, SWE_ERR_NOMEM, SWE_ERR_CUDA. */
int swe_probe_bounded_wait(uint32_t polls, int arrive, int *timed_out, void *stream);

/* ---- One step without device allocation ---------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory -- a plug-in inside an application that
 * owns the GPU's memory pools, or a real-time loop where an allocation could
 * block -- and therefore cannot create a swe_state.
 *
 * One MUSCL-HLLC explicit Euler step in FP32 (the same kernels as swe_step
 * with SWE_KERNEL_SPLIT) on caller-owned device buffers, with a given dt.
 * Inputs, in the library's cell order (see swe_mesh_export):
 *  nbr[3n]  packed neighbour words: (nbr << 3) | (nbr_edge << 1) | owner for
 *           an interior edge, owner = 1 when perm[i] < perm[nbr]; -1 - btag on
 *           a boundary edge;
 *  ln[3n][2] scaled outward normals (lnx, lny; the centroid offsets of the
 *           gradient are derived from them), z[n] bed, manning_n[n] (may be
 *           NULL), h, hu, hv[n];
 *  p: scheme SWE_SCHEME_MUSCL, precision SWE_FP32 and hr_order 1 (g, h_eps,
 *     r_eps, block are used); inflow_qlen[n_inflow] inflow discharge per unit
 *     length (m^2/s) per group; level[n_level] fixed levels; dt finite and
 *     >= 0; stream a cudaStream_t.
 * Outputs h_out, hu_out, hv_out[n]: no output may overlap another output or
 * any input (else SWE_ERR_ARG).
 * The face values (48 bytes per wet cell) go to a scratch array compiled
 * into the library (about 12.6 MB per GPU, held until the process exits), so
 * n_cells must not exceed SWE_NOALLOC_MAX_CELLS (else SWE_ERR_ARG).  The
 * first call on a GPU looks the array up (cudaGetSymbolAddress) with that GPU
 * current; make that first call before any stream capture.  All calls on a
 * GPU share the array, so calls that overlap on the GPU race.  Each call
 * enqueues three kernels on `stream` (dt travels as a kernel argument,
 * nothing is copied from the host) and returns without waiting; no status is
 * read back. */
#define SWE_NOALLOC_MAX_CELLS 262144
int swe_muscl_step_noalloc(int64_t n_cells, const int32_t *nbr, const float *ln, const float *z,
                           const float *manning_n, const float *h, const float *hu,
                           const float *hv, float *h_out, float *hu_out, float *hv_out, double dt,
                           const swe_params *p, const float *inflow_qlen, int n_inflow,
                           const float *level, int n_level, void *stream);

/* ---- Autotuner ----------------------------------------------------------- */

/* Not in the paper.  Time trial_steps CFL steps of each kernel configuration
 * (split kernels with 128/256/512 threads per block; for LSQ MUSCL and HLLC
 * with hr_order 1 also the tile step with tiles of 128/256/512 cells) on a
 * copy of the current state and keep the fastest; the simulation state, time
 * and step count are left as they were (every configuration computes the
 * same bits).  m is the state's mesh (needed to plan the tiles; NULL limits
 * the search to the split kernels).  With the split kernels it then times the
 * prep kernel's own block size (64/128/256 threads; 128 until tuned).
 * Outputs (may be NULL): SWE_KERNEL_*, threads per block of the flux kernel
 * or cells per tile, ms per step. */
int swe_autotune(swe_state *s, const swe_mesh *m, int trial_steps, double cfl, int *kernel, int *block,
                 double *ms_per_step);

/* ---- Partitions and the boundary-first schedule --------------------------- */

/* Not a multi-GPU path (one GPU here): the single-GPU rehearsal of the
 * paper's sub-domain schedule (Sec. 6.4).  A partition cuts a mesh into
 * n_parts contiguous ranges of its (Morton) cell order, of equal size to
 * within one cell, and records per part two halo layers (halo1: cells of
 * other parts next to the part; halo2: cells of other parts next to halo1,
 * which the second-order reconstructions of halo1 cells read), its boundary
 * cells (owned cells that another part holds in a halo) and the rest, its
 * interior.  Cell ids are in the library's (new) order, see swe_mesh_export.
 * Errors: SWE_ERR_ARG (n_parts outside 1 .. min(1024, cells)). */
int swe_partition_create(const swe_mesh *m, int n_parts, swe_partition **out);
int swe_partition_destroy(swe_partition *p);
/* Part `part`: owned cells [owned_begin, owned_end) and the list sizes. */
int swe_partition_info(const swe_partition *p, int part, int64_t *owned_begin, int64_t *owned_end,
                       int64_t *n_halo1, int64_t *n_halo2, int64_t *n_boundary);
/* The sorted cell lists of part `part` (caller-allocated, sized by
 * swe_partition_info; any pointer may be NULL). */
int swe_partition_export(const swe_partition *p, int part, int32_t *halo1, int32_t *halo2, int32_t *boundary);
/* Step the state with the boundary-first schedule of a partition of its mesh
 * (NULL: the plain schedule): every step updates all parts' boundary cells
 * first, then packs every part's halo (halo1 then halo2, from the new state)
 * into exchange buffers on a second stream while it updates the interior
 * cells.  The results are those of the plain schedule, bit for bit.  Needs
 * the split kernels and Euler steps (SWE_ERR_ARG otherwise); the partition
 * may be destroyed afterwards. */
int swe_set_partition(swe_state *s, const swe_partition *p);
/* The exchange buffer of part `part` after the last step: the state of its
 * halo1 then halo2 cells, as FP64 host arrays (synchronises). */
int swe_halo_get(swe_state *s, int part, double *h, double *hu, double *hv);

/* ---- Ensemble ---------------------------------------------------------- */

/* Group independent states so that one batched launch per step (two for the
 * split kernels) advances all of them, each with its own CFL time step, its
 * own boundary values and its own time (the batched form of running many
 * scenarios; cf. the paper's one-sub-domain-per-GPU layout, Sec. 6.4).
 * Members must share precision, scheme, hr_order, Euler time stepping, kernel, block,
 * stream and step phase (steps taken mod 6; freshly initialised states do).
 * Each state may appear once (SWE_ERR_ARG otherwise).  Members stay owned by
 * the caller, must outlive the ensemble, and can be queried (swe_get_state,
 * swe_mass, swe_time) as usual. */
int swe_ensemble_create(swe_state *const *members, int n_members, swe_ensemble **out);
int swe_ensemble_destroy(swe_ensemble *e);
/* Advance every member n_steps explicit steps, each with its own CFL time
 * step dt = cfl * r_min / max_wet(sqrt(g h)+|u|) of Sec. 6.1 (asynchronous). */
int swe_ensemble_step(swe_ensemble *e, int n_steps, double cfl);
/* Wait for the members' stream and return the first member error, if any. */
int swe_ensemble_sync(swe_ensemble *e);
/* Autotune the members' common kernel configuration on the whole ensemble
 * (as swe_autotune; meshes[i] is member i's mesh, NULL for split kernels only). */
int swe_ensemble_autotune(swe_ensemble *e, const swe_mesh *const *meshes, int trial_steps, double cfl,
                          int *kernel, int *block, double *ms_per_step);

#ifdef __cplusplus
}
#endif
#endif
