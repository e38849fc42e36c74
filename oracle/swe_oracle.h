/*
 * swe_oracle.h -- plain FP64 CPU oracle for the explicit finite-volume step of
 * the 2D shallow-water equations on triangles (Delmas & Soulaimani,
 * arXiv 2307.16758, Section 6).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no source with the CUDA path.
 *
 * Every array is in the caller's (original) cell order.  Cell ids are int32.
 * Boundary tags: tag = type + 4*group with type 0 WALL, 1 OPEN (transmissive),
 * 2 INFLOW (group selects the discharge), 3 LEVEL (group selects the level).
 */
#ifndef SWE_ORACLE_H
#define SWE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct om_mesh om_mesh;

/* Build the mesh: orientation, edge adjacency, boundary tags, geometry.
 * Returns 0 or a negative error code (-2 bad mesh). */
int om_mesh_build(const double *node_xy, int64_t n_nodes,
                  const int32_t *tri, int64_t n_tri,
                  const int32_t *bnd_edges, const int32_t *bnd_tag, int64_t n_bnd,
                  const int32_t *cut_edges, int64_t n_cut, om_mesh **out);
void om_mesh_free(om_mesh *m);
int64_t om_mesh_ncells(const om_mesh *m);

/* Export in original order.  Any pointer may be NULL.
 *  tri[n][3] oriented CCW; nbr[n][3] neighbour id or -1 on a boundary;
 *  nbr_edge[n][3] local edge index in the neighbour (-1 on a boundary);
 *  btag[n][3] boundary tag (-1 on interior edges);
 *  lnx,lny[n][3] outward normal scaled by the edge length;
 *  area[n], cx[n], cy[n], rin[n] inscribed radius;
 *  dx,dy[n][3] centroid offset to the neighbour (0 on a boundary). */
int om_mesh_export(const om_mesh *m, int32_t *tri, int32_t *nbr, int32_t *nbr_edge,
                   int32_t *btag, double *lnx, double *lny, double *area,
                   double *cx, double *cy, double *rin, double *dx, double *dy);

/* Locality orders: perm[new] = old.  Morton: 21-bit per axis of the centroid
 * in the square box of the centroids, stable by old id.  RCM: breadth-first
 * from the lowest-degree cell (ties: lowest id), neighbours by (degree, id),
 * restarted per component, then reversed. */
int om_morton_order(const om_mesh *m, int32_t *perm);
int om_rcm_order(const om_mesh *m, int32_t *perm);

/* Options of one run. */
typedef struct {
    int scheme;        /* 0 first-order HLLC, 1 MUSCL (LSQ + Barth-Jespersen) + HLLC, 2 WAF,
                          3 the paper's MUSCL (edge-upwind slopes, beta-limiter) + HLLC */
    int time_scheme;   /* 0 explicit Euler, 1 Heun (SSP-RK2, order studies only) */
    int waf_limiter;   /* 0 SUPERBEE, 1 phi = 1 (no limiting), 2 phi = 0, 3 MINBEE, 4 van Leer */
    int threads;       /* OpenMP threads (0 = default); results do not depend on it */
    double g;
    double h_eps;      /* velocity desingularisation / dry threshold [m] */
    double r_eps;      /* WAF: |local change| below r_eps*max(1,|q|) gives r = 0 */
    double cfl;
    int cfl_local;     /* 0: dt = CFL min_i r_i / max_wet s_i (Sec. 6.1, global form);
                          1: dt = CFL min over wet cells of r_i / s_i (per-cell form) */
    double beta;       /* scheme 3: limiter parameter (1 MINBEE, 2 SUPERBEE) */
    int hr_order;      /* scheme 1: 1 hydrostatic reconstruction on the cell bed (R6),
                          2 second order with a linear bed in each cell (R16) */
    int waf_surface;   /* scheme 2: 0 the ratio r_L, r_R on the depth h (Sec. 6.2.2),
                          1 on the free surface eta (R17) */
} om_opts;

/* Advance n_steps.  h,hu,hv are updated in place.  dt_given (length n_steps)
 * replays a time-step sequence; NULL uses the CFL rule.  dt_used may be NULL.
 * q_in[group] is the inflow discharge in m^3/s, spread per unit length over
 * the INFLOW edges of that group; level[group] is the LEVEL free surface.
 * diag[0] += simulated time, diag[1] += mass added by clipping negative depths,
 * diag[2] += net mass that entered through the boundary (m^3).
 * Returns 0, -4 if no cell is wet under the CFL rule, -5 on a non-finite value. */
int om_run(const om_mesh *m, const om_opts *o,
           const double *z, const double *nman,
           const double *q_in, int n_in, const double *level, int n_level,
           double *h, double *hu, double *hv, int n_steps,
           const double *dt_given, double *dt_used, double *diag);

/* Limited (and unlimited, if non-NULL) gradients of (eta, u, v):
 * grad[n][6] = (deta/dx, deta/dy, du/dx, du/dy, dv/dx, dv/dy). */
int om_gradients(const om_mesh *m, const om_opts *o, const double *z,
                 const double *h, const double *hu, const double *hv,
                 double *grad_limited, double *grad_unlimited);

/* One interior edge in the rotated frame (normal pointing from L to R).
 * in[10] = (hface_L, hstar_L, hcell_L, uL, vL, hface_R, hstar_R, hcell_R, uR, vR)
 * with u the normal and v the tangential velocity; for WAF also
 * waf[8] = (dt_over_dx, hupw_L, hupw_R, vupw_L, vupw_R, hcell_L, hcell_R, unused) (NULL for HLLC).
 * out[4] = (M, P_L, P_R, T): mass flux, the normal momentum flux seen by each
 * side (hydrostatic-reconstruction form, cell-centre pressure removed) and
 * the tangential momentum flux. */
int om_edge_flux(const om_opts *o, const double *in, const double *waf, double *out);

/* The limited slope of the paper's MUSCL (Sec. 6.2.3) from the slope "up"
 * behind the cell and the slope "dn" towards the other side of the edge:
 * dn > 0: max(0, min(beta up, dn), min(up, beta dn));
 * dn < 0: min(0, max(beta up, dn), max(up, beta dn)); dn = 0: 0. */
double om_beta_limit(double beta, double up, double dn);

/* Sum of area*h in FP64 with Neumaier compensation, in cell order. */
double om_mass(const om_mesh *m, const double *h);

#ifdef __cplusplus
}
#endif
#endif
