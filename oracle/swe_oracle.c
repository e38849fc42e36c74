/*
 * swe_oracle.c -- plain FP64 CPU oracle for the explicit finite-volume
 * shallow-water step of Delmas & Soulaimani (arXiv 2307.16758), Section 6.
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by the tests, by the smoke check
 * and by the benchmark's CPU-baseline leg; the product library never links,
 * includes or calls it, and it shares no code with the CUDA path.
 *
 * It is written to be read against the paper, not to be fast: one loop per
 * step of the algorithm, in the order of Sec. 6.1-6.2, FP64 throughout.
 * Parity status of each function (what pins it) is listed in the tests and in
 * the design notes; every function here is pinned (nothing is "parity
 * unpinned").
 *
 * Readings of passages the paper leaves open (the numbering is the one used
 * in the design notes):
 *  R1  p_k of the HLL speed estimate (Sec. 6.2.1) is dimensionally garbled;
 *      it is read as p_k = sqrt(h*(h*+h_k)/2)/h_k for h* > h_k, else 1.
 *  R1b two-rarefaction h*: the bracket is clipped at 0 before squaring
 *      (a vacuum forms when it is negative).
 *  R2  HLLC third component (Sec. 6.2.1): the upwind tangential velocity is
 *      v_L when S* >= 0 and v_R otherwise (the printed cases are swapped;
 *      the WAF passive weights of Sec. 6.2.2 agree with this reading).
 *  R3  WAF limited weights (Sec. 6.2.2): Toro's TVD form,
 *      w_L=(1+sgn(c_L)A_L)/2, w_LR=(sgn(c_R)A_R-sgn(c_L)A_L)/2,
 *      w_R=(1-sgn(c_R)A_R)/2, w_L*=(1+sgn(c*)A*)/2, w_R*=(1-sgn(c*)A*)/2,
 *      sgn(0)=+1.  The weights sum to 1; phi=1 gives the unlimited weights.
 *      A(r,c) = 1 - (1-|c|) phi(r) with phi a classical flux limiter: SUPERBEE
 *      (the paper's choice, its branch table) or, as options, MINBEE
 *      phi = max(0, min(1, r)) and van Leer phi = (r + |r|)/(1 + |r|).
 *  R4  WAF on triangles: dx = |c_R - c_L|; r = 0 when the local change is
 *      below r_eps*max(1,|q_L|,|q_R|); a missing upwind cell uses the cell
 *      itself; boundary edges use the first-order HLLC boundary flux.  The
 *      ratios' quantity q for the nonlinear waves: the paper takes the depth
 *      of the Riemann problem; with the hydrostatic reconstruction (Sec.
 *      6.2.3) that problem is posed on h*_s = eta_s - z_f, whose differences
 *      are those of the free surface eta (z_f is one value per edge), so the
 *      ratios are taken on eta (default; on a flat bed it is the cell depth's
 *      ratio exactly).  The cell depth h itself remains an option (R17).
 *  R5  Dry sides of the Riemann problem (h* <= h_eps): Toro's dry-bed speeds;
 *      both sides dry gives a zero numerical flux.
 *  R6  Bed and hydrostatic reconstruction: piecewise-constant bed per cell;
 *      Audusse et al. (2004) at each edge, z_f = max(z_L,z_R),
 *      h*_s = max(0, eta_s - z_f).  Each side's flux is written in
 *      flux-difference form (F - G(U*_s)) and the cell-centre pressure
 *      g/2 h_i^2 n (which sums to zero round a closed triangle) is removed, so
 *      that a lake at rest is preserved bit for bit.
 *  R7  Inflow (Sec. 6.1): mass flux -q enters the cell; normal momentum flux
 *      q^2/h + g h^2/2 (the q^2/h term dropped when h <= h_eps); q = Q / total
 *      length of the inflow edges of the group.
 *  R8  Fixed-level boundary (not in the paper): ghost depth
 *      max(0, eta_out - z_i), ghost velocity = inner velocity, HLLC.
 *  R9  Manning friction (named in Sec. 6.1, no formula): point-implicit
 *      (hu,hv) <- (hu,hv) / (1 + dt g n^2 |u| h^(-4/3)) after the flux update.
 *  R10 Explicit Euler (Sec. 6.1) is the time scheme; Heun is offered only for
 *      the convergence-order study.
 *  R11 CFL (Sec. 6.1): dt = CFL * min_i r_i / max_wet(sqrt(g h)+|u|); as an
 *      option, per cell: dt = CFL * min over wet cells of r_i / s_i.
 *  R12 Each interior edge is evaluated in one canonical orientation (L = the
 *      cell with the lower original id), so both cells see the same flux.
 *  R13 MUSCL: unweighted least-squares gradients of (eta,u,v) over the face
 *      neighbours, Barth-Jespersen limiting at the three edge midpoints; zero
 *      gradient if the cell or a neighbour is dry or the 2x2 system is
 *      singular.  u = hu/h if h > h_eps else 0.  Depth below 0 after the
 *      update is set to 0 and the mass that adds is recorded; momentum is
 *      zeroed where h <= h_eps.
 *  R16 Second-order hydrostatic reconstruction (the paper's future work,
 *      Sec. 7; scheme 1 with hr_order 2): h is reconstructed like eta (LSQ +
 *      Barth-Jespersen, zero gradient next to a dry cell), the bed at a face
 *      is z_f = z_i + (grad eta - grad h).(m_k - c_i) (a linear bed in the
 *      cell), the Riemann problem takes z_f* = max of the two face beds, and
 *      the cell's own pressure term of a face is g/2 (h_f + h_i)(eta_f - eta_i)
 *      (wet face) -- the first-order correction of R6 plus the centred bed
 *      source g (h_f + h_i)/2 (z_f - z_i) L n of that face.
 *  R15 The paper's own MUSCL (Sec. 6.2.3, scheme 3): the reconstructed
 *      variables are (eta, u, v), as in R13; x_RL is the edge midpoint and
 *      distances are Euclidean; the upwind value of a side is the mean over
 *      its cell's two other neighbours and sits at the mean of their
 *      centroids (a missing neighbour stands in with the cell, as in R4); an
 *      upwind distance of 0 (no other neighbour) gives an upwind slope of 0;
 *      the limited slope is 0 when its condition difference is 0, and when
 *      the side's cell, the other cell or one of its upwind cells is dry;
 *      boundary edges use the cell-centre values.  HR, Riemann flux and
 *      update are those of the other schemes.
 *  R17 WAF ratio on the cell depth h (an option; the default of R4 takes
 *      eta): over a steep bed h varies with the bed even at rest, the limiter
 *      reacts to the bathymetry, and on the river workload WAF-SUPERBEE grows
 *      spurious speeds next to the inflow until it blows up (R14).
 *  R18 WAF weights need a wet star region between S_L and S_R.  Where the
 *      Riemann problem has none -- a dry side (a cell with h <= h_eps, or a
 *      reconstructed depth h* <= h_eps; with first-order faces h* <= h, so
 *      the cell test only settles rounding at the threshold), or two
 *      rarefactions that open a dry gap (u_R - u_L >= 2(a_L + a_R), the
 *      vacuum condition) -- the paper's weights are undefined and the edge
 *      takes A = 1 for all three waves, i.e. its HLLC flux.  Without this the
 *      ratio on eta at such an edge is ill-conditioned (the waves carry a large
 *      velocity jump over a tiny change of eta), SUPERBEE switches between
 *      A = 1 and A = 2|c| - 1 from one step to the next, and the mass flux
 *      alternates between about G(U_L) and G(U_R) (R14).
 */
#include "swe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct om_mesh {
    int64_t n;          /* cells */
    int32_t *tri;       /* [n][3] oriented counter-clockwise */
    int32_t *nbr;       /* [n][3] neighbour or -1 */
    int32_t *nbr_edge;  /* [n][3] local edge index inside the neighbour or -1 */
    int32_t *btag;      /* [n][3] boundary tag or -1 */
    double *lnx, *lny;  /* [n][3] outward normal times edge length */
    double *len;        /* [n][3] edge length */
    double *mx, *my;    /* [n][3] edge midpoint minus centroid */
    double *area, *cx, *cy, *rin;
};

enum { BC_WALL = 0, BC_OPEN = 1, BC_INFLOW = 2, BC_LEVEL = 3 };

/* ------------------------------------------------------------------------ */
/* Mesh                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t lo, hi, cell, k; } edge_rec;
typedef struct { int32_t lo, hi, tag; } key_rec;

static int cmp_edge(const void *a, const void *b)
{
    const edge_rec *x = a, *y = b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return x->k < y->k ? -1 : (x->k > y->k);
}

static int cmp_key(const void *a, const void *b)
{
    const key_rec *x = a, *y = b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    return x->hi < y->hi ? -1 : (x->hi > y->hi);
}

static const key_rec *find_key(const key_rec *keys, int64_t n, int32_t lo, int32_t hi)
{
    key_rec probe = {lo, hi, 0};
    return bsearch(&probe, keys, (size_t)n, sizeof(key_rec), cmp_key);
}

void om_mesh_free(om_mesh *m)
{
    if (!m) return;
    free(m->tri); free(m->nbr); free(m->nbr_edge); free(m->btag);
    free(m->lnx); free(m->lny); free(m->len); free(m->mx); free(m->my);
    free(m->area); free(m->cx); free(m->cy); free(m->rin);
    free(m);
}

int64_t om_mesh_ncells(const om_mesh *m) { return m ? m->n : 0; }

int om_mesh_build(const double *xy, int64_t n_nodes, const int32_t *tri_in, int64_t n,
                  const int32_t *bnd, const int32_t *bnd_tag, int64_t n_bnd,
                  const int32_t *cut, int64_t n_cut, om_mesh **out)
{
    *out = NULL;
    if (n <= 0 || n_nodes < 3 || n > (1LL << 28)) return -1;
    om_mesh *m = calloc(1, sizeof(om_mesh));
    m->n = n;
    m->tri = malloc(sizeof(int32_t) * 3 * n);
    m->nbr = malloc(sizeof(int32_t) * 3 * n);
    m->nbr_edge = malloc(sizeof(int32_t) * 3 * n);
    m->btag = malloc(sizeof(int32_t) * 3 * n);
    m->lnx = malloc(sizeof(double) * 3 * n);
    m->lny = malloc(sizeof(double) * 3 * n);
    m->len = malloc(sizeof(double) * 3 * n);
    m->mx = malloc(sizeof(double) * 3 * n);
    m->my = malloc(sizeof(double) * 3 * n);
    m->area = malloc(sizeof(double) * n);
    m->cx = malloc(sizeof(double) * n);
    m->cy = malloc(sizeof(double) * n);
    m->rin = malloc(sizeof(double) * n);

    /* Orientation: counter-clockwise, so that (dy, -dx) of each edge points out. */
    for (int64_t i = 0; i < n; i++) {
        int32_t a = tri_in[3 * i], b = tri_in[3 * i + 1], c = tri_in[3 * i + 2];
        if (a < 0 || b < 0 || c < 0 || a >= n_nodes || b >= n_nodes || c >= n_nodes) goto bad;
        double cross = (xy[2 * b] - xy[2 * a]) * (xy[2 * c + 1] - xy[2 * a + 1])
                     - (xy[2 * b + 1] - xy[2 * a + 1]) * (xy[2 * c] - xy[2 * a]);
        if (cross == 0.0) goto bad;
        if (cross < 0.0) { int32_t t = b; b = c; c = t; }
        m->tri[3 * i] = a; m->tri[3 * i + 1] = b; m->tri[3 * i + 2] = c;
        m->area[i] = 0.5 * fabs(cross);
    }

    /* Adjacency: every local edge keyed by its unordered node pair, sorted;
     * a key seen twice is an interior edge, once a boundary edge. */
    edge_rec *e = malloc(sizeof(edge_rec) * 3 * n);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            int32_t p = m->tri[3 * i + k], q = m->tri[3 * i + (k + 1) % 3];
            edge_rec r = {p < q ? p : q, p < q ? q : p, (int32_t)i, k};
            e[3 * i + k] = r;
        }
    qsort(e, (size_t)(3 * n), sizeof(edge_rec), cmp_edge);
    for (int64_t i = 0; i < 3 * n; i++) { m->nbr[i] = -1; m->nbr_edge[i] = -1; m->btag[i] = -1; }
    for (int64_t s = 0; s < 3 * n;) {
        int64_t t = s + 1;
        while (t < 3 * n && e[t].lo == e[s].lo && e[t].hi == e[s].hi) t++;
        if (t - s > 2) { free(e); goto bad; }
        if (t - s == 2) {
            edge_rec x = e[s], y = e[s + 1];
            /* both cells counter-clockwise: they must walk the edge in opposite directions */
            if (m->tri[3 * x.cell + x.k] == m->tri[3 * y.cell + y.k]) { free(e); goto bad; }
            m->nbr[3 * x.cell + x.k] = y.cell; m->nbr_edge[3 * x.cell + x.k] = y.k;
            m->nbr[3 * y.cell + y.k] = x.cell; m->nbr_edge[3 * y.cell + y.k] = x.k;
        }
        s = t;
    }
    free(e);

    /* Internal walls (cut edges): both sides become walls. */
    if (n_cut > 0) {
        key_rec *ck = malloc(sizeof(key_rec) * n_cut);
        for (int64_t i = 0; i < n_cut; i++) {
            int32_t p = cut[2 * i], q = cut[2 * i + 1];
            key_rec r = {p < q ? p : q, p < q ? q : p, 0};
            ck[i] = r;
        }
        qsort(ck, (size_t)n_cut, sizeof(key_rec), cmp_key);
        int64_t found = 0;
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < 3; k++) {
                if (m->nbr[3 * i + k] < 0) continue;
                int32_t p = m->tri[3 * i + k], q = m->tri[3 * i + (k + 1) % 3];
                if (find_key(ck, n_cut, p < q ? p : q, p < q ? q : p)) {
                    m->nbr[3 * i + k] = -1; m->nbr_edge[3 * i + k] = -1;
                    m->btag[3 * i + k] = BC_WALL;
                    found++;
                }
            }
        free(ck);
        if (found != 2 * n_cut) goto bad;   /* each cut edge must be an interior edge, listed once */
    }

    /* Boundary tags: listed edges take their tag, the others are walls. */
    key_rec *bk = NULL;
    if (n_bnd > 0) {
        bk = malloc(sizeof(key_rec) * n_bnd);
        for (int64_t i = 0; i < n_bnd; i++) {
            int32_t p = bnd[2 * i], q = bnd[2 * i + 1];
            if (bnd_tag[i] < 0) { free(bk); goto bad; }
            key_rec r = {p < q ? p : q, p < q ? q : p, bnd_tag[i]};
            bk[i] = r;
        }
        qsort(bk, (size_t)n_bnd, sizeof(key_rec), cmp_key);
        for (int64_t i = 1; i < n_bnd; i++)
            if (bk[i].lo == bk[i - 1].lo && bk[i].hi == bk[i - 1].hi) { free(bk); goto bad; }
    }
    int64_t matched = 0;
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            if (m->nbr[3 * i + k] >= 0 || m->btag[3 * i + k] >= 0) continue;
            int32_t p = m->tri[3 * i + k], q = m->tri[3 * i + (k + 1) % 3];
            const key_rec *f = bk ? find_key(bk, n_bnd, p < q ? p : q, p < q ? q : p) : NULL;
            m->btag[3 * i + k] = f ? f->tag : BC_WALL;
            matched += f != NULL;
        }
    free(bk);
    if (matched != n_bnd) goto bad;   /* a listed boundary edge is not on the boundary */

    /* Geometry (Sec. 6.1: |Omega_i|, L_ij, n_ij; inscribed radius R_L of the CFL rule). */
    for (int64_t i = 0; i < n; i++) {
        const int32_t *t = &m->tri[3 * i];
        double x0 = xy[2 * t[0]], y0 = xy[2 * t[0] + 1];
        double x1 = xy[2 * t[1]], y1 = xy[2 * t[1] + 1];
        double x2 = xy[2 * t[2]], y2 = xy[2 * t[2] + 1];
        m->cx[i] = (x0 + x1 + x2) / 3.0;
        m->cy[i] = (y0 + y1 + y2) / 3.0;
        double px[3] = {x0, x1, x2}, py[3] = {y0, y1, y2};
        double perim = 0.0;
        for (int k = 0; k < 3; k++) {
            int k1 = (k + 1) % 3;
            m->lnx[3 * i + k] = py[k1] - py[k];
            m->lny[3 * i + k] = -(px[k1] - px[k]);
            m->len[3 * i + k] = sqrt(m->lnx[3 * i + k] * m->lnx[3 * i + k] + m->lny[3 * i + k] * m->lny[3 * i + k]);
            perim += m->len[3 * i + k];
            m->mx[3 * i + k] = 0.5 * (px[k] + px[k1]) - m->cx[i];
            m->my[3 * i + k] = 0.5 * (py[k] + py[k1]) - m->cy[i];
        }
        m->rin[i] = 2.0 * m->area[i] / perim;
    }
    *out = m;
    return 0;
bad:
    om_mesh_free(m);
    return -2;
}

int om_mesh_export(const om_mesh *m, int32_t *tri, int32_t *nbr, int32_t *nbr_edge,
                   int32_t *btag, double *lnx, double *lny, double *area,
                   double *cx, double *cy, double *rin, double *dx, double *dy)
{
    int64_t n = m->n;
    if (tri) memcpy(tri, m->tri, sizeof(int32_t) * 3 * n);
    if (nbr) memcpy(nbr, m->nbr, sizeof(int32_t) * 3 * n);
    if (nbr_edge) memcpy(nbr_edge, m->nbr_edge, sizeof(int32_t) * 3 * n);
    if (btag) memcpy(btag, m->btag, sizeof(int32_t) * 3 * n);
    if (lnx) memcpy(lnx, m->lnx, sizeof(double) * 3 * n);
    if (lny) memcpy(lny, m->lny, sizeof(double) * 3 * n);
    if (area) memcpy(area, m->area, sizeof(double) * n);
    if (cx) memcpy(cx, m->cx, sizeof(double) * n);
    if (cy) memcpy(cy, m->cy, sizeof(double) * n);
    if (rin) memcpy(rin, m->rin, sizeof(double) * n);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            int32_t j = m->nbr[3 * i + k];
            if (dx) dx[3 * i + k] = j >= 0 ? m->cx[j] - m->cx[i] : 0.0;
            if (dy) dy[3 * i + k] = j >= 0 ? m->cy[j] - m->cy[i] : 0.0;
        }
    return 0;
}

/* ---- locality orders ---------------------------------------------------- */

typedef struct { uint64_t key; int32_t id; } sort_rec;

static int cmp_sort(const void *a, const void *b)
{
    const sort_rec *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

int om_morton_order(const om_mesh *m, int32_t *perm)
{
    int64_t n = m->n;
    double xmin = m->cx[0], xmax = m->cx[0], ymin = m->cy[0], ymax = m->cy[0];
    for (int64_t i = 1; i < n; i++) {
        if (m->cx[i] < xmin) xmin = m->cx[i];
        if (m->cx[i] > xmax) xmax = m->cx[i];
        if (m->cy[i] < ymin) ymin = m->cy[i];
        if (m->cy[i] > ymax) ymax = m->cy[i];
    }
    double ext = xmax - xmin > ymax - ymin ? xmax - xmin : ymax - ymin;
    if (!(ext > 0.0)) ext = 1.0;
    double s = 2097151.0 / ext;
    sort_rec *r = malloc(sizeof(sort_rec) * n);
    for (int64_t i = 0; i < n; i++) {
        double fx = floor((m->cx[i] - xmin) * s), fy = floor((m->cy[i] - ymin) * s);
        if (fx < 0) fx = 0;
        if (fx > 2097151.0) fx = 2097151.0;
        if (fy < 0) fy = 0;
        if (fy > 2097151.0) fy = 2097151.0;
        uint64_t qx = (uint64_t)fx, qy = (uint64_t)fy, key = 0;
        for (int b = 0; b < 21; b++) {
            key |= ((qx >> b) & 1ULL) << (2 * b);
            key |= ((qy >> b) & 1ULL) << (2 * b + 1);
        }
        r[i].key = key; r[i].id = (int32_t)i;
    }
    qsort(r, (size_t)n, sizeof(sort_rec), cmp_sort);
    for (int64_t i = 0; i < n; i++) perm[i] = r[i].id;
    free(r);
    return 0;
}

int om_rcm_order(const om_mesh *m, int32_t *perm)
{
    int64_t n = m->n;
    int *deg = calloc((size_t)n, sizeof(int));
    char *seen = calloc((size_t)n, 1);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) deg[i] += m->nbr[3 * i + k] >= 0;
    /* candidate starts sorted by (degree, id) */
    sort_rec *start = malloc(sizeof(sort_rec) * n);
    for (int64_t i = 0; i < n; i++) { start[i].key = (uint64_t)deg[i]; start[i].id = (int32_t)i; }
    qsort(start, (size_t)n, sizeof(sort_rec), cmp_sort);
    int64_t head = 0, tail = 0, sp = 0;
    while (tail < n) {
        while (seen[start[sp].id]) sp++;
        perm[tail++] = start[sp].id;
        seen[start[sp].id] = 1;
        while (head < tail) {
            int32_t c = perm[head++];
            sort_rec nb[3];
            int cnt = 0;
            for (int k = 0; k < 3; k++) {
                int32_t j = m->nbr[3 * c + k];
                if (j >= 0 && !seen[j]) { nb[cnt].key = (uint64_t)deg[j]; nb[cnt].id = j; cnt++; }
            }
            qsort(nb, (size_t)cnt, sizeof(sort_rec), cmp_sort);
            for (int q = 0; q < cnt; q++) {
                if (seen[nb[q].id]) continue;
                seen[nb[q].id] = 1;
                perm[tail++] = nb[q].id;
            }
        }
    }
    for (int64_t i = 0; i < n / 2; i++) { int32_t t = perm[i]; perm[i] = perm[n - 1 - i]; perm[n - 1 - i] = t; }
    free(deg); free(seen); free(start);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Riemann problem in the rotated frame (Sec. 6.2.1 and 5.2.2)               */
/* ------------------------------------------------------------------------ */

/* Wave-speed estimates S_L, S_R of Sec. 6.2.1 with readings R1, R1b, R5. */
static void hll_speeds(double g, double h_eps, double hL, double uL, double hR, double uR,
                       double *SL, double *SR)
{
    double aL = sqrt(g * hL), aR = sqrt(g * hR);
    if (hL <= h_eps) {            /* dry left bed: Toro's dry-bed speeds */
        *SL = uR - 2.0 * aR;
        *SR = uR + aR;
        return;
    }
    if (hR <= h_eps) {
        *SL = uL - aL;
        *SR = uL + 2.0 * aL;
        return;
    }
    /* first guess h*_0, then two-rarefaction or two-shock estimate */
    double h0 = (hL + hR) / 2.0 - (uR - uL) * (hL + hR) / (4.0 * (aR + aL));
    double hs;
    if (h0 <= (hL < hR ? hL : hR)) {
        double br = (aR + aL) / 2.0 + (uL - uR) / 4.0;
        if (br < 0.0) br = 0.0;
        hs = br * br / g;
    } else {
        double gL = sqrt(g * (h0 + hL) / (2.0 * h0 * hL));
        double gR = sqrt(g * (h0 + hR) / (2.0 * h0 * hR));
        hs = (hL * gL + hR * gR + uL - uR) / (gL + gR);
    }
    double pL = hs > hL ? sqrt(hs * (hs + hL) / 2.0) / hL : 1.0;
    double pR = hs > hR ? sqrt(hs * (hs + hR) / 2.0) / hR : 1.0;
    *SL = uL - aL * pL;
    *SR = uR + aR * pR;
}

/* WAF limiter A(r,c) of Sec. 6.2.2: SUPERBEE's branch table as printed, the
 * phi = 1 / phi = 0 variants, and A = 1 - (1-|c|) phi(r) for MINBEE and van
 * Leer (R3). */
static double waf_A(int lim, double r, double c)
{
    double ac = fabs(c);
    if (lim == 1) return ac;      /* phi = 1: unlimited weights */
    if (lim == 2) return 1.0;     /* phi = 0: upwind */
    if (lim == 3) return 1.0 - (1.0 - ac) * (r <= 0.0 ? 0.0 : (r < 1.0 ? r : 1.0));
    if (lim == 4) return 1.0 - (1.0 - ac) * (r <= 0.0 ? 0.0 : 2.0 * r / (1.0 + r));
    if (r <= 0.0) return 1.0;
    if (r <= 0.5) return 1.0 - 2.0 * (1.0 - ac) * r;
    if (r <= 1.0) return ac;
    if (r <= 2.0) return 1.0 - (1.0 - ac) * r;
    return 2.0 * ac - 1.0;
}

static double waf_ratio(double r_eps, double upw, double qL, double qR)
{
    double loc = qR - qL;
    double sc = fabs(qL) > fabs(qR) ? fabs(qL) : fabs(qR);
    if (sc < 1.0) sc = 1.0;
    if (fabs(loc) <= r_eps * sc) return 0.0;
    return upw / loc;
}

/* The edge flux; see om_edge_flux in the header for in/waf/out.
 * For each side s the numerical flux is written as G(U*_s) + D_s with
 * D_s = F - G(U*_s):  HLL (three branches of Sec. 6.2.1) gives, in the star
 * region, D_L = S_L (S_R dU - dG)/(S_R - S_L) and D_R = S_R (S_L dU - dG)/(S_R - S_L),
 * which is the printed star flux minus G_L or G_R rearranged (R6). */
static void edge_flux(const om_opts *o, int scheme, const double *in, const double *waf, double *out)
{
    const double g = o->g, h_eps = o->h_eps;
    double hfL = in[0], hsL = in[1], hcL = in[2], uL = in[3], vL = in[4];
    double hfR = in[5], hsR = in[6], hcR = in[7], uR = in[8], vR = in[9];
    /* physical fluxes G(U) in the rotated frame, first two components */
    double GL1 = hsL * uL, GL2 = hsL * uL * uL + 0.5 * g * hsL * hsL;
    double GR1 = hsR * uR, GR2 = hsR * uR * uR + 0.5 * g * hsR * hsR;
    double dU1 = hsR - hsL, dU2 = hsR * uR - hsL * uL;
    double dG1 = GR1 - GL1, dG2 = GR2 - GL2;
    double M, T, DL1, DL2, DR1, DR2;

    if (hsL <= h_eps && hsR <= h_eps) {      /* R5: both sides dry, zero flux */
        M = 0.0; T = 0.0;
        DL1 = -GL1; DL2 = -GL2; DR1 = -GR1; DR2 = -GR2;
    } else {
        double SL, SR;
        hll_speeds(g, h_eps, hsL, uL, hsR, uR, &SL, &SR);
        /* S* of Sec. 6.2.1 */
        double num = SL * hsR * (uR - SR) - SR * hsL * (uL - SL);
        double den = hsR * (uR - SR) - hsL * (uL - SL);
        double Ss = den != 0.0 ? num / den : 0.0;
        /* HLL, Sec. 6.2.1, as differences to G_L and G_R */
        double hL1, hL2, hR1, hR2;
        if (SL >= 0.0) {
            hL1 = 0.0; hL2 = 0.0; hR1 = -dG1; hR2 = -dG2;
        } else if (SR <= 0.0) {
            hL1 = dG1; hL2 = dG2; hR1 = 0.0; hR2 = 0.0;
        } else {
            double w = SR - SL;
            hL1 = SL * (SR * dU1 - dG1) / w; hL2 = SL * (SR * dU2 - dG2) / w;
            hR1 = SR * (SL * dU1 - dG1) / w; hR2 = SR * (SL * dU2 - dG2) / w;
        }
        if (scheme != 2 || waf == NULL) {
            /* HLLC: components 1 and 2 are HLL; the third is G1 times the upwind v (R2) */
            DL1 = hL1; DL2 = hL2; DR1 = hR1; DR2 = hR2;
            M = GL1 + DL1;
            if (SR <= 0.0 && !(SL >= 0.0)) M = GR1;
            T = M * (Ss >= 0.0 ? vL : vR);
        } else {
            /* WAF of Sec. 6.2.2 with the TVD weights of reading R3 */
            double dtdx = waf[0];
            double hupL = waf[1], hupR = waf[2], vupL = waf[3], vupR = waf[4];
            double hcl = waf[5], hcr = waf[6];
            double cL = SL * dtdx, cR = SR * dtdx, cs = Ss * dtdx;
            double rL = waf_ratio(o->r_eps, SL >= 0.0 ? hcl - hupL : hupR - hcr, hcl, hcr);
            double rR = waf_ratio(o->r_eps, SR >= 0.0 ? hcl - hupL : hupR - hcr, hcl, hcr);
            double rs = waf_ratio(o->r_eps, Ss >= 0.0 ? vL - vupL : vupR - vR, vL, vR);
            double sgL = cL >= 0.0 ? 1.0 : -1.0, sgR = cR >= 0.0 ? 1.0 : -1.0, sgs = cs >= 0.0 ? 1.0 : -1.0;
            double AL = waf_A(o->waf_limiter, rL, cL);
            double AR = waf_A(o->waf_limiter, rR, cR);
            double As = waf_A(o->waf_limiter, rs, cs);
            /* R18: no wet star region (a dry side: a dry cell or a dry reconstructed
             * depth; or the vacuum condition) */
            if (hsL <= h_eps || hsR <= h_eps || hcL <= h_eps || hcR <= h_eps ||
                uR - uL >= 2.0 * (sqrt(g * hsL) + sqrt(g * hsR))) {
                AL = 1.0; AR = 1.0; As = 1.0;
            }
            double wL = (1.0 + sgL * AL) / 2.0;
            double wLR = (sgR * AR - sgL * AL) / 2.0;
            double wR = (1.0 - sgR * AR) / 2.0;
            double wLs = (1.0 + sgs * As) / 2.0, wRs = (1.0 - sgs * As) / 2.0;
            /* F = wL G_L + wLR F_HLL + wR G_R, written as differences to G_L / G_R */
            DL1 = wLR * hL1 + wR * dG1; DL2 = wLR * hL2 + wR * dG2;
            DR1 = -wL * dG1 + wLR * hR1; DR2 = -wL * dG2 + wLR * hR2;
            M = GL1 + DL1;
            T = (wLs * vL + wRs * vR) * M;
        }
    }
    (void)DR1;
    /* normal momentum seen by each side: advective part of G(U*_s) + D_s +
     * g/2 (hface_s^2 - hcell_s^2)  (Audusse reconstruction, R6) */
    out[0] = M;
    out[1] = hsL * uL * uL + DL2 + 0.5 * g * (hfL - hcL) * (hfL + hcL);
    out[2] = hsR * uR * uR + DR2 + 0.5 * g * (hfR - hcR) * (hfR + hcR);
    out[3] = T;
}

int om_edge_flux(const om_opts *o, const double *in, const double *waf, double *out)
{
    edge_flux(o, waf ? 2 : 0, in, waf, out);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradients: least squares + Barth-Jespersen (R13)                         */
/* ------------------------------------------------------------------------ */

/* Limited gradients of (eta, u, v) and, when hq is given (R16), of h as a
 * fourth quantity: gl[2 s], gl[2 s + 1] for quantity s. */
static void cell_gradient(const om_mesh *m, const om_opts *o, int64_t i,
                          const double *eta, const double *u, const double *v, const double *h,
                          double *gl, double *gu, const double *hq)
{
    const int nq = hq ? 4 : 3;
    for (int q = 0; q < 2 * nq; q++) { gl[q] = 0.0; if (gu) gu[q] = 0.0; }
    if (h[i] <= o->h_eps) return;
    double Mxx = 0, Mxy = 0, Myy = 0;
    double b[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const double *q[4] = {eta, u, v, hq};
    int cnt = 0;
    for (int k = 0; k < 3; k++) {
        int32_t j = m->nbr[3 * i + k];
        if (j < 0) continue;
        if (h[j] <= o->h_eps) return;            /* dry neighbour: first order */
        double dx = m->cx[j] - m->cx[i], dy = m->cy[j] - m->cy[i];
        Mxx += dx * dx; Mxy += dx * dy; Myy += dy * dy;
        for (int s = 0; s < nq; s++) {
            double dq = q[s][j] - q[s][i];
            b[s][0] += dx * dq; b[s][1] += dy * dq;
        }
        cnt++;
    }
    double det = Mxx * Myy - Mxy * Mxy, tr = Mxx + Myy;
    if (cnt < 2 || det <= 1e-12 * tr * tr) return;  /* singular: first order */
    for (int s = 0; s < nq; s++) {
        /* Cramer's rule for the 2x2 normal equations */
        double gx = (Myy * b[s][0] - Mxy * b[s][1]) / det;
        double gy = (Mxx * b[s][1] - Mxy * b[s][0]) / det;
        if (gu) { gu[2 * s] = gx; gu[2 * s + 1] = gy; }
        double qi = q[s][i], qmin = qi, qmax = qi;
        for (int k = 0; k < 3; k++) {
            int32_t j = m->nbr[3 * i + k];
            if (j < 0) continue;
            if (q[s][j] < qmin) qmin = q[s][j];
            if (q[s][j] > qmax) qmax = q[s][j];
        }
        double phi = 1.0;
        for (int k = 0; k < 3; k++) {
            double d = gx * m->mx[3 * i + k] + gy * m->my[3 * i + k];
            double ph = 1.0;
            if (d > 0.0) ph = (qmax - qi) / d;
            else if (d < 0.0) ph = (qmin - qi) / d;
            if (ph < phi) phi = ph;
        }
        gl[2 * s] = phi * gx; gl[2 * s + 1] = phi * gy;
    }
}

static void primitives(const om_mesh *m, const om_opts *o, const double *z,
                       const double *h, const double *hu, const double *hv,
                       double *eta, double *u, double *v)
{
    int64_t n = m->n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        eta[i] = h[i] + z[i];
        u[i] = h[i] > o->h_eps ? hu[i] / h[i] : 0.0;
        v[i] = h[i] > o->h_eps ? hv[i] / h[i] : 0.0;
    }
}

int om_gradients(const om_mesh *m, const om_opts *o, const double *z,
                 const double *h, const double *hu, const double *hv,
                 double *gl, double *gu)
{
    int64_t n = m->n;
    double *eta = malloc(sizeof(double) * n), *u = malloc(sizeof(double) * n), *v = malloc(sizeof(double) * n);
    primitives(m, o, z, h, hu, hv, eta, u, v);
    for (int64_t i = 0; i < n; i++) cell_gradient(m, o, i, eta, u, v, h, gl + 6 * i, gu ? gu + 6 * i : NULL, NULL);
    free(eta); free(u); free(v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One explicit Euler step (Sec. 6.1, eq. of the semi-discrete form)         */
/* ------------------------------------------------------------------------ */

typedef struct {
    double *eta, *u, *v, *grad, *clip, *bflux;
} work_t;

/* face values (eta, u, v) of cell i at the midpoint of its local edge k, and
 * f[3] the bed there: z_i, or with the second-order reconstruction (R16)
 * z_i + (grad eta - grad h) . (m_k - c_i), the bed that the reconstructed
 * eta and h imply */
static void face_values(const om_mesh *m, const om_opts *o, const work_t *w, const double *z, int scheme,
                        int64_t i, int k, double *f)
{
    f[0] = w->eta[i]; f[1] = w->u[i]; f[2] = w->v[i]; f[3] = z[i];
    if (scheme == 1) {
        const double *gr = w->grad + 8 * i;
        double ox = m->mx[3 * i + k], oy = m->my[3 * i + k];
        f[0] += gr[0] * ox + gr[1] * oy;
        f[1] += gr[2] * ox + gr[3] * oy;
        f[2] += gr[4] * ox + gr[5] * oy;
        if (o->hr_order == 2) f[3] += (gr[0] - gr[6]) * ox + (gr[1] - gr[7]) * oy;
    }
}

/* mean of q and of the velocity over the two other neighbours of cell i
 * (its edges k+1 and k+2); a missing neighbour stands in with cell i (R4).
 * q is the free surface eta (R4), or the depth h with the option of R17. */
static void upwind_means(const om_mesh *m, const work_t *w, const double *q, int64_t i, int k,
                         double *hm, double *um, double *vm)
{
    double sh = 0, su = 0, sv = 0;
    for (int d = 1; d <= 2; d++) {
        int32_t j = m->nbr[3 * i + (k + d) % 3];
        int64_t c = j >= 0 ? j : i;
        sh += q[c]; su += w->u[c]; sv += w->v[c];
    }
    *hm = sh / 2.0; *um = su / 2.0; *vm = sv / 2.0;
}

/* Sec. 6.2.3: the limited slope of the paper's MUSCL (see om_beta_limit). */
double om_beta_limit(double beta, double up, double dn)
{
    if (dn > 0.0) {
        double p = fmin(beta * up, dn), q = fmin(up, beta * dn);
        return fmax(0.0, fmax(p, q));
    }
    if (dn < 0.0) {
        double p = fmax(beta * up, dn), q = fmax(up, beta * dn);
        return fmin(0.0, fmin(p, q));
    }
    return 0.0;
}

/* upwind data of cell c for its edge e: mean of (eta, u, v) over its two
 * other neighbours, the position of that mean (mean of their centroids), and
 * whether those cells are wet; a missing neighbour stands in with c (R15) */
static void paper_upwind(const om_mesh *m, const om_opts *o, const work_t *w, const double *h, int64_t c, int e,
                         double *q, double *px, double *py, int *wet)
{
    q[0] = q[1] = q[2] = 0.0;
    *px = *py = 0.0;
    *wet = 1;
    for (int d = 1; d <= 2; d++) {
        int32_t j = m->nbr[3 * c + (e + d) % 3];
        int64_t s = j >= 0 ? j : c;
        q[0] += w->eta[s] / 2.0; q[1] += w->u[s] / 2.0; q[2] += w->v[s] / 2.0;
        *px += m->cx[s] / 2.0; *py += m->cy[s] / 2.0;
        if (h[s] <= o->h_eps) *wet = 0;
    }
}

/* Reconstructed states of the paper's MUSCL (Sec. 6.2.3) at the edge between
 * L (cell l, its local edge kl) and R (cell r, edge kr), as printed:
 *   U~_L = U_L + |x_RL - x_L| dU_L,   U~_R = U_R - |x_R - x_RL| dU_R,
 *   dU_L = lim((U_L - U_Lupw)/|x_L - x_Lupw|, (U_R - U_L)/|x_R - x_L|),
 *   dU_R = lim((U_R - U_L)/|x_R - x_L|, (U_Rupw - U_R)/|x_Rupw - x_R|),
 * componentwise for (eta, u, v), with the readings of R15. */
static void paper_edge_states(const om_mesh *m, const om_opts *o, const work_t *w, const double *h,
                              int64_t l, int kl, int64_t r, int kr, double *fl, double *fr)
{
    const double ql[3] = {w->eta[l], w->u[l], w->v[l]}, qr[3] = {w->eta[r], w->u[r], w->v[r]};
    double ul[3], ur[3], lx, ly, rx, ry;
    int wl, wr;
    paper_upwind(m, o, w, h, l, kl, ul, &lx, &ly, &wl);
    paper_upwind(m, o, w, h, r, kr, ur, &rx, &ry, &wr);
    const double d_lr = hypot(m->cx[r] - m->cx[l], m->cy[r] - m->cy[l]);
    const double d_lu = hypot(m->cx[l] - lx, m->cy[l] - ly), d_ru = hypot(rx - m->cx[r], ry - m->cy[r]);
    const double m_l = hypot(m->mx[3 * l + kl], m->my[3 * l + kl]);   /* |x_RL - x_L| */
    const double m_r = hypot(m->mx[3 * r + kr], m->my[3 * r + kr]);   /* |x_R - x_RL| */
    const int wet_lr = h[l] > o->h_eps && h[r] > o->h_eps;
    for (int s = 0; s < 3; s++) {
        const double s_lr = (qr[s] - ql[s]) / d_lr;
        double dl = 0.0, dr = 0.0;
        if (wet_lr && wl) dl = om_beta_limit(o->beta, d_lu > 0.0 ? (ql[s] - ul[s]) / d_lu : 0.0, s_lr);
        if (wet_lr && wr) dr = om_beta_limit(o->beta, s_lr, d_ru > 0.0 ? (ur[s] - qr[s]) / d_ru : 0.0);
        fl[s] = ql[s] + m_l * dl;
        fr[s] = qr[s] - m_r * dr;
    }
}

/* R16: the own-side pressure term of a face with the linear bed, g/2 (h_f^2 -
 * h_i^2) + g (h_f + h_i)/2 (z_f - z_i): the first-order correction plus the
 * centred bed source of the face, written as g/2 (h_f + h_i)(eta_f - eta_i)
 * on a wet face (h_f = eta_f - z_f) and g/2 (h_f + h_i)(z_f - eta_i) on a dry
 * one, so that a lake at rest gives an exact zero.  f = (eta_f, u, v, z_f). */
static double hyd2(double g, double hf, double hc, const double *f, double eta_c)
{
    return 0.5 * g * (hf + hc) * ((hf > 0.0 ? f[0] : f[3]) - eta_c);
}

static void euler_stage(const om_mesh *m, const om_opts *o, work_t *w,
                        const double *z, const double *nman, const double *qlen, const double *level,
                        const double *h, const double *hu, const double *hv,
                        double *h1, double *hu1, double *hv1, double dt)
{
    const int64_t n = m->n;
    const int scheme = o->scheme;
    const double g = o->g;
    primitives(m, o, z, h, hu, hv, w->eta, w->u, w->v);
    if (scheme == 1) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            cell_gradient(m, o, i, w->eta, w->u, w->v, h, w->grad + 8 * i, NULL, o->hr_order == 2 ? h : NULL);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double R[3] = {0.0, 0.0, 0.0};
        double bsum = 0.0;
        for (int k = 0; k < 3; k++) {
            double L = m->len[3 * i + k];
            double nx = m->lnx[3 * i + k] / L, ny = m->lny[3 * i + k] / L;
            int32_t j = m->nbr[3 * i + k];
            double fi[4];
            face_values(m, o, w, z, scheme, i, k, fi);
            double hfi = fi[0] - fi[3];
            if (hfi < 0.0) hfi = 0.0;
            double M, P, T, sgn;
            if (j >= 0) {
                /* canonical orientation (R12): L = lower id, normal from L to R */
                int32_t kj = m->nbr_edge[3 * i + k];
                int64_t a = i < j ? i : j, b = i < j ? j : i;
                int ka = i < j ? k : kj, kb = i < j ? kj : k;
                double cnx = i < j ? nx : -nx, cny = i < j ? ny : -ny;
                double fa[4], fb[4];
                if (scheme == 3) {
                    paper_edge_states(m, o, w, h, a, ka, b, kb, fa, fb);
                    fa[3] = z[a]; fb[3] = z[b];
                } else {
                    face_values(m, o, w, z, scheme, a, ka, fa);
                    face_values(m, o, w, z, scheme, b, kb, fb);
                }
                double hfa = fa[0] - fa[3]; if (hfa < 0.0) hfa = 0.0;
                double hfb = fb[0] - fb[3]; if (hfb < 0.0) hfb = 0.0;
                double zf = fa[3] > fb[3] ? fa[3] : fb[3];        /* R6 (face beds: R16) */
                double hsa = fa[0] - zf; if (hsa < 0.0) hsa = 0.0;
                double hsb = fb[0] - zf; if (hsb < 0.0) hsb = 0.0;
                /* R16: the cell-centre pressure term is replaced by hyd2 below (so
                 * edge_flux gets hcell = hface and adds nothing) */
                const int hr2 = scheme == 1 && o->hr_order == 2;
                double in[10] = {hfa, hsa, hr2 ? hfa : h[a], fa[1] * cnx + fa[2] * cny, -fa[1] * cny + fa[2] * cnx,
                                 hfb, hsb, hr2 ? hfb : h[b], fb[1] * cnx + fb[2] * cny, -fb[1] * cny + fb[2] * cnx};
                double out[4];
                if (scheme == 2) {
                    double hma, uma, vma, hmb, umb, vmb;
                    const double *q = o->waf_surface ? w->eta : h;     /* R4 / R17 */
                    upwind_means(m, w, q, a, ka, &hma, &uma, &vma);
                    upwind_means(m, w, q, b, kb, &hmb, &umb, &vmb);
                    double ddx = m->cx[b] - m->cx[a], ddy = m->cy[b] - m->cy[a];
                    double wf[8] = {dt / sqrt(ddx * ddx + ddy * ddy), hma, hmb,
                                    -uma * cny + vma * cnx, -umb * cny + vmb * cnx, q[a], q[b], 0.0};
                    edge_flux(o, scheme, in, wf, out);
                } else {
                    edge_flux(o, scheme, in, NULL, out);
                }
                M = out[0]; T = out[3];
                P = i < j ? out[1] : out[2];
                if (hr2) P += hyd2(g, hfi, h[i], fi, w->eta[i]);
                sgn = i < j ? 1.0 : -1.0;
                /* sgn * (M, P n_c + T t_c) with n_c = sgn * n  ==  (sgn M, P n + T t) */
                R[0] += L * sgn * M;
                R[1] += L * (P * nx - T * ny);
                R[2] += L * (P * ny + T * nx);
                continue;
            }
            /* boundary edge: cell i is the left state, normal outward (Sec. 6.1) */
            int tag = m->btag[3 * i + k], type = tag & 3, grp = tag >> 2;
            double un = fi[1] * nx + fi[2] * ny, vt = -fi[1] * ny + fi[2] * nx;
            double hyd = (scheme == 1 && o->hr_order == 2) ? hyd2(g, hfi, h[i], fi, w->eta[i])
                                                           : 0.5 * g * (hfi - h[i]) * (hfi + h[i]);
            if (type == BC_WALL) {
                M = 0.0; P = hyd; T = 0.0;
            } else if (type == BC_OPEN) {
                M = hfi * un; P = hfi * un * un + hyd; T = M * vt;
            } else if (type == BC_INFLOW) {
                double q = qlen[grp];
                M = -q; P = (hfi > o->h_eps ? q * q / hfi : 0.0) + hyd; T = 0.0;
            } else {
                double hg = level[grp] - fi[3];
                if (hg < 0.0) hg = 0.0;
                const int hr2 = scheme == 1 && o->hr_order == 2;
                double in[10] = {hfi, hfi, hr2 ? hfi : h[i], un, vt, hg, hg, hg, un, vt};
                double out[4];
                edge_flux(o, 0, in, NULL, out);
                M = out[0]; P = out[1] + (hr2 ? hyd : 0.0); T = out[3];
            }
            R[0] += L * M;
            R[1] += L * (P * nx - T * ny);
            R[2] += L * (P * ny + T * nx);
            bsum -= L * M;
        }
        double r = dt / m->area[i];
        double hn = h[i] - r * R[0], hun = hu[i] - r * R[1], hvn = hv[i] - r * R[2];
        double clip = 0.0;
        if (hn < 0.0) { clip = -hn * m->area[i]; hn = 0.0; }
        if (hn <= o->h_eps) { hun = 0.0; hvn = 0.0; }
        else if (nman[i] > 0.0) {
            /* R9: point-implicit Manning friction */
            double sp = sqrt(hun * hun + hvn * hvn) / hn;
            double f = 1.0 + dt * g * nman[i] * nman[i] * sp / pow(hn, 4.0 / 3.0);
            hun /= f; hvn /= f;
        }
        h1[i] = hn; hu1[i] = hun; hv1[i] = hvn;
        w->clip[i] = clip;
        w->bflux[i] = bsum * dt;
    }
}

static double sum_fixed(const double *x, int64_t n)
{
    double s = 0.0, c = 0.0;            /* Neumaier */
    for (int64_t i = 0; i < n; i++) {
        double t = s + x[i];
        if (fabs(s) >= fabs(x[i])) c += (s - t) + x[i];
        else c += (x[i] - t) + s;
        s = t;
    }
    return s + c;
}

double om_mass(const om_mesh *m, const double *h)
{
    double *x = malloc(sizeof(double) * m->n);
    for (int64_t i = 0; i < m->n; i++) x[i] = m->area[i] * h[i];
    double s = sum_fixed(x, m->n);
    free(x);
    return s;
}

int om_run(const om_mesh *m, const om_opts *o,
           const double *z, const double *nman,
           const double *q_in, int n_in, const double *level, int n_level,
           double *h, double *hu, double *hv, int n_steps,
           const double *dt_given, double *dt_used, double *diag)
{
    (void)n_level;
    const int64_t n = m->n;
#ifdef _OPENMP
    int saved = omp_get_max_threads();
    if (o->threads > 0) omp_set_num_threads(o->threads);
#endif
    /* inflow per unit length: Q spread over the total length of the group's edges (R7) */
    double qlen[64];
    for (int gi = 0; gi < 64; gi++) qlen[gi] = 0.0;
    if (n_in > 64) n_in = 64;
    for (int gi = 0; gi < n_in; gi++) {
        double tot = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < 3; k++) {
                int t = m->btag[3 * i + k];
                if (m->nbr[3 * i + k] < 0 && t >= 0 && (t & 3) == BC_INFLOW && (t >> 2) == gi) tot += m->len[3 * i + k];
            }
        qlen[gi] = tot > 0.0 ? q_in[gi] / tot : 0.0;
    }
    double rmin = m->rin[0];
    for (int64_t i = 1; i < n; i++) if (m->rin[i] < rmin) rmin = m->rin[i];

    work_t w;
    w.eta = malloc(sizeof(double) * n); w.u = malloc(sizeof(double) * n); w.v = malloc(sizeof(double) * n);
    w.grad = malloc(sizeof(double) * 8 * n);
    w.clip = malloc(sizeof(double) * n); w.bflux = malloc(sizeof(double) * n);
    double *h1 = malloc(sizeof(double) * n), *hu1 = malloc(sizeof(double) * n), *hv1 = malloc(sizeof(double) * n);
    double *h2 = NULL, *hu2 = NULL, *hv2 = NULL;
    if (o->time_scheme == 1) {
        h2 = malloc(sizeof(double) * n); hu2 = malloc(sizeof(double) * n); hv2 = malloc(sizeof(double) * n);
    }
    int rc = 0;
    for (int s = 0; s < n_steps && rc == 0; s++) {
        double dt;
        if (dt_given) {
            dt = dt_given[s];
        } else {
            /* CFL rule of Sec. 6.1 with d = inscribed radius (R11): the global
             * form min_i r_i / max_i s_i, or per cell min_i (r_i / s_i) */
            double smax = 0.0, rs_min = INFINITY;
            for (int64_t i = 0; i < n; i++) {
                if (h[i] <= o->h_eps) continue;
                double u = hu[i] / h[i], v = hv[i] / h[i];
                double sp = sqrt(o->g * h[i]) + sqrt(u * u + v * v);
                if (sp > smax) smax = sp;
                if (sp > 0.0 && m->rin[i] / sp < rs_min) rs_min = m->rin[i] / sp;
            }
            if (!(smax > 0.0)) { rc = -4; break; }
            dt = o->cfl_local ? o->cfl * rs_min : o->cfl * rmin / smax;
        }
        if (dt_used) dt_used[s] = dt;
        euler_stage(m, o, &w, z, nman, qlen, level, h, hu, hv, h1, hu1, hv1, dt);
        double clip = sum_fixed(w.clip, n), bin = sum_fixed(w.bflux, n);
        if (o->time_scheme == 1) {
            euler_stage(m, o, &w, z, nman, qlen, level, h1, hu1, hv1, h2, hu2, hv2, dt);
            clip = 0.5 * (clip + sum_fixed(w.clip, n));
            bin = 0.5 * (bin + sum_fixed(w.bflux, n));
            for (int64_t i = 0; i < n; i++) {
                h[i] = 0.5 * (h[i] + h2[i]); hu[i] = 0.5 * (hu[i] + hu2[i]); hv[i] = 0.5 * (hv[i] + hv2[i]);
            }
        } else {
            memcpy(h, h1, sizeof(double) * n); memcpy(hu, hu1, sizeof(double) * n); memcpy(hv, hv1, sizeof(double) * n);
        }
        if (diag) { diag[0] += dt; diag[1] += clip; diag[2] += bin; }
        for (int64_t i = 0; i < n; i++)
            if (!isfinite(h[i]) || !isfinite(hu[i]) || !isfinite(hv[i])) { rc = -5; break; }
    }
    free(w.eta); free(w.u); free(w.v); free(w.grad); free(w.clip); free(w.bflux);
    free(h1); free(hu1); free(hv1); free(h2); free(hu2); free(hv2);
#ifdef _OPENMP
    omp_set_num_threads(saved);
#endif
    return rc;
}
