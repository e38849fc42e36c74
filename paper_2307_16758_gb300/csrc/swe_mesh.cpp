// Host mesh builder: orientation, edge adjacency, boundary tags, geometry and
// a locality renumbering (Morton or reverse Cuthill-McKee).
//
// The adjacency follows the idea of the paper's pre-processing (Sec. 3.1: cells
// are connected through their shared edges, found from a map of edges); here
// the edges are sorted by their node pair instead of hashed, which keeps the
// result deterministic.  The renumbering plays the role of the paper's
// renumbering for locality (Sec. 3.3) on a single GPU.  Geometry follows the
// notation of Sec. 6.1 (|Omega_i|, L_ij, n_ij) and the inscribed radius R_L
// of the CFL rule.  Compiled without floating-point contraction so that every
// geometric quantity is reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>

#include "swe_mesh.h"

void swe_set_error(const std::string &msg);

namespace {

struct EdgeKey {
    uint64_t key;     // (lo << 32) | hi
    int32_t cell;
    int32_t k;
};

inline uint64_t node_key(int32_t a, int32_t b)
{
    uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
    return ((uint64_t)lo << 32) | hi;
}

uint64_t morton_interleave(uint64_t qx, uint64_t qy)
{
    uint64_t key = 0;
    for (int b = 0; b < 21; b++) {
        key |= ((qx >> b) & 1ULL) << (2 * b);
        key |= ((qy >> b) & 1ULL) << (2 * b + 1);
    }
    return key;
}

// Z-order of the centroids in their square bounding box, 21 bits per axis,
// equal keys by original id.
void morton_perm(const std::vector<double> &cx, const std::vector<double> &cy, std::vector<int32_t> &perm)
{
    const int64_t n = (int64_t)cx.size();
    double xmin = cx[0], xmax = cx[0], ymin = cy[0], ymax = cy[0];
    for (int64_t i = 1; i < n; i++) {
        xmin = std::min(xmin, cx[i]); xmax = std::max(xmax, cx[i]);
        ymin = std::min(ymin, cy[i]); ymax = std::max(ymax, cy[i]);
    }
    double ext = std::max(xmax - xmin, ymax - ymin);
    if (!(ext > 0.0)) ext = 1.0;
    const double s = 2097151.0 / ext;
    std::vector<std::pair<uint64_t, int32_t>> keys((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        double fx = std::floor((cx[i] - xmin) * s), fy = std::floor((cy[i] - ymin) * s);
        fx = std::min(std::max(fx, 0.0), 2097151.0);
        fy = std::min(std::max(fy, 0.0), 2097151.0);
        keys[i] = {morton_interleave((uint64_t)fx, (uint64_t)fy), (int32_t)i};
    }
    std::sort(keys.begin(), keys.end());
    perm.resize((size_t)n);
    for (int64_t i = 0; i < n; i++) perm[i] = keys[i].second;
}

// Reverse Cuthill-McKee: breadth-first from the unvisited cell of lowest
// (degree, id), neighbours visited by (degree, id), then the order reversed.
void rcm_perm(const std::vector<int32_t> &nbr, int64_t n, std::vector<int32_t> &perm)
{
    std::vector<int> deg((size_t)n, 0);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) deg[i] += nbr[3 * i + k] >= 0;
    std::vector<int32_t> start((size_t)n);
    std::iota(start.begin(), start.end(), 0);
    std::stable_sort(start.begin(), start.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
    std::vector<char> seen((size_t)n, 0);
    perm.assign((size_t)n, 0);
    int64_t head = 0, tail = 0, sp = 0;
    while (tail < n) {
        while (seen[start[sp]]) sp++;
        perm[tail++] = start[sp];
        seen[start[sp]] = 1;
        while (head < tail) {
            int32_t c = perm[head++];
            int32_t cand[3];
            int cnt = 0;
            for (int k = 0; k < 3; k++) {
                int32_t j = nbr[3 * c + k];
                if (j >= 0 && !seen[j]) cand[cnt++] = j;
            }
            std::sort(cand, cand + cnt, [&](int32_t a, int32_t b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            for (int q = 0; q < cnt; q++) {
                if (seen[cand[q]]) continue;
                seen[cand[q]] = 1;
                perm[tail++] = cand[q];
            }
        }
    }
    std::reverse(perm.begin(), perm.end());
}

}  // namespace

int swe_mesh_build_host(const double *xy, int64_t n_nodes, const int32_t *tri_in, int64_t n,
                        const int32_t *bnd, const int32_t *bnd_tag, int64_t n_bnd,
                        const int32_t *cut, int64_t n_cut, int reorder, swe_mesh **out)
{
    if (!xy || !tri_in || !out || n <= 0 || n_nodes < 3 || n >= (1LL << 28) || n_nodes >= (1LL << 31) ||
        n_bnd < 0 || n_cut < 0 || (n_bnd > 0 && (!bnd || !bnd_tag)) || (n_cut > 0 && !cut) ||
        reorder < SWE_REORDER_NONE || reorder > SWE_REORDER_RCM) {
        swe_set_error("swe_mesh_create: bad argument");
        return SWE_ERR_ARG;
    }
    // --- orientation and area, original order ---
    std::vector<int32_t> t0((size_t)(3 * n));
    std::vector<double> area0((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        int32_t a = tri_in[3 * i], b = tri_in[3 * i + 1], c = tri_in[3 * i + 2];
        if (a < 0 || b < 0 || c < 0 || a >= n_nodes || b >= n_nodes || c >= n_nodes) {
            swe_set_error("swe_mesh_create: node id out of range in triangle " + std::to_string(i));
            return SWE_ERR_MESH;
        }
        double cross = (xy[2 * b] - xy[2 * a]) * (xy[2 * c + 1] - xy[2 * a + 1])
                     - (xy[2 * b + 1] - xy[2 * a + 1]) * (xy[2 * c] - xy[2 * a]);
        if (cross == 0.0) {
            swe_set_error("swe_mesh_create: degenerate triangle " + std::to_string(i));
            return SWE_ERR_MESH;
        }
        if (cross < 0.0) std::swap(b, c);
        t0[3 * i] = a; t0[3 * i + 1] = b; t0[3 * i + 2] = c;
        area0[i] = 0.5 * std::fabs(cross);
    }
    // --- adjacency by sorted node-pair keys ---
    std::vector<EdgeKey> ek((size_t)(3 * n));
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++)
            ek[3 * i + k] = {node_key(t0[3 * i + k], t0[3 * i + (k + 1) % 3]), (int32_t)i, k};
    std::sort(ek.begin(), ek.end(), [](const EdgeKey &x, const EdgeKey &y) {
        return x.key != y.key ? x.key < y.key : (x.cell != y.cell ? x.cell < y.cell : x.k < y.k);
    });
    std::vector<int32_t> nb0((size_t)(3 * n), -1), ne0((size_t)(3 * n), -1), bt0((size_t)(3 * n), -1);
    for (size_t s = 0; s < ek.size();) {
        size_t t = s + 1;
        while (t < ek.size() && ek[t].key == ek[s].key) t++;
        if (t - s > 2) {
            swe_set_error("swe_mesh_create: edge shared by more than two triangles");
            return SWE_ERR_MESH;
        }
        if (t - s == 2) {
            const EdgeKey &x = ek[s], &y = ek[s + 1];
            if (t0[3 * x.cell + x.k] == t0[3 * y.cell + y.k]) {
                swe_set_error("swe_mesh_create: folded mesh (neighbours walk an edge the same way)");
                return SWE_ERR_MESH;
            }
            nb0[3 * x.cell + x.k] = y.cell; ne0[3 * x.cell + x.k] = y.k;
            nb0[3 * y.cell + y.k] = x.cell; ne0[3 * y.cell + y.k] = x.k;
        }
        s = t;
    }
    ek.clear(); ek.shrink_to_fit();
    // --- internal walls ---
    if (n_cut > 0) {
        std::vector<uint64_t> ck((size_t)n_cut);
        for (int64_t i = 0; i < n_cut; i++) ck[i] = node_key(cut[2 * i], cut[2 * i + 1]);
        std::sort(ck.begin(), ck.end());
        int64_t found = 0;
        for (int64_t e = 0; e < 3 * n; e++) {
            if (nb0[e] < 0) continue;
            int64_t i = e / 3; int k = (int)(e % 3);
            uint64_t key = node_key(t0[3 * i + k], t0[3 * i + (k + 1) % 3]);
            if (std::binary_search(ck.begin(), ck.end(), key)) {
                nb0[e] = -1; ne0[e] = -1; bt0[e] = SWE_WALL;
                found++;
            }
        }
        if (found != 2 * n_cut) {
            swe_set_error("swe_mesh_create: a cut edge is not an interior edge (or is listed twice)");
            return SWE_ERR_MESH;
        }
    }
    // --- boundary tags ---
    std::vector<std::pair<uint64_t, int32_t>> bk((size_t)n_bnd);
    for (int64_t i = 0; i < n_bnd; i++) {
        int32_t tg = bnd_tag[i];
        if (tg < 0 || (tg >> 2) >= SWE_MAX_GROUPS) {
            swe_set_error("swe_mesh_create: boundary tag out of range");
            return SWE_ERR_MESH;
        }
        bk[i] = {node_key(bnd[2 * i], bnd[2 * i + 1]), tg};
    }
    std::sort(bk.begin(), bk.end());
    for (int64_t i = 1; i < n_bnd; i++)
        if (bk[i].first == bk[i - 1].first) {
            swe_set_error("swe_mesh_create: boundary edge listed twice");
            return SWE_ERR_MESH;
        }
    int64_t matched = 0;
    for (int64_t e = 0; e < 3 * n; e++) {
        if (nb0[e] >= 0 || bt0[e] >= 0) continue;
        int64_t i = e / 3; int k = (int)(e % 3);
        uint64_t key = node_key(t0[3 * i + k], t0[3 * i + (k + 1) % 3]);
        auto it = std::lower_bound(bk.begin(), bk.end(), std::make_pair(key, INT32_MIN));
        if (it != bk.end() && it->first == key) { bt0[e] = it->second; matched++; }
        else bt0[e] = SWE_WALL;
    }
    if (matched != n_bnd) {
        swe_set_error("swe_mesh_create: a listed boundary edge is not on the boundary");
        return SWE_ERR_MESH;
    }
    // --- geometry, original order ---
    std::vector<double> cx0((size_t)n), cy0((size_t)n), lnx0((size_t)(3 * n)), lny0((size_t)(3 * n)),
        len0((size_t)(3 * n)), rin0((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        const int32_t *t = &t0[3 * i];
        double px[3] = {xy[2 * t[0]], xy[2 * t[1]], xy[2 * t[2]]};
        double py[3] = {xy[2 * t[0] + 1], xy[2 * t[1] + 1], xy[2 * t[2] + 1]};
        cx0[i] = (px[0] + px[1] + px[2]) / 3.0;
        cy0[i] = (py[0] + py[1] + py[2]) / 3.0;
        double perim = 0.0;
        for (int k = 0; k < 3; k++) {
            int k1 = (k + 1) % 3;
            double lx = py[k1] - py[k], ly = -(px[k1] - px[k]);
            lnx0[3 * i + k] = lx; lny0[3 * i + k] = ly;
            len0[3 * i + k] = std::sqrt(lx * lx + ly * ly);
            perim += len0[3 * i + k];
        }
        rin0[i] = 2.0 * area0[i] / perim;
    }
    // --- renumbering ---
    auto *m = new swe_mesh();
    m->n = n;
    if (reorder == SWE_REORDER_MORTON) morton_perm(cx0, cy0, m->perm);
    else if (reorder == SWE_REORDER_RCM) rcm_perm(nb0, n, m->perm);
    else { m->perm.resize((size_t)n); std::iota(m->perm.begin(), m->perm.end(), 0); }
    m->inv.resize((size_t)n);
    for (int64_t i = 0; i < n; i++) m->inv[m->perm[i]] = (int32_t)i;
    // --- new-order arrays ---
    m->tri.resize((size_t)(3 * n)); m->nbr.resize((size_t)(3 * n)); m->nbr_edge.resize((size_t)(3 * n));
    m->btag.resize((size_t)(3 * n)); m->owner.resize((size_t)(3 * n));
    m->lnx.resize((size_t)(3 * n)); m->lny.resize((size_t)(3 * n)); m->len.resize((size_t)(3 * n));
    m->dx.resize((size_t)(3 * n)); m->dy.resize((size_t)(3 * n));
    m->area.resize((size_t)n); m->cx.resize((size_t)n); m->cy.resize((size_t)n); m->rin.resize((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        int32_t o = m->perm[i];
        m->area[i] = area0[o]; m->cx[i] = cx0[o]; m->cy[i] = cy0[o]; m->rin[i] = rin0[o];
        for (int k = 0; k < 3; k++) {
            int64_t e = 3 * i + k, eo = 3 * (int64_t)o + k;
            int32_t j = nb0[eo];
            m->tri[e] = t0[eo];
            m->nbr[e] = j >= 0 ? m->inv[j] : -1;
            m->nbr_edge[e] = ne0[eo];
            m->btag[e] = bt0[eo];
            // canonical orientation by original id, so that renumbering
            // does not change which side is the left state of the edge
            m->owner[e] = j >= 0 && o < j;
            m->lnx[e] = lnx0[eo]; m->lny[e] = lny0[eo]; m->len[e] = len0[eo];
            m->dx[e] = j >= 0 ? cx0[j] - cx0[o] : 0.0;
            m->dy[e] = j >= 0 ? cy0[j] - cy0[o] : 0.0;
            if (j < 0 && (bt0[eo] & 3) == SWE_INFLOW) m->group_len[bt0[eo] >> 2] += len0[eo];
        }
    }
    m->r_min = m->rin[0];
    for (int64_t i = 1; i < n; i++) m->r_min = std::min(m->r_min, m->rin[i]);
    *out = m;
    return SWE_OK;
}
