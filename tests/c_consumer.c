/*
 * A plain C99 program against the library's C ABI (host-only calls, so it
 * runs without a GPU): the headers must compile as C, the library must link
 * from C, and the host calls must behave as documented.
 *
 * Mesh: the unit square of 2 x 2 squares, each split by its "/" diagonal
 * (8 triangles), walls all round except an inflow edge on x = 0.
 * Prints "ok" and exits 0 when every check passes, else names the check.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "swe.h"
#include "swe_tile_plan.h"

#define CHECK(c)                                                             \
    do {                                                                     \
        if (!(c)) {                                                          \
            printf("failed: %s (line %d): %s\n", #c, __LINE__, swe_last_error()); \
            return 1;                                                        \
        }                                                                    \
    } while (0)

int main(void)
{
    double xy[9][2];
    int32_t tri[8][3];
    int32_t bnd[8][2], tag[8];
    int i, j, k, n_tri = 0, n_bnd = 0;
    for (j = 0; j < 3; j++)
        for (i = 0; i < 3; i++) { xy[3 * j + i][0] = 0.5 * i; xy[3 * j + i][1] = 0.5 * j; }
    for (j = 0; j < 2; j++)
        for (i = 0; i < 2; i++) {
            int32_t p00 = 3 * j + i, p10 = p00 + 1, p01 = p00 + 3, p11 = p00 + 4;
            tri[n_tri][0] = p00; tri[n_tri][1] = p10; tri[n_tri][2] = p11; n_tri++;
            tri[n_tri][0] = p00; tri[n_tri][1] = p11; tri[n_tri][2] = p01; n_tri++;
        }
    for (i = 0; i < 2; i++) {                    /* bottom, top, right: walls */
        bnd[n_bnd][0] = i; bnd[n_bnd][1] = i + 1; tag[n_bnd++] = SWE_WALL;
        bnd[n_bnd][0] = 6 + i; bnd[n_bnd][1] = 7 + i; tag[n_bnd++] = SWE_WALL;
        bnd[n_bnd][0] = 3 * i + 2; bnd[n_bnd][1] = 3 * i + 5; tag[n_bnd++] = SWE_WALL;
    }
    bnd[n_bnd][0] = 0; bnd[n_bnd][1] = 3; tag[n_bnd++] = SWE_INFLOW;   /* left: inflow group 0 */
    bnd[n_bnd][0] = 3; bnd[n_bnd][1] = 6; tag[n_bnd++] = SWE_WALL;

    swe_params p;
    CHECK(swe_params_default(&p, SWE_SCHEME_MUSCL, SWE_FP32) == SWE_OK);
    CHECK(p.precision == SWE_FP32 && p.scheme == SWE_SCHEME_MUSCL && p.g == 9.81 && p.hr_order == 1);
    CHECK(swe_params_default(&p, 99, SWE_FP32) == SWE_ERR_ARG && strlen(swe_last_error()) > 0);

    swe_mesh *m = NULL;
    CHECK(swe_mesh_create(&xy[0][0], 9, &tri[0][0], n_tri, &bnd[0][0], tag, n_bnd, NULL, 0,
                          SWE_REORDER_MORTON, &m) == SWE_OK && m != NULL);
    int64_t n = 0;
    double r_min = 0.0;
    CHECK(swe_mesh_info(m, &n, &r_min) == SWE_OK && n == 8);
    /* inscribed radius of a right isosceles triangle with legs 0.5: 0.5 / (2 + sqrt 2) */
    CHECK(r_min > 0.146446 && r_min < 0.146447);

    int32_t perm[8], nbr[8][3], btag[8][3];
    double area[8];
    CHECK(swe_mesh_export(m, perm, NULL, &nbr[0][0], NULL, &btag[0][0], NULL, NULL, area, NULL, NULL, NULL,
                          NULL, NULL) == SWE_OK);
    {
        int seen[8] = {0}, n_interior = 0, n_inflow = 0;
        double total = 0.0;
        for (i = 0; i < 8; i++) {
            CHECK(perm[i] >= 0 && perm[i] < 8 && !seen[perm[i]]);
            seen[perm[i]] = 1;
            total += area[i];
            for (k = 0; k < 3; k++) {
                if (nbr[i][k] >= 0) {
                    int32_t q = nbr[i][k], back = 0;
                    for (j = 0; j < 3; j++) back += nbr[q][j] == i;
                    CHECK(back == 1 && btag[i][k] == -1);
                    n_interior++;
                } else {
                    n_inflow += btag[i][k] == SWE_INFLOW;
                }
            }
        }
        CHECK(total > 1.0 - 1e-15 && total < 1.0 + 1e-15);
        CHECK(n_interior == 2 * 8 && n_inflow == 1);    /* 8 interior edges, seen from both sides */
    }

    int64_t n_tiles = 0, n_words = 0;
    int32_t hmax = -1, h1max = -1, wmax = -1;
    CHECK(swe_tile_plan_info(m, 32, &n_tiles, &hmax, &h1max, &wmax, &n_words) == SWE_OK);
    CHECK(n_tiles == 1 && hmax == 0 && h1max == 0 && wmax % 8 == 0 && n_words == wmax);
    {
        int32_t *hdr = (int32_t *)malloc(sizeof(int32_t) * 8 * (size_t)n_tiles);
        int32_t *words = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_words);
        CHECK(hdr && words);
        CHECK(swe_tile_plan_export(m, 32, hdr, words) == SWE_OK);
        CHECK(hdr[0] == 0 && hdr[1] == 0 && hdr[3] == 8 && hdr[4] == 0 && hdr[5] == wmax);
        free(hdr);
        free(words);
    }
    CHECK(swe_tile_plan_info(m, 48, NULL, NULL, NULL, NULL, NULL) == SWE_ERR_ARG);
    CHECK(swe_tile_plan_info(NULL, 32, NULL, NULL, NULL, NULL, NULL) == SWE_ERR_ARG);

    swe_partition *part = NULL;
    int64_t a = -1, b = -1, n1 = -1, n2 = -1, nb = -1;
    CHECK(swe_partition_create(m, 2, &part) == SWE_OK);
    CHECK(swe_partition_info(part, 0, &a, &b, &n1, &n2, &nb) == SWE_OK && a == 0 && b == 4 && n1 > 0);
    CHECK(swe_partition_info(part, 2, &a, &b, &n1, &n2, &nb) == SWE_ERR_ARG);
    CHECK(swe_partition_destroy(part) == SWE_OK);

    /* a degenerate triangle is a mesh error */
    {
        int32_t bad[1][3] = {{0, 1, 2}};
        swe_mesh *m2 = NULL;
        CHECK(swe_mesh_create(&xy[0][0], 9, &bad[0][0], 1, NULL, NULL, 0, NULL, 0, SWE_REORDER_NONE, &m2) ==
              SWE_ERR_MESH && m2 == NULL);
    }
    CHECK(swe_mesh_destroy(m) == SWE_OK);
    printf("ok\n");
    return 0;
}
