/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Neighbor lists for double-precision particle data (the paper's Sec. 2.2:
 * many MD codes keep 64-bit particle data; the tree only needs enclosing
 * lower-precision boxes).  Only the tests, the smoke check and the
 * benchmark's CPU arms may load this code.
 *
 * The result is the neighbor-search problem of Sec. 1 with the distance
 * decision fixed as one FP64 expression (built with -ffp-contract=off):
 *     dx = xj - xi;   dx = dx - L * rint(dx * Linv);      (same for y, z)
 *     d2 = (dx*dx + dy*dy) + dz*dz;     j in N(i)  iff  d2 < rl2
 * with Linv = 1.0 / L and rl2 = rl * rl in FP64, rl the FP32 list radius
 * converted exactly to FP64.  j == i is never a neighbor (Sec. 2.1, Fig. 2).
 *
 *   or_nlist64_brute  O(N^2) over all pairs.
 *   or_nlist64_cell   27-cell stencil over a uniform cell list (Sec. 1,
 *                     Fig. 1b), same decision; brute force below 3 cells/axis.
 *
 * Rows are written sorted ascending; counts[i] is the full count even when it
 * exceeds cap (rows then hold the first cap neighbors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline double mi_d2_64(const double *xi, const double *xj, double L, double Linv)
{
    double dx = xj[0] - xi[0];
    double dy = xj[1] - xi[1];
    double dz = xj[2] - xi[2];
    dx = dx - L * rint(dx * Linv);
    dy = dy - L * rint(dy * Linv);
    dz = dz - L * rint(dz * Linv);
    return (dx * dx + dy * dy) + dz * dz;
}

static int cmp_int64(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* pos [n][3] float64, types [n] in [0, nt), rl [nt][nt] FP32 list radii. */
int or_nlist64_brute(int n, const double *pos, const int *types, double L, int nt,
                     const float *rl, int cap, int *rows, int *counts)
{
    double Linv = 1.0 / L;
    double rl2[64];
    if (nt < 1 || nt > 8) return -1;
    for (int k = 0; k < nt * nt; ++k) rl2[k] = (double)rl[k] * (double)rl[k];
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        const double *xi = pos + 3 * (size_t)i;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d2 = mi_d2_64(xi, pos + 3 * (size_t)j, L, Linv);
            if (d2 < rl2[types[i] * nt + types[j]]) {
                if (c < cap) rows[(size_t)i * cap + c] = j;
                ++c;
            }
        }
        counts[i] = c;
    }
    return 0;
}

int or_nlist64_cell(int n, const double *pos, const int *types, double L, int nt,
                    const float *rl, int cap, int *rows, int *counts)
{
    double rmax = 0.0;
    if (nt < 1 || nt > 8) return -1;
    for (int k = 0; k < nt * nt; ++k) rmax = (double)rl[k] > rmax ? (double)rl[k] : rmax;
    /* cells at least rmax wide, 0.1% margin for the binning round-off */
    int nc = (int)floor(L / (rmax * 1.001));
    if (nc > 1024) nc = 1024;
    if (nc < 3) return or_nlist64_brute(n, pos, types, L, nt, rl, cap, rows, counts);
    double inv_w = (double)nc / L;
    size_t ncell = (size_t)nc * nc * nc;
    int *start = (int *)calloc(ncell + 1, sizeof(int));
    int *list = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cid = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cc = (int *)malloc(sizeof(int) * 3 * (size_t)(n > 0 ? n : 1));
    if (!start || !list || !cid || !cc) {
        free(start); free(list); free(cid); free(cc);
        return -2;
    }
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            int c = (int)floor(pos[3 * (size_t)i + a] * inv_w);
            c = c < 0 ? 0 : (c >= nc ? nc - 1 : c);
            cc[3 * (size_t)i + a] = c;
        }
        cid[i] = (cc[3 * (size_t)i] * nc + cc[3 * (size_t)i + 1]) * nc + cc[3 * (size_t)i + 2];
        start[cid[i] + 1]++;
    }
    for (size_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    int *fill = (int *)malloc(sizeof(int) * ncell);
    memcpy(fill, start, sizeof(int) * ncell);
    for (int i = 0; i < n; ++i) list[fill[cid[i]]++] = i;
    free(fill);
    double Linv = 1.0 / L;
    double rl2[64];
    for (int k = 0; k < nt * nt; ++k) rl2[k] = (double)rl[k] * (double)rl[k];
#pragma omp parallel
    {
        int tmp_cap = 4096;
        int *tmp = (int *)malloc(sizeof(int) * tmp_cap);
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            const double *xi = pos + 3 * (size_t)i;
            int cx = cc[3 * (size_t)i], cy = cc[3 * (size_t)i + 1], cz = cc[3 * (size_t)i + 2];
            int c = 0;
            for (int ox = -1; ox <= 1; ++ox)
                for (int oy = -1; oy <= 1; ++oy)
                    for (int oz = -1; oz <= 1; ++oz) {
                        int ax = (cx + ox + nc) % nc, ay = (cy + oy + nc) % nc, az = (cz + oz + nc) % nc;
                        int cell = (ax * nc + ay) * nc + az;
                        for (int p = start[cell]; p < start[cell + 1]; ++p) {
                            int j = list[p];
                            if (j == i) continue;
                            double d2 = mi_d2_64(xi, pos + 3 * (size_t)j, L, Linv);
                            if (d2 < rl2[types[i] * nt + types[j]]) {
                                if (c == tmp_cap) {
                                    tmp_cap *= 2;
                                    tmp = (int *)realloc(tmp, sizeof(int) * tmp_cap);
                                }
                                tmp[c++] = j;
                            }
                        }
                    }
            qsort(tmp, (size_t)c, sizeof(int), cmp_int64);
            for (int k = 0; k < c && k < cap; ++k) rows[(size_t)i * cap + k] = tmp[k];
            counts[i] = c;
        }
        free(tmp);
    }
    free(start); free(list); free(cid); free(cc);
    return 0;
}
