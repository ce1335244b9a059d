/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously-correct neighbor lists used to check the CUDA path.
 * Only the tests, the smoke check and the benchmark's CPU-baseline arm may
 * load this code; the product library never links or calls it.
 *
 * The result being checked is the paper's neighbor-search problem (Sec. 1,
 * Fig. 1a; Sec. 4 first paragraph): for each particle i, every particle j != i
 * (a particle is not its own neighbor, Sec. 2.1 Fig. 2 caption) within the
 * list radius under periodic boundary conditions, saved as a Verlet list.
 * The paper accepts false positives (Sec. 2.3); the exact list is the set it
 * over-approximates, with the leaf filter the paper allows ("filtered or
 * rejected in a later stage", Sec. 2.3).
 *
 * The distance decision is fixed as one FP32 expression (built with
 * -ffp-contract=off, no fast-math):
 *     dx = xj - xi;   dx = dx - L * rintf(dx * Linv);     (same for y, z)
 *     d2 = (dx*dx + dy*dy) + dz*dz;     j in N(i)  iff  d2 < rl2
 * with Linv = 1.0f / L and rl2 = rl * rl computed once in FP32.
 *
 * Functions:
 *   or_nlist_brute  O(N^2) over all pairs.
 *   or_nlist_cell   27-cell stencil over a uniform cell list (Sec. 1, Fig. 1b),
 *                   same decision expression; falls back to brute force when
 *                   fewer than 3 cells fit per axis.
 *   or_band_check   FP64 confirmation: outside a relative band around the
 *                   list radius, the FP32 decision must equal the exact one.
 *
 * Rows are written sorted ascending; counts[i] is the full neighbor count even
 * when it exceeds cap (rows then hold the first cap neighbors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* FP32 minimum-image squared distance, the pinned decision expression. */
static inline float mi_d2(const float *xi, const float *xj, float L, float Linv)
{
    float dx = xj[0] - xi[0];
    float dy = xj[1] - xi[1];
    float dz = xj[2] - xi[2];
    dx = dx - L * rintf(dx * Linv);
    dy = dy - L * rintf(dy * Linv);
    dz = dz - L * rintf(dz * Linv);
    return (dx * dx + dy * dy) + dz * dz;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/*
 * pos   [n][3] float32, types [n] in [0, nt), rl [nt][nt] list radii.
 * rows  [n][cap] int32 out, counts [n] int32 out.
 */
int or_nlist_brute(int n, const float *pos, const int *types, float L, int nt,
                   const float *rl, int cap, int *rows, int *counts)
{
    float Linv = 1.0f / L;
    float rl2[64];
    if (nt < 1 || nt > 8) return -1;
    for (int k = 0; k < nt * nt; ++k) rl2[k] = rl[k] * rl[k];
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        const float *xi = pos + 3 * (size_t)i;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            float d2 = mi_d2(xi, pos + 3 * (size_t)j, L, Linv);
            if (d2 < rl2[types[i] * nt + types[j]]) {
                if (c < cap) rows[(size_t)i * cap + c] = j;
                ++c;
            }
        }
        counts[i] = c;
        /* j ascends in the loop, so the row is already sorted. */
    }
    return 0;
}

/* Uniform cell grid shared by the cell-list oracle and the FP64 band check. */
typedef struct {
    int nc;          /* cells per axis */
    float inv_w;     /* nc / L */
    int *start;      /* [nc^3 + 1] */
    int *list;       /* [n] particle ids grouped by cell, ascending inside a cell */
} grid_t;

static int cell_coord(float x, const grid_t *g)
{
    int c = (int)floorf(x * g->inv_w);
    if (c < 0) c = 0;
    if (c >= g->nc) c = g->nc - 1;
    return c;
}

static int cell_of(const float *x, const grid_t *g)
{
    int cx = cell_coord(x[0], g), cy = cell_coord(x[1], g), cz = cell_coord(x[2], g);
    return (cx * g->nc + cy) * g->nc + cz;
}

/* Cells at least rmax wide with a 0.1% margin that absorbs binning round-off. */
static int grid_build(grid_t *g, int n, const float *pos, float L, float rmax)
{
    double w = (double)rmax * 1.001;
    int nc = (int)floor((double)L / w);
    if (nc < 3) return -1;
    if (nc > 1024) nc = 1024;
    g->nc = nc;
    g->inv_w = (float)nc / L;
    size_t ncell = (size_t)nc * nc * nc;
    g->start = (int *)calloc(ncell + 1, sizeof(int));
    g->list = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cid = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!g->start || !g->list || !cid) { free(cid); return -2; }
    for (int i = 0; i < n; ++i) {
        cid[i] = cell_of(pos + 3 * (size_t)i, g);
        g->start[cid[i] + 1]++;
    }
    for (size_t c = 0; c < ncell; ++c) g->start[c + 1] += g->start[c];
    int *fill = (int *)malloc(sizeof(int) * ncell);
    memcpy(fill, g->start, sizeof(int) * ncell);
    for (int i = 0; i < n; ++i) g->list[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
    return 0;
}

static void grid_free(grid_t *g)
{
    free(g->start);
    free(g->list);
}

int or_nlist_cell(int n, const float *pos, const int *types, float L, int nt,
                  const float *rl, int cap, int *rows, int *counts)
{
    float rmax = 0.0f;
    if (nt < 1 || nt > 8) return -1;
    for (int k = 0; k < nt * nt; ++k) rmax = rl[k] > rmax ? rl[k] : rmax;
    grid_t g;
    if (grid_build(&g, n, pos, L, rmax) != 0)
        return or_nlist_brute(n, pos, types, L, nt, rl, cap, rows, counts);
    float Linv = 1.0f / L;
    float rl2[64];
    for (int k = 0; k < nt * nt; ++k) rl2[k] = rl[k] * rl[k];
    int nc = g.nc;
    int err = 0;
#pragma omp parallel
    {
        int tmp_cap = 4096;
        int *tmp = (int *)malloc(sizeof(int) * tmp_cap);
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            const float *xi = pos + 3 * (size_t)i;
            int cx = cell_coord(xi[0], &g), cy = cell_coord(xi[1], &g), cz = cell_coord(xi[2], &g);
            int c = 0;
            for (int ox = -1; ox <= 1; ++ox)
                for (int oy = -1; oy <= 1; ++oy)
                    for (int oz = -1; oz <= 1; ++oz) {
                        int ax = (cx + ox + nc) % nc, ay = (cy + oy + nc) % nc, az = (cz + oz + nc) % nc;
                        int cell = (ax * nc + ay) * nc + az;
                        for (int p = g.start[cell]; p < g.start[cell + 1]; ++p) {
                            int j = g.list[p];
                            if (j == i) continue;
                            float d2 = mi_d2(xi, pos + 3 * (size_t)j, L, Linv);
                            if (d2 < rl2[types[i] * nt + types[j]]) {
                                if (c == tmp_cap) {
                                    tmp_cap *= 2;
                                    tmp = (int *)realloc(tmp, sizeof(int) * tmp_cap);
                                }
                                tmp[c++] = j;
                            }
                        }
                    }
            qsort(tmp, (size_t)c, sizeof(int), cmp_int);
            /* with nc >= 3 the 27 cells are distinct, so no j repeats */
            for (int k = 0; k < c && k < cap; ++k) rows[(size_t)i * cap + k] = tmp[k];
            counts[i] = c;
        }
        free(tmp);
    }
    grid_free(&g);
    return err;
}

/*
 * FP64 check of an FP32 neighbor list.  For each row i in `sample` (all rows
 * when sample == NULL), the exact FP64 minimum-image distance d64 of every j
 * is compared with the list: a pair with d64 < rl*(1-band) must be listed, a
 * listed pair must have d64 < rl*(1+band).  Pairs inside the band are not
 * judged.  Returns the number of violations (missed + spurious); the first
 * few offending (i, j) pairs go to bad[2*k], bad[2*k+1].
 */
long or_band_check(int n, const float *pos, const int *types, float L, int nt,
                   const float *rl, double band, int cap, const int *rows,
                   const int *counts, int n_sample, const int *sample,
                   int max_bad, int *bad)
{
    float rmax = 0.0f;
    for (int k = 0; k < nt * nt; ++k) rmax = rl[k] > rmax ? rl[k] : rmax;
    grid_t g;
    int use_grid = grid_build(&g, n, pos, L, (float)(rmax * (1.0 + 4 * band) + 1e-4f)) == 0;
    double Ld = (double)L;
    long nbad = 0;
    int nlog = 0;
    int rows_to_check = sample ? n_sample : n;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nbad)
    for (int s = 0; s < rows_to_check; ++s) {
        int i = sample ? sample[s] : s;
        const float *xi = pos + 3 * (size_t)i;
        int ci = counts[i] < cap ? counts[i] : cap;
        const int *row = rows + (size_t)i * cap;
        /* every listed j: not spurious */
        for (int k = 0; k < ci; ++k) {
            int j = row[k];
            double r = (double)rl[types[i] * nt + types[j]];
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double d = (double)pos[3 * (size_t)j + a] - (double)xi[a];
                d -= Ld * rint(d / Ld);
                d2 += d * d;
            }
            if (j == i || sqrt(d2) >= r * (1.0 + band)) {
#pragma omp critical
                {
                    if (nlog < max_bad && bad) { bad[2 * nlog] = i; bad[2 * nlog + 1] = j; nlog++; }
                }
                nbad++;
            }
        }
        /* every j with d64 clearly inside: listed */
        int cx = 0, cy = 0, cz = 0, span = 1, nc = 1;
        if (use_grid) {
            nc = g.nc;
            cx = cell_coord(xi[0], &g); cy = cell_coord(xi[1], &g); cz = cell_coord(xi[2], &g);
        }
        for (int ox = -span; ox <= span; ++ox)
            for (int oy = -span; oy <= span; ++oy)
                for (int oz = -span; oz <= span; ++oz) {
                    int p0, p1;
                    if (use_grid) {
                        int ax = (cx + ox + nc) % nc, ay = (cy + oy + nc) % nc, az = (cz + oz + nc) % nc;
                        int cell = (ax * nc + ay) * nc + az;
                        p0 = g.start[cell]; p1 = g.start[cell + 1];
                    } else {
                        if (ox || oy || oz) continue;
                        p0 = 0; p1 = n;
                    }
                    for (int p = p0; p < p1; ++p) {
                        int j = use_grid ? g.list[p] : p;
                        if (j == i) continue;
                        double r = (double)rl[types[i] * nt + types[j]];
                        double d2 = 0.0;
                        for (int a = 0; a < 3; ++a) {
                            double d = (double)pos[3 * (size_t)j + a] - (double)xi[a];
                            d -= Ld * rint(d / Ld);
                            d2 += d * d;
                        }
                        if (sqrt(d2) < r * (1.0 - band)) {
                            int found = 0;
                            for (int k = 0; k < ci; ++k)
                                if (row[k] == j) { found = 1; break; }
                            if (!found && counts[i] <= cap) {
#pragma omp critical
                                {
                                    if (nlog < max_bad && bad) { bad[2 * nlog] = i; bad[2 * nlog + 1] = j; nlog++; }
                                }
                                nbad++;
                            }
                        }
                    }
                }
    }
    if (use_grid) grid_free(&g);
    return nbad;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
