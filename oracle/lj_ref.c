/*
 * CPU ORACLE -- test infrastructure only (never linked into the product).
 *
 * FP64 truncated-and-shifted Lennard-Jones energy over a given neighbor list,
 * with forces and gradients with respect to the per-type-pair parameters.
 *
 * Pair potential, Eq. 1 of the paper, truncated and shifted to zero at r_c
 * (Sec. 1):
 *     phi(r)  = 4 eps [ (sig/r)^12 - (sig/r)^6 ]
 *     u(r)    = phi(r) - phi(r_c)      for r < r_c,   0 otherwise.
 * Total energy over a full (i,j and j,i) list:
 *     U = 1/2 sum_i sum_{j in N(i)} u(r_ij; eps[t_i][t_j], sig[t_i][t_j], rc[t_i][t_j])
 * Derived quantities (all in FP64):
 *     F_i          = -dU/dx_i = sum_j 24 eps (2 s^2 - s) / r^2 * (x_i - x_j),  s = (sig/r)^6
 *     dU/deps[a][b] = 1/2 sum_{i: t_i=a} sum_{j: t_j=b} u / eps
 *     dU/dsig[a][b] = 1/2 sum_{i: t_i=a} sum_{j: t_j=b}
 *                      (24 eps / sig) [ (2 s^2 - s) - (2 s_c^2 - s_c) ],  s_c = (sig/r_c)^6
 * (each matrix entry is its own parameter; a symmetric model sums the [a][b]
 * and [b][a] entries.)
 *
 * Which pairs interact is decided with the same FP32 minimum-image expression
 * as the neighbor list (d2 < fl(rc*rc) on the float32 positions `pos32`), so
 * that the comparison with an FP32 kernel measures arithmetic error only; the
 * values are then computed in FP64 from `pos64` (pos32 promoted, or perturbed
 * copies for finite differences, where the pair set must stay fixed).
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

static inline float mi_d2_f(const float *xi, const float *xj, float L, float Linv)
{
    float dx = xj[0] - xi[0];
    float dy = xj[1] - xi[1];
    float dz = xj[2] - xi[2];
    dx = dx - L * rintf(dx * Linv);
    dy = dy - L * rintf(dy * Linv);
    dz = dz - L * rintf(dz * Linv);
    return (dx * dx + dy * dy) + dz * dz;
}

/*
 * Outputs may be NULL.  U[0] total energy, e[n] per-particle energy
 * (1/2 of its row), F[n][3] forces, dE/dS [nt][nt] parameter gradients.
 */
int or_lj_fp64(int n, const float *pos32, const double *pos64, const int *types, float L,
               int nt, const double *eps, const double *sig, const float *rcut, int cap,
               const int *rows, const int *counts, double *U, double *e, double *F,
               double *dE, double *dS)
{
    if (nt < 1 || nt > 8) return -1;
    float Linv = 1.0f / L;
    double Ld = (double)L;
    float rc2f[64];
    double sc6[64], phic[64];
    for (int k = 0; k < nt * nt; ++k) {
        rc2f[k] = rcut[k] * rcut[k];
        double rc = (double)rcut[k];
        double s2 = (sig[k] * sig[k]) / (rc * rc);
        sc6[k] = s2 * s2 * s2;
        phic[k] = 4.0 * eps[k] * (sc6[k] * sc6[k] - sc6[k]);
    }
    double Utot = 0.0;
    double gE[64], gS[64];
    memset(gE, 0, sizeof gE);
    memset(gS, 0, sizeof gS);
    for (int i = 0; i < n; ++i) {
        int ti = types[i];
        int c = counts[i] < cap ? counts[i] : cap;
        double ei = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        const int *row = rows + (size_t)i * cap;
        for (int k = 0; k < c; ++k) {
            int j = row[k];
            int p = ti * nt + types[j];
            if (!(mi_d2_f(pos32 + 3 * (size_t)i, pos32 + 3 * (size_t)j, L, Linv) < rc2f[p]))
                continue;
            double d[3];
            for (int a = 0; a < 3; ++a) {
                double v = pos64[3 * (size_t)j + a] - pos64[3 * (size_t)i + a];
                d[a] = v - Ld * rint(v / Ld);
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double s2 = (sig[p] * sig[p]) / r2;
            double s6 = s2 * s2 * s2;
            double u = 4.0 * eps[p] * (s6 * s6 - s6) - phic[p];
            double w = 24.0 * eps[p] * (2.0 * s6 * s6 - s6) / r2;
            ei += 0.5 * u;
            fx -= w * d[0];
            fy -= w * d[1];
            fz -= w * d[2];
            gE[p] += 0.5 * u / eps[p];
            gS[p] += 0.5 * (24.0 * eps[p] / sig[p]) *
                     ((2.0 * s6 * s6 - s6) - (2.0 * sc6[p] * sc6[p] - sc6[p]));
        }
        Utot += ei;
        if (e) e[i] = ei;
        if (F) {
            F[3 * (size_t)i] = fx;
            F[3 * (size_t)i + 1] = fy;
            F[3 * (size_t)i + 2] = fz;
        }
    }
    if (U) U[0] = Utot;
    for (int k = 0; k < nt * nt; ++k) {
        if (dE) dE[k] = gE[k];
        if (dS) dS[k] = gS[k];
    }
    return 0;
}
