/*
 * CPU ORACLE -- test infrastructure only (never linked into the product).
 *
 * Candidate lists of Alg. 1 as written, without the exact leaf filter: the
 * paper lists every particle whose quantized leaf box the search sphere
 * overlaps and leaves false positives to a later stage (Sec. 2.3); how many
 * depends on the precision of the leaf boxes (10-bit, 21-bit, or the FP32
 * point, Sec. 2.2).  Written here as the plain set the rope walk reaches, by
 * brute force over all leaves:
 *
 *   for particle i of type a, every tree b (the particles of type b) with
 *   r = r_list[a][b] > 0, and every periodic image n in {-1, 0, 1}^3
 *   (Sec. 2.3, the 27-bit image set):
 *     - the image is walked when the padded sphere around fl(x_i + n L)
 *       overlaps tree b's root AABB (the exact FP32 min/max of its points);
 *     - leaf j != i of tree b is listed once for that image when the padded
 *       sphere overlaps j's leaf box, quantized outward against the tree's
 *       frame and decoded outward (Sec. 2.2, Fig. 3b, Alg. 1).
 *
 * With quantized nodes every ancestor's decoded box contains the leaf's, and
 * the overlap test below is monotone in the box, so the walk reaches exactly
 * these leaves.
 *
 * Readings of the paper taken here (the paper fixes neither the padding nor
 * the rounding of the overlap tests):
 *   - padded radius rs = up(fl64(r (1 + 2^-20) + 2^-19 L)), rs2 = up(rs * rs),
 *     products formed in FP64 and rounded up to FP32;
 *   - image test against the root box: per axis the gap
 *     g = max(rd(lo - p), rd(p - hi), 0), then
 *     d2 = fma_rd(gx, gx, fma_rd(gy, gy, rd(gz * gz))), walked iff d2 <= rs2;
 *   - leaf test (Eq. 2, nearest point of the box): y = clamp(p, lo', hi') per
 *     axis, d = rz(p - y), d2 = fma_rz(dz, dz, rz(rz(dx * dx) + rz(dy * dy))),
 *     listed iff d2 <= rs2.
 * Both distances are rounded toward zero (rd equals rz on the non-negative
 * gaps), so neither test can reject a box the sphere overlaps in exact
 * arithmetic.
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

void or_quantize_box_q(const float *lo, const float *hi, const float *R_lo, const float *h, long qmax,
                       uint32_t *qlo, uint32_t *qhi);
void or_frame_width(const float *R_lo, const float *R_hi, long qmax, float *h);
void or_dequantize(const uint32_t *qlo, const uint32_t *qhi, const float *R_lo, const float *h,
                   float *lo, float *hi);

/* one operation in the caller's rounding mode, kept from being folded */
static float c_add(float a, float b) { volatile float x = a, y = b; volatile float r = x + y; return r; }
static float c_sub(float a, float b) { volatile float x = a, y = b; volatile float r = x - y; return r; }
static float c_mul(float a, float b) { volatile float x = a, y = b; volatile float r = x * y; return r; }
static float c_fma(float a, float b, float c)
{
    volatile float x = a, y = b, z = c;
    volatile float r = fmaf(x, y, z);
    return r;
}

static float round_up_to_float(double v)
{
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}

/* image test: padded sphere around p against the box [lo, hi] (gap form) */
static int image_overlaps(const float *p, const float *lo, const float *hi, float rs2)
{
    float g[3];
    fesetround(FE_DOWNWARD);
    for (int d = 0; d < 3; ++d) g[d] = fmaxf(fmaxf(c_sub(lo[d], p[d]), c_sub(p[d], hi[d])), 0.f);
    const float d2 = c_fma(g[0], g[0], c_fma(g[1], g[1], c_mul(g[2], g[2])));
    fesetround(FE_TONEAREST);
    return d2 <= rs2;
}

/* leaf test: padded sphere around p against the box [lo, hi] (nearest
 * point); the caller has selected rounding toward zero */
static int leaf_overlaps(const float *p, const float *lo, const float *hi, float rs2)
{
    float dd[3];
    for (int d = 0; d < 3; ++d) dd[d] = c_sub(p[d], fminf(fmaxf(p[d], lo[d]), hi[d]));
    const float d2 = c_fma(dd[2], dd[2], c_add(c_mul(dd[0], dd[0]), c_mul(dd[1], dd[1])));
    return d2 <= rs2;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/*
 * pos [n][3] float32 in [0, L), types [n] in [0, nt), rl [nt][nt] list radii,
 * root [nt][6] (lo xyz, hi xyz) and frame [nt][6] (R_lo xyz, h xyz) of each
 * type's tree as the LBVH build makes them (the 10-bit frame).
 * leaf_bits: precision of the leaf boxes the candidates are tested against:
 *   10 = 10-bit quantized (Fig. 3b, the frame given), 21 = 21-bit quantized
 *   (bin width from the root box with 2^21 - 1 bins, or_frame_width), 0 = the
 *   FP32 point itself (the leaf of an uncompressed tree, Fig. 3a).
 * rows [n][cap] out (sorted ascending, an index repeated once per image that
 * lists it), counts [n] out (full count even past cap).
 * Returns 0, or -1 on bad input.
 */
int or_candidates(int n, const float *pos, const int *types, float L, int nt, const float *rl,
                  const float *root, const float *frame, int leaf_bits, int cap, int *rows, int *counts)
{
    if (n < 0 || nt < 1 || cap < 1 || !(L > 0.f)) return -1;
    if (leaf_bits != 0 && leaf_bits != 10 && leaf_bits != 21) return -1;
    for (int i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= nt) return -1;
    /* decoded leaf boxes */
    float *blo = (float *)malloc(sizeof(float) * 3 * (size_t)(n > 0 ? n : 1));
    float *bhi = (float *)malloc(sizeof(float) * 3 * (size_t)(n > 0 ? n : 1));
    int *cnt_t = (int *)calloc((size_t)nt, sizeof(int));
    if (!blo || !bhi || !cnt_t) {
        free(blo);
        free(bhi);
        free(cnt_t);
        return -1;
    }
    for (int j = 0; j < n; ++j) {
        const float *fr = frame + 6 * types[j];
        const float *x = pos + 3 * (size_t)j;
        cnt_t[types[j]]++;
        if (leaf_bits == 0) {
            for (int d = 0; d < 3; ++d) blo[3 * (size_t)j + d] = bhi[3 * (size_t)j + d] = x[d];
            continue;
        }
        float h[3];
        const long qmax = leaf_bits == 21 ? (1L << 21) - 1 : 1023;
        if (leaf_bits == 21) or_frame_width(root + 6 * types[j], root + 6 * types[j] + 3, qmax, h);
        else for (int d = 0; d < 3; ++d) h[d] = fr[3 + d];
        uint32_t qlo[3], qhi[3];
        or_quantize_box_q(x, x, fr, h, qmax, qlo, qhi);
        or_dequantize(qlo, qhi, fr, h, blo + 3 * (size_t)j, bhi + 3 * (size_t)j);
    }
    /* padded radii and their squares */
    float rs2[64];
    for (int p = 0; p < nt * nt; ++p) {
        const double v = (double)rl[p] * (1.0 + ldexp(1.0, -20)) + ldexp((double)L, -19);
        const float rs = round_up_to_float(v);
        rs2[p] = round_up_to_float((double)rs * (double)rs);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        const int a = types[i];
        int *row = rows + (size_t)i * cap;
        int c = 0;
        for (int b = 0; b < nt; ++b) {
            if (!(rl[a * nt + b] > 0.f) || cnt_t[b] == 0) continue;
            const float r2 = rs2[a * nt + b];
            const float *rlo = root + 6 * b, *rhi = root + 6 * b + 3;
            for (int m = 0; m < 27; ++m) {
                const int sh[3] = {m / 9 - 1, (m / 3) % 3 - 1, m % 3 - 1};
                float p[3];
                for (int d = 0; d < 3; ++d) {
                    const float x = pos[3 * (size_t)i + d];
                    p[d] = sh[d] == 0 ? x : (sh[d] > 0 ? x + L : x - L);   /* round to nearest */
                }
                if (!image_overlaps(p, rlo, rhi, r2)) continue;
                fesetround(FE_TOWARDZERO);
                for (int j = 0; j < n; ++j) {
                    if (j == i || types[j] != b) continue;
                    if (leaf_overlaps(p, blo + 3 * (size_t)j, bhi + 3 * (size_t)j, r2)) {
                        if (c < cap) row[c] = j;
                        ++c;
                    }
                }
                fesetround(FE_TONEAREST);
            }
        }
        counts[i] = c;
        qsort(row, (size_t)(c < cap ? c : cap), sizeof(int), cmp_int);
    }
    free(blo);
    free(bhi);
    free(cnt_t);
    return 0;
}
