/*
 * CPU ORACLE -- test infrastructure only (never linked into the product).
 *
 * Reference construction of the quantized linear BVH, step by step in the
 * order the paper gives them (Sec. 2.1, Sec. 2.2, Fig. 3):
 *
 *   1. Morton binning: each axis of the box is cut into 2^10 - 1 bins, the
 *      10-bit bin coordinates are interleaved into a 30-bit code (Sec. 2.1).
 *   2. Sort along the Z-order curve (Sec. 2.1), stable: equal codes keep
 *      input order (Sec. 3 asks for a deterministic, stable sort).
 *   3. Hierarchy: the radix tree of the sorted keys, written here as its plain
 *      recursive definition -- a range of sorted leaves is split where the
 *      highest bit differing between its first and last key turns from 0 to 1;
 *      equal codes are told apart by their sorted position.  This is the tree
 *      Karras's parallel construction (cited in Sec. 2.1) builds: N-1
 *      internal nodes, each with exactly two children.
 *   4. Fit: every node's AABB is the min/max over the particles below it.
 *   5. Ropes (Sec. 2.1, stackless traversal): the rope of a node is the node
 *      visited next in pre-order once its subtree is skipped; computed here
 *      by a depth-first walk (left child's rope = right sibling, right child's
 *      rope = parent's rope, root's rope = end).
 *   6. Quantization (Sec. 2.2, Fig. 3b,c): the root AABB is split into 2^10 - 1
 *      bins per axis; lower bounds are rounded down and upper bounds up onto
 *      the 1024 bin edges 0..1023, three 10-bit values packed per 32-bit word.
 *      Directed rounding uses the IEEE round-down / round-up modes (Sec. 3),
 *      selected here with fesetround().
 *
 * Where the paper leaves a detail open, this file takes these readings:
 *   - bin index b = min((int)(x * fl(1023 / L)), 1022), x in [0, L);
 *   - code bit 3k+2 = x_k, 3k+1 = y_k, 3k = z_k (x most significant);
 *   - frame of quantization: the fitted root AABB [R_lo, R_hi] of each tree;
 *     h = max(fl_up((R_hi - R_lo) / 1023), FLT_MIN) per axis,
 *     q_lo = floor(fl_down(fl_down(lo - R_lo) / h)),
 *     q_hi = ceil(fl_up(fl_up(hi - R_lo) / h)), both clamped to [0, 1023];
 *   - packed word = qx << 20 | qy << 10 | qz, bits 30-31 free;
 *   - indices: internal node k >= 0, leaf k stored as ~k (negative, Fig. 3 /
 *     Sec. 2.2 sign convention), end of traversal = INT32_MIN;
 *   - node numbering: root = first leaf of its tree, a left child takes the
 *     index of its last leaf, a right child the index of its first leaf
 *     (Karras's numbering), so internal slot k of every tree's last leaf is
 *     unused;
 *   - node word layout (16 bytes, Fig. 3b):
 *       x = packed lo | (bundle << 31), y = packed hi,
 *       z = left child id, or for a bundle node its first leaf index,
 *       w = rope id;
 *     a bundle node is an internal node with at most K leaves (K >= 2); a
 *     traversal that reaches it tests its leaves directly instead of
 *     descending (the subtree collapse Sec. 2.3 proposes);
 *   - leaf word: x, y, z = position, w = original index | (rope is an
 *     internal node) << 31.
 *
 * Several trees ("segments") are built at once: segment s holds the particles
 * with seg[i] == s, binned in a cubic box of edge Lseg[s].
 */
#include <fenv.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#pragma STDC FENV_ACCESS ON

#define OR_END ((int32_t)0x80000000)

static uint32_t interleave3(uint32_t bx, uint32_t by, uint32_t bz)
{
    uint32_t code = 0;
    for (int k = 0; k < 10; ++k) {
        code |= ((bx >> k) & 1u) << (3 * k + 2);
        code |= ((by >> k) & 1u) << (3 * k + 1);
        code |= ((bz >> k) & 1u) << (3 * k);
    }
    return code;
}

static uint32_t bin_of(float x, float s)
{
    int b = (int)(x * s);
    if (b < 0) b = 0;
    if (b > 1022) b = 1022;
    return (uint32_t)b;
}

/* Morton code of every particle in input order. */
void or_morton(int n, const float *pos, const int *seg, const float *Lseg, uint32_t *codes)
{
    for (int i = 0; i < n; ++i) {
        float s = 1023.0f / Lseg[seg[i]];
        const float *x = pos + 3 * (size_t)i;
        codes[i] = interleave3(bin_of(x[0], s), bin_of(x[1], s), bin_of(x[2], s));
    }
}

typedef struct {
    int seg;
    uint32_t code;
    int idx;
} key_t_;

static int cmp_key(const void *a, const void *b)
{
    const key_t_ *p = (const key_t_ *)a, *q = (const key_t_ *)b;
    if (p->seg != q->seg) return p->seg < q->seg ? -1 : 1;
    if (p->code != q->code) return p->code < q->code ? -1 : 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

/* ---- recursive hierarchy ------------------------------------------------ */

typedef struct {
    const uint32_t *code;   /* sorted codes */
    int32_t *left, *right;  /* child ids of internal node k */
    int32_t *first, *last;  /* leaf range of internal node k */
    int32_t *rope_int;      /* rope of internal node k */
    int32_t *rope_leaf;     /* rope of leaf k */
} tree_t;

static int highest_bit(uint32_t v)
{
    int b = 31;
    while (b >= 0 && !((v >> b) & 1u)) --b;
    return b;
}

/* Split of sorted range [f, l] (f < l): last index of the left half. */
static int split_of(const uint32_t *code, int f, int l)
{
    if (code[f] != code[l]) {
        int b = highest_bit(code[f] ^ code[l]);
        int g = f;
        while (g + 1 <= l && !((code[g + 1] >> b) & 1u)) ++g;
        return g;
    }
    /* equal codes: the sorted positions themselves are the distinguishing key */
    int b = highest_bit((uint32_t)f ^ (uint32_t)l);
    int g = f;
    while (g + 1 <= l && !(((uint32_t)(g + 1) >> b) & 1u)) ++g;
    return g;
}

/* Build the subtree over [f, l] with Karras id `id`, set its rope; returns id. */
static void build_rec(tree_t *t, int f, int l, int id, int32_t rope)
{
    if (f == l) {
        t->rope_leaf[f] = rope;
        return;
    }
    int g = split_of(t->code, f, l);
    int32_t lid = (g == f) ? ~g : g;           /* left child [f, g] */
    int32_t rid = (g + 1 == l) ? ~(g + 1) : g + 1; /* right child [g+1, l] */
    t->left[id] = lid;
    t->right[id] = rid;
    t->first[id] = f;
    t->last[id] = l;
    t->rope_int[id] = rope;
    build_rec(t, f, g, g, rid);        /* left child's rope = right sibling */
    build_rec(t, g + 1, l, g + 1, rope); /* right child's rope = parent's rope */
}

/* ---- directed-rounding helpers (mode set by the caller) ------------------ */

static float v_sub(float a, float b)
{
    volatile float x = a, y = b;
    volatile float r = x - y;
    return r;
}

static float v_div(float a, float b)
{
    volatile float x = a, y = b;
    volatile float r = x / y;
    return r;
}

/*
 * Build all trees.
 *   n, pos [n][3], seg [n] in [0, n_seg), Lseg [n_seg], bundle_k (<= 1: none)
 * outputs:
 *   codes   [n]       Morton code per particle (input order)
 *   order   [n]       sorted position -> original index
 *   seg_start [n_seg+1]
 *   nodes   [n][4]    int32 internal node words (unused slots zero)
 *   leaves  [n][4]    float32 leaf words (w holds int bits)
 *   root    [n_seg][6] fitted root AABB lo xyz, hi xyz (zeros for empty trees)
 *   frame   [n_seg][6] quantization frame R_lo xyz, h xyz
 * Returns 0, or -1 on bad input.
 */
int or_lbvh_build(int n, const float *pos, const int *seg, int n_seg, const float *Lseg,
                  int bundle_k, uint32_t *codes, int32_t *order, int32_t *seg_start,
                  int32_t *nodes, float *leaves, float *root, float *frame)
{
    if (n < 0 || n_seg < 1) return -1;
    for (int i = 0; i < n; ++i)
        if (seg[i] < 0 || seg[i] >= n_seg) return -1;
    or_morton(n, pos, seg, Lseg, codes);

    key_t_ *keys = (key_t_ *)malloc(sizeof(key_t_) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        keys[i].seg = seg[i];
        keys[i].code = codes[i];
        keys[i].idx = i;
    }
    qsort(keys, (size_t)n, sizeof(key_t_), cmp_key);

    uint32_t *scode = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n; ++k) {
        order[k] = keys[k].idx;
        scode[k] = keys[k].code;
    }
    for (int s = 0; s <= n_seg; ++s) seg_start[s] = 0;
    for (int k = 0; k < n; ++k) seg_start[keys[k].seg + 1]++;
    for (int s = 0; s < n_seg; ++s) seg_start[s + 1] += seg_start[s];

    size_t nn = (size_t)(n > 0 ? n : 1);
    tree_t t;
    t.code = scode;
    t.left = (int32_t *)calloc(nn, 4);
    t.right = (int32_t *)calloc(nn, 4);
    t.first = (int32_t *)calloc(nn, 4);
    t.last = (int32_t *)calloc(nn, 4);
    t.rope_int = (int32_t *)calloc(nn, 4);
    t.rope_leaf = (int32_t *)calloc(nn, 4);
    float *lo = (float *)calloc(nn * 3, 4), *hi = (float *)calloc(nn * 3, 4);

    memset(nodes, 0, sizeof(int32_t) * 4 * (size_t)n);
    memset(root, 0, sizeof(float) * 6 * (size_t)n_seg);
    memset(frame, 0, sizeof(float) * 6 * (size_t)n_seg);

    for (int s = 0; s < n_seg; ++s) {
        int a = seg_start[s], b = seg_start[s + 1] - 1;
        if (b < a) continue;
        if (a == b) {
            t.rope_leaf[a] = OR_END;
        } else {
            build_rec(&t, a, b, a, OR_END);
        }
        /* fit: min/max of the particle positions under each internal node */
        float rlo[3], rhi[3];
        for (int d = 0; d < 3; ++d) {
            rlo[d] = INFINITY;
            rhi[d] = -INFINITY;
        }
        for (int k = a; k <= b; ++k)
            for (int d = 0; d < 3; ++d) {
                float x = pos[3 * (size_t)order[k] + d];
                rlo[d] = fminf(rlo[d], x);
                rhi[d] = fmaxf(rhi[d], x);
            }
        for (int k = a; k < b; ++k) {
            for (int d = 0; d < 3; ++d) {
                float mn = INFINITY, mx = -INFINITY;
                for (int m = t.first[k]; m <= t.last[k]; ++m) {
                    float x = pos[3 * (size_t)order[m] + d];
                    mn = fminf(mn, x);
                    mx = fmaxf(mx, x);
                }
                lo[3 * (size_t)k + d] = mn;
                hi[3 * (size_t)k + d] = mx;
            }
        }
        /* quantization frame of this tree */
        float h[3];
        fesetround(FE_UPWARD);
        for (int d = 0; d < 3; ++d) {
            h[d] = v_div(v_sub(rhi[d], rlo[d]), 1023.0f);
        }
        fesetround(FE_TONEAREST);
        for (int d = 0; d < 3; ++d) {
            if (!(h[d] >= FLT_MIN)) h[d] = FLT_MIN;
            root[6 * s + d] = rlo[d];
            root[6 * s + 3 + d] = rhi[d];
            frame[6 * s + d] = rlo[d];
            frame[6 * s + 3 + d] = h[d];
        }
        /* outward quantization of every internal node */
        for (int k = a; k < b; ++k) {
            uint32_t qlo[3], qhi[3];
            fesetround(FE_DOWNWARD);
            for (int d = 0; d < 3; ++d) {
                float v = v_div(v_sub(lo[3 * (size_t)k + d], rlo[d]), h[d]);
                long q = (long)floorf(v);
                qlo[d] = (uint32_t)(q < 0 ? 0 : (q > 1023 ? 1023 : q));
            }
            fesetround(FE_UPWARD);
            for (int d = 0; d < 3; ++d) {
                float v = v_div(v_sub(hi[3 * (size_t)k + d], rlo[d]), h[d]);
                long q = (long)ceilf(v);
                qhi[d] = (uint32_t)(q < 0 ? 0 : (q > 1023 ? 1023 : q));
            }
            fesetround(FE_TONEAREST);
            uint32_t plo = qlo[0] << 20 | qlo[1] << 10 | qlo[2];
            uint32_t phi = qhi[0] << 20 | qhi[1] << 10 | qhi[2];
            int count = t.last[k] - t.first[k] + 1;
            int bundle = (bundle_k >= 2 && count <= bundle_k);
            int32_t *w = nodes + 4 * (size_t)k;
            w[0] = (int32_t)(plo | ((uint32_t)bundle << 31));
            w[1] = (int32_t)phi;
            w[2] = bundle ? t.first[k] : t.left[k];
            w[3] = t.rope_int[k];
        }
        for (int k = a; k <= b; ++k) {
            float *w = leaves + 4 * (size_t)k;
            const float *x = pos + 3 * (size_t)order[k];
            w[0] = x[0];
            w[1] = x[1];
            w[2] = x[2];
            uint32_t tag = (uint32_t)order[k] | ((t.rope_leaf[k] >= 0 ? 1u : 0u) << 31);
            memcpy(&w[3], &tag, 4);
        }
    }
    /* export child ids and ranges for the structural checks */
    free(keys);
    free(scode);
    free(t.left);
    free(t.right);
    free(t.first);
    free(t.last);
    free(t.rope_int);
    free(t.rope_leaf);
    free(lo);
    free(hi);
    return 0;
}

/*
 * Structural view of the same trees for the invariant tests: per internal
 * slot k the child ids, leaf range and rope; per leaf its rope.
 */
int or_lbvh_topology(int n, const float *pos, const int *seg, int n_seg, const float *Lseg,
                     int32_t *left, int32_t *right, int32_t *first, int32_t *last,
                     int32_t *rope_int, int32_t *rope_leaf, int32_t *order, int32_t *seg_start)
{
    if (n < 0 || n_seg < 1) return -1;
    uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    or_morton(n, pos, seg, Lseg, codes);
    key_t_ *keys = (key_t_ *)malloc(sizeof(key_t_) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        keys[i].seg = seg[i];
        keys[i].code = codes[i];
        keys[i].idx = i;
    }
    qsort(keys, (size_t)n, sizeof(key_t_), cmp_key);
    uint32_t *scode = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n; ++k) {
        order[k] = keys[k].idx;
        scode[k] = keys[k].code;
    }
    for (int s = 0; s <= n_seg; ++s) seg_start[s] = 0;
    for (int k = 0; k < n; ++k) seg_start[keys[k].seg + 1]++;
    for (int s = 0; s < n_seg; ++s) seg_start[s + 1] += seg_start[s];
    tree_t t = {scode, left, right, first, last, rope_int, rope_leaf};
    for (int k = 0; k < n; ++k) {
        left[k] = right[k] = first[k] = last[k] = rope_int[k] = 0;
        rope_leaf[k] = 0;
    }
    for (int s = 0; s < n_seg; ++s) {
        int a = seg_start[s], b = seg_start[s + 1] - 1;
        if (b < a) continue;
        if (a == b)
            rope_leaf[a] = OR_END;
        else
            build_rec(&t, a, b, a, OR_END);
    }
    free(codes);
    free(keys);
    free(scode);
    return 0;
}

/*
 * Quantize one AABB against a frame onto the bin edges 0..qmax (qmax = 1023
 * for the 10-bit words of Fig. 3b, 2^21 - 1 for 21-bit words: the bit width
 * that trades node size against false positives, Sec. 2.2), lower bound
 * rounded down and upper bound up as above.
 */
void or_quantize_box_q(const float *lo, const float *hi, const float *R_lo, const float *h, long qmax,
                       uint32_t *qlo, uint32_t *qhi)
{
    fesetround(FE_DOWNWARD);
    for (int d = 0; d < 3; ++d) {
        long q = (long)floorf(v_div(v_sub(lo[d], R_lo[d]), h[d]));
        qlo[d] = (uint32_t)(q < 0 ? 0 : (q > qmax ? qmax : q));
    }
    fesetround(FE_UPWARD);
    for (int d = 0; d < 3; ++d) {
        long q = (long)ceilf(v_div(v_sub(hi[d], R_lo[d]), h[d]));
        qhi[d] = (uint32_t)(q < 0 ? 0 : (q > qmax ? qmax : q));
    }
    fesetround(FE_TONEAREST);
}

/* The 10-bit case, exposed for the containment tests. */
void or_quantize_box(const float *lo, const float *hi, const float *R_lo, const float *h,
                     uint32_t *qlo, uint32_t *qhi)
{
    or_quantize_box_q(lo, hi, R_lo, h, 1023, qlo, qhi);
}

/* Bin width of a frame with qmax bins per axis: (R_hi - R_lo) / qmax rounded
 * up, at least the smallest normal float (a root of zero width). */
void or_frame_width(const float *R_lo, const float *R_hi, long qmax, float *h)
{
    fesetround(FE_UPWARD);
    for (int d = 0; d < 3; ++d) h[d] = v_div(v_sub(R_hi[d], R_lo[d]), (float)qmax);
    fesetround(FE_TONEAREST);
    for (int d = 0; d < 3; ++d)
        if (!(h[d] >= FLT_MIN)) h[d] = FLT_MIN;
}

/*
 * Decompression of quantized bounds back to FP32 (Alg. 1, decode before the
 * overlap test): lower edge rounded down, upper edge rounded up, each as one
 * fused multiply-add q*h + R_lo in the directed mode.
 */
void or_dequantize(const uint32_t *qlo, const uint32_t *qhi, const float *R_lo, const float *h,
                   float *lo, float *hi)
{
    fesetround(FE_DOWNWARD);
    for (int d = 0; d < 3; ++d) {
        volatile float q = (float)qlo[d], hh = h[d], r = R_lo[d];
        volatile float v = fmaf(q, hh, r);
        lo[d] = v;
    }
    fesetround(FE_UPWARD);
    for (int d = 0; d < 3; ++d) {
        volatile float q = (float)qhi[d], hh = h[d], r = R_lo[d];
        volatile float v = fmaf(q, hh, r);
        hi[d] = v;
    }
    fesetround(FE_TONEAREST);
}
