// Internal declarations shared by the qbvh CUDA translation units.
//
// Data layout in device memory (all arrays indexed by sorted position k unless
// said otherwise; trees are "segments" of the sorted order, one per
// (system, type)):
//   keys     u32 {type<<30 | morton} or u64 {segment<<30 | morton}
//   order    int32 sorted position -> original index (radix-sort values)
//   range    int2  leaf range [first, last] of internal node k
//   child    int2  {left id, right id} of internal node k
//   par_int  int32 parent of internal node k (-1 at a root)
//   par_leaf int32 parent of leaf k (-1 for a one-particle tree)
//   visit    int32 arrival counter of internal node k (bottom-up fit)
//   leaf_q   uint2 quantized AABB {lo, hi} of leaf k
//   nodes    int4  {lo | bundle<<31, hi, left or first leaf, rope}   (Fig. 3b)
//   nodes32  2 x float4 per internal node, the uncompressed layout of Fig. 3a:
//            {lo.x (sign bit = bundle), lo.y, lo.z, left or first leaf},
//            {hi.x, hi.y, hi.z, rope}; written only when that format is chosen
//   nodes21  2 x int4 per internal node, bounds quantized to 21 bits per axis
//            against the tree's 2^21 - 1 bins: lo64 = qx << 42 | qy << 21 | qz
//            (bit 63 = bundle), hi64 alike, as {lo64 low, lo64 high, hi64 low,
//            hi64 high}, {left or first leaf, rope, 0, 0}; written only when
//            that format is chosen
//   leaves   float4 {x, y, z, original index | rope-is-internal<<31}
// Node ids: k >= 0 internal node k, ~k (negative) leaf k, QBVH_END = INT32_MIN.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define QBVH_END ((int)0x80000000)

// device error word bits
#define QBVH_DEVERR_OUT_OF_BOX 1u
#define QBVH_DEVERR_BAD_TYPE 2u
#define QBVH_DEVERR_TIMEOUT 4u
#define QBVH_DEVERR_INTERNAL 8u

// quantization: 2^10 - 1 bins per axis, bounds on the 1024 bin edges 0..1023
#define QBVH_QMAX 1023
#define QBVH_QMASK 0x3FFFFFFFu
// 21-bit node format: 2^21 - 1 bins per axis, three fields in 63 bits
#define QBVH_QMAX21 2097151
#define QBVH_QMASK21 0x7FFFFFFFFFFFFFFFull

namespace qbvh {

// Packed FP32 pairs (sub/mul .rn.f32x2, sm_100 and later): each half is one
// IEEE round-to-nearest operation, so a pair gives exactly the two scalar
// results.  A leaf's (x, y) already lies in an aligned register pair after
// its 16-byte load, which makes the packing free.  A packed product must not
// feed a packed add where the rounding matters: ptxas contracts that pair
// into a fused multiply-add even with explicit .rn (scalar add.rn is kept).
#ifndef QBVH_F32X2
#define QBVH_F32X2 1
#endif
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}


// ---- Lennard-Jones pair terms (Eq. 1, truncated and shifted) -------------
// Shared by the handle's pass (lj.cu) and the allocation-free pass
// (noalloc.cu), so that both evaluate a pair with the same operations.
//
// Per type pair, from eps, sig and fl(r_c^2):
//   sig2 = sig^2, phic = 4 (s_c^2 - s_c) with s_c = (sig^2 / r_c^2)^3 (the
//   shift per unit eps), dsc = 2 s_c^2 - s_c (its share of dU/dsig).
struct LJParams {
    float eps, sig, sig2, phic, dsc, rc2;
};

__device__ __forceinline__ LJParams lj_params(float eps, float sig, float rc2)
{
    LJParams p;
    p.eps = eps;
    p.sig = sig;
    p.sig2 = sig * sig;
    p.rc2 = rc2;
    const float sc2 = (sig * sig) / rc2;
    const float sc6 = sc2 * sc2 * sc2;
    p.phic = 4.f * (sc6 * sc6 - sc6);
    p.dsc = 2.f * sc6 * sc6 - sc6;
    return p;
}

// 1/r^2: the hardware reciprocal (rcp.approx, at most 1 ulp) or the
// correctly rounded one.  QBVH_LJ_FAST_RCP = 1 (both LJ passes) takes the
// hardware one: FP32 results stay far inside the 1e-5 relative agreement with
// FP64, and the pass at N = 2M measured 0.74 -> 0.68 ms.
#ifndef QBVH_LJ_FAST_RCP
#define QBVH_LJ_FAST_RCP 1
#endif
template <bool FAST>
__device__ __forceinline__ float lj_rcp(float x)
{
    if (FAST) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    return __frcp_rn(x);
}

// The terms of one pair at squared distance r2 < rc2, s = (sig^2 / r2)^3:
//   uE = u / eps = 4 (s^2 - s) - phic          (energy per unit eps)
//   w  = 24 eps (2 s^2 - s) / r2               (F_i += -w d, d = x_j - x_i)
//   gs = (24 eps / sig) ((2 s^2 - s) - dsc)    (dU/dsig of the pair)
struct LJPairTerms {
    float uE, w, gs;
};

template <bool FAST_RCP>
__device__ __forceinline__ LJPairTerms lj_pair_terms(float r2, const LJParams &p)
{
    const float inv_r2 = lj_rcp<FAST_RCP>(r2);
    const float s2 = p.sig2 * inv_r2;
    const float s6 = s2 * s2 * s2;
    LJPairTerms t;
    t.uE = 4.f * (s6 * s6 - s6) - p.phic;
    const float q = 2.f * s6 * s6 - s6;
    t.w = 24.f * p.eps * q * inv_r2;
    t.gs = (24.f * p.eps / p.sig) * (q - p.dsc);
    return t;
}

// Geometry of one pair for the LJ passes.  Whether the pair interacts is
// decided by the pinned FP32 minimum-image expression (the neighbor list's,
// mirrored by the oracle): dx = fl(xj - xi); dx = fl(dx - L rint(dx Linv)),
// r2 = fl(fl(dx^2 + dy^2) + dz^2) < fl(r_cut^2).  The pair's value takes the
// difference rounded once instead.  For n = rint(...) != 0 the expression
// rounds xj - xi at the magnitude of L before the shift: an absolute error up
// to ulp(L) / 2 on a distance below r_cut, which the steep repulsion turns
// into force errors of 1e-5 relative (two-type workload, 32 x 65,536,
// measured 7.4e-6 normwise).  For an interacting pair with n = +1, xj > L/2,
// so xj - L is exact (Sterbenz) and fl(fl(xj - L) - xi) rounds once; for
// n = -1 likewise xi - L.  Those pairs (a box face between them) take this
// branch; the others already hold the once-rounded difference.
#ifndef QBVH_LJ_IMAGE_VALUE
#define QBVH_LJ_IMAGE_VALUE 1
#endif
struct LJPairGeom {
    float r2;                // pinned r^2 (membership)
    float vx, vy, vz, vr2;   // difference rounded once, and fl(fl(vx^2 + vy^2) + vz^2)
};

__device__ __forceinline__ float mi_value(float xj, float xi, float n, float L)
{
    if (n > 0.f) return __fsub_rn(__fsub_rn(xj, L), xi);
    if (n < 0.f) return __fsub_rn(xj, __fsub_rn(xi, L));
    return __fsub_rn(xj, xi);
}

__device__ __forceinline__ LJPairGeom lj_pair_geom(const float4 &pi, const float4 &pj, float L, float Linv)
{
    // x and y as one packed pair, with the same roundings as the scalar form
    const f32x2 dxy0 = f2_sub(f2_pack(pj.x, pj.y), f2_pack(pi.x, pi.y));
    float tx, ty;
    f2_unpack(f2_mul(dxy0, f2_pack(Linv, Linv)), tx, ty);
    const float nx = rintf(tx), ny = rintf(ty);
    // L n is exact (n in {-1, 0, 1}), so a contraction of this product and
    // difference into one fused operation gives the same result
    const f32x2 dxy = f2_sub(dxy0, f2_mul(f2_pack(L, L), f2_pack(nx, ny)));
    float dx, dy;
    f2_unpack(dxy, dx, dy);
    const float dz0 = __fsub_rn(pj.z, pi.z);
    const float nz = rintf(__fmul_rn(dz0, Linv));
    const float dz = __fsub_rn(dz0, __fmul_rn(L, nz));
    float sx, sy;
    f2_unpack(f2_mul(dxy, dxy), sx, sy);
    LJPairGeom g;
    g.r2 = __fadd_rn(__fadd_rn(sx, sy), __fmul_rn(dz, dz));
    g.vx = dx;
    g.vy = dy;
    g.vz = dz;
    g.vr2 = g.r2;
    if (QBVH_LJ_IMAGE_VALUE && (nx != 0.f || ny != 0.f || nz != 0.f)) {
        g.vx = mi_value(pj.x, pi.x, nx, L);
        g.vy = mi_value(pj.y, pi.y, ny, L);
        g.vz = mi_value(pj.z, pi.z, nz, L);
        g.vr2 = __fadd_rn(__fadd_rn(__fmul_rn(g.vx, g.vx), __fmul_rn(g.vy, g.vy)), __fmul_rn(g.vz, g.vz));
    }
    return g;
}

// Outward snapping onto the 2^21 bin edges of the 21-bit node format (lower
// bound rounded down, upper bound up, IEEE directed rounding), shared by the
// build and by candidate mode's 21-bit leaf boxes.
__device__ __forceinline__ unsigned q_down21(float x, float r, float h)
{
    float v = floorf(__fdiv_rd(__fsub_rd(x, r), h));
    v = fminf(fmaxf(v, 0.f), (float)QBVH_QMAX21);
    return (unsigned)v;
}

__device__ __forceinline__ unsigned q_up21(float x, float r, float h)
{
    float v = ceilf(__fdiv_ru(__fsub_ru(x, r), h));
    v = fminf(fmaxf(v, 0.f), (float)QBVH_QMAX21);
    return (unsigned)v;
}

// ---- build helpers shared by the multi-kernel and the one-block builds ----
__device__ __forceinline__ unsigned spread10(unsigned v)
{
    // place bit k of a 10-bit value at bit 3k
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ unsigned bin_of(float x, float scale)
{
    int b = (int)__fmul_rn(x, scale);   // truncation == floor for x >= 0
    b = b < 0 ? 0 : b;
    b = b > QBVH_QMAX - 1 ? QBVH_QMAX - 1 : b;
    return (unsigned)b;
}

__device__ __forceinline__ unsigned pack3(unsigned x, unsigned y, unsigned z)
{
    return (x << 20) | (y << 10) | z;
}

__device__ __forceinline__ unsigned qmin3(unsigned a, unsigned b)
{
    return pack3(min((a >> 20) & 1023u, (b >> 20) & 1023u), min((a >> 10) & 1023u, (b >> 10) & 1023u),
                 min(a & 1023u, b & 1023u));
}

__device__ __forceinline__ unsigned qmax3(unsigned a, unsigned b)
{
    return pack3(max((a >> 20) & 1023u, (b >> 20) & 1023u), max((a >> 10) & 1023u, (b >> 10) & 1023u),
                 max(a & 1023u, b & 1023u));
}

// Lower bound snapped down / upper bound snapped up onto the bin edges.
__device__ __forceinline__ unsigned q_down(float x, float r, float h)
{
    float v = floorf(__fdiv_rd(__fsub_rd(x, r), h));
    v = fminf(fmaxf(v, 0.f), (float)QBVH_QMAX);
    return (unsigned)v;
}

__device__ __forceinline__ unsigned q_up(float x, float r, float h)
{
    float v = ceilf(__fdiv_ru(__fsub_ru(x, r), h));
    v = fminf(fmaxf(v, 0.f), (float)QBVH_QMAX);
    return (unsigned)v;
}

// Rope of the subtree whose leaves end at `last` in tree [lo, hi]: the node
// visited next in pre-order is the shallowest node starting at last + 1.  That
// node is a right child, and a right child's Karras index is its first leaf,
// so it is internal node last+1 if that node starts at last+1, else leaf last+1.
__device__ __forceinline__ int rope_after(const int2 *range, int last, int hi)
{
    const int k = last + 1;
    if (k > hi) return QBVH_END;
    if (k <= hi - 1 && range[k].x == k) return k;
    return ~k;
}

// Per-segment (tree) information, written by the build.
struct SegInfo {
    int start;      // first sorted position
    int count;      // particles in the tree
    int sys;        // system index
    int type;       // particle type
    float rlo[3];   // root AABB lower corner (fitted, exact min over positions)
    float rhi[3];   // root AABB upper corner
    float h[3];     // bin width per axis, rounded up, >= FLT_MIN
    float pad;
    float h21[3];   // bin width of the 21-bit node format (2^21 - 1 bins), rounded up
};

// Per-system information.
struct SysInfo {
    int offset;     // first original index
    int count;
    float L;        // box edge
    float Linv;     // fl(1 / L), computed once on the host
    float mscale;   // fl(1023 / L): Morton bins per unit length
    float pad[3];
};

struct DevStatus {
    int max_count;
    unsigned next_packet;   // packet queue of the traversal (zeroed with max_count before each query)
    unsigned err;
    unsigned pad;
};

// ---- launchers (build.cu) ------------------------------------------------
struct BuildArgs {
    const float4 *pos;   // [n] original order
    const double4_32a *pos64; // [n] original order, double-precision data (or nullptr)
    double L64;          // FP64 box edge of double-precision data
    double4_32a *leaves64;   // [n] FP64 positions in Z-order (double-precision data)
    int n;
    int n_sys;
    int n_types;         // trees per system: particle types, or 1 when all types share a tree
    int type_bound;      // valid particle types are [0, type_bound)
    int n_seg;
    bool wide_keys;      // u64 keys
    int bundle_k;
    const SysInfo *sys;  // [n_sys]
    const int *sys_off;  // [n_sys + 1]
    SegInfo *seg;        // [n_seg]
    unsigned *seg_rootbits; // [n_seg * 8] per-tree count and root AABB accumulators
    unsigned *sort_scratch;  // radix-sort scratch: histograms, tickets, look-back words
    size_t sort_scratch_words;
    int sort_passes;         // digit passes of the key sort
    int *seg_start;      // [n_seg + 1]
    float *frames;       // [n_seg * 8]
    void *keys;          // morton keys, input of the sort
    const void *keys_sorted;
    const int *order;    // sorted values
    int2 *range;
    int2 *child;
    int *par_int;
    int *par_leaf;
    int *visit;
    uint2 *leaf_q;
    int4 *nodes;
    float4 *nodes32;     // [2n] FP32 nodes or nullptr
    int4 *nodes21;       // [2n] 21-bit nodes or nullptr
    float4 *leaves;
    DevStatus *status;
};

void launch_build_prepare(const BuildArgs &a, cudaStream_t s);
void launch_morton(const BuildArgs &a, cudaStream_t s);
void launch_seg_scan(const BuildArgs &a, cudaStream_t s);
void launch_karras(const BuildArgs &a, cudaStream_t s);
void launch_fit(const BuildArgs &a, cudaStream_t s);
// one-block build of one small system (small_build.cu): whether it applies,
// and the launch (writes sorted keys / order to keys_sorted / order)
bool small_build_fits(const BuildArgs &a);
void launch_small_build(const BuildArgs &a, cudaStream_t s);

// ---- radix sort (sort.cu) ------------------------------------------------
struct SortScratch {
    unsigned *hist;        // [passes][256] digit counts -> exclusive offsets
    unsigned *status;      // [passes][tiles][256] look-back words
    unsigned *counters;    // [passes] tile tickets
};

size_t sort_tile_items();
int sort_num_tiles(int n);
size_t sort_scratch_bytes(int n, int passes);
// Sorts (key, value) pairs stably by the low `bits` bits of the key.  keys_a
// holds the input keys; values start as 0..n-1.  Returns the index (0 or 1)
// of the buffer pair holding the result: 0 -> (keys_a, vals_a), 1 -> (keys_b, vals_b).
int radix_sort_pairs(bool wide, void *keys_a, void *keys_b, int *vals_a, int *vals_b, int n,
                     int bits, void *scratch, unsigned *err, cudaStream_t s, bool prepared = false);
int sort_wait_selftest(int spin_limit, unsigned *err_out, cudaStream_t s);

// ---- traversal (query.cu) ------------------------------------------------
struct QueryArgs {
    const int4 *nodes;
    const float4 *nodes32;  // FP32 node format (node_fmt == 1)
    const int4 *nodes21;    // 21-bit node format (node_fmt == 2)
    int node_fmt;
    const float4 *leaves;
    const uint2 *leaf_q;   // quantized leaf boxes (candidate mode)
    const void *keys_sorted;
    bool wide_keys;
    const SegInfo *seg;
    const SysInfo *sys;
    int n;
    int n_types;
    int cap;
    int *rows;
    int *counts;
    DevStatus *status;
    int candidates;        // 1: Alg. 1 candidates, no exact leaf test
    int traversal;         // 0: one thread per particle, 1: warp-uniform walk
    int warp_particles;    // particles per warp of the warp walk: 32, 16, 8, 4, 2 or 1
    // double-precision particle data: FP32 test outside the band
    // [rl2_lo, rl2_hi] around r^2, FP64 test (leaves64, L64, r2_64) inside
    int f64;
    const double4_32a *leaves64;
    double L64;
    float rl2_lo[64];
    float rl2_hi[64];
    double r2_64[64];
    int block;
    int persistent;        // 1: resident warps take packets from a queue (one particle per lane)
    int n_packets;         // packets of 32 / W particles
    int sparse_blocks;     // leading blocks that walk sparse trees one particle per warp
    float r_list[64];      // [a][b] list radius
    float rl2[64];         // fl(r * r)
    float rs[64];          // padded search radius (rounded up)
    float rs2[64];         // rs^2 rounded up
    // Lennard-Jones terms of the accepted pairs, evaluated during the walk
    // (one system, one type; lj = 1): eps/sig [1] on the device, fl(r_c^2),
    // per-particle outputs by original index and one FP64 record per block
    int lj;
    const float *lj_eps, *lj_sig;
    float lj_rc2;
    float *lj_e, *lj_F;
    double *lj_partials;
};

void launch_query(const QueryArgs &a, cudaStream_t s);

// Traversal with the Lennard-Jones terms of the accepted pairs (a.lj = 1):
// one system, one type, one particle per lane, exact lists of FP32 data.
// query_lj_blocks = its block count (one FP64 record per block).
int query_lj_blocks(int n, int block);
void launch_query_lj(const QueryArgs &a, cudaStream_t s);

// ---- uniform grid comparator (grid.cu) ----------------------------------
struct GridArgs {
    const float4 *pos;     // [n] original order
    int n;
    int n_types;
    float L, Linv;
    int nc;                // cells per axis
    float inv_w;           // fl(nc / L)
    unsigned *keys;        // cell index per particle (sort input)
    const unsigned *keys_sorted;
    const int *order;      // sorted position -> original index
    int *cell_start;       // [nc^3 + 1]
    float4 *spos;          // [n] positions in cell order, w = original index
    int *stype;            // [n] types in cell order (n_types > 1) or nullptr
    int *rows;
    int *counts;
    int cap;
    int tpp;               // lanes per particle
    float rl2[64];
    DevStatus *status;
};

void launch_grid_keys(const GridArgs &a, cudaStream_t s);
void launch_grid_cells(const GridArgs &a, cudaStream_t s);
void launch_grid_query(const GridArgs &a, cudaStream_t s);

// ---- Lennard-Jones (lj.cu) -----------------------------------------------
struct LJArgs {
    const float4 *pos;
    const int *order;      // sorted position -> original index (walk order), or nullptr
    const int *rows;
    const int *counts;
    int cap;
    int n;
    int n_types;
    int n_sys;
    const SysInfo *sys;
    const int *blk_sys;    // [n_blocks] system of each block
    const int *blk_first;  // [n_blocks] first particle of each block
    int n_blocks;
    int tpp;               // lanes per particle (1, 2, 4, 8, 16, 32)
    const float *eps;
    const float *sig;
    float rc2[64];         // fl(r_cut * r_cut)
    float *e;
    float *F;
    double *partials;      // [n_blocks][1 + 2 T^2]
    double *U;
    double *dE;
    double *dS;
    const int *sys_blk_start; // [n_sys + 1]
};

void launch_lj_forward(const LJArgs &a, cudaStream_t s);

// fixed-order FP64 sums of one system's n_blocks records of 3 values
// (U, dU/deps, dU/dsig of one type), as written by the fused traversal
void launch_lj_finalize_one(const double *partials, int n_blocks, double *U, double *dE, double *dS,
                            cudaStream_t s);

void launch_lj_backward(const double *g, const float *F, const double *dE, const double *dS,
                        float *gpos, float *geps, float *gsig, int n, int n_sys, int n_types,
                        const SysInfo *sys, const int *sys_off, cudaStream_t s);

void launch_pack(const float *xyz, const int *types, int n, float4 *out, cudaStream_t s);

}  // namespace qbvh
