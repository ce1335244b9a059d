// Neighbor-list traversal (Alg. 1 of the paper).
//
// Particles are taken in Z-order so that neighbouring threads walk nearby
// parts of the tree (Sec. 3).  For every tree the particle interacts with (one
// tree per type, per-type-pair radius):
//   1. test the 27 periodic images of the search sphere against the root AABB
//      and keep the overlapping ones in a bitset (Sec. 2.3; Alg. 1 image loop);
//   2. for each image: stackless traversal from the root -- on overlap descend
//      to the left child, otherwise follow the rope, stop at the end marker
//      (Sec. 2.1; Alg. 1 inner loop);
//   3. node test: the sphere against the node's box through the nearest point
//      y = min(max(x, a), b) (Eq. 2).  Quantized bounds are decompressed
//      outward first (lower bound rounded down, upper up; Sec. 2.3, Sec. 3);
//      the squared distance is rounded toward zero, so a true overlap is
//      never rejected;
//   4. leaf: the paper lists the particle when the sphere overlaps the leaf
//      (Sec. 2.3) and allows the false positives to be filtered later; here
//      the exact FP32 distance test is that filter, so the list is exact.
//      Internal nodes with at most K leaves ("bundles", the subtree collapse
//      suggested at the end of Sec. 2.3) are not descended: their leaves,
//      contiguous in Z-order, are tested directly.
//
// Two mappings of particles to threads:
//   query_thread_kernel: one thread per particle, Alg. 1 as written;
//   query_warp_kernel:   one warp per 32 consecutive Z-order particles.  The
//     warp takes the same rope walk together: at every node each lane tests
//     its own sphere and the warp descends when any lane overlaps; at a leaf
//     or bundle every lane runs the exact test on the same (broadcast) leaf.
//     Control flow is warp-uniform.
//
// Conservativeness.  The search radius is padded on the host:
//   r_search = r_list (1 + 2^-20) + 2^-19 L, rounded up; r_search^2 rounded up.
// If the exact test accepts j under image n, rounding in that test and in the
// image centre fl(x_i + nL) moves the real distance |x_i + nL - x_j| by at
// most r_list * 4.1 u + 5.2 u L (u = 2^-24), below the padding; x_j lies in
// every decoded ancestor box, so every ancestor passes: no pair is lost.
//
// Exact test and image choice.  The list's decision expression is
//   dx = fl(xj - xi); dx = fl(dx - fl(L rint(fl(dx Linv)))), same for y, z,
//   d2 = fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) < fl(r^2).
// Under image n the kernel computes d2 from fl(fl(xj - xi) - nL) and accepts
// when d2 < fl(r^2), without evaluating rint.  This is the same decision: the
// host requires r < (L/2)(1 - 2^-20).  If the shifted d2 < fl(r^2) then every
// shifted component satisfies |dx'| < r (1 + 2.1 u) < (L/2)(1 - 2^-21); for
// n != 0, Sterbenz's lemma makes fl(dx - nL) exact, so dx = nL + dx' and
// fl(dx * Linv) lies strictly inside (n - 1/2, n + 1/2): rint gives n, the
// expression's own choice.  Hence a pair is accepted under exactly one image,
// the one rint selects, with the same d2 -- and rows hold no duplicates.
#include "qbvh_internal.cuh"

namespace qbvh {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
struct Frame {
    float rx, ry, rz;   // R_lo
    float hx, hy, hz;   // bin width
};

// A node's bounds (decoded to FP32, outward) and links.
struct Node {
    float lx, ly, lz, hx, hy, hz;
    int left;     // left child id, or first leaf index of a bundle
    int rope;
    bool bundle;
};

// 10-bit field -> float, exact: OR the value into the mantissa of 2^23, then
// subtract 2^23.
__device__ __forceinline__ float q_at(unsigned w, int shift)
{
    return __uint_as_float(((w >> shift) & 1023u) | 0x4B000000u) - 8388608.f;
}

__device__ __forceinline__ Node decode_q(const int4 w, const Frame &f)
{
    Node n;
    const unsigned lo = (unsigned)w.x, hi = (unsigned)w.y;
    n.lx = __fmaf_rd(q_at(lo, 20), f.hx, f.rx);
    n.ly = __fmaf_rd(q_at(lo, 10), f.hy, f.ry);
    n.lz = __fmaf_rd(q_at(lo, 0), f.hz, f.rz);
    n.hx = __fmaf_ru(q_at(hi, 20), f.hx, f.rx);
    n.hy = __fmaf_ru(q_at(hi, 10), f.hy, f.ry);
    n.hz = __fmaf_ru(q_at(hi, 0), f.hz, f.rz);
    n.left = w.z;
    n.rope = w.w;
    n.bundle = w.x < 0;
    return n;
}

__device__ __forceinline__ Node decode_f(const float4 a, const float4 b)
{
    Node n;
    n.bundle = __float_as_int(a.x) < 0;
    n.lx = __int_as_float(__float_as_int(a.x) & 0x7FFFFFFF);
    n.ly = a.y;
    n.lz = a.z;
    n.hx = b.x;
    n.hy = b.y;
    n.hz = b.z;
    n.left = __float_as_int(a.w);
    n.rope = __float_as_int(b.w);
    return n;
}

// 21-bit node (2 x int4 read as 8 floats): bounds decoded outward like the
// 10-bit ones, fields x << 42 | y << 21 | z of two 64-bit words.
__device__ __forceinline__ float q21_at(unsigned long long w, int shift)
{
    return __uint_as_float(((unsigned)(w >> shift) & (unsigned)QBVH_QMAX21) | 0x4B000000u) - 8388608.f;
}

__device__ __forceinline__ Node decode_21(const float4 a, const float4 b, const Frame &f)
{
    const unsigned long long lo = ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
    const unsigned long long hi = ((unsigned long long)__float_as_uint(a.w) << 32) | __float_as_uint(a.z);
    Node n;
    n.lx = __fmaf_rd(q21_at(lo, 42), f.hx, f.rx);
    n.ly = __fmaf_rd(q21_at(lo, 21), f.hy, f.ry);
    n.lz = __fmaf_rd(q21_at(lo, 0), f.hz, f.rz);
    n.hx = __fmaf_ru(q21_at(hi, 42), f.hx, f.rx);
    n.hy = __fmaf_ru(q21_at(hi, 21), f.hy, f.ry);
    n.hz = __fmaf_ru(q21_at(hi, 0), f.hz, f.rz);
    n.left = __float_as_int(b.x);
    n.rope = __float_as_int(b.y);
    n.bundle = (lo >> 63) != 0ull;
    return n;
}

// Read-only loads of tree words (nodes, leaves).  QBVH_TREE_EVICT_LAST = 1
// marks them evict-last in L2, so that list writes streaming through L2 evict
// them after everything else.  That paid while the list went out as 4-byte
// stores (1.4 GB of DRAM writes per launch at N = 2M: query 1.92 -> 1.84 ms);
// with whole-sector row writes (1.0 GB) plain loads are faster (10-bit nodes
// 1.266 -> 1.240 ms, FP32 nodes 1.243 -> 1.237 ms), so it is off.
// QBVH_NODE_V8 = 1 reads a 32-byte FP32 node with one 256-bit load (sm_100
// and later) instead of two 128-bit ones (same speed, one instruction).
#ifndef QBVH_TREE_EVICT_LAST
#define QBVH_TREE_EVICT_LAST 0
#endif
#ifndef QBVH_NODE_V8
#define QBVH_NODE_V8 1
#endif
__device__ __forceinline__ float4 tree_ld(const float4 *p)
{
#if QBVH_TREE_EVICT_LAST
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
    return v;
#else
    return __ldg(p);
#endif
}
__device__ __forceinline__ int4 tree_ld(const int4 *p)
{
#if QBVH_TREE_EVICT_LAST
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    int4 v;
    asm("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
    return v;
#else
    return __ldg(p);
#endif
}
// both halves of a 32-byte FP32 node (32-byte aligned: node arrays come from
// the allocator's 256-byte aligned blocks)
__device__ __forceinline__ void node32_ld(const float4 *p, float4 &a, float4 &b)
{
#if QBVH_NODE_V8 && QBVH_TREE_EVICT_LAST
    asm("ld.global.nc.L2::evict_last.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w) : "l"(p));
#elif QBVH_NODE_V8
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w) : "l"(p));
#else
    a = tree_ld(p);
    b = tree_ld(p + 1);
#endif
}

// Raw words of a node, loaded ahead of use.
struct Raw {
    int4 q;
    float4 a, b;
};

template <int FMT>
__device__ __forceinline__ Raw load_raw(const QueryArgs &A, int id)
{
    Raw r;
    if (FMT == 0) {
        r.q = tree_ld(A.nodes + id);
    } else if (FMT == 1) {
        node32_ld(A.nodes32 + 2 * (size_t)id, r.a, r.b);
    } else {
        node32_ld(reinterpret_cast<const float4 *>(A.nodes21) + 2 * (size_t)id, r.a, r.b);
    }
    return r;
}

template <int FMT>
__device__ __forceinline__ Node decode(const Raw &r, const Frame &f)
{
    if (FMT == 0) return decode_q(r.q, f);
    if (FMT == 1) return decode_f(r.a, r.b);
    return decode_21(r.a, r.b, f);
}

// Sphere (centre p, squared radius rs2) against a box: lower bound of the
// squared distance from p to the box, compared with the rounded-up rs2.
// Nearest point of the box y = min(max(p, lo), hi) (Eq. 2, exact); the
// differences p - y, their squares and the sum are rounded toward zero, so
// the result never exceeds the true squared distance.  x and y go as one
// packed f32x2 pair.  (Same speed as the gap form max(lo - p, p - hi, 0) with
// downward rounding, kept under QBVH_NODE_CLAMP=0: 1.94 ms at N = 2M either
// way, the walk waits on its dependent node loads, not on this arithmetic.)
#ifndef QBVH_NODE_CLAMP
#define QBVH_NODE_CLAMP 1
#endif
__device__ __forceinline__ bool overlap(float px, float py, float pz, const Node &n, float rs2)
{
#if QBVH_NODE_CLAMP
    const float yx = fminf(fmaxf(px, n.lx), n.hx);
    const float yy = fminf(fmaxf(py, n.ly), n.hy);
    const float yz = fminf(fmaxf(pz, n.lz), n.hz);
    f32x2 dxy;
    asm("sub.rz.f32x2 %0, %1, %2;" : "=l"(dxy) : "l"(f2_pack(px, py)), "l"(f2_pack(yx, yy)));
    f32x2 sxy;
    asm("mul.rz.f32x2 %0, %1, %1;" : "=l"(sxy) : "l"(dxy));
    float sx, sy;
    f2_unpack(sxy, sx, sy);
    const float dz = __fsub_rz(pz, yz);
    const float d2 = __fmaf_rz(dz, dz, __fadd_rz(sx, sy));
#else
    const float gx = fmaxf(fmaxf(__fsub_rd(n.lx, px), __fsub_rd(px, n.hx)), 0.f);
    const float gy = fmaxf(fmaxf(__fsub_rd(n.ly, py), __fsub_rd(py, n.hy)), 0.f);
    const float gz = fmaxf(fmaxf(__fsub_rd(n.lz, pz), __fsub_rd(pz, n.hz)), 0.f);
    const float d2 = __fmaf_rd(gx, gx, __fmaf_rd(gy, gy, __fmul_rd(gz, gz)));
#endif
    return d2 <= rs2;
}

__device__ __forceinline__ bool overlap_q(float px, float py, float pz, uint2 q, const Frame &f, float rs2)
{
    const Node n = decode_q(make_int4((int)q.x, (int)q.y, 0, 0), f);
    return overlap(px, py, pz, n, rs2);
}

// Store of one list entry.  QBVH_ROW_STORE: 0 = streaming (evict-first),
// 1 = cache at L2 (.cg), 2 = default write-back.
#ifndef QBVH_ROW_STORE
#define QBVH_ROW_STORE 0
#endif
__device__ __forceinline__ void row_store(int *p, int v)
{
#if QBVH_ROW_STORE == 0
    __stcs(p, v);
#elif QBVH_ROW_STORE == 1
    __stcg(p, v);
#else
    *p = v;
#endif
}

// Row writer.  Entries past cap are counted, not written.  The list is never
// read back by the traversal, so it is stored with the streaming (evict-first)
// hint and does not push the tree out of L2.  (Gathering four entries into
// one 16-byte store was measured slower: the extra selects and registers cost
// more than the narrower stores.)
// Row staging (QBVH_ROW_STAGING = 1): a lane's entries first go to its
// slots of a per-warp ring in shared memory, 16 entries (two 32-byte
// sectors) per lane, slot k of lane l at ring[32 k + l] (conflict-free).
// Rows start on 32-byte boundaries (the row capacity is a multiple of 8), so
// a completed sector of 8 entries leaves with two 16-byte stores that fill
// one whole DRAM sector, and the L2 sees one write per 8 entries instead of
// one per entry.  The survivor loop (below) stages every tested survivor
// without a branch (the slot after the last entry is free, and the count
// only advances on acceptance) and checks for completed sectors once per 8
// survivors and at the end of each chunk, so the lanes that completed one
// write it together; with one ring sector of slack, at most one sector is
// complete at a check.  Other pushes write a completed sector at once.  The
// partial last sector is written at the end of the particle's walks.
// Measured at N = 2M: the 4-byte row stores took 0.62 of 1.91 ms before
// staging; a flush on every sector completion issued the sector write for
// one or two lanes at a time, on most survivors.
#ifndef QBVH_ROW_STAGING
#define QBVH_ROW_STAGING 1
#endif
// zero image and the other images in two launches (see query_warp_kernel)
#ifndef QBVH_QUERY_SPLIT_IMAGES
#define QBVH_QUERY_SPLIT_IMAGES 0
#endif
__device__ __forceinline__ void store_sector(int *dst, const int *ring)
{
    const int4 lo = make_int4(ring[0], ring[32], ring[64], ring[96]);
    const int4 hi = make_int4(ring[128], ring[160], ring[192], ring[224]);
    __stcs(reinterpret_cast<int4 *>(dst), lo);
    __stcs(reinterpret_cast<int4 *>(dst) + 1, hi);
}

struct Row {
    int *row;
    int cap;
    int count;
    int *ring;   // this lane's slot 0 in the warp's staging ring, or nullptr
    int base;    // staging: entries [0, base) have left the ring (a multiple of 8)
    int fill;    // staging with W lanes per particle: entries the group has written to the row

    // the completed sector [base, base + 8) (staging only)
    __device__ __forceinline__ void flush()
    {
        if (base + 8 <= cap) store_sector(row + base, ring + 32 * (base & 15));
        base += 8;
    }

    // a completed sector, if any (staging only; at most one between checks)
    __device__ __forceinline__ void check()
    {
        if (count - base >= 8) flush();
    }

    // entry j, tested by the caller
    __device__ __forceinline__ void push(int j)
    {
        if (ring) {
            ring[32 * (count & 15)] = j;
            ++count;
            check();
            return;
        }
        if (count < cap) row_store(row + count, j);
        ++count;
    }

    // entry j if acc, without a branch (staging only; the caller checks
    // within every 8 staged candidates)
    __device__ __forceinline__ void stage(int j, bool acc)
    {
        ring[32 * (count & 15)] = j;
        count += acc ? 1 : 0;
    }

    // the entries of the last, partial sector (staging only)
    __device__ __forceinline__ void drain()
    {
        if (!ring) return;
        check();
        const int end = min(count, cap);
        for (int k = base; k < end; ++k) row_store(row + k, ring[32 * (k & 15)]);
    }

    // With W > 1 lanes per particle (the lanes in `same`) every lane stages
    // the survivors it tests in its own ring and counts its own accepted
    // entries; the group shares the row.  A completed sector goes to the next
    // free 8 slots of the row, in lane order among the lanes that flush
    // together.  Every lane of the warp calls this together.
    __device__ __forceinline__ void check_group(unsigned same)
    {
        const bool f = count - base >= 8;
        const unsigned b = __ballot_sync(0xFFFFFFFFu, f) & same;
        if (f) {
            unsigned lt;
            asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
            const int off = fill + 8 * __popc(b & lt);
            if (off + 8 <= cap) store_sector(row + off, ring + 32 * (base & 15));
            base += 8;
        }
        fill += 8 * __popc(b);
    }

    // The group's partial sectors after its complete ones, in lane order; then
    // count holds the particle's total.  Every lane of the warp calls this
    // together; `first` is the group's first lane, G the lane stride.
    template <int W>
    __device__ __forceinline__ void drain_group(unsigned same, int first, int G, int wsub)
    {
        check_group(same);
        const int k = count - base;
        int pre = 0, tot_left = 0, total = 0;
#pragma unroll
        for (int m = 0; m < W; ++m) {
            const int km = __shfl_sync(0xFFFFFFFFu, k, first + m * G);
            const int cm = __shfl_sync(0xFFFFFFFFu, count, first + m * G);
            if (m < wsub) pre += km;
            tot_left += km;
            total += cm;
        }
        const int start = fill + pre;
        for (int i = 0; i < k; ++i)
            if (start + i < cap) row_store(row + start + i, ring[32 * ((base + i) & 15)]);
        fill += tot_left;
        count = total;
    }
};

struct Query {
    float xi, yi, zi;     // own position
    int self;             // own sorted index
    int self_id;          // own original index
    float nLx, nLy, nLz;  // image shift n L
    float px, py, pz;     // image centre fl(x_i + n L)
    float rl2;
    float rl2_lo, rl2_hi; // double-precision data: band of the FP32 test around rl2
    int pair;             // double-precision data: type pair of the current tree
    // Lennard-Jones value of an image pair (fused option): per axis the
    // difference fl(fl(xj - v1) - v2), the once-rounded x_j - x_i - n L
    float vx1, vy1, vz1, vx2, vy2, vz2;
};

// d2 of the exact test (see the header comment) for leaf position q.
// SHIFT = false is the zero image, where subtracting n L = 0 is the identity.
template <bool SHIFT>
__device__ __forceinline__ float exact_d2(const Query &c, const float4 q)
{
#if QBVH_F32X2
    f32x2 dxy = f2_sub(f2_pack(q.x, q.y), f2_pack(c.xi, c.yi));
    float dz = __fsub_rn(q.z, c.zi);
    if (SHIFT) {
        dxy = f2_sub(dxy, f2_pack(c.nLx, c.nLy));
        dz = __fsub_rn(dz, c.nLz);
    }
    float sx, sy;
    f2_unpack(f2_mul(dxy, dxy), sx, sy);
    return __fadd_rn(__fadd_rn(sx, sy), __fmul_rn(dz, dz));
#else
    float dx = __fsub_rn(q.x, c.xi);
    float dy = __fsub_rn(q.y, c.yi);
    float dz = __fsub_rn(q.z, c.zi);
    if (SHIFT) {
        dx = __fsub_rn(dx, c.nLx);
        dy = __fsub_rn(dy, c.nLy);
        dz = __fsub_rn(dz, c.nLz);
    }
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
#endif
}

// Double-precision particle data (Sec. 2.2).  The list's decision is the
// pinned FP64 expression
//   dx = fl(xj - xi); dx = fl(dx - L rint(fl(dx Linv))), same for y, z,
//   d2 = fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) < fl(r^2),
// taken under the walk's image without rint, as in FP32 (the argument in the
// header comment holds with the FP64 unit roundoff).  The leaf words hold
// the positions rounded to FP32, and the FP32 d2 of those decides whenever
// it lies outside [rl2_lo, rl2_hi]: the host sets that band from a bound on
// the difference of the two computations for pairs within the radius
// (per component at most 2^-21 L, see qbvh_query), so it cannot change a
// decision.  Inside the band the FP64 positions decide.
template <bool SHIFT>
__device__ __forceinline__ double exact_d2_64(const QueryArgs &A, const Query &c, int j)
{
    const double2 *pj = reinterpret_cast<const double2 *>(A.leaves64 + j);
    const double2 *pi = reinterpret_cast<const double2 *>(A.leaves64 + c.self);
    const double2 jxy = __ldg(pj), jz = __ldg(pj + 1), ixy = __ldg(pi), iz = __ldg(pi + 1);
    double dx = __dsub_rn(jxy.x, ixy.x);
    double dy = __dsub_rn(jxy.y, ixy.y);
    double dz = __dsub_rn(jz.x, iz.x);
    if (SHIFT) {
        const double L = A.L64;
        if (c.nLx != 0.f) dx = __dsub_rn(dx, c.nLx > 0.f ? L : -L);
        if (c.nLy != 0.f) dy = __dsub_rn(dy, c.nLy > 0.f ? L : -L);
        if (c.nLz != 0.f) dz = __dsub_rn(dz, c.nLz > 0.f ? L : -L);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// The exact decision for leaf j under the current image (j != self).  SELF =
// false leaves out the self test where the caller knows j cannot be the
// particle itself.  (Under a non-zero image the particle's own copy is never
// accepted anyway: its difference is -nL exactly, so d2 >= L^2 > r^2.)
template <bool SHIFT, bool F64, bool SELF = true>
__device__ __forceinline__ bool exact_accept(const QueryArgs &A, const Query &c, int j, const float4 q)
{
    const float d2 = exact_d2<SHIFT>(c, q);
    if (!F64) return d2 < c.rl2 && (!SELF || j != c.self);
    if (SELF && j == c.self) return false;
    if (d2 < c.rl2_lo) return true;
    if (!(d2 <= c.rl2_hi)) return false;
    return exact_d2_64<SHIFT>(A, c, j) < A.r2_64[c.pair];
}

// The exact test of leaf j under the current image.
template <bool SHIFT, bool F64, bool SELF = true>
__device__ __forceinline__ void exact_leaf(const QueryArgs &A, const Query &c, Row &out, int j, const float4 q)
{
    if (exact_accept<SHIFT, F64, SELF>(A, c, j, q)) out.push(__float_as_int(q.w) & 0x7FFFFFFF);
}

// Alg. 1 without the exact filter: the sphere against leaf j's box at the
// node format's precision (Sec. 2.2): the 10-bit quantized box (FMT 0), the
// FP32 point itself (FMT 1) or the 21-bit quantized box (FMT 2, snapped and
// decoded outward against the tree's 21-bit frame f).
template <int FMT>
__device__ __forceinline__ bool cand_overlap(const QueryArgs &A, const Query &c, int j, const float4 q,
                                             const Frame &f, float rs2)
{
    if (FMT == 0) return overlap_q(c.px, c.py, c.pz, __ldg(A.leaf_q + j), f, rs2);
    Node n;
    if (FMT == 1) {
        n.lx = n.hx = q.x;
        n.ly = n.hy = q.y;
        n.lz = n.hz = q.z;
    } else {
        n.lx = __fmaf_rd((float)q_down21(q.x, f.rx, f.hx), f.hx, f.rx);
        n.ly = __fmaf_rd((float)q_down21(q.y, f.ry, f.hy), f.hy, f.ry);
        n.lz = __fmaf_rd((float)q_down21(q.z, f.rz, f.hz), f.hz, f.rz);
        n.hx = __fmaf_ru((float)q_up21(q.x, f.rx, f.hx), f.hx, f.rx);
        n.hy = __fmaf_ru((float)q_up21(q.y, f.ry, f.hy), f.hy, f.ry);
        n.hz = __fmaf_ru((float)q_up21(q.z, f.rz, f.hz), f.hz, f.rz);
    }
    return overlap(c.px, c.py, c.pz, n, rs2);
}

// List j when the sphere overlaps its leaf box (false positives included).
template <int FMT>
__device__ __forceinline__ void candidate_leaf(const QueryArgs &A, const Query &c, Row &out, int j, const float4 q,
                                               const Frame &f, float rs2)
{
    if (j != c.self && cand_overlap<FMT>(A, c, j, q, f, rs2)) out.push(__float_as_int(q.w) & 0x7FFFFFFF);
}

template <bool CAND, bool SHIFT = true, bool F64 = false, bool SELF = true, int FMT = 0>
__device__ __forceinline__ void test_leaf(const QueryArgs &A, const Query &c, Row &out, int j, const float4 q,
                                          const Frame &f, float rs2)
{
    if (CAND)
        candidate_leaf<FMT>(A, c, out, j, q, f, rs2);
    else
        exact_leaf<SHIFT, F64, SELF>(A, c, out, j, q);
}

// The same decisions as exact_leaf / candidate_leaf, returned instead of
// appended (used when several lanes share one particle's row).
template <bool CAND, bool SHIFT, bool F64 = false, int FMT = 0>
__device__ __forceinline__ bool leaf_accepts(const QueryArgs &A, const Query &c, int j, const float4 q,
                                             const Frame &f, float rs2)
{
    if (j == c.self) return false;
    if (CAND) return cand_overlap<FMT>(A, c, j, q, f, rs2);
    return exact_accept<SHIFT, F64>(A, c, j, q);
}

// Append for W lanes sharing a row: the lanes of one particle are `same`
// (a bit pattern over the warp); accepted entries are packed in lane order.
// Every lane of the warp must call this together.
__device__ __forceinline__ void push_shared(Row &out, bool acc, int j, unsigned same)
{
    const unsigned m = __ballot_sync(0xFFFFFFFFu, acc) & same;
    if (acc) {
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        const int slot = out.count + __popc(m & lt);
        if (slot < out.cap) row_store(out.row + slot, j);
    }
    out.count += __popc(m);
}

// 27-bit set of the periodic images whose padded search sphere overlaps the
// root AABB of a tree (Sec. 2.3): bit 9 (nx+1) + 3 (ny+1) + (nz+1).
__device__ __forceinline__ unsigned image_mask(float x, float y, float z, float L, const SegInfo &g, float rs2)
{
    float gap[3][3];
    const float xs[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float p = (m == 1) ? xs[d] : __fadd_rn(xs[d], (m == 0) ? -L : L);
            gap[d][m] = fmaxf(fmaxf(__fsub_rd(g.rlo[d], p), __fsub_rd(p, g.rhi[d])), 0.f);
        }
    }
    unsigned mask = 0u;
#pragma unroll
    for (int mx = 0; mx < 3; ++mx)
#pragma unroll
        for (int my = 0; my < 3; ++my)
#pragma unroll
            for (int mz = 0; mz < 3; ++mz) {
                const float d2 = __fmaf_rd(gap[0][mx], gap[0][mx],
                                           __fmaf_rd(gap[1][my], gap[1][my], __fmul_rd(gap[2][mz], gap[2][mz])));
                if (d2 <= rs2) mask |= 1u << (mx * 9 + my * 3 + mz);
            }
    return mask;
}

__device__ __forceinline__ void set_image(Query &c, int img, float L)
{
    const int nx = img / 9 - 1, ny = (img / 3) % 3 - 1, nz = img % 3 - 1;
    c.nLx = nx == 0 ? 0.f : (nx > 0 ? L : -L);
    c.nLy = ny == 0 ? 0.f : (ny > 0 ? L : -L);
    c.nLz = nz == 0 ? 0.f : (nz > 0 ? L : -L);
    c.px = nx == 0 ? c.xi : __fadd_rn(c.xi, c.nLx);
    c.py = ny == 0 ? c.yi : __fadd_rn(c.yi, c.nLy);
    c.pz = nz == 0 ? c.zi : __fadd_rn(c.zi, c.nLz);
}

template <bool WIDE>
__device__ __forceinline__ int seg_of_sorted(const QueryArgs &a, int s)
{
    if (WIDE) return (int)(__ldg(reinterpret_cast<const unsigned long long *>(a.keys_sorted) + s) >> 30);
    if (a.n_types > 1) return (int)(__ldg(reinterpret_cast<const unsigned *>(a.keys_sorted) + s) >> 30);
    return 0;
}

// the frame of the 21-bit node format: same corner, 2^21 - 1 bins
__device__ __forceinline__ Frame frame21_of(const SegInfo &g)
{
    Frame f;
    f.rx = g.rlo[0];
    f.ry = g.rlo[1];
    f.rz = g.rlo[2];
    f.hx = g.h21[0];
    f.hy = g.h21[1];
    f.hz = g.h21[2];
    return f;
}

__device__ __forceinline__ Frame frame_of(const SegInfo &g)
{
    Frame f;
    f.rx = g.rlo[0];
    f.ry = g.rlo[1];
    f.rz = g.rlo[2];
    f.hx = g.h[0];
    f.hy = g.h[1];
    f.hz = g.h[2];
    return f;
}

// node id outside the tree [start, last] -> broken structure (one unsigned
// compare on the node's or the leaf's index)
__device__ __forceinline__ bool bad_node(int node, const SegInfo &g, int last)
{
    const int idx = node ^ (node >> 31);   // node for internal ids, ~node for leaves
    return (unsigned)(idx - g.start) > (unsigned)(last - g.start);
}

// Largest row count: one atomic per warp, skipped when it cannot raise the maximum.
__device__ __forceinline__ void warp_max_count(int my_count, DevStatus *status)
{
    const int m = __reduce_max_sync(FULL, my_count);
    if ((threadIdx.x & 31) == 0 && m > 0 && m > __ldcg(&status->max_count)) atomicMax(&status->max_count, m);
}

// Last leaf of a bundle: the leaf before the rope target, or the tree's last leaf.
__device__ __forceinline__ int bundle_last(const Node &nd, int last)
{
    return (nd.rope == QBVH_END) ? last : ((nd.rope >= 0 ? nd.rope : ~nd.rope) - 1);
}

// ---- one thread per particle: Alg. 1 as written -------------------------
template <bool WIDE, bool CAND, int FMT>
__global__ void query_thread_kernel(const __grid_constant__ QueryArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int my_count = 0;
    if (s < a.n) {
        const float4 me = __ldg(a.leaves + s);
        int i_orig = __float_as_int(me.w) & 0x7FFFFFFF;
        if (i_orig >= a.n) {
            atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            i_orig = s;
        }
        const int seg_i = seg_of_sorted<WIDE>(a, s);
        const int T = a.n_types;
        const int sys = seg_i / T;
        const int ta = seg_i - sys * T;
        const float L = a.sys[sys].L;

        Query c;
        c.xi = me.x;
        c.yi = me.y;
        c.zi = me.z;
        c.self = s;
        c.self_id = i_orig;
        Row out;
        out.row = a.rows + (size_t)i_orig * a.cap;
        out.cap = a.cap;
        out.count = 0;
        out.ring = nullptr;
        out.base = 0;

        for (int tb = 0; tb < T; ++tb) {
            const float rl = a.r_list[ta * T + tb];
            if (!(rl > 0.f)) continue;
            const SegInfo g = a.seg[sys * T + tb];
            if (g.count == 0) continue;
            c.rl2 = a.rl2[ta * T + tb];
            const float rs2 = a.rs2[ta * T + tb];
            const Frame f = FMT == 2 ? frame21_of(g) : frame_of(g);
            unsigned mask = image_mask(me.x, me.y, me.z, L, g, rs2);
            const int root = g.count >= 2 ? g.start : ~g.start;
            const int last = g.start + g.count - 1;
            while (mask) {
                const int img = __ffs(mask) - 1;
                mask &= mask - 1u;
                set_image(c, img, L);
                int node = root;
                int budget = 2 * g.count;   // pre-order visits each node at most once
                while (node != QBVH_END) {
                    if (--budget < 0 || bad_node(node, g, last)) {
                        atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                        break;
                    }
                    if (node >= 0) {
                        const Node nd = decode<FMT>(load_raw<FMT>(a, node), f);
                        if (overlap(c.px, c.py, c.pz, nd, rs2)) {
                            if (nd.bundle) {
                                int l = bundle_last(nd, last);
                                if (nd.left < g.start || l > last) {
                                    atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                                    l = nd.left - 1;
                                }
                                for (int j = nd.left; j <= l; ++j)
                                    test_leaf<CAND, true, false, true, FMT>(a, c, out, j, tree_ld(a.leaves + j), f,
                                                                           rs2);
                                node = nd.rope;
                            } else {
                                node = nd.left;
                            }
                        } else {
                            node = nd.rope;
                        }
                    } else {
                        const int j = ~node;
                        const float4 q = tree_ld(a.leaves + j);
                        test_leaf<CAND, true, false, true, FMT>(a, c, out, j, q, f, rs2);
                        node = (j == last) ? QBVH_END : ((__float_as_int(q.w) < 0) ? j + 1 : ~(j + 1));
                    }
                }
            }
        }
        a.counts[i_orig] = out.count;
        my_count = out.count;
    }
    warp_max_count(my_count, a.status);
}

// Bundles that few lanes overlap.  Every lane testing every leaf costs the
// warp one trip per leaf however few lanes overlap the bundle box.  Instead,
// the overlapping lanes' tests are spread over the warp: the bundle's leaves
// go to S = 16 (or 32) consecutive lanes, loaded once, and each trip serves
// 32 / S overlapping particles, whose centre, row and count come by shuffle.
// A particle's accepted leaves are packed in leaf order, so rows are the same
// as with the per-lane loop.  Every lane of the warp calls this together;
// `hm` (warp-uniform) holds the overlapping lanes, cnt <= 32 leaves.
// Used when at most QBVH_SPREAD_MAX lanes overlap (N = 2M, density 0.8,
// K = 16; query ms by threshold: 0: 2.15, 4: 2.09, 8: 2.05, 12: 1.99,
// 16: 1.97, 20: 2.04, 32: 2.42).
#ifndef QBVH_SPREAD_MAX
#define QBVH_SPREAD_MAX 16
#endif
template <bool SHIFT, bool F64, bool SELF>
__device__ __forceinline__ void bundle_spread(const QueryArgs &a, const Query &c, Row &out, int first, int cnt,
                                              unsigned hm)
{
    const int lane = threadIdx.x & 31;
    const bool wide = cnt > 16;               // warp-uniform
    const int half = wide ? 0 : (lane >> 4);  // which particle of the trip this lane serves
    const int k = wide ? lane : (lane & 15);  // leaf slot
    const int j = first + k;
    const bool jv = k < cnt;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (jv) q = tree_ld(a.leaves + j);
    const int id = __float_as_int(q.w) & 0x7FFFFFFF;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const unsigned gmask = wide ? 0xFFFFFFFFu : (half ? 0xFFFF0000u : 0x0000FFFFu);
    while (hm) {
        const int o0 = __ffs(hm) - 1;
        hm &= hm - 1u;
        int o1 = -1;
        if (!wide && hm) {
            o1 = __ffs(hm) - 1;
            hm &= hm - 1u;
        }
        const int owner = half ? o1 : o0;
        const int src = owner < 0 ? lane : owner;
        Query t = c;
        t.xi = __shfl_sync(FULL, c.xi, src);
        t.yi = __shfl_sync(FULL, c.yi, src);
        t.zi = __shfl_sync(FULL, c.zi, src);
        t.self = c.self - lane + src;
        const int ocount = __shfl_sync(FULL, out.count, src);
        int *orow = reinterpret_cast<int *>(__shfl_sync(FULL, reinterpret_cast<unsigned long long>(out.row), src));
        const bool acc = owner >= 0 && jv && exact_accept<SHIFT, F64, SELF>(a, t, j, q);
        const unsigned m = __ballot_sync(FULL, acc);
        if (acc) {
            const int slot = ocount + __popc(m & gmask & lt);
            if (slot < out.cap) row_store(orow + slot, id);
        }
        if (lane == o0) out.count += __popc(m & (wide ? 0xFFFFFFFFu : 0x0000FFFFu));
        if (lane == o1) out.count += __popc(m & 0xFFFF0000u);
    }
}

// ---- 10-bit nodes tested in the integer domain ---------------------------
// With quantized nodes (Fig. 3b) the walk does not decode the node bounds.
// Each lane turns the bounding cube of its padded search sphere into the
// tree's lattice once per image: per axis the cells [ceil((p - rs - R) / h),
// floor((p + rs - R) / h)], with the divisions rounded outward and clamped to
// [0, 1023], packed like the node words (x << 20 | y << 10 | z).  A node
// passes when its packed [lo, hi] overlaps that cube on every axis.  A node
// box the sphere overlaps overlaps the cube too (the cube contains the
// sphere, and a node's real box R + [lo, hi] h with integer lo, hi meets
// [p - rs, p + rs] exactly when lo <= floor(..) and hi >= ceil(..)), so the
// test never rejects a node the sphere test of Eq. 2 accepts; it accepts a
// few more (the cube's corners).  All three fields are compared at once: for
// 10-bit fields a and b, (b | G) - (a & ~G) with G the top bit of every field
// borrows nothing across fields, its top bits say whether the low 9 bits of b
// are >= those of a, and (b & ~a) | (~(a ^ b) & t) at the top bits then says
// b >= a for the whole field.  On the N = 262,144 fluid (CPU walk of the
// oracle's tree, K = 32) a warp visits 176 nodes against 170 with the FP32
// sphere test, for about 8 integer operations per node.
#ifndef QBVH_QCUBE
#define QBVH_QCUBE 1
#endif
constexpr unsigned kFieldTops = (1u << 29) | (1u << 19) | (1u << 9);
constexpr unsigned kFieldLows = ~kFieldTops & QBVH_QMASK;

struct LaneCube {
    unsigned lo, hi;   // packed lattice cells of the search cube
    unsigned lo_l;     // lo with the fields' top bits cleared
    unsigned hi_g;     // hi with the fields' top bits set
    unsigned gm;       // kFieldTops, or 0 for a lane that does not walk this image
};

__device__ __forceinline__ unsigned cell_lo(float p, float rs, float R, float h)
{
    const float v = ceilf(__fdiv_rd(__fsub_rd(__fsub_rd(p, rs), R), h));
    return (unsigned)fminf(fmaxf(v, 0.f), (float)QBVH_QMAX);
}

__device__ __forceinline__ unsigned cell_hi(float p, float rs, float R, float h)
{
    const float v = floorf(__fdiv_ru(__fsub_ru(__fadd_ru(p, rs), R), h));
    return (unsigned)fminf(fmaxf(v, 0.f), (float)QBVH_QMAX);
}

__device__ __forceinline__ LaneCube lane_cube(const Query &c, bool on, const Frame &f, float rs)
{
    LaneCube q;
    q.lo = (cell_lo(c.px, rs, f.rx, f.hx) << 20) | (cell_lo(c.py, rs, f.ry, f.hy) << 10) |
           cell_lo(c.pz, rs, f.rz, f.hz);
    q.hi = (cell_hi(c.px, rs, f.rx, f.hx) << 20) | (cell_hi(c.py, rs, f.ry, f.hy) << 10) |
           cell_hi(c.pz, rs, f.rz, f.hz);
    q.lo_l = q.lo & kFieldLows;
    q.hi_g = q.hi | kFieldTops;
    q.gm = on ? kFieldTops : 0u;
    return q;
}

// field-wise b >= a at the fields' top bits, given t = (b | G) - (a & ~G)
__device__ __forceinline__ unsigned fields_ge(unsigned a, unsigned b, unsigned t)
{
    return (b & ~a) | (~(a ^ b) & t);
}

// node words lo (bit 31: bundle flag) and hi against the lane's cube
__device__ __forceinline__ bool cube_overlap(unsigned nlo, unsigned nhi, const LaneCube &q)
{
    const unsigned x1 = fields_ge(nlo, q.hi, q.hi_g - (nlo & kFieldLows));   // node lo <= cube hi
    const unsigned x2 = fields_ge(q.lo, nhi, (nhi | kFieldTops) - q.lo_l);   // cube lo <= node hi
    return (x1 & x2 & q.gm) == kFieldTops;
}

// ---- bundles filtered against the warp's box of search centres -------------
// At a bundle every lane first loads one of its (at most 32) leaves and
// tests it against the box of the warp's image centres grown by the search
// radius: the distance from the leaf to that box, rounded down, against the
// rounded-up r_search^2.  If some lane's exact test accepts the leaf, its
// centre lies in the box and the leaf within the padded radius of it (the
// conservativeness argument in the header comment), so the leaf survives.
// Survivors are packed into per-warp shared memory (x, y, z and original
// index as separate arrays, so that two survivors load as one f32x2 pair),
// and only they are tested exactly.  On the N = 262,144 fluid (K = 32) a warp
// tests 517 survivors instead of 1,333 bundle leaves; the union of its 32
// spheres holds 439 particles (CPU walk of the oracle's tree).
#ifndef QBVH_PREFILTER
#define QBVH_PREFILTER 1
#endif
#ifndef QBVH_FILTER_SPREAD
#define QBVH_FILTER_SPREAD 1
#endif
#ifndef QBVH_FILTER_SPREAD_MAX
#define QBVH_FILTER_SPREAD_MAX 16
#endif
#ifndef QBVH_SPREAD_COST
#define QBVH_SPREAD_COST 25
#endif
#ifndef QBVH_LOOP_COST
#define QBVH_LOOP_COST 14
#endif
// the walks that filter bundles: exact lists with one particle per lane (FP32
// or double-precision data), or of FP32 data with 2 or 4 lanes per particle
// (those share a row through the staging ring, so they need it, and the
// one-launch walk)
#ifndef QBVH_MULTI_LANE_FILTER
#define QBVH_MULTI_LANE_FILTER 1
#endif
__host__ __device__ constexpr bool stage_on(int W, bool CAND, bool F64)
{
    return QBVH_PREFILTER && !CAND &&
           (W == 1 || (!F64 && QBVH_MULTI_LANE_FILTER && (W == 2 || W == 4) && QBVH_ROW_STAGING &&
                       !QBVH_QUERY_SPLIT_IMAGES));
}

// A bundle's survivors (at most 64, padded to an even count) are staged
// before they are tested, so that every bundle runs one survivor loop.
constexpr int kStage = 64;
struct BundleStage {
    float4 blo, bhi;      // the warp's box of image centres (x, y, z)
    float x[kStage], y[kStage], z[kStage];   // 16-byte aligned: four survivors per load
    int id[kStage];       // original indices of the survivors
    union {
        int owner[32];    // overlapping lanes, in lane order (spread, without staging)
        int ring[16 * 32];   // row staging: slot k of lane l at ring[32 k + l]
    };
};

// Box of the image centres fl(x_i + n L) of the lanes that walk this image.
// Positions are in [0, L), so their bit patterns order like the values once
// -0 is folded into +0; fl(x + n L) is monotone in x, so shifting the
// unshifted box's corners gives the box of the shifted centres.
__device__ __forceinline__ void packet_box(const Query &c, bool on, BundleStage *st)
{
    const unsigned bx = __float_as_uint(c.xi + 0.f), by = __float_as_uint(c.yi + 0.f),
                   bz = __float_as_uint(c.zi + 0.f);
    const float lx = __uint_as_float(__reduce_min_sync(FULL, on ? bx : 0xFFFFFFFFu));
    const float ly = __uint_as_float(__reduce_min_sync(FULL, on ? by : 0xFFFFFFFFu));
    const float lz = __uint_as_float(__reduce_min_sync(FULL, on ? bz : 0xFFFFFFFFu));
    const float hx = __uint_as_float(__reduce_max_sync(FULL, on ? bx : 0u));
    const float hy = __uint_as_float(__reduce_max_sync(FULL, on ? by : 0u));
    const float hz = __uint_as_float(__reduce_max_sync(FULL, on ? bz : 0u));
    if ((threadIdx.x & 31) == 0) {
        st->blo = make_float4(__fadd_rn(lx, c.nLx), __fadd_rn(ly, c.nLy), __fadd_rn(lz, c.nLz), 0.f);
        st->bhi = make_float4(__fadd_rn(hx, c.nLx), __fadd_rn(hy, c.nLy), __fadd_rn(hz, c.nLz), 0.f);
    }
    __syncwarp();
}

// ---- Lennard-Jones terms of the accepted pairs (fused option) ------------
// With QueryArgs::lj set (one system, one type) the walk evaluates the
// truncated and shifted pair energy of Eq. 1 for every pair it accepts with
// d2 < fl(r_c^2), from the positions it already holds, so that the list is
// not read back by a second pass.  Per lane (one particle) it sums, two
// survivors per packed step, with s = (sig^2 / r^2)^3:
//   t = sum (s^2 - s),  q = sum (2 s^2 - s),  f = sum (2 s^2 - s) / r^2 v,
//   n = number of interacting pairs,
// and at the end forms e_i = eps (4 t - phic n), F_i = -24 eps f,
// dU/deps = 1/2 sum_i (4 t - phic n), dU/dsig = 1/2 sum_i (24 eps / sig) (q - dsc n)
// (the same terms as the list pass, summed in another order).  Membership
// is the list's pinned d2 < fl(r_c^2); the value takes v = x_j - x_i - n L
// rounded once, as the list pass does.  A pair that does not interact gets
// r^2 = 1e30: its s underflows to zero and every term vanishes.
struct LJAcc {
    f32x2 t, q, fx, fy, fz;
    float n;
};

__device__ __forceinline__ float lj_rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void lj_terms2(LJAcc &A, float sig2, bool l0, bool l1, float r0, float r1, f32x2 vx,
                                          f32x2 vy, f32x2 vz)
{
    const f32x2 inv = f2_pack(lj_rcp_fast(l0 ? r0 : 1e30f), lj_rcp_fast(l1 ? r1 : 1e30f));
    const f32x2 s2 = f2_mul(f2_pack(sig2, sig2), inv);
    const f32x2 s4 = f2_mul(s2, s2);
    const f32x2 s6 = f2_mul(s4, s2);
    const f32x2 s12 = f2_mul(s6, s6);
    A.t = f2_add(A.t, f2_sub(s12, s6));
    const f32x2 q = f2_sub(f2_add(s12, s12), s6);
    A.q = f2_add(A.q, q);
    const f32x2 w = f2_mul(q, inv);
    A.fx = f2_fma(w, vx, A.fx);
    A.fy = f2_fma(w, vy, A.fy);
    A.fz = f2_fma(w, vz, A.fz);
    A.n += (l0 ? 1.f : 0.f) + (l1 ? 1.f : 0.f);
}

// value offsets of the current image (see Query): n > 0: fl(fl(xj - L) - xi);
// n < 0: fl(xj - fl(xi - L)) (fl(xi + n L) is the image centre); n = 0: fl(xj - xi)
__device__ __forceinline__ void set_lj_value(Query &c, float L)
{
    c.vx1 = c.nLx > 0.f ? L : c.px;
    c.vy1 = c.nLy > 0.f ? L : c.py;
    c.vz1 = c.nLz > 0.f ? L : c.pz;
    c.vx2 = c.nLx > 0.f ? c.xi : 0.f;
    c.vy2 = c.nLy > 0.f ? c.yi : 0.f;
    c.vz2 = c.nLz > 0.f ? c.zi : 0.f;
}

// LJ terms of one pair already tested (scalar: odd survivors, single leaves)
template <bool SHIFT>
__device__ __forceinline__ void lj_single(LJAcc &A, const Query &c, float sig2, float rc2, bool acc, float d2,
                                          float4 q)
{
    float vx, vy, vz, r2;
    if (SHIFT) {
        vx = __fsub_rn(__fsub_rn(q.x, c.vx1), c.vx2);
        vy = __fsub_rn(__fsub_rn(q.y, c.vy1), c.vy2);
        vz = __fsub_rn(__fsub_rn(q.z, c.vz1), c.vz2);
        r2 = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
    } else {
        vx = __fsub_rn(q.x, c.xi);
        vy = __fsub_rn(q.y, c.yi);
        vz = __fsub_rn(q.z, c.zi);
        r2 = d2;
    }
    lj_terms2(A, sig2, acc && d2 < rc2, false, r2, 1e30f, f2_pack(vx, 0.f), f2_pack(vy, 0.f), f2_pack(vz, 0.f));
}

struct LJCtx {
    LJAcc *acc;   // nullptr: no LJ terms
    float sig2, rc2;
};

// Two survivors (x, y, z as packed pairs, original indices id) against the
// lane's particle.
// Z-order indices of a warp's survivors (double-precision data only): a
// second array after the block's stages in dynamic shared memory.
__device__ __forceinline__ const int *stage_zid(const BundleStage *st)
{
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    return reinterpret_cast<const int *>(st - warp + nw) + warp * kStage;
}

// Double-precision data: the decision for a survivor (Z-order index j) whose
// FP32 d2 lies inside the band around r^2 (see exact_d2_64).
template <bool SHIFT>
__device__ __forceinline__ bool band_decide(const QueryArgs &A, const Query &c, int j)
{
    return exact_d2_64<SHIFT>(A, c, j) < A.r2_64[c.pair];
}

template <bool SHIFT, bool SELF, bool LJ = false, bool F64 = false>
__device__ __forceinline__ void survivor_vals(const Query &c, Row &out, const f32x2 X, const f32x2 Y, const f32x2 Z,
                                              const int2 id, bool on, bool staged, const LJCtx &lj,
                                              const QueryArgs *A = nullptr, const BundleStage *st = nullptr,
                                              int t = 0)
{
    f32x2 dx = f2_sub(X, f2_pack(c.xi, c.xi)), dy = f2_sub(Y, f2_pack(c.yi, c.yi)),
          dz = f2_sub(Z, f2_pack(c.zi, c.zi));
    if (SHIFT) {
        dx = f2_sub(dx, f2_pack(c.nLx, c.nLx));
        dy = f2_sub(dy, f2_pack(c.nLy, c.nLy));
        dz = f2_sub(dz, f2_pack(c.nLz, c.nLz));
    }
    float sx0, sx1, sy0, sy1, sz0, sz1;
    f2_unpack(f2_mul(dx, dx), sx0, sx1);
    f2_unpack(f2_mul(dy, dy), sy0, sy1);
    f2_unpack(f2_mul(dz, dz), sz0, sz1);
    const float d0 = __fadd_rn(__fadd_rn(sx0, sy0), sz0);
    const float d1 = __fadd_rn(__fadd_rn(sx1, sy1), sz1);
    bool a0, a1;
    if (F64) {
        // FP32 decides outside the band [rl2_lo, rl2_hi], FP64 inside it (rare)
        const bool s0 = on && (!SELF || id.x != c.self_id), s1 = on && (!SELF || id.y != c.self_id);
        a0 = s0 && d0 < c.rl2_lo;
        a1 = s1 && d1 < c.rl2_lo;
        const bool b0 = s0 && !(d0 < c.rl2_lo) && d0 <= c.rl2_hi;
        const bool b1 = s1 && !(d1 < c.rl2_lo) && d1 <= c.rl2_hi;
        if (b0 || b1) {
            const int *zid = stage_zid(st);
            if (b0) a0 = band_decide<SHIFT>(*A, c, zid[t]);
            if (b1) a1 = band_decide<SHIFT>(*A, c, zid[t + 1]);
        }
    } else {
        a0 = on && d0 < c.rl2 && (!SELF || id.x != c.self_id);
        a1 = on && d1 < c.rl2 && (!SELF || id.y != c.self_id);
    }
    if (LJ) {
        f32x2 vx = dx, vy = dy, vz = dz;
        float r0 = d0, r1 = d1;
        if (SHIFT) {
            vx = f2_sub(f2_sub(X, f2_pack(c.vx1, c.vx1)), f2_pack(c.vx2, c.vx2));
            vy = f2_sub(f2_sub(Y, f2_pack(c.vy1, c.vy1)), f2_pack(c.vy2, c.vy2));
            vz = f2_sub(f2_sub(Z, f2_pack(c.vz1, c.vz1)), f2_pack(c.vz2, c.vz2));
            float ux0, ux1, uy0, uy1, uz0, uz1;
            f2_unpack(f2_mul(vx, vx), ux0, ux1);
            f2_unpack(f2_mul(vy, vy), uy0, uy1);
            f2_unpack(f2_mul(vz, vz), uz0, uz1);
            r0 = __fadd_rn(__fadd_rn(ux0, uy0), uz0);
            r1 = __fadd_rn(__fadd_rn(ux1, uy1), uz1);
        }
        lj_terms2(*lj.acc, lj.sig2, a0 && d0 < lj.rc2, a1 && d1 < lj.rc2, r0, r1, vx, vy, vz);
    }
    if (staged) {
        out.stage(id.x, a0);
        out.stage(id.y, a1);
    } else {
        if (a0) out.push(id.x);
        if (a1) out.push(id.y);
    }
}

// survivors t, t + 1 of the stage (8-byte loads)
template <bool SHIFT, bool SELF, bool LJ = false, bool F64 = false>
__device__ __forceinline__ void survivor_pair(const Query &c, Row &out, int t, bool on, const BundleStage *st,
                                              bool staged, const LJCtx &lj = LJCtx{}, const QueryArgs *A = nullptr)
{
    survivor_vals<SHIFT, SELF, LJ, F64>(c, out, *reinterpret_cast<const f32x2 *>(st->x + t),
                                        *reinterpret_cast<const f32x2 *>(st->y + t),
                                        *reinterpret_cast<const f32x2 *>(st->z + t),
                                        *reinterpret_cast<const int2 *>(st->id + t), on, staged, lj, A, st, t);
}

// survivors t .. t + 3 of the stage, t a multiple of 4 (16-byte loads; each
// half of a loaded float4 is an aligned register pair).  QBVH_SURVIVOR_QUAD = 0
// loads two survivors at a time instead.
#ifndef QBVH_SURVIVOR_QUAD
#define QBVH_SURVIVOR_QUAD 1
#endif
template <bool SHIFT, bool SELF, bool LJ = false, bool F64 = false>
__device__ __forceinline__ void survivor_quad(const Query &c, Row &out, int t, bool on, const BundleStage *st,
                                              const LJCtx &lj, const QueryArgs *A = nullptr)
{
    const float4 X = *reinterpret_cast<const float4 *>(st->x + t);
    const float4 Y = *reinterpret_cast<const float4 *>(st->y + t);
    const float4 Z = *reinterpret_cast<const float4 *>(st->z + t);
    const int4 I = *reinterpret_cast<const int4 *>(st->id + t);
    survivor_vals<SHIFT, SELF, LJ, F64>(c, out, f2_pack(X.x, X.y), f2_pack(Y.x, Y.y), f2_pack(Z.x, Z.y),
                                        make_int2(I.x, I.y), on, true, lj, A, st, t);
    survivor_vals<SHIFT, SELF, LJ, F64>(c, out, f2_pack(X.z, X.w), f2_pack(Y.z, Y.w), f2_pack(Z.z, Z.w),
                                        make_int2(I.z, I.w), on, true, lj, A, st, t + 2);
}

// Every lane tests every survivor (one particle per lane), two per step: the
// differences and squares as packed f32x2 pairs, the two sums as scalar adds
// -- the same operations in the same order as exact_d2.  (ptxas contracts a
// packed mul.rn.f32x2 feeding a packed add.rn.f32x2 into one fused
// multiply-add, which changes the rounding of d2: measured on GB300, 8 rows
// of the N = 2M list differed at d = r_list.  Scalar add.rn is not contracted.)
// With row staging the accepted entries are staged without a branch and the
// completed sectors written once per 8 survivors and at the end.
template <bool SHIFT, bool SELF, bool LJ = false, bool F64 = false>
__device__ __forceinline__ void survivors_loop(const Query &c, Row &out, int s, bool on, const BundleStage *st,
                                               const LJCtx &lj = LJCtx{}, const QueryArgs *A = nullptr)
{
    const bool staged = out.ring != nullptr;
    int t = 0;
    if (staged) {
        for (; t + 8 <= s; t += 8) {
#if QBVH_SURVIVOR_QUAD
            survivor_quad<SHIFT, SELF, LJ, F64>(c, out, t, on, st, lj, A);
            survivor_quad<SHIFT, SELF, LJ, F64>(c, out, t + 4, on, st, lj, A);
#else
            survivor_pair<SHIFT, SELF, LJ, F64>(c, out, t, on, st, true, lj, A);
            survivor_pair<SHIFT, SELF, LJ, F64>(c, out, t + 2, on, st, true, lj, A);
            survivor_pair<SHIFT, SELF, LJ, F64>(c, out, t + 4, on, st, true, lj, A);
            survivor_pair<SHIFT, SELF, LJ, F64>(c, out, t + 6, on, st, true, lj, A);
#endif
            out.check();
        }
    }
    for (; t + 1 < s; t += 2) survivor_pair<SHIFT, SELF, LJ, F64>(c, out, t, on, st, staged, lj, A);
    if (t < s) {
        const float4 q = make_float4(st->x[t], st->y[t], st->z[t], 0.f);
        const int id = st->id[t];
        const float d2 = exact_d2<SHIFT>(c, q);
        bool acc = on && d2 < (F64 ? c.rl2_lo : c.rl2) && (!SELF || id != c.self_id);
        if (F64 && on && (!SELF || id != c.self_id) && !(d2 < c.rl2_lo) && d2 <= c.rl2_hi)
            acc = band_decide<SHIFT>(*A, c, stage_zid(st)[t]);
        if (LJ) lj_single<SHIFT>(*lj.acc, c, lj.sig2, lj.rc2, acc, d2, q);
        if (staged) out.stage(id, acc);
        else if (acc) out.push(id);
    }
    if (staged) out.check();
}

// W > 1 lanes per particle: lane wsub of a particle tests the survivor pairs
// 2 (k W + wsub), k = 0, 1, ..., and stages what it accepts in its own ring
// (s is a multiple of 2 W).  Between two checks a lane stages 8 survivors.
template <bool SHIFT, bool SELF, int W>
__device__ __forceinline__ void survivors_loop_w(const Query &c, Row &out, int s, bool on, const BundleStage *st,
                                                 int wsub, unsigned same)
{
    const int steps = s / (2 * W);
    int t = 2 * wsub;
    int k = 0;
    for (; k + 4 <= steps; k += 4) {
        survivor_pair<SHIFT, SELF>(c, out, t, on, st, true);
        survivor_pair<SHIFT, SELF>(c, out, t + 2 * W, on, st, true);
        survivor_pair<SHIFT, SELF>(c, out, t + 4 * W, on, st, true);
        survivor_pair<SHIFT, SELF>(c, out, t + 6 * W, on, st, true);
        t += 8 * W;
        out.check_group(same);
    }
    for (; k < steps; ++k) {
        survivor_pair<SHIFT, SELF>(c, out, t, on, st, true);
        t += 2 * W;
    }
    out.check_group(same);
}

// Survivors spread over the warp when few lanes overlap the bundle: the s
// survivors occupy s lanes of each of kk = 32 / width slots (width 32, 16 or
// 8 lanes), and each trip serves kk overlapping particles, whose centre,
// index and count come by shuffle.  A particle's accepted survivors are
// packed in survivor order, so the row is the same as with the loop above.
template <bool SHIFT, bool SELF>
__device__ __forceinline__ void survivors_spread(const QueryArgs &a, const Query &c, Row &out, int s, int m, int wsh,
                                                 unsigned hm, const BundleStage *st)
{
    const int lane = threadIdx.x & 31;
    const int kk = 32 >> wsh;                       // particles per trip
    const int slot = lane >> wsh;
    const int t = lane & ((1 << wsh) - 1);
    const bool tv = t < s;
    const int tt = tv ? t : 0;
    const float4 q = make_float4(st->x[tt], st->y[tt], st->z[tt], 0.f);
    const int id = st->id[tt];
    const unsigned wmask = wsh == 5 ? FULL : ((1u << (1 << wsh)) - 1u);
    const unsigned smask = wmask << (slot << wsh);  // lanes of my slot
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const int my_rank = ((hm >> lane) & 1u) ? __popc(hm & lt) : -1;
    for (int base = 0; base < m; base += kk) {
        const int oi = base + slot;
        const int owner = oi < m ? st->owner[oi] : -1;
        const int src = owner < 0 ? lane : owner;
        Query u = c;
        u.xi = __shfl_sync(FULL, c.xi, src);
        u.yi = __shfl_sync(FULL, c.yi, src);
        u.zi = __shfl_sync(FULL, c.zi, src);
        const int ocount = __shfl_sync(FULL, out.count, src);
        const int oid = __shfl_sync(FULL, c.self_id, src);
        const bool acc = owner >= 0 && tv && exact_d2<SHIFT>(u, q) < c.rl2 && (!SELF || id != oid);
        const unsigned mb = __ballot_sync(FULL, acc);
        if (acc) {
            const int pos = ocount + __popc(mb & smask & lt);
            if (pos < out.cap) row_store(a.rows + (size_t)oid * out.cap + pos, id);
        }
        const int sl = my_rank - base;
        if (sl >= 0 && sl < kk) out.count += __popc(mb & (wmask << (sl << wsh)));
    }
}

// A chunk of cnt <= 32 leaves starting at `first` of a bundle overlapped by
// the lanes in hm (warp-uniform).  Every lane of the warp calls this together.
template <bool SHIFT, bool SELF, bool LJ = false>
__device__ __forceinline__ void bundle_chunk(const QueryArgs &a, const Query &c, Row &out, int first, int cnt,
                                             unsigned hm, bool on, float rs2, BundleStage *st,
                                             const LJCtx &lj = LJCtx{})
{
    const int lane = threadIdx.x & 31;
    const bool v = lane < cnt;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v) q = tree_ld(a.leaves + first + lane);
    const float4 lo = st->blo, hi = st->bhi;
    const float gx = fmaxf(fmaxf(__fsub_rd(lo.x, q.x), __fsub_rd(q.x, hi.x)), 0.f);
    const float gy = fmaxf(fmaxf(__fsub_rd(lo.y, q.y), __fsub_rd(q.y, hi.y)), 0.f);
    const float gz = fmaxf(fmaxf(__fsub_rd(lo.z, q.z), __fsub_rd(q.z, hi.z)), 0.f);
    const float g2 = __fmaf_rd(gx, gx, __fmaf_rd(gy, gy, __fmul_rd(gz, gz)));
    const bool surv = v && g2 <= rs2;
    const unsigned S = __ballot_sync(FULL, surv);
    if (S == 0u) return;
    const int s = __popc(S);
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    if (surv) {
        const int r = __popc(S & lt);
        st->x[r] = q.x;
        st->y[r] = q.y;
        st->z[r] = q.z;
        st->id[r] = __float_as_int(q.w) & 0x7FFFFFFF;
    }
    // spread when it takes fewer instructions than the loop (about 25 + 3 kk
    // per trip against 14 per survivor step)
    const int m = __popc(hm);
    const int wsh = s <= 8 ? 3 : (s <= 16 ? 4 : 5);
    const int kk = 32 >> wsh;
    const bool spread = QBVH_FILTER_SPREAD && !QBVH_ROW_STAGING && !LJ && m <= QBVH_FILTER_SPREAD_MAX &&
                        (QBVH_SPREAD_COST + 3 * kk) * ((m + kk - 1) / kk) < QBVH_LOOP_COST * s;
    if (spread && ((hm >> lane) & 1u)) st->owner[__popc(hm & lt)] = lane;
    __syncwarp();
    if (spread) survivors_spread<SHIFT, SELF>(a, c, out, s, m, wsh, hm, st);
    else survivors_loop<SHIFT, SELF, LJ>(c, out, s, on, st, lj);
    __syncwarp();   // the next bundle rewrites the stage
}

// The filter of a chunk of cnt <= 32 leaves starting at `first`: its
// survivors are appended to the stage after the s already there; returns the
// new count (warp-uniform).  Every lane of the warp calls this together.
template <bool F64 = false>
__device__ __forceinline__ int chunk_filter(const QueryArgs &a, int first, int cnt, float rs2, BundleStage *st,
                                            int s)
{
    const int lane = threadIdx.x & 31;
    const bool v = lane < cnt;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v) q = tree_ld(a.leaves + first + lane);
    const float4 lo = st->blo, hi = st->bhi;
    const float gx = fmaxf(fmaxf(__fsub_rd(lo.x, q.x), __fsub_rd(q.x, hi.x)), 0.f);
    const float gy = fmaxf(fmaxf(__fsub_rd(lo.y, q.y), __fsub_rd(q.y, hi.y)), 0.f);
    const float gz = fmaxf(fmaxf(__fsub_rd(lo.z, q.z), __fsub_rd(q.z, hi.z)), 0.f);
    const float g2 = __fmaf_rd(gx, gx, __fmaf_rd(gy, gy, __fmul_rd(gz, gz)));
    const bool surv = v && g2 <= rs2;
    const unsigned S = __ballot_sync(FULL, surv);
    if (surv) {
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        const int r = s + __popc(S & lt);
        st->x[r] = q.x;
        st->y[r] = q.y;
        st->z[r] = q.z;
        st->id[r] = __float_as_int(q.w) & 0x7FFFFFFF;
        if (F64) const_cast<int *>(stage_zid(st))[r] = first + lane;
    }
    return s + __popc(S);
}

// A bundle of cnt <= 64 leaves.  Both 32-leaf chunks are filtered into the
// stage first and the survivors tested in one loop.  The count is padded to a
// multiple of 2 W with points at 1e30 in every coordinate: their squared
// distance overflows to +inf, so no lane accepts them, and their LJ terms are
// zero.  (With the spread of few-lane bundles, a build option without row
// staging, chunks are tested one at a time.)
template <bool SHIFT, bool SELF, bool LJ = false, int W = 1, bool F64 = false>
__device__ __forceinline__ void bundle_filtered(const QueryArgs &a, const Query &c, Row &out, int first, int cnt,
                                                unsigned hm, bool on, float rs2, BundleStage *st,
                                                const LJCtx &lj = LJCtx{}, int wsub = 0, unsigned same = 0u)
{
    constexpr bool PER_CHUNK = QBVH_FILTER_SPREAD && !QBVH_ROW_STAGING;
    if (PER_CHUNK) {
        for (int base = 0; base < cnt; base += 32)
            bundle_chunk<SHIFT, SELF, LJ>(a, c, out, first + base, min(32, cnt - base), hm, on, rs2, st, lj);
        return;
    }
    int s = 0;
    for (int base = 0; base < cnt; base += 32)
        s = chunk_filter<F64>(a, first + base, min(32, cnt - base), rs2, st, s);
    if (s == 0) return;
    const int pad = (2 * W - s % (2 * W)) % (2 * W);   // s <= 64, a multiple of 2 W: s + pad <= 64
    const int lane = threadIdx.x & 31;
    if (lane < pad) {
        st->x[s + lane] = 1e30f;
        st->y[s + lane] = 1e30f;
        st->z[s + lane] = 1e30f;
        st->id[s + lane] = 0;
        if (F64) const_cast<int *>(stage_zid(st))[s + lane] = first;   // never read: +inf is outside the band
    }
    s += pad;
    __syncwarp();
    if (W == 1) survivors_loop<SHIFT, SELF, LJ, F64>(c, out, s, on, st, lj, &a);
    else survivors_loop_w<SHIFT, SELF, W>(c, out, s, on, st, wsub, same);
    __syncwarp();   // the next bundle rewrites the stage
}

// bundle leaves tested two per step (two loads in flight; measured 2.25 ->
// 2.20 ms at N = 2M) or one per step
#ifndef QBVH_LEAF_PAIRS
#define QBVH_LEAF_PAIRS 1
#endif
// Every lane tests every leaf j..l of a bundle (one particle per lane).
template <bool CAND, bool SHIFT, bool F64, bool SELF, int FMT>
__device__ __forceinline__ void bundle_loop(const QueryArgs &a, const Query &c, Row &out, int j, int l,
                                            const Frame &f, float rs2, bool on)
{
#if QBVH_LEAF_PAIRS
    for (; j < l; j += 2) {   // two leaves per step: two loads in flight
        const float4 q0 = tree_ld(a.leaves + j);
        const float4 q1 = tree_ld(a.leaves + j + 1);
        if (on) {
            test_leaf<CAND, SHIFT, F64, SELF, FMT>(a, c, out, j, q0, f, rs2);
            test_leaf<CAND, SHIFT, F64, SELF, FMT>(a, c, out, j + 1, q1, f, rs2);
        }
    }
#endif
    for (; j <= l; ++j) {
        const float4 q = tree_ld(a.leaves + j);
        if (on) test_leaf<CAND, SHIFT, F64, SELF, FMT>(a, c, out, j, q, f, rs2);
    }
}

// Registers are capped so that 8 blocks of 256 threads (64 warps) fit on an
// SM: the walk is latency-bound and more resident warps hide more of it
// (measured 2.37 -> 2.23 ms at N = 2M despite a few spilled bytes).
#ifndef QBVH_QUERY_MIN_BLOCKS
#define QBVH_QUERY_MIN_BLOCKS 8
#endif
// ---- one warp per 32 consecutive Z-order particles ----------------------
// The warp-uniform rope walk of one tree under one periodic image.
template <bool CAND, int FMT, bool SHIFT, int W, bool F64, bool LJ = false>
__device__ __forceinline__ void warp_walk(const QueryArgs &a, const Query &c, Row &out, const SegInfo &g,
                                          const Frame &f, int root, int last, bool on, float rs2, int wsub,
                                          unsigned same, BundleStage *st = nullptr, float rs = 0.f,
                                          const LJCtx &lj = LJCtx{})
{
    static_assert(!LJ || (stage_on(W, CAND, F64) && !CAND && !F64 && W == 1), "LJ terms need the filtered walk");
    // bundles filtered against the warp's box (one particle per lane, exact lists of FP32 data)
    constexpr bool FILTER = stage_on(W, CAND, F64);
    // 10-bit nodes tested in the integer domain on the same walks
    constexpr bool QCUBE = FILTER && FMT == 0 && QBVH_QCUBE;
    if (FILTER) packet_box(c, on, st);
    LaneCube cube;
    if (QCUBE) cube = lane_cube(c, on, f, rs);
    const float lrs2 = on ? rs2 : -1.f;   // a negative squared radius overlaps nothing
    int node = root;
    int budget = 2 * g.count;
    while (node != QBVH_END) {
        if (--budget < 0 || bad_node(node, g, last)) {
            atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            break;
        }
        if (node >= 0) {
            const Raw w = load_raw<FMT>(a, node);
            Node nd;
            bool hit;
            if (QCUBE) {
                hit = cube_overlap((unsigned)w.q.x, (unsigned)w.q.y, cube);
                nd.left = w.q.z;
                nd.rope = w.q.w;
                nd.bundle = w.q.x < 0;
            } else {
                nd = decode<FMT>(w, f);
                hit = overlap(c.px, c.py, c.pz, nd, lrs2);
            }
            const unsigned hm = __ballot_sync(FULL, hit);
            if (hm) {
                if (nd.bundle) {
                    int l = bundle_last(nd, last);
                    if (nd.left < g.start || l > last) {
                        atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                        l = nd.left - 1;
                    }
                    int j = nd.left;
                    // only a bundle holding one of the warp's own particles can
                    // hand a lane its own leaf, and only under the zero image
                    const bool self_here =
                        !SHIFT && __any_sync(FULL, (unsigned)(c.self - j) <= (unsigned)(l - j));
                    if (FILTER && l - j < 64) {
                        if (self_here)
                            bundle_filtered<SHIFT, true, LJ, W, F64>(a, c, out, j, l - j + 1, hm, on, rs2, st, lj,
                                                                     wsub, same);
                        else
                            bundle_filtered<SHIFT, false, LJ, W, F64>(a, c, out, j, l - j + 1, hm, on, rs2, st, lj,
                                                                      wsub, same);
                    } else if (W == 1 && !CAND && l - j < 32 && __popc(hm) <= QBVH_SPREAD_MAX) {
                        if (self_here) bundle_spread<SHIFT, F64, true>(a, c, out, j, l - j + 1, hm);
                        else bundle_spread<SHIFT, F64, false>(a, c, out, j, l - j + 1, hm);
                    } else if (W == 1) {
                        if (self_here || CAND) bundle_loop<CAND, SHIFT, F64, true, FMT>(a, c, out, j, l, f, rs2, on);
                        else bundle_loop<CAND, SHIFT, F64, false, FMT>(a, c, out, j, l, f, rs2, on);
                    } else {
                        // the W lanes of a particle take every W-th leaf
                        for (; j <= l; j += W) {
                            const int jj = j + wsub;
                            bool acc = false;
                            int id = 0;
                            if (jj <= l) {
                                const float4 q = tree_ld(a.leaves + jj);
                                acc = on && leaf_accepts<CAND, SHIFT, F64, FMT>(a, c, jj, q, f, rs2);
                                id = __float_as_int(q.w) & 0x7FFFFFFF;
                            }
                            push_shared(out, acc, id, same);
                        }
                    }
                    node = nd.rope;
                } else {
                    node = nd.left;
                }
            } else {
                node = nd.rope;
            }
        } else {
            const int j = ~node;
            const float4 q = tree_ld(a.leaves + j);
            if (LJ) {
                const float d2 = exact_d2<SHIFT>(c, q);
                const bool acc = on && d2 < c.rl2 && j != c.self;
                lj_single<SHIFT>(*lj.acc, c, lj.sig2, lj.rc2, acc, d2, q);
                if (acc) out.push(__float_as_int(q.w) & 0x7FFFFFFF);
            } else if (W == 1) {
                if (on) test_leaf<CAND, SHIFT, F64, true, FMT>(a, c, out, j, q, f, rs2);
            } else if (FILTER) {
                // the group's row goes through the staging rings
                const bool acc = wsub == 0 && on && leaf_accepts<CAND, SHIFT, F64, FMT>(a, c, j, q, f, rs2);
                out.stage(__float_as_int(q.w) & 0x7FFFFFFF, acc);
                out.check_group(same);
            } else {
                const bool acc = wsub == 0 && on && leaf_accepts<CAND, SHIFT, F64, FMT>(a, c, j, q, f, rs2);
                push_shared(out, acc, __float_as_int(q.w) & 0x7FFFFFFF, same);
            }
            node = (j == last) ? QBVH_END : ((__float_as_int(q.w) < 0) ? j + 1 : ~(j + 1));
        }
    }
}

#if QBVH_QUERY_MIN_BLOCKS > 0
#define QBVH_QUERY_BOUNDS __launch_bounds__(256, QBVH_QUERY_MIN_BLOCKS)
#else
#define QBVH_QUERY_BOUNDS
#endif

// W lanes per particle: a warp serves 32 / W consecutive Z-order particles;
// lane l works for particle l % (32 / W) and takes every W-th leaf of a bundle
// starting at l / (32 / W).
//
// PHASE 2 (the default) walks every periodic image in one launch.  With
// QBVH_QUERY_SPLIT_IMAGES = 1 the images go to two launches instead: PHASE 0
// walks the zero image of every tree (a particle lies inside its own box, so
// this image is never empty) and PHASE 1 the other images, which only
// particles within the search radius of a box face need, appending after the
// phase-0 entries (the count comes from counts[]).  The split removes the
// register spills of the zero-image walk but the image launch runs with few
// busy warps: 1.92 ms in one launch against 2.01 ms in two at N = 2M.
// ONE: a single tree (one system, one type), segment and type loops
// compiled out.
#ifndef QBVH_QUERY_SPLIT_IMAGES
#define QBVH_QUERY_SPLIT_IMAGES 0
#endif
#ifndef QBVH_REVERSE_BLOCKS
#define QBVH_REVERSE_BLOCKS 1
#endif
// ---- sparse trees: one particle per warp ---------------------------------
// A tree of few, widely spaced particles (the large spheres of a
// size-asymmetric mixture) makes poor packets: 32 consecutive Z-order
// particles then span much of the box, so a packet walk is 32 separate
// walks run one after another on one warp, and the few such warps end long
// after the rest (mixture L = 100: the 400 large particles' walks of the
// small-particle tree took 1.5 ms against 0.55 ms for all small-small
// pairs).  Tree `ta` of a single-system FP32 build of 2 to 4 types (32-bit
// keys) is walked one particle per warp instead when it holds at most
// QBVH_SPARSE_MAX particles and a packet of 32 spans more than twice its
// largest list radius:
// 32 L^3 / count > (2 r_max)^3.  The choice changes only which warp walks a
// particle: the walk visits the same nodes and leaves in the same order, so
// rows are the same either way.
#ifndef QBVH_SPARSE_TREES
#define QBVH_SPARSE_TREES 1
#endif
#ifndef QBVH_SPARSE_MAX
#define QBVH_SPARSE_MAX 4096
#endif
__device__ __forceinline__ bool sparse_tree(const QueryArgs &a, int ta)
{
    const int count = a.seg[ta].count;
    if (count == 0 || count > QBVH_SPARSE_MAX) return false;
    const int T = a.n_types;
    float r = 0.f;
    for (int tb = 0; tb < T; ++tb) r = fmaxf(r, a.r_list[ta * T + tb]);
    const float L = a.sys[0].L, d = 2.f * r;
    return 32.f * L * L * L > (float)count * d * d * d;
}

// The leading a.sparse_blocks blocks: every particle of a sparse tree gets a
// whole warp (W = 32: the lanes share the walk and split each bundle's
// leaves), warps taking particles in a grid-stride loop.
template <int FMT>
__device__ __forceinline__ void sparse_walks(const QueryArgs &a)
{
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((a.sparse_blocks * blockDim.x) >> 5);
    const int T = a.n_types;
    const float L = a.sys[0].L;
    for (int ta = 0; ta < T; ++ta) {
        if (!sparse_tree(a, ta)) continue;
        const int start = a.seg[ta].start, count = a.seg[ta].count;
        for (int p = gw; p < count; p += nw) {
            const int s = start + p;
            const float4 me = __ldg(a.leaves + s);
            int i_orig = __float_as_int(me.w) & 0x7FFFFFFF;
            if (i_orig >= a.n) {
                atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                i_orig = s;
            }
            Query c;
            c.xi = me.x;
            c.yi = me.y;
            c.zi = me.z;
            c.self = s;
            c.self_id = i_orig;
            Row out;
            out.row = a.rows + (size_t)i_orig * a.cap;
            out.cap = a.cap;
            out.count = 0;
            out.ring = nullptr;
            out.base = 0;
            for (int tb = 0; tb < T; ++tb) {
                if (!(a.r_list[ta * T + tb] > 0.f)) continue;
                const SegInfo g = a.seg[tb];
                if (g.count == 0) continue;
                c.rl2 = a.rl2[ta * T + tb];
                const float rs2 = a.rs2[ta * T + tb];
                const Frame f = FMT == 2 ? frame21_of(g) : frame_of(g);
                const int root = g.count >= 2 ? g.start : ~g.start;
                const int last = g.start + g.count - 1;
                unsigned mask = image_mask(me.x, me.y, me.z, L, g, rs2);
                while (mask) {
                    const int img = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    set_image(c, img, L);
                    if (img == 13)
                        warp_walk<false, FMT, false, 32, false>(a, c, out, g, f, root, last, true, rs2, lane, FULL);
                    else
                        warp_walk<false, FMT, true, 32, false>(a, c, out, g, f, root, last, true, rs2, lane, FULL);
                }
            }
            if (lane == 0) a.counts[i_orig] = out.count;
            warp_max_count(out.count, a.status);
        }
    }
}

// lanes 0, G, 2G, ... of a warp with W lanes per particle (G = 32 / W
// particles): the lanes of particle 0
__host__ __device__ constexpr unsigned same_lanes(int W)
{
    unsigned m = 0u;
    for (int k = 0; k < W; ++k) m |= 1u << (k * (32 / W));
    return m;
}

// Register cap of the traversal that also sums the LJ terms: its eleven
// accumulators do not fit under the plain walk's 32 registers.
#ifndef QBVH_QUERY_LJ_MIN_BLOCKS
#define QBVH_QUERY_LJ_MIN_BLOCKS 5
#endif

// FP64 record of one block: the fixed-order sum over its lanes of U, dU/deps
// and dU/dsig (the same three values the list pass writes per block)
__device__ __forceinline__ void lj_block_record(const QueryArgs &a, double v0, double v1, double v2)
{
    __shared__ double s_red[8][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(FULL, v0, o);
        v1 += __shfl_down_sync(FULL, v1, o);
        v2 += __shfl_down_sync(FULL, v2, o);
    }
    if (lane == 0) {
        s_red[warp][0] = v0;
        s_red[warp][1] = v1;
        s_red[warp][2] = v2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += s_red[w][threadIdx.x];
        a.lj_partials[(size_t)blockIdx.x * 3 + threadIdx.x] = x;
    }
}

// One packet: the G = 32 / W consecutive Z-order particles p G, ..., p G + G - 1
// walked by this warp.  Every lane of the warp calls this together.
template <bool WIDE, bool CAND, int FMT, int W, bool ONE, int PHASE, bool F64, bool LJ>
__device__ __forceinline__ void warp_packet(const QueryArgs &a, int p)
{
    static_assert(!LJ || (ONE && W == 1 && !CAND && !F64 && PHASE == 2), "LJ terms: one tree, filtered walk");
    constexpr int G = 32 / W;
    // sparse trees (above) exist for single-system builds with several types
    constexpr bool SPARSE = QBVH_SPARSE_TREES && !WIDE && !ONE && !CAND && !F64 && PHASE == 2;
    const int lane = threadIdx.x & 31;
    const int pidx = lane % G;
    const int wsub = lane / G;
    const unsigned same = same_lanes(W) << pidx;
    const int s = p * G + pidx;
    const bool active = s < a.n;
    float4 me = make_float4(0.f, 0.f, 0.f, 0.f);
    int i_orig = 0, seg_i = -1;
    if (active) {
        me = __ldg(a.leaves + s);
        i_orig = __float_as_int(me.w) & 0x7FFFFFFF;
        if (i_orig >= a.n) {
            if (PHASE == 0) atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            i_orig = s;
        }
        seg_i = ONE ? 0 : seg_of_sorted<WIDE>(a, s);
    }
    Query c;
    c.xi = me.x;
    c.yi = me.y;
    c.zi = me.z;
    c.self = s;
    c.self_id = i_orig;
    Row out;
    out.row = a.rows + (size_t)i_orig * a.cap;
    out.cap = a.cap;
    out.count = (PHASE == 1 && active) ? a.counts[i_orig] : 0;
    constexpr bool STAGE = stage_on(W, CAND, F64);
    // one BundleStage per warp, in dynamic shared memory sized to the block
    extern __shared__ BundleStage stage[];
    BundleStage *st = STAGE ? &stage[threadIdx.x >> 5] : nullptr;
    // row staging on the filtered walks (every push of those walks goes through it)
    constexpr bool RING = STAGE && QBVH_ROW_STAGING && PHASE == 2;
    out.ring = RING ? st->ring + lane : nullptr;
    out.base = 0;
    out.fill = 0;
    bool walked = PHASE != 1;
    bool elsewhere = false;   // particle of a sparse tree: walked by the leading blocks
    LJAcc acc;
    LJCtx lj;
    if (LJ) {
        acc.t = acc.q = acc.fx = acc.fy = acc.fz = f2_pack(0.f, 0.f);
        acc.n = 0.f;
        const float sg = __ldg(a.lj_sig);
        lj.acc = &acc;
        lj.sig2 = sg * sg;
        lj.rc2 = a.lj_rc2;
    }
    const int T = ONE ? 1 : a.n_types;
    // the warp's particles may belong to several trees (segment boundaries):
    // take one segment value at a time
    unsigned remaining = __ballot_sync(FULL, active);
    while (remaining) {
        const int seg = ONE ? 0 : __shfl_sync(FULL, seg_i, __ffs(remaining) - 1);
        const bool part = ONE ? active : (active && seg_i == seg);
        remaining = ONE ? 0u : (remaining & ~__ballot_sync(FULL, part));
        if (SPARSE && a.sparse_blocks > 0 && sparse_tree(a, seg)) {
            elsewhere = elsewhere || part;
            continue;
        }
        const int sys = seg / T;
        const int ta = seg - sys * T;
        const float L = a.sys[sys].L;
        for (int tb = 0; tb < T; ++tb) {
            const float rl = a.r_list[ta * T + tb];
            if (!(rl > 0.f)) continue;
            const SegInfo g = a.seg[sys * T + tb];
            if (g.count == 0) continue;
            c.rl2 = a.rl2[ta * T + tb];
            if (F64) {
                c.rl2_lo = a.rl2_lo[ta * T + tb];
                c.rl2_hi = a.rl2_hi[ta * T + tb];
                c.pair = ta * T + tb;
            }
            const float rs2 = a.rs2[ta * T + tb];
            const float rs = a.rs[ta * T + tb];
            const Frame f = FMT == 2 ? frame21_of(g) : frame_of(g);
            const int root = g.count >= 2 ? g.start : ~g.start;
            const int last = g.start + g.count - 1;
            if (PHASE == 0) {
                // zero image: the walk's own root test decides whether it is empty
                set_image(c, 13, L);
                warp_walk<CAND, FMT, false, W, F64>(a, c, out, g, f, root, last, part, rs2, wsub, same, st, rs);
                continue;
            }
            unsigned mine = part ? image_mask(me.x, me.y, me.z, L, g, rs2) : 0u;
            if (PHASE == 1) mine &= ~(1u << 13);
            unsigned mask = __reduce_or_sync(FULL, mine);
            walked = walked || mask != 0u;
            while (mask) {
                const int img = __ffs(mask) - 1;
                mask &= mask - 1u;
                set_image(c, img, L);
                if (LJ) set_lj_value(c, L);
                const bool on = (mine >> img) & 1u;
                if (PHASE == 2 && img == 13)
                    warp_walk<CAND, FMT, false, W, F64, LJ>(a, c, out, g, f, root, last, on, rs2, wsub, same, st,
                                                            rs, lj);
                else
                    warp_walk<CAND, FMT, true, W, F64, LJ>(a, c, out, g, f, root, last, on, rs2, wsub, same, st,
                                                           rs, lj);
            }
        }
    }
    if (!walked) return;   // phase 1, no image to add for this warp: counts stay
    if (RING) {
        if (W == 1) {
            if (active && !elsewhere) out.drain();
        } else {
            out.drain_group<W>(same, pidx, G, wsub);   // lanes pidx + m G, every lane together
        }
    }
    // the row index again (not kept live across the walk)
    int io = 0;
    if (active) {
        io = __float_as_int(__ldg(a.leaves + s).w) & 0x7FFFFFFF;
        io = io < a.n ? io : s;
    }
    if (active && wsub == 0 && !elsewhere) a.counts[io] = out.count;
    warp_max_count(active && !elsewhere ? out.count : 0, a.status);
    if (LJ) {
        float t0, t1, q0, q1, x0, x1, y0, y1, z0, z1;
        f2_unpack(acc.t, t0, t1);
        f2_unpack(acc.q, q0, q1);
        f2_unpack(acc.fx, x0, x1);
        f2_unpack(acc.fy, y0, y1);
        f2_unpack(acc.fz, z0, z1);
        const float eps = __ldg(a.lj_eps), sig = __ldg(a.lj_sig);
        const LJParams p = lj_params(eps, sig, a.lj_rc2);
        const float uE = __fsub_rn(4.f * __fadd_rn(t0, t1), p.phic * acc.n);   // sum of u / eps
        const float e = eps * uE;
        const float c24 = -24.f * eps;
        if (active) {
            if (a.lj_e) a.lj_e[io] = 0.5f * e;
            if (a.lj_F) {
                a.lj_F[3 * (size_t)io] = c24 * __fadd_rn(x0, x1);
                a.lj_F[3 * (size_t)io + 1] = c24 * __fadd_rn(y0, y1);
                a.lj_F[3 * (size_t)io + 2] = c24 * __fadd_rn(z0, z1);
            }
        }
        const float gs = (24.f * eps / sig) * __fsub_rn(__fadd_rn(q0, q1), p.dsc * acc.n);
        lj_block_record(a, 0.5 * (double)e, 0.5 * (double)uE, 0.5 * (double)gs);
    }
}

// Packets to warps.  Without PERSIST every warp of the grid walks one packet
// (its index in the grid).  With PERSIST the grid holds about as many warps
// as the GPU keeps resident, and each warp takes packets from a device
// counter until they run out, so that a warp that ends early starts the next
// packet instead of idling until its block's last warp ends.  The counter
// only grows, so the loop ends.  With several types packets are taken from
// the end of the sorted order first: the last trees (in a size-asymmetric
// mixture the large particles, whose packets span wide regions and walk
// longest) start first and overlap the rest instead of running alone at the
// end (mixture L = 100: 2.05 -> 1.89 ms before sparse trees; one type gains
// nothing from it, 1.84 -> 1.87 ms at N = 2M).
template <bool WIDE, bool CAND, int FMT, int W, bool ONE, int PHASE, bool F64, bool LJ, bool PERSIST>
__device__ __forceinline__ void warp_query(const QueryArgs &a)
{
    static_assert(!PERSIST || (!LJ && PHASE == 2), "packet queue: one launch, no per-block LJ records");
    constexpr bool SPARSE = QBVH_SPARSE_TREES && !WIDE && !ONE && !CAND && !F64 && PHASE == 2;
    int bid = (int)blockIdx.x, nblk = (int)gridDim.x;
    if (SPARSE && a.sparse_blocks > 0) {
        if (bid < a.sparse_blocks) {
            sparse_walks<FMT>(a);
            return;
        }
        bid -= a.sparse_blocks;
        nblk -= a.sparse_blocks;
    }
    const bool rev = QBVH_REVERSE_BLOCKS && (ONE ? 1 : a.n_types) > 1;
    if (PERSIST) {
        const int lane = threadIdx.x & 31;
        for (;;) {
            int p = 0;
            if (lane == 0) p = (int)atomicAdd(&a.status->next_packet, 1u);
            p = __shfl_sync(FULL, p, 0);
            if (p >= a.n_packets) break;
            warp_packet<WIDE, CAND, FMT, W, ONE, PHASE, F64, LJ>(a, rev ? a.n_packets - 1 - p : p);
        }
        return;
    }
    const int blk = rev ? nblk - 1 - bid : bid;
    warp_packet<WIDE, CAND, FMT, W, ONE, PHASE, F64, LJ>(a, (int)((blk * blockDim.x + threadIdx.x) >> 5));
}

template <bool WIDE, bool CAND, int FMT, int W, bool ONE, int PHASE, bool F64 = false>
__global__ void QBVH_QUERY_BOUNDS query_warp_kernel(const __grid_constant__ QueryArgs a)
{
    warp_query<WIDE, CAND, FMT, W, ONE, PHASE, F64, false, false>(a);
}

// Double-precision data: the filtered walk of one particle per lane, with its
// own register cap (the FP64 band decision needs more registers than the
// FP32 walk's 32)
#ifndef QBVH_QUERY_F64_MIN_BLOCKS
#define QBVH_QUERY_F64_MIN_BLOCKS 6
#endif
template <int FMT, bool ONE>
__global__ void __launch_bounds__(256, QBVH_QUERY_F64_MIN_BLOCKS) query_f64_kernel(const __grid_constant__ QueryArgs a)
{
    warp_query<false, false, FMT, 1, ONE, 2, true, false, false>(a);
}

// the one-particle-per-lane walk of exact FP32 lists with the packet queue
template <bool WIDE, int FMT, bool ONE>
__global__ void QBVH_QUERY_BOUNDS query_queue_kernel(const __grid_constant__ QueryArgs a)
{
    warp_query<WIDE, false, FMT, 1, ONE, 2, false, false, true>(a);
}

// the walk of one system of one type that also sums the LJ terms of its pairs
template <int FMT>
__global__ void __launch_bounds__(256, QBVH_QUERY_LJ_MIN_BLOCKS) query_warp_lj_kernel(const __grid_constant__ QueryArgs a)
{
    warp_query<false, false, FMT, 1, true, 2, false, true, false>(a);
}

}  // namespace

// SM count of the current device, looked up once per device (the value
// only sizes the sparse-tree blocks: a stale or racing read costs speed, not
// correctness; the table is written once per slot with the same value)
static int sm_count_current()
{
    constexpr int kMaxDev = 64;
    static int sms[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 152;
    }
    int v = __atomic_load_n(&sms[dev], __ATOMIC_RELAXED);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        __atomic_store_n(&sms[dev], v, __ATOMIC_RELAXED);
    }
    return v;
}

// leading blocks for sparse trees: about 8 warps per SM
static int sparse_blocks_for(const QueryArgs &a)
{
    return sm_count_current() * (256 / a.block);
}

// dynamic shared memory of a traversal block: one BundleStage per warp
static size_t stage_bytes(int block, bool stage, bool f64 = false)
{
    // double-precision data: the survivors' Z-order indices after the stages
    return stage ? (size_t)(block / 32) * (sizeof(BundleStage) + (f64 ? kStage * sizeof(int) : 0)) : 0;
}

// Blocks of `kernel` that one SM keeps resident at `block` threads and
// `smem` bytes of dynamic shared memory (at least 1).
static int resident_blocks(const void *kernel, int block, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

// The packet-queue walk: at most as many blocks as stay resident, plus the
// sparse-tree blocks.
template <int FMT, bool WIDE, bool ONE>
static void launch_queue(QueryArgs a, cudaStream_t s, int grid, size_t sm)
{
    const void *k = reinterpret_cast<const void *>(&query_queue_kernel<WIDE, FMT, ONE>);
    const int resident = sm_count_current() * resident_blocks(k, a.block, sm);
    const int g = min(grid, resident) + a.sparse_blocks;
    query_queue_kernel<WIDE, FMT, ONE><<<g, a.block, sm, s>>>(a);
}

template <int FMT, int W, int PHASE>
static void launch_warp_phase(QueryArgs a, cudaStream_t s, int grid)
{
    const int b = a.block;
    a.sparse_blocks = 0;
    a.n_packets = grid * (b / 32);
    if (QBVH_SPARSE_TREES && PHASE == 2 && !a.wide_keys && !a.candidates && a.n_types > 1) {
        a.sparse_blocks = sparse_blocks_for(a);
        grid += a.sparse_blocks;
    }
    const size_t sm = stage_bytes(b, stage_on(W, a.candidates != 0, false));
    if (PHASE == 2 && W == 1 && a.persistent && !a.candidates) {
        if (a.wide_keys) launch_queue<FMT, true, false>(a, s, grid - a.sparse_blocks, sm);
        else if (a.n_types == 1) launch_queue<FMT, false, true>(a, s, grid - a.sparse_blocks, sm);
        else launch_queue<FMT, false, false>(a, s, grid - a.sparse_blocks, sm);
        return;
    }
    if (a.wide_keys) {
        if (a.candidates) query_warp_kernel<true, true, FMT, W, false, PHASE><<<grid, b, sm, s>>>(a);
        else query_warp_kernel<true, false, FMT, W, false, PHASE><<<grid, b, sm, s>>>(a);
    } else if (a.candidates) {
        query_warp_kernel<false, true, FMT, W, false, PHASE><<<grid, b, sm, s>>>(a);
    } else if (a.n_types == 1) {
        query_warp_kernel<false, false, FMT, W, true, PHASE><<<grid, b, sm, s>>>(a);
    } else {
        query_warp_kernel<false, false, FMT, W, false, PHASE><<<grid, b, sm, s>>>(a);
    }
}

template <int FMT, int W>
static void launch_warp(const QueryArgs &a, cudaStream_t s)
{
    const int b = a.block;
    const long long threads = (long long)((a.n + (32 / W) - 1) / (32 / W)) * 32;
    const int grid = (int)((threads + b - 1) / b);
#if QBVH_QUERY_SPLIT_IMAGES
    launch_warp_phase<FMT, W, 0>(a, s, grid);
    launch_warp_phase<FMT, W, 1>(a, s, grid);
#else
    launch_warp_phase<FMT, W, 2>(a, s, grid);
#endif
}

template <int FMT>
static void launch_thread(const QueryArgs &a, cudaStream_t s)
{
    const int b = a.block;
    const int grid = (a.n + b - 1) / b;
    if (a.wide_keys) {
        if (a.candidates) query_thread_kernel<true, true, FMT><<<grid, b, 0, s>>>(a);
        else query_thread_kernel<true, false, FMT><<<grid, b, 0, s>>>(a);
    } else {
        if (a.candidates) query_thread_kernel<false, true, FMT><<<grid, b, 0, s>>>(a);
        else query_thread_kernel<false, false, FMT><<<grid, b, 0, s>>>(a);
    }
}

// Double-precision particle data: the exact list of one system through the
// warp walk with one particle per lane.
template <int FMT>
static void launch_f64(const QueryArgs &a, cudaStream_t s)
{
    const int b = a.block;
    const int grid = (int)(((long long)((a.n + 31) / 32) * 32 + b - 1) / b);
    const size_t sm = stage_bytes(b, stage_on(1, false, true), true);
    if (a.n_types == 1) query_f64_kernel<FMT, true><<<grid, b, sm, s>>>(a);
    else query_f64_kernel<FMT, false><<<grid, b, sm, s>>>(a);
}

int query_lj_blocks(int n, int block)
{
    const long long threads = (long long)((n + 31) / 32) * 32;
    return (int)((threads + block - 1) / block);
}

void launch_query_lj(const QueryArgs &a, cudaStream_t s)
{
    if (a.n == 0) return;
    const int b = a.block;
    const int grid = query_lj_blocks(a.n, b);
    const size_t sm = stage_bytes(b, true);
    if (a.node_fmt == 0) query_warp_lj_kernel<0><<<grid, b, sm, s>>>(a);
    else if (a.node_fmt == 1) query_warp_lj_kernel<1><<<grid, b, sm, s>>>(a);
    else query_warp_lj_kernel<2><<<grid, b, sm, s>>>(a);
}

void launch_query(const QueryArgs &a, cudaStream_t s)
{
    if (a.n == 0) return;
    if (a.f64) {
        if (a.node_fmt == 0) launch_f64<0>(a, s);
        else if (a.node_fmt == 1) launch_f64<1>(a, s);
        else launch_f64<2>(a, s);
        return;
    }
    if (a.traversal == 0) {
        if (a.node_fmt == 0) launch_thread<0>(a, s);
        else if (a.node_fmt == 1) launch_thread<1>(a, s);
        else launch_thread<2>(a, s);
        return;
    }
    const int W = 32 / a.warp_particles;
    if (a.node_fmt == 0) {
        switch (W) {
        case 1: launch_warp<0, 1>(a, s); break;
        case 2: launch_warp<0, 2>(a, s); break;
        case 4: launch_warp<0, 4>(a, s); break;
        case 8: launch_warp<0, 8>(a, s); break;
        case 16: launch_warp<0, 16>(a, s); break;
        default: launch_warp<0, 32>(a, s); break;
        }
    } else if (a.node_fmt == 1) {
        switch (W) {
        case 1: launch_warp<1, 1>(a, s); break;
        case 2: launch_warp<1, 2>(a, s); break;
        case 4: launch_warp<1, 4>(a, s); break;
        case 8: launch_warp<1, 8>(a, s); break;
        case 16: launch_warp<1, 16>(a, s); break;
        default: launch_warp<1, 32>(a, s); break;
        }
    } else {
        switch (W) {
        case 1: launch_warp<2, 1>(a, s); break;
        case 2: launch_warp<2, 2>(a, s); break;
        case 4: launch_warp<2, 4>(a, s); break;
        case 8: launch_warp<2, 8>(a, s); break;
        case 16: launch_warp<2, 16>(a, s); break;
        default: launch_warp<2, 32>(a, s); break;
        }
    }
}

}  // namespace qbvh
