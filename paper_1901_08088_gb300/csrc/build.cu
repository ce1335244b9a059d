// Build of the quantized LBVH (Sec. 2.1, Sec. 2.2, Fig. 3 of the paper).
//
//   prepare  : reset per-tree accumulators and the device status word
//   morton   : Morton binning of every particle (2^10 - 1 bins per axis, 30-bit
//              code, Sec. 2.1), per-tree particle count and root AABB
//   seg_scan : tree start offsets and quantization frames (root AABB split
//              into 2^10 - 1 bins per axis, bin width rounded up, Sec. 2.2)
//   (radix sort of the codes: sort.cu)
//   karras   : binary radix tree of the sorted codes (Karras's construction,
//              cited in Sec. 2.1): N-1 internal nodes with two children each
//   fit      : bottom-up walk from the leaves (Sec. 2.1); each internal node
//              is completed by the second child to arrive
//
// Quantization is done in the fit, in the integer domain: a leaf's bounds are
// snapped outward onto the bin edges (lower bound rounded down, upper bound
// up, IEEE directed rounding, Sec. 3) and an internal node's quantized bounds
// are the per-axis min / max of its children's.  Outward snapping is monotone,
// so the min of snapped children equals the snapped min of the children: this
// is the quantization of the node's FP32 AABB (Sec. 2.2) without ever storing
// the FP32 boxes.
#include <float.h>

#include "qbvh_internal.cuh"

namespace qbvh {

namespace {

constexpr int kBlock = 256;
constexpr int kLocalSegs = 64;
constexpr int kMortonItems = 8;   // particles per thread of the Morton pass

__device__ __forceinline__ int sys_of(const int *off, int n_sys, int i)
{
    // largest k with off[k] <= i
    int lo = 0, hi = n_sys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-tree accumulator layout (8 words): [0] count, [1..3] min bits of x,y,z,
// [4..6] max bits, [7] unused.  Valid positions are >= 0, where the order of
// IEEE floats equals the order of their bit patterns as unsigned integers.
__device__ __forceinline__ unsigned acc_init(int f) { return (f >= 1 && f <= 3) ? 0x7F800000u : 0u; }

// Resets the per-tree accumulators, the status word and the radix-sort scratch
// (histograms, tickets, look-back words) in one grid-stride pass.
__global__ void prepare_kernel(unsigned *acc, int n_seg, DevStatus *status, unsigned *scratch, size_t words)
{
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t t = t0; t < (size_t)n_seg * 8; t += stride) acc[t] = acc_init((int)(t & 7));
    for (size_t t = t0; t < words; t += stride) scratch[t] = 0u;
    if (t0 == 0) {
        status->max_count = 0;
        status->err = 0u;
    }
}

// Double-precision particle data (Sec. 2.2): a coordinate x is bounded by
// the FP32 box [rd(x), ru(x)], rounded down and up, so every FP32 or
// quantized box built over it encloses the exact point.  NaN and negative
// coordinates are read as 0 (the morton pass has flagged the build).
__device__ __forceinline__ void read_pos64(const BuildArgs &a, int idx, float3 &lo, float3 &hi, float3 &mid,
                                           double3 &xyz)
{
    const double4_32a q = a.pos64[idx];
    const double x = (q.x >= 0.0) ? q.x : 0.0;
    const double y = (q.y >= 0.0) ? q.y : 0.0;
    const double z = (q.z >= 0.0) ? q.z : 0.0;
    lo = make_float3(__double2float_rd(x), __double2float_rd(y), __double2float_rd(z));
    hi = make_float3(__double2float_ru(x), __double2float_ru(y), __double2float_ru(z));
    mid = make_float3(__double2float_rn(x), __double2float_rn(y), __double2float_rn(z));
    xyz = make_double3(x, y, z);
}

template <bool WIDE, bool F64>
__global__ void __launch_bounds__(kBlock) morton_kernel(const BuildArgs a, unsigned *acc)
{
    __shared__ unsigned s_acc[kLocalSegs * 8];
    __shared__ unsigned s_hist[8 * 256];
    __shared__ int s_seg0, s_span;
    const int T = a.n_types;        // trees per system
    const int TV = a.type_bound;    // valid types
    const int npass = a.sort_passes;
    for (int t = threadIdx.x; t < npass * 256; t += kBlock) s_hist[t] = 0u;
    if (threadIdx.x == 0) {
        int first = blockIdx.x * kBlock * kMortonItems;
        int last = min(first + kBlock * kMortonItems, a.n) - 1;
        int k0 = a.n_sys > 1 ? sys_of(a.sys_off, a.n_sys, first) : 0;
        int k1 = a.n_sys > 1 ? sys_of(a.sys_off, a.n_sys, last) : 0;
        s_seg0 = k0 * T;
        s_span = (k1 - k0 + 1) * T;
    }
    for (int t = threadIdx.x; t < kLocalSegs * 8; t += kBlock) s_acc[t] = acc_init(t & 7);
    __syncthreads();
    const bool local = s_span <= kLocalSegs;

    // kMortonItems particles per thread, in kBlock-wide strides: the block's
    // histograms and tree accumulators go to global memory once per
    // kBlock * kMortonItems particles
    for (int it = 0; it < kMortonItems; ++it) {
    const int i = (blockIdx.x * kMortonItems + it) * kBlock + threadIdx.x;
    if (i < a.n) {
        // fresh arrival counters and parent links for the fit (a missing link
        // ends a walk instead of sending it to an arbitrary index)
        a.visit[i] = 0;
        a.par_int[i] = -1;
        a.par_leaf[i] = -1;
    }
    unsigned err = 0u;
    int seg = -1;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);   // lower corner of the particle's box
    float3 ph = make_float3(0.f, 0.f, 0.f);        // upper corner
    if (i < a.n) {
        const int k = a.n_sys > 1 ? sys_of(a.sys_off, a.n_sys, i) : 0;
        const SysInfo sy = a.sys[k];
        int type;
        if (F64) {
            const double4_32a q = a.pos64[i];
            const bool type_ok = q.w >= 0.0 && q.w < (double)TV && (double)(int)q.w == q.w;
            if (!type_ok) err |= QBVH_DEVERR_BAD_TYPE;
            if (!(q.x >= 0.0 && q.x < a.L64 && q.y >= 0.0 && q.y < a.L64 && q.z >= 0.0 && q.z < a.L64))
                err |= QBVH_DEVERR_OUT_OF_BOX;
            type = type_ok ? (int)q.w : 0;
            float3 lo, hi, mid;
            double3 xyz;
            read_pos64(a, i, lo, hi, mid, xyz);
            p = make_float4(lo.x, lo.y, lo.z, 0.f);
            ph = hi;
        } else {
            p = __ldg(a.pos + i);
            type = __float_as_int(p.w);
            if (type < 0 || type >= TV) {
                err |= QBVH_DEVERR_BAD_TYPE;
                type = 0;
            }
            if (!(p.x >= 0.f && p.x < sy.L && p.y >= 0.f && p.y < sy.L && p.z >= 0.f && p.z < sy.L)) {
                err |= QBVH_DEVERR_OUT_OF_BOX;
                // keep the accumulators in the non-negative range; the build is
                // reported as failed at the next query
                p.x = fmaxf(p.x, 0.f);
                p.y = fmaxf(p.y, 0.f);
                p.z = fmaxf(p.z, 0.f);
                if (!(p.x == p.x)) p.x = 0.f;
                if (!(p.y == p.y)) p.y = 0.f;
                if (!(p.z == p.z)) p.z = 0.f;
            }
            ph = make_float3(p.x, p.y, p.z);
        }
        const unsigned code = (spread10(bin_of(p.x, sy.mscale)) << 2) |
                              (spread10(bin_of(p.y, sy.mscale)) << 1) |
                              spread10(bin_of(p.z, sy.mscale));
        if (T == 1) type = 0;   // every type in the system's one tree
        seg = k * T + type;
        const unsigned long long key = WIDE ? (((unsigned long long)seg << 30) | code)
                                            : (unsigned long long)(((unsigned)type << 30) | code);
        if (WIDE)
            reinterpret_cast<unsigned long long *>(a.keys)[i] = key;
        else
            reinterpret_cast<unsigned *>(a.keys)[i] = (unsigned)key;
        // digit histograms of the key sort, one per 8-bit pass
        for (int p = 0; p < npass; ++p) atomicAdd(&s_hist[p * 256 + (unsigned)((key >> (8 * p)) & 255u)], 1u);
    }
    if (err) atomicOr(&a.status->err, err);

    // per-tree count and root AABB: warp-aggregate when the warp is uniform
    const unsigned full = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int seg0 = __shfl_sync(full, seg, 0);
    const bool uniform = __all_sync(full, seg == seg0) && seg0 >= 0;
    unsigned v[7];
    v[0] = 1u;
    v[1] = __float_as_uint(p.x);
    v[2] = __float_as_uint(p.y);
    v[3] = __float_as_uint(p.z);
    v[4] = __float_as_uint(ph.x);
    v[5] = __float_as_uint(ph.y);
    v[6] = __float_as_uint(ph.z);
    unsigned *dst_base = nullptr;
    if (uniform) {
        v[0] = __reduce_add_sync(full, 1u);
        for (int f = 1; f <= 3; ++f) v[f] = __reduce_min_sync(full, v[f]);
        for (int f = 4; f <= 6; ++f) v[f] = __reduce_max_sync(full, v[f]);
        if (lane == 0) {
            dst_base = local ? s_acc + (seg0 - s_seg0) * 8 : acc + (size_t)seg0 * 8;
        }
    } else if (seg >= 0) {
        dst_base = local ? s_acc + (seg - s_seg0) * 8 : acc + (size_t)seg * 8;
    }
    if (dst_base) {
        atomicAdd(dst_base, v[0]);
        for (int f = 1; f <= 3; ++f) atomicMin(dst_base + f, v[f]);
        for (int f = 4; f <= 6; ++f) atomicMax(dst_base + f, v[f]);
    }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < npass * 256; t += kBlock)
        if (s_hist[t]) atomicAdd(a.sort_scratch + t, s_hist[t]);   // histograms lead the scratch
    if (local) {
        for (int t = threadIdx.x; t < s_span * 8; t += kBlock) {
            const int f = t & 7;
            const unsigned x = s_acc[t];
            const unsigned cnt = s_acc[t & ~7];
            if (cnt == 0u || f == 7) continue;
            unsigned *g = acc + (size_t)s_seg0 * 8 + t;
            if (f == 0) atomicAdd(g, x);
            else if (f <= 3) atomicMin(g, x);
            else atomicMax(g, x);
        }
    }
}

// One block: exclusive scan of the tree counts, tree records and frames.
__global__ void __launch_bounds__(1024) seg_scan_kernel(const BuildArgs a, const unsigned *acc)
{
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < a.n_seg; base += 1024) {
        const int s = base + tid;
        const int c = s < a.n_seg ? (int)acc[(size_t)s * 8] : 0;
        int x = c;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? s_warp[warp - 1] : 0) + s_carry;
        const int start = incl - c;
        if (s < a.n_seg) {
            SegInfo g;
            g.start = start;
            g.count = c;
            g.sys = s / a.n_types;
            g.type = s % a.n_types;
            g.pad = 0.f;
            float *fr = a.frames + (size_t)s * 8;
            for (int d = 0; d < 3; ++d) {
                float lo = __uint_as_float(acc[(size_t)s * 8 + 1 + d]);
                float hi = __uint_as_float(acc[(size_t)s * 8 + 4 + d]);
                if (c == 0) lo = hi = 0.f;
                // bin width: (R_hi - R_lo) / 1023 rounded up, so 1023 bins cover the root
                float h = __fdiv_ru(__fsub_ru(hi, lo), (float)QBVH_QMAX);
                if (!(h >= FLT_MIN)) h = FLT_MIN;
                // and for the 21-bit node format, 2^21 - 1 bins
                float h21 = __fdiv_ru(__fsub_ru(hi, lo), (float)QBVH_QMAX21);
                if (!(h21 >= FLT_MIN)) h21 = FLT_MIN;
                g.rlo[d] = lo;
                g.rhi[d] = hi;
                g.h[d] = h;
                g.h21[d] = h21;
                fr[d] = lo;
                fr[3 + d] = h;
            }
            fr[6] = 0.f;
            fr[7] = 0.f;
            a.seg[s] = g;
            a.seg_start[s] = start;
            if (s == a.n_seg - 1) a.seg_start[a.n_seg] = incl;
        }
        __syncthreads();
        if (tid == 1023) s_carry = incl;
        __syncthreads();
    }
}

template <bool WIDE>
__device__ __forceinline__ unsigned long long key_at(const void *keys, int k)
{
    if (WIDE) return __ldg(reinterpret_cast<const unsigned long long *>(keys) + k);
    return __ldg(reinterpret_cast<const unsigned *>(keys) + k);
}

template <bool WIDE>
__device__ __forceinline__ int seg_of_key(unsigned long long key, int n_types)
{
    if (WIDE) return (int)(key >> 30);
    return n_types > 1 ? (int)(key >> 30) : 0;
}

// Length of the common prefix of the augmented keys (code, sorted position)
// of leaves i and j inside [a, b]; -1 outside.
template <bool WIDE>
__device__ __forceinline__ int delta(const void *keys, int i, unsigned ci, int j, int a, int b)
{
    if (j < a || j > b) return -1;
    const unsigned cj = (unsigned)key_at<WIDE>(keys, j) & QBVH_QMASK;
    if (ci != cj) return __clz(ci ^ cj);
    return 32 + __clz((unsigned)i ^ (unsigned)j);
}

template <bool WIDE>
__global__ void __launch_bounds__(kBlock) karras_kernel(const BuildArgs a)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= a.n) return;
    const unsigned long long key = key_at<WIDE>(a.keys_sorted, i);
    const int s = seg_of_key<WIDE>(key, a.n_types);
    const SegInfo g = a.seg[s];
    const int lo = g.start, hi = g.start + g.count - 1;
    if (i == hi) {
        if (g.count == 1) a.par_leaf[i] = -1;
        return;   // no internal node at a tree's last leaf
    }
    const unsigned ci = (unsigned)key & QBVH_QMASK;
    const void *K = a.keys_sorted;
    // direction of the range
    const int d = (delta<WIDE>(K, i, ci, i + 1, lo, hi) - delta<WIDE>(K, i, ci, i - 1, lo, hi)) > 0 ? 1 : -1;
    const int dmin = delta<WIDE>(K, i, ci, i - d, lo, hi);
    // upper bound on the range length, then binary search for the other end
    int lmax = 2;
    while (delta<WIDE>(K, i, ci, i + lmax * d, lo, hi) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta<WIDE>(K, i, ci, i + (l + t) * d, lo, hi) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta<WIDE>(K, i, ci, j, lo, hi);
    // binary search for the split position
    int sp = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta<WIDE>(K, i, ci, i + (sp + t) * d, lo, hi) > dnode) sp += t;
    } while (t > 1);
    const int gamma = i + sp * d + min(d, 0);
    const int first = min(i, j), last = max(i, j);
    const int left = (first == gamma) ? ~gamma : gamma;
    const int right = (last == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    a.range[i] = make_int2(first, last);
    a.child[i] = make_int2(left, right);
    if (left >= 0) a.par_int[left] = i; else a.par_leaf[~left] = i;
    if (right >= 0) a.par_int[right] = i; else a.par_leaf[~right] = i;
    if (i == lo) a.par_int[i] = -1;   // node lo of a tree is its root
}

// 21-bit fields, three per 64-bit word (x << 42 | y << 21 | z)
__device__ __forceinline__ unsigned long long pack21(unsigned x, unsigned y, unsigned z)
{
    return ((unsigned long long)x << 42) | ((unsigned long long)y << 21) | z;
}

__device__ __forceinline__ unsigned field21(unsigned long long w, int shift)
{
    return (unsigned)(w >> shift) & (unsigned)QBVH_QMAX21;
}

__device__ __forceinline__ unsigned long long qmin21(unsigned long long a, unsigned long long b)
{
    return pack21(min(field21(a, 42), field21(b, 42)), min(field21(a, 21), field21(b, 21)),
                  min(field21(a, 0), field21(b, 0)));
}

__device__ __forceinline__ unsigned long long qmax21(unsigned long long a, unsigned long long b)
{
    return pack21(max(field21(a, 42), field21(b, 42)), max(field21(a, 21), field21(b, 21)),
                  max(field21(a, 0), field21(b, 0)));
}

// the 21-bit box {lo64, hi64} of an FP32 box against tree g
__device__ __forceinline__ ulonglong2 quantize21(const float3 &lo, const float3 &hi, const SegInfo &g)
{
    ulonglong2 q;
    q.x = pack21(q_down21(lo.x, g.rlo[0], g.h21[0]), q_down21(lo.y, g.rlo[1], g.h21[1]),
                 q_down21(lo.z, g.rlo[2], g.h21[2]));
    q.y = pack21(q_up21(hi.x, g.rlo[0], g.h21[0]), q_up21(hi.y, g.rlo[1], g.h21[1]),
                 q_up21(hi.z, g.rlo[2], g.h21[2]));
    return q;
}

__device__ __forceinline__ float clear_sign(float x) { return __int_as_float(__float_as_int(x) & 0x7FFFFFFF); }

// atomic increment with acquire-release semantics at device scope; returns the old value
__device__ __forceinline__ int arrive_acq_rel(int *p)
{
    int old;
    asm volatile("atom.add.acq_rel.gpu.s32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

// Bottom-up fit, in two parts.
//
// Block part.  A block owns leaves [b0, b1] and the internal nodes with the
// same indices.  An internal node whose leaf range lies inside [b0, b1] is
// "local": its Karras index (an end of its range) is then in [b0, b1] too,
// and so are its children.  Every thread loads the words of its own leaf and
// node (coalesced), then the block settles its local nodes level by level:
// in each round a node whose children are done is computed from the
// children's boxes in shared memory; a barrier separates the rounds.
//
// Global part.  Nodes whose range crosses a block boundary are completed by
// climbing: the thread of every local subtree root (and of every leaf whose
// parent crosses) arrives at the parent through a device-scope
// acquire-release counter; the second arrival computes the parent from its
// children's words in global memory (every node and leaf is written there)
// and climbs on.
template <bool WIDE, bool F32>
__device__ __forceinline__ void fit_compute(const BuildArgs &a, int node, const int2 r, const int2 c, int rope,
                                            uint2 bl, uint2 br, const float4 &lo_a, const float4 &hi_a,
                                            const float4 &lo_b, const float4 &hi_b, uint2 *q_out, float4 *lo_out,
                                            float4 *hi_out, const ulonglong2 &b21l, const ulonglong2 &b21r,
                                            ulonglong2 *q21_out)
{
    const unsigned qlo = qmin3(bl.x, br.x);
    const unsigned qhi = qmax3(bl.y, br.y);
    const int count = r.y - r.x + 1;
    const int bundle = (a.bundle_k >= 2 && count <= a.bundle_k) ? 1 : 0;
    int4 w;
    w.x = (int)(qlo | ((unsigned)bundle << 31));
    w.y = (int)qhi;
    w.z = bundle ? r.x : c.x;
    w.w = rope;
    __stcg(a.nodes + node, w);
    if (q_out) *q_out = make_uint2(qlo, qhi);
    if (a.nodes21) {
        // 21-bit bounds: per-field min / max of the children's (Sec. 2.2 at a
        // wider bit width), the bundle flag in bit 63
        const unsigned long long lo21 = qmin21(b21l.x, b21r.x), hi21 = qmax21(b21l.y, b21r.y);
        if (q21_out) *q21_out = make_ulonglong2(lo21, hi21);
        const unsigned long long lw = lo21 | ((unsigned long long)bundle << 63);
        __stcg(a.nodes21 + 2 * (size_t)node,
               make_int4((int)(unsigned)lw, (int)(unsigned)(lw >> 32), (int)(unsigned)hi21, (int)(unsigned)(hi21 >> 32)));
        __stcg(a.nodes21 + 2 * (size_t)node + 1, make_int4(w.z, w.w, 0, 0));
    }
    if (F32) {
        // exact FP32 AABB: min / max of the children's boxes (Fig. 3a layout)
        const float4 lo = make_float4(fminf(lo_a.x, lo_b.x), fminf(lo_a.y, lo_b.y), fminf(lo_a.z, lo_b.z), 0.f);
        const float4 hb = make_float4(fmaxf(hi_a.x, hi_b.x), fmaxf(hi_a.y, hi_b.y), fmaxf(hi_a.z, hi_b.z), 0.f);
        if (lo_out) {
            *lo_out = lo;
            *hi_out = hb;
        }
        float lx = lo.x;
        if (bundle) lx = __int_as_float(__float_as_int(lx) | 0x80000000);
        __stcg(a.nodes32 + 2 * (size_t)node, make_float4(lx, lo.y, lo.z, __int_as_float(w.z)));
        __stcg(a.nodes32 + 2 * (size_t)node + 1, make_float4(hb.x, hb.y, hb.z, __int_as_float(w.w)));
    }
}

// FP32 box of leaf k as written in global memory: the point itself, or for
// double-precision data the outward-rounded box of the FP64 point.
template <bool F64>
__device__ __forceinline__ void leaf_box(const BuildArgs &a, int k, float4 &lo, float4 &hi)
{
    if (F64) {
        const double2 *d2 = reinterpret_cast<const double2 *>(a.leaves64 + k);
        const double2 xy = __ldcg(d2), zw = __ldcg(d2 + 1);
        lo = make_float4(__double2float_rd(xy.x), __double2float_rd(xy.y), __double2float_rd(zw.x), 0.f);
        hi = make_float4(__double2float_ru(xy.x), __double2float_ru(xy.y), __double2float_ru(zw.x), 0.f);
    } else {
        lo = hi = __ldcg(a.leaves + k);
    }
}

// 21-bit box of internal node k as written in global memory
__device__ __forceinline__ ulonglong2 node21_box(const BuildArgs &a, int k)
{
    const int4 w = __ldcg(a.nodes21 + 2 * (size_t)k);
    const unsigned long long lo = ((unsigned long long)(unsigned)w.y << 32) | (unsigned)w.x;
    const unsigned long long hi = ((unsigned long long)(unsigned)w.w << 32) | (unsigned)w.z;
    return make_ulonglong2(lo & QBVH_QMASK21, hi);
}

// 21-bit box of leaf k (recomputed from the leaf's FP32 box)
template <bool F64>
__device__ __forceinline__ ulonglong2 leaf21_box(const BuildArgs &a, int k, const SegInfo &g)
{
    float4 lo, hi;
    leaf_box<F64>(a, k, lo, hi);
    return quantize21(make_float3(lo.x, lo.y, lo.z), make_float3(hi.x, hi.y, hi.z), g);
}

// Climb from `node` while this thread is the second arrival (global part).
template <bool WIDE, bool F32, bool F64>
__device__ __forceinline__ void fit_climb(const BuildArgs &a, int node, int hi, int sg)
{
    // a radix tree over 62-bit keys (30-bit code + 32-bit position) is at most
    // 63 levels deep; a longer walk means a broken parent link
    for (int depth = 0; node >= 0; ++depth) {
        if (node >= a.n || depth > 64) {
            atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            return;
        }
        // the node's own words do not depend on the arrival: load them first
        const int2 r = a.range[node];
        const int2 c = a.child[node];
        const int up = a.par_int[node];
        const int rope = rope_after(a.range, r.y, hi);
        // release publishes this child's bounds, acquire makes the sibling's
        // bounds visible to the thread that continues upward
        if (arrive_acq_rel(a.visit + node) == 0) return;   // sibling not done yet
        if (c.x >= a.n || ~c.x >= a.n || c.y >= a.n || ~c.y >= a.n) {
            atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            return;
        }
        uint2 bl, br;
        float4 lo_a, hi_a, lo_b, hi_b;
        if (c.x >= 0) {
            int4 w = __ldcg(a.nodes + c.x);
            bl = make_uint2((unsigned)w.x & QBVH_QMASK, (unsigned)w.y);
        } else {
            bl = __ldcg(a.leaf_q + ~c.x);
        }
        if (c.y >= 0) {
            int4 w = __ldcg(a.nodes + c.y);
            br = make_uint2((unsigned)w.x & QBVH_QMASK, (unsigned)w.y);
        } else {
            br = __ldcg(a.leaf_q + ~c.y);
        }
        if (F32) {
            if (c.x >= 0) {
                lo_a = __ldcg(a.nodes32 + 2 * (size_t)c.x);
                hi_a = __ldcg(a.nodes32 + 2 * (size_t)c.x + 1);
                lo_a.x = clear_sign(lo_a.x);
            } else {
                leaf_box<F64>(a, ~c.x, lo_a, hi_a);
            }
            if (c.y >= 0) {
                lo_b = __ldcg(a.nodes32 + 2 * (size_t)c.y);
                hi_b = __ldcg(a.nodes32 + 2 * (size_t)c.y + 1);
                lo_b.x = clear_sign(lo_b.x);
            } else {
                leaf_box<F64>(a, ~c.y, lo_b, hi_b);
            }
        }
        ulonglong2 b21l = make_ulonglong2(0ull, 0ull), b21r = b21l;
        if (a.nodes21) {
            const SegInfo &g = a.seg[sg];
            b21l = c.x >= 0 ? node21_box(a, c.x) : leaf21_box<F64>(a, ~c.x, g);
            b21r = c.y >= 0 ? node21_box(a, c.y) : leaf21_box<F64>(a, ~c.y, g);
        }
        fit_compute<WIDE, F32>(a, node, r, c, rope, bl, br, lo_a, hi_a, lo_b, hi_b, nullptr, nullptr, nullptr, b21l,
                               b21r, nullptr);
        node = up;
    }
}

// Resident blocks of the fit per SM (register cap).  The climb keeps blocks
// alive, so more of them hide more of its latency: 8 blocks of 256 (32
// registers, a few spilled) measured build 0.359 -> 0.348 ms at N = 2M
// against 5 (48 registers, no spills).
#ifndef QBVH_FIT_MIN_BLOCKS
#define QBVH_FIT_MIN_BLOCKS 8
#endif
template <bool WIDE, bool F32, bool F64, bool Q21>
__global__ void __launch_bounds__(kBlock, Q21 ? 4 : QBVH_FIT_MIN_BLOCKS) fit_kernel(const BuildArgs a)
{
    __shared__ ulonglong2 s_q21[Q21 ? kBlock : 1];  // 21-bit box of internal node b0 + t
    __shared__ ulonglong2 s_lq21[Q21 ? kBlock : 1]; // 21-bit box of leaf b0 + t
    __shared__ int s_done[kBlock];                  // local internal node b0 + t settled
    __shared__ uint2 s_q[kBlock];                   // quantized box of internal node b0 + t
    __shared__ uint2 s_lq[kBlock];                  // quantized box of leaf b0 + t
    __shared__ float4 s_lo[F32 ? kBlock : 1];       // FP32 box of internal node b0 + t
    __shared__ float4 s_hi[F32 ? kBlock : 1];
    __shared__ float4 s_leaf[F32 ? kBlock : 1];     // FP32 box of leaf b0 + t: lower corner
    __shared__ float4 s_leafhi[F32 && F64 ? kBlock : 1];   // upper corner (double-precision data)
    const int t = threadIdx.x;
    const int b0 = blockIdx.x * kBlock;
    const int b1 = min(b0 + kBlock, a.n) - 1;
    const int k = b0 + t;
    const bool live = k < a.n;
    s_done[t] = 0;

    // ---- leaf k and the words of internal node k --------------------------
    int hi = 0, leaf_up = -1, sg = 0;
    bool node_valid = false;
    int2 r = make_int2(0, -1), c = make_int2(0, 0);
    int up = -1, rope = QBVH_END;
    if (live) {
        const unsigned long long key = key_at<WIDE>(a.keys_sorted, k);
        sg = seg_of_key<WIDE>(key, a.n_types);
        const SegInfo g = a.seg[sg];
        hi = g.start + g.count - 1;
        int orig = __ldg(a.order + k);
        if ((unsigned)orig >= (unsigned)a.n) {
            atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            orig = 0;
        }
        // the leaf's box: the FP32 point, or for double-precision data the
        // outward-rounded box [rd(x), ru(x)] with the nearest FP32 point as
        // the leaf word the traversal tests first
        float3 blo, bhi, mid;
        if (F64) {
            double3 x64;
            read_pos64(a, orig, blo, bhi, mid, x64);
            double4_32a w64;
            w64.x = x64.x;
            w64.y = x64.y;
            w64.z = x64.z;
            w64.w = 0.0;
            a.leaves64[k] = w64;
        } else {
            const float4 p = __ldg(a.pos + orig);
            blo = bhi = mid = make_float3(p.x, p.y, p.z);
        }
        const int leaf_rope = rope_after(a.range, k, hi);
        const unsigned tag = (unsigned)orig | ((leaf_rope >= 0 ? 1u : 0u) << 31);
        const float4 leaf = make_float4(mid.x, mid.y, mid.z, __uint_as_float(tag));
        a.leaves[k] = leaf;
        uint2 q;
        q.x = pack3(q_down(blo.x, g.rlo[0], g.h[0]), q_down(blo.y, g.rlo[1], g.h[1]),
                    q_down(blo.z, g.rlo[2], g.h[2]));
        q.y = pack3(q_up(bhi.x, g.rlo[0], g.h[0]), q_up(bhi.y, g.rlo[1], g.h[1]), q_up(bhi.z, g.rlo[2], g.h[2]));
        a.leaf_q[k] = q;
        s_lq[t] = q;
        if (Q21) s_lq21[t] = quantize21(blo, bhi, g);
        if (F32) {
            s_leaf[t] = F64 ? make_float4(blo.x, blo.y, blo.z, 0.f) : leaf;
            if (F64) s_leafhi[t] = make_float4(bhi.x, bhi.y, bhi.z, 0.f);
        }
        leaf_up = a.par_leaf[k];
        // internal node k exists for every leaf index of a tree but its last
        node_valid = k <= hi - 1;
        if (node_valid) {
            r = a.range[k];
            c = a.child[k];
            up = a.par_int[k];
            rope = rope_after(a.range, r.y, hi);
        }
    }
    const bool local = node_valid && r.x >= b0 && r.y <= b1;
    if (local && (k < r.x || k > r.y)) atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
    bool pending = local && k >= r.x && k <= r.y;
    __syncthreads();

    // ---- block part: rounds over the local nodes -----------------------------
    for (int round = 0; round < kBlock; ++round) {
        bool done_now = false;
        if (pending) {
            const int ia = (c.x >= 0 ? c.x : ~c.x) - b0, ib = (c.y >= 0 ? c.y : ~c.y) - b0;
            if ((unsigned)ia >= (unsigned)kBlock || (unsigned)ib >= (unsigned)kBlock) {
                atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                pending = false;
            } else if ((c.x < 0 || s_done[ia]) && (c.y < 0 || s_done[ib])) {
                const uint2 bl = c.x >= 0 ? s_q[ia] : s_lq[ia];
                const uint2 br = c.y >= 0 ? s_q[ib] : s_lq[ib];
                float4 lo_a, hi_a, lo_b, hi_b;
                if (F32) {
                    lo_a = c.x >= 0 ? s_lo[ia] : s_leaf[ia];
                    hi_a = c.x >= 0 ? s_hi[ia] : (F64 ? s_leafhi[ia] : s_leaf[ia]);
                    lo_b = c.y >= 0 ? s_lo[ib] : s_leaf[ib];
                    hi_b = c.y >= 0 ? s_hi[ib] : (F64 ? s_leafhi[ib] : s_leaf[ib]);
                }
                ulonglong2 b21l = make_ulonglong2(0ull, 0ull), b21r = b21l;
                if (Q21) {
                    b21l = c.x >= 0 ? s_q21[ia] : s_lq21[ia];
                    b21r = c.y >= 0 ? s_q21[ib] : s_lq21[ib];
                }
                fit_compute<WIDE, F32>(a, k, r, c, rope, bl, br, lo_a, hi_a, lo_b, hi_b, &s_q[t],
                                       F32 ? &s_lo[t] : nullptr, F32 ? &s_hi[t] : nullptr, b21l, b21r,
                                       Q21 ? &s_q21[t] : nullptr);
                done_now = true;
                pending = false;
            }
        }
        __syncthreads();                 // this round's boxes are written
        if (done_now) s_done[t] = 1;
        if (!__syncthreads_or(pending)) break;   // and its flags visible
    }
    if (pending) atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);   // a cycle: broken links

    // ---- global part: climb from the roots of the local subtrees -------------
    // (a leaf or local node whose parent is not local; the parent's range
    // decides, and a parent's range contains its child's)
    if (live && leaf_up >= 0 && leaf_up < a.n) {
        const int2 pr = a.range[leaf_up];
        if (!(pr.x >= b0 && pr.y <= b1)) fit_climb<WIDE, F32, F64>(a, leaf_up, hi, sg);
    } else if (live && leaf_up >= a.n) {
        atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
    }
    if (local && up >= 0 && up < a.n) {
        const int2 pr = a.range[up];
        if (!(pr.x >= b0 && pr.y <= b1)) fit_climb<WIDE, F32, F64>(a, up, hi, sg);
    } else if (local && up >= a.n) {
        atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
    }
}

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

}  // namespace

void launch_build_prepare(const BuildArgs &a, cudaStream_t s)
{
    const size_t work = (size_t)a.n_seg * 8 > a.sort_scratch_words ? (size_t)a.n_seg * 8 : a.sort_scratch_words;
    int blocks = (int)((work + kBlock - 1) / kBlock);
    blocks = blocks < 1 ? 1 : (blocks > 1216 ? 1216 : blocks);
    prepare_kernel<<<blocks, kBlock, 0, s>>>(a.seg_rootbits, a.n_seg, a.status, a.sort_scratch,
                                             a.sort_scratch_words);
}

void launch_morton(const BuildArgs &a, cudaStream_t s)
{
    if (a.n == 0) return;
    if (a.wide_keys)
        morton_kernel<true, false><<<blocks_for(a.n, kBlock * kMortonItems), kBlock, 0, s>>>(a, a.seg_rootbits);
    else if (a.pos64)
        morton_kernel<false, true><<<blocks_for(a.n, kBlock * kMortonItems), kBlock, 0, s>>>(a, a.seg_rootbits);
    else
        morton_kernel<false, false><<<blocks_for(a.n, kBlock * kMortonItems), kBlock, 0, s>>>(a, a.seg_rootbits);
}

void launch_seg_scan(const BuildArgs &a, cudaStream_t s)
{
    seg_scan_kernel<<<1, 1024, 0, s>>>(a, a.seg_rootbits);
}

void launch_karras(const BuildArgs &a, cudaStream_t s)
{
    if (a.n == 0) return;
    if (a.wide_keys)
        karras_kernel<true><<<blocks_for(a.n, kBlock), kBlock, 0, s>>>(a);
    else
        karras_kernel<false><<<blocks_for(a.n, kBlock), kBlock, 0, s>>>(a);
}

void launch_fit(const BuildArgs &a, cudaStream_t s)
{
    if (a.n == 0) return;
    const int g = blocks_for(a.n, kBlock);
    if (a.wide_keys) {
        if (a.nodes32) fit_kernel<true, true, false, false><<<g, kBlock, 0, s>>>(a);
        else if (a.nodes21) fit_kernel<true, false, false, true><<<g, kBlock, 0, s>>>(a);
        else fit_kernel<true, false, false, false><<<g, kBlock, 0, s>>>(a);
    } else if (a.pos64) {
        if (a.nodes32) fit_kernel<false, true, true, false><<<g, kBlock, 0, s>>>(a);
        else if (a.nodes21) fit_kernel<false, false, true, true><<<g, kBlock, 0, s>>>(a);
        else fit_kernel<false, false, true, false><<<g, kBlock, 0, s>>>(a);
    } else {
        if (a.nodes32) fit_kernel<false, true, false, false><<<g, kBlock, 0, s>>>(a);
        else if (a.nodes21) fit_kernel<false, false, false, true><<<g, kBlock, 0, s>>>(a);
        else fit_kernel<false, false, false, false><<<g, kBlock, 0, s>>>(a);
    }
}

}  // namespace qbvh
