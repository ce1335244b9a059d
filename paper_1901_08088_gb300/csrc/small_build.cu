// One-block build of a small system (Sec. 2.1, Sec. 2.2, Fig. 3 of the paper).
//
// For one periodic system of at most kSmallUse particles (FP32 data, at most
// four trees, 10-bit or FP32 nodes) the whole build runs in a single block of
// 1024 threads: Morton binning and validation, the per-tree count and root
// box, a stable LSD radix sort of the keys in shared memory, Karras's
// hierarchy and the bottom-up fit by climbing from the leaves.  It writes the same words as the
// multi-kernel build (build.cu + sort.cu): sorted keys and order, tree
// records and frames, 10-bit nodes, FP32 nodes, leaves and leaf boxes.  The
// multi-kernel build is nine latency-bound launches; one launch keeps the
// whole tree in one SM's shared memory.
#include <float.h>

#include "qbvh_internal.cuh"

namespace qbvh {

namespace {

constexpr int kSB = 1024;                    // threads of the block
constexpr int kSmallMax = 4096;              // largest system
constexpr int kItems = kSmallMax / kSB;      // keys per thread
constexpr int kWarps = kSB / 32;
constexpr int kMaxTrees = 4;
constexpr int kMaxDepth = 64;                // a radix tree over 30 + 12 key bits is at most 43 deep

// dynamic shared memory: the sort's two key / value buffers and per-warp
// digit histograms (96 KB; the second buffers and the histograms later hold
// the node ranges and children), then the 10-bit boxes of internal nodes and
// leaves, the parents of internal nodes and leaves and the fit's arrival
// counters (112 KB)
constexpr size_t kSortBytes = 4 * kSmallMax * 4 + kWarps * 256 * 4;
constexpr size_t kFitBytes = 2 * kSmallMax * sizeof(uint2) + 3 * kSmallMax * sizeof(int);
constexpr size_t kSmemBytes = kSortBytes + kFitBytes;

__device__ __forceinline__ unsigned lane_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Length of the common prefix of the augmented keys (code, sorted position)
// of leaves i and j inside [lo, hi]; -1 outside (Karras's delta).
__device__ __forceinline__ int delta_s(const unsigned *keys, int i, unsigned ci, int j, int lo, int hi)
{
    if (j < lo || j > hi) return -1;
    const unsigned cj = keys[j] & QBVH_QMASK;
    if (ci != cj) return __clz(ci ^ cj);
    return 32 + __clz((unsigned)i ^ (unsigned)j);
}

template <bool F32>
__global__ void __launch_bounds__(kSB, 1) small_build_kernel(const BuildArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned *kA = reinterpret_cast<unsigned *>(smem);
    int *vA = reinterpret_cast<int *>(kA + kSmallMax);
    unsigned *kB = reinterpret_cast<unsigned *>(vA + kSmallMax);
    int *vB = reinterpret_cast<int *>(kB + kSmallMax);
    unsigned *hist = reinterpret_cast<unsigned *>(vB + kSmallMax);   // [kWarps][256]
    int2 *s_range = reinterpret_cast<int2 *>(kB);                   // after the sort
    int2 *s_child = reinterpret_cast<int2 *>(hist);                 // after the sort
    uint2 *s_q = reinterpret_cast<uint2 *>(smem + kSortBytes);      // internal node k
    uint2 *s_lq = s_q + kSmallMax;                                  // leaf k
    int *s_par_int = reinterpret_cast<int *>(s_lq + kSmallMax);     // parent of internal node k
    int *s_par_leaf = s_par_int + kSmallMax;                        // parent of leaf k
    int *s_visit = s_par_leaf + kSmallMax;                          // arrivals at internal node k
    __shared__ unsigned s_acc[kMaxTrees * 8];   // count, min bits xyz, max bits xyz
    __shared__ SegInfo s_seg[kMaxTrees];
    __shared__ unsigned s_tot[256], s_dstart[256], s_wsum[8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = a.n, T = a.n_types, TV = a.type_bound;
    const SysInfo sy = a.sys[0];
    if (tid < kMaxTrees * 8) s_acc[tid] = ((tid & 7) >= 1 && (tid & 7) <= 3) ? 0x7F800000u : 0u;
    if (tid == 0) {
        a.status->max_count = 0;
        a.status->err = 0u;
    }
    __syncthreads();

    // ---- keys, validation, per-tree count and root box -------------------
    // item `it` of lane l in warp w is key w * 32 kItems + it * 32 + l: each
    // warp owns a contiguous run, the order the sort's ranking keeps
    unsigned err = 0u;
    // per-tree count and box of this thread's keys, then of the warp's
    unsigned acc[kMaxTrees][7];
#pragma unroll
    for (int t = 0; t < kMaxTrees; ++t) {
        acc[t][0] = 0u;
        acc[t][1] = acc[t][2] = acc[t][3] = 0xFFFFFFFFu;
        acc[t][4] = acc[t][5] = acc[t][6] = 0u;
    }
    float4 pin[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int i = warp * 32 * kItems + it * 32 + lane;
        pin[it] = i < n ? __ldg(a.pos + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int i = warp * 32 * kItems + it * 32 + lane;
        unsigned key = 0xFFFFFFFFu;   // past n: ranks last
        if (i < n) {
            float4 p = pin[it];
            int type = __float_as_int(p.w);
            if (type < 0 || type >= TV) {
                err |= QBVH_DEVERR_BAD_TYPE;
                type = 0;
            }
            if (!(p.x >= 0.f && p.x < sy.L && p.y >= 0.f && p.y < sy.L && p.z >= 0.f && p.z < sy.L)) {
                err |= QBVH_DEVERR_OUT_OF_BOX;
                p.x = fmaxf(p.x, 0.f);
                p.y = fmaxf(p.y, 0.f);
                p.z = fmaxf(p.z, 0.f);
                if (!(p.x == p.x)) p.x = 0.f;
                if (!(p.y == p.y)) p.y = 0.f;
                if (!(p.z == p.z)) p.z = 0.f;
            }
            const unsigned code = (spread10(bin_of(p.x, sy.mscale)) << 2) | (spread10(bin_of(p.y, sy.mscale)) << 1) |
                                  spread10(bin_of(p.z, sy.mscale));
            if (T == 1) type = 0;   // every type in the system's one tree
            key = T > 1 ? (((unsigned)type << 30) | code) : code;
#pragma unroll
            for (int t = 0; t < kMaxTrees; ++t) {
                if (t != type) continue;
                acc[t][0] += 1u;
                acc[t][1] = min(acc[t][1], __float_as_uint(p.x));
                acc[t][2] = min(acc[t][2], __float_as_uint(p.y));
                acc[t][3] = min(acc[t][3], __float_as_uint(p.z));
                acc[t][4] = max(acc[t][4], __float_as_uint(p.x));
                acc[t][5] = max(acc[t][5], __float_as_uint(p.y));
                acc[t][6] = max(acc[t][6], __float_as_uint(p.z));
            }
        }
        kA[i] = key;
        vA[i] = i;
    }
#pragma unroll
    for (int t = 0; t < kMaxTrees; ++t) {
        if (t >= T) break;
        const unsigned cnt = __reduce_add_sync(0xFFFFFFFFu, acc[t][0]);
        if (cnt == 0u) continue;
        unsigned v[7];
        v[0] = cnt;
#pragma unroll
        for (int f = 1; f <= 3; ++f) v[f] = __reduce_min_sync(0xFFFFFFFFu, acc[t][f]);
#pragma unroll
        for (int f = 4; f <= 6; ++f) v[f] = __reduce_max_sync(0xFFFFFFFFu, acc[t][f]);
        if (lane == 0) {
            unsigned *g = s_acc + 8 * t;
            atomicAdd(g, v[0]);
#pragma unroll
            for (int f = 1; f <= 3; ++f) atomicMin(g + f, v[f]);
#pragma unroll
            for (int f = 4; f <= 6; ++f) atomicMax(g + f, v[f]);
        }
    }
    err = __reduce_or_sync(0xFFFFFFFFu, err);
    if (lane == 0 && err) atomicOr(&a.status->err, err);
    __syncthreads();

    // ---- tree records and quantization frames (as seg_scan_kernel) ---------
    if (tid < T) {
        int start = 0;
        for (int t = 0; t < tid; ++t) start += (int)s_acc[8 * t];
        const int c = (int)s_acc[8 * tid];
        SegInfo g;
        g.start = start;
        g.count = c;
        g.sys = 0;
        g.type = tid;
        g.pad = 0.f;
        float *fr = a.frames + (size_t)tid * 8;
        for (int d = 0; d < 3; ++d) {
            float lo = __uint_as_float(s_acc[8 * tid + 1 + d]);
            float hi = __uint_as_float(s_acc[8 * tid + 4 + d]);
            if (c == 0) lo = hi = 0.f;
            float h = __fdiv_ru(__fsub_ru(hi, lo), (float)QBVH_QMAX);
            if (!(h >= FLT_MIN)) h = FLT_MIN;
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
        s_seg[tid] = g;
        a.seg[tid] = g;
        a.seg_start[tid] = start;
        if (tid == T - 1) a.seg_start[T] = start + c;
    }

    // ---- stable LSD radix sort of (key, input index), 8-bit digits ---------
    // (each warp ranks its run row by row, lanes in order; runs keep the warp
    // order, so equal digits keep their order: the sort is stable, and with
    // the input index as the value equal codes end in input order)
    unsigned *src_k = kA, *dst_k = kB;
    int *src_v = vA, *dst_v = vB;
    const unsigned lt = lane_lt();
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        for (int t = tid; t < kWarps * 256; t += kSB) hist[t] = 0u;
        __syncthreads();
        unsigned key[kItems], rank[kItems];
        int val[kItems];
        unsigned *wh = hist + warp * 256;
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const int idx = warp * 32 * kItems + it * 32 + lane;
            key[it] = src_k[idx];
            val[it] = src_v[idx];
            const unsigned d = (key[it] >> shift) & 255u;
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
            const unsigned prev = wh[d];
            __syncwarp();
            const unsigned r = __popc(peers & lt);
            if (r == 0) wh[d] = prev + __popc(peers);
            __syncwarp();
            rank[it] = prev + r;
        }
        __syncthreads();
        // per digit: the warps' offsets, then the digits' starts
        if (tid < 256) {
            unsigned cnt = 0u;
            for (int w = 0; w < kWarps; ++w) {
                const unsigned c = hist[w * 256 + tid];
                hist[w * 256 + tid] = cnt;
                cnt += c;
            }
            s_tot[tid] = cnt;
            unsigned x = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wsum[warp] = x;
            s_dstart[tid] = x - cnt;   // exclusive within the warp
        }
        __syncthreads();
        if (tid < 256) {
            unsigned before = 0u;
            for (int w = 0; w < warp; ++w) before += s_wsum[w];
            s_dstart[tid] += before;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const unsigned d = (key[it] >> shift) & 255u;
            const unsigned pos = s_dstart[d] + wh[d] + rank[it];
            dst_k[pos] = key[it];
            dst_v[pos] = val[it];
        }
        __syncthreads();
        unsigned *tk = src_k;
        src_k = dst_k;
        dst_k = tk;
        int *tv = src_v;
        src_v = dst_v;
        dst_v = tv;
    }
    // four passes: the result is back in kA / vA
    unsigned *out_keys = const_cast<unsigned *>(reinterpret_cast<const unsigned *>(a.keys_sorted));
    int *out_order = const_cast<int *>(a.order);
    for (int k = tid; k < n; k += kSB) {
        out_keys[k] = kA[k];
        out_order[k] = vA[k];
    }

    // ---- Karras hierarchy: internal node i of the tree holding leaf i ------
    for (int i = tid; i < kSmallMax; i += kSB) {
        s_range[i] = make_int2(0, -1);
        s_child[i] = make_int2(0, 0);
        s_par_int[i] = -1;
        s_par_leaf[i] = -1;
        s_visit[i] = 0;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kSB) {
        const unsigned key = kA[i];
        const SegInfo &g = s_seg[T > 1 ? (int)(key >> 30) : 0];
        const int lo = g.start, hi = g.start + g.count - 1;
        if (i >= hi) continue;   // no internal node at a tree's last leaf
        const unsigned ci = key & QBVH_QMASK;
        const int d = (delta_s(kA, i, ci, i + 1, lo, hi) - delta_s(kA, i, ci, i - 1, lo, hi)) > 0 ? 1 : -1;
        const int dmin = delta_s(kA, i, ci, i - d, lo, hi);
        int lmax = 2;
        while (delta_s(kA, i, ci, i + lmax * d, lo, hi) > dmin) lmax <<= 1;
        int l = 0;
        for (int t = lmax >> 1; t >= 1; t >>= 1)
            if (delta_s(kA, i, ci, i + (l + t) * d, lo, hi) > dmin) l += t;
        const int j = i + l * d;
        const int dnode = delta_s(kA, i, ci, j, lo, hi);
        int sp = 0, t = l;
        do {
            t = (t + 1) >> 1;
            if (delta_s(kA, i, ci, i + (sp + t) * d, lo, hi) > dnode) sp += t;
        } while (t > 1);
        const int gamma = i + sp * d + min(d, 0);
        const int first = min(i, j), last = max(i, j);
        const int left = (first == gamma) ? ~gamma : gamma, right = (last == gamma + 1) ? ~(gamma + 1) : gamma + 1;
        s_range[i] = make_int2(first, last);
        s_child[i] = make_int2(left, right);
        if (left >= 0) s_par_int[left] = i; else s_par_leaf[~left] = i;
        if (right >= 0) s_par_int[right] = i; else s_par_leaf[~right] = i;
    }
    __syncthreads();

    // ---- leaves: words, 10-bit boxes ----------------------------------------
    {
        float4 pl[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const int k = tid + it * kSB;
            pl[it] = k < n ? __ldg(a.pos + vA[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const int k = tid + it * kSB;
            if (k >= n) continue;
            const unsigned key = kA[k];
            const SegInfo &g = s_seg[T > 1 ? (int)(key >> 30) : 0];
            const int hi = g.start + g.count - 1;
            const float4 p = pl[it];
            const int leaf_rope = rope_after(s_range, k, hi);
            const unsigned tag = (unsigned)vA[k] | ((leaf_rope >= 0 ? 1u : 0u) << 31);
            a.leaves[k] = make_float4(p.x, p.y, p.z, __uint_as_float(tag));
            uint2 q;
            q.x = pack3(q_down(p.x, g.rlo[0], g.h[0]), q_down(p.y, g.rlo[1], g.h[1]), q_down(p.z, g.rlo[2], g.h[2]));
            q.y = pack3(q_up(p.x, g.rlo[0], g.h[0]), q_up(p.y, g.rlo[1], g.h[1]), q_up(p.z, g.rlo[2], g.h[2]));
            a.leaf_q[k] = q;
            s_lq[k] = q;
        }
    }
    __syncthreads();

    // ---- bottom-up fit: every leaf's thread climbs; at each internal node the
    // first child to arrive stops and the second computes the node (Sec. 2.1),
    // the arrival counted in shared memory; the fences order each child's
    // box before its arrival and the sibling's box after it
    for (int k = tid; k < n; k += kSB) {
        const unsigned key = kA[k];
        const SegInfo &g = s_seg[T > 1 ? (int)(key >> 30) : 0];
        const int hi = g.start + g.count - 1;
        int p = s_par_leaf[k];
        for (int depth = 0; p >= 0; ++depth) {
            if (p >= n || depth > kMaxDepth) {
                atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                break;
            }
            __threadfence_block();
            if (atomicAdd(&s_visit[p], 1) == 0) break;   // the sibling is not done yet
            __threadfence_block();
            const int2 c = s_child[p];
            const int ia = c.x >= 0 ? c.x : ~c.x, ib = c.y >= 0 ? c.y : ~c.y;
            if ((unsigned)ia >= (unsigned)n || (unsigned)ib >= (unsigned)n) {
                atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                break;
            }
            const int2 r = s_range[p];
            const uint2 bl = c.x >= 0 ? s_q[c.x] : s_lq[ia];
            const uint2 br = c.y >= 0 ? s_q[c.y] : s_lq[ib];
            const unsigned qlo = qmin3(bl.x, br.x), qhi = qmax3(bl.y, br.y);
            const int count = r.y - r.x + 1;
            const int bundle = (a.bundle_k >= 2 && count <= a.bundle_k) ? 1 : 0;
            int4 w;
            w.x = (int)(qlo | ((unsigned)bundle << 31));
            w.y = (int)qhi;
            w.z = bundle ? r.x : c.x;
            w.w = rope_after(s_range, r.y, hi);
            a.nodes[p] = w;
            s_q[p] = make_uint2(qlo, qhi);
            if (F32) {
                // exact FP32 box: an internal child's from this launch's own
                // writes (L2), a leaf child's from its input point
                float4 la, ha, lb, hb;
                if (c.x >= 0) {
                    la = __ldcg(a.nodes32 + 2 * (size_t)c.x);
                    ha = __ldcg(a.nodes32 + 2 * (size_t)c.x + 1);
                    la.x = __int_as_float(__float_as_int(la.x) & 0x7FFFFFFF);
                } else {
                    la = ha = __ldg(a.pos + vA[ia]);
                }
                if (c.y >= 0) {
                    lb = __ldcg(a.nodes32 + 2 * (size_t)c.y);
                    hb = __ldcg(a.nodes32 + 2 * (size_t)c.y + 1);
                    lb.x = __int_as_float(__float_as_int(lb.x) & 0x7FFFFFFF);
                } else {
                    lb = hb = __ldg(a.pos + vA[ib]);
                }
                float lx = fminf(la.x, lb.x);
                if (bundle) lx = __int_as_float(__float_as_int(lx) | 0x80000000);
                __stcg(a.nodes32 + 2 * (size_t)p, make_float4(lx, fminf(la.y, lb.y), fminf(la.z, lb.z),
                                                              __int_as_float(w.z)));
                __stcg(a.nodes32 + 2 * (size_t)p + 1, make_float4(fmaxf(ha.x, hb.x), fmaxf(ha.y, hb.y),
                                                                  fmaxf(ha.z, hb.z), __int_as_float(w.w)));
            }
            p = s_par_int[p];
        }
    }
}

}  // namespace

// Used up to 3072 particles: build + query of one system measured against the
// multi-kernel build (rho 0.6, r_list 3.4, best particles per warp; eager /
// replayed from a CUDA graph, ms): N = 500 0.075 / 0.061 vs 0.118 / 0.086,
// N = 1000 0.091 / 0.076 vs 0.134 / 0.108, N = 3000 0.127 / 0.114 vs 0.155 /
// 0.130, N = 4096 0.142 / 0.132 vs 0.142 / 0.117.  At 4096 one SM's sort
// (51k cycles), hierarchy (32k) and fit (27k) no longer beat 152 SMs.
// (Measured again later, build alone at N = 4096: 0.083 ms eager against
// 0.088 ms for the nine-launch build, which replays faster from a graph; a
// bitonic sort of unique 64-bit keys instead of the radix sort measured
// slower: 0.082 against 0.067 ms at N = 3072.)
#ifndef QBVH_SMALL_USE
#define QBVH_SMALL_USE 3072
#endif
constexpr int kSmallUse = QBVH_SMALL_USE;

bool small_build_fits(const BuildArgs &a)
{
    return a.n >= 2 && a.n <= kSmallUse && a.n_sys == 1 && !a.wide_keys && !a.pos64 && !a.nodes21 &&
           a.n_types <= kMaxTrees;
}

void launch_small_build(const BuildArgs &a, cudaStream_t s)
{
    static bool attr_set[2] = {false, false};
    if (a.nodes32) {
        if (!attr_set[1]) {
            cudaFuncSetAttribute(small_build_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
            attr_set[1] = true;
        }
        small_build_kernel<true><<<1, kSB, kSmemBytes, s>>>(a);
    } else {
        if (!attr_set[0]) {
            cudaFuncSetAttribute(small_build_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
            attr_set[0] = true;
        }
        small_build_kernel<false><<<1, kSB, kSmemBytes, s>>>(a);
    }
}

}  // namespace qbvh
