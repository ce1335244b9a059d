// Neighbor-list traversal (Alg. 1 of the paper).
//
// One thread per particle, particles taken in Z-order so that the threads of a
// warp walk nearby parts of the tree (Sec. 3).  For every tree the particle
// interacts with (one tree per type, per-type-pair radius):
//   1. test the 27 periodic images of the search sphere against the root
//      AABB and keep the overlapping ones in a bitset (Sec. 2.3; Alg. 1 image
//      loop);
//   2. for each image: stackless traversal from the root -- on overlap descend
//      to the left child, otherwise follow the rope, stop at the end marker
//      (Sec. 2.1; Alg. 1 inner loop);
//   3. node test: decompress the 10-bit bounds outward (lower bound rounded
//      down, upper up, Sec. 2.3 and Sec. 3) and test the sphere against the
//      box through the nearest point y = min(max(x, a), b) (Eq. 2), with every
//      rounding in the direction that can only enlarge the overlap;
//   4. leaf: the paper lists the particle as soon as the sphere overlaps the
//      leaf (Sec. 2.3), accepting false positives it allows to be filtered
//      later; here the exact FP32 minimum-image test is that filter, so the
//      list is exact.  Internal nodes with at most K leaves ("bundles", the
//      subtree collapse suggested at the end of Sec. 2.3) are tested leaf by
//      leaf without descending.
//
// Conservativeness.  The sphere radius is padded on the host:
//   r_search = r_list (1 + 2^-20) + 2^-19 L, rounded up, r_search^2 rounded up.
// If the exact test accepts j for image n (d2 < fl(r_list^2)), rounding in
// that expression and in the image position fl(x_i + n L) moves the real
// distance |x_i + nL - x_j| by at most r_list * 4.1 u + 5.2 u L (u = 2^-24),
// below the padding, and x_j lies in every decoded ancestor box, so every
// ancestor passes the round-down sphere test: no pair is lost.
//
// Duplicates.  A leaf may overlap the padded sphere of two images; it is
// accepted only under the image n = rint(fl((x_j - x_i) / L)) that the exact
// expression itself selects, so each j appears at most once per row.
#include "qbvh_internal.cuh"

namespace qbvh {

namespace {

struct Frame {
    float rx, ry, rz;   // R_lo
    float hx, hy, hz;   // bin width
};

__device__ __forceinline__ float q_at(unsigned w, int shift) { return (float)((w >> shift) & 1023u); }

// Sphere (centre p, squared radius rs2) against the quantized box of a node.
// Decoded bounds are rounded outward and the squared distance to the box is a
// lower bound, so a true overlap is never rejected.
__device__ __forceinline__ bool overlap_q(float px, float py, float pz, unsigned wlo, unsigned whi,
                                          const Frame &f, float rs2)
{
    const float lox = __fmaf_rd(q_at(wlo, 20), f.hx, f.rx);
    const float loy = __fmaf_rd(q_at(wlo, 10), f.hy, f.ry);
    const float loz = __fmaf_rd(q_at(wlo, 0), f.hz, f.rz);
    const float hix = __fmaf_ru(q_at(whi, 20), f.hx, f.rx);
    const float hiy = __fmaf_ru(q_at(whi, 10), f.hy, f.ry);
    const float hiz = __fmaf_ru(q_at(whi, 0), f.hz, f.rz);
    const float gx = fmaxf(fmaxf(__fsub_rd(lox, px), __fsub_rd(px, hix)), 0.f);
    const float gy = fmaxf(fmaxf(__fsub_rd(loy, py), __fsub_rd(py, hiy)), 0.f);
    const float gz = fmaxf(fmaxf(__fsub_rd(loz, pz), __fsub_rd(pz, hiz)), 0.f);
    const float d2 = __fmaf_rd(gx, gx, __fmaf_rd(gy, gy, __fmul_rd(gz, gz)));
    return d2 <= rs2;
}

// rint(t) == n for n in {-1, 0, 1} and |t| < 1.5 (always true for valid
// positions), written as range tests; rint rounds half to even, so +-0.5 -> 0.
__device__ __forceinline__ bool image_is(float t, int n)
{
    return n == 0 ? (fabsf(t) <= 0.5f) : (n > 0 ? (t > 0.5f) : (t < -0.5f));
}

struct Ctx {
    float xi, yi, zi;   // own position
    int self;           // own sorted index
    float L, Linv;
    float rl2;
    int nx, ny, nz;     // current image
    float nLx, nLy, nLz;
    int *row;
    int cap;
    int count;
};

// The exact FP32 minimum-image test (pinned expression) for leaf j under the
// current image; appends the original index on success.
__device__ __forceinline__ void exact_leaf(Ctx &c, int j, const float4 q)
{
    if (j == c.self) return;
    float dx = __fsub_rn(q.x, c.xi);
    float dy = __fsub_rn(q.y, c.yi);
    float dz = __fsub_rn(q.z, c.zi);
    if (!image_is(__fmul_rn(dx, c.Linv), c.nx) || !image_is(__fmul_rn(dy, c.Linv), c.ny) ||
        !image_is(__fmul_rn(dz, c.Linv), c.nz))
        return;
    dx = __fsub_rn(dx, c.nLx);
    dy = __fsub_rn(dy, c.nLy);
    dz = __fsub_rn(dz, c.nLz);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (d2 < c.rl2) {
        if (c.count < c.cap) c.row[c.count] = __float_as_int(q.w) & 0x7FFFFFFF;
        ++c.count;
    }
}

// Alg. 1 without the exact filter: list j when the sphere overlaps its
// quantized leaf box (false positives included).
__device__ __forceinline__ void candidate_leaf(Ctx &c, int j, const float4 q, const uint2 lq, const Frame &f,
                                               float px, float py, float pz, float rs2)
{
    if (j == c.self) return;
    if (overlap_q(px, py, pz, lq.x, lq.y, f, rs2)) {
        if (c.count < c.cap) c.row[c.count] = __float_as_int(q.w) & 0x7FFFFFFF;
        ++c.count;
    }
}

template <bool WIDE, bool CAND>
__global__ void query_kernel(const __grid_constant__ QueryArgs a)
{
    const uint2 *__restrict__ leaf_q = a.leaf_q;
    __shared__ int s_max[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int my_count = 0;
    if (s < a.n) {
        const float4 me = __ldg(a.leaves + s);
        int i_orig = __float_as_int(me.w) & 0x7FFFFFFF;
        if (i_orig >= a.n) {
            atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            i_orig = s;
        }
        int seg_i = 0;
        if (WIDE)
            seg_i = (int)(__ldg(reinterpret_cast<const unsigned long long *>(a.keys_sorted) + s) >> 30);
        else if (a.n_types > 1)
            seg_i = (int)(__ldg(reinterpret_cast<const unsigned *>(a.keys_sorted) + s) >> 30);
        const int T = a.n_types;
        const int sys = seg_i / T;
        const int ta = seg_i - sys * T;
        const SysInfo sy = a.sys[sys];

        Ctx c;
        c.xi = me.x;
        c.yi = me.y;
        c.zi = me.z;
        c.self = s;
        c.L = sy.L;
        c.Linv = sy.Linv;
        c.row = a.rows + (size_t)i_orig * a.cap;
        c.cap = a.cap;
        c.count = 0;

        for (int tb = 0; tb < T; ++tb) {
            const float rl = a.r_list[ta * T + tb];
            if (!(rl > 0.f)) continue;
            const SegInfo g = a.seg[sys * T + tb];
            if (g.count == 0) continue;
            c.rl2 = a.rl2[ta * T + tb];
            const float rs2 = a.rs2[ta * T + tb];
            Frame f;
            f.rx = g.rlo[0];
            f.ry = g.rlo[1];
            f.rz = g.rlo[2];
            f.hx = g.h[0];
            f.hy = g.h[1];
            f.hz = g.h[2];
            // per-axis lower bounds of the gap between each image and the root
            float gap[3][3];
            const float xs[3] = {me.x, me.y, me.z};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float p = (m == 1) ? xs[d] : __fadd_rn(xs[d], (m == 0) ? -c.L : c.L);
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
                                                   __fmaf_rd(gap[1][my], gap[1][my],
                                                             __fmul_rd(gap[2][mz], gap[2][mz])));
                        if (d2 <= rs2) mask |= 1u << (mx * 9 + my * 3 + mz);
                    }
            const int root = g.count >= 2 ? g.start : ~g.start;
            const int last = g.start + g.count - 1;
            while (mask) {
                const int img = __ffs(mask) - 1;
                mask &= mask - 1u;
                c.nx = img / 9 - 1;
                c.ny = (img / 3) % 3 - 1;
                c.nz = img % 3 - 1;
                c.nLx = c.nx == 0 ? 0.f : (c.nx > 0 ? c.L : -c.L);
                c.nLy = c.ny == 0 ? 0.f : (c.ny > 0 ? c.L : -c.L);
                c.nLz = c.nz == 0 ? 0.f : (c.nz > 0 ? c.L : -c.L);
                const float px = c.nx == 0 ? me.x : __fadd_rn(me.x, c.nLx);
                const float py = c.ny == 0 ? me.y : __fadd_rn(me.y, c.nLy);
                const float pz = c.nz == 0 ? me.z : __fadd_rn(me.z, c.nLz);
                int node = root;
                // pre-order visits every node at most once: 2 count - 1 steps
                int budget = 2 * g.count;
                while (node != QBVH_END) {
                    if (--budget < 0 || node > last || ~node > last || (node >= 0 && node < g.start) ||
                        (node < 0 && ~node < g.start)) {
                        atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                        break;
                    }
                    if (node >= 0) {
                        const int4 w = __ldg(a.nodes + node);
                        if (overlap_q(px, py, pz, (unsigned)w.x, (unsigned)w.y, f, rs2)) {
                            if (w.x < 0) {   // bundle: test its leaves directly
                                int l = (w.w == QBVH_END) ? last : ((w.w >= 0 ? w.w : ~w.w) - 1);
                                if (w.z < g.start || l > last) {
                                    atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
                                    l = w.z - 1;
                                }
                                for (int j = w.z; j <= l; ++j) {
                                    const float4 q = __ldg(a.leaves + j);
                                    if (CAND)
                                        candidate_leaf(c, j, q, __ldg(leaf_q + j), f, px, py, pz, rs2);
                                    else
                                        exact_leaf(c, j, q);
                                }
                                node = w.w;
                            } else {
                                node = w.z;
                            }
                        } else {
                            node = w.w;
                        }
                    } else {
                        const int j = ~node;
                        const float4 q = __ldg(a.leaves + j);
                        if (CAND)
                            candidate_leaf(c, j, q, __ldg(leaf_q + j), f, px, py, pz, rs2);
                        else
                            exact_leaf(c, j, q);
                        node = (j == last) ? QBVH_END : ((__float_as_int(q.w) < 0) ? j + 1 : ~(j + 1));
                    }
                }
            }
        }
        a.counts[i_orig] = c.count;
        my_count = c.count;
    }
    // largest row count of the block -> one atomic
    int m = __reduce_max_sync(0xFFFFFFFFu, my_count);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_max[warp] = m;
    __syncthreads();
    if (warp == 0) {
        m = (lane < (int)(blockDim.x >> 5)) ? s_max[lane] : 0;
        m = __reduce_max_sync(0xFFFFFFFFu, m);
        if (lane == 0 && m > 0) atomicMax(&a.status->max_count, m);
    }
}

}  // namespace

void launch_query(const QueryArgs &a, cudaStream_t s)
{
    if (a.n == 0) return;
    const int b = a.block;
    const int grid = (a.n + b - 1) / b;
    if (a.wide_keys) {
        if (a.candidates)
            query_kernel<true, true><<<grid, b, 0, s>>>(a);
        else
            query_kernel<true, false><<<grid, b, 0, s>>>(a);
    } else {
        if (a.candidates)
            query_kernel<false, true><<<grid, b, 0, s>>>(a);
        else
            query_kernel<false, false><<<grid, b, 0, s>>>(a);
    }
}

}  // namespace qbvh
