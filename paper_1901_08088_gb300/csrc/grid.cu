// Uniform-grid (cell list) neighbor search: the comparator of the paper
// (Sec. 3, P "equivalent uniform grid algorithm"; Sec. 1, Fig. 1b).
//
//   grid_key_kernel   : bin every particle into cells at least the list radius
//                       wide (cells of size r_c, Sec. 3); key = cell index
//   (stable radix sort of the keys: sort.cu -- the sort-based, deterministic,
//    memory-compact grid build the paper compares against)
//   grid_range_kernel : first sorted particle of every cell (binary search)
//   grid_gather_kernel: positions in cell order, w = original index
//   grid_query_kernel : n lanes per particle (n a power of two, Sec. 3) walk
//                       the 27-cell stencil; each lane tests every n-th
//                       particle of a cell with the same exact FP32 expression
//                       as the tree traversal, and the group compacts its
//                       accepted neighbours with a ballot into the row.
//
// With at least 3 cells per axis the 27 stencil cells are distinct, so every
// particle within the list radius is seen exactly once per row.
#include "qbvh_internal.cuh"

namespace qbvh {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ int cell_coord(float x, float inv_w, int nc)
{
    int c = (int)__fmul_rn(x, inv_w);
    c = c < 0 ? 0 : c;
    return c >= nc ? nc - 1 : c;
}

__global__ void __launch_bounds__(kBlock) grid_key_kernel(GridArgs a)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= a.n) return;
    float4 p = __ldg(a.pos + i);
    unsigned err = 0u;
    const int type = __float_as_int(p.w);
    if (type < 0 || type >= a.n_types) err |= QBVH_DEVERR_BAD_TYPE;
    if (!(p.x >= 0.f && p.x < a.L && p.y >= 0.f && p.y < a.L && p.z >= 0.f && p.z < a.L)) {
        err |= QBVH_DEVERR_OUT_OF_BOX;
        p.x = (p.x == p.x) ? p.x : 0.f;   // NaN -> cell 0 (the run is reported as failed)
        p.y = (p.y == p.y) ? p.y : 0.f;
        p.z = (p.z == p.z) ? p.z : 0.f;
    }
    if (err) atomicOr(&a.status->err, err);
    const int nc = a.nc;
    const unsigned key = (unsigned)((cell_coord(p.x, a.inv_w, nc) * nc + cell_coord(p.y, a.inv_w, nc)) * nc +
                                    cell_coord(p.z, a.inv_w, nc));
    a.keys[i] = key;
}

// start[c] = first sorted index whose cell is >= c, for c in [0, nc^3]
__global__ void __launch_bounds__(kBlock) grid_range_kernel(GridArgs a)
{
    const int c = blockIdx.x * kBlock + threadIdx.x;
    const int ncell = a.nc * a.nc * a.nc;
    if (c > ncell) return;
    int lo = 0, hi = a.n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a.keys_sorted + mid) < (unsigned)c) lo = mid + 1; else hi = mid;
    }
    a.cell_start[c] = lo;
}

__global__ void __launch_bounds__(kBlock) grid_gather_kernel(GridArgs a)
{
    const int s = blockIdx.x * kBlock + threadIdx.x;
    if (s >= a.n) return;
    int orig = __ldg(a.order + s);
    if ((unsigned)orig >= (unsigned)a.n) {
        atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
        orig = 0;
    }
    const float4 p = __ldg(a.pos + orig);
    a.spos[s] = make_float4(p.x, p.y, p.z, __int_as_float(orig));
    if (a.stype) {
        int t = __float_as_int(p.w);
        a.stype[s] = t < 0 ? 0 : (t >= a.n_types ? a.n_types - 1 : t);
    }
}

__device__ __forceinline__ float min_image(float d, float L, float Linv)
{
    return __fsub_rn(d, __fmul_rn(L, rintf(__fmul_rn(d, Linv))));
}

template <int TPP>
__global__ void __launch_bounds__(kBlock) grid_query_kernel(const __grid_constant__ GridArgs a)
{
    const int lane = threadIdx.x & 31;
    const int sub = lane % TPP;
    const int gbase = lane - sub;                      // first lane of this group
    const unsigned gmask = (TPP == 32) ? 0xFFFFFFFFu : (((1u << TPP) - 1u) << gbase);
    const int s = (blockIdx.x * kBlock + threadIdx.x) / TPP;
    const bool active = s < a.n;
    int count = 0;
    if (active) {
        const float4 me = __ldg(a.spos + s);
        int i_orig = __float_as_int(me.w);
        if ((unsigned)i_orig >= (unsigned)a.n) {
            atomicOr(&a.status->err, QBVH_DEVERR_INTERNAL);
            i_orig = s;
        }
        const int ta = a.stype ? __ldg(a.stype + s) : 0;
        int *row = a.rows + (size_t)i_orig * a.cap;
        const int nc = a.nc;
        const unsigned key = __ldg(a.keys_sorted + s);
        const int cz = key % nc, cy = (key / nc) % nc, cx = key / (nc * nc);
        for (int ox = -1; ox <= 1; ++ox) {
            const int x = (cx + ox + nc) % nc;
            for (int oy = -1; oy <= 1; ++oy) {
                const int y = (cy + oy + nc) % nc;
                for (int oz = -1; oz <= 1; ++oz) {
                    const int z = (cz + oz + nc) % nc;
                    const int cell = (x * nc + y) * nc + z;
                    const int b = __ldg(a.cell_start + cell), e = __ldg(a.cell_start + cell + 1);
                    // every lane of the group runs the same number of rounds
                    for (int k0 = b; k0 < e; k0 += TPP) {
                        const int k = k0 + sub;
                        bool acc = false;
                        int j = 0;
                        if (k < e) {
                            const float4 q = __ldg(a.spos + k);
                            const int tb = a.stype ? __ldg(a.stype + k) : 0;
                            const float dx = min_image(__fsub_rn(q.x, me.x), a.L, a.Linv);
                            const float dy = min_image(__fsub_rn(q.y, me.y), a.L, a.Linv);
                            const float dz = min_image(__fsub_rn(q.z, me.z), a.L, a.Linv);
                            const float d2 =
                                __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                            acc = d2 < a.rl2[ta * a.n_types + tb] && k != s;
                            j = __float_as_int(q.w);
                        }
                        // compact the group's accepted neighbours into the row
                        const unsigned m = __ballot_sync(gmask, acc) & gmask;
                        if (acc) {
                            const int slot = count + __popc(m & ((1u << lane) - 1u));
                            if (slot < a.cap) __stcs(row + slot, j);
                        }
                        count += __popc(m);
                    }
                }
            }
        }
        if (sub == 0) a.counts[i_orig] = count;
    }
    const int mx = __reduce_max_sync(0xFFFFFFFFu, active ? count : 0);
    if (lane == 0 && mx > 0 && mx > __ldcg(&a.status->max_count)) atomicMax(&a.status->max_count, mx);
}

inline int blocks_for(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_grid_keys(const GridArgs &a, cudaStream_t s)
{
    if (a.n > 0) grid_key_kernel<<<blocks_for(a.n, kBlock), kBlock, 0, s>>>(a);
}

void launch_grid_cells(const GridArgs &a, cudaStream_t s)
{
    const long long ncell = (long long)a.nc * a.nc * a.nc;
    grid_range_kernel<<<blocks_for(ncell + 1, kBlock), kBlock, 0, s>>>(a);
    if (a.n > 0) grid_gather_kernel<<<blocks_for(a.n, kBlock), kBlock, 0, s>>>(a);
}

void launch_grid_query(const GridArgs &a, cudaStream_t s)
{
    if (a.n == 0) return;
    const int g = blocks_for((long long)a.n * a.tpp, kBlock);
    switch (a.tpp) {
    case 1: grid_query_kernel<1><<<g, kBlock, 0, s>>>(a); break;
    case 2: grid_query_kernel<2><<<g, kBlock, 0, s>>>(a); break;
    case 4: grid_query_kernel<4><<<g, kBlock, 0, s>>>(a); break;
    case 8: grid_query_kernel<8><<<g, kBlock, 0, s>>>(a); break;
    case 16: grid_query_kernel<16><<<g, kBlock, 0, s>>>(a); break;
    default: grid_query_kernel<32><<<g, kBlock, 0, s>>>(a); break;
    }
}

}  // namespace qbvh
