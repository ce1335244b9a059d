// C ABI of the qbvh library (declarations and contracts: include/qbvh.h).
//
// Host side of the method: argument validation, buffer ownership, the launch
// sequence of the build (Sec. 2.1-2.2) and of the traversal (Alg. 1), the
// row-capacity overflow check and retry, and the Lennard-Jones pass.
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/qbvh.h"
#include "qbvh_internal.cuh"

using namespace qbvh;

namespace qbvh {
int lj_particles_per_block();
}

// 1: one system of at most 3072 particles is built by one block (small_build.cu)
#ifndef QBVH_SMALL_BUILD
#define QBVH_SMALL_BUILD 1
#endif

namespace {

// Named host ranges around each stage for timeline tools (NVTX; header-only,
// a no-op unless a profiler attaches).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    bool grown = false;   // set when the last ensure() reallocated
};

enum Fault { FAULT_NONE = 0, FAULT_ALLOC = 1, FAULT_TIMEOUT = 2, FAULT_OVERFLOW = 3 };

int read_fault_env()
{
    const char *f = getenv("QBVH_FAULT");
    if (!f) return FAULT_NONE;
    if (!strcmp(f, "alloc")) return FAULT_ALLOC;
    if (!strcmp(f, "timeout")) return FAULT_TIMEOUT;
    if (!strcmp(f, "overflow")) return FAULT_OVERFLOW;
    return FAULT_NONE;
}

}  // namespace

struct qbvh_ctx {
    int device = 0;
    int fault = FAULT_NONE;
    // options
    int bundle_k = 16;
    int query_block = 128;
    int candidates = 0;
    int traversal = 1;
    int warp_particles = 32;
    int node_fmt = 0;      // 0: 10-bit quantized nodes (Fig. 3b), 1: FP32 nodes (Fig. 3a), 2: 21-bit nodes
    int lj_tpp = 2;        // lanes per particle in the LJ pass
    int lj_zorder = 1;     // LJ pass walks particles in the tree's Z-order
    int method = 0;        // 0: quantized BVH, 1: uniform grid comparator
    int grid_tpp = 8;      // lanes per particle of the grid traversal
    int type_trees = 1;    // 1: one tree per (system, type); 0: one tree per system
    int fused_lj = 0;      // qbvh_query_lj_async: LJ terms inside the traversal where supported
    int persistent = 0;    // traversal warps take packets from a queue
    int built_method = 0;
    const void *grid_pos = nullptr;   // positions recorded by a grid-method build
    int built_fmt = 0;     // node format of the last build
    // last build
    bool built = false;
    int n = 0, n_sys = 0, n_types = 0, n_seg = 0;
    int tree_types = 0;   // trees per system: n_types, or 1 when all types share a tree
    bool wide = false;
    int sorted = 0;   // which key/value buffer pair holds the sorted result
    std::vector<int> off;
    std::vector<float> L;
    std::vector<SysInfo> sysinfo;
    float L_min = 0.f, L_max = 0.f;
    bool f64 = false;        // last build was of double-precision particle data
    double L64 = 0.0;        // its FP64 box edge
    // last query
    bool have_list = false;
    int cap = 0;
    int max_count = 0;
    float r_list[64];
    // device buffers
    DevBuf keys[2], vals[2], sort_scratch, nodes, nodes32, nodes21, leaves, leaf_q, range, child, par_int, par_leaf,
        visit;
    DevBuf seg, acc, seg_start, frames, sys, sys_off, status;
    DevBuf rows, counts;
    DevBuf cell_start, stype;
    DevBuf leaves64;
    DevBuf lj_partials, lj_blk_sys, lj_blk_first, lj_sys_blk;
    std::vector<int> lj_layout_off;   // offsets the LJ block tables were built for
    int lj_n_blocks = 0;
    // uploads cached by content
    std::vector<SysInfo> up_sys;
    std::vector<int> up_off;
    // pinned host status
    DevStatus *h_status = nullptr;
};

namespace {

struct DeviceGuard {
    int prev = -1, want;
    explicit DeviceGuard(int d) : want(d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

int ensure(qbvh_ctx *h, DevBuf &b, size_t bytes)
{
    b.grown = false;
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return QBVH_OK;
    if (h->fault == FAULT_ALLOC) return QBVH_ERR_OOM;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return QBVH_ERR_OOM;
    }
    b.cap = bytes;
    b.grown = true;
    return QBVH_OK;
}

void release(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

int cuda_status()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QBVH_OK : QBVH_ERR_CUDA;
}

int ceil_log2(int v)
{
    int b = 0;
    while ((1 << b) < v) ++b;
    return b;
}

template <typename T>
int upload_if_changed(qbvh_ctx *h, DevBuf &dst, std::vector<T> &cache, const std::vector<T> &src,
                      cudaStream_t s)
{
    const size_t bytes = src.size() * sizeof(T);
    int rc = ensure(h, dst, bytes);
    if (rc) return rc;
    if (!dst.grown && cache.size() == src.size() && !memcmp(cache.data(), src.data(), bytes)) return QBVH_OK;
    if (cudaMemcpyAsync(dst.p, src.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return QBVH_ERR_CUDA;
    cache = src;
    return QBVH_OK;
}

float round_up_f(double v)
{
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}

int map_dev_err(unsigned err)
{
    if (err & QBVH_DEVERR_OUT_OF_BOX) return QBVH_ERR_OUT_OF_BOX;
    if (err & QBVH_DEVERR_BAD_TYPE) return QBVH_ERR_BAD_TYPE;
    if (err & QBVH_DEVERR_TIMEOUT) return QBVH_ERR_DEVICE_TIMEOUT;
    if (err & QBVH_DEVERR_INTERNAL) return QBVH_ERR_INTERNAL;
    return QBVH_OK;
}

// pos64_dev != nullptr: double-precision particle data of one system
// (double4 {x, y, z, type}, 32-byte aligned) with FP64 box edge L64; L[0] is
// then its nearest FP32 value.
int build_impl(qbvh_ctx *h, const void *pos_dev, int n, int n_sys, const int *off, const float *L, int n_types,
               cudaStream_t s, const void *pos64_dev = nullptr, double L64 = 0.0)
{
    NvtxRange range("qbvh_build");
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (n < 0 || n >= (1 << 30) || n_sys < 1 || n_sys > 65536) return QBVH_ERR_INVALID_ARG;
    if (n_types < 1 || n_types > QBVH_MAX_TYPES || n_sys * n_types > 65536) return QBVH_ERR_INVALID_ARG;
    const bool f64 = pos64_dev != nullptr || L64 != 0.0;
    if (f64) {
        // one system, narrow keys (at most 4 types), the BVH method
        if (n_sys != 1 || n_types > 4 || h->method != 0) return QBVH_ERR_INVALID_ARG;
        if (n > 0 && (!pos64_dev || ((uintptr_t)pos64_dev & 31u))) return QBVH_ERR_INVALID_ARG;
        if (!(L64 > 0.0) || !isfinite(L64)) return QBVH_ERR_INVALID_ARG;
    } else if (n > 0 && (!pos_dev || ((uintptr_t)pos_dev & 15u))) {
        return QBVH_ERR_INVALID_ARG;
    }
    if (!off || !L) return QBVH_ERR_INVALID_ARG;
    if (off[0] != 0 || off[n_sys] != n) return QBVH_ERR_INVALID_ARG;
    for (int k = 0; k < n_sys; ++k) {
        if (off[k + 1] < off[k]) return QBVH_ERR_INVALID_ARG;
        if (!(L[k] > 0.f) || !isfinite(L[k])) return QBVH_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    h->built = false;
    h->have_list = false;
    h->f64 = f64;
    h->L64 = f64 ? L64 : 0.0;
    h->n = n;
    h->n_sys = n_sys;
    h->n_types = n_types;
    h->tree_types = h->type_trees ? n_types : 1;
    h->n_seg = n_sys * h->tree_types;
    h->wide = (n_sys > 1) || (h->tree_types > 4);
    h->off.assign(off, off + n_sys + 1);
    h->L.assign(L, L + n_sys);
    h->sysinfo.resize(n_sys);
    h->L_min = INFINITY;
    h->L_max = 0.f;
    for (int k = 0; k < n_sys; ++k) {
        SysInfo si;
        memset(&si, 0, sizeof si);
        si.offset = off[k];
        si.count = off[k + 1] - off[k];
        si.L = L[k];
        si.Linv = 1.0f / L[k];
        si.mscale = 1023.0f / L[k];
        h->sysinfo[k] = si;
        h->L_min = fminf(h->L_min, L[k]);
        h->L_max = fmaxf(h->L_max, L[k]);
    }
    h->built_method = h->method;
    if (h->method == 1) {
        // grid comparator: the cell width is the list radius, known at the query;
        // the build records the input and the system description only
        if (n_sys != 1) return QBVH_ERR_INVALID_ARG;
        int rc0 = ensure(h, h->status, sizeof(DevStatus));
        rc0 = rc0 ? rc0 : upload_if_changed(h, h->sys, h->up_sys, h->sysinfo, s);
        rc0 = rc0 ? rc0 : upload_if_changed(h, h->sys_off, h->up_off, h->off, s);
        if (rc0) return rc0;
        if (cudaMemsetAsync(h->status.p, 0, sizeof(DevStatus), s) != cudaSuccess) return QBVH_ERR_CUDA;
        h->grid_pos = pos_dev;
        h->built = true;
        return QBVH_OK;
    }
    const int bits = h->wide ? 30 + ceil_log2(h->n_seg) : (h->tree_types > 1 ? 32 : 30);
    const int passes = (bits + 7) / 8;
    const size_t kb = h->wide ? 8 : 4;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int rc = QBVH_OK;
    rc = rc ? rc : ensure(h, h->keys[0], nn * kb);
    rc = rc ? rc : ensure(h, h->keys[1], nn * kb);
    rc = rc ? rc : ensure(h, h->vals[0], nn * 4);
    rc = rc ? rc : ensure(h, h->vals[1], nn * 4);
    rc = rc ? rc : ensure(h, h->sort_scratch, sort_scratch_bytes(n, passes));
    rc = rc ? rc : ensure(h, h->nodes, nn * sizeof(int4));
    if (h->node_fmt == 1) rc = rc ? rc : ensure(h, h->nodes32, nn * 2 * sizeof(float4));
    if (h->node_fmt == 2) rc = rc ? rc : ensure(h, h->nodes21, nn * 2 * sizeof(int4));
    rc = rc ? rc : ensure(h, h->leaves, nn * sizeof(float4));
    if (f64) rc = rc ? rc : ensure(h, h->leaves64, nn * 4 * sizeof(double));
    rc = rc ? rc : ensure(h, h->leaf_q, nn * sizeof(uint2));
    rc = rc ? rc : ensure(h, h->range, nn * sizeof(int2));
    rc = rc ? rc : ensure(h, h->child, nn * sizeof(int2));
    rc = rc ? rc : ensure(h, h->par_int, nn * 4);
    rc = rc ? rc : ensure(h, h->par_leaf, nn * 4);
    rc = rc ? rc : ensure(h, h->visit, nn * 4);
    rc = rc ? rc : ensure(h, h->seg, (size_t)h->n_seg * sizeof(SegInfo));
    rc = rc ? rc : ensure(h, h->acc, (size_t)h->n_seg * 8 * 4);
    rc = rc ? rc : ensure(h, h->seg_start, (size_t)(h->n_seg + 1) * 4);
    rc = rc ? rc : ensure(h, h->frames, (size_t)h->n_seg * 8 * 4);
    rc = rc ? rc : ensure(h, h->status, sizeof(DevStatus));
    if (rc) return rc;
    rc = upload_if_changed(h, h->sys, h->up_sys, h->sysinfo, s);
    if (rc) return rc;
    rc = upload_if_changed(h, h->sys_off, h->up_off, h->off, s);
    if (rc) return rc;

    BuildArgs a;
    memset(&a, 0, sizeof a);
    a.pos = reinterpret_cast<const float4 *>(pos_dev);
    a.pos64 = f64 ? reinterpret_cast<const double4_32a *>(pos64_dev) : nullptr;
    a.L64 = L64;
    a.leaves64 = f64 ? reinterpret_cast<double4_32a *>(h->leaves64.p) : nullptr;
    a.n = n;
    a.n_sys = n_sys;
    a.n_types = h->tree_types;
    a.type_bound = n_types;
    a.n_seg = h->n_seg;
    a.wide_keys = h->wide;
    a.bundle_k = h->bundle_k;
    a.sys = reinterpret_cast<const SysInfo *>(h->sys.p);
    a.sys_off = reinterpret_cast<const int *>(h->sys_off.p);
    a.seg = reinterpret_cast<SegInfo *>(h->seg.p);
    a.seg_rootbits = reinterpret_cast<unsigned *>(h->acc.p);
    a.seg_start = reinterpret_cast<int *>(h->seg_start.p);
    a.frames = reinterpret_cast<float *>(h->frames.p);
    a.keys = h->keys[0].p;
    a.range = reinterpret_cast<int2 *>(h->range.p);
    a.child = reinterpret_cast<int2 *>(h->child.p);
    a.par_int = reinterpret_cast<int *>(h->par_int.p);
    a.par_leaf = reinterpret_cast<int *>(h->par_leaf.p);
    a.visit = reinterpret_cast<int *>(h->visit.p);
    a.leaf_q = reinterpret_cast<uint2 *>(h->leaf_q.p);
    a.nodes = reinterpret_cast<int4 *>(h->nodes.p);
    a.nodes32 = h->node_fmt == 1 ? reinterpret_cast<float4 *>(h->nodes32.p) : nullptr;
    a.nodes21 = h->node_fmt == 2 ? reinterpret_cast<int4 *>(h->nodes21.p) : nullptr;
    a.leaves = reinterpret_cast<float4 *>(h->leaves.p);
    a.status = reinterpret_cast<DevStatus *>(h->status.p);
    a.sort_scratch = reinterpret_cast<unsigned *>(h->sort_scratch.p);
    a.sort_scratch_words = sort_scratch_bytes(n, passes) / sizeof(unsigned);
    a.sort_passes = passes;
    h->built_fmt = h->node_fmt;

    if (QBVH_SMALL_BUILD && small_build_fits(a)) {
        // one small system (small_build_fits): the whole build in one block
        h->sorted = 0;
        a.keys_sorted = h->keys[0].p;
        a.order = reinterpret_cast<const int *>(h->vals[0].p);
        launch_small_build(a, s);
    } else {
        launch_build_prepare(a, s);
        launch_morton(a, s);
        launch_seg_scan(a, s);
        h->sorted = radix_sort_pairs(h->wide, h->keys[0].p, h->keys[1].p, reinterpret_cast<int *>(h->vals[0].p),
                                     reinterpret_cast<int *>(h->vals[1].p), n, bits, h->sort_scratch.p,
                                     &a.status->err, s, /*prepared=*/true);
        a.keys_sorted = h->keys[h->sorted].p;
        a.order = reinterpret_cast<const int *>(h->vals[h->sorted].p);
        launch_karras(a, s);
        launch_fit(a, s);
    }
    rc = cuda_status();
    if (rc) return rc;
    h->built = true;
    return QBVH_OK;
}

// Grid comparator: bin into cells at least the largest list radius wide (with
// a 2^-14 relative margin that absorbs the FP32 binning round-off, so two
// particles closer than the radius always sit in adjacent cells), sort by
// cell, find every cell's first particle, gather, walk the 27-cell stencil.
int grid_enqueue(qbvh_ctx *h, const float *r_list, const float *rl2, int cap, cudaStream_t s)
{
    const int T = h->n_types;
    float rmax = 0.f;
    for (int p = 0; p < T * T; ++p) rmax = fmaxf(rmax, r_list[p]);
    const float L = h->L[0];
    const int n = h->n;
    int nc = rmax > 0.f ? (int)floor((double)L / ((double)rmax * (1.0 + ldexp(1.0, -14)))) : 1023;
    // no more than about 2 cells per particle (wider cells stay correct)
    const int nc_cap = (int)ceil(cbrt(2.0 * (n > 27 ? n : 27)));
    if (nc > nc_cap) nc = nc_cap;
    if (nc > 1023) nc = 1023;
    if (nc < 3) return QBVH_ERR_CUTOFF_TOO_LARGE;
    const long long ncell = (long long)nc * nc * nc;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int rc = QBVH_OK;
    rc = rc ? rc : ensure(h, h->keys[0], nn * 4);
    rc = rc ? rc : ensure(h, h->keys[1], nn * 4);
    rc = rc ? rc : ensure(h, h->vals[0], nn * 4);
    rc = rc ? rc : ensure(h, h->vals[1], nn * 4);
    const int bits = ceil_log2((int)ncell + 1);
    rc = rc ? rc : ensure(h, h->sort_scratch, sort_scratch_bytes(n, (bits + 7) / 8));
    rc = rc ? rc : ensure(h, h->cell_start, (size_t)(ncell + 1) * 4);
    rc = rc ? rc : ensure(h, h->leaves, nn * sizeof(float4));
    if (T > 1) rc = rc ? rc : ensure(h, h->stype, nn * 4);
    if (rc) return rc;
    GridArgs a;
    memset(&a, 0, sizeof a);
    a.pos = reinterpret_cast<const float4 *>(h->grid_pos);
    a.n = n;
    a.n_types = T;
    a.L = L;
    a.Linv = 1.0f / L;
    a.nc = nc;
    a.inv_w = (float)nc / L;
    a.keys = reinterpret_cast<unsigned *>(h->keys[0].p);
    a.cell_start = reinterpret_cast<int *>(h->cell_start.p);
    a.spos = reinterpret_cast<float4 *>(h->leaves.p);
    a.stype = T > 1 ? reinterpret_cast<int *>(h->stype.p) : nullptr;
    a.rows = reinterpret_cast<int *>(h->rows.p);
    a.counts = reinterpret_cast<int *>(h->counts.p);
    a.cap = cap;
    a.tpp = h->grid_tpp;
    for (int p = 0; p < T * T; ++p) a.rl2[p] = r_list[p] > 0.f ? rl2[p] : -1.f;
    a.status = reinterpret_cast<DevStatus *>(h->status.p);
    launch_grid_keys(a, s);
    h->sorted = radix_sort_pairs(false, h->keys[0].p, h->keys[1].p, reinterpret_cast<int *>(h->vals[0].p),
                                 reinterpret_cast<int *>(h->vals[1].p), n, bits, h->sort_scratch.p, &a.status->err,
                                 s);
    a.keys_sorted = reinterpret_cast<const unsigned *>(h->keys[h->sorted].p);
    a.order = reinterpret_cast<const int *>(h->vals[h->sorted].p);
    launch_grid_cells(a, s);
    launch_grid_query(a, s);
    return cuda_status();
}

// LJ outputs requested with the traversal (qbvh_query_lj_async)
struct QueryLJ {
    const void *pos;
    const float *eps, *sig, *r_cut;
    float *e;
    double *U;
    float *F;
    double *dE, *dS;
};

// The traversal sums the LJ terms itself for one system of one type walked
// one particle per lane (exact lists of FP32 data, quantized BVH).
bool fused_lj_ok(const qbvh_ctx *h)
{
    return h->fused_lj && h->built_method == 0 && !h->f64 && !h->candidates && h->traversal == 1 &&
           h->warp_particles == 32 && h->n_sys == 1 && h->n_types == 1 && h->n > 0;
}

int query_enqueue(qbvh_ctx *h, const float *r_list_host, int cap, cudaStream_t s, const QueryLJ *lj = nullptr)
{
    NvtxRange range("qbvh_query");
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (!h->built) return QBVH_ERR_NOT_BUILT;
    if (!r_list_host || cap < 1 || cap > (1 << 28)) return QBVH_ERR_INVALID_ARG;
    cap = (cap + 7) & ~7;   // rows start on 32-byte boundaries (whole sectors are written)
    const int T = h->n_types;
    if ((long long)h->n * cap >= (1LL << 40)) return QBVH_ERR_INVALID_ARG;
    // all types in one tree per system: the leaf test cannot tell types
    // apart, so every type pair must share one radius
    const bool merged = h->built_method == 0 && h->tree_types != T;
    if (merged)
        for (int p = 0; p < T * T; ++p)
            if (!(r_list_host[p] == r_list_host[0])) return QBVH_ERR_INVALID_ARG;
    const int Tq = merged ? 1 : T;   // radius matrix of the trees
    // the traversal numbers its threads in 32 bits: n particles with 32 / p
    // lanes each (p particles per warp, or the grid's lanes per particle)
    // must stay below 2^32 threads, with room for the last block's rounding
    const int lanes = h->built_method == 1 ? h->grid_tpp
                      : (h->traversal == 1 && !h->f64) ? 32 / h->warp_particles : 1;
    if ((long long)h->n * lanes > (1LL << 32) - 1024) return QBVH_ERR_INVALID_ARG;
    QueryArgs q;
    memset(&q, 0, sizeof q);
    if (h->f64 && h->candidates) return QBVH_ERR_INVALID_ARG;   // exact lists only for FP64 data
    const double L_half = h->f64 ? h->L64 : (double)h->L_min;
    for (int a = 0; a < Tq; ++a)
        for (int b = 0; b < Tq; ++b) {
            const float r = r_list_host[a * T + b];
            if (!(r >= 0.f) || !isfinite(r) || r != r_list_host[b * T + a]) return QBVH_ERR_INVALID_ARG;
            // below half the box by a relative 2^-20: then a pair is found under
            // exactly one periodic image, the one the exact test selects
            if (h->n > 0 && r > 0.f && !((double)r < 0.5 * L_half * (1.0 - ldexp(1.0, -20))))
                return QBVH_ERR_CUTOFF_TOO_LARGE;
            if (h->f64) {
                // FP32 test of the rounded positions vs the FP64 decision: each
                // component differs by at most eps = 2^-21 L for pairs within
                // the radius (rounding of both positions and of L, 2^-24 L
                // each, and of the two FP32 subtractions), so
                // |d2_32 - d2_64| <= 2 sqrt(3) r eps + 3 eps^2 + 3 * 2^-24 (r + eps)^2
                // < M below; outside [r^2 - M, r^2 + M] the FP32 test decides
                const double r64 = (double)r, eps = ldexp(h->L64, -21);
                const double r2 = r64 * r64;
                const double M = 8.0 * r64 * eps + 4.0 * eps * eps + ldexp((r64 + eps) * (r64 + eps), -20);
                float lo = (float)(r2 - M);
                if ((double)lo > r2 - M) lo = nextafterf(lo, -INFINITY);
                q.rl2_lo[a * Tq + b] = lo;
                q.rl2_hi[a * Tq + b] = round_up_f(r2 + M);
                q.r2_64[a * Tq + b] = r2;
            }
            q.r_list[a * Tq + b] = r;
            q.rl2[a * Tq + b] = r * r;
            // padded search radius: covers FP32 rounding of the image position
            // and of the exact test (see query.cu), rounded up
            const float rs = round_up_f((double)r * (1.0 + ldexp(1.0, -20)) + ldexp((double)h->L_max, -19));
            q.rs[a * Tq + b] = rs;
            q.rs2[a * Tq + b] = round_up_f((double)rs * (double)rs);
        }
    DeviceGuard g(h->device);
    int rc = ensure(h, h->rows, (size_t)(h->n > 0 ? h->n : 1) * cap * 4);
    rc = rc ? rc : ensure(h, h->counts, (size_t)(h->n > 0 ? h->n : 1) * 4);
    if (rc) return rc;
    DevStatus *st = reinterpret_cast<DevStatus *>(h->status.p);
    // the largest count and the traversal's packet queue start at zero (the
    // error word keeps what the build found)
    if (cudaMemsetAsync(&st->max_count, 0, 2 * sizeof(int), s) != cudaSuccess) return QBVH_ERR_CUDA;
    if (h->built_method == 1) {
        rc = grid_enqueue(h, q.r_list, q.rl2, cap, s);
        if (rc) return rc;
        if (cudaMemcpyAsync(h->h_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return QBVH_ERR_CUDA;
        rc = cuda_status();
        if (rc) return rc;
        h->cap = cap;
        memcpy(h->r_list, r_list_host, sizeof(float) * T * T);
        h->have_list = true;
        return QBVH_OK;
    }
    q.nodes = reinterpret_cast<const int4 *>(h->nodes.p);
    q.nodes32 = reinterpret_cast<const float4 *>(h->nodes32.p);
    q.nodes21 = reinterpret_cast<const int4 *>(h->nodes21.p);
    q.node_fmt = h->built_fmt;
    q.leaves = reinterpret_cast<const float4 *>(h->leaves.p);
    q.leaf_q = reinterpret_cast<const uint2 *>(h->leaf_q.p);
    q.keys_sorted = h->keys[h->sorted].p;
    q.wide_keys = h->wide;
    q.seg = reinterpret_cast<const SegInfo *>(h->seg.p);
    q.sys = reinterpret_cast<const SysInfo *>(h->sys.p);
    q.n = h->n;
    q.n_types = Tq;
    q.cap = cap;
    q.rows = reinterpret_cast<int *>(h->rows.p);
    q.counts = reinterpret_cast<int *>(h->counts.p);
    q.status = st;
    q.candidates = h->candidates;
    q.traversal = h->traversal;
    q.warp_particles = h->warp_particles;
    q.block = h->query_block;
    q.persistent = h->persistent;
    q.f64 = h->f64 ? 1 : 0;
    q.leaves64 = h->f64 ? reinterpret_cast<const double4_32a *>(h->leaves64.p) : nullptr;
    q.L64 = h->L64;
    if (lj && fused_lj_ok(h)) {
        const int nb = query_lj_blocks(h->n, h->query_block);
        rc = ensure(h, h->lj_partials, (size_t)nb * 3 * 8);
        if (rc) return rc;
        const float rc_ = lj->r_cut[0];
        q.lj = 1;
        q.lj_eps = lj->eps;
        q.lj_sig = lj->sig;
        q.lj_rc2 = rc_ * rc_;
        q.lj_e = lj->e;
        q.lj_F = lj->F;
        q.lj_partials = reinterpret_cast<double *>(h->lj_partials.p);
        launch_query_lj(q, s);
        launch_lj_finalize_one(q.lj_partials, nb, lj->U, lj->dE, lj->dS, s);
    } else {
        launch_query(q, s);
    }
    if (cudaMemcpyAsync(h->h_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVH_ERR_CUDA;
    rc = cuda_status();
    if (rc) return rc;
    h->cap = cap;
    memcpy(h->r_list, r_list_host, sizeof(float) * T * T);
    h->have_list = true;
    return QBVH_OK;
}

int status_check(qbvh_ctx *h)
{
    h->max_count = h->h_status->max_count;
    int rc = map_dev_err(h->h_status->err);
    if (h->fault == FAULT_TIMEOUT) rc = QBVH_ERR_DEVICE_TIMEOUT;
    if (rc) return rc;
    if (h->fault == FAULT_OVERFLOW && h->max_count <= h->cap) h->max_count = h->cap + 1;
    if (h->max_count > h->cap) return QBVH_ERR_OVERFLOW;
    return QBVH_OK;
}

}  // namespace

extern "C" {

const char *qbvh_strerror(int code)
{
    switch (code) {
    case QBVH_OK: return "ok";
    case QBVH_ERR_INVALID_ARG: return "invalid argument";
    case QBVH_ERR_OUT_OF_BOX: return "position outside [0, L) or not finite";
    case QBVH_ERR_BAD_TYPE: return "particle type outside [0, n_types)";
    case QBVH_ERR_CUTOFF_TOO_LARGE: return "list radius must be below half the box edge";
    case QBVH_ERR_OVERFLOW: return "neighbor row capacity exceeded after all retries";
    case QBVH_ERR_DEVICE_TIMEOUT: return "bounded device-side wait gave up";
    case QBVH_ERR_CUDA: return "CUDA runtime error";
    case QBVH_ERR_OOM: return "out of memory";
    case QBVH_ERR_NOT_BUILT: return "no tree or list built yet";
    case QBVH_ERR_INTERNAL: return "device-side consistency check failed";
    default: return "unknown status";
    }
}

int qbvh_create(qbvh_handle *out, int device)
{
    if (!out) return QBVH_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return QBVH_ERR_CUDA;
    }
    qbvh_ctx *h = new qbvh_ctx();
    h->device = device;
    h->fault = read_fault_env();
    DeviceGuard g(device);
    if (cudaMallocHost(&h->h_status, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return QBVH_ERR_OOM;
    }
    memset(h->h_status, 0, sizeof(DevStatus));
    *out = h;
    return QBVH_OK;
}

int qbvh_destroy(qbvh_handle h)
{
    if (!h) return QBVH_ERR_INVALID_ARG;
    {
        DeviceGuard g(h->device);
        cudaDeviceSynchronize();
        DevBuf *all[] = {&h->keys[0], &h->keys[1], &h->vals[0], &h->vals[1], &h->sort_scratch, &h->nodes, &h->nodes32,
                         &h->nodes21,
                         &h->leaves, &h->leaf_q, &h->range, &h->child, &h->par_int, &h->par_leaf, &h->visit,
                         &h->seg, &h->acc, &h->seg_start, &h->frames, &h->sys, &h->sys_off, &h->status,
                         &h->rows, &h->counts, &h->cell_start, &h->stype, &h->lj_partials, &h->lj_blk_sys, &h->lj_blk_first,
                         &h->lj_sys_blk, &h->leaves64};
        for (DevBuf *b : all) release(*b);
        if (h->h_status) cudaFreeHost(h->h_status);
    }
    delete h;
    return QBVH_OK;
}

int qbvh_set_option(qbvh_handle h, int option, int value)
{
    if (!h) return QBVH_ERR_INVALID_ARG;
    switch (option) {
    case QBVH_OPT_BUNDLE:
        if (value < 1 || value > 64) return QBVH_ERR_INVALID_ARG;
        h->bundle_k = value;
        return QBVH_OK;
    case QBVH_OPT_QUERY_BLOCK:
        if (value < 32 || value > 256 || (value & 31)) return QBVH_ERR_INVALID_ARG;
        h->query_block = value;
        return QBVH_OK;
    case QBVH_OPT_CANDIDATES:
        if (value != 0 && value != 1) return QBVH_ERR_INVALID_ARG;
        h->candidates = value;
        return QBVH_OK;
    case QBVH_OPT_TRAVERSAL:
        if (value != 0 && value != 1) return QBVH_ERR_INVALID_ARG;
        h->traversal = value;
        return QBVH_OK;
    case QBVH_OPT_NODE_FORMAT:
        if (value < 0 || value > 2) return QBVH_ERR_INVALID_ARG;
        h->node_fmt = value;
        return QBVH_OK;
    case QBVH_OPT_LJ_LANES:
        if (value < 1 || value > 32 || (value & (value - 1))) return QBVH_ERR_INVALID_ARG;
        h->lj_tpp = value;
        return QBVH_OK;
    case QBVH_OPT_LJ_ZORDER:
        if (value != 0 && value != 1) return QBVH_ERR_INVALID_ARG;
        h->lj_zorder = value;
        return QBVH_OK;
    case QBVH_OPT_WARP_PARTICLES:
        if (value < 1 || value > 32 || (value & (value - 1))) return QBVH_ERR_INVALID_ARG;
        h->warp_particles = value;
        return QBVH_OK;
    case QBVH_OPT_METHOD:
        if (value != 0 && value != 1) return QBVH_ERR_INVALID_ARG;
        h->method = value;
        return QBVH_OK;
    case QBVH_OPT_GRID_LANES:
        if (value < 1 || value > 32 || (value & (value - 1))) return QBVH_ERR_INVALID_ARG;
        h->grid_tpp = value;
        return QBVH_OK;
    case QBVH_OPT_TYPE_TREES:
        if (value != 0 && value != 1) return QBVH_ERR_INVALID_ARG;
        h->type_trees = value;
        return QBVH_OK;
    case QBVH_OPT_FUSED_LJ:
        if (value != 0 && value != 1) return QBVH_ERR_INVALID_ARG;
        h->fused_lj = value;
        return QBVH_OK;
    case QBVH_OPT_PERSISTENT:
        if (value != 0 && value != 1) return QBVH_ERR_INVALID_ARG;
        h->persistent = value;
        return QBVH_OK;
    default: return QBVH_ERR_INVALID_ARG;
    }
}

int qbvh_get_option(qbvh_handle h, int option, int *value)
{
    if (!h || !value) return QBVH_ERR_INVALID_ARG;
    switch (option) {
    case QBVH_OPT_BUNDLE: *value = h->bundle_k; return QBVH_OK;
    case QBVH_OPT_QUERY_BLOCK: *value = h->query_block; return QBVH_OK;
    case QBVH_OPT_CANDIDATES: *value = h->candidates; return QBVH_OK;
    case QBVH_OPT_TRAVERSAL: *value = h->traversal; return QBVH_OK;
    case QBVH_OPT_NODE_FORMAT: *value = h->node_fmt; return QBVH_OK;
    case QBVH_OPT_LJ_LANES: *value = h->lj_tpp; return QBVH_OK;
    case QBVH_OPT_LJ_ZORDER: *value = h->lj_zorder; return QBVH_OK;
    case QBVH_OPT_WARP_PARTICLES: *value = h->warp_particles; return QBVH_OK;
    case QBVH_OPT_METHOD: *value = h->method; return QBVH_OK;
    case QBVH_OPT_GRID_LANES: *value = h->grid_tpp; return QBVH_OK;
    case QBVH_OPT_TYPE_TREES: *value = h->type_trees; return QBVH_OK;
    case QBVH_OPT_FUSED_LJ: *value = h->fused_lj; return QBVH_OK;
    case QBVH_OPT_PERSISTENT: *value = h->persistent; return QBVH_OK;
    default: return QBVH_ERR_INVALID_ARG;
    }
}

int qbvh_build(qbvh_handle h, const void *pos_dev, int n, float L, int n_types, cudaStream_t stream)
{
    int off[2] = {0, n};
    return build_impl(h, pos_dev, n, 1, off, &L, n_types, stream);
}

int qbvh_build_f64(qbvh_handle h, const void *pos64_dev, int n, double L, int n_types, cudaStream_t stream)
{
    if (!h || !(L > 0.0) || !isfinite(L)) return QBVH_ERR_INVALID_ARG;
    const float L32 = (float)L;
    if (!(L32 > 0.f) || !isfinite(L32)) return QBVH_ERR_INVALID_ARG;
    int off[2] = {0, n};
    return build_impl(h, nullptr, n, 1, off, &L32, n_types, stream, pos64_dev, L);
}

int qbvh_build_batched(qbvh_handle h, const void *pos_dev, int n_total, int n_sys, const int *sys_offsets_host,
                       const float *L_host, int n_types, cudaStream_t stream)
{
    return build_impl(h, pos_dev, n_total, n_sys, sys_offsets_host, L_host, n_types, stream);
}

int qbvh_query_async(qbvh_handle h, const float *r_list_host, int cap, cudaStream_t stream)
{
    return query_enqueue(h, r_list_host, cap, stream);
}

int qbvh_query_lj_async(qbvh_handle h, const void *pos_dev, const float *r_list_host, int cap,
                        const float *eps_dev, const float *sig_dev, const float *r_cut_host, float *e_dev,
                        double *U_dev, float *F_dev, double *dE_dev, double *dS_dev, cudaStream_t stream)
{
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (!h->built) return QBVH_ERR_NOT_BUILT;
    if (!r_list_host || !eps_dev || !sig_dev || !r_cut_host || !U_dev) return QBVH_ERR_INVALID_ARG;
    if (h->n > 0 && (!pos_dev || ((uintptr_t)pos_dev & 15u))) return QBVH_ERR_INVALID_ARG;
    const int T = h->n_types;
    for (int p = 0; p < T * T; ++p) {
        const float rc = r_cut_host[p];
        if (!(rc > 0.f) || !isfinite(rc) || rc > r_list_host[p]) return QBVH_ERR_INVALID_ARG;
    }
    const QueryLJ lj{pos_dev, eps_dev, sig_dev, r_cut_host, e_dev, U_dev, F_dev, dE_dev, dS_dev};
    const bool fused = fused_lj_ok(h);
    int rc = query_enqueue(h, r_list_host, cap, stream, &lj);
    if (rc || fused) return rc;
    return qbvh_lj_forward(h, pos_dev, eps_dev, sig_dev, r_cut_host, e_dev, U_dev, F_dev, dE_dev, dS_dev, stream);
}

int qbvh_query_status(qbvh_handle h, int *max_count)
{
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (!h->have_list) return QBVH_ERR_NOT_BUILT;
    int rc = status_check(h);
    if (max_count) *max_count = h->max_count;
    return rc;
}

int qbvh_query(qbvh_handle h, const float *r_list_host, int cap, int max_retries, cudaStream_t stream)
{
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (max_retries < 0) return QBVH_ERR_INVALID_ARG;
    for (int attempt = 0;; ++attempt) {
        int rc = query_enqueue(h, r_list_host, cap, stream);
        if (rc) return rc;
        {
            DeviceGuard g(h->device);
            if (cudaStreamSynchronize(stream) != cudaSuccess) {
                cudaGetLastError();
                return QBVH_ERR_CUDA;
            }
        }
        rc = status_check(h);
        if (rc != QBVH_ERR_OVERFLOW) return rc;
        if (attempt >= max_retries) return QBVH_ERR_OVERFLOW;
        cap = ((h->max_count + 31) / 32) * 32;
    }
}

int nlist_get(qbvh_handle h, const int **rows, const int **counts, int *cap, int *max_count)
{
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (!h->have_list) return QBVH_ERR_NOT_BUILT;
    if (rows) *rows = reinterpret_cast<const int *>(h->rows.p);
    if (counts) *counts = reinterpret_cast<const int *>(h->counts.p);
    if (cap) *cap = h->cap;
    if (max_count) *max_count = h->max_count;
    return QBVH_OK;
}

int qbvh_tree_get(qbvh_handle h, const void **nodes, const void **leaves, const int **order, const int **seg_start,
                  const float **frames, int *n_seg)
{
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (!h->built || h->built_method != 0) return QBVH_ERR_NOT_BUILT;
    if (nodes) *nodes = h->nodes.p;
    if (leaves) *leaves = h->leaves.p;
    if (order) *order = reinterpret_cast<const int *>(h->vals[h->sorted].p);
    if (seg_start) *seg_start = reinterpret_cast<const int *>(h->seg_start.p);
    if (frames) *frames = reinterpret_cast<const float *>(h->frames.p);
    if (n_seg) *n_seg = h->n_seg;
    return QBVH_OK;
}

int qbvh_lj_forward(qbvh_handle h, const void *pos_dev, const float *eps_dev, const float *sig_dev,
                    const float *r_cut_host, float *e_dev, double *U_dev, float *F_dev, double *dE_dev,
                    double *dS_dev, cudaStream_t stream)
{
    NvtxRange range("qbvh_lj_forward");
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (!h->have_list) return QBVH_ERR_NOT_BUILT;
    if (!eps_dev || !sig_dev || !r_cut_host || !U_dev) return QBVH_ERR_INVALID_ARG;
    if (h->n > 0 && (!pos_dev || ((uintptr_t)pos_dev & 15u))) return QBVH_ERR_INVALID_ARG;
    const int T = h->n_types;
    LJArgs a;
    memset(&a, 0, sizeof a);
    for (int p = 0; p < T * T; ++p) {
        const float rc = r_cut_host[p];
        if (!(rc > 0.f) || !isfinite(rc) || rc > h->r_list[p]) return QBVH_ERR_INVALID_ARG;
        a.rc2[p] = rc * rc;
    }
    DeviceGuard g(h->device);
    // block tables: every block covers particles of one system
    const int B = lj_particles_per_block();
    int rc = QBVH_OK;
    if (h->lj_layout_off != h->off || h->lj_blk_sys.p == nullptr) {
        std::vector<int> blk_sys, blk_first, sys_blk(h->n_sys + 1, 0);
        for (int k = 0; k < h->n_sys; ++k) {
            sys_blk[k] = (int)blk_sys.size();
            for (int f = h->off[k]; f < h->off[k + 1]; f += B) {
                blk_sys.push_back(k);
                blk_first.push_back(f);
            }
        }
        sys_blk[h->n_sys] = (int)blk_sys.size();
        h->lj_n_blocks = (int)blk_sys.size();
        if (blk_sys.empty()) {
            blk_sys.push_back(0);
            blk_first.push_back(0);
        }
        rc = rc ? rc : ensure(h, h->lj_blk_sys, blk_sys.size() * 4);
        rc = rc ? rc : ensure(h, h->lj_blk_first, blk_first.size() * 4);
        rc = rc ? rc : ensure(h, h->lj_sys_blk, sys_blk.size() * 4);
        if (rc) return rc;
        if (cudaMemcpyAsync(h->lj_blk_sys.p, blk_sys.data(), blk_sys.size() * 4, cudaMemcpyHostToDevice, stream) ||
            cudaMemcpyAsync(h->lj_blk_first.p, blk_first.data(), blk_first.size() * 4, cudaMemcpyHostToDevice,
                            stream) ||
            cudaMemcpyAsync(h->lj_sys_blk.p, sys_blk.data(), sys_blk.size() * 4, cudaMemcpyHostToDevice, stream))
            return QBVH_ERR_CUDA;
        h->lj_layout_off = h->off;
    }
    const int np = 1 + 2 * T * T;
    rc = ensure(h, h->lj_partials, (size_t)(h->lj_n_blocks > 0 ? h->lj_n_blocks : 1) * np * 8);
    if (rc) return rc;
    a.pos = reinterpret_cast<const float4 *>(pos_dev);
    a.order = h->lj_zorder ? reinterpret_cast<const int *>(h->vals[h->sorted].p) : nullptr;
    a.rows = reinterpret_cast<const int *>(h->rows.p);
    a.counts = reinterpret_cast<const int *>(h->counts.p);
    a.cap = h->cap;
    a.n = h->n;
    a.n_types = T;
    a.n_sys = h->n_sys;
    a.sys = reinterpret_cast<const SysInfo *>(h->sys.p);
    a.blk_sys = reinterpret_cast<const int *>(h->lj_blk_sys.p);
    a.blk_first = reinterpret_cast<const int *>(h->lj_blk_first.p);
    a.n_blocks = h->lj_n_blocks;
    a.tpp = h->lj_tpp;
    a.eps = eps_dev;
    a.sig = sig_dev;
    a.e = e_dev;
    a.F = F_dev;
    a.partials = reinterpret_cast<double *>(h->lj_partials.p);
    a.U = U_dev;
    a.dE = dE_dev;
    a.dS = dS_dev;
    a.sys_blk_start = reinterpret_cast<const int *>(h->lj_sys_blk.p);
    launch_lj_forward(a, stream);
    return cuda_status();
}

int qbvh_lj_backward(qbvh_handle h, const double *g_dev, const float *F_dev, const double *dE_dev,
                     const double *dS_dev, float *grad_pos_dev, float *grad_eps_dev, float *grad_sig_dev,
                     cudaStream_t stream)
{
    NvtxRange range("qbvh_lj_backward");
    if (!h) return QBVH_ERR_INVALID_ARG;
    if (!h->built) return QBVH_ERR_NOT_BUILT;
    if (!g_dev) return QBVH_ERR_INVALID_ARG;
    if (grad_pos_dev && !F_dev) return QBVH_ERR_INVALID_ARG;
    if (grad_eps_dev && !dE_dev) return QBVH_ERR_INVALID_ARG;
    if (grad_sig_dev && !dS_dev) return QBVH_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    launch_lj_backward(g_dev, F_dev, dE_dev, dS_dev, grad_pos_dev, grad_eps_dev, grad_sig_dev, h->n, h->n_sys,
                       h->n_types, reinterpret_cast<const SysInfo *>(h->sys.p),
                       reinterpret_cast<const int *>(h->sys_off.p), stream);
    return cuda_status();
}

int qbvh_selftest_wait_timeout(int device, cudaStream_t stream)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return QBVH_ERR_CUDA;
    }
    DeviceGuard g(device);
    unsigned *err = nullptr;
    if (cudaMallocHost(&err, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return QBVH_ERR_OOM;
    }
    *err = 0u;
    int rc = sort_wait_selftest(4096, err, stream) == 0 ? map_dev_err(*err) : QBVH_ERR_CUDA;
    cudaFreeHost(err);
    return rc;
}

int qbvh_pack_positions(const float *xyz_dev, const int *types_dev, int n, void *pos4_dev, cudaStream_t stream)
{
    if (n < 0) return QBVH_ERR_INVALID_ARG;
    if (n > 0 && (!xyz_dev || !pos4_dev || ((uintptr_t)pos4_dev & 15u))) return QBVH_ERR_INVALID_ARG;
    launch_pack(xyz_dev, types_dev, n, reinterpret_cast<float4 *>(pos4_dev), stream);
    return cuda_status();
}

}  // extern "C"
