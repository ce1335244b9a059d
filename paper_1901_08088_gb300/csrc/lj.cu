// Truncated-and-shifted Lennard-Jones energy over a neighbor list (Eq. 1 of
// the paper, shifted to zero at r_c as described in Sec. 1), in one fused pass
// that also produces the forces and the gradients with respect to the
// per-type-pair parameters:
//
//   s = (sig / r)^6,  s_c = (sig / r_c)^6
//   u(r)          = 4 eps (s^2 - s) - 4 eps (s_c^2 - s_c)           (r < r_c)
//   e_i           = 1/2 sum_{j in N(i)} u(r_ij)          (full list: each pair twice)
//   F_i           = sum_j 24 eps (2 s^2 - s) / r^2 (x_i - x_j)
//   dU/deps[a][b] = 1/2 sum_{i:a, j:b} u / eps
//   dU/dsig[a][b] = 1/2 sum_{i:a, j:b} (24 eps / sig) [(2 s^2 - s) - (2 s_c^2 - s_c)]
//
// Per-particle sums are FP32 in registers.  Each block covers particles of a
// single system and reduces its FP32 contributions in FP64 into one partial
// record; a second kernel adds the records of each system in a fixed order,
// so the FP64 totals are deterministic.
#include "qbvh_internal.cuh"

namespace qbvh {

namespace {

constexpr int kLJBlock = 128;
#ifndef QBVH_LJ_PARTICLES
#define QBVH_LJ_PARTICLES 256
#endif
constexpr int kLJParticles = QBVH_LJ_PARTICLES;   // particles per block, taken in rounds of kLJBlock / TPP

// Register cap of the one-type pass: 9 blocks of 128 threads (56 registers)
// keep it free of spills and measured 0.683 -> 0.668 ms at N = 2M; the
// passes with several types spill under that cap and keep the default.
#ifndef QBVH_LJ_MIN_BLOCKS_ONE
#define QBVH_LJ_MIN_BLOCKS_ONE 9
#endif
// row entries per load: 4 (16 bytes; 2 measured 0.74 -> 0.83 ms)
#ifndef QBVH_LJ_PREFETCH
#define QBVH_LJ_PREFETCH 1
#endif
#ifndef QBVH_LJ_VEC
#define QBVH_LJ_VEC 4
#endif
// TPP lanes share one particle: lane r of the group takes row entries
// r, r + TPP, ..., so that a group reads its row in contiguous chunks.
template <int T, int TPP>
__global__ void __launch_bounds__(kLJBlock, T == 1 ? QBVH_LJ_MIN_BLOCKS_ONE : 1)
lj_forward_kernel(const __grid_constant__ LJArgs a)
{
    constexpr int NP = 1 + 2 * T * T;
    __shared__ LJParams s_par[T * T];
    __shared__ double s_red[kLJBlock / 32][NP];
    const int tid = threadIdx.x;
    if (tid < T * T) s_par[tid] = lj_params(a.eps[tid], a.sig[tid], a.rc2[tid]);
    __syncthreads();
    const int sys = a.blk_sys[blockIdx.x];
    const SysInfo sy = a.sys[sys];
    const int sub = tid % TPP;
    const int end = min(a.blk_first[blockIdx.x] + kLJParticles, sy.offset + sy.count);
    double v[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) v[q] = 0.0;
    for (int base = a.blk_first[blockIdx.x]; base < end; base += kLJBlock / TPP) {
        // position in the walk order: Z-order when the tree's order is given, so
        // that a block's particles are close and their neighbours' positions are
        // shared in L1; systems occupy the same index range in both orders
        const int sidx = base + tid / TPP;
        const bool active = sidx < end;
        const int i = active ? (a.order ? __ldg(a.order + sidx) : sidx) : 0;
        float e = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        float gE[T], gS[T];
#pragma unroll
        for (int b = 0; b < T; ++b) gE[b] = gS[b] = 0.f;
        int ta = 0;
        if (active) {
            const float4 pi = __ldg(a.pos + i);
            ta = T > 1 ? __float_as_int(pi.w) : 0;
            ta = ta < 0 ? 0 : (ta >= T ? T - 1 : ta);
            const int c = min(__ldg(a.counts + i), a.cap);
            const int *row = a.rows + (size_t)i * a.cap;
            // each lane reads QBVH_LJ_VEC consecutive row entries with one
            // 16- or 8-byte load (rows are 16-byte aligned: the capacity is a
            // multiple of 4), then their positions, then does the arithmetic
            constexpr int V = QBVH_LJ_VEC;
            // with 4 entries per load the next chunk's entries are loaded one
            // iteration ahead (QBVH_LJ_PREFETCH), so that a row load is in
            // flight while the current chunk's positions are gathered
            int4 vnext = make_int4(-1, -1, -1, -1);
            if (QBVH_LJ_PREFETCH && V == 4 && V * sub < c)
                vnext = __ldg(reinterpret_cast<const int4 *>(row) + ((V * sub) >> 2));
            for (int k0 = V * sub; k0 < c; k0 += V * TPP) {
                int jj[V];
                if (V == 4) {
                    int4 v;
                    if (QBVH_LJ_PREFETCH) {
                        v = vnext;
                        const int kn = k0 + V * TPP;
                        if (kn < c) vnext = __ldg(reinterpret_cast<const int4 *>(row) + (kn >> 2));
                    } else {
                        v = __ldg(reinterpret_cast<const int4 *>(row) + (k0 >> 2));
                    }
                    jj[0] = v.x;
                    jj[V > 1 ? 1 : 0] = v.y;
                    jj[V > 2 ? 2 : 0] = v.z;
                    jj[V > 3 ? 3 : 0] = v.w;
                } else if (V == 2) {
                    const int2 v = __ldg(reinterpret_cast<const int2 *>(row) + (k0 >> 1));
                    jj[0] = v.x;
                    jj[V > 1 ? 1 : 0] = v.y;
                } else {
                    jj[0] = __ldg(row + k0);
                }
                float4 pp[V];
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    if (k0 + u >= c) jj[u] = -1;   // past the row end
                    if ((unsigned)jj[u] < (unsigned)a.n) pp[u] = __ldg(a.pos + jj[u]);
                }
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    if ((unsigned)jj[u] >= (unsigned)a.n) continue;
                    const float4 pj = pp[u];
                    int tb = T > 1 ? __float_as_int(pj.w) : 0;
                    tb = tb < 0 ? 0 : (tb >= T ? T - 1 : tb);
                    const int p = ta * T + tb;
                    const LJPairGeom gm = lj_pair_geom(pi, pj, sy.L, sy.Linv);
                    const LJParams &par = s_par[p];
                    if (!(gm.r2 < par.rc2)) continue;
                    const LJPairTerms t = lj_pair_terms<QBVH_LJ_FAST_RCP>(gm.vr2, par);
                    e += par.eps * t.uE;
                    fx -= t.w * gm.vx;
                    fy -= t.w * gm.vy;
                    fz -= t.w * gm.vz;
#pragma unroll
                    for (int b = 0; b < T; ++b) {
                        if (b == tb) {
                            gE[b] += t.uE;
                            gS[b] += t.gs;
                        }
                    }
                }
            }
        }
        // per-particle results: FP32 sums over the group's lanes
        float ei = e, fxi = fx, fyi = fy, fzi = fz;
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) {
            ei += __shfl_xor_sync(0xFFFFFFFFu, ei, o);
            fxi += __shfl_xor_sync(0xFFFFFFFFu, fxi, o);
            fyi += __shfl_xor_sync(0xFFFFFFFFu, fyi, o);
            fzi += __shfl_xor_sync(0xFFFFFFFFu, fzi, o);
        }
        if (active && sub == 0) {
            if (a.e) a.e[i] = 0.5f * ei;
            if (a.F) {
                a.F[3 * (size_t)i] = fxi;
                a.F[3 * (size_t)i + 1] = fyi;
                a.F[3 * (size_t)i + 2] = fzi;
            }
        }
        // FP64 accumulation of the energy and the parameter-gradient terms
        v[0] += 0.5 * (double)e;
        if (active) {
#pragma unroll
            for (int b = 0; b < T; ++b) {
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    if (t == ta) {
                        v[1 + t * T + b] += 0.5 * (double)gE[b];
                        v[1 + T * T + t * T + b] += 0.5 * (double)gS[b];
                    }
                }
            }
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) s_red[warp][q] = x;
    }
    __syncthreads();
    for (int q = tid; q < NP; q += kLJBlock) {
        double x = 0.0;
        for (int w = 0; w < kLJBlock / 32; ++w) x += s_red[w][q];
        a.partials[(size_t)blockIdx.x * NP + q] = x;
    }
}

// One block per system: fixed-order FP64 sum of the block records.  Thread
// t sums its own contiguous run of records in order (the loads of a run are
// independent, so they are in flight together), then a fixed-order tree
// adds the 1024 run sums: the same order on every call.
constexpr int kFinThreads = 1024;
// Without a block table (sys_blk_start == nullptr) one system owns records
// [0, n_blocks).
__global__ void __launch_bounds__(kFinThreads) lj_finalize_kernel(const double *partials, const int *sys_blk_start,
                                                                  int np, int T, double *U, double *dE, double *dS,
                                                                  int n_blocks = 0)
{
    __shared__ double s[kFinThreads];
    const int sys = blockIdx.x;
    const int t = threadIdx.x;
    const int b0 = sys_blk_start ? sys_blk_start[sys] : 0;
    const int b1 = sys_blk_start ? sys_blk_start[sys + 1] : n_blocks;
    const int run = (b1 - b0 + kFinThreads - 1) / kFinThreads;
    const int r0 = b0 + t * run, r1 = min(r0 + run, b1);
    for (int q = 0; q < np; ++q) {
        double x = 0.0;
#pragma unroll 8
        for (int b = r0; b < r1; ++b) x += partials[(size_t)b * np + q];
        s[t] = x;
        __syncthreads();
        for (int o = kFinThreads / 2; o > 0; o >>= 1) {
            if (t < o) s[t] += s[t + o];
            __syncthreads();
        }
        if (t == 0) {
            const double tot = s[0];
            if (q == 0) U[sys] = tot;
            else if (q <= T * T) { if (dE) dE[(size_t)sys * T * T + (q - 1)] = tot; }
            else if (dS) dS[(size_t)sys * T * T + (q - 1 - T * T)] = tot;
        }
        __syncthreads();
    }
}

__global__ void lj_backward_pos_kernel(const double *g, const float *F, float *gpos, int n, int n_sys,
                                       const int *sys_off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_sys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(sys_off + mid) <= i) lo = mid; else hi = mid - 1;
    }
    const float gs = (float)g[lo];
    for (int d = 0; d < 3; ++d) gpos[3 * (size_t)i + d] = -gs * F[3 * (size_t)i + d];
}

__global__ void lj_backward_param_kernel(const double *g, const double *dE, const double *dS, float *geps,
                                         float *gsig, int n_sys, int TT)
{
    const int q = threadIdx.x;
    if (q >= TT) return;
    double xe = 0.0, xs = 0.0;
    for (int k = 0; k < n_sys; ++k) {
        if (dE) xe += g[k] * dE[(size_t)k * TT + q];
        if (dS) xs += g[k] * dS[(size_t)k * TT + q];
    }
    if (geps) geps[q] = (float)xe;
    if (gsig) gsig[q] = (float)xs;
}

__global__ void pack_kernel(const float *xyz, const int *types, int n, float4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = types ? types[i] : 0;
    out[i] = make_float4(xyz[3 * (size_t)i], xyz[3 * (size_t)i + 1], xyz[3 * (size_t)i + 2], __int_as_float(t));
}

}  // namespace

int lj_particles_per_block() { return kLJParticles; }

template <int T>
static void launch_lj_t(const LJArgs &a, cudaStream_t s)
{
    switch (a.tpp) {
    case 1: lj_forward_kernel<T, 1><<<a.n_blocks, kLJBlock, 0, s>>>(a); break;
    case 2: lj_forward_kernel<T, 2><<<a.n_blocks, kLJBlock, 0, s>>>(a); break;
    case 4: lj_forward_kernel<T, 4><<<a.n_blocks, kLJBlock, 0, s>>>(a); break;
    case 8: lj_forward_kernel<T, 8><<<a.n_blocks, kLJBlock, 0, s>>>(a); break;
    case 16: lj_forward_kernel<T, 16><<<a.n_blocks, kLJBlock, 0, s>>>(a); break;
    default: lj_forward_kernel<T, 32><<<a.n_blocks, kLJBlock, 0, s>>>(a); break;
    }
}

void launch_lj_forward(const LJArgs &a, cudaStream_t s)
{
    if (a.n_blocks > 0) {
        switch (a.n_types) {
        case 1: launch_lj_t<1>(a, s); break;
        case 2: launch_lj_t<2>(a, s); break;
        case 3: launch_lj_t<3>(a, s); break;
        case 4: launch_lj_t<4>(a, s); break;
        case 5: launch_lj_t<5>(a, s); break;
        case 6: launch_lj_t<6>(a, s); break;
        case 7: launch_lj_t<7>(a, s); break;
        default: launch_lj_t<8>(a, s); break;
        }
    }
    const int T = a.n_types;
    lj_finalize_kernel<<<a.n_sys, kFinThreads, 0, s>>>(a.partials, a.sys_blk_start, 1 + 2 * T * T, T, a.U, a.dE, a.dS);
}

void launch_lj_finalize_one(const double *partials, int n_blocks, double *U, double *dE, double *dS,
                            cudaStream_t s)
{
    lj_finalize_kernel<<<1, kFinThreads, 0, s>>>(partials, nullptr, 3, 1, U, dE, dS, n_blocks);
}

void launch_lj_backward(const double *g, const float *F, const double *dE, const double *dS, float *gpos,
                        float *geps, float *gsig, int n, int n_sys, int n_types, const SysInfo *sys,
                        const int *sys_off, cudaStream_t s)
{
    (void)sys;
    if (gpos && F && n > 0) lj_backward_pos_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, F, gpos, n, n_sys, sys_off);
    if (geps || gsig) lj_backward_param_kernel<<<1, 64, 0, s>>>(g, dE, dS, geps, gsig, n_sys, n_types * n_types);
}

void launch_pack(const float *xyz, const int *types, int n, float4 *out, cudaStream_t s)
{
    if (n > 0) pack_kernel<<<(n + 255) / 256, 256, 0, s>>>(xyz, types, n, out);
}

}  // namespace qbvh
