// Allocation-free Lennard-Jones pass: qbvh_lj_forward_noalloc (include/qbvh.h).
//
// Some callers cannot allocate GPU memory at the point where they need forces:
// code running under a memory pool or an allocator that is locked for the
// duration of a step, plugins embedded in a host program that owns every
// device allocation, or real-time loops where cudaMalloc/cudaFree (which can
// synchronize the device) are not allowed.  This entry point computes the same
// energies, forces and parameter gradients as qbvh_lj_forward for one periodic
// system and a caller-provided neighbor list, and allocates nothing: the only
// memory it needs besides its inputs and outputs -- one FP64 record per block
// for the deterministic energy/gradient sums -- lives in the fixed array below.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it (kBlocks * kMaxRecord doubles, about 321 KB) until the
// process exits.  Its device address is looked up once per device with
// cudaGetSymbolAddress, on that device's first call (see qbvh.h).  Every call
// overwrites every record it reads, so nothing has to be cleared between
// calls; calls that overlap on the GPU (different streams, or several host
// threads) share the array and race.
#include <mutex>

#include "../../include/qbvh.h"
#include "qbvh_internal.cuh"

namespace {

constexpr int kBlocks = 1216;      // fixed grid: 8 blocks on each of 152 SMs
constexpr int kThreads = 128;
constexpr int kLanes = 4;          // lanes sharing one particle's row
constexpr int kMaxTypes = 4;
constexpr int kMaxRecord = 1 + 2 * kMaxTypes * kMaxTypes;
constexpr int kMaxDevices = 64;

// per-block FP64 records: energy, dU/deps[T][T], dU/dsig[T][T]
static __device__ __align__(256) double g_lj_records[kBlocks * kMaxRecord];

std::mutex g_mu;
double *g_records[kMaxDevices] = {};

// squared cutoffs fl(r_cut * r_cut), passed by value
struct Rc2 {
    float v[kMaxTypes * kMaxTypes];
};

__device__ __forceinline__ float min_image(float d, float L, float Linv)
{
    return __fsub_rn(d, __fmul_rn(L, rintf(__fmul_rn(d, Linv))));
}

// Grid-stride over particles; each block folds its particles' contributions
// into its own FP64 record, so the record count is fixed by the grid.
template <int T>
__global__ void __launch_bounds__(kThreads) lj_noalloc_kernel(const float4 *__restrict__ pos, int n, float L,
                                                              float Linv, const int *__restrict__ rows,
                                                              const int *__restrict__ counts, int cap,
                                                              const float *eps, const float *sig, const Rc2 rc2_in,
                                                              float *e_out, float *F_out, double *records)
{
    constexpr int NP = 1 + 2 * T * T;
    __shared__ float s_eps[T * T], s_sig[T * T], s_sig2[T * T], s_phic[T * T], s_dsc[T * T], s_rc2[T * T];
    __shared__ double s_red[kThreads / 32][NP];
    const int tid = threadIdx.x;
    if (tid < T * T) {
        const float ep = eps[tid], sg = sig[tid], rc2 = rc2_in.v[tid];
        s_eps[tid] = ep;
        s_sig[tid] = sg;
        s_sig2[tid] = sg * sg;
        s_rc2[tid] = rc2;
        const float sc2 = (sg * sg) / rc2;
        const float sc6 = sc2 * sc2 * sc2;
        s_phic[tid] = 4.f * (sc6 * sc6 - sc6);
        s_dsc[tid] = 2.f * sc6 * sc6 - sc6;
    }
    __syncthreads();
    const int sub = tid % kLanes;
    const int per_block = kThreads / kLanes;
    double v[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) v[q] = 0.0;
    for (int base = blockIdx.x * per_block; base < n; base += gridDim.x * per_block) {
        const int i = base + tid / kLanes;
        const bool active = i < n;
        float e = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        float gE[T], gS[T];
#pragma unroll
        for (int b = 0; b < T; ++b) gE[b] = gS[b] = 0.f;
        int ta = 0;
        if (active) {
            const float4 pi = __ldg(pos + i);
            ta = T > 1 ? __float_as_int(pi.w) : 0;
            ta = ta < 0 ? 0 : (ta >= T ? T - 1 : ta);
            const int c = min(__ldg(counts + i), cap);
            const int *row = rows + (size_t)i * cap;
            for (int k = sub; k < c; k += kLanes) {
                const int j = __ldg(row + k);
                if ((unsigned)j >= (unsigned)n) continue;
                const float4 pj = __ldg(pos + j);
                int tb = T > 1 ? __float_as_int(pj.w) : 0;
                tb = tb < 0 ? 0 : (tb >= T ? T - 1 : tb);
                const int p = ta * T + tb;
                const float dx = min_image(__fsub_rn(pj.x, pi.x), L, Linv);
                const float dy = min_image(__fsub_rn(pj.y, pi.y), L, Linv);
                const float dz = min_image(__fsub_rn(pj.z, pi.z), L, Linv);
                const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                if (!(r2 < s_rc2[p])) continue;
                const float inv_r2 = __frcp_rn(r2);
                const float s2 = s_sig2[p] * inv_r2;
                const float s6 = s2 * s2 * s2;
                const float uE = 4.f * (s6 * s6 - s6) - s_phic[p];
                const float q = 2.f * s6 * s6 - s6;
                const float w = 24.f * s_eps[p] * q * inv_r2;
                e += s_eps[p] * uE;
                fx -= w * dx;
                fy -= w * dy;
                fz -= w * dz;
#pragma unroll
                for (int b = 0; b < T; ++b) {
                    if (b == tb) {
                        gE[b] += uE;
                        gS[b] += (24.f * s_eps[p] / s_sig[p]) * (q - s_dsc[p]);
                    }
                }
            }
        }
        float ei = e, fxi = fx, fyi = fy, fzi = fz;
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) {
            ei += __shfl_xor_sync(0xFFFFFFFFu, ei, o);
            fxi += __shfl_xor_sync(0xFFFFFFFFu, fxi, o);
            fyi += __shfl_xor_sync(0xFFFFFFFFu, fyi, o);
            fzi += __shfl_xor_sync(0xFFFFFFFFu, fzi, o);
        }
        if (active && sub == 0) {
            if (e_out) e_out[i] = 0.5f * ei;
            if (F_out) {
                F_out[3 * (size_t)i] = fxi;
                F_out[3 * (size_t)i + 1] = fyi;
                F_out[3 * (size_t)i + 2] = fzi;
            }
        }
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
    // every block writes its whole record, also when it had no particles
    for (int q = tid; q < NP; q += kThreads) {
        double x = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) x += s_red[w][q];
        records[(size_t)blockIdx.x * NP + q] = x;
    }
}

// One block: fixed-order FP64 sum of the kBlocks records.
__global__ void lj_noalloc_finalize(const double *records, int np, int T, double *U, double *dE, double *dS)
{
    __shared__ double s[256];
    for (int q = 0; q < np; ++q) {
        double x = 0.0;
        for (int b = threadIdx.x; b < kBlocks; b += blockDim.x) x += records[(size_t)b * np + q];
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double tot = s[0];
            if (q == 0) U[0] = tot;
            else if (q <= T * T) { if (dE) dE[q - 1] = tot; }
            else if (dS) dS[q - 1 - T * T] = tot;
        }
        __syncthreads();
    }
}

// Device address of the record array on the current device, looked up once.
int records_on_device(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return QBVH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_records[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lj_records) != cudaSuccess || !p) {
            cudaGetLastError();
            return QBVH_ERR_CUDA;
        }
        g_records[dev] = reinterpret_cast<double *>(p);
    }
    *out = g_records[dev];
    return QBVH_OK;
}

template <int T>
void launch(const float4 *pos, int n, float L, float Linv, const int *rows, const int *counts, int cap,
            const float *eps, const float *sig, const Rc2 &rc2, float *e, float *F, double *rec, double *U,
            double *dE, double *dS, cudaStream_t s)
{
    lj_noalloc_kernel<T><<<kBlocks, kThreads, 0, s>>>(pos, n, L, Linv, rows, counts, cap, eps, sig, rc2, e, F, rec);
    lj_noalloc_finalize<<<1, 256, 0, s>>>(rec, 1 + 2 * T * T, T, U, dE, dS);
}

}  // namespace

extern "C" int qbvh_lj_forward_noalloc(const void *pos_dev, int n, float L, int n_types, const int *rows_dev,
                                       const int *counts_dev, int cap, const float *eps_dev, const float *sig_dev,
                                       const float *r_cut_host, float *e_dev, double *U_dev, float *F_dev,
                                       double *dE_dev, double *dS_dev, cudaStream_t stream)
{
    if (n_types < 1 || n_types > kMaxTypes) return QBVH_ERR_INVALID_ARG;   // beyond the fixed records
    if (n < 0 || n >= (1 << 30) || cap < 1 || !(L > 0.f) || !isfinite(L)) return QBVH_ERR_INVALID_ARG;
    if (!eps_dev || !sig_dev || !r_cut_host || !U_dev) return QBVH_ERR_INVALID_ARG;
    Rc2 rc2;
    for (int p = 0; p < kMaxTypes * kMaxTypes; ++p) rc2.v[p] = 0.f;
    for (int p = 0; p < n_types * n_types; ++p) {
        const float rc = r_cut_host[p];
        if (!(rc > 0.f) || !isfinite(rc)) return QBVH_ERR_INVALID_ARG;
        rc2.v[p] = rc * rc;
    }
    if (n > 0 && (!pos_dev || ((uintptr_t)pos_dev & 15u) || !rows_dev || !counts_dev)) return QBVH_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QBVH_ERR_CUDA;
    }
    double *rec = nullptr;
    int rc = records_on_device(dev, &rec);
    if (rc) return rc;
    const float Linv = 1.0f / L;
    const float4 *pos = reinterpret_cast<const float4 *>(pos_dev);
    switch (n_types) {
    case 1: launch<1>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, rec,
                      U_dev, dE_dev, dS_dev, stream); break;
    case 2: launch<2>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, rec,
                      U_dev, dE_dev, dS_dev, stream); break;
    case 3: launch<3>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, rec,
                      U_dev, dE_dev, dS_dev, stream); break;
    default: launch<4>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, rec,
                       U_dev, dE_dev, dS_dev, stream); break;
    }
    return cudaGetLastError() == cudaSuccess ? QBVH_OK : QBVH_ERR_CUDA;
}
