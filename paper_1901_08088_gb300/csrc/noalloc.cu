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
// for the deterministic energy/gradient sums, and one error word -- lives in
// the fixed scratch variable below.
//
// The scratch is a file-scope __device__ variable, so every GPU that loads
// this library holds it (kBlocks * kMaxRecord doubles plus one word, about
// 321 KB) until the process exits.  In host code its name stands for a host
// copy, not for device memory, so the kernels get the device address looked
// up with cudaGetSymbolAddress.  That lookup runs once per device and CUDA
// context, on the first call that finds the device's current context new
// (see qbvh.h).  Every call rewrites every record it reads and clears the
// error word on its stream before its kernels run; calls that overlap on the
// GPU (different streams, or several host threads) share the scratch and race.
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

// error bits of one call
constexpr unsigned kErrBadType = 1u;    // a particle type outside [0, n_types)
constexpr unsigned kErrBadIndex = 2u;   // a row entry outside [0, n)

struct Scratch {
    double records[kBlocks * kMaxRecord];   // per block: energy, dU/deps[T][T], dU/dsig[T][T]
    unsigned err;                           // error bits, cleared by every call
};

static __device__ __align__(256) Scratch g_noalloc_scratch;

// Device address of the scratch, per device, valid for the CUDA context it
// was looked up in.
struct Cached {
    unsigned long long ctx_id = 0;
    Scratch *ptr = nullptr;
};
std::mutex g_mu;
Cached g_cache[kMaxDevices];

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Identity of the current CUDA context (0 when the driver cannot tell): a
// device reset gives the device a new context, where the variable may sit at
// another address, so the cache is keyed on it.
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch on the current device.  Called with that
// device current; looks the address up again whenever the device's context
// changed since the last lookup (or cannot be identified).
int scratch_on_device(int dev, Scratch **out)
{
    if (dev < 0 || dev >= kMaxDevices) return QBVH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long ctx = current_context_id();
    Cached &c = g_cache[dev];
    if (!c.ptr || ctx == 0 || c.ctx_id != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            c.ptr = nullptr;
            return QBVH_ERR_CUDA;
        }
        c.ptr = reinterpret_cast<Scratch *>(p);
        c.ctx_id = ctx;
    }
    *out = c.ptr;
    return QBVH_OK;
}

// squared cutoffs fl(r_cut * r_cut), passed by value
struct Rc2 {
    float v[kMaxTypes * kMaxTypes];
};

// Grid-stride over particles; each block folds its particles' contributions
// into its own FP64 record, so the record count is fixed by the grid.  A
// particle whose type lies outside [0, T) contributes nothing (its outputs
// are zero), and neither does a pair whose partner has such a type or whose
// row entry lies outside [0, n); each case sets its error bit.
template <int T>
__global__ void __launch_bounds__(kThreads) lj_noalloc_kernel(const float4 *__restrict__ pos, int n, float L,
                                                              float Linv, const int *__restrict__ rows,
                                                              const int *__restrict__ counts, int cap,
                                                              const float *eps, const float *sig, const Rc2 rc2_in,
                                                              float *e_out, float *F_out, Scratch *scratch)
{
    constexpr int NP = 1 + 2 * T * T;
    __shared__ qbvh::LJParams s_par[T * T];
    __shared__ double s_red[kThreads / 32][NP];
    const int tid = threadIdx.x;
    if (tid < T * T) s_par[tid] = qbvh::lj_params(eps[tid], sig[tid], rc2_in.v[tid]);
    __syncthreads();
    const int sub = tid % kLanes;
    const int per_block = kThreads / kLanes;
    unsigned err = 0u;
    double v[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) v[q] = 0.0;
    for (int base = blockIdx.x * per_block; base < n; base += gridDim.x * per_block) {
        const int i = base + tid / kLanes;
        float e = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        float gE[T], gS[T];
#pragma unroll
        for (int b = 0; b < T; ++b) gE[b] = gS[b] = 0.f;
        int ta = 0;
        bool active = i < n;
        if (active) {
            const float4 pi = __ldg(pos + i);
            ta = T > 1 ? __float_as_int(pi.w) : 0;
            if ((unsigned)ta >= (unsigned)T) {
                err |= kErrBadType;
                active = false;
            }
            const int c = active ? min(__ldg(counts + i), cap) : 0;
            const int *row = rows + (size_t)i * cap;
            for (int k = sub; k < c; k += kLanes) {
                const int j = __ldg(row + k);
                if ((unsigned)j >= (unsigned)n) {
                    err |= kErrBadIndex;
                    continue;
                }
                const float4 pj = __ldg(pos + j);
                const int tb = T > 1 ? __float_as_int(pj.w) : 0;
                if ((unsigned)tb >= (unsigned)T) {
                    err |= kErrBadType;
                    continue;
                }
                const qbvh::LJParams &par = s_par[ta * T + tb];
                const qbvh::LJPairGeom gm = qbvh::lj_pair_geom(pi, pj, L, Linv);
                if (!(gm.r2 < par.rc2)) continue;
                const qbvh::LJPairTerms t = qbvh::lj_pair_terms<QBVH_LJ_FAST_RCP>(gm.vr2, par);
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
        float ei = e, fxi = fx, fyi = fy, fzi = fz;
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) {
            ei += __shfl_xor_sync(0xFFFFFFFFu, ei, o);
            fxi += __shfl_xor_sync(0xFFFFFFFFu, fxi, o);
            fyi += __shfl_xor_sync(0xFFFFFFFFu, fyi, o);
            fzi += __shfl_xor_sync(0xFFFFFFFFu, fzi, o);
        }
        if (i < n && sub == 0) {
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
    err = __reduce_or_sync(0xFFFFFFFFu, err);
    if (lane == 0 && err) atomicOr(&scratch->err, err);
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
        scratch->records[(size_t)blockIdx.x * NP + q] = x;
    }
}

// One block: fixed-order FP64 sum of the kBlocks records, and the call's
// status (an error also makes the energy NaN, so that it cannot pass for a
// valid total).
__global__ void lj_noalloc_finalize(const Scratch *scratch, int np, int T, double *U, double *dE, double *dS,
                                    int *status)
{
    __shared__ double s[256];
    const unsigned err = scratch->err;
    for (int q = 0; q < np; ++q) {
        double x = 0.0;
        for (int b = threadIdx.x; b < kBlocks; b += blockDim.x) x += scratch->records[(size_t)b * np + q];
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double tot = s[0];
            if (q == 0) U[0] = err ? __longlong_as_double(0x7FF8000000000000LL) : tot;
            else if (q <= T * T) { if (dE) dE[q - 1] = tot; }
            else if (dS) dS[q - 1 - T * T] = tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        status[0] = (err & kErrBadType) ? QBVH_ERR_BAD_TYPE : ((err & kErrBadIndex) ? QBVH_ERR_INTERNAL : QBVH_OK);
}

template <int T>
void launch(const float4 *pos, int n, float L, float Linv, const int *rows, const int *counts, int cap,
            const float *eps, const float *sig, const Rc2 &rc2, float *e, float *F, Scratch *scratch, double *U,
            double *dE, double *dS, int *status, cudaStream_t s)
{
    lj_noalloc_kernel<T><<<kBlocks, kThreads, 0, s>>>(pos, n, L, Linv, rows, counts, cap, eps, sig, rc2, e, F,
                                                       scratch);
    lj_noalloc_finalize<<<1, 256, 0, s>>>(scratch, 1 + 2 * T * T, T, U, dE, dS, status);
}

}  // namespace

extern "C" int qbvh_lj_forward_noalloc(const void *pos_dev, int n, float L, int n_types, const int *rows_dev,
                                       const int *counts_dev, int cap, const float *eps_dev, const float *sig_dev,
                                       const float *r_cut_host, float *e_dev, double *U_dev, float *F_dev,
                                       double *dE_dev, double *dS_dev, int *status_dev, cudaStream_t stream)
{
    if (n_types < 1 || n_types > kMaxTypes) return QBVH_ERR_INVALID_ARG;   // beyond the fixed records
    if (n < 0 || n >= (1 << 30) || cap < 1 || !(L > 0.f) || !isfinite(L)) return QBVH_ERR_INVALID_ARG;
    if (!eps_dev || !sig_dev || !r_cut_host || !U_dev || !status_dev) return QBVH_ERR_INVALID_ARG;
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
    Scratch *scratch = nullptr;
    int rc = scratch_on_device(dev, &scratch);
    if (rc) return rc;
    // the error word must start at zero; the records are all rewritten
    if (cudaMemsetAsync(&scratch->err, 0, sizeof(unsigned), stream) != cudaSuccess) {
        cudaGetLastError();
        return QBVH_ERR_CUDA;
    }
    const float Linv = 1.0f / L;
    const float4 *pos = reinterpret_cast<const float4 *>(pos_dev);
    switch (n_types) {
    case 1: launch<1>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, scratch,
                      U_dev, dE_dev, dS_dev, status_dev, stream); break;
    case 2: launch<2>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, scratch,
                      U_dev, dE_dev, dS_dev, status_dev, stream); break;
    case 3: launch<3>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, scratch,
                      U_dev, dE_dev, dS_dev, status_dev, stream); break;
    default: launch<4>(pos, n, L, Linv, rows_dev, counts_dev, cap, eps_dev, sig_dev, rc2, e_dev, F_dev, scratch,
                       U_dev, dE_dev, dS_dev, status_dev, stream); break;
    }
    return cudaGetLastError() == cudaSuccess ? QBVH_OK : QBVH_ERR_CUDA;
}
