// Stable LSD radix sort of (key, value) pairs, one kernel per 8-bit digit
// ("onesweep": every tile ranks its keys locally, then learns where its digit
// buckets start from the tiles before it through a decoupled look-back).
//
// The paper sorts the Morton codes with a library sort and notes that sorting
// is a large part of the build (Sec. 2.2, Sec. 3); it asks for a stable sort
// so that the particle order is deterministic (Sec. 3).
//
// Kernels:
//   hist  : one read of the keys, 256-bin histograms of every digit (the
//           build computes them in its Morton pass instead)
//   pass  : one per digit; tile 0 scans the digit histogram into global bucket
//           starts; tiles of keys are taken in ticket order, so a
//           tile only ever waits for tiles whose blocks are already running.
//           The wait is bounded: after kSpinLimit polls the block records
//           QBVH_DEVERR_TIMEOUT in the error word and continues (the result is
//           then wrong but every access stays in bounds).
#include "qbvh_internal.cuh"

namespace qbvh {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// keys per thread: 8 keeps 2048-key tiles, 27 KB of shared memory per block
// and twice the blocks of 16 items (the pass is latency-bound: more resident
// tiles hide more of the ranking and look-back latency)
#ifndef QBVH_SORT_ITEMS
#define QBVH_SORT_ITEMS 8
#endif
constexpr int kItems = QBVH_SORT_ITEMS;
constexpr int kTile = kThreads * kItems;
constexpr int kRadix = 256;
constexpr unsigned kFlagAgg = 1u << 30;
constexpr unsigned kFlagPre = 2u << 30;
constexpr unsigned kValMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 8;
constexpr int kSpinLimit = 1 << 20;
#ifndef QBVH_SORT_LOOKBACK
#define QBVH_SORT_LOOKBACK 8
#endif
// predecessor flags read per look-back round (build at N = 2M: 8 -> 0.38 ms,
// 16 -> 0.384 ms, 32 -> 0.395 ms)
constexpr int kLookBatch = QBVH_SORT_LOOKBACK;

__device__ __forceinline__ void st_relaxed(unsigned *p, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename K>
__global__ void __launch_bounds__(kThreads) hist_kernel(const K *__restrict__ keys, int n, int npass,
                                                        unsigned *__restrict__ hist)
{
    __shared__ unsigned sh[kMaxPasses * kRadix];
    for (int t = threadIdx.x; t < npass * kRadix; t += kThreads) sh[t] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const K k = keys[i];
        for (int p = 0; p < npass; ++p) atomicAdd(&sh[p * kRadix + ((unsigned)(k >> (8 * p)) & 255u)], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < npass * kRadix; t += kThreads)
        if (sh[t]) atomicAdd(hist + t, sh[t]);
}

// exclusive scan of 256 values held one per thread of a 256-thread block
__device__ __forceinline__ unsigned block_excl_scan256(unsigned v, unsigned *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    unsigned before = 0u;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    __syncthreads();
    return before + x - v;
}

template <typename K>
__global__ void __launch_bounds__(kThreads) pass_kernel(const K *__restrict__ kin, const int *__restrict__ vin,
                                                        K *__restrict__ kout, int *__restrict__ vout, int n,
                                                        int shift, const unsigned *__restrict__ bucket_base,
                                                        unsigned *status, unsigned *ticket, unsigned *err,
                                                        int spin_limit)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned *s_whist = reinterpret_cast<unsigned *>(smem);   // [kWarps][256]
    unsigned *s_dstart = s_whist + kWarps * kRadix;            // [256]
    unsigned *s_excl = s_dstart + kRadix;                      // [256]
    unsigned *s_misc = s_excl + kRadix;                        // [16]
    K *s_keys = reinterpret_cast<K *>(s_misc + 16);
    int *s_vals = reinterpret_cast<int *>(s_keys + kTile);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < kWarps * kRadix; t += kThreads) s_whist[t] = 0u;
    if (tid == 0) s_misc[0] = atomicAdd(ticket, 1u);
    __syncthreads();
    const int tile = (int)s_misc[0];
    const int base = tile * kTile + warp * (32 * kItems);
    // tile 0 turns the pass's digit histogram into global bucket starts
    unsigned bucket_start = 0u;
    if (tile == 0) bucket_start = block_excl_scan256(bucket_base[tid], s_misc + 1);

    K key[kItems];
    int val[kItems];
    unsigned rank[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int idx = base + it * 32 + lane;
        const bool ok = idx < n;
        key[it] = ok ? kin[idx] : ~K(0);   // out-of-range items rank last, digit 255
        val[it] = ok ? (vin ? vin[idx] : idx) : 0;
    }
    // warp-local stable ranking, row by row
    const unsigned lt = lanemask_lt();
    unsigned *wh = s_whist + warp * kRadix;
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const unsigned d = (unsigned)(key[it] >> shift) & 255u;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const unsigned prev = wh[d];
        __syncwarp();
        const unsigned r = __popc(peers & lt);
        if (r == 0) wh[d] = prev + __popc(peers);
        __syncwarp();
        rank[it] = prev + r;
    }
    __syncthreads();

    // per digit: offsets of the warps, the tile's count, and its global start
    unsigned cnt = 0u;
    {
        const int d = tid;   // kThreads == kRadix
        for (int w = 0; w < kWarps; ++w) {
            const unsigned c = s_whist[w * kRadix + d];
            s_whist[w * kRadix + d] = cnt;
            cnt += c;
        }
        unsigned *mine = status + (size_t)tile * kRadix + d;
        unsigned excl;
        if (tile == 0) {
            excl = bucket_start;   // this digit's global start
            st_relaxed(mine, kFlagPre | (excl + cnt));
        } else {
            st_relaxed(mine, kFlagAgg | cnt);
            excl = 0u;
            int j = tile - 1;
            int spins = 0;
            bool done = false;
            // predecessors are read kLookBatch at a time (independent loads)
            // and consumed newest first: aggregates add up until an inclusive
            // prefix ends the walk; an unpublished slot is polled again
            while (!done) {
                unsigned v[kLookBatch];
#pragma unroll
                for (int b = 0; b < kLookBatch; ++b)
                    v[b] = (j - b >= 0) ? ld_relaxed(status + (size_t)(j - b) * kRadix + d) : kFlagPre;
#pragma unroll
                for (int b = 0; b < kLookBatch; ++b) {
                    if (done) break;
                    const unsigned f = v[b] & ~kValMask;
                    if (f == 0u) break;           // not yet published: poll from here
                    excl += v[b] & kValMask;      // kFlagPre past tile 0 carries value 0
                    --j;
                    if (f == kFlagPre || j < 0) done = true;
                }
                if (done) break;
                const unsigned f0 = ld_relaxed(status + (size_t)j * kRadix + d) & ~kValMask;
                if (f0 == 0u) {
                    if (++spins > spin_limit) {
                        atomicOr(err, QBVH_DEVERR_TIMEOUT);
                        break;
                    }
                    if (spins > 64) __nanosleep(100);
                }
            }
            st_relaxed(mine, kFlagPre | ((excl + cnt) & kValMask));
        }
        s_excl[d] = excl;
    }
    const unsigned dstart = block_excl_scan256(cnt, s_misc + 1);
    s_dstart[tid] = dstart;
    __syncthreads();

    // scatter into shared memory in digit order
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const unsigned d = (unsigned)(key[it] >> shift) & 255u;
        const unsigned pos = s_dstart[d] + s_whist[warp * kRadix + d] + rank[it];
        s_keys[pos] = key[it];
        s_vals[pos] = val[it];
    }
    __syncthreads();
    // coalesced write-out: consecutive positions of a bucket go to consecutive addresses
    const int valid = min(kTile, n - tile * kTile);
    for (int p = tid; p < valid; p += kThreads) {
        const K k = s_keys[p];
        const unsigned d = (unsigned)(k >> shift) & 255u;
        const unsigned g = s_excl[d] + ((unsigned)p - s_dstart[d]);
        if (g < (unsigned)n) {
            kout[g] = k;
            vout[g] = s_vals[p];
        }
    }
}

template <typename K>
size_t pass_smem()
{
    return sizeof(unsigned) * (kWarps * kRadix + 2 * kRadix + 16) + (sizeof(K) + sizeof(int)) * kTile;
}

template <typename K>
int sort_impl(K *ka, K *kb, int *va, int *vb, int n, int bits, void *scratch, unsigned *err, bool prepared,
              cudaStream_t s)
{
    const int npass = (bits + 7) / 8;
    const int tiles = sort_num_tiles(n);
    unsigned *hist = reinterpret_cast<unsigned *>(scratch);
    unsigned *ticket = hist + kMaxPasses * kRadix;
    unsigned *status = ticket + kMaxPasses * 4;
    if (!prepared) {
        // zeroed scratch and digit histograms, unless the caller's kernels made them
        cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n, npass), s);
        int hb = (n + kThreads * 8 - 1) / (kThreads * 8);
        hb = hb < 1 ? 1 : (hb > 1216 ? 1216 : hb);
        hist_kernel<K><<<hb, kThreads, 0, s>>>(ka, n, npass, hist);
    }
    static bool attr_set = false;
    const size_t smem = pass_smem<K>();
    if (!attr_set) {
        cudaFuncSetAttribute(pass_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    K *src_k = ka, *dst_k = kb;
    int *src_v = nullptr, *dst_v = vb;
    int *v_first_dst = vb;
    (void)v_first_dst;
    for (int p = 0; p < npass; ++p) {
        pass_kernel<K><<<tiles, kThreads, smem, s>>>(src_k, src_v, dst_k, dst_v, n, 8 * p, hist + p * kRadix,
                                                     status + (size_t)p * tiles * kRadix, ticket + p * 4, err,
                                                     kSpinLimit);
        // ping-pong
        K *tk = src_k;
        src_k = dst_k;
        dst_k = tk;
        int *tv = src_v;
        src_v = dst_v;
        dst_v = (tv == nullptr) ? va : tv;
    }
    return (src_k == ka) ? 0 : 1;
}

}  // namespace

size_t sort_tile_items() { return kTile; }

int sort_num_tiles(int n) { return n <= 0 ? 1 : (n + kTile - 1) / kTile; }

size_t sort_scratch_bytes(int n, int passes)
{
    return sizeof(unsigned) * ((size_t)kMaxPasses * kRadix + kMaxPasses * 4 +
                               (size_t)passes * sort_num_tiles(n) * kRadix);
}

// One tile (tile 1) of a pass whose predecessor (tile 0) never publishes: the
// look-back gives up after `spin_limit` polls and records QBVH_DEVERR_TIMEOUT.
// Every access stays inside the 2-tile buffers.  Returns the device error word.
int sort_wait_selftest(int spin_limit, unsigned *err_out, cudaStream_t s)
{
    const int n = 2 * kTile;
    unsigned *kin = nullptr, *kout = nullptr, *misc = nullptr;
    int *vout = nullptr;
    const size_t misc_words = kRadix + 4 + 2 * kRadix + 1;   // bucket base, ticket, status of 2 tiles, err
    if (cudaMalloc(&kin, n * sizeof(unsigned)) != cudaSuccess || cudaMalloc(&kout, n * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&vout, n * sizeof(int)) != cudaSuccess || cudaMalloc(&misc, misc_words * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(kin);
        cudaFree(kout);
        cudaFree(vout);
        cudaFree(misc);
        return -1;
    }
    unsigned *base = misc, *ticket = misc + kRadix, *status = misc + kRadix + 4, *err = status + 2 * kRadix;
    cudaMemsetAsync(kin, 0, n * sizeof(unsigned), s);
    cudaMemsetAsync(misc, 0, misc_words * sizeof(unsigned), s);
    const unsigned one = 1u;
    cudaMemcpyAsync(ticket, &one, sizeof one, cudaMemcpyHostToDevice, s);   // the block takes tile 1
    const size_t smem = pass_smem<unsigned>();
    cudaFuncSetAttribute(pass_kernel<unsigned>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pass_kernel<unsigned><<<1, kThreads, smem, s>>>(kin, nullptr, kout, vout, n, 0, base, status, ticket, err,
                                                    spin_limit);   // tile 1: never scans
    cudaMemcpyAsync(err_out, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(kin);
    cudaFree(kout);
    cudaFree(vout);
    cudaFree(misc);
    return e == cudaSuccess ? 0 : -1;
}

int radix_sort_pairs(bool wide, void *keys_a, void *keys_b, int *vals_a, int *vals_b, int n, int bits,
                     void *scratch, unsigned *err, cudaStream_t s, bool prepared)
{
    if (n <= 0) return 0;
    if (wide)
        return sort_impl<unsigned long long>(reinterpret_cast<unsigned long long *>(keys_a),
                                             reinterpret_cast<unsigned long long *>(keys_b), vals_a, vals_b, n,
                                             bits, scratch, err, prepared, s);
    return sort_impl<unsigned>(reinterpret_cast<unsigned *>(keys_a), reinterpret_cast<unsigned *>(keys_b), vals_a,
                               vals_b, n, bits, scratch, err, prepared, s);
}

}  // namespace qbvh
