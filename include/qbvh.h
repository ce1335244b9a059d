/*
 * qbvh -- neighbor lists through a linear bounding volume hierarchy with
 * quantized node bounds, for one NVIDIA GB300 (sm_103a).
 *
 * Method: Howard, Statt, Madutsa, Truskett, Panagiotopoulos, "Quantized
 * bounding volume hierarchies for neighbor search in molecular simulations on
 * graphics processing units" (arXiv:1901.08088).
 *
 * The problem this library solves is the paper's (Sec. 1, Fig. 1a; Sec. 4):
 * given particle positions in a periodic cubic box, a particle type per
 * particle and a list radius per type pair, find for every particle i all
 * particles j != i closer than the list radius, and store them as a Verlet
 * (neighbor) list.  The list is exact: the distance of every pair found by
 * the tree traversal is re-tested with one fixed FP32 expression,
 *
 *     dx = xj - xi;  dx = dx - L * rint(dx * Linv);      (same for y and z)
 *     d2 = (dx*dx + dy*dy) + dz*dz;    j in N(i)  iff  d2 < r*r,
 *
 * with Linv = 1.0f / L and r*r rounded once in FP32, so the list is
 * bit-identical to a brute-force search with that expression.
 *
 * Conventions for every entry point
 *   - Return value: QBVH_OK (0) or one of the QBVH_ERR_* codes below.
 *   - Pointers named *_dev are device pointers on the handle's device; *_host
 *     are host pointers read before the call returns.
 *   - All GPU work is enqueued on `stream` (0 = legacy default stream) and is
 *     asynchronous unless stated otherwise.  The caller keeps every input
 *     device buffer alive, unmodified, until that work has completed.
 *   - Buffers returned by the library (nlist_get, qbvh_tree_get) belong to the
 *     handle and stay valid until the next build/query/destroy on that handle.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - Counts: 0 <= n < 2^30 particles, 1 <= n_types <= 8 types.
 */
#ifndef QBVH_H
#define QBVH_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define QBVH_OK 0
#define QBVH_ERR_INVALID_ARG 1      /* bad pointer, size, alignment or option      */
#define QBVH_ERR_OUT_OF_BOX 2       /* a position is outside [0, L) or not finite  */
#define QBVH_ERR_BAD_TYPE 3         /* a particle type is outside [0, n_types)     */
#define QBVH_ERR_CUTOFF_TOO_LARGE 4 /* list radius >= L/2 for some system          */
#define QBVH_ERR_OVERFLOW 5         /* a row still exceeded its capacity after the
                                       allowed retries; counts are complete,
                                       rows are truncated at cap                    */
#define QBVH_ERR_DEVICE_TIMEOUT 6   /* a bounded device-side wait gave up          */
#define QBVH_ERR_CUDA 7             /* a CUDA runtime call failed                  */
#define QBVH_ERR_OOM 8              /* device or pinned allocation failed          */
#define QBVH_ERR_NOT_BUILT 9        /* query/get before a successful build         */
#define QBVH_ERR_INTERNAL 10        /* a device-side consistency check failed (an
                                       index out of range or a walk longer than
                                       the tree); the access was skipped          */

/* Largest number of particle types a handle accepts. */
#define QBVH_MAX_TYPES 8

/* Opaque handle: owns the tree, the neighbor list and all scratch memory. */
typedef struct qbvh_ctx *qbvh_handle;

/* Human-readable name of a status code (static string, never NULL). */
const char *qbvh_strerror(int code);

/*
 * Create a handle bound to CUDA device `device`.  Allocates only a few bytes
 * of pinned host memory; device buffers are allocated by the first build and
 * grown when a later call needs more.
 * Errors: INVALID_ARG (out == NULL), CUDA (no such device), OOM.
 */
int qbvh_create(qbvh_handle *out, int device);

/* Release every buffer of the handle.  Synchronizes the handle's device. */
int qbvh_destroy(qbvh_handle h);

/* ---- tuning options (qbvh_set_option) ---------------------------------- */
/* Subtree collapse (Sec. 2.3, final paragraph): internal nodes with at most K
 * leaves are traversed by testing their leaves directly.  K = 1 keeps the
 * paper's one-particle leaves.  Values 1..64, default 16.  Takes effect at
 * the next build. */
#define QBVH_OPT_BUNDLE 1
/* Threads per block of the traversal kernel: 32..256, multiple of 32,
 * default 128 (the warp walk is compiled for at most 256 threads per block
 * so that 8 blocks fit on an SM).  Takes effect at the next query. */
#define QBVH_OPT_QUERY_BLOCK 2
/* 1 = skip the exact leaf test and list every particle whose node the search
 * sphere overlaps, as Alg. 1 does (candidates, false positives included).
 * 0 (default) = exact list. */
#define QBVH_OPT_CANDIDATES 3
/* Traversal mapping: 0 = one thread per particle (Alg. 1 as written);
 * 1 (default) = one warp per 32 consecutive Z-order particles walking the
 * tree together (same rope walk, warp-uniform control flow, each lane testing
 * its own sphere).  Both give the same list.  Takes effect at the next query. */
#define QBVH_OPT_TRAVERSAL 4
/* Node storage: 0 (default) = 16-byte nodes with 10-bit quantized bounds
 * (Fig. 3b); 1 = 32-byte nodes with exact FP32 bounds (Fig. 3a); 2 = 32-byte
 * nodes with bounds quantized to 21 bits per axis (2^21 - 1 bins on the root
 * box, the wider bit width Sec. 2.2 weighs against false positives).  All
 * give the same list; in candidate mode (QBVH_OPT_CANDIDATES) the leaves are
 * tested at the format's precision (10-bit box, FP32 point, 21-bit box), so
 * the false positives differ.  qbvh_tree_get returns the 10-bit nodes, which
 * every build writes.  Takes effect at the next build. */
#define QBVH_OPT_NODE_FORMAT 5
/* Lanes that share one particle's row in qbvh_lj_forward: 1, 2, 4, 8, 16 or
 * 32 (default 2).  More lanes read a row in longer contiguous chunks. */
#define QBVH_OPT_LJ_LANES 6
/* 1 (default): qbvh_lj_forward visits particles in the Z-order of the last
 * build (neighbouring particles share cached positions); 0: original order.
 * Results are the same up to FP32 rounding of the per-block FP64 sums'
 * inputs (each particle's own sums are unchanged). */
#define QBVH_OPT_LJ_ZORDER 7
/* Search method: 0 (default) = the quantized BVH; 1 = the paper's comparison
 * method, a sort-based uniform grid (cell list) with cells as wide as the
 * largest list radius and a 27-cell stencil walked by QBVH_OPT_GRID_LANES
 * lanes per particle (Sec. 3).  Same exact list.  With the grid, qbvh_build
 * only records the input (one system, positions kept alive by the caller
 * until the query has run) and the grid is built inside qbvh_query, because
 * the cell width is the list radius; qbvh_tree_get is not available.
 * Takes effect at the next build. */
#define QBVH_OPT_METHOD 8
/* Lanes per particle of the grid traversal: 1, 2, 4, 8, 16 or 32 (default 8);
 * n * value must stay below 2^32 (else qbvh_query: QBVH_ERR_INVALID_ARG). */
#define QBVH_OPT_GRID_LANES 9
/* Particles per warp of the warp-uniform walk: 32 (default), 16, 8, 4, 2 or
 * 1; with fewer particles each particle gets 32/value lanes.  With 2 or 4 lanes
 * per particle (16 or 8 per warp) the lanes split the survivors of each
 * bundle's filter and share the particle's row through their staging rings;
 * with more lanes they split a bundle's leaves and pack their accepted
 * neighbours with a ballot.  Fewer particles
 * per warp means more warps (small systems fill the GPU) and a smaller union
 * of search spheres per walk.  In a single-system build of 2 to 4 types,
 * a type of at most 4096 particles so sparse that 32 of them span more than
 * twice its largest list radius (32 L^3 / count > (2 r_max)^3) is walked
 * one particle per warp whatever this value.  The traversal launches
 * n * 32/value threads, which must stay below 2^32 (one particle per warp:
 * n < 2^27); qbvh_query returns QBVH_ERR_INVALID_ARG otherwise. */
#define QBVH_OPT_WARP_PARTICLES 10
/* Trees per system: 1 (default) = one tree per particle type, each pair of
 * types (a, b) searched with its own radius r_list[a][b] (Sec. 1, Sec. 5);
 * 0 = one tree per system holding every type.  With 0 the leaf test does not
 * see types, so qbvh_query then requires the same radius for every type pair
 * (else QBVH_ERR_INVALID_ARG); the list is the same, and each particle walks
 * one tree instead of one per type.  Types are still validated at the build
 * and still select the Lennard-Jones parameters.  Takes effect at the next
 * build. */
#define QBVH_OPT_TYPE_TREES 11
/* qbvh_query_lj_async: 1 = the traversal evaluates the LJ terms of the pairs
 * it accepts where it supports that (one system, one type, 32 particles per
 * warp, exact lists of FP32 data); 0 (default) = the traversal followed by
 * the separate pass of qbvh_lj_forward.  The summing traversal evaluates the
 * terms for every pair it tests, about four per listed pair, so at large N
 * the two passes are faster; the autotuner decides per workload.  Takes
 * effect at the next call. */
#define QBVH_OPT_FUSED_LJ 12
/* Traversal work distribution for the one-particle-per-lane walk of exact
 * FP32 lists: 0 (default) = one warp of the grid per packet of 32 Z-order
 * particles; 1 = about as many warps as the GPU keeps resident, each taking
 * packets from a device-side queue until none are left (a warp that ends
 * early starts another packet instead of waiting for its block).  The list
 * is the same either way.  Takes effect at the next query. */
#define QBVH_OPT_PERSISTENT 13

int qbvh_set_option(qbvh_handle h, int option, int value);
int qbvh_get_option(qbvh_handle h, int option, int *value);

/*
 * Build the quantized LBVH of one periodic system (Sec. 2.1, 2.2, Fig. 3):
 * Morton binning into 2^10-1 bins per axis, stable radix sort of the 30-bit
 * codes, Karras hierarchy (N-1 internal nodes with two children each),
 * bottom-up fit, ropes for stackless traversal and outward-rounded 10-bit
 * quantization of every node against the root AABB.  With n_types > 1 one
 * tree is built per type (per-type trees for size-asymmetric mixtures,
 * Sec. 1 and Sec. 5).
 *
 * pos_dev : [n] float4 {x, y, z, w}, 16-byte aligned, x,y,z in [0, L),
 *           w = the particle's type as int32 bits (0 when n_types == 1).
 * n       : number of particles (0 allowed: empty tree).
 * L       : cubic box edge, finite and > 0.
 * n_types : 1..QBVH_MAX_TYPES.
 * Positions and types are validated on the device; a violation is reported
 * by the next qbvh_query (QBVH_ERR_OUT_OF_BOX / QBVH_ERR_BAD_TYPE).
 * Errors here: INVALID_ARG, OOM, CUDA.
 */
int qbvh_build(qbvh_handle h, const void *pos_dev, int n, float L, int n_types,
               cudaStream_t stream);

/*
 * Build the LBVH of one periodic system whose particle data is in double
 * precision (Sec. 2.2: the boxes need not be; every FP32 or quantized box
 * must enclose the exact particle, so a coordinate x enters the tree as the
 * FP32 box [round-down(x), round-up(x)]).  The list the next qbvh_query
 * writes is exact for the FP64 positions: j is a neighbor of i when the FP64
 * minimum-image expression
 *     dx = xj - xi;  dx = dx - L * rint(dx * (1/L))   (y, z alike)
 *     d2 = (dx*dx + dy*dy) + dz*dz  <  (double)r_list * (double)r_list
 * holds in IEEE double arithmetic without contraction.  The traversal runs
 * in FP32 with the padded search sphere of Sec. 2.3; the leaf test takes
 * FP32 positions rounded to nearest and defers to the FP64 positions only
 * for the pairs within a proven error band of r_list (qbvh_query).
 *
 * pos64_dev : [n] double4 {x, y, z, w}, 32-byte aligned, x,y,z in [0, L),
 *             w = the particle's type as a whole number in [0, n_types).
 * L         : cubic box edge in FP64, finite and > 0 (its nearest FP32
 *             value is used for the FP32 parts).
 * n_types   : 1..4.
 * The uniform-grid method and the candidate mode do not take FP64 data
 * (QBVH_ERR_INVALID_ARG); the traversal of FP64 data is always the warp walk
 * with 32 particles per warp (QBVH_OPT_TRAVERSAL and QBVH_OPT_WARP_PARTICLES
 * do not apply).  Errors and device-side validation as qbvh_build.
 */
int qbvh_build_f64(qbvh_handle h, const void *pos64_dev, int n, double L, int n_types,
                   cudaStream_t stream);

/*
 * Build the trees of n_sys independent periodic systems in one launch
 * sequence (one tree per system and type).  System k owns particles
 * [sys_offsets_host[k], sys_offsets_host[k+1]) of pos_dev and the cubic box
 * of edge L_host[k].  sys_offsets_host has n_sys+1 non-decreasing entries,
 * starting at 0 and ending at n_total.  1 <= n_sys <= 65536 and
 * n_sys * n_types <= 65536.  Same pos_dev layout and errors as qbvh_build.
 */
int qbvh_build_batched(qbvh_handle h, const void *pos_dev, int n_total, int n_sys,
                       const int *sys_offsets_host, const float *L_host, int n_types,
                       cudaStream_t stream);

/*
 * Neighbor list from the last build: stackless rope traversal (Alg. 1) of
 * every particle in Z-order over the periodic images whose search sphere
 * overlaps the root (27-bit image set, Sec. 2.3), sphere-AABB test against
 * the decompressed node bounds (Eq. 2) with directed rounding (Sec. 3), the
 * exact FP32 distance test at the leaves, and compaction into rows.
 *
 * r_list_host : [n_types][n_types] list radii (r_cut + skin), symmetric,
 *               each 0 <= r < (L/2)(1 - 2^-20) for every system's L
 *               (0 = type pair never listed); all equal when the build
 *               put every type in one tree (QBVH_OPT_TYPE_TREES = 0).
 * cap         : initial row capacity, >= 1; rounded up to a multiple of 8
 *               (nlist_get reports the capacity in use).
 * max_retries : when some row has more than cap neighbors the capacity is
 *               raised to the largest count rounded up to 32 and the traversal
 *               rerun (tree reused), at most max_retries times.
 * Blocks the host on one 16-byte readback per traversal (the largest count and
 * the device error word).
 * Errors: NOT_BUILT, INVALID_ARG, CUTOFF_TOO_LARGE, OUT_OF_BOX, BAD_TYPE,
 *         OVERFLOW (counts complete, rows truncated), DEVICE_TIMEOUT, OOM, CUDA.
 */
int qbvh_query(qbvh_handle h, const float *r_list_host, int cap, int max_retries,
               cudaStream_t stream);

/*
 * Enqueue one traversal without waiting: the list is written with capacity
 * cap and the 16-byte status is copied to the handle's pinned host memory on
 * `stream`.  No host synchronization, no allocation once the row buffer
 * holds n*cap entries, so the call may be recorded into a CUDA graph after a
 * first call at the same sizes.  Read the outcome with qbvh_query_status once
 * the stream has completed.
 */
int qbvh_query_async(qbvh_handle h, const float *r_list_host, int cap, cudaStream_t stream);

/*
 * Outcome of the last traversal enqueued on the handle; valid after the
 * caller has synchronized that stream.  *max_count = largest row count,
 * return value = QBVH_OK, OUT_OF_BOX, BAD_TYPE, DEVICE_TIMEOUT or OVERFLOW
 * (max_count > cap).
 */
int qbvh_query_status(qbvh_handle h, int *max_count);

/*
 * Borrow the neighbor list of the last query (Sec. 1: the Verlet list).
 * rows   : [n][cap] int32, row i lists the original indices j of particle i's
 *          neighbors in unspecified order; entries past counts[i] are unset.
 * counts : [n] int32 number of neighbors of particle i (may exceed cap only
 *          after QBVH_ERR_OVERFLOW).
 * Indices are positions in the pos_dev array of the build (concatenated over
 * systems for a batched build).  Any output pointer may be NULL.
 */
int nlist_get(qbvh_handle h, const int **rows, const int **counts, int *cap, int *max_count);

/*
 * Borrow the tree of the last build, for inspection and tests.
 * nodes     : [n] int4 internal nodes by Karras index, each
 *             {lo | bundle<<31, hi, left child or first leaf, rope},
 *             lo/hi = qx<<20 | qy<<10 | qz (Fig. 3b), ids >= 0 internal,
 *             ~k leaf k, INT32_MIN end of traversal; slot of each tree's
 *             last leaf unused.
 * leaves    : [n] float4 {x, y, z, original index | (rope is internal)<<31}
 *             in Z-order.
 * order     : [n] int32 sorted position -> original index.
 * seg_start : [n_seg + 1] int32 first sorted position of each tree, tree
 *             s = system * n_types + type.
 * frames    : [n_seg] 8 floats {R_lo xyz, h xyz, -, -}: quantization frame
 *             of each tree (root AABB corner and bin width).
 * n_seg     : number of trees.
 */
int qbvh_tree_get(qbvh_handle h, const void **nodes, const void **leaves, const int **order,
                  const int **seg_start, const float **frames, int *n_seg);

/*
 * Truncated-and-shifted Lennard-Jones energy (Eq. 1, shifted to zero at
 * r_cut, Sec. 1) over the handle's last neighbor list, in one fused pass:
 * per-particle energy, forces and the gradients with respect to the
 * per-type-pair parameters.  Pairs interact when the FP32 distance
 * expression above gives d2 < r_cut*r_cut.  Accumulation is FP32 per
 * particle; the per-system sums are FP64.
 *
 * pos_dev      : [n] float4 as for the build (original order).
 * eps_dev, sig_dev : [n_types][n_types] float32 device arrays.
 * r_cut_host   : [n_types][n_types] float32, each <= the list radius used.
 * e_dev        : [n] float32 out, 1/2 of particle i's pair energies (or NULL).
 * U_dev        : [n_sys] float64 out, total energy of each system (required).
 * F_dev        : [n][3] float32 out, F_i = -dU/dx_i (or NULL).
 * dE_dev, dS_dev : [n_sys][n_types][n_types] float64 out, dU/deps[a][b] and
 *                dU/dsig[a][b] of each system, each matrix entry treated as
 *                its own parameter (or NULL).
 * Errors: NOT_BUILT (no list), INVALID_ARG, CUDA.
 */
int qbvh_lj_forward(qbvh_handle h, const void *pos_dev, const float *eps_dev,
                    const float *sig_dev, const float *r_cut_host, float *e_dev, double *U_dev,
                    float *F_dev, double *dE_dev, double *dS_dev, cudaStream_t stream);

/*
 * Traversal and Lennard-Jones forward in one call: enqueues qbvh_query_async
 * (same arguments r_list_host, cap) and the energies, forces and eps/sigma
 * gradients of qbvh_lj_forward over the list it writes (same arguments and
 * outputs; pos_dev = the positions of the last build).  This is the step of
 * a simulation that rebuilds its Verlet list (Sec. 1): the pair energy of
 * Eq. 1, truncated and shifted at r_cut, is needed for the same pairs the
 * search has just found.
 *
 * With QBVH_OPT_FUSED_LJ = 1, for one system of one type walked 32
 * particles per warp (the default mapping) with exact lists of FP32 data,
 * the traversal sums the pair terms of every pair it accepts with
 * d2 < r_cut^2, from the positions it already holds, and the list is not
 * read back.  The per-particle sums then run in the walk's order instead of the
 * row order: the results agree with qbvh_lj_forward to FP32 rounding, not bit
 * for bit, and are deterministic.  Otherwise the two passes run back to back.
 * The LJ outputs are valid when qbvh_query_status returns QBVH_OK: after an
 * overflow the fused sums include the pairs past cap, the separate pass does
 * not.  No host synchronization.
 * Errors: NOT_BUILT, INVALID_ARG (as either call), and the enqueue errors of
 *         qbvh_query_async.
 */
int qbvh_query_lj_async(qbvh_handle h, const void *pos_dev, const float *r_list_host, int cap,
                        const float *eps_dev, const float *sig_dev, const float *r_cut_host, float *e_dev,
                        double *U_dev, float *F_dev, double *dE_dev, double *dS_dev, cudaStream_t stream);

/*
 * Chain rule for a scalar loss of the per-system energies: with g = dLoss/dU
 * ([n_sys] float64 device), writes grad_pos[i] = -g[sys(i)] * F[i] ([n][3]
 * float32) and grad_eps = sum_k g[k] dE[k], grad_sig likewise ([n_types^2]
 * float32).  F, dE, dS are the outputs of qbvh_lj_forward.  Any output may
 * be NULL.
 */
int qbvh_lj_backward(qbvh_handle h, const double *g_dev, const float *F_dev,
                     const double *dE_dev, const double *dS_dev, float *grad_pos_dev,
                     float *grad_eps_dev, float *grad_sig_dev, cudaStream_t stream);

/*
 * Allocation-free variant of qbvh_lj_forward, for callers that cannot allocate
 * device memory when they need forces: an allocator locked for the length of
 * a step, a plugin inside a host program that owns every device allocation,
 * or a loop where cudaMalloc/cudaFree (which may synchronize the device) are
 * not allowed.  The paper has no counterpart; this is an interface choice of
 * this library.
 *
 * Same energies, forces and eps/sigma gradients as qbvh_lj_forward, for ONE
 * periodic system of edge L and a neighbor list the caller passes in
 * (rows_dev [n][cap], counts_dev [n], as nlist_get returns them); no handle.
 * pos_dev, eps_dev, sig_dev, e_dev, F_dev: as for qbvh_lj_forward;
 * r_cut_host: [n_types][n_types] float32 on the host; U_dev: [1] float64;
 * dE_dev, dS_dev: [n_types][n_types] float64 (or NULL).
 * status_dev: [1] int32 device, required: written on the stream with
 *   QBVH_OK, QBVH_ERR_BAD_TYPE (some particle's type w is outside
 *   [0, n_types): that particle and every pair with it are left out) or
 *   QBVH_ERR_INTERNAL (some row entry is outside [0, n): that entry is left
 *   out).  On either error *U_dev is NaN.  Types are not clamped.
 *
 * Nothing is allocated: the per-block FP64 sums and the error word live in a
 * fixed variable of 1216 x 33 doubles plus one word (about 321 KB) inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  Limit: n_types <= 4 (larger counts return QBVH_ERR_INVALID_ARG
 * because their sums would not fit that variable).  The device address of
 * the variable is looked up (cudaGetSymbolAddress) by the first call on each
 * device, and again by the first call after that device's CUDA context has
 * changed (for example after cudaDeviceReset); make such a first call before
 * any stream capture.  Every call clears the error word and rewrites the
 * sums it reads on its stream, so nothing carries over from one call to the
 * next, but calls that overlap on the GPU (several streams or host threads)
 * share the variable and race.  Runs on the current device and is
 * asynchronous.  Errors returned: INVALID_ARG, CUDA.
 */
int qbvh_lj_forward_noalloc(const void *pos_dev, int n, float L, int n_types, const int *rows_dev,
                            const int *counts_dev, int cap, const float *eps_dev, const float *sig_dev,
                            const float *r_cut_host, float *e_dev, double *U_dev, float *F_dev,
                            double *dE_dev, double *dS_dev, int *status_dev, cudaStream_t stream);

/*
 * Self-test of the bounded device-side waits (failure detection without a
 * GPU fault).  Runs one tile of a radix-sort pass (the decoupled look-back of
 * the Morton-code sort, Sec. 3) whose predecessor never publishes its counts,
 * with a short poll limit (4096 polls).  The kernel gives up, records the
 * timeout in its error word and finishes with every access in bounds; the
 * expected return value is QBVH_ERR_DEVICE_TIMEOUT (QBVH_OK would mean the
 * wait did not give up).  Allocates and frees about 50 KB on `device`;
 * synchronizes `stream`.
 */
int qbvh_selftest_wait_timeout(int device, cudaStream_t stream);

/*
 * Pack positions [n][3] float32 and types [n] int32 (types_dev may be NULL
 * for all-zero) into the float4 layout the build reads.
 */
int qbvh_pack_positions(const float *xyz_dev, const int *types_dev, int n, void *pos4_dev,
                        cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* QBVH_H */
