/*
 * psr.h - C ABI of libpsr, the GB300 (sm_103a) library for the truncated
 * short-range particle-particle (P2P) gravity of the PM-FMM method
 * (Wang & Meng, "PhotoNs-GPU", arXiv:2107.14008).
 *
 * What is computed (paper, Section 2, Eq. tr): for every particle i of a
 * periodic box of side L,
 *
 *   a_i = G sum_j sum_{n in Z^3} [j != i or n != 0] [0 < |d| < r_c]
 *           m_j d T(|d| / (2 r_s)) / |d|^3,      d = x_j + n L - x_i,
 *   T(x) = erfc(x) + (2x / sqrt(pi)) exp(-x^2),
 *
 * i.e. the short-range pair force F_s = -(r/r^3) T of Section 2 per unit
 * target mass, truncated at the cutoff r_c, with the split radius
 * r_s = 1.2 L / N_PM.  The sum runs over the leaf pairs of an octree whose
 * leaves hold at most max_leaf particles (Sections 2 and 3.1-3.2: particles
 * grouped into contiguous leaves, a task list of <target leaf, source leaf>
 * pairs grouped by target leaf).  The list holds every leaf pair whose
 * bounding boxes come closer than r_c, so it adds no approximation.
 *
 * Conventions for every entry point:
 *  - Status: 0 (PSR_OK) or a negative PSR_E_* code; psr_last_error() gives a
 *    message (thread-local, valid until the next call on that thread).
 *    Nothing throws across the ABI.
 *  - Host pointers are marked "host", device pointers "device".  Device
 *    memory is always owned by the caller; the library never allocates or
 *    frees device memory and never synchronises inside psr_p2p_forces or
 *    psr_p2p_adjoint (both only enqueue work on the given stream).
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - Arrays of vectors are row-major n x 3.
 *  - Calls that use the same psr_leaves must be ordered on one stream; two
 *    such calls running concurrently on different streams race on the
 *    workspace's scheduler counters.
 */
#ifndef PSR_H
#define PSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status codes */
#define PSR_OK 0
#define PSR_E_ARG (-1)       /* bad argument (NULL, size, NaN position ...)   */
#define PSR_E_CUTOFF (-2)    /* r_c >= L or r_c <= 0: only n in {-1,0,1}^3
                                images are summed, which needs r_c < L       */
#define PSR_E_WORKSPACE (-3) /* workspace missing, too small or misaligned   */
#define PSR_E_CUDA (-4)      /* a CUDA runtime call failed                   */
#define PSR_E_DEVICE (-5)    /* a kernel's bounds check set the error word   */
#define PSR_E_TIMEOUT (-6)   /* a bounded host wait on the device ran out    */
#define PSR_E_NOMEM (-7)     /* host allocation failed                       */
#define PSR_E_STATE (-8)     /* call order violated (e.g. not uploaded)      */

/* ------------------------------------------------------------ options */
/* precision of the pair arithmetic */
#define PSR_FP64 0        /* FP64 throughout, T from erfc/exp; with interp
                             PSR_TAYLOR2/4 the paper's double-precision table
                             path instead (Section 3.3: the Taylor table in
                             FP64 about the nearest node, 1/r by Newton-
                             Raphson from an FP32 estimate; forward only, not
                             in psr_p2p_forces_noalloc)                     */
#define PSR_FP32_EXACT 1  /* FP32 pair math, T from erfcf/expf              */
#define PSR_FP32_TABLE 2  /* FP32 pair math, T interpolated from a table
                             in shared memory (Section 3.3)                 */
/* interpolation of the table (PSR_FP32_TABLE; the Taylor levels also
   select PSR_FP64's table path) */
#define PSR_LINEAR 0      /* chord between nodes                            */
#define PSR_CUBIC 1       /* cubic Hermite on (T_k, T'_k = x_k^2 E_k)       */
#define PSR_TAYLOR2 2     /* the paper's Taylor table (Section 3.3, Eq. int)
                             to level T_[2] about the nearest node; forward
                             only                                           */
#define PSR_TAYLOR4 3     /* the same to level T_[4]                        */
/* inner loop of the FP32 forward kernels */
#define PSR_KERNEL_AUTO 0   /* the library's default (scalar streams)          */
#define PSR_KERNEL_SCALAR 1 /* one source particle per lane and iteration      */
#define PSR_KERNEL_PAPER 3  /* the paper's mapping (Section 3.2, Algorithms 1
                               and 2): one thread block per target leaf, one
                               thread per target particle, each source leaf
                               staged in shared memory between two barriers;
                               same pair arithmetic and tables (prior art,
                               kept for comparison)                           */
#define PSR_KERNEL_PACKED 2 /* two source particles per lane and iteration in
                               packed f32x2 arithmetic (sm_100+) for leaves
                               that take one target per lane; the scalar
                               two- and three-targets paths for the others  */
/* accumulation of FP32 partial sums across source leaves */
#define PSR_ACC_FP64 0    /* fold into FP64 accumulators                    */
#define PSR_ACC_KAHAN32 1 /* fold with compensated (two-sum) FP32           */

typedef struct {
    double L;   /* box side; positions are wrapped into [0, L)              */
    double r_s; /* split radius (1.2 L / N_PM in the paper, Section 2)      */
    double r_c; /* cutoff radius, 0 < r_c < L                                */
    double G;   /* gravitational constant                                    */
} psr_box;

typedef struct {
    int precision;       /* PSR_FP64 | PSR_FP32_EXACT | PSR_FP32_TABLE        */
    int table_n;         /* table intervals on [0, x_c]: a power of two in
                            [64, 8192] for PSR_LINEAR / PSR_CUBIC (0 = 1024);
                            any value in [64, 2048] for the Taylor tables
                            (0 = 384, the paper's node spacing 3/512 at
                            x_c = 2.25)                                       */
    int interp;          /* PSR_LINEAR | PSR_CUBIC | PSR_TAYLOR2 | PSR_TAYLOR4
                            (the adjoint takes PSR_LINEAR | PSR_CUBIC)        */
    int accum;           /* PSR_ACC_FP64 | PSR_ACC_KAHAN32                    */
    int warps_per_block; /* 1..8; 0 = default (8)                            */
    int blocks_per_sm;   /* 0 = default (occupancy-derived)                   */
    int fold_every;      /* source particles summed in FP32 before a fold;
                            0 = default (64)                                  */
    int count_pairs;     /* 1: also count pairs with 0 < r < r_c (slower)     */
    int kernel;          /* PSR_KERNEL_AUTO | _SCALAR | _PACKED | _PAPER (FP32 forward;
                            the FP32 adjoint runs its packed variant for
                            _PACKED, its scalar one otherwise)               */
    int source_tile;     /* FP32 kernels: source particles staged per warp in
                            shared memory, 64 | 128 | 256 and >= the largest
                            leaf; 0 = default (forward 256, adjoint 128)    */
    int shard_count;     /* split the target leaves over shard_count launches
                            (one per GPU, inputs replicated): this launch
                            computes the targets of schedule entries
                            shard_index, shard_index + shard_count, ... (the
                            schedule is largest-work first, so the shards are
                            balanced) and leaves every other output element
                            untouched; 0 or 1 = all targets                  */
    int shard_index;     /* 0 <= shard_index < max(shard_count, 1)          */
    int reserved[4];     /* must be zero                                      */
} psr_opts;

typedef struct {
    int64_t n;               /* particles (all boxes)                          */
    int64_t n_leaves;        /* octree leaves                                  */
    int64_t n_pairs;         /* leaf-pair entries (including i = j)            */
    int64_t n_items;         /* scheduled target leaves (= n_leaves)           */
    int64_t nbox;            /* boxes                                          */
    int64_t evaluated_pairs; /* sum over leaf pairs of n_I * n_J               */
    size_t device_bytes;     /* workspace size psr_upload needs                */
    int max_leaf;            /* largest leaf occupancy                          */
    int max_row;             /* most source leaves of one target leaf          */
    double build_seconds;    /* host time of psr_build_leaves*                 */
    const int64_t* perm;     /* host, n: sorted index -> original index
                                (owned by the handle); NULL for a handle built
                                on the device                                  */
    int64_t n_far;           /* well-separated (M2L) leaf-pair entries of a
                                psr_device_build_split handle, else 0; n_pairs
                                then counts the near (P2P) entries only        */
    double theta;            /* acceptance parameter of that split, else 0    */
    int64_t rows_walked_twice; /* device builds: target leaves whose pair row
                                the count walk could not keep in the pair
                                cache, walked again by psr_device_build_finish
                                (every row for a split or when the cache's
                                per-row slot is below 16 runs); else 0      */
    int equal_mass;          /* 1 if within every box all particles have one
                                mass: the FP32 kernels then apply it once per
                                target instead of once per pair (the paper's
                                kernel carries a single GM, Algorithm 2)    */
} psr_info;

typedef struct psr_leaves psr_leaves; /* opaque, host-owned */

/* Build flags */
#define PSR_BUILD_ORB 2     /* host builder: the paper's ORB tree (Section 2:
                               a cell's particles split in two equal halves
                               along the longest axis of their box) instead
                               of the Morton octree; leaf centres (lcen) are
                               the leaf boxes' centres on the L / 2^22 grid */
#define PSR_BUILD_UNPACKED 4 /* plain octree leaves.  By default both
                               builders pack them: consecutive sibling cells
                               that would each be a leaf share one leaf (their
                               parent's cell) while their total stays within
                               max_leaf, taken greedily in Morton order (a
                               pack of one keeps its own cell); fuller leaves
                               whose boxes stay inside the parent cell      */
#define PSR_BUILD_SPLIT_GAUSSIAN 8 /* psr_device_build_split: also measure
                               the cells against the Gaussian length of the
                               kernel (see there)                           */
#define PSR_BUILD_NO_FP64 1 /* omit the FP64 particle copy (PSR_FP64 and the
                               FP64 adjoint are then unavailable)            */

/*
 * psr_build_leaves - host: sort particles along a Morton curve, cut the
 * octree into leaves of at most max_leaf particles (each leaf a contiguous
 * pack, Section 2), and build the near-field leaf-pair list grouped by
 * target leaf (the TaskGroup/GroupIdx of Section 3.2) with a periodic image
 * code per entry.
 *   pos      host, n x 3 FP64, any real values (wrapped into [0, L));
 *            may be NULL when n = 0
 *   mass     host, n FP64, or NULL for equal masses 1/n
 *   box      host, box parameters
 *   max_leaf 1..64
 *   flags    PSR_BUILD_* bits
 *   out      receives the handle; free with psr_free_leaves
 * n = 0 gives an empty handle: the device calls then do nothing.
 * Errors: PSR_E_ARG (NULL, n < 0, n >= 2^31, non-finite input, max_leaf out
 * of range, r_s <= 0), PSR_E_CUTOFF (r_c <= 0 or r_c >= L), PSR_E_NOMEM.
 */
int psr_build_leaves(const double* pos, const double* mass, int64_t n, const psr_box* box,
                     int max_leaf, int flags, psr_leaves** out);

/*
 * psr_build_leaves_batch - host: as psr_build_leaves for nbox independent
 * boxes in one handle; one launch then serves every box.  Particles are
 * numbered box after box (box 0's n[0] particles first).  All boxes must
 * share the ratio r_c / r_s (one interpolation table).
 */
int psr_build_leaves_batch(int nbox, const double* const* pos, const double* const* mass,
                           const int64_t* n, const psr_box* boxes, int max_leaf, int flags,
                           psr_leaves** out);

/* psr_leaves_info - host: sizes of a built handle (see psr_info). */
int psr_leaves_info(const psr_leaves* h, psr_info* info);

/*
 * psr_upload - copy the handle's arrays into a caller-owned device
 * workspace of at least info.device_bytes bytes, 256-byte aligned, on
 * `cuda_stream` (the host side is pageable, so the call returns once the
 * copies are staged).  The workspace must stay allocated, and unchanged by
 * the caller, while the handle uses it.
 * Errors: PSR_E_WORKSPACE (NULL, too small, misaligned), PSR_E_CUDA.
 */
int psr_upload(psr_leaves* h, void* d_workspace, size_t bytes, void* cuda_stream);

/*
 * psr_p2p_forces - device: accelerations of every particle (Section 2 pair
 * force, Section 3.2 kernel), one persistent launch over all target leaves
 * of all boxes.
 *   d_acc  device, n x 3, in the ORIGINAL particle order; FP64 when
 *          opts->precision == PSR_FP64, FP32 otherwise.  Overwritten.
 * The first call with a new (precision, table_n, interp) also builds the
 * interpolation table in the workspace (one small extra launch).
 * Errors: PSR_E_ARG, PSR_E_STATE (not uploaded; FP64 payload omitted),
 * PSR_E_CUDA (launch failure).
 */
int psr_p2p_forces(psr_leaves* h, const psr_opts* opts, void* d_acc, void* cuda_stream);

/*
 * psr_p2p_adjoint - device: gradients of L = sum_i c_i . a_i (not in the
 * paper; derived from the pair force and the n = 2 truncated prefactor f_(2)
 * of Section 2):
 *   dL/dx_k = G sum_j K(d_kj) (m_k c_j - m_j c_k),
 *   K(d)    = g I + (g'(r)/r) d d^T,  g = T/r^3,  g'(r)/r = -f_(2),
 *   dL/dm_k = -G sum_j g(r_kj) d_kj . c_j,
 * over the same pairs as the forward sum.
 *   d_cot       device, n x 3 cotangent, original order
 *   d_grad_pos  device, n x 3, original order, overwritten
 *   d_grad_mass device, n, original order, overwritten (may be NULL)
 * All three are FP64 when opts->precision == PSR_FP64, FP32 otherwise.
 */
int psr_p2p_adjoint(psr_leaves* h, const psr_opts* opts, const void* d_cot, void* d_grad_pos,
                    void* d_grad_mass, void* cuda_stream);

/*
 * psr_p2p_forces_noalloc - device: the same accelerations as psr_p2p_forces
 * (same kernels, same options), for callers that cannot allocate device
 * memory - code that runs inside a memory pool or arena owned by a host
 * framework, in a context where an allocation may block, or under a policy
 * that forbids allocations after start-up.  The paper has no counterpart;
 * this is an interface addition of this library.
 *   h      a handle uploaded with psr_upload (its workspace holds the inputs)
 *   d_acc  device, n x 3, original order, as for psr_p2p_forces
 * The kernel's scratch (work counters, error word and interpolation table)
 * is a fixed 66,048-byte __device__ array in the library instead of the
 * workspace; each device that loads the library holds one copy until the
 * process exits.  The call never calls cudaMalloc, cudaFree or any other
 * allocating routine.
 * Limits and behaviour:
 *  - PSR_FP32_TABLE accepts table_n <= 4096; larger tables return PSR_E_ARG.
 *  - Set-up: the first call on each device (with that device current) looks
 *    up the array's device address with cudaGetSymbolAddress and caches it.
 *    Under CUDA's default lazy module loading that look-up is what loads the
 *    library's module holding the array onto the device, and the driver
 *    allocates the array's storage at that moment.  A caller that cannot
 *    allow even that makes one call on each device at start-up, before any
 *    stream capture (or runs with CUDA_MODULE_LOADING=EAGER, which loads the
 *    modules when the context is created); later calls allocate nothing.
 *  - Every call on a device shares the array: each call clears its counters
 *    and rebuilds the table it needs first, and two calls that overlap on
 *    the GPU (different streams, no ordering) race on it.
 *  - Bounds-check errors of these calls land in the shared array and are
 *    not reported by psr_check; count_pairs results are not readable either.
 * Errors: as psr_p2p_forces, plus PSR_E_ARG for an oversized table.
 */
int psr_p2p_forces_noalloc(psr_leaves* h, const psr_opts* opts, void* d_acc, void* cuda_stream);

/*
 * psr_autotune - host + device: pick the tile shape of the FP32 forward
 * kernel for this leaf set.  Starting from *base (precision, table, interp
 * and accumulation are kept), times every candidate of
 *   kernel      PSR_KERNEL_SCALAR | PSR_KERNEL_PACKED  (sources per lane
 *               and iteration: 1 | 2)
 *   warps       4 | 8 per block
 *   source_tile 64 | 128 | 256 staged source particles per warp
 * that fits shared memory and the largest leaf, with CUDA events on
 * `cuda_stream` (one warm-up and `reps` timed launches each, best time
 * kept), writing the accelerations to d_acc (n x 3 FP32, overwritten).
 * The best options go to *best and their time in milliseconds to *best_ms
 * (may be NULL).  Synchronises the stream; every wait is bounded by
 * timeout_ms (PSR_E_TIMEOUT).  Errors: PSR_E_ARG (FP64 precision, reps < 1),
 * PSR_E_STATE (not uploaded), PSR_E_CUDA, PSR_E_TIMEOUT.
 */
int psr_autotune(psr_leaves* h, const psr_opts* base, void* d_acc, void* cuda_stream, int reps,
                 int timeout_ms, psr_opts* best, float* best_ms);

/*
 * psr_fp32_peak - host + device: measure the FP32 fused multiply-add rate
 * of the current device, the denominator of the FP32 kernels' roofline (the
 * paper, Section 5, states its kernel throughput as a fraction of the SP
 * peak).  Not part of the method.  Launches `launches` times a kernel of
 * (SMs x 4) blocks of 256 threads in which every thread runs 8 independent
 * chains x <- x a + b (a = 0.9999, b = 1e-4: the values stay near 1) for
 * iters x 8 steps, timing each launch with CUDA events on `cuda_stream`, and
 * writes the best rate, 2 FLOP per FMA, to *flops_per_s.
 *   d_sink      caller-owned device buffer of sink_bytes bytes; it receives
 *               one float per thread (so that no chain is optimised away)
 *               and must hold SMs x 4 x 256 floats (4 MB covers any device
 *               of up to 1024 SMs)
 * Synchronises the stream; every wait is bounded by timeout_ms.
 * Errors: PSR_E_ARG (null pointer, iters or launches < 1, sink too small:
 * the message states the size needed), PSR_E_CUDA, PSR_E_TIMEOUT.
 */
int psr_fp32_peak(void* d_sink, size_t sink_bytes, int iters, int launches, void* cuda_stream,
                  int timeout_ms, double* flops_per_s);

/*
 * psr_pair_count - host: number of pairs with 0 < r < r_c counted by the
 * last psr_p2p_forces call made with opts->count_pairs = 1 (waits up to
 * timeout_ms for the stream).  Errors: PSR_E_STATE, PSR_E_TIMEOUT.
 */
int psr_pair_count(psr_leaves* h, void* cuda_stream, int timeout_ms, int64_t* count);

/*
 * psr_evaluated_count - host: number of pair terms the kernel of the last
 * psr_p2p_forces call made with opts->count_pairs = 1 evaluated (target
 * particles x source particles it ran the pair arithmetic on, self pairs
 * included; waits up to timeout_ms for the stream).  The FP32 warp-per-leaf
 * kernels drop staged sources that lie at least r_c from the target leaf's
 * particle box (those pairs are zero by the truncation of Eq. tr), so their
 * count lies between psr_pair_count's and the leaf-pair tiles' total
 * (psr_info.evaluated_pairs); the FP64 and PSR_KERNEL_PAPER kernels evaluate
 * every tile pair.  Errors: PSR_E_STATE, PSR_E_TIMEOUT.
 */
int psr_evaluated_count(psr_leaves* h, void* cuda_stream, int timeout_ms, int64_t* count);

/*
 * psr_check - host: wait (at most timeout_ms) for `cuda_stream`, then read
 * and clear the workspace's device error word.  Returns PSR_E_DEVICE if a
 * kernel found an out-of-range index (the offending entry was skipped),
 * PSR_E_TIMEOUT if the stream did not finish in time.
 */
int psr_check(psr_leaves* h, void* cuda_stream, int timeout_ms);

/*
 * psr_table - device: write the interpolation table the FP32 table path
 * uses for (table_n, interp) over [0, x_c] into d_out (float4 entries,
 * table_n + 1 of them; entry table_n is the zero sentinel beyond the
 * cutoff).  Linear: (M_k, D_k, A_k, 0) with T = M_k + f D_k, f in
 * [-1/2, 1/2] about the interval midpoint, equivalently T = A_k + (k + f) D_k
 * (A_k = M_k - k D_k, the form the forward kernel evaluates); cubic:
 * (c0, c1, c2, c3) with
 * T = c0 + f (c1 + f (c2 + f c3)).  Taylor (table_n in [64, 2048]): two
 * float4 per node k = 0..table_n, (c0, c1, c2, c3) and (c4, 0, 0, 0), with
 * T = c0 + f (c1 + f (c2 + f (c3 + f c4))), f = (x - x_k) table_n / x_c the
 * offset from the nearest node (c3 = c4 = 0 for PSR_TAYLOR2).  For tests and
 * inspection.
 */
int psr_table(int table_n, int interp, double x_c, void* d_out, void* cuda_stream);

/*
 * psr_leaves_host_arrays - host: read-only views of the handle's host copies
 * of what psr_upload sends to the device (for tests and inspection).  Valid
 * until psr_free_leaves.  Layouts:
 *   pf     n x 4 FP32: (x, y, z) - leaf-cell centre, divided by 2 r_s; mass
 *   pd     n x 4 FP64: wrapped x, y, z; mass (NULL with PSR_BUILD_NO_FP64)
 *   leaf   n_leaves x 4 int32: first sorted particle, count, box, 0
 *   lcen   n_leaves x 4 int32: cell centre in units of L / 2^22 (x, y, z),
 *          octree level
 *   rowptr n_leaves + 1 int64: entries of target leaf I are
 *          pairs[rowptr[I] .. rowptr[I+1])
 *   pairs  n_pairs uint32: (source leaf << 5) | (nx+1)*9 + (ny+1)*3 + (nz+1)
 *   items  n_leaves int32: target leaves in the order the kernels take them
 */
typedef struct {
    const float* pf;
    const double* pd;
    const int32_t* leaf;
    const int32_t* lcen;
    const int64_t* rowptr;
    const uint32_t* pairs;
    const int32_t* items;
} psr_host_arrays;
int psr_leaves_host_arrays(const psr_leaves* h, psr_host_arrays* out);

/*
 * psr_leaves_regions - host: byte offsets of the arrays inside the device
 * workspace, with the layouts of psr_host_arrays, plus perm (n int32: sorted
 * index -> original index) and the workspace size.  pd is meaningful only
 * without PSR_BUILD_NO_FP64.  For reading a workspace on the device, e.g.
 * the permutation of a device-built handle.  Errors: PSR_E_ARG (NULL).
 */
typedef struct {
    size_t pf, pd, perm, leaf, lcen, rowptr, pairs, items;
    size_t frow, fpairs, fcen, fofs; /* multipole split only: far CSR
                                  (n_leaves + 1 int64), far entries (n_far
                                  uint32, the pair list's encoding), expansion
                                  centres (n_leaves x 4 FP64: x, y, z, radius),
                                  their offsets from the cell centres lcen
                                  (n_leaves x 4 FP32: x, y, z, radius)       */
    size_t total;
} psr_regions;
int psr_leaves_regions(const psr_leaves* h, psr_regions* out);

/* ------------------------------------------------- device leaf builder */
/*
 * The leaf set of psr_build_leaves built on the GPU from device-resident
 * positions (one box): the same leaves, pair list and schedule, bit for bit
 * (paper, Section 2 and Section 3.2; the tree is a binary radix tree over
 * the Morton-ordered leaf cells, whose walk keeps the same leaf pairs in the
 * same order as the host's octree walk).  Two calls, so that the caller can
 * size the workspace from the counts:
 *
 * psr_device_build_scratch_bytes - host: scratch bytes psr_device_build
 * needs for n particles (about 430 per particle, 64 of them a cache of the
 * pair rows the counting walk finds, which psr_device_build_finish then
 * copies instead of walking the tree again).  Errors: PSR_E_ARG
 * (n < 1 or n > 2^28, NULL).
 *
 * psr_device_build - enqueue key, radix sort, leaf, radix tree and pair
 * count kernels on cuda_stream, wait for them (each wait at most timeout_ms;
 * <= 0 means 60 s) and read back the leaf and pair counts; returns a handle
 * whose workspace is not yet written (psr_leaves_info works on it).
 *   d_pos     device, n x 3 FP64, any real values (wrapped into [0, L));
 *             consumed before the call returns
 *   d_mass    device, n FP64, or NULL for equal masses 1/n; consumed before
 *             the call returns
 *   n         1 .. 2^28
 *   d_scratch device, >= psr_device_build_scratch_bytes(n) bytes, 256-byte
 *             aligned, owned by the caller; it holds the build state until
 *             the work psr_device_build_finish enqueues has run
 * The box must have r_c >= 1e-10 and L <= 1e12 (the walk's FP32 bounds
 * stay rigorous there).  Not capturable in a CUDA graph (it waits on the
 * stream).  Errors: PSR_E_ARG (argument, box outside that range, non-finite
 * position or mass), PSR_E_CUTOFF,
 * PSR_E_WORKSPACE (scratch missing, small or misaligned), PSR_E_CUDA,
 * PSR_E_TIMEOUT, PSR_E_DEVICE (a tree bound check fired: traversal stack
 * overflow or a malformed tree; the build is abandoned), PSR_E_NOMEM.
 *
 * psr_device_build_finish - enqueue on cuda_stream the kernels that write
 * the workspace (psr_leaves_info().device_bytes, 256-byte aligned, owned by
 * the caller) from the scratch; afterwards the handle is as after
 * psr_upload.  On a device-built handle psr_upload and
 * psr_leaves_host_arrays return PSR_E_STATE and psr_info.perm is NULL (the
 * permutation is in the workspace at psr_leaves_regions().perm).  Errors:
 * PSR_E_STATE (no pending device build), PSR_E_WORKSPACE, PSR_E_CUDA.
 */
int psr_device_build_scratch_bytes(int64_t n, size_t* bytes);
int psr_device_build(const double* d_pos, const double* d_mass, int64_t n, const psr_box* box,
                     int max_leaf, int flags, void* d_scratch, size_t scratch_bytes,
                     void* cuda_stream, int timeout_ms, psr_leaves** out);
int psr_device_build_finish(psr_leaves* h, void* d_ws, size_t bytes, void* cuda_stream);

/*
 * psr_device_build_split - psr_device_build with the multipole split of the
 * paper's PM-FMM short range (Section 2: cell pairs that are well separated
 * interact through M2L, the rest through P2P).  Every leaf-pair entry the
 * walk finds within r_c goes to exactly one of two lists:
 *   far   the particle boxes' centres are R apart with theta |R| >= rho_I +
 *         rho_J (rho: half the box diagonal; with PSR_BUILD_SPLIT_GAUSSIAN
 *         also theta 2 r_s^2 / |R| >= rho_I + rho_J, 2 r_s^2 / |R| being the
 *         length on which the kernel's Gaussian truncation varies) and every
 *         point of one box lies within r_c of every point of the other (so
 *         the hard cutoff removes no pair of the expansion);
 *   near  every other entry, including i = j.
 * The handle's pair list (what psr_p2p_forces and psr_p2p_adjoint evaluate)
 * holds the near entries only; the far list and the expansion centres are
 * in the workspace (psr_leaves_regions: frow, fpairs, fcen) for
 * psr_fmm_forces.  The union of the two lists is the list psr_device_build
 * writes.  theta in (0, 1].  The classification is made in FP32: the
 * inside test rigorously (boxes rounded outward, distances rounded up,
 * against r_c^2 (1 - 1e-6) rounded down), the opening test with plain
 * rounding, so that an entry within about 1e-6 of the opening threshold may
 * fall on either side.
 * Errors: those of psr_device_build; PSR_E_ARG for theta outside (0, 1].
 */
int psr_device_build_split(const double* d_pos, const double* d_mass, int64_t n,
                           const psr_box* box, int max_leaf, int flags, double theta,
                           void* d_scratch, size_t scratch_bytes, void* cuda_stream,
                           int timeout_ms, psr_leaves** out);

/* ------------------------------------------------- long-range PM part */
/*
 * The long-range part of the PM-FMM split (paper, Section 2): phi_long solves
 * Poisson's equation on an N_PM^3 mesh with the Gaussian-filtered Green's
 * function -4 pi G exp(-k^2 r_s^2) / k^2 (the Fourier complement of the
 * short-range erfc(r / 2 r_s) of Eq. tr; the paper prints exp(-k^2/4r_s^2),
 * which is not its complement), k = 0 dropped.  Cloud-in-cell (CIC) mass
 * assignment onto mesh points g L / N_PM, FFT (cuFFT), division by the
 * squared CIC window unless PSR_PM_NO_DECONVOLVE, spectral gradient -i k
 * (Nyquist planes zeroed), inverse FFT per axis, CIC interpolation back.
 * psr_p2p_forces + psr_pm_forces (PSR_PM_ACCUMULATE) is the total periodic
 * acceleration of the split, short range truncated at r_c.
 *
 * psr_pm_create - host: cuFFT plans for an n_pm^3 mesh (n_pm even, in
 *   [8, 1024]); cuFFT may allocate plan data here, never the FFT work area.
 *   Errors: PSR_E_ARG, PSR_E_NOMEM, PSR_E_CUDA.
 * psr_pm_scratch_bytes - host: scratch psr_pm_forces needs (about 28 n_pm^3
 *   bytes plus the cuFFT work area).
 * psr_pm_forces - device, asynchronous on cuda_stream, allocates nothing:
 *   d_pos   device, n x 3 FP64, any real values (wrapped into [0, L)); a
 *           particle with a non-finite coordinate deposits nothing and its
 *           output is left unchanged
 *   d_mass  device, n FP64, or NULL for equal masses 1/n
 *   box     L, r_s, G (r_c unused)
 *   flags   PSR_PM_ACCUMULATE: add to d_acc instead of overwriting it;
 *           PSR_PM_NO_DECONVOLVE: keep the CIC windows
 *   d_scratch device, >= psr_pm_scratch_bytes, 256-byte aligned, caller-owned
 *   d_acc   device, n x 3 FP32, original particle order
 *   Calls on one psr_pm must not overlap in time (they share its plans).
 *   Mass is deposited with FP32 atomics, so the result varies with the
 *   order of the additions at the level of FP32 rounding.
 *   Errors: PSR_E_ARG, PSR_E_WORKSPACE, PSR_E_CUDA.
 * psr_pm_free - host: destroy the plans (NULL is ignored).
 */
#define PSR_PM_ACCUMULATE 1
#define PSR_PM_NO_DECONVOLVE 2
typedef struct psr_pm psr_pm; /* opaque, host-owned */
int psr_pm_create(int n_pm, psr_pm** out);
int psr_pm_scratch_bytes(const psr_pm* pm, size_t* bytes);
int psr_pm_forces(psr_pm* pm, const double* d_pos, const double* d_mass, int64_t n,
                  const psr_box* box, int flags, void* d_scratch, size_t scratch_bytes,
                  float* d_acc, void* cuda_stream);
void psr_pm_free(psr_pm* pm);

/* ------------------------------------------- truncated multipole part */
/*
 * The truncated multipole operators of the PM-FMM short range (paper,
 * Section 2: P2M, M2L with the truncated prefactors f_(n), L2P).  Kernel
 * psi(r) = erfc(r / 2 r_s) / r, f_(k) = (1/r d/dr)^k psi from the paper's
 * closed form, derivative tensors D_n(R) = d^n psi(R) from the f_(k).
 * Cells are CSR ranges [first[c], first[c+1]) of a particle array.
 * Expansions to order p (1 <= p <= 6), multi-indices |n| <= p in graded
 * order (|n|, then n1 descending, then n2 descending), coefficients scaled
 * by a caller-chosen length h so that FP32 holds them (the cell size or r_s
 * are good choices; each M2L entry forms its derivatives at the scale |R|
 * and rescales by (h/|R|)^(|k|+1), so any h with (h/|R|)^(p+1) and
 * (|R|/h)^(p+1) inside the FP32 range works):
 *   Mh_m = sum_j m_j ((z_A - x_j)/h)^m / m!                       (P2M)
 *   Lh_n = sum_{|m| <= p-|n|} Mh_m h^(|n|+|m|+1) D_{n+m}(z_B - z_A) (M2L)
 *   a_c(x) = (G/h^2) sum_{|k| <= p-1} Lh_{k+e_c} ((x - z_B)/h)^k / k!  (L2P)
 * so that a(x) approximates G sum_j m_j grad psi(x - x_j) over the source
 * cells (the smooth truncated kernel, no hard cutoff).  All three are
 * asynchronous on cuda_stream and allocate nothing; FP32 coefficients.
 *
 * psr_fmm_ncoef - host: (p+1)(p+2)(p+3)/6 coefficients per cell.
 * psr_fmm_p2m - d_first (ncell+1) int64, d_pos n x 3 FP64, d_mass n FP64 or
 *   NULL for 1/n, d_centre ncell x 3 FP64 -> d_M ncell x ncoef FP32.
 * psr_fmm_m2l - target cells t: entries d_pairs[d_rowptr[t] .. d_rowptr[t+1])
 *   = (source cell << 5) | image code (nx+1)*9 + (ny+1)*3 + (nz+1), the source
 *   centre taken at c_s + n L (box->L); box->r_s sets the kernel.  Writes
 *   d_L ntarget x ncoef.  d_status (device uint32, may be NULL) gets bit 0
 *   for an entry out of range and bit 1 for coincident centres (both
 *   skipped).
 * psr_fmm_l2p - accelerations of the particles of each cell from its local
 *   coefficients, times box->G; PSR_FMM_ACCUMULATE adds into d_acc (n x 3
 *   FP32) instead of overwriting.
 * psr_fmm_forces - the far part of the short range on a psr_device_build_split
 *   handle (after psr_device_build_finish; the FP64 particle copy must be
 *   present): P2M on every leaf about its expansion centre, M2L over the
 *   far list, L2P on every leaf, with h = box r_s.  d_M and d_L: device
 *   scratch of n_leaves x ncoef4 FP32 each (ncoef rounded up to a multiple
 *   of 4: the rows load as float4), 16-byte aligned.  d_acc: n x 3 in the ORIGINAL
 *   particle order (as psr_p2p_forces), FP32, or FP64 with PSR_FMM_F64;
 *   PSR_FMM_ACCUMULATE adds into it (e.g. onto the near part from
 *   psr_p2p_forces).  d_status as for psr_fmm_m2l.
 *   Three launches, asynchronous, graph-capturable.
 * Errors: PSR_E_ARG (order, scale, NULL, counts, flags), PSR_E_STATE (not a
 * split handle with its workspace written and its FP64 copy), PSR_E_CUDA.
 */
#define PSR_FMM_ACCUMULATE 1
#define PSR_FMM_F64 2
int psr_fmm_ncoef(int p, int* ncoef);
int psr_fmm_p2m(int p, double h, int64_t n, int64_t ncell, const int64_t* d_first,
                const double* d_pos, const double* d_mass, const double* d_centre, float* d_M,
                void* cuda_stream);
int psr_fmm_m2l(int p, double h, const psr_box* box, int64_t ntarget, int64_t nsource,
                const int64_t* d_rowptr, const uint32_t* d_pairs, const double* d_centre_t,
                const double* d_centre_s, const float* d_M, float* d_L, unsigned* d_status,
                void* cuda_stream);
int psr_fmm_l2p(int p, double h, const psr_box* box, int64_t ncell, const int64_t* d_first,
                const double* d_pos, const double* d_centre, const float* d_L, float* d_acc,
                int flags, void* cuda_stream);
int psr_fmm_forces(const psr_leaves* h, int p, int flags, float* d_M, float* d_L, void* d_acc,
                   unsigned* d_status, void* cuda_stream);

/* psr_free_leaves - host: free a handle (NULL is ignored). */
void psr_free_leaves(psr_leaves* h);

/* psr_last_error - message of the last failing call on this thread. */
const char* psr_last_error(void);

/* psr_version - library version string. */
const char* psr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSR_H */
