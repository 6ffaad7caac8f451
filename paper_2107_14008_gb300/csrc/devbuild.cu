// Device-side leaf and leaf-pair builder: the GPU counterpart of builder.cpp
// (paper, Section 2: contiguous leaves of at most MAXLEAF particles; Section
// 3.2: the task list grouped by target leaf, with start and length per leaf).
// It produces the arrays the host builder produces, bit for bit and in the
// same order:
//   1. keys      wrap positions into [0, L), 21-bit quantisation, 63-bit Morton key
//   2. sort      stable LSD radix sort of (key, index), 8 passes of 8 bits
//   3. leaves    a particle's leaf is its first ancestor cell, from the root, that
//                holds at most max_leaf particles; level-21 cells beyond max_leaf
//                are cut into chunks of max_leaf.  Since that cell contains the
//                particle and at most max_leaf particles, its extent is found by
//                binary searches inside a window of +-(max_leaf + 1) sorted keys.
//   4. tree      a binary radix tree over the leaf cell keys (Karras 2012, equal
//                keys ordered by leaf index) with bottom-up bounding boxes
//   5. pairs     per target leaf and periodic image, a depth-first traversal that
//                keeps every leaf whose box comes closer than r_c.  A node's box
//                contains its leaves' boxes, so the kept set is exactly the set of
//                leaves that pass the leaf test, which the host's octree keeps too;
//                the left-first order visits them in leaf order like the host's
//                Morton-ordered octree walk.  Counted in one pass, which also
//                stores each row in a pair cache of 16 words per particle; after
//                a prefix sum of the counts the cached rows are copied into
//                place and only the rows the cache could not hold are walked a
//                second time (the multipole split walks twice).  The walk prunes with
//                FP32 bounds (directed rounding) and falls back to the host's FP64
//                leaf test only where the bounds cannot decide (gap^2 within about
//                1e-5 of the cutoff): FP64 throughput on this part is 1/64 of FP32.
//   6. schedule  target leaves sorted by evaluated work, largest first (stable)
// The FP64 steps use the same operations as the host (no contraction).
//
// Two calls: psr_device_build runs 1-5 (counting) on the caller's scratch and
// reads back the sizes; psr_device_build_finish writes the workspace.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>

#include "kcommon.cuh"

namespace psr {

void set_last_error(const std::string& msg);

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per block
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 values per block
constexpr int64_t kScanMaxTiles = 65536;              // the top level scans in one block
constexpr int kStackDepth = 128;                      // tree depth <= 63 key + 27 index bits
constexpr int kDefaultTimeoutMs = 60000;
constexpr int64_t kMaxN = (int64_t)1 << 28;           // scan limit: 65536 tiles of 4096

// counters in the scratch (int64 words)
enum : int {
    kCntMaxLeaf = 0,
    kCntPairs = 1,
    kCntEvaluated = 2,
    kCntMaxCost = 3,
    kCntMaxRow = 4,
    kCntError = 5,  // bit 0 non-finite input, bit 1 stack overflow, bit 2 malformed tree
    kCntFar = 6,    // well-separated (M2L) entries of the multipole split
    kCntUncached = 7,  // rows the pair cache could not hold (re-walked by the write pass)
    kCntMassDiff = 8,  // nonzero if some particle's mass differs from particle 0's
    kCntMass0 = 9,     // particle 0's mass (the bits of a double)
    kCntWords = 10,
};

// The pair cache: the count walk also records each row as runs of
// consecutive leaves of one image (the first leaf with its image code, and the
// run length: 8 bytes, one run for about ten entries on clustered sets), in a
// slot of equal size per row, so that the write step expands the runs instead
// of walking the tree again.  A row with more runs than its slot holds is
// walked again instead; with slots below kMinRuns runs the cache is not used.
constexpr int kCacheWordsPerParticle = 16;
constexpr int kMinRuns = 16;

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch regions (byte offsets); leaf arrays are sized for n leaves (max_leaf 1).
struct Scratch {
    size_t wpos, key0, key1, val0, val1, flag, lid, lfirst, llevel, lkey, lbox, lrec, lcnt,
        lfar, lout, lcost, tnode, tspan, tparl, tpari, tbox, nodef, tflag, hist, tiles, total, cnt,
        lruns, cache, bytes;
    int64_t ncache;  // pair cache capacity in runs
};

Scratch scratch_layout(int64_t n)
{
    Scratch s{};
    size_t o = 0;
    const size_t N = (size_t)(n > 0 ? n : 1);
    const size_t nb = (N + kSortTile - 1) / kSortTile;
    const size_t hist = 256 * nb;
    const size_t big = hist > N + 1 ? hist : N + 1;  // longest scanned array
    const size_t ntiles = (big + kScanTile - 1) / kScanTile;
    s.wpos = o;   o = a256(o + 32 * N);  // x, y, z, m (wrapped, FP64)
    s.key0 = o;   o = a256(o + 8 * N);
    s.key1 = o;   o = a256(o + 8 * N);
    s.val0 = o;   o = a256(o + 4 * N);
    s.val1 = o;   o = a256(o + 4 * N);
    s.flag = o;   o = a256(o + 8 * N);
    s.lid = o;    o = a256(o + 8 * N);
    s.lfirst = o; o = a256(o + 4 * (N + 1));
    s.llevel = o; o = a256(o + 4 * N);
    s.lkey = o;   o = a256(o + 8 * N);
    s.lbox = o;   o = a256(o + 48 * N);
    s.lrec = o;   o = a256(o + 32 * N);  // FP32 inward leaf box and count
    s.lcnt = o;   o = a256(o + 8 * N);
    s.lfar = o;   o = a256(o + 8 * N);   // far entries per leaf (multipole split)
    s.lout = o;   o = a256(o + 32 * N);  // FP32 leaf box rounded outward (multipole split)
    s.lcost = o;  o = a256(o + 8 * N);
    s.tnode = o;  o = a256(o + 8 * N);
    s.tspan = o;  o = a256(o + 8 * N);   // leaf range [lo, hi] of each internal node
    s.tparl = o;  o = a256(o + 4 * N);
    s.tpari = o;  o = a256(o + 4 * N);
    s.tbox = o;   o = a256(o + 48 * N);
    s.nodef = o;  o = a256(o + 64 * N);  // internal nodes: children and their FP32 boxes
    s.tflag = o;  o = a256(o + 4 * N);
    s.hist = o;   o = a256(o + 8 * hist);
    s.tiles = o;  o = a256(o + 8 * ntiles);
    s.total = o;  o = a256(o + 8);
    s.cnt = o;    o = a256(o + 8 * kCntWords);
    s.lruns = o;  o = a256(o + 4 * N);   // runs cached per row (-1: not cached)
    s.ncache = (int64_t)(kCacheWordsPerParticle / 2 * N);
    s.cache = o;  o = a256(o + 8 * (size_t)s.ncache);  // uint2 (first leaf << 5 | code, length)
    s.bytes = o;
    return s;
}

struct BoxK {
    double L, scale, unit, inv2rs, rc2m;  // rc2m = r_c^2 (1 + 1e-5), the host's margin
    float thi, tlo;  // FP32 thresholds: thi >= rc2m (1 + 1e-6), tlo <= rc2m (1 - 1e-6)
    float theta2;    // multipole split: theta^2 (0: no split)
    float gt2;       //   and theta^2 (2 r_s^2)^2 (the Gaussian length of the kernel)
    float rc2far;    // FP32 at most r_c^2 (1 - 1e-6): a far pair lies wholly inside the cutoff
};

// ------------------------------------------------------------ utilities --

__device__ __forceinline__ uint64_t spread3_d(uint64_t v)
{
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

__device__ __forceinline__ uint32_t compact3_d(uint64_t v)
{
    v &= 0x1249249249249249ULL;
    v = (v | (v >> 2)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v >> 4)) & 0x100f00f00f00f00fULL;
    v = (v | (v >> 8)) & 0x1f0000ff0000ffULL;
    v = (v | (v >> 16)) & 0x1f00000000ffffULL;
    v = (v | (v >> 32)) & 0x1fffffULL;
    return (uint32_t)v;
}

// first index in [lo, hi) with a[index] >= x (hi if none)
__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t lo,
                                                   int64_t hi, uint64_t x)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// FP64 gap^2 between box A and box B shifted by sh, in the host builder's
// order of operations (explicit roundings: no contraction).
__device__ __forceinline__ double gap2_d(const double* A, const double* B, const double sh[3])
{
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double l = __dadd_rn(B[a], sh[a]), h = __dadd_rn(B[3 + a], sh[a]);
        const double g = fmax(0.0, fmax(__dsub_rn(l, A[3 + a]), __dsub_rn(A[a], h)));
        s = __dadd_rn(s, __dmul_rn(g, g));
    }
    return s;
}

// ------------------------------------------------------------------ scan --
// Exclusive prefix sum of int64 values: tile sums, one block scanning the tile
// sums, then tile scans with their offsets.  In-place use (in == out) is safe.

__global__ void __launch_bounds__(1024) k_scan_tiles(const int64_t* in, int64_t m,
                                                     int64_t* __restrict__ sums)
{
    __shared__ int64_t red[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < m) v += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// Block-wide exclusive scan of one value per thread (blockDim.x == 1024);
// returns the block total.
__device__ int64_t block_exclusive(int64_t v, int64_t* ex, int64_t* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int64_t s = sh[lane];
        int64_t si = s;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, si, o);
            if (lane >= o) si += t;
        }
        sh[lane] = si - s;
        if (lane == 31) sh[32] = si;
    }
    __syncthreads();
    *ex = inc - v + sh[w];
    const int64_t total = sh[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(1024) k_scan_top(int64_t* __restrict__ sums, int64_t nt,
                                                   int64_t* __restrict__ total)
{
    __shared__ int64_t sh[33];
    const int64_t per = (nt + kScanThreads - 1) / kScanThreads;
    const int64_t b = (int64_t)threadIdx.x * per, e = b + per < nt ? b + per : nt;
    int64_t v = 0;
    for (int64_t k = b; k < e; ++k) v += sums[k];
    int64_t ex;
    const int64_t t = block_exclusive(v, &ex, sh);
    for (int64_t k = b; k < e; ++k) {
        const int64_t c = sums[k];
        sums[k] = ex;
        ex += c;
    }
    if (threadIdx.x == 0) *total = t;
}

__global__ void __launch_bounds__(1024) k_scan_apply(const int64_t* in, int64_t m,
                                                     const int64_t* __restrict__ sums, int64_t* out)
{
    __shared__ int64_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems], v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = base + k < m ? in[base + k] : 0;
        v += loc[k];
    }
    int64_t ex;
    block_exclusive(v, &ex, sh);
    ex += sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < m) out[base + k] = ex;
        ex += loc[k];
    }
}

int scan_exclusive(const int64_t* in, int64_t* out, int64_t m, int64_t* tiles, int64_t* total,
                   cudaStream_t st)
{
    const int64_t nt = (m + kScanTile - 1) / kScanTile;
    if (nt > kScanMaxTiles) return (int)cudaErrorInvalidValue;
    if (nt == 0) return (int)cudaMemsetAsync(total, 0, 8, st);
    k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, st>>>(in, m, tiles);
    k_scan_top<<<1, kScanThreads, 0, st>>>(tiles, nt, total);
    k_scan_apply<<<(unsigned)nt, kScanThreads, 0, st>>>(in, m, tiles, out);
    return (int)cudaGetLastError();
}

// ------------------------------------------------------------ radix sort --
// Stable LSD radix sort of (64-bit key, int32 value), 8 bits per pass.  Per
// pass: digit counts per tile (digit-major), their exclusive scan, and a
// stable scatter: item t of a tile is w*256 + it*32 + lane, ranked warp by
// warp, iteration by iteration and lane by lane, i.e. in item order.

__device__ __forceinline__ int64_t tile_item(int w, int it, int lane)
{
    return (int64_t)w * (kSortItems * 32) + it * 32 + lane;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys,
                                                             int64_t n, int shift,
                                                             int64_t* __restrict__ hist,
                                                             int64_t nblocks)
{
    __shared__ unsigned cnt[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int it = 0; it < kSortItems; ++it) {
        const int64_t j = base + tile_item(w, it, lane);
        if (j < n) atomicAdd(&cnt[(keys[j] >> shift) & 255], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x)
        hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    int32_t* __restrict__ vout, int64_t n, int shift, const int64_t* __restrict__ off,
    int64_t nblocks)
{
    __shared__ unsigned whist[kSortThreads / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) whist[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    uint64_t key[kSortItems];
    int32_t val[kSortItems];
    unsigned rank[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int64_t j = base + tile_item(w, it, lane);
        const bool ok = j < n;
        key[it] = ok ? kin[j] : 0;
        val[it] = ok ? vin[j] : 0;
        const unsigned d = ok ? (unsigned)((key[it] >> shift) & 255) : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        rank[it] = ok ? whist[w][d] + __popc(peers & lt) : 0u;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) whist[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {  // exclusive over warps, per digit
        unsigned s = 0;
        for (int k = 0; k < kSortThreads / 32; ++k) {
            const unsigned c = whist[k][d];
            whist[k][d] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int64_t j = base + tile_item(w, it, lane);
        if (j < n) {
            const unsigned d = (unsigned)((key[it] >> shift) & 255);
            const int64_t pos = off[(int64_t)d * nblocks + blockIdx.x] + whist[w][d] + rank[it];
            kout[pos] = key[it];
            vout[pos] = val[it];
        }
    }
}

// Sorts on bits [0, bits) of the keys (bits <= 64); the result ends in (k0, v0).
int radix_sort(uint64_t* k0, int32_t* v0, uint64_t* k1, int32_t* v1, int64_t n, int bits,
               int64_t* hist, int64_t* tiles, int64_t* total, cudaStream_t st)
{
    if (n <= 1) return 0;
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    int passes = (bits + 7) / 8;
    if (passes & 1) ++passes;  // an even count leaves the result in (k0, v0); <= 8
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        uint64_t* ki = (p & 1) ? k1 : k0;
        int32_t* vi = (p & 1) ? v1 : v0;
        uint64_t* ko = (p & 1) ? k0 : k1;
        int32_t* vo = (p & 1) ? v0 : v1;
        k_radix_hist<<<(unsigned)nb, kSortThreads, 0, st>>>(ki, n, shift, hist, nb);
        int e = scan_exclusive(hist, hist, 256 * nb, tiles, total, st);
        if (e) return e;
        k_radix_scatter<<<(unsigned)nb, kSortThreads, 0, st>>>(ki, vi, ko, vo, n, shift, hist, nb);
        if ((e = (int)cudaGetLastError())) return e;
    }
    return 0;
}

// -------------------------------------------------------- keys and leaves --

__global__ void k_keys(const double* __restrict__ pos, const double* __restrict__ mass, int64_t n,
                       BoxK bx, double* __restrict__ wpos, uint64_t* __restrict__ key,
                       int32_t* __restrict__ idx, long long* __restrict__ cnt)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t q[3];
    bool bad = false;
    for (int a = 0; a < 3; ++a) {
        double v = pos[3 * i + a];
        if (!isfinite(v)) {
            bad = true;
            v = 0.0;
        }
        if (!(v >= 0.0 && v < bx.L)) {  // fmod is exact, so values inside [0, L) keep their bits
            v = fmod(v, bx.L);
            if (v < 0) v += bx.L;
            if (!(v < bx.L)) v = 0.0;
        }
        wpos[4 * i + a] = v;
        double qq = floor(__dmul_rn(v, bx.scale));
        if (qq < 0) qq = 0;
        if (qq > (double)((1u << kMortonBits) - 1)) qq = (double)((1u << kMortonBits) - 1);
        q[a] = (uint64_t)qq;
    }
    double m = mass ? mass[i] : 1.0 / (double)n;
    if (!isfinite(m)) {
        bad = true;
        m = 0.0;
    }
    wpos[4 * i + 3] = m;
    if (bad) atomicOr((unsigned long long*)(cnt + kCntError), 1ULL);
    // one mass for every particle lets the FP32 kernels apply it once per target
    const double m0 = mass ? mass[0] : 1.0 / (double)n;
    if (m != m0) atomicOr((unsigned long long*)(cnt + kCntMassDiff), 1ULL);
    if (i == 0) cnt[kCntMass0] = __double_as_longlong(m);
    key[i] = (spread3_d(q[0]) << 2) | (spread3_d(q[1]) << 1) | spread3_d(q[2]);
    idx[i] = (int32_t)i;
}

__device__ __forceinline__ uint64_t cell_prefix(uint64_t k, int level)
{
    const int sh = 3 * (kMortonBits - level);
    return sh >= 64 ? 0ULL : (k >> sh) << sh;
}

// [a, b) = the sorted indices of i's level-`level` cell, searched in [lo, hi)
__device__ __forceinline__ void cell_range(const uint64_t* __restrict__ key, int64_t i, int level,
                                           int64_t lo, int64_t hi, int64_t& a, int64_t& b)
{
    const int sh = 3 * (kMortonBits - level);
    const uint64_t p = cell_prefix(key[i], level);
    a = lower_bound_u64(key, lo, i, p);
    b = sh >= 63 ? hi : lower_bound_u64(key, i + 1, hi, p + (1ULL << sh));
}

// Leaf level and leaf-start flag of each sorted particle.  In the window
// [i - max_leaf - 1, i + max_leaf + 2) a cell's clipped count exceeds
// max_leaf exactly when its full count does, and is exact when it does not.
__global__ void k_leaf_level(const uint64_t* __restrict__ key, int64_t n, int max_leaf,
                             int64_t* __restrict__ flag, int32_t* __restrict__ level)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t lo = i - max_leaf - 1 > 0 ? i - max_leaf - 1 : 0;
    const int64_t hi = i + max_leaf + 2 < n ? i + max_leaf + 2 : n;
    int64_t a, b;
    cell_range(key, i, kMortonBits, lo, hi, a, b);
    bool start;
    int L;
    if (b - a > max_leaf) {  // over-full finest cell: chunks of max_leaf from its start
        L = kMortonBits;
        const int64_t a0 = lower_bound_u64(key, 0, i, key[i]);
        start = ((i - a0) % max_leaf) == 0;
    } else {  // smallest level whose cell holds at most max_leaf (counts fall with level)
        int l0 = 0, l1 = kMortonBits;
        while (l0 < l1) {
            const int mid = (l0 + l1) >> 1;
            cell_range(key, i, mid, lo, hi, a, b);
            if (b - a <= max_leaf) l1 = mid;
            else l0 = mid + 1;
        }
        L = l0;
        cell_range(key, i, L, lo, hi, a, b);
        start = i == a;
    }
    flag[i] = start ? 1 : 0;
    level[i] = L;
}

__global__ void k_leaf_fill(const int64_t* __restrict__ flag, const int64_t* __restrict__ lid,
                            const int32_t* __restrict__ level, const uint64_t* __restrict__ key,
                            int64_t n, int32_t* __restrict__ lfirst, int32_t* __restrict__ llevel,
                            uint64_t* __restrict__ lkey)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == n - 1) lfirst[lid[i] + flag[i]] = (int32_t)n;  // lfirst[nl] = n
    if (i >= n || !flag[i]) return;
    const int64_t g = lid[i];
    lfirst[g] = (int32_t)i;
    llevel[g] = level[i];
    lkey[g] = cell_prefix(key[i], level[i]);
}

// Leaf packing (the host builder's rule): consecutive sibling leaves (the
// same level L >= 1 and the same parent cell; chunks of an over-full finest
// cell excluded) share one leaf while their total stays within max_leaf,
// taken greedily in Morton order.  A pack of several leaves takes the
// parent's cell (its level; its key stays that of its first member, whose
// top bits name the parent), a pack of one keeps its own.  The first leaf of each run of
// siblings (at most 8) packs the run: pstart[g] = 1 where a pack begins,
// psize[g] = the leaves of the pack that begins at g.
__device__ __forceinline__ bool packable(const int32_t* __restrict__ llevel,
                                         const uint64_t* __restrict__ lkey, int64_t nl, int64_t g)
{
    const int L = llevel[g];
    if (L < 1) return false;
    if (L == kMortonBits)  // a chunk of an over-full finest cell shares its key with a neighbour
        return !((g > 0 && llevel[g - 1] == L && lkey[g - 1] == lkey[g]) ||
                 (g + 1 < nl && llevel[g + 1] == L && lkey[g + 1] == lkey[g]));
    return true;
}

__device__ __forceinline__ bool siblings(const int32_t* __restrict__ llevel,
                                         const uint64_t* __restrict__ lkey, int64_t nl, int64_t g)
{
    const int L = llevel[g];
    return g > 0 && llevel[g - 1] == L && packable(llevel, lkey, nl, g - 1) &&
           packable(llevel, lkey, nl, g) &&
           cell_prefix(lkey[g - 1], L - 1) == cell_prefix(lkey[g], L - 1);
}

__global__ void k_pack_mark(const int32_t* __restrict__ lfirst, const int32_t* __restrict__ llevel,
                            const uint64_t* __restrict__ lkey, int64_t nl, int max_leaf,
                            int64_t* __restrict__ pstart, int32_t* __restrict__ psize)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nl || siblings(llevel, lkey, nl, g)) return;  // not the first of its run
    int64_t start = g;
    int cnt = 0, k = 0;
    for (int64_t j = g; j < nl && (j == g || siblings(llevel, lkey, nl, j)); ++j) {
        const int c = lfirst[j + 1] - lfirst[j];
        if (j == g || cnt + c > max_leaf) {
            if (j > g) psize[start] = k;
            pstart[j] = 1;
            start = j;
            cnt = c;
            k = 1;
        } else {
            pstart[j] = 0;
            cnt += c;
            ++k;
        }
    }
    psize[start] = k;
}

__global__ void k_pack_fill(const int64_t* __restrict__ pstart, const int64_t* __restrict__ pid,
                            const int32_t* __restrict__ psize, const int32_t* __restrict__ lfirst,
                            const int32_t* __restrict__ llevel, const uint64_t* __restrict__ lkey,
                            int64_t nl, int32_t* __restrict__ lfirst2, int32_t* __restrict__ llevel2,
                            uint64_t* __restrict__ lkey2)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g == nl - 1) lfirst2[pid[g] + pstart[g]] = lfirst[nl];  // lfirst[packs] = n
    if (g >= nl || !pstart[g]) return;
    const int64_t p = pid[g];
    const bool multi = psize[g] > 1;
    lfirst2[p] = lfirst[g];
    llevel2[p] = multi ? llevel[g] - 1 : llevel[g];
    lkey2[p] = lkey[g];  // the first member's key keeps the keys sorted (an earlier,
                         // deeper sibling subtree can hold keys above the parent's prefix)
}

__global__ void k_leaf_box(const int32_t* __restrict__ lfirst, int64_t nl, int64_t n,
                           const double* __restrict__ wpos, const int32_t* __restrict__ idx,
                           double* __restrict__ lbox, float4* __restrict__ lrec,
                           float4* __restrict__ lout, long long* __restrict__ cnt)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nl) return;
    const int64_t f = lfirst[g], e = g + 1 < nl ? lfirst[g + 1] : n;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t k = f; k < e; ++k) {
        const int64_t p = idx[k];
        for (int a = 0; a < 3; ++a) {
            const double v = wpos[4 * p + a];
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    }
    for (int a = 0; a < 3; ++a) {
        lbox[6 * g + a] = lo[a];
        lbox[6 * g + 3 + a] = hi[a];
    }
    // walk record: the box rounded inward (lo up, hi down) and the count
    lrec[2 * g] = make_float4(__double2float_ru(lo[0]), __double2float_ru(lo[1]),
                              __double2float_ru(lo[2]), __int_as_float((int)(e - f)));
    lrec[2 * g + 1] = make_float4(__double2float_rd(hi[0]), __double2float_rd(hi[1]),
                                  __double2float_rd(hi[2]), 0.f);
    // the box rounded outward (lo down, hi up) and half its diagonal, for
    // the multipole split
    const float ol[3] = {__double2float_rd(lo[0]), __double2float_rd(lo[1]),
                         __double2float_rd(lo[2])};
    const float oh[3] = {__double2float_ru(hi[0]), __double2float_ru(hi[1]),
                         __double2float_ru(hi[2])};
    float r2 = 0.f;
    for (int a = 0; a < 3; ++a) {
        const float ea = __fmul_rn(0.5f, __fsub_rn(oh[a], ol[a]));
        r2 = __fmaf_rn(ea, ea, r2);
    }
    lout[2 * g] = make_float4(ol[0], ol[1], ol[2], 0.f);
    lout[2 * g + 1] = make_float4(oh[0], oh[1], oh[2], __fsqrt_rn(r2));
    atomicMax(cnt + kCntMaxLeaf, (long long)(e - f));
}

// ------------------------------------------------------------------ tree --
// Internal node i (0 <= i < nl - 1) of the binary radix tree over the sorted
// leaf cell keys, node 0 the root.  A child code with bit 31 set is a leaf.

constexpr int kLeafBit = (int)0x80000000u;

__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int64_t nl, int64_t i, int64_t j)
{
    if (j < 0 || j >= nl) return -1;
    const uint64_t a = k[i], b = k[j];
    if (a == b) return 64 + __clz((unsigned)(i ^ j));
    return __clzll(a ^ b);
}

__global__ void k_tree_nodes(const uint64_t* __restrict__ k, int64_t nl, int2* __restrict__ node,
                             int2* __restrict__ span, int32_t* __restrict__ parl,
                             int32_t* __restrict__ pari)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nl - 1) return;
    const int d = delta(k, nl, i, i + 1) > delta(k, nl, i, i - 1) ? 1 : -1;
    const int dmin = delta(k, nl, i, i - d);
    int64_t lmax = 2;
    while (delta(k, nl, i, i + lmax * d) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t t = lmax / 2; t >= 1; t /= 2)
        if (delta(k, nl, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(k, nl, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(k, nl, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int2 c;
    if (lo == gamma) {
        c.x = (int)gamma | kLeafBit;
        parl[gamma] = (int)i;
    } else {
        c.x = (int)gamma;
        pari[gamma] = (int)i;
    }
    if (hi == gamma + 1) {
        c.y = (int)(gamma + 1) | kLeafBit;
        parl[gamma + 1] = (int)i;
    } else {
        c.y = (int)(gamma + 1);
        pari[gamma + 1] = (int)i;
    }
    node[i] = c;
    span[i] = make_int2((int)lo, (int)hi);
    if (i == 0) pari[0] = -1;
}

__device__ __forceinline__ const double* child_box(int c, const double* lbox, const double* tbox)
{
    return c < 0 ? lbox + 6 * (int64_t)(c & 0x7fffffff) : tbox + 6 * (int64_t)c;
}

// Bottom-up boxes: of the two threads that reach a node, the second one
// (whose sibling subtree is then complete) computes it and moves up.
__global__ void k_tree_boxes(int64_t nl, const int2* __restrict__ node,
                             const int32_t* __restrict__ parl, const int32_t* __restrict__ pari,
                             const double* __restrict__ lbox, double* tbox, int* flags,
                             long long* cnt)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nl) return;
    int p = parl[g];
    for (int step = 0; p >= 0; ++step) {
        if (step > kStackDepth || p >= nl - 1) {
            atomicOr((unsigned long long*)(cnt + kCntError), 4ULL);
            return;
        }
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;
        __threadfence();
        const int2 c = node[p];
        const double* A = child_box(c.x, lbox, tbox);
        const double* B = child_box(c.y, lbox, tbox);
        for (int a = 0; a < 3; ++a) {
            tbox[6 * (int64_t)p + a] = fmin(__ldcg(A + a), __ldcg(B + a));
            tbox[6 * (int64_t)p + 3 + a] = fmax(__ldcg(A + 3 + a), __ldcg(B + 3 + a));
        }
        p = pari[p];
    }
}

// ----------------------------------------------------------------- pairs --
// Internal node i packed for the walk (64 bytes): its children's boxes in
// FP32 rounded outward (lo down, hi up) and their codes:
//   q[0] = (l.lo.x, l.lo.y, l.lo.z, l.hi.x)   q[1] = (l.hi.y, l.hi.z, r.lo.x, r.lo.y)
//   q[2] = (r.lo.z, r.hi.x, r.hi.y, r.hi.z)   q[3] = bits(left, right, lo, hi)
// where [lo, hi] is the node's leaf range: left covers [lo, gamma], right
// [gamma + 1, hi], gamma = the left child's index (leaf or internal).
__global__ void k_tree_pack(int64_t nl, const int2* __restrict__ node,
                            const int2* __restrict__ span, const double* __restrict__ lbox,
                            const double* __restrict__ tbox, float4* __restrict__ nodef)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nl - 1) return;
    const int2 c = node[i];
    const double* A = child_box(c.x, lbox, tbox);
    const double* B = child_box(c.y, lbox, tbox);
    float v[12];
    for (int a = 0; a < 3; ++a) {
        v[a] = __double2float_rd(A[a]);
        v[3 + a] = __double2float_ru(A[3 + a]);
        v[6 + a] = __double2float_rd(B[a]);
        v[9 + a] = __double2float_ru(B[3 + a]);
    }
    float4* q = nodef + 4 * i;
    q[0] = make_float4(v[0], v[1], v[2], v[3]);
    q[1] = make_float4(v[4], v[5], v[6], v[7]);
    q[2] = make_float4(v[8], v[9], v[10], v[11]);
    const int2 sp = span[i];
    q[3] = make_float4(__int_as_float(c.x), __int_as_float(c.y), __int_as_float(sp.x),
                       __int_as_float(sp.y));
}

// Bounds on the exact gap^2 between a target box A and a box B shifted by
// sh, in FP32 with every operation rounded toward the bound (shift given
// rounded down, sd, and up, su).  Lower bound: boxes rounded outward.
__device__ __forceinline__ float gap2_lower(const float* alo, const float* ahi, const float* blo,
                                            const float* bhi, const float* sd, const float* su)
{
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d1 = __fsub_rd(__fadd_rd(blo[a], sd[a]), ahi[a]);
        const float d2 = __fsub_rd(alo[a], __fadd_ru(bhi[a], su[a]));
        const float g = fmaxf(0.f, fmaxf(d1, d2));
        s = __fadd_rd(s, __fmul_rd(g, g));
    }
    return s;
}

// Upper bound: boxes rounded inward (lo up, hi down).
__device__ __forceinline__ float gap2_upper(const float* alo, const float* ahi, const float* blo,
                                            const float* bhi, const float* sd, const float* su)
{
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d1 = __fsub_ru(__fadd_ru(blo[a], su[a]), ahi[a]);
        const float d2 = __fsub_ru(alo[a], __fadd_rd(bhi[a], sd[a]));
        const float g = fmaxf(0.f, fmaxf(d1, d2));
        s = __fadd_ru(s, __fmul_ru(g, g));
    }
    return s;
}

// Upper bound on the largest gap^2 between A and any point of box B + sh,
// which bounds the gap^2 of every leaf inside B: B rounded outward, A
// rounded inward (alo up, ahi down).
__device__ __forceinline__ float maxgap2_upper(const float* alo, const float* ahi, const float* blo,
                                               const float* bhi, const float* sd, const float* su)
{
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float e1 = __fsub_ru(__fadd_ru(bhi[a], su[a]), ahi[a]);
        const float e2 = __fsub_ru(alo[a], __fadd_rd(blo[a], sd[a]));
        const float g = fmaxf(0.f, fmaxf(e1, e2));
        s = __fadd_ru(s, __fmul_ru(g, g));
    }
    return s;
}

// The multipole split: leaf J + shift is well separated from leaf I when
// every point of one box lies within r_c of every point of the other (a
// rigorous FP32 upper bound of the largest point-pair distance, from boxes
// rounded outward, against r_c^2 (1 - 1e-6) rounded down: the cutoff then
// removes no pair the expansion includes) and the box centres are R apart
// with theta |R| >= rho_I + rho_J (rho: half the diagonal of the outward
// box), and, with PSR_BUILD_SPLIT_GAUSSIAN, also theta 2 r_s^2 / |R| >=
// rho_I + rho_J: 2 r_s^2 / |R| is the length on which the kernel's Gaussian
// truncation varies (d/dR of -R^2 / 4 r_s^2), shorter than |R| beyond
// r = sqrt(2) r_s (gt2 = theta^2 (2 r_s^2)^2, or infinity without the flag).
// The opening test is taken in FP32 with explicit roundings so that the
// count and the write pass decide alike.
// alo/ahi, ra: box I and its rho; b0 = (lo of box J), b1 = (hi of box J,
// rho_J); sd/su: the shift rounded down and up.
__device__ __forceinline__ bool far_pair(const float* alo, const float* ahi, float ra, float4 b0,
                                         float4 b1, const float* sd, const float* su,
                                         float theta2, float gt2, float rc2far)
{
    const float blo[3] = {b0.x, b0.y, b0.z}, bhi[3] = {b1.x, b1.y, b1.z};
    float m2 = 0.f, d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float bl = __fadd_rd(blo[a], sd[a]), bh = __fadd_ru(bhi[a], su[a]);
        const float mx = fmaxf(__fsub_ru(bh, alo[a]), __fsub_ru(ahi[a], bl));
        m2 = __fmaf_ru(mx, mx, m2);
        const float d = __fsub_rn(__fmul_rn(0.5f, __fadd_rn(bl, bh)),
                                  __fmul_rn(0.5f, __fadd_rn(alo[a], ahi[a])));
        d2 = __fmaf_rn(d, d, d2);
    }
    const float r = __fadd_rn(ra, b1.w);
    const float r2 = __fmul_rn(r, r);
    return d2 > 0.f && m2 < rc2far && __fmul_rn(theta2, d2) >= r2 && __fmul_rn(r2, d2) <= gt2;
}

// One thread per target leaf.  WRITE = false counts the row and its work
// and, given a pair cache of kslot runs per row, records the row's runs there
// in walk order (lruns[I]: their number, or -1 when the slot is too small);
// WRITE = true writes the row at rowptr, skipping the rows a given lruns
// marks as cached (k_pairs_expand writes those).
// Row order: a warp takes 32 consecutive leaves (neighbours, whose walks
// share most of their paths), or, with interleave, lane k of warp w takes
// leaf k W + w (W = ceil(n_leaves / 32)).  When every row fits in one wave of
// resident warps the launch lasts as long as its slowest warp, a warp of 32
// leaves of the densest region walking one after another where their paths
// part; spread over 32 warps those walks run side by side (the bench
// workload's count walk: 2.79 against 3.02 ms per build).  With more rows
// than that the launch is bound by the total work, and the neighbours'
// shared paths win (8-particle leaves: 9.3 against 11.2 ms).  Nodes are pruned when the FP32
// lower bound of their gap^2 reaches thi (then the host's FP64 test fails
// for every leaf below); a leaf is kept when the FP32 upper bound is below
// tlo (then the host's FP64 test passes); only the leaves in between take
// the host's FP64 test itself.  The walk keeps its current node in a
// register and stacks a right child only while it descends the left one.
// Each walk visits at most 2 nl - 1 nodes; more means a malformed tree,
// reported, never looped on.
template <bool WRITE>
__global__ void __launch_bounds__(128, 8) k_pairs(
    int64_t nl, int64_t n, BoxK bx, const int32_t* __restrict__ lfirst,
    const double* __restrict__ lbox, const float4* __restrict__ lrec,
    const float4* __restrict__ nodef, const double* __restrict__ rootbox,
    int64_t* __restrict__ lcnt, int64_t* __restrict__ lcost, const int64_t* __restrict__ rowptr,
    uint32_t* __restrict__ pairs, long long* __restrict__ cnt, unsigned* __restrict__ err,
    int32_t* __restrict__ lruns, uint2* __restrict__ cache, int kslot, int interleave)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t W = (nl + 31) >> 5;
    const int64_t I = !interleave ? t : (t >> 5) < W ? (t & 31) * W + (t >> 5) : nl;
    if (I >= nl) return;
    if (WRITE && lruns && lruns[I] >= 0) return;
    double A[6];
    float aolo[3], aohi[3], ailo[3], aihi[3], rlo[3], rhi[3];
    for (int a = 0; a < 3; ++a) {
        A[a] = lbox[6 * I + a];
        A[3 + a] = lbox[6 * I + 3 + a];
        aolo[a] = __double2float_rd(A[a]);
        aohi[a] = __double2float_ru(A[3 + a]);
        ailo[a] = __double2float_ru(A[a]);
        aihi[a] = __double2float_rd(A[3 + a]);
        rlo[a] = __double2float_rd(rootbox[a]);
        rhi[a] = __double2float_ru(rootbox[3 + a]);
    }
    // stack entries: (node code, -1) or a leaf range (first, last) kept whole
    int2 stack[kStackDepth];
    int64_t c = 0, src = 0;
    int64_t w = WRITE ? rowptr[I] : 0;
    const int64_t wend = WRITE ? rowptr[I + 1] : 0;
    bool bad = false;
    // pair cache state: the open run (first entry word, length) and the runs
    // stored so far in this row's slot
    const bool caching = !WRITE && cache != nullptr;
    bool cok = caching;
    uint2* const slot = caching ? cache + I * (int64_t)kslot : nullptr;
    uint32_t run0 = 0, runn = 0;
    int nrun = 0;
    // keeps leaves [f, l] of this image
    auto take = [&](int f, int l, int code) {
        c += l - f + 1;
        src += lfirst[l + 1] - lfirst[f];
        if (WRITE) {
            if (w + (l - f + 1) > wend) {
                atomicOr(err, 4u);
                bad = true;
                return;
            }
            for (int J = f; J <= l; ++J) pairs[w++] = ((uint32_t)J << 5) | (uint32_t)code;
        } else if (cok) {
            const uint32_t e0 = ((uint32_t)f << 5) | (uint32_t)code;
            if (runn > 0 && e0 == run0 + (runn << 5)) {  // continues the open run
                runn += (uint32_t)(l - f + 1);
            } else {
                if (runn > 0) {
                    if (nrun == kslot) {
                        cok = false;
                        return;
                    }
                    slot[nrun++] = make_uint2(run0, runn);
                }
                run0 = e0;
                runn = (uint32_t)(l - f + 1);
            }
        }
    };
    for (int code = 0; code < kShiftCodes && !bad; ++code) {
        const double sh[3] = {(code / 9 - 1) * bx.L, ((code / 3) % 3 - 1) * bx.L,
                              (code % 3 - 1) * bx.L};
        float sd[3], su[3];
        for (int a = 0; a < 3; ++a) {
            sd[a] = __double2float_rd(sh[a]);
            su[a] = __double2float_ru(sh[a]);
        }
        if (gap2_lower(aolo, aohi, rlo, rhi, sd, su) >= bx.thi) continue;
        if (maxgap2_upper(ailo, aihi, rlo, rhi, sd, su) < bx.tlo) {
            take(0, (int)nl - 1, code);
            continue;
        }
        int sp = 0;
        int2 cur = make_int2(nl >= 2 ? 0 : kLeafBit, -1);
        int64_t visits = 0;
        for (;;) {
            if (++visits > 2 * nl) {
                atomicOr(err, 4u);
                bad = true;
                break;
            }
            int2 next = make_int2(0, -2);  // y == -2: take the next stacked entry
            if (cur.y >= 0) {  // a whole leaf range deferred behind a left subtree
                take(cur.x, cur.y, code);
            } else if (cur.x < 0) {  // a leaf that passed the lower-bound test
                const int J = cur.x & 0x7fffffff;
                const float4 r0 = lrec[2 * (int64_t)J], r1 = lrec[2 * (int64_t)J + 1];
                const float bi_lo[3] = {r0.x, r0.y, r0.z}, bi_hi[3] = {r1.x, r1.y, r1.z};
                if (gap2_upper(ailo, aihi, bi_lo, bi_hi, sd, su) < bx.tlo ||
                    gap2_d(A, lbox + 6 * (int64_t)J, sh) < bx.rc2m)
                    take(J, J, code);
            } else {
                const float4* q = nodef + 4 * (int64_t)cur.x;
                const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
                const float llo[3] = {q0.x, q0.y, q0.z}, lhi[3] = {q0.w, q1.x, q1.y};
                const float blo[3] = {q1.z, q1.w, q2.x}, bhi[3] = {q2.y, q2.z, q2.w};
                const int lc = __float_as_int(q3.x), rc = __float_as_int(q3.y);
                const int lo = __float_as_int(q3.z), hi = __float_as_int(q3.w);
                const int gamma = lc & 0x7fffffff;
                const bool pl = gap2_lower(aolo, aohi, llo, lhi, sd, su) < bx.thi;
                const bool pr = gap2_lower(aolo, aohi, blo, bhi, sd, su) < bx.thi;
                const bool fl = pl && maxgap2_upper(ailo, aihi, llo, lhi, sd, su) < bx.tlo;
                const bool fr = pr && maxgap2_upper(ailo, aihi, blo, bhi, sd, su) < bx.tlo;
                if (fl) take(lo, gamma, code);
                if (pl && !fl) {  // the left child needs a visit; the right one waits
                    if (pr) {
                        if (sp >= kStackDepth) {
                            atomicOr(err, 2u);
                            bad = true;
                            break;
                        }
                        stack[sp++] = fr ? make_int2(gamma + 1, hi) : make_int2(rc, -1);
                    }
                    next = make_int2(lc, -1);
                } else if (fr) {
                    take(gamma + 1, hi, code);
                } else if (pr) {
                    next = make_int2(rc, -1);
                }
            }
            if (bad) break;
            if (next.y != -2) {
                cur = next;
            } else if (sp > 0) {
                cur = stack[--sp];
            } else {
                break;
            }
        }
    }
    if (WRITE && !bad && w != wend) atomicOr(err, 4u);
    if (!WRITE) {
        const int64_t nI = lfirst[I + 1] - lfirst[I];
        lcnt[I] = c;
        lcost[I] = src * nI;
        if (caching) {
            if (cok && runn > 0) {
                if (nrun == kslot)
                    cok = false;
                else
                    slot[nrun++] = make_uint2(run0, runn);
            }
            lruns[I] = cok ? nrun : -1;
            if (!cok) atomicAdd((unsigned long long*)(cnt + kCntUncached), 1ULL);
        }
        atomicAdd((unsigned long long*)(cnt + kCntPairs), (unsigned long long)c);
        atomicAdd((unsigned long long*)(cnt + kCntEvaluated), (unsigned long long)(src * nI));
        atomicMax(cnt + kCntMaxCost, (long long)(src * nI));
        atomicMax(cnt + kCntMaxRow, (long long)c);
    }
}

// Writes the cached rows at rowptr.  One warp per row: lane k loads run k of
// a group of 32 (one coalesced load), a warp scan of the run lengths gives
// each run's first entry, and the group's entries are written 32 at a time,
// entry e finding its run by a binary search over the lanes (shuffles).  A
// run list that does not add up to the row's length (a corrupt cache) sets
// error bit 4.
__global__ void __launch_bounds__(256) k_pairs_expand(int64_t nl, const int32_t* __restrict__ lruns,
                                                      const uint2* __restrict__ cache, int kslot,
                                                      const int64_t* __restrict__ rowptr,
                                                      uint32_t* __restrict__ pairs,
                                                      unsigned* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t I = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); I < nl; I += nw) {
        const int nrun = lruns[I];
        if (nrun <= 0) continue;  // empty, or walked by the write pass
        const uint2* slot = cache + I * (int64_t)kslot;
        const int64_t row0 = rowptr[I], len = rowptr[I + 1] - row0;
        int64_t done = 0;  // entries of the earlier groups
        bool bad = false;
        for (int r0 = 0; r0 < nrun; r0 += 32) {
            const int nv = nrun - r0 < 32 ? nrun - r0 : 32;
            const uint2 run = lane < nv ? slot[r0 + lane] : make_uint2(0u, 0u);
            int64_t inc = run.y;  // inclusive scan of the run lengths
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t v = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += v;
            }
            const int64_t tot = __shfl_sync(kFull, inc, 31);
            const int64_t exc = inc - run.y;
            if (done + tot > len) {
                bad = true;
                break;
            }
            for (int64_t e0 = 0; e0 < tot; e0 += 32) {
                const int64_t e = e0 + lane;
                int lo = 0;  // the last run whose first entry is <= e
                for (int step = 16; step > 0; step >>= 1) {
                    const int cand = lo + step;
                    const int64_t v = __shfl_sync(kFull, exc, cand & 31);
                    if (cand < nv && v <= e) lo = cand;
                }
                const uint32_t x = __shfl_sync(kFull, run.x, lo);
                const int64_t first = __shfl_sync(kFull, exc, lo);
                if (e < tot) pairs[row0 + done + e] = x + ((uint32_t)(e - first) << 5);
            }
            done += tot;
        }
        if ((bad || done != len) && lane == 0) atomicOr(err, 4u);
    }
}

// The walk of k_pairs with the multipole split.  A lane's walk does not
// classify the leaves it keeps: it queues the kept ranges (first, last,
// image) in shared memory, and whenever a lane's queue is nearly full, or
// every lane's walk has ended, the warp classifies all queued ranges of all
// its lanes as one list, 32 source leaves per step (far_pair then runs with
// every lane busy, where inside a divergent walk it ran one lane at a time),
// and counts or writes the near and far entries of each owning row in walk
// order.  Every lane runs the same number of flushes (lanes past the last
// leaf have ended from the start), so the warp-wide steps see all 32 lanes.
// With a pair cache the count pass also records each row's queued ranges as
// runs (as k_pairs does), and the write pass replays a recorded row's runs
// into the queue instead of walking it again (lruns[I] >= 0).  Rows are
// interleaved over the warps as in k_pairs (here 6.33 -> 5.57 ms per split
// build on the bench workload: a warp runs until its slowest lane is done).
constexpr int kSplitQ = 8;  // queued ranges per lane (a walk step queues at most 2)

template <bool WRITE>
__global__ void __launch_bounds__(128, 4) k_pairs_split(
    int64_t nl, BoxK bx, const int32_t* __restrict__ lfirst, const double* __restrict__ lbox,
    const float4* __restrict__ lrec, const float4* __restrict__ lout,
    const float4* __restrict__ nodef, const double* __restrict__ rootbox,
    int64_t* __restrict__ lcnt, int64_t* __restrict__ lcost, int64_t* __restrict__ lfar,
    const int64_t* __restrict__ rowptr, uint32_t* __restrict__ pairs,
    const int64_t* __restrict__ frowptr, uint32_t* __restrict__ fpairs,
    long long* __restrict__ cnt, unsigned* __restrict__ err, int32_t* __restrict__ lruns,
    uint2* __restrict__ cache, int kslot, int interleave)
{
    constexpr int kQ = kSplitQ, kSlots = 32 * kSplitQ, kWarps = 4;
    __shared__ int4 sq[kWarps][kSlots];            // (first, last, image, owning lane)
    __shared__ long long spre[kWarps][kSlots];     // leaves queued before each slot
    __shared__ float4 sbox[kWarps][32][2];         // owning lane's box rounded outward, rho
    __shared__ long long sw[kWarps][32], sfw[kWarps][32];    // write positions
    __shared__ long long swe[kWarps][32], sfwe[kWarps][32];  // row ends
    __shared__ long long sc[kWarps][32], scf[kWarps][32], ssrc[kWarps][32];  // counts
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t W = (nl + 31) >> 5;
    const int64_t I = !interleave ? t : (t >> 5) < W ? (t & 31) * W + (t >> 5) : nl;
    const bool live = I < nl;
    double A[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    float aolo[3] = {0.f, 0.f, 0.f}, aohi[3] = {0.f, 0.f, 0.f};
    float ailo[3] = {0.f, 0.f, 0.f}, aihi[3] = {0.f, 0.f, 0.f};
    float rlo[3] = {0.f, 0.f, 0.f}, rhi[3] = {0.f, 0.f, 0.f};
    sbox[wp][lane][0] = sbox[wp][lane][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    sw[wp][lane] = sfw[wp][lane] = swe[wp][lane] = sfwe[wp][lane] = 0;
    sc[wp][lane] = scf[wp][lane] = ssrc[wp][lane] = 0;
    if (live) {
        for (int a = 0; a < 3; ++a) {
            A[a] = lbox[6 * I + a];
            A[3 + a] = lbox[6 * I + 3 + a];
            aolo[a] = __double2float_rd(A[a]);
            aohi[a] = __double2float_ru(A[3 + a]);
            ailo[a] = __double2float_ru(A[a]);
            aihi[a] = __double2float_rd(A[3 + a]);
            rlo[a] = __double2float_rd(rootbox[a]);
            rhi[a] = __double2float_ru(rootbox[3 + a]);
        }
        sbox[wp][lane][0] = lout[2 * I];
        sbox[wp][lane][1] = lout[2 * I + 1];
        if (WRITE) {
            sw[wp][lane] = rowptr[I];
            swe[wp][lane] = rowptr[I + 1];
            sfw[wp][lane] = frowptr[I];
            sfwe[wp][lane] = frowptr[I + 1];
        }
    }
    __syncwarp();
    const float Lrd = __double2float_rd(bx.L), Lru = __double2float_ru(bx.L);
    int2 stack[kStackDepth];
    bool bad = false, done = !live, in_tree = false;
    int code = -1, sp = 0;
    int2 cur = make_int2(0, -1);
    int64_t visits = 0;
    float sd[3] = {0.f, 0.f, 0.f}, su[3] = {0.f, 0.f, 0.f};
    double sh[3] = {0.0, 0.0, 0.0};
    int4* myq = &sq[wp][lane * kQ];
    // pair cache: the count pass records runs (open run run0/runn), the write
    // pass replays a recorded row (nrun runs, the next one at ri)
    bool cok = !WRITE && live && cache != nullptr;
    const bool replay = WRITE && live && lruns != nullptr && lruns[I] >= 0;
    uint2* const slot = (cok || replay) ? cache + I * (int64_t)kslot : nullptr;
    uint32_t run0 = 0, runn = 0;
    int nrun = replay ? lruns[I] : 0, ri = 0;
    int nq = 0;
    auto push = [&](int f, int l, int c) {
        myq[nq++] = make_int4(f, l, c, lane);
        if (!cok) return;
        const uint32_t e0 = ((uint32_t)f << 5) | (uint32_t)c;
        if (runn > 0 && e0 == run0 + (runn << 5)) {
            runn += (uint32_t)(l - f + 1);
        } else {
            if (runn > 0) {
                if (nrun == kslot) {
                    cok = false;
                    return;
                }
                slot[nrun++] = make_uint2(run0, runn);
            }
            run0 = e0;
            runn = (uint32_t)(l - f + 1);
        }
    };
    for (;;) {
        // ---- walk (or replay) until the queue may not take another step's ranges
        nq = 0;
        while (!done && nq <= kQ - 2) {
            if (replay) {
                if (ri == nrun) {
                    done = true;
                    break;
                }
                const uint2 run = slot[ri++];
                const int f = (int)(run.x >> 5);
                myq[nq++] = make_int4(f, f + (int)run.y - 1, (int)(run.x & 31u), lane);
                continue;
            }
            if (!in_tree) {
                if (++code >= kShiftCodes) {
                    done = true;
                    break;
                }
                sh[0] = (code / 9 - 1) * bx.L;
                sh[1] = ((code / 3) % 3 - 1) * bx.L;
                sh[2] = (code % 3 - 1) * bx.L;
                for (int a = 0; a < 3; ++a) {
                    sd[a] = __double2float_rd(sh[a]);
                    su[a] = __double2float_ru(sh[a]);
                }
                if (gap2_lower(aolo, aohi, rlo, rhi, sd, su) >= bx.thi) continue;
                if (maxgap2_upper(ailo, aihi, rlo, rhi, sd, su) < bx.tlo) {
                    push(0, (int)nl - 1, code);
                    continue;
                }
                in_tree = true;
                sp = 0;
                cur = make_int2(nl >= 2 ? 0 : kLeafBit, -1);
                visits = 0;
            }
            if (++visits > 2 * nl) {
                atomicOr(err, 4u);
                bad = done = true;
                break;
            }
            int2 next = make_int2(0, -2);  // y == -2: take the next stacked entry
            if (cur.y >= 0) {  // a whole leaf range deferred behind a left subtree
                push(cur.x, cur.y, code);
            } else if (cur.x < 0) {  // a leaf that passed the lower-bound test
                const int J = cur.x & 0x7fffffff;
                const float4 r0 = lrec[2 * (int64_t)J], r1 = lrec[2 * (int64_t)J + 1];
                const float bi_lo[3] = {r0.x, r0.y, r0.z}, bi_hi[3] = {r1.x, r1.y, r1.z};
                if (gap2_upper(ailo, aihi, bi_lo, bi_hi, sd, su) < bx.tlo ||
                    gap2_d(A, lbox + 6 * (int64_t)J, sh) < bx.rc2m)
                    push(J, J, code);
            } else {
                const float4* qn = nodef + 4 * (int64_t)cur.x;
                const float4 q0 = qn[0], q1 = qn[1], q2 = qn[2], q3 = qn[3];
                const float llo[3] = {q0.x, q0.y, q0.z}, lhi[3] = {q0.w, q1.x, q1.y};
                const float blo[3] = {q1.z, q1.w, q2.x}, bhi[3] = {q2.y, q2.z, q2.w};
                const int lc = __float_as_int(q3.x), rc = __float_as_int(q3.y);
                const int lo = __float_as_int(q3.z), hi = __float_as_int(q3.w);
                const int gamma = lc & 0x7fffffff;
                const bool pl = gap2_lower(aolo, aohi, llo, lhi, sd, su) < bx.thi;
                const bool pr = gap2_lower(aolo, aohi, blo, bhi, sd, su) < bx.thi;
                const bool fl = pl && maxgap2_upper(ailo, aihi, llo, lhi, sd, su) < bx.tlo;
                const bool fr = pr && maxgap2_upper(ailo, aihi, blo, bhi, sd, su) < bx.tlo;
                if (fl) push(lo, gamma, code);
                if (pl && !fl) {  // the left child needs a visit; the right one waits
                    if (pr) {
                        if (sp >= kStackDepth) {
                            atomicOr(err, 2u);
                            bad = done = true;
                            break;
                        }
                        stack[sp++] = fr ? make_int2(gamma + 1, hi) : make_int2(rc, -1);
                    }
                    next = make_int2(lc, -1);
                } else if (fr) {
                    push(gamma + 1, hi, code);
                } else if (pr) {
                    next = make_int2(rc, -1);
                }
            }
            if (next.y != -2) {
                cur = next;
            } else if (sp > 0) {
                cur = stack[--sp];
            } else {
                in_tree = false;
            }
        }
        // ---- the warp classifies the queued ranges of all its lanes
        __syncwarp();
        long long mine = 0;  // leaves this lane queued
        for (int k = 0; k < nq; ++k) mine += (long long)myq[k].y - myq[k].x + 1;
        long long base = mine;  // inclusive scan over lanes, then exclusive
        for (int o = 1; o < 32; o <<= 1) {
            const long long v = __shfl_up_sync(kFull, base, o);
            if (lane >= o) base += v;
        }
        const long long total = __shfl_sync(kFull, base, 31);
        base -= mine;
        {
            long long run = base;
            for (int k = 0; k < kQ; ++k) {
                spre[wp][lane * kQ + k] = run;  // empty slots: zero-length, next lane's base
                if (k < nq) run += (long long)myq[k].y - myq[k].x + 1;
            }
        }
        __syncwarp();
        for (long long v0 = 0; v0 < total; v0 += 32) {
            const long long v = v0 + lane;
            const bool valid = v < total;
            int slot = 0;
            if (valid) {  // the last slot whose prefix is <= v
                int lo = 0, hi = kSlots - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (spre[wp][mid] <= v) lo = mid;
                    else hi = mid - 1;
                }
                slot = lo;
            }
            const int4 r = sq[wp][slot];
            const int owner = valid ? r.w : 32;
            const int J = r.x + (int)(v - spre[wp][slot]);
            bool far = false;
            int nsrc = 0;
            if (valid) {
                const int s3[3] = {r.z / 9 - 1, (r.z / 3) % 3 - 1, r.z % 3 - 1};
                float fd[3], fu[3];
                for (int a = 0; a < 3; ++a) {
                    fd[a] = s3[a] < 0 ? -Lru : (s3[a] > 0 ? Lrd : 0.f);
                    fu[a] = s3[a] < 0 ? -Lrd : (s3[a] > 0 ? Lru : 0.f);
                }
                const float4 b0 = sbox[wp][owner][0], b1 = sbox[wp][owner][1];
                const float alo[3] = {b0.x, b0.y, b0.z}, ahi[3] = {b1.x, b1.y, b1.z};
                far = far_pair(alo, ahi, b1.w, lout[2 * (int64_t)J], lout[2 * (int64_t)J + 1],
                               fd, fu, bx.theta2, bx.gt2, bx.rc2far);
                if (!WRITE && !far) nsrc = lfirst[J + 1] - lfirst[J];
            }
            const unsigned seg = __match_any_sync(kFull, owner);
            const unsigned fb = __ballot_sync(kFull, valid && far) & seg;
            const unsigned nb = __ballot_sync(kFull, valid && !far) & seg;
            const unsigned lt = (1u << lane) - 1u;
            const bool lead = valid && lane == __ffs(seg) - 1;
            if (WRITE && valid) {
                const uint32_t ent = ((uint32_t)J << 5) | (uint32_t)r.z;
                if (far) {
                    const long long pos = sfw[wp][owner] + __popc(fb & lt);
                    if (pos < sfwe[wp][owner]) fpairs[pos] = ent;
                    else atomicOr(err, 4u);
                } else {
                    const long long pos = sw[wp][owner] + __popc(nb & lt);
                    if (pos < swe[wp][owner]) pairs[pos] = ent;
                    else atomicOr(err, 4u);
                }
            }
            if (!WRITE && nsrc) atomicAdd((unsigned long long*)&ssrc[wp][owner], (unsigned long long)nsrc);
            __syncwarp();
            if (lead) {
                sw[wp][owner] += __popc(nb);
                sfw[wp][owner] += __popc(fb);
                sc[wp][owner] += __popc(nb);
                scf[wp][owner] += __popc(fb);
            }
            __syncwarp();
        }
        if (__all_sync(kFull, done)) break;
    }
    if (!live) return;
    const int64_t c = sc[wp][lane], cf = scf[wp][lane], src = ssrc[wp][lane];
    if (WRITE && !bad && (sw[wp][lane] != swe[wp][lane] || sfw[wp][lane] != sfwe[wp][lane]))
        atomicOr(err, 4u);
    if (!WRITE) {
        const int64_t nI = lfirst[I + 1] - lfirst[I];
        lcnt[I] = c;
        lfar[I] = cf;
        lcost[I] = src * nI;
        if (cache) {
            if (cok && runn > 0) {
                if (nrun == kslot)
                    cok = false;
                else
                    slot[nrun++] = make_uint2(run0, runn);
            }
            lruns[I] = cok ? nrun : -1;
            if (!cok) atomicAdd((unsigned long long*)(cnt + kCntUncached), 1ULL);
        }
        atomicAdd((unsigned long long*)(cnt + kCntPairs), (unsigned long long)c);
        atomicAdd((unsigned long long*)(cnt + kCntFar), (unsigned long long)cf);
        atomicAdd((unsigned long long*)(cnt + kCntEvaluated), (unsigned long long)(src * nI));
        atomicMax(cnt + kCntMaxCost, (long long)(src * nI));
        atomicMax(cnt + kCntMaxRow, (long long)c);
    }
}

// Expansion centre and radius of each leaf for the multipole split: the
// centre of its particle box and half the box diagonal; also the centre's
// offset from the leaf's cell centre (lcen, units of L / 2^22) in FP32, so
// that centre differences are an exact integer part plus a small FP32 one.
__global__ void k_fcen(const double* __restrict__ lbox, const int4* __restrict__ lcen,
                       double unit, int64_t nl, double4* __restrict__ fcen,
                       float4* __restrict__ fofs)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nl) return;
    const double* A = lbox + 6 * g;
    const int4 q = lcen[g];
    const int qc[3] = {q.x, q.y, q.z};
    double c[3], o[3], r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double ea = __dmul_rn(0.5, __dsub_rn(A[3 + a], A[a]));
        c[a] = __dmul_rn(0.5, __dadd_rn(A[a], A[3 + a]));
        o[a] = __dsub_rn(c[a], __dmul_rn((double)qc[a], unit));
        r2 = __dadd_rn(r2, __dmul_rn(ea, ea));
    }
    const double r = __dsqrt_rn(r2);
    fcen[g] = make_double4(c[0], c[1], c[2], r);
    fofs[g] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)r);
}

// --------------------------------------------------------------- payload --
// The workspace arrays of one leaf: leaf record, integer cell centre (units
// L / 2^22), leaf-local FP32 coordinates in units of 2 r_s, FP64 copy, perm.
__global__ void k_payload(const int32_t* __restrict__ lfirst, const int32_t* __restrict__ llevel,
                          const uint64_t* __restrict__ lkey, int64_t nl, int64_t n, BoxK bx,
                          const double* __restrict__ wpos, const int32_t* __restrict__ idx,
                          float4* __restrict__ pf, double4* __restrict__ pd,
                          int32_t* __restrict__ perm, int4* __restrict__ leaf,
                          int4* __restrict__ lcen)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nl) return;
    const int64_t f = lfirst[g], e = g + 1 < nl ? lfirst[g + 1] : n;
    const int L = llevel[g];
    const uint64_t k = lkey[g];
    const int sh = kMortonBits - L;
    const uint32_t sc = 1u << sh;
    const int32_t cx = (int32_t)((2 * (compact3_d(k >> 2) >> sh) + 1) * sc);
    const int32_t cy = (int32_t)((2 * (compact3_d(k >> 1) >> sh) + 1) * sc);
    const int32_t cz = (int32_t)((2 * (compact3_d(k) >> sh) + 1) * sc);
    leaf[g] = make_int4((int)f, (int)(e - f), 0, 0);
    lcen[g] = make_int4(cx, cy, cz, L);
    const double c[3] = {__dmul_rn((double)cx, bx.unit), __dmul_rn((double)cy, bx.unit),
                         __dmul_rn((double)cz, bx.unit)};
    for (int64_t q = f; q < e; ++q) {
        const int64_t p = idx[q];
        const double x = wpos[4 * p], y = wpos[4 * p + 1], z = wpos[4 * p + 2], m = wpos[4 * p + 3];
        pf[q] = make_float4((float)__dmul_rn(__dsub_rn(x, c[0]), bx.inv2rs),
                            (float)__dmul_rn(__dsub_rn(y, c[1]), bx.inv2rs),
                            (float)__dmul_rn(__dsub_rn(z, c[2]), bx.inv2rs), (float)m);
        if (pd) pd[q] = make_double4(x, y, z, m);
        perm[q] = (int32_t)p;
    }
}

// schedule keys: maxcost - cost ascending = cost descending; equal costs keep
// leaf order (stable sort)
__global__ void k_sched_keys(const int64_t* __restrict__ lcost, int64_t nl, long long maxcost,
                             uint64_t* __restrict__ key, int32_t* __restrict__ val)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nl) return;
    key[g] = (uint64_t)(maxcost - lcost[g]);
    val[g] = (int32_t)g;
}

__global__ void k_copy_total(int64_t* dst, const int64_t* src) { *dst = *src; }

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int dfail(int code, const std::string& msg)
{
    set_last_error(msg);
    return code;
}

int dcuda(int e, const char* what)
{
    return dfail(PSR_E_CUDA, std::string(what) + ": " + cudaGetErrorString((cudaError_t)e));
}

// Bounded host wait for the stream, then a copy of `bytes` to the host.
// Waits (at most timeout_ms) for the work queued on st, then copies one or
// two small device blocks to the host.  The wait polls without sleeping for
// its first 2 ms (the build's steps between waits take about a millisecond,
// and a sleeping poll wakes up to tens of microseconds late), then every 20
// microseconds.
int read_back(void* dst, const void* src, size_t bytes, cudaStream_t st, int timeout_ms,
              void* dst2 = nullptr, const void* src2 = nullptr, size_t bytes2 = 0)
{
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return dcuda(e, "cudaStreamQuery");
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > timeout_ms) return dfail(PSR_E_TIMEOUT, "device build did not finish within the timeout");
        if (ms > 2.0) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && dst2) e = cudaMemcpyAsync(dst2, src2, bytes2, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PSR_OK : dcuda(e, "cudaMemcpyAsync (device build counters)");
}

float float_at_least(double x)
{
    float f = (float)x;
    return (double)f < x ? std::nextafter(f, INFINITY) : f;
}

float float_at_most(double x)
{
    float f = (float)x;
    return (double)f > x ? std::nextafter(f, -INFINITY) : f;
}

BoxK box_k(const psr_box& b)
{
    BoxK k;
    k.L = b.L;
    k.scale = std::ldexp(1.0, kMortonBits) / b.L;
    k.unit = std::ldexp(b.L, -kCentreShift);
    k.inv2rs = 1.0 / (2.0 * b.r_s);
    k.rc2m = b.r_c * b.r_c * (1.0 + 1e-5);
    k.thi = float_at_least(k.rc2m * (1.0 + 1e-6));
    k.tlo = float_at_most(k.rc2m * (1.0 - 1e-6));
    k.theta2 = 0.0f;
    k.gt2 = 0.0f;
    k.rc2far = float_at_most(b.r_c * b.r_c * (1.0 - 1e-6));
    return k;
}

}  // namespace
}  // namespace psr

using namespace psr;

extern "C" {

int psr_device_build_scratch_bytes(int64_t n, size_t* bytes)
{
    if (!bytes || n < 1 || n > kMaxN)
        return dfail(PSR_E_ARG, "need 1 <= n <= 2^28 and a non-null output");
    *bytes = scratch_layout(n).bytes;
    return PSR_OK;
}

}  // extern "C"

namespace {

int device_build(const double* d_pos, const double* d_mass, int64_t n, const psr_box* box,
                 int max_leaf, int flags, double theta, void* d_scratch, size_t scratch_bytes,
                 void* stream, int timeout_ms, psr_leaves** out)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!out) return dfail(PSR_E_ARG, "null output");
    *out = nullptr;
    if (!d_pos || !box || n < 1 || n > kMaxN)
        return dfail(PSR_E_ARG, "null argument or n outside [1, 2^28]");
    if (max_leaf < 1 || max_leaf > kMaxLeaf) return dfail(PSR_E_ARG, "max_leaf must be in [1, 64]");
    if (flags & ~(PSR_BUILD_NO_FP64 | PSR_BUILD_UNPACKED | PSR_BUILD_SPLIT_GAUSSIAN))
        return dfail(PSR_E_ARG, "the device builder takes PSR_BUILD_NO_FP64, PSR_BUILD_UNPACKED "
                                "and PSR_BUILD_SPLIT_GAUSSIAN (no ORB)");
    if (!(std::isfinite(box->L) && box->L > 0) || !(std::isfinite(box->r_s) && box->r_s > 0) ||
        !std::isfinite(box->G))
        return dfail(PSR_E_ARG, "L, r_s must be finite and positive");
    if (!(box->r_c > 0) || !(box->r_c < box->L)) return dfail(PSR_E_CUTOFF, "need 0 < r_c < L");
    if (!(box->r_c >= 1e-10) || !(box->L <= 1e12))
        return dfail(PSR_E_ARG, "the device builder takes r_c >= 1e-10 and L <= 1e12");
    const Scratch S = scratch_layout(n);
    if (!d_scratch || scratch_bytes < S.bytes || (reinterpret_cast<uintptr_t>(d_scratch) & 255))
        return dfail(PSR_E_WORKSPACE, "scratch must be 256-byte aligned and at least " +
                                          std::to_string(S.bytes) + " bytes");
    if (timeout_ms <= 0) timeout_ms = kDefaultTimeoutMs;
    cudaStream_t st = (cudaStream_t)stream;
    char* s = static_cast<char*>(d_scratch);
    double* wpos = (double*)(s + S.wpos);
    uint64_t* k0 = (uint64_t*)(s + S.key0);
    uint64_t* k1 = (uint64_t*)(s + S.key1);
    int32_t* v0 = (int32_t*)(s + S.val0);
    int32_t* v1 = (int32_t*)(s + S.val1);
    int64_t* flag = (int64_t*)(s + S.flag);
    int64_t* lid = (int64_t*)(s + S.lid);
    int32_t* lfirst = (int32_t*)(s + S.lfirst);
    int32_t* llevel = (int32_t*)(s + S.llevel);
    uint64_t* lkey = (uint64_t*)(s + S.lkey);
    double* lbox = (double*)(s + S.lbox);
    float4* lrec = (float4*)(s + S.lrec);
    int64_t* lcnt = (int64_t*)(s + S.lcnt);
    int64_t* lcost = (int64_t*)(s + S.lcost);
    int2* tnode = (int2*)(s + S.tnode);
    int2* tspan = (int2*)(s + S.tspan);
    int32_t* tparl = (int32_t*)(s + S.tparl);
    int32_t* tpari = (int32_t*)(s + S.tpari);
    double* tbox = (double*)(s + S.tbox);
    float4* nodef = (float4*)(s + S.nodef);
    int* tflag = (int*)(s + S.tflag);
    int64_t* hist = (int64_t*)(s + S.hist);
    int64_t* tiles = (int64_t*)(s + S.tiles);
    int64_t* total = (int64_t*)(s + S.total);
    long long* cnt = (long long*)(s + S.cnt);
    BoxK bx = box_k(*box);
    bx.theta2 = (float)(theta * theta);
    bx.gt2 = (flags & PSR_BUILD_SPLIT_GAUSSIAN) ? (float)(theta * theta * 4.0 * std::pow(box->r_s, 4))
                                               : INFINITY;

    int e;
    if ((e = (int)cudaMemsetAsync(cnt, 0, 8 * kCntWords, st))) return dcuda(e, "cudaMemsetAsync");
    k_keys<<<nblk(n, 256), 256, 0, st>>>(d_pos, d_mass, n, bx, wpos, k0, v0, cnt);
    if ((e = (int)cudaGetLastError())) return dcuda(e, "key kernel");
    if ((e = radix_sort(k0, v0, k1, v1, n, 3 * kMortonBits, hist, tiles, total, st)))
        return dcuda(e, "radix sort");
    k_leaf_level<<<nblk(n, 256), 256, 0, st>>>(k0, n, max_leaf, flag, v1);
    if ((e = (int)cudaGetLastError())) return dcuda(e, "leaf level kernel");
    if ((e = scan_exclusive(flag, lid, n, tiles, total, st))) return dcuda(e, "scan");
    k_leaf_fill<<<nblk(n, 256), 256, 0, st>>>(flag, lid, v1, k0, n, lfirst, llevel, lkey);
    if ((e = (int)cudaGetLastError())) return dcuda(e, "leaf fill kernel");
    long long c[kCntWords];
    int64_t nl = 0;
    if ((e = read_back(&nl, total, 8, st, timeout_ms, c, cnt, sizeof c))) return e;
    if (c[kCntError] & 1) return dfail(PSR_E_ARG, "non-finite position or mass");
    if (nl < 1 || nl > n || nl >= (1 << 27)) return dfail(PSR_E_ARG, "leaf count out of range");
    if (!(flags & PSR_BUILD_UNPACKED)) {
        // pack sibling leaves: marks, pack ids, packed arrays in the (still
        // free) tree regions, copied back over the leaf arrays
        int64_t* pstart = flag;
        int64_t* pid = lid;
        int32_t* psize = tflag;
        int32_t* lfirst2 = (int32_t*)tspan;
        int32_t* llevel2 = tpari;
        uint64_t* lkey2 = (uint64_t*)tnode;
        k_pack_mark<<<nblk(nl, 256), 256, 0, st>>>(lfirst, llevel, lkey, nl, max_leaf, pstart, psize);
        if ((e = (int)cudaGetLastError())) return dcuda(e, "leaf packing kernel");
        if ((e = scan_exclusive(pstart, pid, nl, tiles, total, st))) return dcuda(e, "scan");
        k_pack_fill<<<nblk(nl, 256), 256, 0, st>>>(pstart, pid, psize, lfirst, llevel, lkey, nl,
                                                   lfirst2, llevel2, lkey2);
        if ((e = (int)cudaGetLastError())) return dcuda(e, "leaf packing kernel");
        int64_t np = 0;
        if ((e = read_back(&np, total, 8, st, timeout_ms))) return e;
        if (np < 1 || np > nl) return dfail(PSR_E_DEVICE, "leaf packing failed");
        if ((e = (int)cudaMemcpyAsync(lfirst, lfirst2, 4 * (np + 1), cudaMemcpyDeviceToDevice, st)) ||
            (e = (int)cudaMemcpyAsync(llevel, llevel2, 4 * np, cudaMemcpyDeviceToDevice, st)) ||
            (e = (int)cudaMemcpyAsync(lkey, lkey2, 8 * np, cudaMemcpyDeviceToDevice, st)))
            return dcuda(e, "cudaMemcpyAsync");
        nl = np;
    }
    k_leaf_box<<<nblk(nl, 256), 256, 0, st>>>(lfirst, nl, n, wpos, v0, lbox, lrec,
                                              (float4*)(s + S.lout), cnt);
    if (nl >= 2) {
        if ((e = (int)cudaMemsetAsync(tflag, 0, 4 * (nl - 1), st))) return dcuda(e, "cudaMemsetAsync");
        k_tree_nodes<<<nblk(nl - 1, 256), 256, 0, st>>>(lkey, nl, tnode, tspan, tparl, tpari);
        k_tree_boxes<<<nblk(nl, 256), 256, 0, st>>>(nl, tnode, tparl, tpari, lbox, tbox, tflag, cnt);
        k_tree_pack<<<nblk(nl - 1, 256), 256, 0, st>>>(nl, tnode, tspan, lbox, tbox, nodef);
    }
    const double* rootbox = nl >= 2 ? tbox : lbox;
    // rows interleaved over the warps when they fit in one wave of the count
    // walk's resident warps (32 per SM), two of the split walk's (16 per SM)
    int dev = 0, sms = 0;
    if ((e = (int)cudaGetDevice(&dev))) return dcuda(e, "cudaGetDevice");
    if ((e = (int)cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return dcuda(e, "cudaDeviceGetAttribute");
    const int interleave = nl <= (int64_t)sms * 32 * 32 ? 1 : 0;
    // runs per row in the pair cache (none below kMinRuns: rows walked twice)
    const int64_t ks = S.ncache / nl;
    const int kslot = ks >= kMinRuns ? (int)(ks < (1 << 20) ? ks : (1 << 20)) : 0;
    int32_t* const lruns = kslot ? (int32_t*)(s + S.lruns) : nullptr;
    uint2* const pcache = kslot ? (uint2*)(s + S.cache) : nullptr;
    if (theta > 0.0)
        k_pairs_split<false><<<nblk(nl, 128), 128, 0, st>>>(
            nl, bx, lfirst, lbox, lrec, (const float4*)(s + S.lout), nodef, rootbox, lcnt, lcost,
            (int64_t*)(s + S.lfar), nullptr, nullptr, nullptr, nullptr, cnt,
            (unsigned*)(cnt + kCntError), lruns, pcache, kslot, interleave);
    else {
        k_pairs<false><<<nblk(nl, 128), 128, 0, st>>>(
            nl, n, bx, lfirst, lbox, lrec, nodef, rootbox, lcnt, lcost, nullptr, nullptr, cnt,
            (unsigned*)(cnt + kCntError), lruns, pcache, kslot, interleave);
    }
    if ((e = (int)cudaGetLastError())) return dcuda(e, "pair count kernel");
    if ((e = read_back(c, cnt, sizeof c, st, timeout_ms))) return e;
    if (c[kCntError] & 2) return dfail(PSR_E_DEVICE, "tree traversal stack overflow");
    if (c[kCntError] & 4) return dfail(PSR_E_DEVICE, "malformed radix tree");
    if (c[kCntPairs] >= ((int64_t)1 << 32) || c[kCntFar] >= ((int64_t)1 << 32))
        return dfail(PSR_E_ARG, "more than 2^32 leaf pairs");

    Leaves* h = new (std::nothrow) Leaves();
    if (!h) return dfail(PSR_E_NOMEM, "out of host memory");
    try {
        h->nbox = 1;
        h->boxes.assign(box, box + 1);
        h->box_first = {0, n};
        h->n = n;
        h->max_leaf_req = max_leaf;
        h->flags = flags;
        h->n_leaves = nl;
        h->n_pairs = c[kCntPairs];
        h->evaluated = c[kCntEvaluated];
        h->max_leaf = (int)c[kCntMaxLeaf];
        h->max_row = (int)c[kCntMaxRow];
        h->has_pd = !(flags & PSR_BUILD_NO_FP64);
        h->device_built = true;
        h->has_far = theta > 0.0;
        h->theta = theta;
        h->n_far = theta > 0.0 ? c[kCntFar] : 0;
        h->boxdev = {box_constants(*box)};
        h->equal_mass = c[kCntMassDiff] == 0;
        if (h->equal_mass) {
            double m0;
            std::memcpy(&m0, &c[kCntMass0], sizeof m0);
            h->boxdev[0].m_eq = (float)m0;
        }
        h->lay = make_layout(*h);
    } catch (const std::bad_alloc&) {
        delete h;
        return dfail(PSR_E_NOMEM, "out of host memory");
    }
    h->db_scratch = s;
    h->db_maxcost = c[kCntMaxCost];
    h->db_kslot = kslot;
    h->db_interleave = interleave;
    h->db_uncached = kslot ? c[kCntUncached] : nl;
    h->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = reinterpret_cast<psr_leaves*>(h);
    return PSR_OK;
}

}  // namespace

extern "C" {

int psr_device_build(const double* d_pos, const double* d_mass, int64_t n, const psr_box* box,
                     int max_leaf, int flags, void* d_scratch, size_t scratch_bytes, void* stream,
                     int timeout_ms, psr_leaves** out)
{
    return device_build(d_pos, d_mass, n, box, max_leaf, flags, 0.0, d_scratch, scratch_bytes,
                        stream, timeout_ms, out);
}

int psr_device_build_split(const double* d_pos, const double* d_mass, int64_t n,
                           const psr_box* box, int max_leaf, int flags, double theta,
                           void* d_scratch, size_t scratch_bytes, void* stream, int timeout_ms,
                           psr_leaves** out)
{
    if (out) *out = nullptr;
    if (!(theta > 0.0 && theta <= 1.0)) return dfail(PSR_E_ARG, "theta must be in (0, 1]");
    return device_build(d_pos, d_mass, n, box, max_leaf, flags, theta, d_scratch, scratch_bytes,
                        stream, timeout_ms, out);
}

int psr_device_build_finish(psr_leaves* hh, void* d_ws, size_t bytes, void* stream)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h || !h->db_scratch) return dfail(PSR_E_STATE, "not a pending device build");
    if (!d_ws || bytes < h->lay.total || (reinterpret_cast<uintptr_t>(d_ws) & 255))
        return dfail(PSR_E_WORKSPACE, "workspace must be 256-byte aligned and at least " +
                                          std::to_string(h->lay.total) + " bytes");
    const int64_t n = h->n, nl = h->n_leaves;
    const Scratch S = scratch_layout(n);
    char* s = h->db_scratch;
    char* w = static_cast<char*>(d_ws);
    const Layout& L = h->lay;
    cudaStream_t st = (cudaStream_t)stream;
    const BoxK bx = box_k(h->boxes[0]);
    int e, dev = 0, sms = 0;
    if ((e = (int)cudaGetDevice(&dev))) return dcuda(e, "cudaGetDevice");
    if ((e = (int)cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return dcuda(e, "cudaDeviceGetAttribute");
    // the control words first: the pair write kernel reports into the error
    // word that psr_check reads
    if ((e = (int)cudaMemsetAsync(w + L.ctrl, 0, kCtrlWords * 4, st))) return dcuda(e, "cudaMemsetAsync");
    const int32_t* lfirst = (const int32_t*)(s + S.lfirst);
    k_payload<<<nblk(nl, 128), 128, 0, st>>>(
        lfirst, (const int32_t*)(s + S.llevel), (const uint64_t*)(s + S.lkey), nl, n, bx,
        (const double*)(s + S.wpos), (const int32_t*)(s + S.val0), (float4*)(w + L.pf),
        h->has_pd ? (double4*)(w + L.pd) : nullptr, (int32_t*)(w + L.perm), (int4*)(w + L.leaf),
        (int4*)(w + L.lcen));
    if ((e = (int)cudaGetLastError())) return dcuda(e, "payload kernel");
    // row pointers: exclusive scan of the row lengths, then the total
    int64_t* rowptr = (int64_t*)(w + L.rowptr);
    int64_t* tiles = (int64_t*)(s + S.tiles);
    int64_t* total = (int64_t*)(s + S.total);
    if ((e = scan_exclusive((const int64_t*)(s + S.lcnt), rowptr, nl, tiles, total, st)))
        return dcuda(e, "scan");
    k_copy_total<<<1, 1, 0, st>>>(rowptr + nl, total);
    const double* lbox = (const double*)(s + S.lbox);
    int64_t* frow = h->has_far ? (int64_t*)(w + L.frow) : nullptr;
    if (h->has_far) {
        if ((e = scan_exclusive((const int64_t*)(s + S.lfar), frow, nl, tiles, total, st)))
            return dcuda(e, "scan");
        k_copy_total<<<1, 1, 0, st>>>(frow + nl, total);
        k_fcen<<<nblk(nl, 128), 128, 0, st>>>(lbox, (const int4*)(w + L.lcen), bx.unit, nl,
                                              (double4*)(w + L.fcen), (float4*)(w + L.fofs));
        if ((e = (int)cudaGetLastError())) return dcuda(e, "expansion centre kernel");
    }
    const double* rootbox = nl >= 2 ? (const double*)(s + S.tbox) : lbox;
    if (h->has_far) {
        BoxK bxw = bx;
        bxw.theta2 = (float)(h->theta * h->theta);
        bxw.gt2 = (h->flags & PSR_BUILD_SPLIT_GAUSSIAN)
                      ? (float)(h->theta * h->theta * 4.0 * std::pow(h->boxes[0].r_s, 4))
                      : INFINITY;
        // rows the count pass recorded are replayed; the rest are walked again
        k_pairs_split<true><<<nblk(nl, 128), 128, 0, st>>>(
            nl, bxw, lfirst, lbox, (const float4*)(s + S.lrec), (const float4*)(s + S.lout),
            (const float4*)(s + S.nodef), rootbox, nullptr, nullptr, nullptr, rowptr,
            (uint32_t*)(w + L.pairs), frow, (uint32_t*)(w + L.fpairs), nullptr,
            (unsigned*)(w + L.ctrl) + kCtrlError,
            h->db_kslot ? (int32_t*)(s + S.lruns) : nullptr,
            h->db_kslot ? (uint2*)(s + S.cache) : nullptr, h->db_kslot, h->db_interleave);
    } else {
        // rows the count walk cached are expanded; the rest are walked again
        int32_t* lruns = h->db_kslot ? (int32_t*)(s + S.lruns) : nullptr;
        if (lruns) {
            k_pairs_expand<<<nblk(nl, 8), 256, 0, st>>>(nl, lruns, (const uint2*)(s + S.cache),
                                                       h->db_kslot, rowptr, (uint32_t*)(w + L.pairs),
                                                       (unsigned*)(w + L.ctrl) + kCtrlError);
            if ((e = (int)cudaGetLastError())) return dcuda(e, "pair expand kernel");
        }
        if (h->db_uncached > 0)
            k_pairs<true><<<nblk(nl, 128), 128, 0, st>>>(
                nl, n, bx, lfirst, lbox, (const float4*)(s + S.lrec), (const float4*)(s + S.nodef),
                rootbox, nullptr, nullptr, rowptr, (uint32_t*)(w + L.pairs), nullptr,
                (unsigned*)(w + L.ctrl) + kCtrlError, lruns, nullptr, 0, h->db_interleave);
    }
    if ((e = (int)cudaGetLastError())) return dcuda(e, "pair write kernel");
    // schedule: the particle sort buffers are free again (values in int32
    // views of the flag / lid regions, both >= 4 nl bytes)
    uint64_t* k0 = (uint64_t*)(s + S.key0);
    uint64_t* k1 = (uint64_t*)(s + S.key1);
    int32_t* v0 = (int32_t*)(s + S.flag);
    int32_t* v1 = (int32_t*)(s + S.lid);
    k_sched_keys<<<nblk(nl, 256), 256, 0, st>>>((const int64_t*)(s + S.lcost), nl,
                                                (long long)h->db_maxcost, k0, v0);
    int bits = 1;
    while (bits < 63 && ((uint64_t)h->db_maxcost >> bits)) ++bits;
    if ((e = radix_sort(k0, v0, k1, v1, nl, bits, (int64_t*)(s + S.hist), tiles, total, st)))
        return dcuda(e, "schedule sort");
    if ((e = (int)cudaMemcpyAsync(w + L.items, v0, 4 * nl, cudaMemcpyDeviceToDevice, st)))
        return dcuda(e, "cudaMemcpyAsync");
    if ((e = (int)cudaMemcpyAsync(w + L.boxes, h->boxdev.data(), sizeof(BoxDev),
                                  cudaMemcpyHostToDevice, st)))
        return dcuda(e, "cudaMemcpyAsync");
    h->d_ws = w;
    h->ws_bytes = bytes;
    h->uploaded = true;
    h->table_key = -1;
    h->table_xc = -1.0;
    h->adj_table_key = -1;
    h->sm_count = sms;
    h->device = dev;
    h->db_scratch = nullptr;
    return PSR_OK;
}

}  // extern "C"
