// FP32 forward P2P kernels (paper, Section 3.2, Algorithms 1 and 2, redesigned
// for sm_103a): shared device code of the two kernel variants.
//
// Work decomposition.  The paper gives one thread block to each target leaf
// and one thread to each target particle, with the j-leaf staged in shared
// memory.  Leaves here hold 1-64 particles (mean ~20 on the packed leaves of
// clustered sets, ~9 unpacked), so one WARP takes one target leaf: each lane
// holds R = 1, 2 or 3 target particles (chosen per leaf to fill the most
// lanes), the n_I targets occupy T = ceil(n_I / R) lanes, and the warp's 32
// lanes form S = 32 / T streams.  The row's source leaves are staged chunk by
// chunk into a per-warp shared-memory buffer, already shifted into the target
// leaf's frame and culled against the target leaf's box, and stream s takes
// staged particles s, s+S, ... (one broadcast shared-memory load serves the T
// lanes of a stream).  Two variants of the inner loop: scalar streams (one
// source per iteration) and packed pairs (two sources per iteration in
// sm_100+ f32x2 arithmetic, half the issue slots of the pair arithmetic; used
// for the leaves that take one target per lane).  The
// S partial sums of each target are combined through shared memory at the
// end.  Warps take target leaves from an atomic ticket in largest-work-first
// order (persistent grid, no inter-block waits).
//
// Precision.  Pair arithmetic is FP32 in leaf-local coordinates scaled by
// 1/(2 r_s); the offset between two leaf centres (with the periodic image) is
// an exact integer in units of L/2^22, converted to FP32 once per leaf pair.
// FP32 partial sums over one staged chunk (<= 256 source particles) are folded
// into FP64 (PSR_ACC_FP64) or compensated FP32 (PSR_ACC_KAHAN32) accumulators.
//
// T(x).  Exact: erfcf + expf.  Table: T on [0, x_c] with N intervals, held in
// shared memory: linear (midpoint value, chord difference) or cubic Hermite
// (monomial coefficients about the midpoint); index N is a zero sentinel, so
// the cutoff (x >= x_c) costs no extra instruction.
#pragma once
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace psr {

enum { TM_EXACT = 0, TM_LINEAR = 1, TM_CUBIC = 2, TM_TAYLOR = 3 };

// a * b + c clamped to [0, 1] in one instruction
__device__ __forceinline__ float fma_sat(float a, float b, float c)
{
    float d;
    asm("fma.rn.ftz.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Linear table (entries (A_k, N D_k) in shared memory).  The linear path
// measures distances in units of x_c, so s = sat(r / x_c - 1/(2N)) = t / N
// with t = u - 1/2 (u in table units) already clamped to [0, 1]: rint(s N) is
// the interval (N, the zero sentinel, beyond the cutoff) and T = A_k + s N D_k.
// Below u = 1/2 the clamp holds s at 0, which moves T by under 1e-8 (T is
// flat there: T = 1 - O(x^3)).
__device__ __forceinline__ float linear_T(float s, float nmax, unsigned tab_bias)
{
    const float fk = fmaf(s, nmax, kMagic);
    const float2 c = lds_f2((unsigned)__float_as_int(fk) * 8u + tab_bias);
    return fmaf(s, c.y, c.x);
}

// Paper's Taylor table (Section 3.3, Eq. int) about the nearest node: entry k
// is two float4, (c0, c1, c2, c3) and (c4, 0, 0, 0), the expansion about x_k
// in u - k (table units); nodes k = 0..N all real (x_N = x_c), so the cutoff,
// inside node N's cell, is an explicit select.
__device__ __forceinline__ float taylor_T(float u, float nmax, unsigned tab_bias)
{
    const float t = fminf(u, nmax);
    const float fk = t + kMagic;
    const float f = t - (fk - kMagic);
    const unsigned ad = (unsigned)__float_as_int(fk) * 32u + tab_bias;
    const float4 c = lds_f4(ad);
    const float c4 = lds_f1(ad + 16u);
    const float v = fmaf(f, fmaf(f, fmaf(f, fmaf(f, c4, c.w), c.z), c.y), c.x);
    return u < nmax ? v : 0.0f;
}

// exact T(x) with the hard cutoff
__device__ __forceinline__ float eval_T_exact(float x, float x_c)
{
    float T = erfcf(x) + kTwoOverSqrtPi * x * expf(-x * x);
    return x < x_c ? T : 0.0f;
}

template <int ACC>
struct Acc3 {
    double x = 0, y = 0, z = 0;  // FP64 mode
    float sx = 0, sy = 0, sz = 0, cx = 0, cy = 0, cz = 0;  // Kahan mode
    __device__ __forceinline__ void fold(float& fx, float& fy, float& fz)
    {
        if (ACC == PSR_ACC_FP64) {
            x += (double)fx;
            y += (double)fy;
            z += (double)fz;
        } else {
            float s, e;
            two_sum(sx, fx, s, e); sx = s; cx += e;
            two_sum(sy, fy, s, e); sy = s; cy += e;
            two_sum(sz, fz, s, e); sz = s; cz += e;
        }
        fx = fy = fz = 0.0f;
    }
};

// The target leaf's particle box in the kernel's working frame, and the
// cutoff in working units: a staged source particle whose distance from this
// box is at least the cutoff is beyond the cutoff from every target of the
// leaf, so its pairs contribute nothing (Eq. tr is truncated at r_c) and it is
// not staged.  The leaf-pair list keeps a source leaf when the two leaves'
// boxes come closer than r_c, so a part of each source leaf can lie farther.
//
// cull_box: the warp-wide box of the targets, written to the warp's two box
// slots in shared memory (kept there, not in registers, through the item's
// chunk loop): each lane passes the bounds of its active targets (+inf / -inf
// when it has none).
// The squared cutoff is widened by a factor 1 + 2^-12: the box distance
// computed in FP32 is a lower bound of every target's distance up to a few
// units in the last place, and the pair loop's own cutoff test (the table's
// zero sentinel, or x < x_c) decides each pair the kernel evaluates, so the
// margin only keeps a few extra pairs.
__device__ __forceinline__ void cull_box(float lox, float loy, float loz, float hix, float hiy,
                                         float hiz, float cut, float4* __restrict__ slot)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lox = fminf(lox, __shfl_xor_sync(kFull, lox, o));
        loy = fminf(loy, __shfl_xor_sync(kFull, loy, o));
        loz = fminf(loz, __shfl_xor_sync(kFull, loz, o));
        hix = fmaxf(hix, __shfl_xor_sync(kFull, hix, o));
        hiy = fmaxf(hiy, __shfl_xor_sync(kFull, hiy, o));
        hiz = fmaxf(hiz, __shfl_xor_sync(kFull, hiz, o));
    }
    if ((threadIdx.x & 31) == 0) {
        slot[0] = make_float4(0.5f * (lox + hix), 0.5f * (loy + hiy), 0.5f * (loz + hiz),
                              cut * cut * (1.0f + 1.0f / 4096.0f));
        slot[1] = make_float4(0.5f * (hix - lox), 0.5f * (hiy - loy), 0.5f * (hiz - loz), 0.0f);
    }
    __syncwarp();
}

// Loads from shared memory that the compiler must not hoist, merge or move
// across other volatile accesses: the target box is read at each use instead
// of being held in registers across the staging loop (where the item's
// accumulators already fill them), and the stream loop reads staged sources
// through 32-bit shared addresses that must not be read before the chunk's
// staging stores.
__device__ __forceinline__ float4 lds_f4_v(unsigned a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// true if the point (x, y, z) lies within the cutoff of the box kept at the
// shared-memory address box (two float4: centre and cut^2, half extents)
__device__ __forceinline__ bool cull_keep(unsigned box, float x, float y, float z)
{
    const float4 c = lds_f4_v(box), h = lds_f4_v(box + 16u);
    const float dx = fmaxf(fabsf(x - c.x) - h.x, 0.0f);
    const float dy = fmaxf(fabsf(y - c.y) - h.y, 0.0f);
    const float dz = fmaxf(fabsf(z - c.z) - h.z, 0.0f);
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < c.w;
}

// Per-warp shared-memory staging of a row's source particles.  Up to 32 row
// entries are examined at once (lane k reads entry e0 + k); a warp prefix sum
// of their leaf sizes gives each leaf's slots, and as many whole leaves as fit
// the buffer's free slots are taken.  Each particle is shifted into the target
// leaf's frame (its leaf offset added), tested against the target box
// (CullBox), and the particles within the cutoff are written compacted, in
// entry order, so the compute loop that follows is uniform over the chunk.
// When a window of 32 entries fits whole, the next window is staged behind it,
// so a chunk fills its buffer although the cull drops particles.
constexpr int kMetaPerWarp = 32; // entries per window (one per lane)
constexpr int kWarpMeta = kMetaPerWarp + 2;  // then the two CullBox slots

// Stages one chunk starting at entry e0; returns the number of entries taken
// and sets nst to the number of staged (kept) particles.  Staged coordinates
// are multiplied by sc (the kernels' working unit per FP32 coordinate unit).
// MODE 0: one float4 (x, y, z, m) per particle; MODE 1: particle pairs
// interleaved for packed arithmetic, an odd count padded with a massless
// particle far beyond the cutoff; MODE 2 (adjoint): two float4 per particle,
// (x, y, z, c_z) and (c_x, c_y, m, m), c the cotangent from a.cot_sorted;
// MODE 3 (packed adjoint): particle pairs interleaved, four float4 per pair
// (x0, x1, y0, y1), (z0, z1, m0, m1), (cx0, cx1, cy0, cy1), (cz0, cz1, 0, 0),
// an odd count padded like MODE 1 (zero mass and cotangent).
template <int MODE>
__device__ __forceinline__ int stage_chunk(const FwdArgs& a, long long e0, long long re,
                                           int4 ci, float unit, float sc, int cap,
                                           float4* __restrict__ stage,
                                           float4* __restrict__ meta, int& nst)
{
    const int lane = threadIdx.x & 31;
    const unsigned box = smem_u32(meta + kMetaPerWarp);
    const unsigned lt = (1u << lane) - 1u;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    const int4* __restrict__ lcen = reinterpret_cast<const int4*>(a.lcen);
    // entries as 32-bit offsets into the row (fewer live registers)
    const unsigned* __restrict__ prow = a.pairs + e0;
    const int rem = (int)min(re - e0, (long long)0x7fffffff);
    int nk = 0;  // particles kept so far
    int eb = 0;  // entries taken so far
    for (;;) {
        const int e = eb + lane;
        int cnt = 0, first = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (e < rem) {
            unsigned ent = prow[e];
            int J = (int)(ent >> 5);
            unsigned code = ent & 31u;
            bool ok = J < a.n_leaves && code < (unsigned)kShiftCodes;
            int4 lj = make_int4(0, 0, 0, 0);
            if (ok) {
                lj = leaf[J];
                ok = lj.x >= 0 && lj.y >= 1 && lj.y <= a.max_leaf && (long long)lj.x + lj.y <= a.n;
            }
            if (ok) {
                int4 cj = lcen[J];
                int nx, ny, nz;
                decode_shift(code, nx, ny, nz);
                ox = (float)(cj.x - ci.x + nx * (1 << kCentreShift)) * unit;
                oy = (float)(cj.y - ci.y + ny * (1 << kCentreShift)) * unit;
                oz = (float)(cj.z - ci.z + nz * (1 << kCentreShift)) * unit;
                cnt = lj.y;
                first = lj.x;
            } else {
                // a bad entry becomes one particle placed far beyond the cutoff
                set_error(a.ctrl, kErrLeafIndex);
                cnt = 1;
                first = 0;
                ox = oy = oz = 1e18f;
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned fit = __ballot_sync(kFull, e < rem && incl <= cap - nk);
        const int ntake = __popc(fit);  // the first window takes >= 1: cap >= max_leaf
        if (ntake == 0) break;
        const int nraw = __shfl_sync(kFull, incl, ntake - 1);
        const int excl = incl - cnt;
        if (lane < ntake)
            meta[lane] = make_float4(__int_as_float(first - excl), ox * sc, oy * sc, oz * sc);
        __syncwarp();
        // slot p belongs to the entry k with excl_k <= p < excl_{k+1}: count the
        // entry starts at or before p with a position bitmask per 32-slot round
        int C = 0;
        for (int p0 = 0; p0 < nraw; p0 += 32) {
            const int rel = excl - p0;
            const unsigned bit = (lane < ntake && rel >= 0 && rel < 32) ? (1u << rel) : 0u;
            const unsigned M = __reduce_or_sync(kFull, bit);
            const int k = C + __popc(M & ((2u << lane) - 1u)) - 1;
            C += __popc(M);
            const int p = p0 + lane;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            int src = 0;
            bool keep = false;
            float4 cot = make_float4(0.f, 0.f, 0.f, 0.f);  // adjoint modes
            if (p < nraw) {
                const float4 m = meta[k];
                src = __float_as_int(m.x) + p;
                v = __ldg(pf + src);
                // the cotangent is loaded beside the position, before the
                // cull decides (one round trip instead of two per round)
                if (MODE >= 2) cot = __ldg(reinterpret_cast<const float4*>(a.cot_sorted) + src);
                v.x = fmaf(v.x, sc, m.y);
                v.y = fmaf(v.y, sc, m.z);
                v.z = fmaf(v.z, sc, m.w);
                keep = cull_keep(box, v.x, v.y, v.z);
            }
            const unsigned K = __ballot_sync(kFull, keep);
            const int pos = nk + __popc(K & lt);
            if (keep) {
                if (MODE == 1) {
                    // pair j = pos/2 occupies two float4: (x0, x1, y0, y1), (z0, z1, m0, m1)
                    float* d = reinterpret_cast<float*>(stage) + 8 * (pos >> 1) + (pos & 1);
                    d[0] = v.x;
                    d[2] = v.y;
                    d[4] = v.z;
                    d[6] = v.w;
                } else if (MODE == 0) {
                    stage[pos] = v;
                } else if (MODE == 2) {
                    stage[2 * pos] = make_float4(v.x, v.y, v.z, cot.z);
                    stage[2 * pos + 1] = make_float4(cot.x, cot.y, v.w, v.w);
                } else {
                    const float4 c = cot;
                    float* d = reinterpret_cast<float*>(stage) + 16 * (pos >> 1) + (pos & 1);
                    d[0] = v.x;
                    d[2] = v.y;
                    d[4] = v.z;
                    d[6] = v.w;
                    d[8] = c.x;
                    d[10] = c.y;
                    d[12] = c.z;
                    d[14] = 0.0f;
                }
            }
            nk += __popc(K);
        }
        __syncwarp();
        eb += ntake;
        // a partly taken window means the next leaf does not fit
        if (ntake < 32 || eb >= rem) break;
    }
    if (MODE == 1 && (nk & 1) && lane == 0) {
        // pad an odd chunk with a massless particle far beyond the cutoff
        float* d = reinterpret_cast<float*>(stage) + 8 * (nk >> 1) + 1;
        d[0] = d[2] = d[4] = 1e18f;
        d[6] = 0.0f;
    }
    if (MODE == 3 && (nk & 1) && lane == 0) {
        // the same pad, with a zero cotangent
        float* d = reinterpret_cast<float*>(stage) + 16 * (nk >> 1) + 1;
        d[0] = d[2] = d[4] = 1e18f;
        d[6] = d[8] = d[10] = d[12] = d[14] = 0.0f;
    }
    __syncwarp();
    nst = nk;
    return eb;
}

// Combine the S stream partial sums of each target through shared memory
// (the warp's staging buffer) and write the accelerations, scaled by gout, in
// the original particle order.
template <int ACC, int R>
__device__ __forceinline__ void finish_item(const FwdArgs& a, int4 li, Acc3<ACC>* acc,
                                            const bool* act, int lane, int s, int q, int S, int T,
                                            float gout, float4* __restrict__ stage)
{
    // Each target slot r reduces through its own region of the staging buffer
    // (768 B; two slots fit the smallest per-warp buffer, 64 + 32 float4), with
    // volatile accesses, so one slot's stores cannot overtake another's loads.
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (ACC == PSR_ACC_FP64) {
            volatile double* red = reinterpret_cast<volatile double*>(stage) + 96 * r;
            red[3 * lane + 0] = acc[r].x;
            red[3 * lane + 1] = acc[r].y;
            red[3 * lane + 2] = acc[r].z;
            __syncwarp();
            if (s == 0 && act[r]) {
                double sx = acc[r].x, sy = acc[r].y, sz = acc[r].z;
                for (int t = 1; t < S; ++t) {
                    sx += red[3 * (lane + t * T) + 0];
                    sy += red[3 * (lane + t * T) + 1];
                    sz += red[3 * (lane + t * T) + 2];
                }
                int idx = a.perm[li.x + q + T * r];
                float* out = reinterpret_cast<float*>(a.out) + 3LL * idx;
                out[0] = (float)(sx * (double)gout);
                out[1] = (float)(sy * (double)gout);
                out[2] = (float)(sz * (double)gout);
            }
        } else {
            volatile float* red = reinterpret_cast<volatile float*>(stage) + 192 * r;
            red[6 * lane + 0] = acc[r].sx;
            red[6 * lane + 1] = acc[r].cx;
            red[6 * lane + 2] = acc[r].sy;
            red[6 * lane + 3] = acc[r].cy;
            red[6 * lane + 4] = acc[r].sz;
            red[6 * lane + 5] = acc[r].cz;
            __syncwarp();
            if (s == 0 && act[r]) {
                float sx = acc[r].sx, cx = acc[r].cx, sy = acc[r].sy, cy = acc[r].cy;
                float sz = acc[r].sz, cz = acc[r].cz, u, v;
                for (int t = 1; t < S; ++t) {
                    const volatile float* o = red + 6 * (lane + t * T);
                    two_sum(sx, o[0], u, v); sx = u; cx += o[1] + v;
                    two_sum(sy, o[2], u, v); sy = u; cy += o[3] + v;
                    two_sum(sz, o[4], u, v); sz = u; cz += o[5] + v;
                }
                int idx = a.perm[li.x + q + T * r];
                float* out = reinterpret_cast<float*>(a.out) + 3LL * idx;
                out[0] = (sx + cx) * gout;
                out[1] = (sy + cy) * gout;
                out[2] = (sz + cz) * gout;
            }
        }
        __syncwarp();
    }
}

// Packed FP32 helpers (sm_100+ f32x2 instructions: two lanes of work per issue)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// T for a pair of table coordinates t = u - 1/2, u = x N / x_c (one FFMA of
// r^2 and 1/r when coordinates are in table units).  Table entries: linear
// (M_k, D_k) float2, cubic (c0..c3) float4, entry N = 0 (beyond the cutoff).
// The index comes from the 1.5*2^23 rounding trick: the float bits of
// t + 1.5*2^23 hold rint(t) in their low bits, so an entry address is one
// multiply-add of them.
template <int TM>
__device__ __forceinline__ float2 eval_T2(float2 t, float2 r2, float2 rinv, unsigned tab_bias,
                                          float nmax, float x_c, float xscale)
{
    if (TM == TM_EXACT) {
        return make_float2(eval_T_exact(r2.x * rinv.x * xscale, x_c),
                           eval_T_exact(r2.y * rinv.y * xscale, x_c));
    } else if (TM == TM_TAYLOR) {  // t = u here (nearest node)
        return make_float2(taylor_T(t.x, nmax, tab_bias), taylor_T(t.y, nmax, tab_bias));
    } else if (TM == TM_LINEAR) {  // t = s here (see linear_T)
        const float2 fk = fma2(t, make_float2(nmax, nmax), make_float2(kMagic, kMagic));
        const float2 ca = lds_f2((unsigned)__float_as_int(fk.x) * 8u + tab_bias);
        const float2 cb = lds_f2((unsigned)__float_as_int(fk.y) * 8u + tab_bias);
        // Two scalar FFMAs, not one FFMA2: an f32x2 operand must sit in a
        // register pair, and gathering (ca.y, cb.y) and (ca.x, cb.x) into pairs
        // costs four register moves, which run on the heavy half of the FMA
        // pipe like the f32x2 arithmetic itself (the packed kernel's limit);
        // scalar FFMAs write their results straight into a pair and can run
        // on either half.
        return make_float2(fmaf(t.x, ca.y, ca.x), fmaf(t.y, cb.y, cb.x));
    } else {
        t.x = fminf(t.x, nmax);
        t.y = fminf(t.y, nmax);
        const float2 fk = add2(t, make_float2(kMagic, kMagic));
        const float2 kf = add2(fk, make_float2(-kMagic, -kMagic));
        const float2 f = fma2(kf, make_float2(-1.0f, -1.0f), t);
        const unsigned ka = (unsigned)__float_as_int(fk.x), kb = (unsigned)__float_as_int(fk.y);
        {
            const float4 ca = lds_f4(ka * 16u + tab_bias), cb = lds_f4(kb * 16u + tab_bias);
            return make_float2(fmaf(f.x, fmaf(f.x, fmaf(f.x, ca.w, ca.z), ca.y), ca.x),
                               fmaf(f.y, fmaf(f.y, fmaf(f.y, cb.w, cb.z), cb.y), cb.x));
        }
    }
}

// One target leaf on one warp.  R = targets per lane; T = ceil(n_I / R) lanes
// per stream, S = 32 / T streams.  Each stream takes staged particle PAIRS
// s, s+S, ... and evaluates both particles of a pair at once with packed
// FP32 (f32x2) arithmetic.
template <int TM, int ACC, bool COUNT, bool EQM, int R>
__device__ __forceinline__ void fwd_item_pk(const FwdArgs& a, int I, int4 li, unsigned tab_bias,
                                            float4* __restrict__ stage, float4* __restrict__ meta,
                                         unsigned long long& npairs, unsigned long long& nev)
{
    const int lane = threadIdx.x & 31;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const int4* __restrict__ lcen = reinterpret_cast<const int4*>(a.lcen);
    const int nI = li.y;
    const int T = (nI + R - 1) / R;
    const int S = 32 / T;
    const int s = lane / T;
    const int q = lane - s * T;
    const bool on = s < S;
    const BoxDev& bx = a.boxes[li.z];
    const float x_c = bx.x_c;
    const float nmax = (float)a.table_n;
    // working unit: table intervals (u = x N / x_c) for the table path, x itself
    // for the exact path
    const float sc = TM == TM_EXACT ? 1.0f : TM == TM_LINEAR ? 1.0f / x_c : (float)a.table_n / x_c;
    const float xscale = 1.0f / sc;  // working unit -> x (exact path only)
    const float unit = bx.unit;
    const int4 ci = lcen[I];

    float2 ntx[R], nty[R], ntz[R];  // minus the target coordinates, both halves
    bool act[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = q + T * r;
        act[r] = on && t < nI;
        const float4 v = pf[li.x + (act[r] ? t : 0)];
        ntx[r] = make_float2(-v.x * sc, -v.x * sc);
        nty[r] = make_float2(-v.y * sc, -v.y * sc);
        ntz[r] = make_float2(-v.z * sc, -v.z * sc);
    }
    {  // the target box for the cull (shared memory, after the entry records)
        float lx = kInf, ly = kInf, lz = kInf, hx = -kInf, hy = -kInf, hz = -kInf;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (act[r]) {
                lx = fminf(lx, -ntx[r].x); hx = fmaxf(hx, -ntx[r].x);
                ly = fminf(ly, -nty[r].x); hy = fmaxf(hy, -nty[r].x);
                lz = fminf(lz, -ntz[r].x); hz = fmaxf(hz, -ntz[r].x);
            }
        cull_box(lx, ly, lz, hx, hy, hz, x_c * sc, meta + kMetaPerWarp);
    }
    Acc3<ACC> acc[R];
    float2 fx[R], fy[R], fz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) fx[r] = fy[r] = fz[r] = make_float2(0.0f, 0.0f);
    unsigned cnt = 0;
    const long long re = a.rowptr[I + 1];
    long long e0 = a.rowptr[I];
    const float eps = kEps2 * sc * sc;
    const float2 eps2 = make_float2(eps, eps);
    // table coordinate: u - 1/2 (interval tables), u (Taylor: nearest node)
    const float2 mhalf = TM == TM_TAYLOR ? make_float2(0.0f, 0.0f) : make_float2(-0.5f, -0.5f);
    const float soff = -0.5f / nmax;  // linear path: s = sat(r / x_c - 1/(2N))
    while (e0 < re) {
        int nst;
        e0 += stage_chunk<1>(a, e0, re, ci, unit, sc, a.stage_cap, stage, meta, nst);
        if (COUNT && lane == 0) nev += (unsigned long long)nst * (unsigned)nI;
        if (on) {
            auto evalp = [&](const float4 A, const float4 B) {
                const float2 px = make_float2(A.x, A.y), py = make_float2(A.z, A.w);
                const float2 pz = make_float2(B.x, B.y), pm = make_float2(B.z, B.w);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 dx = add2(px, ntx[r]), dy = add2(py, nty[r]), dz = add2(pz, ntz[r]);
                    const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
                    const float2 rinv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
                    const float2 t = TM == TM_LINEAR
                                         ? make_float2(fma_sat(r2.x, rinv.x, soff), fma_sat(r2.y, rinv.y, soff))
                                         : fma2(r2, rinv, mhalf);
                    const float2 Tv = eval_T2<TM>(t, r2, rinv, tab_bias, nmax, x_c, xscale);
                    // 1/r^3 formed beside the table lookup: two dependent
                    // multiplies after T instead of four
                    const float2 ri3 = mul2(mul2(rinv, rinv), rinv);
                    const float2 w = EQM ? mul2(Tv, ri3) : mul2(mul2(pm, Tv), ri3);
                    fx[r] = fma2(w, dx, fx[r]);
                    fy[r] = fma2(w, dy, fy[r]);
                    fz[r] = fma2(w, dz, fz[r]);
                    if (COUNT) {
                        const float uc = TM == TM_EXACT ? x_c : TM == TM_LINEAR ? 1.0f : nmax;
                        const float ua = r2.x * rinv.x, ub = r2.y * rinv.y;
                        cnt += (act[r] && ua < uc && (dx.x != 0.0f || dy.x != 0.0f || dz.x != 0.0f));
                        cnt += (act[r] && ub < uc && (dx.y != 0.0f || dy.y != 0.0f || dz.y != 0.0f));
                    }
                }
            };
            // Two staged pairs per iteration (k and k + S, then the odd one),
            // in the order of the plain loop: two independent dependency
            // chains per lane, as in the scalar kernel.
            const float4* ps = stage + 2 * s;
            const float4* const pe = stage + 2 * ((nst + 1) >> 1);
#pragma unroll 1
            for (; ps + 2 * S < pe; ps += 4 * S) {
                const float4 A0 = ps[0], B0 = ps[1], A1 = ps[2 * S], B1 = ps[2 * S + 1];
                evalp(A0, B0);
                evalp(A1, B1);
            }
            if (ps < pe) evalp(ps[0], ps[1]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float sx = fx[r].x + fx[r].y, sy = fy[r].x + fy[r].y, sz = fz[r].x + fz[r].y;
                acc[r].fold(sx, sy, sz);
                fx[r] = fy[r] = fz[r] = make_float2(0.0f, 0.0f);
            }
        }
        __syncwarp();
    }
    finish_item<ACC, R>(a, li, acc, act, lane, s, q, S, T,
                        bx.g_acc * sc * sc * (EQM ? bx.m_eq : 1.0f), stage);
    if (COUNT) npairs += cnt;
}

// T for one table coordinate t = u - 1/2 (see eval_T2).
template <int TM>
__device__ __forceinline__ float eval_T1(float t, float r2, float rinv, unsigned tab_bias,
                                         float nmax, float x_c, float xscale)
{
    if (TM == TM_EXACT) return eval_T_exact(r2 * rinv * xscale, x_c);
    if (TM == TM_TAYLOR) return taylor_T(t, nmax, tab_bias);  // t = u here
    if (TM == TM_LINEAR) return linear_T(t, nmax, tab_bias);  // t = s here
    t = fminf(t, nmax);
    const float fk = t + kMagic;
    const unsigned k = (unsigned)__float_as_int(fk);
    const float f = t - (fk - kMagic);
    const float4 c = lds_f4(k * 16u + tab_bias);
    return fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
}

// Scalar-stream variant: stream s takes staged particles s, s+S, ... one at
// a time (two iterations in flight per warp).  d_x and d_y come from one
// f32x2 add of register pairs (the staged (x, y) and the target's
// (-x_k, -y_k)), the same rounding as two scalar subtractions: one
// instruction fewer per pair (2 % on the 128^3 launch, 5 % at 96^3).
template <int TM, int ACC, bool COUNT, bool EQM, int R>
__device__ __forceinline__ void fwd_item_sc(const FwdArgs& a, int I, int4 li, unsigned tab_bias,
                                            float4* __restrict__ stage,
                                            float4* __restrict__ meta, unsigned long long& npairs,
                                            unsigned long long& nev)
{
    const int lane = threadIdx.x & 31;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const int4* __restrict__ lcen = reinterpret_cast<const int4*>(a.lcen);
    const int nI = li.y;
    const int T = (nI + R - 1) / R;
    const int S = 32 / T;
    const int s = lane / T;
    const int q = lane - s * T;
    const bool on = s < S;
    const BoxDev& bx = a.boxes[li.z];
    const float x_c = bx.x_c;
    const float nmax = (float)a.table_n;
    const float soff = -0.5f / nmax;  // linear path: s = sat(r / x_c - 1/(2N))
    const float sc = TM == TM_EXACT ? 1.0f : TM == TM_LINEAR ? 1.0f / x_c : (float)a.table_n / x_c;
    const float xscale = 1.0f / sc;
    const float unit = bx.unit;
    const int4 ci = lcen[I];

    float2 nxy[R];  // (-x_k, -y_k): d_x, d_y in one f32x2 add
    float xz[R];
    bool act[R];
    float lx = kInf, ly = kInf, lz = kInf, hx = -kInf, hy = -kInf, hz = -kInf;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = q + T * r;
        act[r] = on && t < nI;
        const float4 v = pf[li.x + (act[r] ? t : 0)];
        const float x = v.x * sc, y = v.y * sc;
        xz[r] = v.z * sc;
        nxy[r] = make_float2(-x, -y);
        if (act[r]) {
            lx = fminf(lx, x); hx = fmaxf(hx, x);
            ly = fminf(ly, y); hy = fmaxf(hy, y);
            lz = fminf(lz, xz[r]); hz = fmaxf(hz, xz[r]);
        }
    }
    // the target box for the cull (shared memory, after the entry records)
    cull_box(lx, ly, lz, hx, hy, hz, x_c * sc, meta + kMetaPerWarp);
    Acc3<ACC> acc[R];
    float fx[R], fy[R], fz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) fx[r] = fy[r] = fz[r] = 0.0f;
    unsigned cnt = 0;
    const long long re = a.rowptr[I + 1];
    long long e0 = a.rowptr[I];
    const float eps2 = kEps2 * sc * sc;
    while (e0 < re) {
        int nst;
        e0 += stage_chunk<0>(a, e0, re, ci, unit, sc, a.stage_cap, stage, meta, nst);
        if (COUNT && lane == 0) nev += (unsigned long long)nst * (unsigned)nI;
        if (on) {
            auto eval = [&](const float4 p) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 dxy = add2(make_float2(p.x, p.y), nxy[r]);
                    const float dx = dxy.x, dy = dxy.y, dz = p.z - xz[r];
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    float rinv = rsqrt_ftz(r2);
                    const float t = TM == TM_LINEAR ? fma_sat(r2, rinv, soff)
                                                    : fmaf(r2, rinv, TM == TM_TAYLOR ? 0.0f : -0.5f);
                    float Tv = eval_T1<TM>(t, r2, rinv, tab_bias, nmax, x_c, xscale);
                    // 1/r^3 formed beside the table lookup (two dependent
                    // multiplies after T instead of four)
                    const float ri3 = rinv * rinv * rinv;
                    const float w = EQM ? Tv * ri3 : (p.w * Tv) * ri3;
                    fx[r] = fmaf(w, dx, fx[r]);
                    fy[r] = fmaf(w, dy, fy[r]);
                    fz[r] = fmaf(w, dz, fz[r]);
                    if (COUNT) {
                        const float u = r2 * rinv;
                        const float uc = TM == TM_EXACT ? x_c : TM == TM_LINEAR ? 1.0f : nmax;
                        cnt += (act[r] && u < uc && (dx != 0.0f || dy != 0.0f || dz != 0.0f));
                    }
                }
            };
            // Two sources per iteration (s + 2jS and s + (2j+1)S), then the odd
            // one: the same order as a plain loop over k = s, s+S, ..., with
            // half its loop and address instructions (1-3 % faster launches).
// the loop walks 32-bit shared-window addresses (one integer add per
            // step; 1.5 % faster than pointer arithmetic on the bench workload);
            // the loads are volatile so that none moves across the chunk's
            // staging stores
            unsigned sa = smem_u32(stage + s);
            const unsigned se = smem_u32(stage + nst), st1 = 16u * (unsigned)S;
#pragma unroll 1
            for (; sa + st1 < se; sa += 2u * st1) {
                const float4 p0 = lds_f4_v(sa), p1 = lds_f4_v(sa + st1);
                eval(p0);
                eval(p1);
            }
            if (sa < se) eval(lds_f4_v(sa));
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r].fold(fx[r], fy[r], fz[r]);
        }
        __syncwarp();
    }
    finish_item<ACC, R>(a, li, acc, act, lane, s, q, S, T,
                        bx.g_acc * sc * sc * (EQM ? bx.m_eq : 1.0f), stage);
    if (COUNT) npairs += cnt;
}

// Lane-slot efficiency of R targets per lane: n_I * floor(32 / ceil(n_I/R)) / (32 R)
__device__ __forceinline__ bool prefer_two_per_lane(int n)
{
    if (n > 32) return true;
    int t2 = (n + 1) >> 1;
    int e1 = n * (32 / n);          // x 1/32
    int e2 = n * (32 / t2);         // x 1/64
    return e2 > 2 * e1 + (2 * e1) / 16;  // > 6 % better
}

// Targets per lane for the scalar kernel, by cost per useful pair.  One
// iteration of a stream evaluates one staged source against the lane's R
// targets, kPairInstr instructions per target plus kSourceInstr for the
// source itself (its shared-memory load and the loop), and the warp's
// S_R = floor(32 / ceil(n_I / R)) streams serve n_I S_R pairs per iteration:
// the cost per pair is (kPairInstr R + kSourceInstr) / S_R, the cheapest R
// wins, ties going to the smaller.  The per-source term is set to 0, the
// measured best: with 3, 6 or 10 the rule moves leaves of 25-32 particles to
// R = 2 or 3 at equal lane fill, and whole launches ran 2-5 % slower.  So a
// larger R is taken only where it fills strictly more lanes: R = 3 for
// leaves of 3, 6, 9, 11-12, 17-18, 21-24 (24 = 8 lanes x 3 targets x 4
// streams) and 33-48 particles (11-16 lanes x 2 streams, against 17-24 lanes
// x 1 for R = 2; 6 % faster on leaves of up to 64); R = 2 for 19-20 and
// 49-64.  R = 1 needs n_I <= 32; R = 3 needs tiles of at least 128
// particles (its final reduction takes 3 x 768 B of the warp's staging
// buffer).
constexpr int kPairInstr = 20, kSourceInstr = 0;
__device__ __forceinline__ int targets_per_lane(int n, int cap)
{
    int best = 0, bnum = 0, bS = 1;
#pragma unroll
    for (int R = 1; R <= 3; ++R) {
        const int T = (n + R - 1) / R;
        if (T > 32 || (R == 3 && cap < 128)) continue;
        const int S = 32 / T, num = kPairInstr * R + kSourceInstr;
        if (best == 0 || num * bS < bnum * S) {
            best = R;
            bnum = num;
            bS = S;
        }
    }
    return best;
}

// Shared memory: the table, then one staging buffer of stage_cap particles
// plus 32 entry records per warp.
template <int TM, int ACC, bool COUNT, bool WIDE, bool PK, bool EQM>
__global__ void __launch_bounds__(256, 4) p2p_fwd_f32_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const unsigned esize = TM == TM_TAYLOR ? 32u : TM == TM_CUBIC ? 16u : 8u;
    const size_t tab_bytes = TM == TM_EXACT ? 0 : (size_t)(a.table_n + 1) * esize;
    float4* stage = reinterpret_cast<float4*>(smem + ((tab_bytes + 15) & ~(size_t)15)) +
                    (size_t)warp * (a.stage_cap + kWarpMeta);
    float4* meta = stage + a.stage_cap;
    if (TM == TM_TAYLOR) {
        const float4* g = reinterpret_cast<const float4*>(a.table);
        for (int i = threadIdx.x; i < 2 * (a.table_n + 1); i += blockDim.x)
            reinterpret_cast<float4*>(smem)[i] = g[i];
        __syncthreads();
    } else if (TM != TM_EXACT) {
        const float4* g = reinterpret_cast<const float4*>(a.table);
        for (int i = threadIdx.x; i <= a.table_n; i += blockDim.x) {
            const float4 v = g[i];
            if (TM == TM_LINEAR)
                reinterpret_cast<float2*>(smem)[i] = make_float2(v.z, v.y * (float)a.table_n);  // (A_k, N D_k)
            else
                reinterpret_cast<float4*>(smem)[i] = v;
        }
        __syncthreads();
    }
    // entry address = bits(t + 1.5*2^23) * esize + tab_bias (mod 2^32)
    const unsigned tab_bias = smem_u32(smem) - (unsigned)kMagicBits * esize;
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    unsigned long long npairs = 0, nev = 0;
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.ctrl + kCtrlTicketFwd, 1u) * a.item_stride + a.item_offset;
        it = __shfl_sync(kFull, it, 0);
        if (it >= a.n_items) break;
        int I = a.items[it];
        if (I < 0 || I >= a.n_leaves) {
            if (lane == 0) set_error(a.ctrl, kErrItemIndex);
            continue;
        }
        int4 li = leaf[I];
        if (li.y <= 0 || li.y > a.max_leaf || li.y > 64 || (long long)li.x + li.y > a.n ||
            li.z < 0 || li.z >= a.nbox) {
            if (lane == 0) set_error(a.ctrl, kErrParticleRange);
            continue;
        }
        if (PK) {
            // packed pairs where one target per lane fills the lanes as well
            // as any R; elsewhere the scalar two- or three-targets paths,
            // whose lane fill the packed state cannot reach within 64
            // registers (10.59 against 10.78 ms for packed pairs throughout
            // on the bench workload)
            const int R = targets_per_lane(li.y, a.stage_cap);
            if (R == 1)
                fwd_item_pk<TM, ACC, COUNT, EQM, 1>(a, I, li, tab_bias, stage, meta, npairs, nev);
            else if (R == 3)
                fwd_item_sc<TM, ACC, COUNT, EQM, 3>(a, I, li, tab_bias, stage, meta, npairs, nev);
            else
                fwd_item_sc<TM, ACC, COUNT, EQM, 2>(a, I, li, tab_bias, stage, meta, npairs, nev);
        } else {
            const int R = WIDE ? targets_per_lane(li.y, a.stage_cap) : 1;
            if (R == 3)
                fwd_item_sc<TM, ACC, COUNT, EQM, 3>(a, I, li, tab_bias, stage, meta, npairs, nev);
            else if (R == 2)
                fwd_item_sc<TM, ACC, COUNT, EQM, 2>(a, I, li, tab_bias, stage, meta, npairs, nev);
            else
                fwd_item_sc<TM, ACC, COUNT, EQM, 1>(a, I, li, tab_bias, stage, meta, npairs, nev);
        }
    }
    if (COUNT) {
        for (int off = 16; off > 0; off >>= 1) npairs += __shfl_xor_sync(kFull, npairs, off);
        if (lane == 0 && npairs)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlPairsLo), npairs);
        if (lane == 0 && nev)  // lane 0 alone counted the warp's staged pairs
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlEvalLo), nev);
    }
    persistent_exit(a.ctrl + kCtrlTicketFwd, a.ctrl + kCtrlDoneFwd);
}

// Launch and occupancy of the variant PK (explicitly instantiated in
// p2p_fwd_f32_sc.cu and p2p_fwd_f32_pk.cu).
template <int TM, int ACC, bool COUNT, bool PK, bool EQM>
static int launch_t(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    // Both variants carry the scalar two- and three-targets-per-lane paths
    // (targets_per_lane picks per leaf; the packed variant runs its f32x2
    // loop for the leaves that take one target per lane).
    auto k = p2p_fwd_f32_kernel<TM, ACC, COUNT, true, PK, EQM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    k<<<a.blocks, a.warps_per_block * 32, smem, st>>>(a);
    return (int)cudaGetLastError();
}

template <int TM, int ACC, bool PK>
static int launch_c(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    // equal masses: the mass leaves the pair sum (the pair-counting launch,
    // untimed, keeps the general form)
    return a.count_pairs  ? launch_t<TM, ACC, true, PK, false>(a, smem, st)
           : a.equal_mass ? launch_t<TM, ACC, false, PK, true>(a, smem, st)
                          : launch_t<TM, ACC, false, PK, false>(a, smem, st);
}

template <bool PK>
int launch_fwd_f32_variant(const FwdArgs& a, int precision, size_t smem, cudaStream_t st)
{
    if (precision == PSR_FP32_EXACT)
        return a.accum == PSR_ACC_FP64 ? launch_c<TM_EXACT, PSR_ACC_FP64, PK>(a, smem, st)
                                       : launch_c<TM_EXACT, PSR_ACC_KAHAN32, PK>(a, smem, st);
    if (a.interp == PSR_LINEAR)
        return a.accum == PSR_ACC_FP64 ? launch_c<TM_LINEAR, PSR_ACC_FP64, PK>(a, smem, st)
                                       : launch_c<TM_LINEAR, PSR_ACC_KAHAN32, PK>(a, smem, st);
    if (a.interp == PSR_TAYLOR2 || a.interp == PSR_TAYLOR4)
        return a.accum == PSR_ACC_FP64 ? launch_c<TM_TAYLOR, PSR_ACC_FP64, PK>(a, smem, st)
                                       : launch_c<TM_TAYLOR, PSR_ACC_KAHAN32, PK>(a, smem, st);
    return a.accum == PSR_ACC_FP64 ? launch_c<TM_CUBIC, PSR_ACC_FP64, PK>(a, smem, st)
                                   : launch_c<TM_CUBIC, PSR_ACC_KAHAN32, PK>(a, smem, st);
}

template <bool PK>
const void* fwd_f32_kernel_ptr(int precision, int interp, int accum, int max_leaf)
{
#define PSR_PICK(TM, ACC) ((const void*)p2p_fwd_f32_kernel<TM, ACC, false, true, PK, false>)
    if (precision == PSR_FP32_EXACT)
        return accum == PSR_ACC_FP64 ? PSR_PICK(TM_EXACT, PSR_ACC_FP64) : PSR_PICK(TM_EXACT, PSR_ACC_KAHAN32);
    if (interp == PSR_LINEAR)
        return accum == PSR_ACC_FP64 ? PSR_PICK(TM_LINEAR, PSR_ACC_FP64) : PSR_PICK(TM_LINEAR, PSR_ACC_KAHAN32);
    if (interp == PSR_TAYLOR2 || interp == PSR_TAYLOR4)
        return accum == PSR_ACC_FP64 ? PSR_PICK(TM_TAYLOR, PSR_ACC_FP64) : PSR_PICK(TM_TAYLOR, PSR_ACC_KAHAN32);
    return accum == PSR_ACC_FP64 ? PSR_PICK(TM_CUBIC, PSR_ACC_FP64) : PSR_PICK(TM_CUBIC, PSR_ACC_KAHAN32);
#undef PSR_PICK
}

}  // namespace psr
