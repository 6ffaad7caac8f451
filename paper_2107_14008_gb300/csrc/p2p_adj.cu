// Adjoint P2P kernels (not in the paper).  For L = sum_i c_i . a_i with the
// forward sum of Section 2 over a fixed set of pairs:
//   dL/dx_k = G sum_j K(d_kj) (m_k c_j - m_j c_k),  K(d) = g I + (g'(r)/r) d d^T,
//   dL/dm_k = -G sum_j g(r_kj) d_kj . c_j,
// g = T/r^3 and g'(r)/r = -f_(2), the n = 2 truncated prefactor of Section 2:
//   g'(r)/r = -3 T/r^5 - exp(-x^2) / (2 sqrt(pi) r_s^3 r^2).
// In the FP32 kernels' coordinates d' = d/(2 r_s), x = |d'|:
//   dL/dx_k = G/(8 r_s^3) sum_j [ (T/x^3) v + h d' (d'.v) ],  v = m_k c_j - m_j c_k,
//   h = -3 T/x^5 - (4/sqrt(pi)) exp(-x^2)/x^2,
//   dL/dm_k = -G/(4 r_s^2) sum_j (T/x^3) d'.c_j.
// Each pair needs the source payload (x, m, c): the cotangent is first
// gathered into Morton order.  Same work decomposition as the forward.
#include <cuda_runtime.h>

#include "fwd_f32_common.cuh"

namespace psr {

constexpr float kFourOverSqrtPi = 2.2567583341910251f;
constexpr float kLog2E = 1.4426950408889634f;
// Largest 1/r (in units of 1/x_c) the linear path's arithmetic takes: with
// T <= 1 and Q <= c4, T/r^3 and (3 T/r^3 + Q)/r^2 stay finite (3 kRinvMax^5 <
// FLT_MAX).  1/r is clamped here; only pairs closer than 2.5e-8 x_c, below
// the resolution of the FP32 leaf-local coordinates, are affected, and at
// r = 0 the zero table entry makes every term exactly zero.
constexpr float kRinvMax = 4.0e7f;

// PTX ex2.approx.ftz.f32: one SFU instruction, 2^x with a relative error of
// about 2^-22 (PTX ISA); the argument here is -x^2 log2(e) <= 0.
__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// T and Q' = c4 exp(-x^2) (c4 = 4/sqrt(pi) in working units).
// Linear table: distances in units of x_c, the coordinate runs downwards,
// s' = sat(1 + 1/(2N) - r / x_c) = 1 - s with the forward kernel's
// s = r / x_c - 1/(2N), and rint(s' N) = N - rint(s N): entry 0 is the zero
// entry (beyond the cutoff), entry N - k holds interval k as one float4
// (A_T + N D_T, -N D_T, c4 (A_Q + N D_Q), -c4 N D_Q) in intercept form of s'.
// The downward coordinate lets coincident pairs reach the zero entry for
// free: there 1/r = +inf, r^2 (-1/r) is NaN and the saturating FMA flushes
// NaN to 0.  Cubic: t = u - 1/2 in table units (u = x N / x_c), the T and Q
// coefficient float4s in two arrays.  Entry N is zero.
template <int TM>
__device__ __forceinline__ void eval_TQ(float t, float x, float x_c, unsigned tab_bias,
                                        unsigned q_off, float nmax, float c4, float& T, float& Q)
{
    if (TM == TM_EXACT) {
        const float q = expf(-x * x);
        const float tv = erfcf(x) + kTwoOverSqrtPi * x * q;
        const bool in = x < x_c;
        T = in ? tv : 0.0f;
        Q = in ? c4 * q : 0.0f;
    } else if (TM == TM_LINEAR) {  // t = s here
        const float fk = fmaf(t, nmax, kMagic);
        const float4 c = lds_f4((unsigned)__float_as_int(fk) * 16u + tab_bias);
        T = fmaf(t, c.y, c.x);
        Q = fmaf(t, c.w, c.z);
    } else {
        t = fminf(t, nmax);
        const float fk = t + kMagic;
        const unsigned a = (unsigned)__float_as_int(fk) * 16u + tab_bias;
        const float4 c = lds_f4(a);
        {
            const float f = t - (fk - kMagic);
            const float4 d = lds_f4(a + q_off);
            T = fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
            Q = c4 * fmaf(f, fmaf(f, fmaf(f, d.w, d.z), d.y), d.x);
        }
    }
}

template <int ACC>
struct Acc4 {
    double d[4] = {0, 0, 0, 0};
    float s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    __device__ __forceinline__ void fold(float* f)
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (ACC == PSR_ACC_FP64) {
                d[i] += (double)f[i];
            } else {
                float ss, ee;
                two_sum(s[i], f[i], ss, ee);
                s[i] = ss;
                c[i] += ee;
            }
            f[i] = 0.0f;
        }
    }
};

// Combine the S stream partials of each target and write dL/dx (scaled by
// gx = G/(8 r_s^3) sc^3) and dL/dm (gm = -G/(4 r_s^2) sc^2) in the original
// order.
template <int ACC, int R>
__device__ __forceinline__ void adj_finish(const FwdArgs& a, int4 li, Acc4<ACC>* acc,
                                           const bool* act, int lane, int s, int q, int S, int T,
                                           float gx, float gm, float4* __restrict__ stage)
{
    // Combine the S stream partials through the staging buffer: each target
    // slot r has its own region (1 KB) and the accesses are volatile, so no
    // slot's writes can meet another slot's reads whatever the compiler's
    // ordering (a shared region let the second slot's stores overtake the
    // first slot's loads).
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (ACC == PSR_ACC_FP64) {
            volatile double* red = reinterpret_cast<volatile double*>(stage) + 128 * r;
#pragma unroll
            for (int i = 0; i < 4; ++i) red[4 * lane + i] = acc[r].d[i];
            __syncwarp();
            if (s == 0 && act[r]) {
                double t4[4] = {acc[r].d[0], acc[r].d[1], acc[r].d[2], acc[r].d[3]};
                for (int t = 1; t < S; ++t)
#pragma unroll
                    for (int i = 0; i < 4; ++i) t4[i] += red[4 * (lane + t * T) + i];
                const int idx = a.perm[li.x + q + T * r];
                float* o = reinterpret_cast<float*>(a.out) + 3LL * idx;
                o[0] = (float)(t4[0] * (double)gx);
                o[1] = (float)(t4[1] * (double)gx);
                o[2] = (float)(t4[2] * (double)gx);
                if (a.out_m) reinterpret_cast<float*>(a.out_m)[idx] = (float)(t4[3] * (double)gm);
            }
        } else {
            volatile float* red = reinterpret_cast<volatile float*>(stage) + 256 * r;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                red[8 * lane + 2 * i] = acc[r].s[i];
                red[8 * lane + 2 * i + 1] = acc[r].c[i];
            }
            __syncwarp();
            if (s == 0 && act[r]) {
                float hi[4], lo[4], u, v;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    hi[i] = acc[r].s[i];
                    lo[i] = acc[r].c[i];
                }
                for (int t = 1; t < S; ++t)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const volatile float* o = red + 8 * (lane + t * T) + 2 * i;
                        two_sum(hi[i], o[0], u, v);
                        hi[i] = u;
                        lo[i] += o[1] + v;
                    }
                const int idx = a.perm[li.x + q + T * r];
                float* o = reinterpret_cast<float*>(a.out) + 3LL * idx;
                o[0] = (hi[0] + lo[0]) * gx;
                o[1] = (hi[1] + lo[1]) * gx;
                o[2] = (hi[2] + lo[2]) * gx;
                if (a.out_m) reinterpret_cast<float*>(a.out_m)[idx] = (hi[3] + lo[3]) * gm;
            }
        }
        __syncwarp();
    }
}

// Running sums of the two-targets-per-lane path in shared memory: the
// register state of two targets (coordinates, cotangents, chunk partials and
// 2 x 4 FP64 sums) does not fit the 80 registers of 3 blocks per SM, and the
// sums, touched once per staged chunk, are the cheapest part to move out.
// Slot (r, i), target r of the lane and component i (x, y, z, m), is the
// 8-byte word at 256 (4 r + i) + 8 lane of the warp's accumulator block (a
// warp's access to one slot is one conflict-free 256-byte row): one double,
// or the compensated pair (sum, compensation).  The accesses are volatile so
// that none is merged with or moved across another.
constexpr int kAdjAccF4 = 128;  // accumulator block per warp (float4): 2 targets x 4 x 32 lanes x 8 B

__device__ __forceinline__ unsigned acc_slot(unsigned base, int r, int i, int lane)
{
    return base + 256u * (unsigned)(4 * r + i) + 8u * (unsigned)lane;
}

__device__ __forceinline__ double acc_ld_f64(unsigned a)
{
    double d;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(d) : "r"(a) : "memory");
    return d;
}

__device__ __forceinline__ float2 acc_ld_f2(unsigned a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

// zero the lane's R x 4 slots
template <int R>
__device__ __forceinline__ void acc_zero_all(unsigned base, int lane)
{
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm volatile("st.shared.v2.f32 [%0], {%1, %1};" ::"r"(acc_slot(base, r, i, lane)),
                         "f"(0.0f)
                         : "memory");
    __syncwarp();
}

// fold the lane's R x 4 chunk partials into its slots and clear them
template <int ACC, int R>
__device__ __forceinline__ void acc_fold_all(unsigned base, int lane, float (*f)[4])
{
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const unsigned a = acc_slot(base, r, i, lane);
            if (ACC == PSR_ACC_FP64) {
                const double d = acc_ld_f64(a) + (double)f[r][i];
                asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(d) : "memory");
            } else {
                const float2 v = acc_ld_f2(a);
                float ss, ee;
                two_sum(v.x, f[r][i], ss, ee);
                asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(ss), "f"(v.y + ee)
                             : "memory");
            }
            f[r][i] = 0.0f;
        }
}

// adj_finish for sums kept in shared memory: the S stream partials of each
// target are the slots of lanes q, q + T, ..., q + (S-1) T, combined in that
// order (the order of adj_finish).
template <int ACC, int R>
__device__ __forceinline__ void adj_finish_smem(const FwdArgs& a, int4 li, unsigned accb,
                                                const bool* act, int lane, int s, int q, int S,
                                                int T, float gx, float gm)
{
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (s != 0 || !act[r]) continue;
        const int idx = a.perm[li.x + q + T * r];
        float* o = reinterpret_cast<float*>(a.out) + 3LL * idx;
        if (ACC == PSR_ACC_FP64) {
            double t4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) t4[i] = acc_ld_f64(acc_slot(accb, r, i, lane));
            for (int t = 1; t < S; ++t)
#pragma unroll
                for (int i = 0; i < 4; ++i) t4[i] += acc_ld_f64(acc_slot(accb, r, i, lane + t * T));
            o[0] = (float)(t4[0] * (double)gx);
            o[1] = (float)(t4[1] * (double)gx);
            o[2] = (float)(t4[2] * (double)gx);
            if (a.out_m) reinterpret_cast<float*>(a.out_m)[idx] = (float)(t4[3] * (double)gm);
        } else {
            float hi[4], lo[4], u, v;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 w = acc_ld_f2(acc_slot(accb, r, i, lane));
                hi[i] = w.x;
                lo[i] = w.y;
            }
            for (int t = 1; t < S; ++t)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 w = acc_ld_f2(acc_slot(accb, r, i, lane + t * T));
                    two_sum(hi[i], w.x, u, v);
                    hi[i] = u;
                    lo[i] += w.y + v;
                }
            o[0] = (hi[0] + lo[0]) * gx;
            o[1] = (hi[1] + lo[1]) * gx;
            o[2] = (hi[2] + lo[2]) * gx;
            if (a.out_m) reinterpret_cast<float*>(a.out_m)[idx] = (hi[3] + lo[3]) * gm;
        }
    }
    __syncwarp();
}

// One target leaf on one warp (same decomposition as the forward kernels;
// staged payload: two float4 per source particle, (x, y, z, c_z) and
// (c_x, c_y, m, m), so that the x, y halves of d = x_j - x_k and of
// v = m_k c_j - m_j c_k come from register pairs in f32x2 arithmetic: one
// FADD2 and one FMUL2 + FFMA2 instead of five scalar instructions, with the
// same rounding.  The rest of the pair stays scalar, where it spreads over
// both halves of the FMA pipe (f32x2 runs on one).  With two targets per
// lane the running sums live in shared memory (acc_fold_all).
template <int TM, int ACC, bool EQM, int R>
__device__ __forceinline__ void adj_item(const FwdArgs& a, int I, int4 li, unsigned tab_bias,
                                         unsigned q_off, float4* __restrict__ stage,
                                         float4* __restrict__ meta, unsigned accb)
{
    constexpr bool SA = R == 2;  // sums in shared memory
    const int lane = threadIdx.x & 31;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const float4* __restrict__ cs = reinterpret_cast<const float4*>(a.cot_sorted);
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
    // working unit: x for the exact path, x / x_c for the linear table (whose
    // entries carry c4), table intervals for the cubic one
    const float sc = TM == TM_EXACT ? 1.0f : TM == TM_LINEAR ? 1.0f / x_c : (float)a.table_n / x_c;
    const float xscale = 1.0f / sc;
    const float c4 = kFourOverSqrtPi / (sc * sc * sc);  // (4/sqrt(pi)) in working units
    const float sref = 1.0f + 0.5f / nmax;               // linear: s' = sat(1 + 1/(2N) - r / x_c)
    const float unit = bx.unit;
    const int4 ci = lcen[I];

    float4 xi[R];
    float2 nxy[R], mk2[R], nck[R];  // (-x_k, -y_k), (m_k, m_k), (-c_kx, -c_ky)
    float nckz[R];
    bool act[R];
    float f[R][4];
    Acc4<ACC> acc[SA ? 1 : R];
    if (SA) acc_zero_all<R>(accb, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = q + T * r;
        act[r] = on && t < nI;
        xi[r] = pf[li.x + (act[r] ? t : 0)];
        xi[r].x *= sc;
        xi[r].y *= sc;
        xi[r].z *= sc;
        const float4 ck = cs[li.x + (act[r] ? t : 0)];
        nxy[r] = make_float2(-xi[r].x, -xi[r].y);
        mk2[r] = make_float2(xi[r].w, xi[r].w);
        nck[r] = make_float2(-ck.x, -ck.y);
        nckz[r] = -ck.z;
#pragma unroll
        for (int i = 0; i < 4; ++i) f[r][i] = 0.0f;
    }
    {  // the target box for the cull (shared memory, after the entry records)
        float lx = kInf, ly = kInf, lz = kInf, hx = -kInf, hy = -kInf, hz = -kInf;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (act[r]) {
                lx = fminf(lx, xi[r].x); hx = fmaxf(hx, xi[r].x);
                ly = fminf(ly, xi[r].y); hy = fmaxf(hy, xi[r].y);
                lz = fminf(lz, xi[r].z); hz = fmaxf(hz, xi[r].z);
            }
        cull_box(lx, ly, lz, hx, hy, hz, x_c * sc, meta + kMetaPerWarp);
    }
    const long long re = a.rowptr[I + 1];
    long long e0 = a.rowptr[I];
    while (e0 < re) {
        int nst;
        e0 += stage_chunk<2>(a, e0, re, ci, unit, sc, a.stage_cap, stage, meta, nst);
        if (on) {
            // p = (x, y, z, c_z), c = (c_x, c_y, m, m) of one staged source
            auto eval = [&](const float4 p, const float4 c) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 dxy = add2(make_float2(p.x, p.y), nxy[r]);
                    const float dx = dxy.x, dy = dxy.y, dz = p.z - xi[r].z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    // the self pair and coincident pairs contribute nothing:
                    // on the linear path the NaN coordinate at r = 0 selects
                    // the zero entry (T = Q = 0) and the clamped 1/r keeps
                    // every product finite; elsewhere 1/r = 0 makes tr3 and
                    // hh zero (T and Q stay finite)
                    float rinv, tv;
                    if (TM == TM_LINEAR) {
                        const float ri = rsqrt_ftz(r2);
                        tv = fma_sat(r2, -ri, sref);
                        rinv = fminf(ri, kRinvMax);
                    } else {
                        rinv = r2 > 0.0f ? rsqrt_ftz(r2) : 0.0f;
                        tv = fmaf(r2, rinv, -0.5f);
                    }
                    float Tv, Qv;
                    eval_TQ<TM>(tv, r2 * rinv * xscale, x_c, tab_bias, q_off, nmax, c4, Tv, Qv);
                    const float rinv2 = rinv * rinv;
                    const float tr3 = Tv * rinv2 * rinv;                          // T/u^3
                    const float hh = -rinv2 * fmaf(3.0f, tr3, Qv);                // g'(r)/r
                    // v = m_k c_j - m_j c_k
                    // (equal masses: v = m (c_j - c_k), m applied with gx)
                    const float2 vxy = EQM ? add2(make_float2(c.x, c.y), nck[r])
                                           : fma2(mk2[r], make_float2(c.x, c.y),
                                                  mul2(make_float2(c.z, c.w), nck[r]));
                    const float vx = vxy.x, vy = vxy.y;
                    const float vz = EQM ? p.w + nckz[r] : fmaf(xi[r].w, p.w, c.z * nckz[r]);
                    const float hd = hh * fmaf(dx, vx, fmaf(dy, vy, dz * vz));
                    f[r][0] = fmaf(tr3, vx, fmaf(hd, dx, f[r][0]));
                    f[r][1] = fmaf(tr3, vy, fmaf(hd, dy, f[r][1]));
                    f[r][2] = fmaf(tr3, vz, fmaf(hd, dz, f[r][2]));
                    f[r][3] = fmaf(tr3, fmaf(dx, c.x, fmaf(dy, c.y, dz * p.w)), f[r][3]);
                }
            };
            // Stream s takes staged sources s, s + S, ... in that order: four
            // per iteration with one target per lane, two with two targets
            // (then the rest one by one), which halves and quarters the loop
            // instructions (the two-source loop was 4 % faster than the plain
            // one with the FP64 fold, 9 % with the compensated one; four
            // sources gain 0.7 % more).  The loop walks 32-bit shared
            // addresses with volatile loads, as in the forward kernel (3 %
            // faster than pointer arithmetic).
            unsigned sa = smem_u32(stage + 2 * s);
            const unsigned se = smem_u32(stage + 2 * nst), st1 = 32u * (unsigned)S;
            if (R == 1) {
#pragma unroll 1
                for (; sa + 3u * st1 < se; sa += 4u * st1) {
                    const float4 p0 = lds_f4_v(sa), c0 = lds_f4_v(sa + 16u);
                    const float4 p1 = lds_f4_v(sa + st1), c1 = lds_f4_v(sa + st1 + 16u);
                    const float4 p2 = lds_f4_v(sa + 2u * st1), c2 = lds_f4_v(sa + 2u * st1 + 16u);
                    const float4 p3 = lds_f4_v(sa + 3u * st1), c3 = lds_f4_v(sa + 3u * st1 + 16u);
                    eval(p0, c0);
                    eval(p1, c1);
                    eval(p2, c2);
                    eval(p3, c3);
                }
#pragma unroll 1
                for (; sa < se; sa += st1) eval(lds_f4_v(sa), lds_f4_v(sa + 16u));
            } else {
#pragma unroll 1
                for (; sa + st1 < se; sa += 2u * st1) {
                    const float4 p0 = lds_f4_v(sa), c0 = lds_f4_v(sa + 16u);
                    const float4 p1 = lds_f4_v(sa + st1), c1 = lds_f4_v(sa + st1 + 16u);
                    eval(p0, c0);
                    eval(p1, c1);
                }
                if (sa < se) eval(lds_f4_v(sa), lds_f4_v(sa + 16u));
            }
            if (SA) {
                acc_fold_all<ACC, R>(accb, lane, f);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) acc[SA ? 0 : r].fold(f[r]);
            }
        }
        __syncwarp();
    }
    const float gx = bx.g_adj * sc * sc * sc * (EQM ? bx.m_eq : 1.0f);
    if (SA)
        adj_finish_smem<ACC, R>(a, li, accb, act, lane, s, q, S, T, gx, -bx.g_adjm * sc * sc);
    else
        adj_finish<ACC, R>(a, li, acc, act, lane, s, q, S, T, gx, -bx.g_adjm * sc * sc, stage);
}

// Packed variant of adj_item (PSR_KERNEL_PACKED): each stream takes staged
// source PAIRS and evaluates both sources of a pair at once in sm_100+ f32x2
// arithmetic (31 of the 36 FP32 operations of a pair are vector algebra on d,
// v and the cotangents).  The table step and 1/r stay scalar (two lookups, two
// rsqrt); the linear path reads T alone (8-byte entries) and takes exp(-x^2)
// from ex2, zeroed with T beyond the cutoff.  Qn carries -c4, so g'(r)/r is
// rinv2 (-3 T/r^3 + Qn) with no negation.  Same arithmetic per pair as
// adj_item up to rounding order.  It executes 23 % fewer instructions than
// adj_item but is not faster: every f32x2 instruction runs on the heavy half
// of the FMA pipe, whose load and the dependency chains of 24 warps per SM
// hold it at about 60 % of issue.  One target per lane unless leaves exceed
// 32 particles (the two-targets state spills at 80 registers).
template <int TM, int ACC, bool EQM, int R>
__device__ __forceinline__ void adj_item_pk(const FwdArgs& a, int I, int4 li, unsigned tab_bias,
                                            unsigned q_off, float4* __restrict__ stage,
                                            float4* __restrict__ meta)
{
    const int lane = threadIdx.x & 31;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const float4* __restrict__ cs = reinterpret_cast<const float4*>(a.cot_sorted);
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
    const float sc = TM == TM_EXACT ? 1.0f : TM == TM_LINEAR ? 1.0f / x_c : (float)a.table_n / x_c;
    const float xscale = 1.0f / sc;
    const float c4n = -kFourOverSqrtPi / (sc * sc * sc);  // -(4/sqrt(pi)) in working units
    const float soff = -0.5f / nmax;
    const float unit = bx.unit;
    const int4 ci = lcen[I];

    float2 nx[R], ny[R], nz[R], mk[R], ncx[R], ncy[R], ncz[R], fx[R], fy[R], fz[R], fm[R];
    bool act[R];
    Acc4<ACC> acc[R];
    float lx = kInf, ly = kInf, lz = kInf, hx = -kInf, hy = -kInf, hz = -kInf;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = q + T * r;
        act[r] = on && t < nI;
        const float4 v = pf[li.x + (act[r] ? t : 0)];
        const float4 c = cs[li.x + (act[r] ? t : 0)];
        const float x = v.x * sc, y = v.y * sc, z = v.z * sc;
        nx[r] = make_float2(-x, -x);
        ny[r] = make_float2(-y, -y);
        nz[r] = make_float2(-z, -z);
        mk[r] = make_float2(v.w, v.w);
        ncx[r] = make_float2(-c.x, -c.x);
        ncy[r] = make_float2(-c.y, -c.y);
        ncz[r] = make_float2(-c.z, -c.z);
        fx[r] = fy[r] = fz[r] = fm[r] = make_float2(0.0f, 0.0f);
        if (act[r]) {
            lx = fminf(lx, x); hx = fmaxf(hx, x);
            ly = fminf(ly, y); hy = fmaxf(hy, y);
            lz = fminf(lz, z); hz = fmaxf(hz, z);
        }
    }
    cull_box(lx, ly, lz, hx, hy, hz, x_c * sc, meta + kMetaPerWarp);
    const float2 m3 = make_float2(-3.0f, -3.0f);
    const float2 c4n2 = make_float2(c4n, c4n);
    // exp(-x^2) = 2^(r2 qarg): r2 is in units of x_c^2 on the linear path
    const float qarg = -kLog2E * x_c * x_c;
    const long long re = a.rowptr[I + 1];
    long long e0 = a.rowptr[I];
    while (e0 < re) {
        int nst;
        e0 += stage_chunk<3>(a, e0, re, ci, unit, sc, a.stage_cap, stage, meta, nst);
        if (on) {
            const int npair = (nst + 1) >> 1;
#pragma unroll 1
            for (int k = s; k < npair; k += S) {
                const float4 A = stage[4 * k], B = stage[4 * k + 1];
                const float4 C = stage[4 * k + 2], D = stage[4 * k + 3];
                const float2 px = make_float2(A.x, A.y), py = make_float2(A.z, A.w);
                const float2 pz = make_float2(B.x, B.y), pm = make_float2(B.z, B.w);
                const float2 cx = make_float2(C.x, C.y), cy = make_float2(C.z, C.w);
                const float2 cz = make_float2(D.x, D.y);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 dx = add2(px, nx[r]), dy = add2(py, ny[r]), dz = add2(pz, nz[r]);
                    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                    // self and coincident pairs: 1/r = 0 zeroes their terms
                    const float2 rinv = make_float2(r2.x > 0.0f ? rsqrt_ftz(r2.x) : 0.0f,
                                                    r2.y > 0.0f ? rsqrt_ftz(r2.y) : 0.0f);
                    float2 Tv, Qn;
                    if (TM == TM_LINEAR) {
                        // T from the table (8-byte entries, as in the forward);
                        // -c4 exp(-x^2) from ex2, zeroed with T beyond the
                        // cutoff (the table's zero entry): half the table's
                        // shared-memory traffic for one MUFU and three ALU
                        // instructions per pair
                        const float2 sv = make_float2(fma_sat(r2.x, rinv.x, soff),
                                                      fma_sat(r2.y, rinv.y, soff));
                        Tv = make_float2(linear_T(sv.x, nmax, tab_bias), linear_T(sv.y, nmax, tab_bias));
                        const float2 q2 = make_float2(ex2_ftz(r2.x * qarg), ex2_ftz(r2.y * qarg));
                        Qn = mul2(c4n2, make_float2(Tv.x > 0.0f ? q2.x : 0.0f, Tv.y > 0.0f ? q2.y : 0.0f));
                    } else {
                        eval_TQ<TM>(fmaf(r2.x, rinv.x, -0.5f), r2.x * rinv.x * xscale, x_c, tab_bias,
                                    q_off, nmax, c4n, Tv.x, Qn.x);
                        eval_TQ<TM>(fmaf(r2.y, rinv.y, -0.5f), r2.y * rinv.y * xscale, x_c, tab_bias,
                                    q_off, nmax, c4n, Tv.y, Qn.y);
                    }
                    const float2 rinv2 = mul2(rinv, rinv);
                    const float2 tr3 = mul2(Tv, mul2(rinv2, rinv));           // T/u^3
                    const float2 hh = mul2(rinv2, fma2(m3, tr3, Qn));         // g'(r)/r
                    // m_k c_j - m_j c_k (equal masses: c_j - c_k, m applied with gx)
                    const float2 vx = EQM ? add2(cx, ncx[r]) : fma2(mk[r], cx, mul2(pm, ncx[r]));
                    const float2 vy = EQM ? add2(cy, ncy[r]) : fma2(mk[r], cy, mul2(pm, ncy[r]));
                    const float2 vz = EQM ? add2(cz, ncz[r]) : fma2(mk[r], cz, mul2(pm, ncz[r]));
                    const float2 hd = mul2(hh, fma2(dx, vx, fma2(dy, vy, mul2(dz, vz))));
                    fx[r] = fma2(tr3, vx, fma2(hd, dx, fx[r]));
                    fy[r] = fma2(tr3, vy, fma2(hd, dy, fy[r]));
                    fz[r] = fma2(tr3, vz, fma2(hd, dz, fz[r]));
                    fm[r] = fma2(tr3, fma2(dx, cx, fma2(dy, cy, mul2(dz, cz))), fm[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float f4[4] = {fx[r].x + fx[r].y, fy[r].x + fy[r].y, fz[r].x + fz[r].y,
                               fm[r].x + fm[r].y};
                acc[r].fold(f4);
                fx[r] = fy[r] = fz[r] = fm[r] = make_float2(0.0f, 0.0f);
            }
        }
        __syncwarp();
    }
    adj_finish<ACC, R>(a, li, acc, act, lane, s, q, S, T,
                       bx.g_adj * sc * sc * sc * (EQM ? bx.m_eq : 1.0f), -bx.g_adjm * sc * sc, stage);
}

// Shared memory: the table (T and Q), then per warp a staging buffer of
// stage_cap particles x 2 float4, 32 entry records and the two box slots,
// then the accumulator block of the two-targets path (kAdjAccF4).
template <int TM, int ACC, bool WIDE, bool PK, bool EQM>
__global__ void __launch_bounds__(256, 3) p2p_adj_f32_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const size_t tab_bytes = TM == TM_EXACT ? 0
                           : (size_t)(a.table_n + 1) * (TM == TM_LINEAR ? 16 : 32);
    float4* stage = reinterpret_cast<float4*>(smem + tab_bytes) +
                    (size_t)warp * (2 * a.stage_cap + kWarpMeta + kAdjAccF4);
    float4* meta = stage + 2 * a.stage_cap;
    const unsigned accb = smem_u32(meta + kWarpMeta);
    if (TM != TM_EXACT) {
        const float4* g = reinterpret_cast<const float4*>(a.table);
        const float4* gq = g + (kMaxTableN + 1);
        float4* sT = reinterpret_cast<float4*>(smem);
        for (int i = threadIdx.x; i <= a.table_n; i += blockDim.x) {
            if (TM == TM_LINEAR && PK) {
                // the packed variant reads T alone, (A_T, N D_T) as in the
                // forward kernel, and takes exp(-x^2) from ex2 (adj_item_pk)
                const float4 u = g[i];
                reinterpret_cast<float2*>(smem)[i] = make_float2(u.z, (float)a.table_n * u.y);
            } else if (TM == TM_LINEAR) {
                // interval i at entry N - i, in the downward coordinate s'
                // (eval_TQ): (A_T + N D_T, -N D_T, c4 (A_Q + N D_Q), -c4 N D_Q),
                // c4 = (4/sqrt(pi)) x_c^3 (the linear path works in units of
                // x_c; all boxes of a handle share x_c, as they share the
                // table); each entry is formed in FP64 and rounded once
                const float4 u = g[i], v = gq[i];
                const double n = (double)a.table_n, xc = a.boxes[0].x_c;
                const double c4 = 2.2567583341910251 * xc * xc * xc;
                sT[a.table_n - i] = make_float4((float)((double)u.z + n * (double)u.y),
                                                (float)(-n * (double)u.y),
                                                (float)(c4 * ((double)v.z + n * (double)v.y)),
                                                (float)(-c4 * n * (double)v.y));
            } else {
                sT[i] = g[i];
                sT[a.table_n + 1 + i] = gq[i];
            }
        }
        __syncthreads();
    }
    const unsigned tab_bias = smem_u32(smem) - (unsigned)kMagicBits * (TM == TM_LINEAR && PK ? 8u : 16u);
    const unsigned q_off = (unsigned)(a.table_n + 1) * 16u;
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.ctrl + kCtrlTicketAdj, 1u) * a.item_stride + a.item_offset;
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
            if (WIDE && prefer_two_per_lane(li.y))
                adj_item_pk<TM, ACC, EQM, 2>(a, I, li, tab_bias, q_off, stage, meta);
            else
                adj_item_pk<TM, ACC, EQM, 1>(a, I, li, tab_bias, q_off, stage, meta);
        } else if (WIDE && prefer_two_per_lane(li.y)) {
            // leaves of 11-12 and 17-20 particles up to 32 (and all larger
            // ones); at equal lane fill one target per lane is faster (its
            // state fits the registers and its loop takes four sources per
            // iteration): sending the ties to two targets cost 1.4 %
            adj_item<TM, ACC, EQM, 2>(a, I, li, tab_bias, q_off, stage, meta, accb);
        } else {
            adj_item<TM, ACC, EQM, 1>(a, I, li, tab_bias, q_off, stage, meta, accb);
        }
    }
    persistent_exit(a.ctrl + kCtrlTicketAdj, a.ctrl + kCtrlDoneAdj);
}

// ------------------------------------------------------------------ FP64 --
template <int R>
__device__ __forceinline__ void adj64_item(const FwdArgs& a, int I, int4 li)
{
    const int lane = threadIdx.x & 31;
    const double4* __restrict__ pd = reinterpret_cast<const double4*>(a.pd);
    const double4* __restrict__ cs = reinterpret_cast<const double4*>(a.cot_sorted);
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    const int nI = li.y;
    const int lgT = (R == 2) ? 5 : stream_log2(nI);
    const int q = lane & ((1 << lgT) - 1);
    const int s = lane >> lgT;
    const int S = 32 >> lgT;
    const BoxDev& bx = a.boxes[li.z];
    const double L = bx.L, rc2 = bx.rc2, inv2rs = bx.inv_2rs;
    const double c2 = 1.1283791670955126;  // 2/sqrt(pi)
    // exp(-x^2) / (2 sqrt(pi) r_s^3)
    const double cq = 1.0 / (2.0 * 1.7724538509055160 * bx.r_s * bx.r_s * bx.r_s);
    double4 xi[R], ck[R];
    bool act[R];
    double t3[R][3], g[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = q + 32 * r;
        act[r] = t < nI;
        xi[r] = pd[li.x + (act[r] ? t : 0)];
        ck[r] = cs[li.x + (act[r] ? t : 0)];
        for (int i = 0; i < 4; ++i) g[r][i] = 0.0;
        t3[r][0] = t3[r][1] = t3[r][2] = 0.0;
    }
    const long long re = a.rowptr[I + 1];
    long long e = a.rowptr[I] + s;
    int j = 0, jend = 0;
    for (;;) {
        if (j >= jend) {
            bool found = false;
            while (e < re) {
                unsigned ent = a.pairs[e];
                e += S;
                int J = (int)(ent >> 5);
                unsigned code = ent & 31u;
                if (J >= a.n_leaves || code >= (unsigned)kShiftCodes) {
                    set_error(a.ctrl, J >= a.n_leaves ? kErrLeafIndex : kErrShiftCode);
                    continue;
                }
                int4 lj = leaf[J];
                if (lj.x < 0 || lj.y < 0 || (long long)lj.x + lj.y > a.n) {
                    set_error(a.ctrl, kErrParticleRange);
                    continue;
                }
                int nx, ny, nz;
                decode_shift(code, nx, ny, nz);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    t3[r][0] = xi[r].x - nx * L;
                    t3[r][1] = xi[r].y - ny * L;
                    t3[r][2] = xi[r].z - nz * L;
                }
                j = lj.x;
                jend = lj.x + lj.y;
                found = true;
                break;
            }
            if (!found) break;
        }
        const double4 p = pd[j];
        const double4 c = cs[j];
        ++j;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double dx = p.x - t3[r][0], dy = p.y - t3[r][1], dz = p.z - t3[r][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2 && r2 > 0.0) {
                double rr = sqrt(r2);
                double x = rr * inv2rs;
                double Q = exp(-x * x);
                double T = erfc(x) + c2 * x * Q;
                double gg = T / (r2 * rr);
                double hf = -3.0 * gg / r2 - cq * Q / r2;  // g'(r)/r
                double vx = xi[r].w * c.x - p.w * ck[r].x;
                double vy = xi[r].w * c.y - p.w * ck[r].y;
                double vz = xi[r].w * c.z - p.w * ck[r].z;
                double hd = hf * (dx * vx + dy * vy + dz * vz);
                g[r][0] += gg * vx + hd * dx;
                g[r][1] += gg * vy + hd * dy;
                g[r][2] += gg * vz + hd * dz;
                g[r][3] += gg * (dx * c.x + dy * c.y + dz * c.z);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        for (int off = 1 << lgT; off < 32; off <<= 1)
            for (int i = 0; i < 4; ++i) g[r][i] += __shfl_xor_sync(kFull, g[r][i], off);
    if (s == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!act[r]) continue;
            int idx = a.perm[li.x + q + 32 * r];
            double* o = reinterpret_cast<double*>(a.out) + 3LL * idx;
            o[0] = bx.G * g[r][0];
            o[1] = bx.G * g[r][1];
            o[2] = bx.G * g[r][2];
            if (a.out_m) reinterpret_cast<double*>(a.out_m)[idx] = -bx.G * g[r][3];
        }
    }
}

template <bool WIDE>
__global__ void __launch_bounds__(256) p2p_adj_f64_kernel(const FwdArgs a)
{
    const int lane = threadIdx.x & 31;
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.ctrl + kCtrlTicketAdj, 1u) * a.item_stride + a.item_offset;
        it = __shfl_sync(kFull, it, 0);
        if (it >= a.n_items) break;
        int I = a.items[it];
        if (I < 0 || I >= a.n_leaves) {
            if (lane == 0) set_error(a.ctrl, kErrItemIndex);
            continue;
        }
        int4 li = leaf[I];
        if (li.y <= 0 || li.y > a.max_leaf || (long long)li.x + li.y > a.n || li.z < 0 ||
            li.z >= a.nbox) {
            if (lane == 0) set_error(a.ctrl, kErrParticleRange);
            continue;
        }
        if (WIDE && li.y > 32)
            adj64_item<2>(a, I, li);
        else
            adj64_item<1>(a, I, li);
    }
    persistent_exit(a.ctrl + kCtrlTicketAdj, a.ctrl + kCtrlDoneAdj);
}

// Morton-order source payload of the cotangent: cs[k] = (c[perm[k]], 0).
template <typename T, typename T4>
__global__ void gather_cot_kernel(const T* __restrict__ cot, const int32_t* __restrict__ perm,
                                  T4* __restrict__ cs, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    long long i = perm[k];
    T4 v;
    v.x = cot[3 * i];
    v.y = cot[3 * i + 1];
    v.z = cot[3 * i + 2];
    v.w = 0;
    cs[k] = v;
}

size_t adj_f32_smem(int precision, int interp, int table_n, int warps, int cap)
{
    size_t tab = precision != PSR_FP32_TABLE ? 0
               : (size_t)(table_n + 1) * (interp == PSR_LINEAR ? 16 : 32);
    return tab + (size_t)warps * (2 * cap + kWarpMeta + kAdjAccF4) * 16;
}

template <int TM, int ACC, bool EQM>
static int launch_adj_e(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    // always with the two-targets-per-lane path (mid-size leaves fill more lanes)
    // (the packed variant carries it only for leaves above 32 particles: its
    // per-target state would spill)
    auto k = a.variant != PSR_KERNEL_PACKED ? p2p_adj_f32_kernel<TM, ACC, true, false, EQM>
             : a.max_leaf > 32              ? p2p_adj_f32_kernel<TM, ACC, true, true, EQM>
                                            : p2p_adj_f32_kernel<TM, ACC, false, true, EQM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    k<<<a.blocks, a.warps_per_block * 32, smem, st>>>(a);
    return (int)cudaGetLastError();
}

// equal masses: m leaves the pair sums (v = m (c_j - c_k))
template <int TM, int ACC>
static int launch_adj_t(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    return a.equal_mass ? launch_adj_e<TM, ACC, true>(a, smem, st)
                        : launch_adj_e<TM, ACC, false>(a, smem, st);
}

int launch_adj_f32(const FwdArgs& a, int precision, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    long long nb = (a.n + 255) / 256;
    gather_cot_kernel<float, float4><<<(unsigned)nb, 256, 0, st>>>(
        reinterpret_cast<const float*>(a.cot), a.perm, reinterpret_cast<float4*>(a.cot_sorted), a.n);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return (int)e0;
    size_t smem = adj_f32_smem(precision, a.interp, a.table_n, a.warps_per_block, a.stage_cap);
    if (precision == PSR_FP32_EXACT)
        return a.accum == PSR_ACC_FP64 ? launch_adj_t<TM_EXACT, PSR_ACC_FP64>(a, smem, st)
                                       : launch_adj_t<TM_EXACT, PSR_ACC_KAHAN32>(a, smem, st);
    if (a.interp == PSR_LINEAR)
        return a.accum == PSR_ACC_FP64 ? launch_adj_t<TM_LINEAR, PSR_ACC_FP64>(a, smem, st)
                                       : launch_adj_t<TM_LINEAR, PSR_ACC_KAHAN32>(a, smem, st);
    return a.accum == PSR_ACC_FP64 ? launch_adj_t<TM_CUBIC, PSR_ACC_FP64>(a, smem, st)
                                   : launch_adj_t<TM_CUBIC, PSR_ACC_KAHAN32>(a, smem, st);
}

int launch_adj_f64(const FwdArgs& a, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    long long nb = (a.n + 255) / 256;
    gather_cot_kernel<double, double4><<<(unsigned)nb, 256, 0, st>>>(
        reinterpret_cast<const double*>(a.cot), a.perm, reinterpret_cast<double4*>(a.cot_sorted), a.n);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return (int)e0;
    if (a.max_leaf > 32) p2p_adj_f64_kernel<true><<<a.blocks, a.warps_per_block * 32, 0, st>>>(a);
    else p2p_adj_f64_kernel<false><<<a.blocks, a.warps_per_block * 32, 0, st>>>(a);
    return (int)cudaGetLastError();
}

int adj_occupancy(int precision, int interp, int accum, int warps, int max_leaf, int table_n,
                  int cap, int variant, int* out)
{
    const bool wide = max_leaf > 32;
    size_t smem = 0;
    const void* f;
    if (precision == PSR_FP64) {
        f = wide ? (const void*)p2p_adj_f64_kernel<true> : (const void*)p2p_adj_f64_kernel<false>;
    } else {
        smem = adj_f32_smem(precision, interp, table_n, warps, cap);
#define PSR_PICK(TM, ACC) (variant != PSR_KERNEL_PACKED \
                               ? (const void*)p2p_adj_f32_kernel<TM, ACC, true, false, false> \
                               : wide ? (const void*)p2p_adj_f32_kernel<TM, ACC, true, true, false> \
                                      : (const void*)p2p_adj_f32_kernel<TM, ACC, false, true, false>)
        if (precision == PSR_FP32_EXACT)
            f = accum == PSR_ACC_FP64 ? PSR_PICK(TM_EXACT, PSR_ACC_FP64) : PSR_PICK(TM_EXACT, PSR_ACC_KAHAN32);
        else if (interp == PSR_LINEAR)
            f = accum == PSR_ACC_FP64 ? PSR_PICK(TM_LINEAR, PSR_ACC_FP64) : PSR_PICK(TM_LINEAR, PSR_ACC_KAHAN32);
        else
            f = accum == PSR_ACC_FP64 ? PSR_PICK(TM_CUBIC, PSR_ACC_FP64) : PSR_PICK(TM_CUBIC, PSR_ACC_KAHAN32);
#undef PSR_PICK
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
        }
    }
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, warps * 32, smem);
}

}  // namespace psr
