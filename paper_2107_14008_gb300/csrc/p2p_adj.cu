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

#include "kcommon.cuh"

namespace psr {

enum { TA_EXACT = 0, TA_LINEAR = 1, TA_CUBIC = 2 };
constexpr float kFourOverSqrtPi = 2.2567583341910251f;

template <int TM>
__device__ __forceinline__ void eval_TQ(float x, const float* tT, const float* tQ, float inv_h,
                                        float nmax, float x_c, float& T, float& Q)
{
    if (TM == TA_EXACT) {
        float q = expf(-x * x);
        float t = erfcf(x) + kTwoOverSqrtPi * x * q;
        bool in = x < x_c;
        T = in ? t : 0.0f;
        Q = in ? q : 0.0f;
    } else {
        float t = fminf(fmaf(x, inv_h, -0.5f), nmax);
        float fk = t + kMagic;
        int k = __float_as_int(fk) - kMagicBits;
        float f = t - (fk - kMagic);
        if (TM == TA_LINEAR) {
            float4 c = reinterpret_cast<const float4*>(tT)[k];  // (T mid, T diff, Q mid, Q diff)
            T = fmaf(f, c.y, c.x);
            Q = fmaf(f, c.w, c.z);
        } else {
            float4 c = reinterpret_cast<const float4*>(tT)[k];
            float4 d = reinterpret_cast<const float4*>(tQ)[k];
            T = fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
            Q = fmaf(f, fmaf(f, fmaf(f, d.w, d.z), d.y), d.x);
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
    __device__ __forceinline__ void reduce(int lgT)
    {
        for (int off = 1 << lgT; off < 32; off <<= 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (ACC == PSR_ACC_FP64) {
                    d[i] += __shfl_xor_sync(kFull, d[i], off);
                } else {
                    float os = __shfl_xor_sync(kFull, s[i], off), oc = __shfl_xor_sync(kFull, c[i], off);
                    float ss, ee;
                    two_sum(s[i], os, ss, ee);
                    s[i] = ss;
                    c[i] += oc + ee;
                }
            }
        }
    }
    __device__ __forceinline__ float get(int i, float g) const
    {
        return ACC == PSR_ACC_FP64 ? (float)(d[i] * (double)g) : (s[i] + c[i]) * g;
    }
};

template <int TM, int ACC, int R>
__device__ __forceinline__ void adj_item(const FwdArgs& a, int I, int4 li, const float* tT,
                                         const float* tQ)
{
    const int lane = threadIdx.x & 31;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const float4* __restrict__ cs = reinterpret_cast<const float4*>(a.cot_sorted);
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    const int4* __restrict__ lcen = reinterpret_cast<const int4*>(a.lcen);
    const int nI = li.y;
    const int lgT = (R == 2) ? 5 : stream_log2(nI);
    const int q = lane & ((1 << lgT) - 1);
    const int s = lane >> lgT;
    const int S = 32 >> lgT;
    const BoxDev& bx = a.boxes[li.z];
    const float unit = bx.unit, x_c = bx.x_c;
    const float nmax = (float)a.table_n, inv_h = (float)a.table_n / x_c;
    const int4 ci = lcen[I];

    float4 xi[R], ck[R];
    bool act[R];
    float t3[R][3], f[R][4];
    Acc4<ACC> acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = q + 32 * r;
        act[r] = t < nI;
        xi[r] = pf[li.x + (act[r] ? t : 0)];
        ck[r] = cs[li.x + (act[r] ? t : 0)];
#pragma unroll
        for (int i = 0; i < 4; ++i) f[r][i] = 0.0f;
        t3[r][0] = t3[r][1] = t3[r][2] = 0.0f;
    }
    int since = 0;
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
                int4 cj = lcen[J];
                int nx, ny, nz;
                decode_shift(code, nx, ny, nz);
                float ox = (float)(cj.x - ci.x + nx * (1 << kCentreShift)) * unit;
                float oy = (float)(cj.y - ci.y + ny * (1 << kCentreShift)) * unit;
                float oz = (float)(cj.z - ci.z + nz * (1 << kCentreShift)) * unit;
                if (since >= a.fold_every) {
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r].fold(f[r]);
                    since = 0;
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    t3[r][0] = xi[r].x - ox;
                    t3[r][1] = xi[r].y - oy;
                    t3[r][2] = xi[r].z - oz;
                }
                since += lj.y;
                j = lj.x;
                jend = lj.x + lj.y;
                found = true;
                break;
            }
            if (!found) break;
        }
        const float4 p = __ldg(pf + j);
        const float4 c = __ldg(cs + j);
        ++j;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float dx = p.x - t3[r][0], dy = p.y - t3[r][1], dz = p.z - t3[r][2];
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float rinv = rsqrtf(r2);
            float x = r2 * rinv;
            float T, Q;
            eval_TQ<TM>(x, tT, tQ, inv_h, nmax, x_c, T, Q);
            float rinv2 = rinv * rinv;
            float tr3 = T * rinv2 * rinv;                        // T / x^3
            float hh = -rinv2 * fmaf(3.0f, tr3, kFourOverSqrtPi * Q);  // -3T/x^5 - (4/sqrt(pi)) Q/x^2
            bool nz = r2 > 0.0f;
            tr3 = nz ? tr3 : 0.0f;
            hh = nz ? hh : 0.0f;
            float vx = fmaf(xi[r].w, c.x, -p.w * ck[r].x);
            float vy = fmaf(xi[r].w, c.y, -p.w * ck[r].y);
            float vz = fmaf(xi[r].w, c.z, -p.w * ck[r].z);
            float hd = hh * fmaf(dx, vx, fmaf(dy, vy, dz * vz));
            f[r][0] = fmaf(tr3, vx, fmaf(hd, dx, f[r][0]));
            f[r][1] = fmaf(tr3, vy, fmaf(hd, dy, f[r][1]));
            f[r][2] = fmaf(tr3, vz, fmaf(hd, dz, f[r][2]));
            f[r][3] = fmaf(tr3, fmaf(dx, c.x, fmaf(dy, c.y, dz * c.z)), f[r][3]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[r].fold(f[r]);
        acc[r].reduce(lgT);
    }
    if (s == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!act[r]) continue;
            int idx = a.perm[li.x + q + 32 * r];
            float* o = reinterpret_cast<float*>(a.out) + 3LL * idx;
            o[0] = acc[r].get(0, bx.g_adj);
            o[1] = acc[r].get(1, bx.g_adj);
            o[2] = acc[r].get(2, bx.g_adj);
            if (a.out_m) reinterpret_cast<float*>(a.out_m)[idx] = acc[r].get(3, -bx.g_adjm);
        }
    }
}

template <int TM, int ACC, bool WIDE>
__global__ void __launch_bounds__(256) p2p_adj_f32_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    float* tT = reinterpret_cast<float*>(smem);
    float* tQ = tT + 4 * (a.table_n + 1);
    if (TM != TA_EXACT) {
        const float4* g = reinterpret_cast<const float4*>(a.table);
        const float4* gq = g + (kMaxTableN + 1);
        float4* sT = reinterpret_cast<float4*>(tT);
        float4* sQ = reinterpret_cast<float4*>(tQ);
        for (int i = threadIdx.x; i <= a.table_n; i += blockDim.x) {
            if (TM == TA_LINEAR) {
                float4 u = g[i], v = gq[i];
                sT[i] = make_float4(u.x, u.y, v.x, v.y);
            } else {
                sT[i] = g[i];
                sQ[i] = gq[i];
            }
        }
        __syncthreads();
    }
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.ctrl + kCtrlTicketAdj, 1u);
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
            adj_item<TM, ACC, 2>(a, I, li, tT, tQ);
        else
            adj_item<TM, ACC, 1>(a, I, li, tT, tQ);
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
        if (lane == 0) it = (int)atomicAdd(a.ctrl + kCtrlTicketAdj, 1u);
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

static size_t adj_smem(int precision, int interp, int table_n)
{
    if (precision != PSR_FP32_TABLE) return 0;
    return (size_t)(table_n + 1) * (interp == PSR_LINEAR ? 16 : 32);
}

template <int TM, int ACC>
static int launch_adj_t(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    bool wide = a.max_leaf > 32;
    auto k = wide ? p2p_adj_f32_kernel<TM, ACC, true> : p2p_adj_f32_kernel<TM, ACC, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    k<<<a.blocks, a.warps_per_block * 32, smem, st>>>(a);
    return (int)cudaGetLastError();
}

int launch_adj_f32(const FwdArgs& a, int precision, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    long long nb = (a.n + 255) / 256;
    gather_cot_kernel<float, float4><<<(unsigned)nb, 256, 0, st>>>(
        reinterpret_cast<const float*>(a.cot), a.perm, reinterpret_cast<float4*>(a.cot_sorted), a.n);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return (int)e0;
    size_t smem = adj_smem(precision, a.interp, a.table_n);
    if (precision == PSR_FP32_EXACT)
        return a.accum == PSR_ACC_FP64 ? launch_adj_t<TA_EXACT, PSR_ACC_FP64>(a, smem, st)
                                       : launch_adj_t<TA_EXACT, PSR_ACC_KAHAN32>(a, smem, st);
    if (a.interp == PSR_LINEAR)
        return a.accum == PSR_ACC_FP64 ? launch_adj_t<TA_LINEAR, PSR_ACC_FP64>(a, smem, st)
                                       : launch_adj_t<TA_LINEAR, PSR_ACC_KAHAN32>(a, smem, st);
    return a.accum == PSR_ACC_FP64 ? launch_adj_t<TA_CUBIC, PSR_ACC_FP64>(a, smem, st)
                                   : launch_adj_t<TA_CUBIC, PSR_ACC_KAHAN32>(a, smem, st);
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

int adj_occupancy(int precision, int interp, int accum, int warps, int max_leaf, int table_n, int* out)
{
    bool wide = max_leaf > 32;
    size_t smem = adj_smem(precision, interp, table_n);
    const void* f;
    if (precision == PSR_FP64) {
        f = wide ? (const void*)p2p_adj_f64_kernel<true> : (const void*)p2p_adj_f64_kernel<false>;
    } else {
#define PSR_PICK(TM, ACC) (wide ? (const void*)p2p_adj_f32_kernel<TM, ACC, true> \
                                : (const void*)p2p_adj_f32_kernel<TM, ACC, false>)
        if (precision == PSR_FP32_EXACT)
            f = accum == PSR_ACC_FP64 ? PSR_PICK(TA_EXACT, PSR_ACC_FP64) : PSR_PICK(TA_EXACT, PSR_ACC_KAHAN32);
        else if (interp == PSR_LINEAR)
            f = accum == PSR_ACC_FP64 ? PSR_PICK(TA_LINEAR, PSR_ACC_FP64) : PSR_PICK(TA_LINEAR, PSR_ACC_KAHAN32);
        else
            f = accum == PSR_ACC_FP64 ? PSR_PICK(TA_CUBIC, PSR_ACC_FP64) : PSR_PICK(TA_CUBIC, PSR_ACC_KAHAN32);
#undef PSR_PICK
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
        }
    }
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, warps * 32, smem);
}

}  // namespace psr
