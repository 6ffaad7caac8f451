// FP32 forward P2P kernels (paper, Section 3.2, Algorithms 1 and 2, redesigned
// for sm_103a) and the interpolation-table builder (Section 3.3).
//
// Work decomposition.  The paper gives one thread block to each target leaf
// and one thread to each target particle.  Leaves hold 8-32 particles, so
// here one WARP takes one target leaf: its 32 lanes form S = 32 / T streams of
// T lanes (T = the power of two >= leaf size, >= 4); lane q of every stream
// holds target particle q, and stream s walks source leaves s, s+S, ... of the
// target's row, one source particle per iteration (a broadcast load shared by
// the T lanes of the stream).  At the end the S partial sums of each target
// are combined with warp shuffles.  Warps take target leaves from an atomic
// ticket in largest-work-first order (persistent grid, no inter-block waits).
//
// Precision.  Pair arithmetic is FP32 in leaf-local coordinates scaled by
// 1/(2 r_s); the offset between two leaf centres (with the periodic image) is
// an exact integer in units of L/2^22, converted to FP32 once per leaf pair.
// Per-source FP32 partial sums are folded every `fold_every` source particles
// into FP64 (PSR_ACC_FP64) or compensated FP32 (PSR_ACC_KAHAN32) accumulators.
//
// T(x).  Exact: erfcf + expf.  Table: T on [0, x_c] with N intervals, held in
// shared memory: linear (midpoint value, chord difference) or cubic Hermite
// (monomial coefficients about the midpoint); index N is a zero sentinel, so
// the cutoff (x >= x_c) costs no extra instruction.
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace psr {

enum { TM_EXACT = 0, TM_LINEAR = 1, TM_CUBIC = 2 };

template <int TM>
__device__ __forceinline__ float eval_T(float x, const void* tab, float inv_h, float nmax,
                                        float x_c)
{
    if (TM == TM_EXACT) {
        float T = erfcf(x) + kTwoOverSqrtPi * x * expf(-x * x);
        return x < x_c ? T : 0.0f;
    } else {
        float t = fminf(fmaf(x, inv_h, -0.5f), nmax);
        float fk = t + kMagic;
        int k = __float_as_int(fk) - kMagicBits;
        float f = t - (fk - kMagic);
        if (TM == TM_LINEAR) {
            float2 c = reinterpret_cast<const float2*>(tab)[k];
            return fmaf(f, c.y, c.x);
        } else {
            float4 c = reinterpret_cast<const float4*>(tab)[k];
            return fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
        }
    }
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
    // combine the partials of lanes lane ^ off for off = T, 2T, ..., 16
    __device__ __forceinline__ void reduce(int lgT)
    {
        for (int off = 1 << lgT; off < 32; off <<= 1) {
            if (ACC == PSR_ACC_FP64) {
                x += __shfl_xor_sync(kFull, x, off);
                y += __shfl_xor_sync(kFull, y, off);
                z += __shfl_xor_sync(kFull, z, off);
            } else {
                float s, e;
                float osx = __shfl_xor_sync(kFull, sx, off), ocx = __shfl_xor_sync(kFull, cx, off);
                float osy = __shfl_xor_sync(kFull, sy, off), ocy = __shfl_xor_sync(kFull, cy, off);
                float osz = __shfl_xor_sync(kFull, sz, off), ocz = __shfl_xor_sync(kFull, cz, off);
                two_sum(sx, osx, s, e); sx = s; cx += ocx + e;
                two_sum(sy, osy, s, e); sy = s; cy += ocy + e;
                two_sum(sz, osz, s, e); sz = s; cz += ocz + e;
            }
        }
    }
    __device__ __forceinline__ void result(float g, float& ox, float& oy, float& oz) const
    {
        if (ACC == PSR_ACC_FP64) {
            ox = (float)(x * (double)g);
            oy = (float)(y * (double)g);
            oz = (float)(z * (double)g);
        } else {
            ox = (sx + cx) * g;
            oy = (sy + cy) * g;
            oz = (sz + cz) * g;
        }
    }
};

// One target leaf on one warp; R = targets per lane (2 when leaves exceed 32).
template <int TM, int ACC, bool COUNT, int R>
__device__ __forceinline__ void fwd_item(const FwdArgs& a, int I, int4 li, const float* tab,
                                         unsigned long long& npairs)
{
    const int lane = threadIdx.x & 31;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    const int4* __restrict__ lcen = reinterpret_cast<const int4*>(a.lcen);
    const int nI = li.y;
    const int lgT = (R == 2) ? 5 : stream_log2(nI);
    const int q = lane & ((1 << lgT) - 1);
    const int s = lane >> lgT;
    const int S = 32 >> lgT;
    const BoxDev& bx = a.boxes[li.z];
    const float unit = bx.unit;
    const float x_c = bx.x_c;
    const float nmax = (float)a.table_n;
    const float inv_h = (float)a.table_n / x_c;
    const int4 ci = lcen[I];

    float4 xi[R];
    bool act[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = q + 32 * r;
        act[r] = t < nI;
        xi[r] = pf[li.x + (act[r] ? t : 0)];
    }
    Acc3<ACC> acc[R];
    float fx[R], fy[R], fz[R], tx[R], ty[R], tz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        fx[r] = fy[r] = fz[r] = 0.0f;
        tx[r] = ty[r] = tz[r] = 0.0f;
    }
    unsigned cnt = 0;
    int since = 0;
    const long long re = a.rowptr[I + 1];
    long long e = a.rowptr[I] + s;
    int j = 0, jend = 0;
    for (;;) {
        if (j >= jend) {
            // next source leaf of this stream (divergent, once per leaf)
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
                    for (int r = 0; r < R; ++r) acc[r].fold(fx[r], fy[r], fz[r]);
                    since = 0;
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    tx[r] = xi[r].x - ox;
                    ty[r] = xi[r].y - oy;
                    tz[r] = xi[r].z - oz;
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
        ++j;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float dx = p.x - tx[r], dy = p.y - ty[r], dz = p.z - tz[r];
            float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kEps2)));
            float rinv = rsqrtf(r2);
            float x = r2 * rinv;
            float T = eval_T<TM>(x, tab, inv_h, nmax, x_c);
            float w = p.w * T * rinv * rinv * rinv;
            fx[r] = fmaf(w, dx, fx[r]);
            fy[r] = fmaf(w, dy, fy[r]);
            fz[r] = fmaf(w, dz, fz[r]);
            if (COUNT) cnt += (act[r] && x < x_c && (dx != 0.0f || dy != 0.0f || dz != 0.0f));
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[r].fold(fx[r], fy[r], fz[r]);
        acc[r].reduce(lgT);
    }
    if (COUNT) npairs += cnt;
    if (s == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!act[r]) continue;
            float ox, oy, oz;
            acc[r].result(bx.g_acc, ox, oy, oz);
            int idx = a.perm[li.x + q + 32 * r];
            float* out = reinterpret_cast<float*>(a.out) + 3LL * idx;
            out[0] = ox;
            out[1] = oy;
            out[2] = oz;
        }
    }
}

template <int TM, int ACC, bool COUNT, bool WIDE>
__global__ void __launch_bounds__(256) p2p_fwd_f32_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    if (TM != TM_EXACT) {
        const float4* g = reinterpret_cast<const float4*>(a.table);
        if (TM == TM_LINEAR) {
            float2* t = reinterpret_cast<float2*>(smem);
            for (int i = threadIdx.x; i <= a.table_n; i += blockDim.x) {
                float4 v = g[i];
                t[i] = make_float2(v.x, v.y);
            }
        } else {
            float4* t = reinterpret_cast<float4*>(smem);
            for (int i = threadIdx.x; i <= a.table_n; i += blockDim.x) t[i] = g[i];
        }
        __syncthreads();
    }
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    unsigned long long npairs = 0;
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.ctrl + kCtrlTicketFwd, 1u);
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
            fwd_item<TM, ACC, COUNT, 2>(a, I, li, reinterpret_cast<const float*>(smem), npairs);
        else
            fwd_item<TM, ACC, COUNT, 1>(a, I, li, reinterpret_cast<const float*>(smem), npairs);
    }
    if (COUNT) {
        for (int off = 16; off > 0; off >>= 1) npairs += __shfl_xor_sync(kFull, npairs, off);
        if (lane == 0 && npairs)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlPairsLo), npairs);
    }
    persistent_exit(a.ctrl + kCtrlTicketFwd, a.ctrl + kCtrlDoneFwd);
}

// ------------------------------------------------------------------ table --
// Entries k = 0..N-1 describe [x_k, x_{k+1}], x_k = k x_c / N, as functions of
// f = (x - x_k)/h - 1/2 in [-1/2, 1/2]; entry N is zero (beyond the cutoff).
// Second half (offset N+1): the same for Q(x) = exp(-x^2), used by the adjoint.
__global__ void table_kernel(int N, int interp, double x_c, float4* __restrict__ tT,
                             float4* __restrict__ tQ)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > N) return;
    if (k == N) {
        tT[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tQ) tQ[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const double h = x_c / N;
    const double c2 = 1.1283791670955126;  // 2 / sqrt(pi)
    double x0 = k * h, x1 = (k + 1) * h;
    double q0 = exp(-x0 * x0), q1 = exp(-x1 * x1);
    double T0 = erfc(x0) + c2 * x0 * q0, T1 = erfc(x1) + c2 * x1 * q1;
    // T' = x^2 E(x) = -(4/sqrt(pi)) x^2 exp(-x^2); Q' = -2 x exp(-x^2)
    double D0 = -2.0 * c2 * x0 * x0 * q0, D1 = -2.0 * c2 * x1 * x1 * q1;
    double P0 = -2.0 * x0 * q0, P1 = -2.0 * x1 * q1;
    auto make = [&](double f0, double f1, double d0, double d1) {
        if (interp == PSR_LINEAR) return make_float4((float)(0.5 * (f0 + f1)), (float)(f1 - f0), 0.f, 0.f);
        // Hermite cubic in s = f + 1/2: a0 + a1 s + a2 s^2 + a3 s^3
        double a0 = f0, a1 = h * d0;
        double a2 = -3.0 * f0 - 2.0 * h * d0 + 3.0 * f1 - h * d1;
        double a3 = 2.0 * f0 + h * d0 - 2.0 * f1 + h * d1;
        return make_float4((float)(a0 + 0.5 * a1 + 0.25 * a2 + 0.125 * a3),
                           (float)(a1 + a2 + 0.75 * a3), (float)(a2 + 1.5 * a3), (float)a3);
    };
    tT[k] = make(T0, T1, D0, D1);
    if (tQ) tQ[k] = make(q0, q1, P0, P1);
}

int launch_table(int table_n, int interp, double x_c, void* d_out, void* d_q_out, void* stream)
{
    int threads = 256, blocks = (table_n + 1 + threads - 1) / threads;
    table_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(
        table_n, interp, x_c, reinterpret_cast<float4*>(d_out), reinterpret_cast<float4*>(d_q_out));
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- launch --
template <int TM, int ACC, bool COUNT, bool WIDE>
static int launch_t(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    auto k = p2p_fwd_f32_kernel<TM, ACC, COUNT, WIDE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    k<<<a.blocks, a.warps_per_block * 32, smem, st>>>(a);
    return (int)cudaGetLastError();
}

template <int TM, int ACC>
static int launch_c(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    bool wide = a.max_leaf > 32;
    if (a.count_pairs)
        return wide ? launch_t<TM, ACC, true, true>(a, smem, st) : launch_t<TM, ACC, true, false>(a, smem, st);
    return wide ? launch_t<TM, ACC, false, true>(a, smem, st) : launch_t<TM, ACC, false, false>(a, smem, st);
}

static size_t fwd_smem(int precision, int interp, int table_n)
{
    if (precision != PSR_FP32_TABLE) return 0;
    return (size_t)(table_n + 1) * (interp == PSR_LINEAR ? 8 : 16);
}

int launch_fwd_f32(const FwdArgs& a, int precision, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    size_t smem = fwd_smem(precision, a.interp, a.table_n);
    if (precision == PSR_FP32_EXACT)
        return a.accum == PSR_ACC_FP64 ? launch_c<TM_EXACT, PSR_ACC_FP64>(a, smem, st)
                                       : launch_c<TM_EXACT, PSR_ACC_KAHAN32>(a, smem, st);
    if (a.interp == PSR_LINEAR)
        return a.accum == PSR_ACC_FP64 ? launch_c<TM_LINEAR, PSR_ACC_FP64>(a, smem, st)
                                       : launch_c<TM_LINEAR, PSR_ACC_KAHAN32>(a, smem, st);
    return a.accum == PSR_ACC_FP64 ? launch_c<TM_CUBIC, PSR_ACC_FP64>(a, smem, st)
                                   : launch_c<TM_CUBIC, PSR_ACC_KAHAN32>(a, smem, st);
}

int fwd_f32_occupancy(int precision, int interp, int accum, int warps, int max_leaf, int table_n,
                      int* out)
{
    size_t smem = fwd_smem(precision, interp, table_n);
    const void* f;
    bool wide = max_leaf > 32;
#define PSR_PICK(TM, ACC) (wide ? (const void*)p2p_fwd_f32_kernel<TM, ACC, false, true> \
                                : (const void*)p2p_fwd_f32_kernel<TM, ACC, false, false>)
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
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, warps * 32, smem);
}

}  // namespace psr
