// FP32 forward P2P kernels (paper, Section 3.2, Algorithms 1 and 2, redesigned
// for sm_103a) and the interpolation-table builder (Section 3.3).
//
// Work decomposition.  The paper gives one thread block to each target leaf
// and one thread to each target particle, with the j-leaf staged in shared
// memory.  Leaves here hold 1-64 particles (mean ~9 on clustered sets), so one
// WARP takes one target leaf: each lane holds R = 1 or 2 target particles, the
// n_I targets occupy T = ceil(n_I / R) lanes, and the warp's 32 lanes form
// S = 32 / T streams.  The row's source leaves are staged chunk by chunk into a
// per-warp shared-memory buffer, already shifted into the target leaf's frame,
// and stream s takes staged particles s, s+S, ... (one broadcast shared-memory
// load serves the T lanes of a stream).  The S partial sums of each target
// are combined through shared memory at the end.  Warps take target leaves
// from an atomic ticket in largest-work-first order (persistent grid, no
// inter-block waits).
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

// Per-warp shared-memory staging of a row's source particles.  Up to 32 row
// entries are examined at once (lane k reads entry e0 + k); a warp prefix sum
// of their leaf sizes gives each leaf's slot in the buffer, and as many whole
// leaves as fit in kStageCap slots are taken.  Each staged particle is written
// already shifted into the target leaf's frame (its leaf offset added), so the
// compute loop that follows is uniform over the chunk.
constexpr int kStageCap = 256;   // particles per warp buffer (4 KB)
constexpr int kMetaPerWarp = 32; // entries per chunk

// Stages one chunk starting at entry e0; returns the number of entries taken
// and sets nst to the number of staged particles.
__device__ __forceinline__ int stage_chunk(const FwdArgs& a, long long e0, long long re,
                                           int4 ci, float unit, float4* __restrict__ stage,
                                           float4* __restrict__ meta, int& nst)
{
    const int lane = threadIdx.x & 31;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    const int4* __restrict__ lcen = reinterpret_cast<const int4*>(a.lcen);
    const long long e = e0 + lane;
    int cnt = 0, first = 0;
    float ox = 0.f, oy = 0.f, oz = 0.f;
    if (e < re) {
        unsigned ent = a.pairs[e];
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
            ox = oy = oz = 1e30f;
        }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned fit = __ballot_sync(kFull, e < re && incl <= kStageCap);
    const int ntake = __popc(fit);  // >= 1: one leaf always fits
    nst = __shfl_sync(kFull, incl, ntake - 1);
    const int excl = incl - cnt;
    if (lane < ntake) meta[lane] = make_float4(__int_as_float(first - excl), ox, oy, oz);
    __syncwarp();
    // slot p belongs to the entry k with excl_k <= p < excl_{k+1}: count the
    // entry starts at or before p with a position bitmask per 32-slot round
    int C = 0;
    for (int p0 = 0; p0 < nst; p0 += 32) {
        const int rel = excl - p0;
        const unsigned bit = (lane < ntake && rel >= 0 && rel < 32) ? (1u << rel) : 0u;
        const unsigned M = __reduce_or_sync(kFull, bit);
        const int k = C + __popc(M & ((2u << lane) - 1u)) - 1;
        C += __popc(M);
        const int p = p0 + lane;
        if (p < nst) {
            const float4 m = meta[k];
            const float4 v = __ldg(pf + (__float_as_int(m.x) + p));
            stage[p] = make_float4(v.x + m.y, v.y + m.z, v.z + m.w, v.w);
        }
    }
    __syncwarp();
    return ntake;
}

// One target leaf on one warp.  R = targets per lane; T = ceil(n_I / R) lanes
// per stream, S = 32 / T streams; stream s takes staged particles s, s+S, ...
template <int TM, int ACC, bool COUNT, int R>
__device__ __forceinline__ void fwd_item(const FwdArgs& a, int I, int4 li, const float* tab,
                                         float4* __restrict__ stage, float4* __restrict__ meta,
                                         unsigned long long& npairs)
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
    const float unit = bx.unit;
    const float x_c = bx.x_c;
    const float nmax = (float)a.table_n;
    const float inv_h = (float)a.table_n / x_c;
    const int4 ci = lcen[I];

    float4 xi[R];
    bool act[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = q + T * r;
        act[r] = on && t < nI;
        xi[r] = pf[li.x + (act[r] ? t : 0)];
    }
    Acc3<ACC> acc[R];
    float fx[R], fy[R], fz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) fx[r] = fy[r] = fz[r] = 0.0f;
    unsigned cnt = 0;
    const long long re = a.rowptr[I + 1];
    long long e0 = a.rowptr[I];
    while (e0 < re) {
        int nst;
        e0 += stage_chunk(a, e0, re, ci, unit, stage, meta, nst);
        if (on) {
#pragma unroll 2
            for (int k = s; k < nst; k += S) {
                const float4 p = stage[k];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float dx = p.x - xi[r].x, dy = p.y - xi[r].y, dz = p.z - xi[r].z;
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kEps2)));
                    float rinv = rsqrtf(r2);
                    float x = r2 * rinv;
                    float T_ = eval_T<TM>(x, tab, inv_h, nmax, x_c);
                    float w = p.w * T_ * rinv * rinv * rinv;
                    fx[r] = fmaf(w, dx, fx[r]);
                    fy[r] = fmaf(w, dy, fy[r]);
                    fz[r] = fmaf(w, dz, fz[r]);
                    if (COUNT)
                        cnt += (act[r] && x < x_c && (dx != 0.0f || dy != 0.0f || dz != 0.0f));
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r].fold(fx[r], fy[r], fz[r]);
        }
        __syncwarp();
    }
    if (COUNT) npairs += cnt;
    // combine the S stream partials of each target through shared memory
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float ox, oy, oz;
        acc[r].result(1.0f, ox, oy, oz);  // partial sum of this lane, in coordinate units
        if (ACC == PSR_ACC_FP64) {
            double* red = reinterpret_cast<double*>(stage);
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
                out[0] = (float)(sx * (double)bx.g_acc);
                out[1] = (float)(sy * (double)bx.g_acc);
                out[2] = (float)(sz * (double)bx.g_acc);
            }
        } else {
            float* red = reinterpret_cast<float*>(stage);
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
                    const float* o = red + 6 * (lane + t * T);
                    two_sum(sx, o[0], u, v); sx = u; cx += o[1] + v;
                    two_sum(sy, o[2], u, v); sy = u; cy += o[3] + v;
                    two_sum(sz, o[4], u, v); sz = u; cz += o[5] + v;
                }
                int idx = a.perm[li.x + q + T * r];
                float* out = reinterpret_cast<float*>(a.out) + 3LL * idx;
                out[0] = (sx + cx) * bx.g_acc;
                out[1] = (sy + cy) * bx.g_acc;
                out[2] = (sz + cz) * bx.g_acc;
            }
        }
        (void)ox; (void)oy; (void)oz;
        __syncwarp();
    }
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

template <int TM, int ACC, bool COUNT>
__global__ void __launch_bounds__(256) p2p_fwd_f32_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const size_t tab_bytes = TM == TM_EXACT ? 0
                           : (size_t)(a.table_n + 1) * (TM == TM_LINEAR ? 8 : 16);
    float4* stage = reinterpret_cast<float4*>(smem + ((tab_bytes + 15) & ~(size_t)15)) +
                    (size_t)warp * (kStageCap + kMetaPerWarp);
    float4* meta = stage + kStageCap;
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
        if (li.y <= 0 || li.y > a.max_leaf || li.y > 64 || (long long)li.x + li.y > a.n ||
            li.z < 0 || li.z >= a.nbox) {
            if (lane == 0) set_error(a.ctrl, kErrParticleRange);
            continue;
        }
        if (prefer_two_per_lane(li.y))
            fwd_item<TM, ACC, COUNT, 2>(a, I, li, reinterpret_cast<const float*>(smem), stage,
                                        meta, npairs);
        else
            fwd_item<TM, ACC, COUNT, 1>(a, I, li, reinterpret_cast<const float*>(smem), stage,
                                        meta, npairs);
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
template <int TM, int ACC, bool COUNT>
static int launch_t(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    auto k = p2p_fwd_f32_kernel<TM, ACC, COUNT>;
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
    return a.count_pairs ? launch_t<TM, ACC, true>(a, smem, st) : launch_t<TM, ACC, false>(a, smem, st);
}

static size_t fwd_smem(int precision, int interp, int table_n, int warps)
{
    size_t tab = precision != PSR_FP32_TABLE ? 0
               : (size_t)(table_n + 1) * (interp == PSR_LINEAR ? 8 : 16);
    return ((tab + 15) & ~(size_t)15) + (size_t)warps * (kStageCap + kMetaPerWarp) * 16;
}

int launch_fwd_f32(const FwdArgs& a, int precision, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    size_t smem = fwd_smem(precision, a.interp, a.table_n, a.warps_per_block);
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
    size_t smem = fwd_smem(precision, interp, table_n, warps);
    const void* f;
    (void)max_leaf;
#define PSR_PICK(TM, ACC) ((const void*)p2p_fwd_f32_kernel<TM, ACC, false>)
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
