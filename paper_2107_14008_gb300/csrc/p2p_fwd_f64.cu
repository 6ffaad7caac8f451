// FP64 forward P2P kernel: the plain double-precision path (paper, Section 2
// pair force with Eq. tr evaluated by erfc/exp, Section 3.2 kernel layout),
// or, with a Taylor interpolation level, the paper's double-precision table
// path (Section 3.3: the Eq. int expansion about the nearest of N + 1 nodes,
// level T_[4] for double precision) with the table in shared memory and
// 1/r from an FP32 estimate refined by two Newton-Raphson steps in FP64.
// Same work decomposition as the FP32 kernels (warp per target leaf, S
// streams of T lanes, persistent ticket); coordinates are the wrapped FP64
// positions and each leaf pair adds its periodic image n L exactly as the
// definition d = x_j + n L - x_i reads.
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace psr {

// Taylor table in FP64: node k = 0..N, x_k = k h, h = x_c / N; six doubles
// per node, the Eq. int coefficients of eps^m (eps = x - x_k) times h^m, so
// that the expansion is a polynomial in f = x/h - k (zero above the level).
__global__ void table64_kernel(int N, int level, double x_c, double* __restrict__ t)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > N) return;
    const double h = x_c / N, x = k * h, x2 = x * x;
    const double E = -2.0 * 1.1283791670955126 * exp(-x2);  // -4 exp(-x^2) / sqrt(pi)
    double* c = t + 6 * (int64_t)k;
    c[0] = erfc(x) - 0.5 * x * E;
    c[1] = x2 * E * h;
    c[2] = -x * (x2 - 1.0) * E * h * h;
    c[3] = level >= 4 ? (2.0 / 3.0 * x2 * x2 - 5.0 / 3.0 * x2 + 1.0 / 3.0) * E * h * h * h : 0.0;
    c[4] = level >= 4 ? -x * (x2 * x2 / 3.0 - 1.5 * x2 + 1.0) * E * h * h * h * h : 0.0;
    c[5] = 0.0;
}

int launch_table64(int table_n, int interp, double x_c, void* d_out, void* stream)
{
    const int threads = 256, blocks = (table_n + 1 + threads - 1) / threads;
    table64_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(
        table_n, interp == PSR_TAYLOR4 ? 4 : 2, x_c, reinterpret_cast<double*>(d_out));
    return (int)cudaGetLastError();
}

// 1/sqrt(r2) for r2 > 0: an FP32 estimate (FP64 rsqrt where r2 leaves the
// FP32 normal range) refined by two Newton-Raphson steps for 1/sqrt,
// y <- y (3 - r2 y^2) / 2, each of which squares the relative error.
__device__ __forceinline__ double rsqrt_nr(double r2)
{
    const float f = (float)r2;
    double y = (f > 1e-36f && f < 1e36f) ? (double)rsqrtf(f) : rsqrt(r2);
    y = y * fma(-0.5 * r2, y * y, 1.5);
    y = y * fma(-0.5 * r2, y * y, 1.5);
    return y;
}

template <bool COUNT, int R, bool TAYLOR>
__device__ __forceinline__ void fwd64_item(const FwdArgs& a, int I, int4 li, const double* tab,
                                           unsigned long long& npairs, unsigned long long& nev)
{
    const int lane = threadIdx.x & 31;
    const double4* __restrict__ pd = reinterpret_cast<const double4*>(a.pd);
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    const int nI = li.y;
    const int lgT = (R == 2) ? 5 : stream_log2(nI);
    const int q = lane & ((1 << lgT) - 1);
    const int s = lane >> lgT;
    const int S = 32 >> lgT;
    const BoxDev& bx = a.boxes[li.z];
    const double L = bx.L, rc2 = bx.rc2, inv2rs = bx.inv_2rs;
    const double c2 = 1.1283791670955126;  // 2 / sqrt(pi)
    const double nmax = (double)a.table_n;
    const double uscale = nmax / bx.r_c;  // r -> x N / x_c (table units), in FP64

    double4 xi[R];
    bool act[R];
    double ax[R], ay[R], az[R], tx[R], ty[R], tz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = q + 32 * r;
        act[r] = t < nI;
        xi[r] = pd[li.x + (act[r] ? t : 0)];
        ax[r] = ay[r] = az[r] = 0.0;
        tx[r] = ty[r] = tz[r] = 0.0;
    }
    unsigned cnt = 0;
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
                    tx[r] = xi[r].x - nx * L;
                    ty[r] = xi[r].y - ny * L;
                    tz[r] = xi[r].z - nz * L;
                }
                j = lj.x;
                jend = lj.x + lj.y;
                found = true;
                break;
            }
            if (!found) break;
        }
        const double4 p = pd[j];
        ++j;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double dx = p.x - tx[r], dy = p.y - ty[r], dz = p.z - tz[r];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2 && r2 > 0.0) {
                double w;
                if (TAYLOR) {
                    const double ri = rsqrt_nr(r2);
                    const double u = r2 * ri * uscale;
                    const double kf = fmin(rint(u), nmax);
                    const double f = u - kf;
                    const double* c = tab + 6 * (int)kf;
                    const double T = fma(f, fma(f, fma(f, fma(f, c[4], c[3]), c[2]), c[1]), c[0]);
                    w = p.w * T * ri * ri * ri;
                } else {
                    double rr = sqrt(r2);
                    double x = rr * inv2rs;
                    double T = erfc(x) + c2 * x * exp(-x * x);
                    w = p.w * T / (r2 * rr);
                }
                ax[r] += w * dx;
                ay[r] += w * dy;
                az[r] += w * dz;
                if (COUNT) cnt += act[r];
            }
            if (COUNT) nev += act[r];
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        for (int off = 1 << lgT; off < 32; off <<= 1) {
            ax[r] += __shfl_xor_sync(kFull, ax[r], off);
            ay[r] += __shfl_xor_sync(kFull, ay[r], off);
            az[r] += __shfl_xor_sync(kFull, az[r], off);
        }
    if (COUNT) npairs += cnt;
    if (s == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!act[r]) continue;
            int idx = a.perm[li.x + q + 32 * r];
            double* out = reinterpret_cast<double*>(a.out) + 3LL * idx;
            out[0] = bx.G * ax[r];
            out[1] = bx.G * ay[r];
            out[2] = bx.G * az[r];
        }
    }
}

template <bool COUNT, bool WIDE, bool TAYLOR>
__global__ void __launch_bounds__(256) p2p_fwd_f64_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem64[];
    const double* tab = reinterpret_cast<const double*>(smem64);
    if (TAYLOR) {
        const double* g = reinterpret_cast<const double*>(a.table);
        for (int i = threadIdx.x; i < 6 * (a.table_n + 1); i += blockDim.x)
            reinterpret_cast<double*>(smem64)[i] = g[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
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
        if (li.y <= 0 || li.y > a.max_leaf || (long long)li.x + li.y > a.n || li.z < 0 ||
            li.z >= a.nbox) {
            if (lane == 0) set_error(a.ctrl, kErrParticleRange);
            continue;
        }
        if (WIDE && li.y > 32)
            fwd64_item<COUNT, 2, TAYLOR>(a, I, li, tab, npairs, nev);
        else
            fwd64_item<COUNT, 1, TAYLOR>(a, I, li, tab, npairs, nev);
    }
    if (COUNT) {
        for (int off = 16; off > 0; off >>= 1) {
            npairs += __shfl_xor_sync(kFull, npairs, off);
            nev += __shfl_xor_sync(kFull, nev, off);
        }
        if (lane == 0 && npairs)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlPairsLo), npairs);
        if (lane == 0 && nev)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlEvalLo), nev);
    }
    persistent_exit(a.ctrl + kCtrlTicketFwd, a.ctrl + kCtrlDoneFwd);
}

namespace {

bool taylor64(int interp) { return interp == PSR_TAYLOR2 || interp == PSR_TAYLOR4; }

template <bool COUNT, bool WIDE, bool TAYLOR>
int launch64(const FwdArgs& a, size_t smem, cudaStream_t st)
{
    auto k = p2p_fwd_f64_kernel<COUNT, WIDE, TAYLOR>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    k<<<a.blocks, a.warps_per_block * 32, smem, st>>>(a);
    return (int)cudaGetLastError();
}

template <bool TAYLOR>
const void* ptr64(bool wide)
{
    return wide ? (const void*)p2p_fwd_f64_kernel<false, true, TAYLOR>
                : (const void*)p2p_fwd_f64_kernel<false, false, TAYLOR>;
}

}  // namespace

size_t fwd_f64_smem(int interp, int table_n)
{
    return taylor64(interp) ? (size_t)(table_n + 1) * 48 : 0;
}

int launch_fwd_f64(const FwdArgs& a, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const bool wide = a.max_leaf > 32, tay = taylor64(a.interp);
    const size_t smem = fwd_f64_smem(a.interp, a.table_n);
    if (tay) {
        if (a.count_pairs) return wide ? launch64<true, true, true>(a, smem, st) : launch64<true, false, true>(a, smem, st);
        return wide ? launch64<false, true, true>(a, smem, st) : launch64<false, false, true>(a, smem, st);
    }
    if (a.count_pairs) return wide ? launch64<true, true, false>(a, 0, st) : launch64<true, false, false>(a, 0, st);
    return wide ? launch64<false, true, false>(a, 0, st) : launch64<false, false, false>(a, 0, st);
}

int fwd_f64_occupancy(int warps, int max_leaf, int interp, int table_n, int* out)
{
    const bool wide = max_leaf > 32, tay = taylor64(interp);
    const void* f = tay ? ptr64<true>(wide) : ptr64<false>(wide);
    const size_t smem = fwd_f64_smem(interp, table_n);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, warps * 32, smem);
}

}  // namespace psr
