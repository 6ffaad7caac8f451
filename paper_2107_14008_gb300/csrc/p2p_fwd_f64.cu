// FP64 forward P2P kernel: the plain double-precision path (paper, Section 2
// pair force with Eq. tr evaluated by erfc/exp, Section 3.2 kernel layout).
// Same work decomposition as the FP32 kernels (warp per target leaf, S
// streams of T lanes, persistent ticket); coordinates are the wrapped FP64
// positions and each leaf pair adds its periodic image n L exactly as the
// definition d = x_j + n L - x_i reads.
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace psr {

template <bool COUNT, int R>
__device__ __forceinline__ void fwd64_item(const FwdArgs& a, int I, int4 li,
                                           unsigned long long& npairs)
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
                double rr = sqrt(r2);
                double x = rr * inv2rs;
                double T = erfc(x) + c2 * x * exp(-x * x);
                double w = p.w * T / (r2 * rr);
                ax[r] += w * dx;
                ay[r] += w * dy;
                az[r] += w * dz;
                if (COUNT) cnt += act[r];
            }
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

template <bool COUNT, bool WIDE>
__global__ void __launch_bounds__(256) p2p_fwd_f64_kernel(const FwdArgs a)
{
    const int lane = threadIdx.x & 31;
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    unsigned long long npairs = 0;
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
            fwd64_item<COUNT, 2>(a, I, li, npairs);
        else
            fwd64_item<COUNT, 1>(a, I, li, npairs);
    }
    if (COUNT) {
        for (int off = 16; off > 0; off >>= 1) npairs += __shfl_xor_sync(kFull, npairs, off);
        if (lane == 0 && npairs)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlPairsLo), npairs);
    }
    persistent_exit(a.ctrl + kCtrlTicketFwd, a.ctrl + kCtrlDoneFwd);
}

int launch_fwd_f64(const FwdArgs& a, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    bool wide = a.max_leaf > 32;
    if (a.count_pairs) {
        if (wide) p2p_fwd_f64_kernel<true, true><<<a.blocks, a.warps_per_block * 32, 0, st>>>(a);
        else p2p_fwd_f64_kernel<true, false><<<a.blocks, a.warps_per_block * 32, 0, st>>>(a);
    } else {
        if (wide) p2p_fwd_f64_kernel<false, true><<<a.blocks, a.warps_per_block * 32, 0, st>>>(a);
        else p2p_fwd_f64_kernel<false, false><<<a.blocks, a.warps_per_block * 32, 0, st>>>(a);
    }
    return (int)cudaGetLastError();
}

int fwd_f64_occupancy(int warps, int max_leaf, int* out)
{
    const void* f = max_leaf > 32 ? (const void*)p2p_fwd_f64_kernel<false, true>
                                  : (const void*)p2p_fwd_f64_kernel<false, false>;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, warps * 32, 0);
}

}  // namespace psr
