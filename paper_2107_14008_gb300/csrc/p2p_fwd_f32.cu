// FP32 forward P2P: variant dispatch, shared-memory sizing, and the
// interpolation-table builder (paper, Section 3.3).
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace psr {

template <bool PK>
int launch_fwd_f32_variant(const FwdArgs& a, int precision, size_t smem, cudaStream_t st);
template <bool PK>
const void* fwd_f32_kernel_ptr(int precision, int interp, int accum, int max_leaf);

// ------------------------------------------------------------------ table --
// Entries k = 0..N-1 describe [x_k, x_{k+1}], x_k = k x_c / N, as functions of
// f = (x - x_k)/h - 1/2 in [-1/2, 1/2]; entry N is zero (beyond the cutoff).
// Linear entries are (M_k, D_k, A_k, 0): the chord is M_k + f D_k, or, with
// t = u - 1/2 = k + f (u = x/h), A_k + t D_k where A_k = M_k - k D_k, which
// the forward kernel evaluates in one FMA without forming f.
// Second half (offset N+1): the same for Q(x) = exp(-x^2), used by the adjoint.
// Taylor modes (Eq. int of Section 3.3): node k = 0..N, two float4 per node,
// the level-2 or level-4 expansion about x_k in powers of f = (x - x_k)/h:
//   T_k + x_k^2 E_k eps - x_k (x_k^2 - 1) E_k eps^2
//       + (2/3 x_k^4 - 5/3 x_k^2 + 1/3) E_k eps^3 - x_k (x_k^4/3 - 3/2 x_k^2 + 1) E_k eps^4,
// eps = f h, E_k = -4 exp(-x_k^2) / sqrt(pi), T_k = erfc(x_k) - x_k E_k / 2.
__global__ void table_kernel(int N, int interp, double x_c, float4* __restrict__ tT,
                             float4* __restrict__ tQ)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > N) return;
    if (interp == PSR_TAYLOR2 || interp == PSR_TAYLOR4) {
        const double h = x_c / N, x = k * h, x2 = x * x;
        const double E = -2.0 * 1.1283791670955126 * exp(-x2);
        const double c0 = erfc(x) - 0.5 * x * E;
        const double c1 = x2 * E * h;
        const double c2 = -x * (x2 - 1.0) * E * h * h;
        const bool four = interp == PSR_TAYLOR4;
        const double c3 = four ? (2.0 / 3.0 * x2 * x2 - 5.0 / 3.0 * x2 + 1.0 / 3.0) * E * h * h * h : 0.0;
        const double c4 = four ? -x * (x2 * x2 / 3.0 - 1.5 * x2 + 1.0) * E * h * h * h * h : 0.0;
        tT[2 * k] = make_float4((float)c0, (float)c1, (float)c2, (float)c3);
        tT[2 * k + 1] = make_float4((float)c4, 0.f, 0.f, 0.f);
        return;
    }
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
        if (interp == PSR_LINEAR) {
            const double m = 0.5 * (f0 + f1), d = f1 - f0;
            return make_float4((float)m, (float)d, (float)(m - k * d), 0.f);
        }
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

// bytes of one table entry in shared memory (and in global for Taylor)
size_t table_entry_bytes(int interp)
{
    return interp == PSR_LINEAR ? 8 : interp == PSR_CUBIC ? 16 : 32;
}

// ---------------------------------------------------------------- launch --
constexpr int kMetaPerWarpHost = 34;  // 32 entry records + 2 target-box slots

size_t fwd_f32_smem(int precision, int interp, int table_n, int warps, int cap)
{
    size_t tab = precision != PSR_FP32_TABLE ? 0 : (size_t)(table_n + 1) * table_entry_bytes(interp);
    return ((tab + 15) & ~(size_t)15) + (size_t)warps * (cap + kMetaPerWarpHost) * 16;
}

int launch_fwd_f32(const FwdArgs& a, int precision, void* stream)
{
    size_t smem = fwd_f32_smem(precision, a.interp, a.table_n, a.warps_per_block, a.stage_cap);
    cudaStream_t st = (cudaStream_t)stream;
    return a.variant == PSR_KERNEL_PACKED ? launch_fwd_f32_variant<true>(a, precision, smem, st)
                                          : launch_fwd_f32_variant<false>(a, precision, smem, st);
}

int fwd_f32_occupancy(int precision, int interp, int accum, int warps, int max_leaf, int table_n,
                      int cap, int variant, int* out)
{
    size_t smem = fwd_f32_smem(precision, interp, table_n, warps, cap);
    const void* f = variant == PSR_KERNEL_PACKED
                        ? fwd_f32_kernel_ptr<true>(precision, interp, accum, max_leaf)
                        : fwd_f32_kernel_ptr<false>(precision, interp, accum, max_leaf);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, warps * 32, smem);
}

}  // namespace psr
