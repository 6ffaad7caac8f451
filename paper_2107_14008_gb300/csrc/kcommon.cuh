// Device helpers shared by the P2P kernels of libpsr.
#pragma once

#include <cuda_runtime.h>

#include "psr_internal.h"

namespace psr {

constexpr unsigned kFull = 0xffffffffu;
// rint by the 1.5 * 2^23 trick: for |t| < 2^22, (t + M) - M == rint(t) and the
// low mantissa bits of (t + M) hold rint(t) + 2^22.
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;
// The FP32 kernels work in coordinates scaled by 1 / (2 r_s), so the pair
// distance is the paper's x = r / (2 r_s) directly.  A tiny constant is added
// to r^2 so that the self pair (d = 0 exactly) gives a finite 1/r and hence a
// zero term; it moves any pair farther than 1e-7 x-units by < 1e-6 relative.
constexpr float kEps2 = 1e-20f;
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;
constexpr float kInf = __builtin_huge_valf();

__device__ __forceinline__ void set_error(unsigned* ctrl, unsigned bit)
{
    atomicOr(ctrl + kCtrlError, bit);
}

// Shift code (nx+1)*9 + (ny+1)*3 + (nz+1) -> n components.
__device__ __forceinline__ void decode_shift(unsigned code, int& nx, int& ny, int& nz)
{
    nx = (int)(code / 9u) - 1;
    ny = (int)((code / 3u) % 3u) - 1;
    nz = (int)(code % 3u) - 1;
}

// Two-sum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Grid-wide end of a persistent launch: the last block to finish resets the
// work ticket and the done counter, so the next launch (or a graph replay)
// starts from zero without a memset.
__device__ __forceinline__ void persistent_exit(unsigned* ticket, unsigned* done)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned d = atomicAdd(done, 1u);
        if (d == gridDim.x - 1) {
            atomicExch(ticket, 0u);
            atomicExch(done, 0u);
            __threadfence();
        }
    }
}

// PTX rsqrt.approx.ftz.f32: one SFU instruction, max relative error 2^-22.9.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 32-bit shared-window address of a shared-memory pointer.
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Loads from read-only shared data (the interpolation table): no ordering.
__device__ __forceinline__ float lds_f1(unsigned a)
{
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds_f2(unsigned a)
{
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 lds_f4(unsigned a)
{
    float4 v;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
// lanes per stream T (power of two >= n, at least 4), as log2
__device__ __forceinline__ int stream_log2(int n)
{
    return n <= 4 ? 2 : n <= 8 ? 3 : n <= 16 ? 4 : 5;
}

}  // namespace psr
