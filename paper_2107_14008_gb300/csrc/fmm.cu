// Truncated multipole operators of the PM-FMM short range (paper, Section 2):
// P2M, M2L with the truncated prefactors f_(n), L2P.
//
// Kernel psi(r) = erfc(r / 2 r_s) / r (the short-range potential per unit
// mass); f_(k) = (1/r d/dr)^k psi, evaluated from the paper's closed form
//   (-1)^k r_s^(2k+1) f_(k) = (2k-1)!! / 2^(2k+1) erfc(x) / x^(2k+1)
//                            + sum_{q=1..k} 2^(-q-k) (2k-1)!! / (2k-2q+1)!! exp(-x^2) / (sqrt(pi) x^(2q)),
// x = r / 2 r_s.  psi depends on s = r^2/2 only and d/ds = (1/r) d/dr, so
//   D_n(R) = d^n psi = sum_{j <= n/2} prod_a n_a! / (2^j_a j_a! (n_a - 2 j_a)!) R^(n-2j) f_(|n|-|j|).
// Expansions (|n| <= p):
//   P2M  M_m = sum_j m_j (z_A - x_j)^m / m!
//   M2L  L_n = sum_{|m| <= p-|n|} M_m D_{n+m}(z_B - z_A)
//   L2P  a_c = G sum_{|k| <= p-1} L_{k+e_c} (x - z_B)^k / k!
// The library stores scaled coefficients so that FP32 holds every order:
// Mh_m = M_m / r_s^|m| and Lh_n = L_n r_s^(|n|+1), then
//   Lh_n = sum Mh_m Dh_{n+m},  Dh_n = r_s^(|n|+1) D_n (a function of R / r_s),
//   a_c = (G / r_s^2) sum Lh_{k+e_c} (u / r_s)^k / k!.
// Coefficient order: graded by |n|, then n1 descending, then n2 descending:
//   index(n) = K(K+1)(K+2)/6 + (K-n1)(K-n1+1)/2 + (K-n1-n2),  K = |n|.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <type_traits>

#include "kcommon.cuh"
#include "psr_internal.h"

namespace psr {
void set_last_error(const std::string& msg);
}

using namespace psr;

namespace {

constexpr int kMaxOrder = 6;  // p

__host__ __device__ constexpr int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Position of n = (a, b, c) in the graded order.
__host__ __device__ constexpr int cidx(int a, int b, int c)
{
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

__host__ __device__ constexpr int ifact(int n) { return n <= 1 ? 1 : n * ifact(n - 1); }

// (2t+1)!! for t >= -1, with (-1)!! = 1.
__host__ __device__ constexpr int odd_fact(int t) { return t <= 0 ? 1 : (2 * t + 1) * odd_fact(t - 1); }

// n! / (2^j j! (n-2j)!): the number of ways to pick j disjoint pairs out of n.
__host__ __device__ constexpr int pair_count(int n, int j)
{
    return ifact(n) / ((1 << j) * ifact(j) * ifact(n - 2 * j));
}

// Compile-time loop: f(std::integral_constant<int, i>) for i = B .. E-1, so
// that every coefficient index below is a constant and the expansions live
// in registers.
template <int B, int E, class F>
__device__ __forceinline__ void cfor(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        cfor<B + 1, E>(f);
    }
}

#define PSR_CI(v) constexpr int v = decltype(v##_)::value

// Cells of particles: a cell's particles are [first[c], first[c+1]) or, with
// a leaf record, [leaf[c].x, leaf[c].x + leaf[c].y); coordinates and masses
// are read with strides (n x 3 arrays, or the x, y, z, m rows of a
// workspace's FP64 copy).
struct Cells {
    const int64_t* first;
    const int4* leaf;
    const double* pos;
    const double* mass;  // NULL: every mass is m_default
    const double* centre;
    int pstride, mstride, cstride;
    double m_default;
};

__device__ __forceinline__ void cell_range(const Cells& C, int64_t c, int64_t& b, int64_t& e)
{
    if (C.leaf) {
        const int4 r = C.leaf[c];
        b = r.x;
        e = (int64_t)r.x + r.y;
    } else {
        b = C.first[c];
        e = C.first[c + 1];
    }
}

// phi[k] = r^(2k+1) f_(k)(r) for k = 0..P, x = r / 2 r_s.  Written at the
// length scale r itself, the paper's closed form for f_(k) becomes
//   phi_k = (-1)^k (2k-1)!! [erfc(x) + exp(-x^2)/sqrt(pi) S_k],
//   S_k = sum_{t < k} 2^(t+1) x^(2t+1) / (2t+1)!!,
// every term bounded for x <= x_c (phi_0 = erfc(x), phi_1 = -T(x)).
template <int P>
__device__ __forceinline__ void prefactors(float x, float (&phi)[P + 1])
{
    const float e = erfcf(x), g = expf(-x * x) * 0.5641895835477563f;  // exp(-x^2)/sqrt(pi)
    const float x2 = 2.0f * x * x;
    float a = 2.0f * x, S = 0.0f;  // a = 2^(t+1) x^(2t+1) / (2t+1)!!
    phi[0] = e;
    cfor<1, P + 1>([&](auto k_) {
        PSR_CI(k);
        S += a;
        a *= x2 * (1.0f / (float)(2 * k + 1));
        const float v = (float)odd_fact(k - 1) * fmaf(g, S, e);
        phi[k] = (k & 1) ? -v : v;
    });
}

// One M2L entry added into acc: Lh_n += sum_{|m| <= P-|n|} Mh_m Dh_{n+m}.
// u = R / |R| and sigma = h / |R|.  Every Dh_k with |k| <= P is formed once,
//   Dh_k = h^(|k|+1) D_k = sigma^(|k|+1) sum_{j <= k/2} prod_a pair_count(k_a, j_a) u^(k-2j) phi_(|k|-|j|)
// (nothing overflows while sigma^(P+1) stays in range), and scattered into
// every L_n with n <= k componentwise (m = k - n).
template <int P, bool VEC>
__device__ __forceinline__ void m2l_entry(const float (&u)[3], float sigma, float x,
                                          const float* __restrict__ Ms, float (&acc)[ncoef(P)])
{
    constexpr int NC = ncoef(P);
    float phi[P + 1];
    prefactors<P>(x, phi);
    float pw[3][P + 1], sg[P + 1];
    sg[0] = sigma;
#pragma unroll
    for (int k = 1; k <= P; ++k) sg[k] = sg[k - 1] * sigma;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pw[a][0] = 1.0f;
#pragma unroll
        for (int k = 1; k <= P; ++k) pw[a][k] = pw[a][k - 1] * u[a];
    }
    float m[(NC + 3) & ~3];
    if constexpr (VEC) {  // rows padded to a multiple of 4 floats, 16-byte aligned
#pragma unroll
        for (int i = 0; i < (NC + 3) / 4; ++i) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(Ms) + i);
            m[4 * i] = v.x;
            m[4 * i + 1] = v.y;
            m[4 * i + 2] = v.z;
            m[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NC; ++i) m[i] = __ldg(Ms + i);
    }
    cfor<0, P + 1>([&](auto K_) {
        PSR_CI(K);
        cfor<0, K + 1>([&](auto a_) {
            PSR_CI(a);
            cfor<0, K - a + 1>([&](auto b_) {
                PSR_CI(b);
                constexpr int c = K - a - b;
                float d = 0.0f;
                cfor<0, a / 2 + 1>([&](auto ja_) {
                    PSR_CI(ja);
                    cfor<0, b / 2 + 1>([&](auto jb_) {
                        PSR_CI(jb);
                        cfor<0, c / 2 + 1>([&](auto jc_) {
                            PSR_CI(jc);
                            constexpr float cf =
                                (float)(pair_count(a, ja) * pair_count(b, jb) * pair_count(c, jc));
                            d = fmaf(cf * phi[K - ja - jb - jc],
                                     pw[0][a - 2 * ja] * pw[1][b - 2 * jb] * pw[2][c - 2 * jc], d);
                        });
                    });
                });
                d *= sg[K];
                cfor<0, a + 1>([&](auto n1_) {
                    PSR_CI(n1);
                    cfor<0, b + 1>([&](auto n2_) {
                        PSR_CI(n2);
                        cfor<0, c + 1>([&](auto n3_) {
                            PSR_CI(n3);
                            constexpr int i = cidx(n1, n2, n3);
                            acc[i] = fmaf(m[cidx(a - n1, b - n2, c - n3)], d, acc[i]);
                        });
                    });
                });
            });
        });
    });
}

}  // namespace

namespace {

// Mh_m = sum_j m_j ((z_A - x_j)/h)^m / m!, one thread per cell.
template <int P>
__global__ void __launch_bounds__(128) k_p2m(Cells C, double inv_h, int64_t ncell,
                                             float* __restrict__ M, int mstride)
{
    constexpr int NC = ncoef(P);
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    float acc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = 0.0f;
    const double* zc = C.centre + c * C.cstride;
    const double z[3] = {zc[0], zc[1], zc[2]};
    int64_t j, j1;
    cell_range(C, c, j, j1);
    for (; j < j1; ++j) {
        float pw[3][P + 1];  // v^k / k!
        const double* xj = C.pos + j * C.pstride;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = (float)((z[a] - xj[a]) * inv_h);
            pw[a][0] = 1.0f;
#pragma unroll
            for (int k = 1; k <= P; ++k) pw[a][k] = pw[a][k - 1] * v * (1.0f / (float)k);
        }
        const float m = C.mass ? (float)C.mass[j * C.mstride] : (float)C.m_default;
        cfor<0, P + 1>([&](auto K_) {
            PSR_CI(K);
            cfor<0, K + 1>([&](auto a_) {
                PSR_CI(a);
                const float ma = m * pw[0][a];
                cfor<0, K - a + 1>([&](auto b_) {
                    PSR_CI(b);
                    constexpr int i = cidx(a, b, K - a - b);
                    acc[i] = fmaf(ma * pw[1][b], pw[2][K - a - b], acc[i]);
                });
            });
        });
    }
    float* out = M + c * mstride;
#pragma unroll
    for (int i = 0; i < NC; ++i) out[i] = acc[i];
    for (int i = NC; i < mstride; ++i) out[i] = 0.0f;
}

// Centres of the M2L cells: FP64 coordinates (stride cstride), or, for a
// leaf handle (CELL), the exact integer cell centre (lcen, units of
// unit = L / 2^22) plus an FP32 offset (fofs), so that a centre difference
// is an exact integer part plus a small FP32 one and needs no FP64.
struct Centres {
    const double* ct;
    const double* cs;
    int cstride;
    const int4* lcen;
    const float4* fofs;
    float unit;
};

// Lh_n = sum over the row's (source, image) entries of sum_m Mh_m Dh_{n+m}.
// G lanes per target cell (G divides 32): the lanes take the row's entries
// in turn and their partial expansions are summed by shuffles.  Every lane
// of a warp reaches the shuffles (lanes past the last target carry empty
// rows).  Entry = (source << 5) | image code, the code (nx+1)*9 + (ny+1)*3 +
// (nz+1); the source centre is taken at c_s + n L.  Coefficient rows are
// mstride floats apart (CELL: a multiple of 4, 16-byte aligned).
template <int P, int G, bool CELL>
__global__ void __launch_bounds__(128) k_m2l(Centres Z, double inv_h, float inv_hf, float x_per_h,
                                             double L, int64_t ntarget, int64_t nsource,
                                             const int64_t* __restrict__ rowptr,
                                             const uint32_t* __restrict__ pairs,
                                             const float* __restrict__ M, int mstride,
                                             float* __restrict__ Lout, unsigned* __restrict__ err)
{
    constexpr int NC = ncoef(P);
    const int sub = threadIdx.x & (G - 1);
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    const bool live = t < ntarget;
    float acc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = 0.0f;
    int64_t e = 0, e1 = 0;
    double z[3] = {0.0, 0.0, 0.0};
    int4 qt = make_int4(0, 0, 0, 0);
    float4 ot = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        e = rowptr[t] + sub;
        e1 = rowptr[t + 1];
        if constexpr (CELL) {
            qt = Z.lcen[t];
            ot = Z.fofs[t];
        } else {
            z[0] = Z.ct[t * Z.cstride];
            z[1] = Z.ct[t * Z.cstride + 1];
            z[2] = Z.ct[t * Z.cstride + 2];
        }
    }
    for (; e < e1; e += G) {
        const uint32_t ent = pairs[e];
        const int64_t s = ent >> 5;
        const int code = ent & 31;
        if (s >= nsource || code >= 27) {
            if (err) atomicOr(err, 1u);
            continue;
        }
        const int sh[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
        float Rh[3];
        if constexpr (CELL) {
            const int4 qs = Z.lcen[s];
            const float4 os = Z.fofs[s];
            const int dq[3] = {qt.x - qs.x - sh[0] * (1 << kCentreShift),
                               qt.y - qs.y - sh[1] * (1 << kCentreShift),
                               qt.z - qs.z - sh[2] * (1 << kCentreShift)};
            const float dof[3] = {ot.x - os.x, ot.y - os.y, ot.z - os.z};
#pragma unroll
            for (int a = 0; a < 3; ++a) Rh[a] = fmaf((float)dq[a], Z.unit, dof[a]) * inv_hf;
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double d = z[a] - Z.cs[s * Z.cstride + a];
                Rh[a] = (float)((sh[a] == 0 ? d : d - sh[a] * L) * inv_h);
            }
        }
        const float r2 = fmaf(Rh[0], Rh[0], fmaf(Rh[1], Rh[1], Rh[2] * Rh[2]));
        if (!(r2 > 0.0f)) {  // coincident centres: no expansion exists
            if (err) atomicOr(err, 2u);
            continue;
        }
        const float ri = rsqrtf(r2), r = r2 * ri;
        const float u[3] = {Rh[0] * ri, Rh[1] * ri, Rh[2] * ri};
        m2l_entry<P, CELL>(u, ri, r * x_per_h, M + s * mstride, acc);
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        float v = acc[i];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        acc[i] = v;
    }
    if (live && sub == 0) {
        float* out = Lout + t * mstride;
#pragma unroll
        for (int i = 0; i < NC; ++i) out[i] = acc[i];
        for (int i = NC; i < mstride; ++i) out[i] = 0.0f;
    }
}

// a_c(x) = (G / h^2) sum_{|k| <= p-1} Lh_{k+e_c} ((x - z_B)/h)^k / k!, one
// thread per cell; written to, or added into, the n x 3 output (FP32 or
// FP64) at row j, or at row perm[j] when a permutation is given.
template <int P, class OutT>
__global__ void __launch_bounds__(128) k_l2p(Cells C, double inv_h, float g_over_h2,
                                             int64_t ncell, const float* __restrict__ Lin,
                                             int mstride, const int32_t* __restrict__ perm,
                                             OutT* __restrict__ acc, int accumulate)
{
    constexpr int NC = ncoef(P);
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    float Lc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) Lc[i] = Lin[c * mstride + i];
    const double* zc = C.centre + c * C.cstride;
    const double z[3] = {zc[0], zc[1], zc[2]};
    int64_t j, j1;
    cell_range(C, c, j, j1);
    for (; j < j1; ++j) {
        float pw[3][P];  // u^k / k!
        const double* xj = C.pos + j * C.pstride;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float u = (float)((xj[a] - z[a]) * inv_h);
            pw[a][0] = 1.0f;
#pragma unroll
            for (int k = 1; k < P; ++k) pw[a][k] = pw[a][k - 1] * u * (1.0f / (float)k);
        }
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
        cfor<0, P>([&](auto K_) {
            PSR_CI(K);
            cfor<0, K + 1>([&](auto a_) {
                PSR_CI(a);
                cfor<0, K - a + 1>([&](auto b_) {
                    PSR_CI(b);
                    constexpr int d = K - a - b;
                    const float mono = pw[0][a] * pw[1][b] * pw[2][d];
                    s0 = fmaf(Lc[cidx(a + 1, b, d)], mono, s0);
                    s1 = fmaf(Lc[cidx(a, b + 1, d)], mono, s1);
                    s2 = fmaf(Lc[cidx(a, b, d + 1)], mono, s2);
                });
            });
        });
        const float v[3] = {g_over_h2 * s0, g_over_h2 * s1, g_over_h2 * s2};
        OutT* o = acc + 3 * (perm ? (int64_t)perm[j] : j);
#pragma unroll
        for (int a = 0; a < 3; ++a) o[a] = accumulate ? o[a] + (OutT)v[a] : (OutT)v[a];
    }
}

#undef PSR_CI

}  // namespace

namespace {

int ffail(int code, const std::string& msg)
{
    set_last_error(msg);
    return code;
}

int fcuda(const char* what)
{
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PSR_OK
                            : ffail(PSR_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

unsigned fblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Calls f(std::integral_constant<int, p>) for the runtime order p in [1, 6].
template <class F>
void by_order(int p, F&& f)
{
    switch (p) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 5: f(std::integral_constant<int, 5>{}); break;
        default: f(std::integral_constant<int, 6>{}); break;
    }
}

constexpr int kM2LGroup = 8;  // lanes per target cell in M2L

int check_order(int p, double h)
{
    if (p < 1 || p > kMaxOrder) return ffail(PSR_E_ARG, "order p must be in [1, 6]");
    if (!(h > 0) || !std::isfinite(h)) return ffail(PSR_E_ARG, "scale h must be finite and positive");
    return PSR_OK;
}

}  // namespace

namespace {

int launch_p2m(int p, double h, const Cells& C, int64_t ncell, float* M, int mstride,
               cudaStream_t st)
{
    by_order(p, [&](auto P_) {
        constexpr int P = decltype(P_)::value;
        k_p2m<P><<<fblk(ncell, 128), 128, 0, st>>>(C, 1.0 / h, ncell, M, mstride);
    });
    return fcuda("P2M kernel");
}

int launch_m2l(int p, double h, const psr_box& box, int64_t ntarget, int64_t nsource,
               const int64_t* rowptr, const uint32_t* pairs, const Centres& Z, bool cell,
               const float* M, int mstride, float* Lout, unsigned* status, cudaStream_t st)
{
    const unsigned grid = fblk(ntarget * kM2LGroup, 128);
    const double inv_h = 1.0 / h;
    const float xh = (float)(0.5 * h / box.r_s);
    by_order(p, [&](auto P_) {
        constexpr int P = decltype(P_)::value;
        if (cell)
            k_m2l<P, kM2LGroup, true><<<grid, 128, 0, st>>>(Z, inv_h, (float)inv_h, xh, box.L,
                                                            ntarget, nsource, rowptr, pairs, M,
                                                            mstride, Lout, status);
        else
            k_m2l<P, kM2LGroup, false><<<grid, 128, 0, st>>>(Z, inv_h, (float)inv_h, xh, box.L,
                                                             ntarget, nsource, rowptr, pairs, M,
                                                             mstride, Lout, status);
    });
    return fcuda("M2L kernel");
}

int launch_l2p(int p, double h, const psr_box& box, const Cells& C, int64_t ncell,
               const float* Lin, int mstride, const int32_t* perm, void* acc, bool f64,
               bool accumulate, cudaStream_t st)
{
    const float g = (float)(box.G / (h * h));
    by_order(p, [&](auto P_) {
        constexpr int P = decltype(P_)::value;
        if (f64)
            k_l2p<P, double><<<fblk(ncell, 128), 128, 0, st>>>(
                C, 1.0 / h, g, ncell, Lin, mstride, perm, (double*)acc, accumulate ? 1 : 0);
        else
            k_l2p<P, float><<<fblk(ncell, 128), 128, 0, st>>>(
                C, 1.0 / h, g, ncell, Lin, mstride, perm, (float*)acc, accumulate ? 1 : 0);
    });
    return fcuda("L2P kernel");
}

bool kernel_box_ok(const psr_box* box)
{
    return box && box->r_s > 0 && std::isfinite(box->r_s) && box->L > 0 && std::isfinite(box->L);
}

}  // namespace

extern "C" {

int psr_fmm_ncoef(int p, int* ncoef_out)
{
    if (!ncoef_out || p < 0 || p > kMaxOrder) return ffail(PSR_E_ARG, "need 0 <= p <= 6");
    *ncoef_out = ncoef(p);
    return PSR_OK;
}

int psr_fmm_p2m(int p, double h, int64_t n, int64_t ncell, const int64_t* d_first,
                const double* d_pos, const double* d_mass, const double* d_centre, float* d_M,
                void* stream)
{
    int rc = check_order(p, h);
    if (rc) return rc;
    if (ncell < 0 || n < 0 || (ncell > 0 && (!d_first || !d_centre || !d_M || (n > 0 && !d_pos))))
        return ffail(PSR_E_ARG, "null argument or negative count");
    if (ncell == 0) return PSR_OK;
    const Cells C{d_first, nullptr, d_pos, d_mass, d_centre, 3, 1, 3,
                  n > 0 ? 1.0 / (double)n : 0.0};
    return launch_p2m(p, h, C, ncell, d_M, ncoef(p), (cudaStream_t)stream);
}

int psr_fmm_m2l(int p, double h, const psr_box* box, int64_t ntarget, int64_t nsource,
                const int64_t* d_rowptr, const uint32_t* d_pairs, const double* d_centre_t,
                const double* d_centre_s, const float* d_M, float* d_L, unsigned* d_status,
                void* stream)
{
    int rc = check_order(p, h);
    if (rc) return rc;
    if (!kernel_box_ok(box)) return ffail(PSR_E_ARG, "box needs L > 0 and r_s > 0");
    if (ntarget < 0 || nsource < 0 ||
        (ntarget > 0 && (!d_rowptr || !d_centre_t || !d_L || (nsource > 0 && (!d_pairs || !d_centre_s || !d_M)))))
        return ffail(PSR_E_ARG, "null argument or negative count");
    if (ntarget == 0) return PSR_OK;
    const Centres Z{d_centre_t, d_centre_s, 3, nullptr, nullptr, 0.0f};
    return launch_m2l(p, h, *box, ntarget, nsource, d_rowptr, d_pairs, Z, false, d_M, ncoef(p),
                      d_L, d_status, (cudaStream_t)stream);
}

int psr_fmm_l2p(int p, double h, const psr_box* box, int64_t ncell, const int64_t* d_first,
                const double* d_pos, const double* d_centre, const float* d_L, float* d_acc,
                int flags, void* stream)
{
    int rc = check_order(p, h);
    if (rc) return rc;
    if (!box || !std::isfinite(box->G)) return ffail(PSR_E_ARG, "box needs a finite G");
    if (flags & ~PSR_FMM_ACCUMULATE) return ffail(PSR_E_ARG, "unknown L2P flags");
    if (ncell < 0 || (ncell > 0 && (!d_first || !d_pos || !d_centre || !d_L || !d_acc)))
        return ffail(PSR_E_ARG, "null argument or negative count");
    if (ncell == 0) return PSR_OK;
    const Cells C{d_first, nullptr, d_pos, nullptr, d_centre, 3, 1, 3, 0.0};
    return launch_l2p(p, h, *box, C, ncell, d_L, ncoef(p), nullptr, d_acc, false,
                      (flags & PSR_FMM_ACCUMULATE) != 0, (cudaStream_t)stream);
}

int psr_fmm_forces(const psr_leaves* hh, int p, int flags, float* d_M, float* d_L, void* d_acc,
                   unsigned* d_status, void* stream)
{
    const Leaves* h = reinterpret_cast<const Leaves*>(hh);
    if (!h) return ffail(PSR_E_ARG, "null handle");
    if (p < 1 || p > kMaxOrder) return ffail(PSR_E_ARG, "order p must be in [1, 6]");
    if (flags & ~(PSR_FMM_ACCUMULATE | PSR_FMM_F64)) return ffail(PSR_E_ARG, "unknown flags");
    if (!h->has_far) return ffail(PSR_E_STATE, "not a psr_device_build_split handle");
    if (!h->uploaded || !h->d_ws) return ffail(PSR_E_STATE, "workspace not written yet");
    if (!h->has_pd) return ffail(PSR_E_STATE, "the FP64 particle copy is absent (PSR_BUILD_NO_FP64)");
    const int64_t nl = h->n_leaves;
    if (nl == 0) return PSR_OK;
    if (!d_M || !d_L || !d_acc) return ffail(PSR_E_ARG, "null argument");
    if ((reinterpret_cast<uintptr_t>(d_M) | reinterpret_cast<uintptr_t>(d_L)) & 15)
        return ffail(PSR_E_ARG, "d_M and d_L must be 16-byte aligned");
    const psr_box& box = h->boxes[0];
    if (!kernel_box_ok(&box) || !std::isfinite(box.G)) return ffail(PSR_E_ARG, "bad box");
    const double scale = box.r_s;
    const char* w = h->d_ws;
    const Layout& L = h->lay;
    const double* pd = (const double*)(w + L.pd);
    const double* fcen = (const double*)(w + L.fcen);
    const Cells C{nullptr, (const int4*)(w + L.leaf), pd, pd + 3, fcen, 4, 4, 4, 0.0};
    const int ms = (ncoef(p) + 3) & ~3;  // padded rows: float4 loads in M2L
    const Centres Z{nullptr, nullptr, 0, (const int4*)(w + L.lcen), (const float4*)(w + L.fofs),
                    (float)std::ldexp(box.L, -kCentreShift)};
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_p2m(p, scale, C, nl, d_M, ms, st);
    if (rc) return rc;
    rc = launch_m2l(p, scale, box, nl, nl, (const int64_t*)(w + L.frow),
                    (const uint32_t*)(w + L.fpairs), Z, true, d_M, ms, d_L, d_status, st);
    if (rc) return rc;
    return launch_l2p(p, scale, box, C, nl, d_L, ms, (const int32_t*)(w + L.perm), d_acc,
                      (flags & PSR_FMM_F64) != 0, (flags & PSR_FMM_ACCUMULATE) != 0, st);
}

}  // extern "C"
