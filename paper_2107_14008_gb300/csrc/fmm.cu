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

#include "kcommon.cuh"

namespace psr {
void set_last_error(const std::string& msg);
}

using namespace psr;

namespace {

constexpr int kMaxOrder = 6;                                   // p
constexpr int kMaxCoef = (kMaxOrder + 1) * (kMaxOrder + 2) * (kMaxOrder + 3) / 6;       // 84
constexpr int kMaxDOrder = 2 * kMaxOrder;                      // derivatives up to 2p
constexpr int kMaxD = (kMaxDOrder + 1) * (kMaxDOrder + 2) * (kMaxDOrder + 3) / 6;       // 455

__host__ __device__ __forceinline__ int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

__device__ __forceinline__ int cidx(int a, int b, int c)
{
    const int K = a + b + c;
    return K * (K + 1) * (K + 2) / 6 + (K - a) * (K - a + 1) / 2 + (K - a - b);
}

__constant__ float c_fact[kMaxDOrder + 1] = {1.f, 1.f, 2.f, 6.f, 24.f, 120.f, 720.f, 5040.f,
                                             40320.f, 362880.f, 3628800.f, 39916800.f,
                                             479001600.f};

__device__ __forceinline__ float ffact(int n) { return c_fact[n]; }

// phi[k] = h^(2k+1) f_(k)(r) for k = 0..kmax from the closed form, written
// with x = r / 2 r_s, rho = h / r_s and w = rho / x = 2h / r so that no
// intermediate overflows for well-separated cells (w <= 1):
//   phi_k = (-1)^k [ (2k-1)!!/2^(2k+1) erfc(x) w^(2k+1)
//                    + exp(-x^2)/sqrt(pi) sum_q 2^(-q-k) (2k-1)!!/(2k-2q+1)!! rho^(2(k-q)+1) w^(2q) ]
__device__ void scaled_prefactors(float x, float rho, int kmax, float* phi)
{
    const float e = erfcf(x), g = expf(-x * x) * 0.5641895835477563f;  // exp(-x^2)/sqrt(pi)
    const float w = rho / x;
    // ascending powers only (no division, so nothing needed underflows)
    float w2q[kMaxDOrder + 1], rodd[kMaxDOrder + 1], dodd[kMaxDOrder + 1];
    w2q[0] = 1.0f;   // w^(2q)
    rodd[0] = rho;   // rho^(2t+1)
    dodd[0] = 1.0f;  // (2t+1)!!
    for (int t = 1; t <= kmax; ++t) {
        w2q[t] = w2q[t - 1] * w * w;
        rodd[t] = rodd[t - 1] * rho * rho;
        dodd[t] = dodd[t - 1] * (float)(2 * t + 1);
    }
    phi[0] = 0.5f * e * w;
    for (int k = 1; k <= kmax; ++k) {
        const float dk = dodd[k - 1];  // (2k-1)!!
        float t = 0.0f;
        for (int q = 1; q <= k; ++q)  // (2k-1)!!/(2k-2q+1)!! = dk / dodd[k-q]
            t += dk / dodd[k - q] * exp2f((float)(-q - k)) * rodd[k - q] * w2q[q];
        const float v = dk * exp2f((float)(-2 * k - 1)) * e * w2q[k] * w + g * t;
        phi[k] = (k & 1) ? -v : v;
    }
}

}  // namespace

namespace {

// Dh_n = h^(|n|+1) D_n(R) for every |n| <= order, at Rh = R / h (graded order).
__device__ void scaled_derivatives(const float Rh[3], float x, float rho, int order, float* D)
{
    float phi[kMaxDOrder + 1];
    scaled_prefactors(x, rho, order, phi);
    float pw[3][kMaxDOrder + 1];
    for (int a = 0; a < 3; ++a) {
        pw[a][0] = 1.0f;
        for (int k = 1; k <= order; ++k) pw[a][k] = pw[a][k - 1] * Rh[a];
    }
    for (int K = 0; K <= order; ++K)
        for (int n1 = K; n1 >= 0; --n1)
            for (int n2 = K - n1; n2 >= 0; --n2) {
                const int n3 = K - n1 - n2;
                float s = 0.0f;
                for (int j1 = 0; 2 * j1 <= n1; ++j1)
                    for (int j2 = 0; 2 * j2 <= n2; ++j2)
                        for (int j3 = 0; 2 * j3 <= n3; ++j3) {
                            const float c =
                                ffact(n1) / ((float)(1 << j1) * ffact(j1) * ffact(n1 - 2 * j1)) *
                                ffact(n2) / ((float)(1 << j2) * ffact(j2) * ffact(n2 - 2 * j2)) *
                                ffact(n3) / ((float)(1 << j3) * ffact(j3) * ffact(n3 - 2 * j3));
                            s += c * pw[0][n1 - 2 * j1] * pw[1][n2 - 2 * j2] * pw[2][n3 - 2 * j3] *
                                 phi[K - j1 - j2 - j3];
                        }
                D[cidx(n1, n2, n3)] = s;
            }
}

// Mh_m = sum_j m_j ((z_A - x_j)/h)^m / m!, one thread per cell.
__global__ void k_p2m(int p, double inv_h, int64_t ncell, const int64_t* __restrict__ first,
                      const double* __restrict__ pos, const double* __restrict__ mass,
                      double m_default, const double* __restrict__ centre, float* __restrict__ M)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int nc = ncoef(p);
    float acc[kMaxCoef];
    for (int i = 0; i < nc; ++i) acc[i] = 0.0f;
    for (int64_t j = first[c]; j < first[c + 1]; ++j) {
        float pw[3][kMaxOrder + 1];  // v^k / k!
        for (int a = 0; a < 3; ++a) {
            const float v = (float)((centre[3 * c + a] - pos[3 * j + a]) * inv_h);
            pw[a][0] = 1.0f;
            for (int k = 1; k <= p; ++k) pw[a][k] = pw[a][k - 1] * v / (float)k;
        }
        const float m = mass ? (float)mass[j] : (float)m_default;
        for (int K = 0; K <= p; ++K)
            for (int a = K; a >= 0; --a)
                for (int b = K - a; b >= 0; --b)
                    acc[cidx(a, b, K - a - b)] += m * pw[0][a] * pw[1][b] * pw[2][K - a - b];
    }
    for (int i = 0; i < nc; ++i) M[c * nc + i] = acc[i];
}

// Lh_n = sum over the row's (source, image) entries of sum_m Mh_m Dh_{n+m},
// one warp per target cell: the lanes take the row's entries in turn and the
// 32 partial expansions are summed by shuffles.  Entry = (source << 5) |
// image code, the code (nx+1)*9 + (ny+1)*3 + (nz+1); the source centre is
// taken at c_s + n L.
__global__ void k_m2l(int p, double inv_h, float x_per_h, float rho, double L, int64_t ntarget,
                      int64_t nsource, const int64_t* __restrict__ rowptr,
                      const uint32_t* __restrict__ pairs, const double* __restrict__ ct,
                      const double* __restrict__ cs, const float* __restrict__ M,
                      float* __restrict__ Lout, unsigned* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= ntarget) return;  // whole warps only
    const int nc = ncoef(p);
    float acc[kMaxCoef];
    for (int i = 0; i < nc; ++i) acc[i] = 0.0f;
    float D[kMaxD];
    for (int64_t e = rowptr[t] + lane; e < rowptr[t + 1]; e += 32) {
        const uint32_t ent = pairs[e];
        const int64_t s = ent >> 5;
        const int code = ent & 31;
        if (s >= nsource || code >= 27) {
            if (err) atomicOr(err, 1u);
            continue;
        }
        const int sh[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
        float Rh[3];
        float r2 = 0.0f;
        for (int a = 0; a < 3; ++a) {
            Rh[a] = (float)((ct[3 * t + a] - cs[3 * s + a] - sh[a] * L) * inv_h);
            r2 += Rh[a] * Rh[a];
        }
        if (!(r2 > 0.0f)) {  // coincident centres: no expansion exists
            if (err) atomicOr(err, 2u);
            continue;
        }
        scaled_derivatives(Rh, sqrtf(r2) * x_per_h, rho, 2 * p, D);
        const float* Ms = M + s * nc;
        for (int Kn = 0; Kn <= p; ++Kn)
            for (int n1 = Kn; n1 >= 0; --n1)
                for (int n2 = Kn - n1; n2 >= 0; --n2) {
                    const int n3 = Kn - n1 - n2;
                    float v = 0.0f;
                    for (int Km = 0; Km <= p - Kn; ++Km)
                        for (int m1 = Km; m1 >= 0; --m1)
                            for (int m2 = Km - m1; m2 >= 0; --m2) {
                                const int m3 = Km - m1 - m2;
                                v += Ms[cidx(m1, m2, m3)] * D[cidx(n1 + m1, n2 + m2, n3 + m3)];
                            }
                    acc[cidx(n1, n2, n3)] += v;
                }
    }
    for (int i = 0; i < nc; ++i) {
        float v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) Lout[t * nc + i] = v;
    }
}

// a_c(x) = (G / h^2) sum_{|k| <= p-1} Lh_{k+e_c} ((x - z_B)/h)^k / k!, one
// thread per cell; written to, or added into, the output.
__global__ void k_l2p(int p, double inv_h, float g_over_h2, int64_t ncell,
                      const int64_t* __restrict__ first, const double* __restrict__ pos,
                      const double* __restrict__ centre, const float* __restrict__ Lin,
                      float* __restrict__ acc, int accumulate)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int nc = ncoef(p);
    const float* Lc = Lin + c * nc;
    for (int64_t j = first[c]; j < first[c + 1]; ++j) {
        float pw[3][kMaxOrder + 1];  // u^k / k!
        for (int a = 0; a < 3; ++a) {
            const float u = (float)((pos[3 * j + a] - centre[3 * c + a]) * inv_h);
            pw[a][0] = 1.0f;
            for (int k = 1; k <= p; ++k) pw[a][k] = pw[a][k - 1] * u / (float)k;
        }
        float s[3] = {0.f, 0.f, 0.f};
        for (int K = 0; K <= p - 1; ++K)
            for (int a = K; a >= 0; --a)
                for (int b = K - a; b >= 0; --b) {
                    const int d = K - a - b;
                    const float mono = pw[0][a] * pw[1][b] * pw[2][d];
                    s[0] += Lc[cidx(a + 1, b, d)] * mono;
                    s[1] += Lc[cidx(a, b + 1, d)] * mono;
                    s[2] += Lc[cidx(a, b, d + 1)] * mono;
                }
        for (int a = 0; a < 3; ++a) {
            const float v = g_over_h2 * s[a];
            acc[3 * j + a] = accumulate ? acc[3 * j + a] + v : v;
        }
    }
}

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

int check_order(int p, double h)
{
    if (p < 1 || p > kMaxOrder) return ffail(PSR_E_ARG, "order p must be in [1, 6]");
    if (!(h > 0) || !std::isfinite(h)) return ffail(PSR_E_ARG, "scale h must be finite and positive");
    return PSR_OK;
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
    k_p2m<<<fblk(ncell, 128), 128, 0, (cudaStream_t)stream>>>(
        p, 1.0 / h, ncell, d_first, d_pos, d_mass, n > 0 ? 1.0 / (double)n : 0.0, d_centre, d_M);
    return fcuda("P2M kernel");
}

int psr_fmm_m2l(int p, double h, const psr_box* box, int64_t ntarget, int64_t nsource,
                const int64_t* d_rowptr, const uint32_t* d_pairs, const double* d_centre_t,
                const double* d_centre_s, const float* d_M, float* d_L, unsigned* d_status,
                void* stream)
{
    int rc = check_order(p, h);
    if (rc) return rc;
    if (!box || !(box->r_s > 0) || !std::isfinite(box->r_s) || !(box->L > 0))
        return ffail(PSR_E_ARG, "box needs L > 0 and r_s > 0");
    if (ntarget < 0 || nsource < 0 ||
        (ntarget > 0 && (!d_rowptr || !d_centre_t || !d_L || (nsource > 0 && (!d_pairs || !d_centre_s || !d_M)))))
        return ffail(PSR_E_ARG, "null argument or negative count");
    if (ntarget == 0) return PSR_OK;
    const double rho = h / box->r_s;
    k_m2l<<<fblk(ntarget * 32, 128), 128, 0, (cudaStream_t)stream>>>(
        p, 1.0 / h, (float)(0.5 * rho), (float)rho, box->L, ntarget, nsource, d_rowptr, d_pairs,
        d_centre_t, d_centre_s, d_M, d_L, d_status);
    return fcuda("M2L kernel");
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
    k_l2p<<<fblk(ncell, 128), 128, 0, (cudaStream_t)stream>>>(
        p, 1.0 / h, (float)(box->G / (h * h)), ncell, d_first, d_pos, d_centre, d_L, d_acc,
        (flags & PSR_FMM_ACCUMULATE) ? 1 : 0);
    return fcuda("L2P kernel");
}

}  // extern "C"
