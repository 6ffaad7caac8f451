// Long-range particle-mesh (PM) accelerations of the PM-FMM split (paper,
// Section 2: phi_long solves Poisson's equation on a mesh with a Gaussian-
// filtered Green's function; the split radius is r_s = 1.2 L / N_PM).
//
//   1. k_cic_deposit  cloud-in-cell assignment of the masses onto the N^3 mesh
//                     (points at g L/N), FP32 atomics, density m / Delta^3
//   2. cuFFT R2C
//   3. k_pm_green     times -4 pi G exp(-k^2 r_s^2) / k^2, divided by the
//                     squared CIC window (assignment and interpolation) unless
//                     PSR_PM_NO_DECONVOLVE, and by N^3 (cuFFT does not
//                     normalise); zero at k = 0
//   4. per axis c: k_pm_grad (-i k_c, Nyquist plane of axis c zeroed), cuFFT C2R
//   5. k_cic_interp   CIC interpolation of the three component meshes at the
//                     particles, written to (or added into) the output
//
// The filter is exp(-k^2 r_s^2), the Fourier complement of the short-range
// erfc(r/2 r_s) of Eq. tr (the paper prints exp(-k^2/4r_s^2), which is not).
// cuFFT plans are made once per mesh size with automatic work-area allocation
// off: psr_pm_forces runs the FFTs in the caller's scratch.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <new>
#include <string>

#include "kcommon.cuh"

namespace psr {
void set_last_error(const std::string& msg);
}

using namespace psr;

struct psr_pm {
    int n;
    cufftHandle r2c, c2r;
    size_t work;  // bytes of the larger cuFFT work area
};

namespace {

struct Mesh {
    size_t rho, phik, ak, ax, ay, az, work, bytes;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

Mesh mesh_layout(int n, size_t work)
{
    Mesh m{};
    const size_t nr = (size_t)n * n * n, nc = (size_t)n * n * (n / 2 + 1);
    size_t o = 0;
    m.rho = o;  o = a256(o + 4 * nr);
    m.phik = o; o = a256(o + 8 * nc);
    m.ak = o;   o = a256(o + 8 * nc);
    m.ax = o;   o = a256(o + 4 * nr);
    m.ay = o;   o = a256(o + 4 * nr);
    m.az = o;   o = a256(o + 4 * nr);
    m.work = o; o = a256(o + work);
    m.bytes = o;
    return m;
}

struct CicPoint {
    int i[3][2];
    float w[3][2];
};

// wrapped position -> the two mesh points and weights per axis
__device__ __forceinline__ CicPoint cic_point(const double* p, double L, double inv_delta, int n)
{
    CicPoint c;
    for (int a = 0; a < 3; ++a) {
        double v = fmod(p[a], L);
        if (v < 0) v += L;
        if (!(v < L)) v = 0.0;
        const double u = v * inv_delta;
        double fl = floor(u);
        int i0 = (int)fl;
        if (i0 >= n) i0 = n - 1;  // u rounded up to n
        const float f = (float)(u - fl);
        c.i[a][0] = i0;
        c.i[a][1] = i0 + 1 == n ? 0 : i0 + 1;
        c.w[a][0] = 1.0f - f;
        c.w[a][1] = f;
    }
    return c;
}

// A particle with a non-finite coordinate deposits nothing (and is skipped
// by the interpolation).
__global__ void k_cic_deposit(const double* __restrict__ pos, const double* __restrict__ mass,
                              int64_t np, double L, double inv_delta, int n, float m_default,
                              float inv_vol, float* __restrict__ rho)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const double p[3] = {pos[3 * j], pos[3 * j + 1], pos[3 * j + 2]};
    if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) return;
    const float m = (mass ? (float)mass[j] : m_default) * inv_vol;
    const CicPoint c = cic_point(p, L, inv_delta, n);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const size_t row = ((size_t)c.i[0][a] * n + c.i[1][b]) * n;
            const float wab = m * c.w[0][a] * c.w[1][b];
            atomicAdd(rho + row + c.i[2][0], wab * c.w[2][0]);
            atomicAdd(rho + row + c.i[2][1], wab * c.w[2][1]);
        }
}

// signed frequency of FFT index i (index n/2 is the Nyquist frequency -n/2)
__device__ __forceinline__ int freq(int i, int n) { return i < n / 2 ? i : i - n; }

// phik *= Green's function (and 1 / N^3); one thread per complex mode
__global__ void k_pm_green(cufftComplex* __restrict__ phik, int n, float kf, float r_s2, float g4pi,
                           float half_delta, int deconvolve, float inv_n3)
{
    const int64_t nz = n / 2 + 1;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n * nz) return;
    const int iz = (int)(t % nz), iy = (int)((t / nz) % n), ix = (int)(t / (nz * n));
    const float kx = kf * freq(ix, n), ky = kf * freq(iy, n), kz = kf * iz;
    const float k2 = kx * kx + ky * ky + kz * kz;
    float g = 0.0f;
    if (k2 > 0.0f) {
        g = -g4pi * expf(-k2 * r_s2) / k2 * inv_n3;
        if (deconvolve) {
            const float kk[3] = {kx, ky, kz};
            for (int a = 0; a < 3; ++a) {
                const float y = kk[a] * half_delta;
                const float s = y == 0.0f ? 1.0f : sinf(y) / y;
                const float s2 = s * s;
                g /= s2 * s2;
            }
        }
    }
    cufftComplex v = phik[t];
    v.x *= g;
    v.y *= g;
    phik[t] = v;
}

// ak = -i k_c phik; the Nyquist plane of axis c is zeroed
__global__ void k_pm_grad(const cufftComplex* __restrict__ phik, cufftComplex* __restrict__ ak,
                          int n, float kf, int c)
{
    const int64_t nz = n / 2 + 1;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n * nz) return;
    const int iz = (int)(t % nz), iy = (int)((t / nz) % n), ix = (int)(t / (nz * n));
    const int f = c == 0 ? freq(ix, n) : c == 1 ? freq(iy, n) : iz;
    const bool nyq = (n % 2 == 0) && (f == n / 2 || f == -n / 2);
    const float k = nyq ? 0.0f : kf * f;
    const cufftComplex v = phik[t];
    ak[t] = make_float2(k * v.y, -k * v.x);  // -i k (x + i y) = k y - i k x
}

__global__ void k_cic_interp(const double* __restrict__ pos, int64_t np, double L,
                             double inv_delta, int n, const float* __restrict__ gx,
                             const float* __restrict__ gy, const float* __restrict__ gz,
                             float* __restrict__ acc, int accumulate)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const double p[3] = {pos[3 * j], pos[3 * j + 1], pos[3 * j + 2]};
    if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) return;
    const CicPoint c = cic_point(p, L, inv_delta, n);
    float s[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) {
                const size_t q = ((size_t)c.i[0][a] * n + c.i[1][b]) * n + c.i[2][d];
                const float w = c.w[0][a] * c.w[1][b] * c.w[2][d];
                s[0] = fmaf(w, gx[q], s[0]);
                s[1] = fmaf(w, gy[q], s[1]);
                s[2] = fmaf(w, gz[q], s[2]);
            }
    for (int a = 0; a < 3; ++a) acc[3 * j + a] = accumulate ? acc[3 * j + a] + s[a] : s[a];
}

int pfail(int code, const std::string& msg)
{
    set_last_error(msg);
    return code;
}

int cuda_err(cudaError_t e, const char* what)
{
    return pfail(PSR_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int fft_err(cufftResult r, const char* what)
{
    return pfail(PSR_E_CUDA, std::string(what) + ": cuFFT status " + std::to_string((int)r));
}

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" {

int psr_pm_create(int n_pm, psr_pm** out)
{
    if (!out) return pfail(PSR_E_ARG, "null output");
    *out = nullptr;
    if (n_pm < 8 || n_pm > 1024 || (n_pm & 1))
        return pfail(PSR_E_ARG, "n_pm must be even and in [8, 1024]");
    psr_pm* pm = new (std::nothrow) psr_pm();
    if (!pm) return pfail(PSR_E_NOMEM, "out of host memory");
    pm->n = n_pm;
    size_t w1 = 0, w2 = 0;
    cufftResult r;
    if ((r = cufftCreate(&pm->r2c)) != CUFFT_SUCCESS) {
        delete pm;
        return fft_err(r, "cufftCreate");
    }
    if ((r = cufftCreate(&pm->c2r)) != CUFFT_SUCCESS) {
        cufftDestroy(pm->r2c);
        delete pm;
        return fft_err(r, "cufftCreate");
    }
    if ((r = cufftSetAutoAllocation(pm->r2c, 0)) != CUFFT_SUCCESS ||
        (r = cufftSetAutoAllocation(pm->c2r, 0)) != CUFFT_SUCCESS ||
        (r = cufftMakePlan3d(pm->r2c, n_pm, n_pm, n_pm, CUFFT_R2C, &w1)) != CUFFT_SUCCESS ||
        (r = cufftMakePlan3d(pm->c2r, n_pm, n_pm, n_pm, CUFFT_C2R, &w2)) != CUFFT_SUCCESS) {
        cufftDestroy(pm->r2c);
        cufftDestroy(pm->c2r);
        delete pm;
        return fft_err(r, "cuFFT plan");
    }
    pm->work = w1 > w2 ? w1 : w2;
    *out = pm;
    return PSR_OK;
}

int psr_pm_scratch_bytes(const psr_pm* pm, size_t* bytes)
{
    if (!pm || !bytes) return pfail(PSR_E_ARG, "null argument");
    *bytes = mesh_layout(pm->n, pm->work).bytes;
    return PSR_OK;
}

int psr_pm_forces(psr_pm* pm, const double* d_pos, const double* d_mass, int64_t n,
                  const psr_box* box, int flags, void* d_scratch, size_t scratch_bytes,
                  float* d_acc, void* stream)
{
    if (!pm || !box || ((!d_pos || !d_acc) && n > 0) || n < 0)
        return pfail(PSR_E_ARG, "null argument or n < 0");
    if (flags & ~(PSR_PM_ACCUMULATE | PSR_PM_NO_DECONVOLVE))
        return pfail(PSR_E_ARG, "unknown PM flags");
    if (!(std::isfinite(box->L) && box->L > 0) || !(std::isfinite(box->r_s) && box->r_s > 0) ||
        !std::isfinite(box->G))
        return pfail(PSR_E_ARG, "L, r_s must be finite and positive");
    const int N = pm->n;
    const Mesh M = mesh_layout(N, pm->work);
    if (!d_scratch || scratch_bytes < M.bytes || (reinterpret_cast<uintptr_t>(d_scratch) & 255))
        return pfail(PSR_E_WORKSPACE, "scratch must be 256-byte aligned and at least " +
                                          std::to_string(M.bytes) + " bytes");
    if (n == 0) return PSR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char* s = static_cast<char*>(d_scratch);
    float* rho = (float*)(s + M.rho);
    cufftComplex* phik = (cufftComplex*)(s + M.phik);
    cufftComplex* ak = (cufftComplex*)(s + M.ak);
    float* g[3] = {(float*)(s + M.ax), (float*)(s + M.ay), (float*)(s + M.az)};
    const double L = box->L, delta = L / N;
    const int64_t nr = (int64_t)N * N * N, nc = (int64_t)N * N * (N / 2 + 1);
    cudaError_t e;
    cufftResult r;
    if ((e = cudaMemsetAsync(rho, 0, 4 * (size_t)nr, st)) != cudaSuccess) return cuda_err(e, "cudaMemsetAsync");
    k_cic_deposit<<<nblk(n, 256), 256, 0, st>>>(d_pos, d_mass, n, L, 1.0 / delta, N,
                                                (float)(1.0 / (double)n),
                                                (float)(1.0 / (delta * delta * delta)), rho);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "deposit kernel");
    if ((r = cufftSetStream(pm->r2c, st)) != CUFFT_SUCCESS ||
        (r = cufftSetStream(pm->c2r, st)) != CUFFT_SUCCESS ||
        (r = cufftSetWorkArea(pm->r2c, s + M.work)) != CUFFT_SUCCESS ||
        (r = cufftSetWorkArea(pm->c2r, s + M.work)) != CUFFT_SUCCESS)
        return fft_err(r, "cuFFT stream / work area");
    if ((r = cufftExecR2C(pm->r2c, rho, phik)) != CUFFT_SUCCESS) return fft_err(r, "cufftExecR2C");
    const float kf = (float)(2.0 * M_PI / L);
    k_pm_green<<<nblk(nc, 256), 256, 0, st>>>(
        phik, N, kf, (float)(box->r_s * box->r_s), (float)(4.0 * M_PI * box->G),
        (float)(0.5 * delta), (flags & PSR_PM_NO_DECONVOLVE) ? 0 : 1, (float)(1.0 / (double)nr));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "Green kernel");
    for (int c = 0; c < 3; ++c) {
        k_pm_grad<<<nblk(nc, 256), 256, 0, st>>>(phik, ak, N, kf, c);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "gradient kernel");
        if ((r = cufftExecC2R(pm->c2r, ak, g[c])) != CUFFT_SUCCESS) return fft_err(r, "cufftExecC2R");
    }
    k_cic_interp<<<nblk(n, 256), 256, 0, st>>>(d_pos, n, L, 1.0 / delta, N, g[0], g[1], g[2], d_acc,
                                               (flags & PSR_PM_ACCUMULATE) ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "interpolation kernel");
    return PSR_OK;
}

void psr_pm_free(psr_pm* pm)
{
    if (!pm) return;
    cufftDestroy(pm->r2c);
    cufftDestroy(pm->c2r);
    delete pm;
}

}  // extern "C"
