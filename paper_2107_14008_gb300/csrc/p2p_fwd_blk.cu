// The paper's P2P work mapping (Section 3.2, Algorithms 1 and 2) as a
// prior-art variant (psr_opts.kernel = PSR_KERNEL_PAPER): one thread block
// per target leaf, target leaves taken in schedule order with a grid stride;
// one thread per target particle; each source leaf of the row staged into
// shared memory between two barriers; the Core loop over the staged
// particles.  Pair arithmetic, tables and accumulation are those of the
// warp-per-leaf kernels (leaf-local FP32 coordinates, exact leaf-centre
// offsets, FP32 partial sums folded into FP64 or compensated FP32, and with
// one mass for all particles, as in the paper's Core function with its
// single GM, the mass applied once per target), so that only the work
// mapping differs.  Blocks hold 32 threads, or 64 when a leaf holds more
// than 32 particles.
#include "fwd_f32_common.cuh"

namespace psr {

template <int TM, int ACC, bool COUNT, bool EQM>
__global__ void __launch_bounds__(64) p2p_fwd_blk_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x;
    const unsigned esize = TM == TM_TAYLOR ? 32u : TM == TM_CUBIC ? 16u : 8u;
    const size_t tab_bytes = TM == TM_EXACT ? 0 : (size_t)(a.table_n + 1) * esize;
    float4* sj = reinterpret_cast<float4*>(smem + ((tab_bytes + 15) & ~(size_t)15));
    if (TM == TM_TAYLOR) {
        const float4* g = reinterpret_cast<const float4*>(a.table);
        for (int i = t; i < 2 * (a.table_n + 1); i += blockDim.x)
            reinterpret_cast<float4*>(smem)[i] = g[i];
    } else if (TM != TM_EXACT) {
        const float4* g = reinterpret_cast<const float4*>(a.table);
        for (int i = t; i <= a.table_n; i += blockDim.x) {
            const float4 v = g[i];
            if (TM == TM_LINEAR)
                reinterpret_cast<float2*>(smem)[i] = make_float2(v.z, v.y * (float)a.table_n);
            else
                reinterpret_cast<float4*>(smem)[i] = v;
        }
    }
    __syncthreads();
    const unsigned tab_bias = smem_u32(smem) - (unsigned)kMagicBits * esize;
    const float4* __restrict__ pf = reinterpret_cast<const float4*>(a.pf);
    const int4* __restrict__ leaf = reinterpret_cast<const int4*>(a.leaf);
    const int4* __restrict__ lcen = reinterpret_cast<const int4*>(a.lcen);
    unsigned long long npairs = 0, nev = 0;
    for (long long b = blockIdx.x;; b += gridDim.x) {
        const long long it = b * a.item_stride + a.item_offset;
        if (it >= a.n_items) break;
        const int I = a.items[it];
        if (I < 0 || I >= a.n_leaves) {
            if (t == 0) set_error(a.ctrl, kErrItemIndex);
            continue;
        }
        const int4 li = leaf[I];
        if (li.y <= 0 || li.y > a.max_leaf || li.y > (int)blockDim.x ||
            (long long)li.x + li.y > a.n || li.z < 0 || li.z >= a.nbox) {
            if (t == 0) set_error(a.ctrl, kErrParticleRange);
            continue;
        }
        const BoxDev& bx = a.boxes[li.z];
        const float x_c = bx.x_c;
        const float nmax = (float)a.table_n;
        const float soff = -0.5f / nmax;
        const float sc = TM == TM_EXACT ? 1.0f : TM == TM_LINEAR ? 1.0f / x_c : (float)a.table_n / x_c;
        const float xscale = 1.0f / sc;
        const float unit = bx.unit;
        const int4 ci = lcen[I];
        const bool act = t < li.y;
        float4 xi = pf[li.x + (act ? t : 0)];
        xi.x *= sc;
        xi.y *= sc;
        xi.z *= sc;
        Acc3<ACC> acc;
        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
        const float eps2 = kEps2 * sc * sc;
        int since = 0;
        unsigned cnt = 0;
        const long long re = a.rowptr[I + 1];
        for (long long e = a.rowptr[I]; e < re; ++e) {
            const unsigned ent = a.pairs[e];
            const int J = (int)(ent >> 5);
            const unsigned code = ent & 31u;
            bool ok = J < a.n_leaves && code < (unsigned)kShiftCodes;
            int4 lj = make_int4(0, 0, 0, 0);
            if (ok) {
                lj = leaf[J];
                ok = lj.x >= 0 && lj.y >= 1 && lj.y <= a.max_leaf && lj.y <= (int)blockDim.x &&
                     (long long)lj.x + lj.y <= a.n;
            }
            if (!ok) {  // the same entry for every thread: the block skips it together
                if (t == 0) set_error(a.ctrl, kErrLeafIndex);
                continue;
            }
            const int4 cj = lcen[J];
            int nx, ny, nz;
            decode_shift(code, nx, ny, nz);
            const float ox = (float)(cj.x - ci.x + nx * (1 << kCentreShift)) * unit * sc;
            const float oy = (float)(cj.y - ci.y + ny * (1 << kCentreShift)) * unit * sc;
            const float oz = (float)(cj.z - ci.z + nz * (1 << kCentreShift)) * unit * sc;
            __syncthreads();  // the previous source leaf has been read
            if (t < lj.y) {
                const float4 v = __ldg(pf + lj.x + t);
                sj[t] = make_float4(fmaf(v.x, sc, ox), fmaf(v.y, sc, oy), fmaf(v.z, sc, oz), v.w);
            }
            __syncthreads();
            if (act) {
                for (int k = 0; k < lj.y; ++k) {
                    const float4 p = sj[k];
                    const float dx = p.x - xi.x, dy = p.y - xi.y, dz = p.z - xi.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    const float rinv = rsqrt_ftz(r2);
                    const float tt = TM == TM_LINEAR ? fma_sat(r2, rinv, soff)
                                                     : fmaf(r2, rinv, TM == TM_TAYLOR ? 0.0f : -0.5f);
                    const float Tv = eval_T1<TM>(tt, r2, rinv, tab_bias, nmax, x_c, xscale);
                    const float w = EQM ? Tv * rinv * rinv * rinv : p.w * Tv * rinv * rinv * rinv;
                    fx = fmaf(w, dx, fx);
                    fy = fmaf(w, dy, fy);
                    fz = fmaf(w, dz, fz);
                    if (COUNT) {
                        const float u = r2 * rinv;
                        const float uc = TM == TM_EXACT ? x_c : TM == TM_LINEAR ? 1.0f : nmax;
                        cnt += (u < uc && (dx != 0.0f || dy != 0.0f || dz != 0.0f));
                    }
                }
                since += lj.y;
                if (COUNT) nev += (unsigned)lj.y;
                if (since >= a.fold_every) {
                    acc.fold(fx, fy, fz);
                    since = 0;
                }
            }
        }
        if (act) {
            acc.fold(fx, fy, fz);
            const float gout = bx.g_acc * sc * sc * (EQM ? bx.m_eq : 1.0f);
            float* out = reinterpret_cast<float*>(a.out) + 3LL * a.perm[li.x + t];
            if (ACC == PSR_ACC_FP64) {
                out[0] = (float)(acc.x * (double)gout);
                out[1] = (float)(acc.y * (double)gout);
                out[2] = (float)(acc.z * (double)gout);
            } else {
                out[0] = (acc.sx + acc.cx) * gout;
                out[1] = (acc.sy + acc.cy) * gout;
                out[2] = (acc.sz + acc.cz) * gout;
            }
        }
        if (COUNT) npairs += cnt;
    }
    if (COUNT && npairs)
        atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlPairsLo), npairs);
    if (COUNT && nev)
        atomicAdd(reinterpret_cast<unsigned long long*>(a.ctrl + kCtrlEvalLo), nev);
}

namespace {

size_t blk_smem(int precision, int interp, int table_n, int threads)
{
    const size_t tab = precision != PSR_FP32_TABLE ? 0 : (size_t)(table_n + 1) * table_entry_bytes(interp);
    return ((tab + 15) & ~(size_t)15) + (size_t)threads * 16;
}

template <int TM, int ACC, bool COUNT, bool EQM>
int launch_t(const FwdArgs& a, size_t smem, int threads, cudaStream_t st)
{
    auto k = p2p_fwd_blk_kernel<TM, ACC, COUNT, EQM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    k<<<a.blocks, threads, smem, st>>>(a);
    return (int)cudaGetLastError();
}

template <int TM, int ACC>
int launch_c(const FwdArgs& a, size_t smem, int threads, cudaStream_t st)
{
    return a.count_pairs  ? launch_t<TM, ACC, true, false>(a, smem, threads, st)
           : a.equal_mass ? launch_t<TM, ACC, false, true>(a, smem, threads, st)
                          : launch_t<TM, ACC, false, false>(a, smem, threads, st);
}

template <int TM, int ACC>
const void* ptr_c() { return (const void*)p2p_fwd_blk_kernel<TM, ACC, false, false>; }

int pick_tm(int precision, int interp)
{
    if (precision == PSR_FP32_EXACT) return TM_EXACT;
    if (interp == PSR_LINEAR) return TM_LINEAR;
    if (interp == PSR_TAYLOR2 || interp == PSR_TAYLOR4) return TM_TAYLOR;
    return TM_CUBIC;
}

}  // namespace

int blk_threads(int max_leaf) { return max_leaf > 32 ? 64 : 32; }

int launch_fwd_blk(const FwdArgs& a, int precision, void* stream)
{
    const int threads = blk_threads(a.max_leaf);
    const size_t smem = blk_smem(precision, a.interp, a.table_n, threads);
    cudaStream_t st = (cudaStream_t)stream;
    const bool f64 = a.accum == PSR_ACC_FP64;
    switch (pick_tm(precision, a.interp)) {
        case TM_EXACT:
            return f64 ? launch_c<TM_EXACT, PSR_ACC_FP64>(a, smem, threads, st)
                       : launch_c<TM_EXACT, PSR_ACC_KAHAN32>(a, smem, threads, st);
        case TM_LINEAR:
            return f64 ? launch_c<TM_LINEAR, PSR_ACC_FP64>(a, smem, threads, st)
                       : launch_c<TM_LINEAR, PSR_ACC_KAHAN32>(a, smem, threads, st);
        case TM_TAYLOR:
            return f64 ? launch_c<TM_TAYLOR, PSR_ACC_FP64>(a, smem, threads, st)
                       : launch_c<TM_TAYLOR, PSR_ACC_KAHAN32>(a, smem, threads, st);
        default:
            return f64 ? launch_c<TM_CUBIC, PSR_ACC_FP64>(a, smem, threads, st)
                       : launch_c<TM_CUBIC, PSR_ACC_KAHAN32>(a, smem, threads, st);
    }
}

int fwd_blk_occupancy(int precision, int interp, int accum, int max_leaf, int table_n, int* out)
{
    const int threads = blk_threads(max_leaf);
    const size_t smem = blk_smem(precision, interp, table_n, threads);
    const bool f64 = accum == PSR_ACC_FP64;
    const void* f;
    switch (pick_tm(precision, interp)) {
        case TM_EXACT: f = f64 ? ptr_c<TM_EXACT, PSR_ACC_FP64>() : ptr_c<TM_EXACT, PSR_ACC_KAHAN32>(); break;
        case TM_LINEAR: f = f64 ? ptr_c<TM_LINEAR, PSR_ACC_FP64>() : ptr_c<TM_LINEAR, PSR_ACC_KAHAN32>(); break;
        case TM_TAYLOR: f = f64 ? ptr_c<TM_TAYLOR, PSR_ACC_FP64>() : ptr_c<TM_TAYLOR, PSR_ACC_KAHAN32>(); break;
        default: f = f64 ? ptr_c<TM_CUBIC, PSR_ACC_FP64>() : ptr_c<TM_CUBIC, PSR_ACC_KAHAN32>(); break;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, threads, smem);
}

}  // namespace psr
