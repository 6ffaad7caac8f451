// C ABI of libpsr (declared in include/psr.h): argument checks, workspace
// upload, table caching and kernel launches.  No device allocation happens
// here; psr_p2p_forces and psr_p2p_adjoint only enqueue work.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>

#include "psr_internal.h"

using namespace psr;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(PSR_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Poll the stream until it is idle or timeout_ms has passed.
int wait_stream(cudaStream_t st, int timeout_ms)
{
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return PSR_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaStreamQuery");
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > timeout_ms) return fail(PSR_E_TIMEOUT, "stream did not finish within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

struct Opts {
    int precision, table_n, interp, accum, warps, bps, fold, count, kernel, tile, nshard, shard;
};

int check_opts(const psr_opts* o, Opts* out)
{
    psr_opts d{};
    d.precision = PSR_FP32_TABLE;
    if (!o) o = &d;
    for (int i = 0; i < 4; ++i)
        if (o->reserved[i] != 0) return fail(PSR_E_ARG, "psr_opts.reserved must be zero");
    const int nshard = o->shard_count > 1 ? o->shard_count : 1;
    if (o->shard_count < 0 || o->shard_index < 0 || o->shard_index >= nshard)
        return fail(PSR_E_ARG, "psr_opts.shard_index must be in [0, shard_count)");
    if (o->source_tile != 0 && o->source_tile != 64 && o->source_tile != 128 &&
        o->source_tile != 256)
        return fail(PSR_E_ARG, "psr_opts.source_tile must be 0, 64, 128 or 256");
    if (o->kernel < PSR_KERNEL_AUTO || o->kernel > PSR_KERNEL_PAPER)
        return fail(PSR_E_ARG, "psr_opts.kernel out of range");
    if (o->precision < PSR_FP64 || o->precision > PSR_FP32_TABLE)
        return fail(PSR_E_ARG, "psr_opts.precision out of range");
    if (o->interp < PSR_LINEAR || o->interp > PSR_TAYLOR4)
        return fail(PSR_E_ARG, "psr_opts.interp out of range");
    const bool taylor = o->interp == PSR_TAYLOR2 || o->interp == PSR_TAYLOR4;
    int tn = o->table_n ? o->table_n : (taylor ? kTaylorPaperN : 1024);
    if (taylor && (tn < 64 || tn > kMaxTaylorN))
        return fail(PSR_E_ARG, "psr_opts.table_n must be in [64, 2048] for the Taylor tables");
    if (!taylor && (tn < 64 || tn > kMaxTableN || (tn & (tn - 1))))
        return fail(PSR_E_ARG, "psr_opts.table_n must be a power of two in [64, 8192]");
    if (o->accum != PSR_ACC_FP64 && o->accum != PSR_ACC_KAHAN32)
        return fail(PSR_E_ARG, "psr_opts.accum out of range");
    int w = o->warps_per_block;
    if (w < 0 || w > 32) return fail(PSR_E_ARG, "psr_opts.warps_per_block must be in [0, 32]");
    if (o->blocks_per_sm < 0 || o->blocks_per_sm > 64)
        return fail(PSR_E_ARG, "psr_opts.blocks_per_sm must be in [0, 64]");
    int fold = o->fold_every ? o->fold_every : 64;
    if (fold < 1) return fail(PSR_E_ARG, "psr_opts.fold_every must be positive");
    *out = Opts{o->precision, tn, o->interp, o->accum, w, o->blocks_per_sm, fold,
                o->count_pairs ? 1 : 0, o->kernel == PSR_KERNEL_AUTO ? PSR_KERNEL_SCALAR : o->kernel,
                o->source_tile, nshard, o->shard_index};
    return PSR_OK;
}

// Warps per block: every kernel is built for at most 256 threads (8 warps).
int resolve_warps(Opts& o, bool fwd32)
{
    (void)fwd32;
    if (o.warps == 0) o.warps = 8;
    if (o.warps > 8) return fail(PSR_E_ARG, "warps_per_block must be in [1, 8]");
    return PSR_OK;
}

constexpr int kAdjStageCap = 128;  // adjoint staged particles per warp (2 float4 each)

// Staging capacity per warp; the table and the staging buffers must fit in one
// block's shared memory.
int fwd32_smem_config(const Opts& o, int* cap)
{
    *cap = o.tile ? o.tile : 256;
    if (fwd_f32_smem(o.precision, o.interp, o.table_n, o.warps, *cap) > kSmemPerBlock)
        return fail(PSR_E_ARG, "table and staging buffers exceed shared memory; use fewer warps");
    return PSR_OK;
}

// A staged chunk always holds at least one whole leaf.
int check_tile(const Leaves* h, int cap)
{
    if (cap < h->max_leaf)
        return fail(PSR_E_ARG, "source_tile " + std::to_string(cap) + " is below the largest leaf (" +
                                   std::to_string(h->max_leaf) + " particles)");
    return PSR_OK;
}

FwdArgs base_args(Leaves* h, const Opts& o)
{
    FwdArgs a{};
    char* w = h->d_ws;
    const Layout& L = h->lay;
    a.pf = w + L.pf;
    a.pd = h->has_pd ? w + L.pd : nullptr;
    a.perm = reinterpret_cast<const int32_t*>(w + L.perm);
    a.leaf = reinterpret_cast<const int32_t*>(w + L.leaf);
    a.lcen = reinterpret_cast<const int32_t*>(w + L.lcen);
    a.rowptr = reinterpret_cast<const int64_t*>(w + L.rowptr);
    a.pairs = reinterpret_cast<const uint32_t*>(w + L.pairs);
    a.items = reinterpret_cast<const int32_t*>(w + L.items);
    a.boxes = reinterpret_cast<const BoxDev*>(w + L.boxes);
    a.table = w + L.table;
    a.ctrl = reinterpret_cast<unsigned*>(w + L.ctrl);
    a.cot_sorted = w + L.cotf;
    a.n = h->n;
    a.n_leaves = h->n_leaves;
    a.n_pairs = h->n_pairs;
    a.n_items = (int)h->n_leaves;
    a.nbox = h->nbox;
    a.table_n = o.table_n;
    a.interp = o.interp;
    a.accum = o.accum;
    a.fold_every = o.fold;
    a.count_pairs = o.count;
    a.warps_per_block = o.warps;
    a.max_leaf = h->max_leaf;
    a.variant = o.kernel;
    a.item_stride = o.nshard;
    a.item_offset = o.shard;
    a.equal_mass = h->equal_mass ? 1 : 0;
    return a;
}

bool fp64_taylor(const Opts& o)
{
    return o.precision == PSR_FP64 && (o.interp == PSR_TAYLOR2 || o.interp == PSR_TAYLOR4);
}

int ensure_table(Leaves* h, const Opts& o, cudaStream_t st)
{
    const bool t64 = fp64_taylor(o);
    if (o.precision != PSR_FP32_TABLE && !t64) return PSR_OK;
    const double x_c = h->boxes[0].r_c / (2.0 * h->boxes[0].r_s);
    int key = (o.table_n * 4 + o.interp) * 2 + (t64 ? 1 : 0);
    if (key == h->table_key && x_c == h->table_xc) return PSR_OK;
    char* t = h->d_ws + h->lay.table;
    int e = t64 ? launch_table64(o.table_n, o.interp, x_c, t, st)
                : launch_table(o.table_n, o.interp, x_c, t, t + (size_t)(kMaxTableN + 1) * 16, st);
    if (e) return cuda_fail((cudaError_t)e, "table kernel launch");
    h->table_key = key;
    h->table_xc = x_c;
    return PSR_OK;
}

int grid_blocks(Leaves* h, const Opts& o, int adjoint, int* blocks)
{
    int bps = o.bps;
    if (bps == 0) {
        int occ = 0, e;
        if (adjoint)
            e = adj_occupancy(o.precision, o.interp, o.accum, o.warps, h->max_leaf, o.table_n,
                              o.tile ? o.tile : kAdjStageCap, o.kernel, &occ);
        else if (o.precision == PSR_FP64)
            e = fwd_f64_occupancy(o.warps, h->max_leaf, o.interp, o.table_n, &occ);
        else if (o.kernel == PSR_KERNEL_PAPER)
            e = fwd_blk_occupancy(o.precision, o.interp, o.accum, h->max_leaf, o.table_n, &occ);
        else {
            int cap;
            if ((e = fwd32_smem_config(o, &cap))) return e;
            if ((e = check_tile(h, cap))) return e;
            e = fwd_f32_occupancy(o.precision, o.interp, o.accum, o.warps, h->max_leaf, o.table_n,
                                  cap, o.kernel, &occ);
        }
        if (e) return cuda_fail((cudaError_t)e, "occupancy query");
        bps = occ > 0 ? occ : 1;
    }
    *blocks = bps * (h->sm_count > 0 ? h->sm_count : 1);
    return PSR_OK;
}

}  // namespace

namespace psr {

// Helpers for the allocation-free entry point in noalloc.cu.
void set_last_error(const std::string& msg) { g_err = msg; }

int prepare_forward(Leaves* h, const psr_opts* opts, FwdArgs* a, int* precision)
{
    if (!h->uploaded) return fail(PSR_E_STATE, "psr_upload has not been called");
    Opts o;
    int rc = check_opts(opts, &o);
    if (rc) return rc;
    if (o.precision == PSR_FP64 && !h->has_pd)
        return fail(PSR_E_STATE, "built with PSR_BUILD_NO_FP64: no FP64 payload");
    const bool fwd32 = o.precision != PSR_FP64;
    if ((rc = resolve_warps(o, fwd32))) return rc;
    *a = base_args(h, o);
    if (fwd32 && (rc = fwd32_smem_config(o, &a->stage_cap))) return rc;
    if (fwd32 && (rc = check_tile(h, a->stage_cap))) return rc;
    if ((rc = grid_blocks(h, o, 0, &a->blocks))) return rc;
    *precision = o.precision;
    return PSR_OK;
}

}  // namespace psr

extern "C" {

const char* psr_last_error(void) { return g_err.c_str(); }

const char* psr_version(void) { return "psr 0.1 (sm_103a)"; }

int psr_build_leaves(const double* pos, const double* mass, int64_t n, const psr_box* box,
                     int max_leaf, int flags, psr_leaves** out)
{
    if (!box) return fail(PSR_E_ARG, "null box");
    const double* p[1] = {pos};
    const double* m[1] = {mass};
    int64_t nn[1] = {n};
    Leaves* h = nullptr;
    std::string err;
    int rc = build_batch(1, p, mass ? m : nullptr, nn, box, max_leaf, flags, &h, &err);
    if (rc) return fail(rc, err);
    *out = reinterpret_cast<psr_leaves*>(h);
    return PSR_OK;
}

int psr_build_leaves_batch(int nbox, const double* const* pos, const double* const* mass,
                           const int64_t* n, const psr_box* boxes, int max_leaf, int flags,
                           psr_leaves** out)
{
    Leaves* h = nullptr;
    std::string err;
    int rc = build_batch(nbox, pos, mass, n, boxes, max_leaf, flags, &h, &err);
    if (rc) return fail(rc, err);
    *out = reinterpret_cast<psr_leaves*>(h);
    return PSR_OK;
}

int psr_leaves_info(const psr_leaves* hh, psr_info* info)
{
    const Leaves* h = reinterpret_cast<const Leaves*>(hh);
    if (!h || !info) return fail(PSR_E_ARG, "null argument");
    std::memset(info, 0, sizeof *info);
    info->n = h->n;
    info->n_leaves = h->n_leaves;
    info->n_pairs = h->n_pairs;
    info->n_items = h->n_leaves;
    info->nbox = h->nbox;
    info->evaluated_pairs = h->evaluated;
    info->device_bytes = h->lay.total;
    info->max_leaf = h->max_leaf;
    info->max_row = h->max_row;
    info->build_seconds = h->build_seconds;
    info->perm = h->device_built ? nullptr : h->perm.data();
    info->n_far = h->n_far;
    info->theta = h->theta;
    info->rows_walked_twice = h->device_built ? h->db_uncached : 0;
    info->equal_mass = h->equal_mass ? 1 : 0;
    return PSR_OK;
}

int psr_upload(psr_leaves* hh, void* d_ws, size_t bytes, void* stream)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h) return fail(PSR_E_ARG, "null handle");
    if (h->device_built)
        return fail(PSR_E_STATE, "a device-built handle is written by psr_device_build_finish");
    if (!d_ws || bytes < h->lay.total || (reinterpret_cast<uintptr_t>(d_ws) & 255))
        return fail(PSR_E_WORKSPACE, "workspace must be 256-byte aligned and at least " +
                                         std::to_string(h->lay.total) + " bytes");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    char* w = static_cast<char*>(d_ws);
    const Layout& L = h->lay;
    struct Cp { size_t off; const void* src; size_t bytes; } cps[] = {
        {L.pf, h->pf.data(), h->pf.size() * sizeof(float)},
        {L.pd, h->pd.data(), h->pd.size() * sizeof(double)},
        {L.perm, h->perm32.data(), h->perm32.size() * sizeof(int32_t)},
        {L.leaf, h->leaf.data(), h->leaf.size() * sizeof(int32_t)},
        {L.lcen, h->lcen.data(), h->lcen.size() * sizeof(int32_t)},
        {L.rowptr, h->rowptr.data(), h->rowptr.size() * sizeof(int64_t)},
        {L.pairs, h->pairs.data(), h->pairs.size() * sizeof(uint32_t)},
        {L.items, h->items.data(), h->items.size() * sizeof(int32_t)},
        {L.boxes, h->boxdev.data(), h->boxdev.size() * sizeof(BoxDev)},
    };
    for (const Cp& c : cps) {
        if (!c.bytes) continue;
        if ((e = cudaMemcpyAsync(w + c.off, c.src, c.bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync (upload)");
    }
    if ((e = cudaMemsetAsync(w + L.ctrl, 0, kCtrlWords * 4, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync (ctrl)");
    h->d_ws = w;
    h->ws_bytes = bytes;
    h->uploaded = true;
    h->table_key = -1;
    h->table_xc = -1.0;
    h->sm_count = sms;
    h->device = dev;
    return PSR_OK;
}

int psr_p2p_forces(psr_leaves* hh, const psr_opts* opts, void* d_acc, void* stream)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h || (!d_acc && h->n > 0)) return fail(PSR_E_ARG, "null argument");
    if (!h->uploaded) return fail(PSR_E_STATE, "psr_upload has not been called");
    Opts o;
    int rc = check_opts(opts, &o);
    if (rc) return rc;
    if (h->n == 0) return PSR_OK;  // nothing to compute
    if (o.precision == PSR_FP64 && !h->has_pd)
        return fail(PSR_E_STATE, "built with PSR_BUILD_NO_FP64: no FP64 payload");
    cudaStream_t st = (cudaStream_t)stream;
    const bool fwd32 = o.precision != PSR_FP64;
    if ((rc = resolve_warps(o, fwd32))) return rc;
    if ((rc = ensure_table(h, o, st))) return rc;
    FwdArgs a = base_args(h, o);
    a.out = d_acc;
    if (fwd32 && (rc = fwd32_smem_config(o, &a.stage_cap))) return rc;
    if (fwd32 && (rc = check_tile(h, a.stage_cap))) return rc;
    if ((rc = grid_blocks(h, o, 0, &a.blocks))) return rc;
    if (o.count) {
        cudaError_t e = cudaMemsetAsync(a.ctrl + kCtrlPairsLo, 0, 16, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (pair counters)");
    }
    int e = (o.precision == PSR_FP64)          ? launch_fwd_f64(a, st)
            : (o.kernel == PSR_KERNEL_PAPER) ? launch_fwd_blk(a, o.precision, st)
                                             : launch_fwd_f32(a, o.precision, st);
    if (e) return cuda_fail((cudaError_t)e, "forward kernel launch");
    return PSR_OK;
}

int psr_p2p_adjoint(psr_leaves* hh, const psr_opts* opts, const void* d_cot, void* d_grad_pos,
                    void* d_grad_mass, void* stream)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h || ((!d_cot || !d_grad_pos) && h->n > 0)) return fail(PSR_E_ARG, "null argument");
    if (!h->uploaded) return fail(PSR_E_STATE, "psr_upload has not been called");
    Opts o;
    int rc = check_opts(opts, &o);
    if (rc) return rc;
    if (o.precision == PSR_FP32_TABLE && o.interp != PSR_LINEAR && o.interp != PSR_CUBIC)
        return fail(PSR_E_ARG, "the adjoint takes PSR_LINEAR or PSR_CUBIC tables");
    if (fp64_taylor(o))
        return fail(PSR_E_ARG, "the FP64 Taylor table path is forward-only (the FP64 adjoint is plain)");
    if (h->n == 0) return PSR_OK;  // nothing to compute
    if (o.precision == PSR_FP64 && !h->has_pd)
        return fail(PSR_E_STATE, "built with PSR_BUILD_NO_FP64: no FP64 payload");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = resolve_warps(o, false))) return rc;
    if ((rc = ensure_table(h, o, st))) return rc;
    FwdArgs a = base_args(h, o);
    a.cot = d_cot;
    a.stage_cap = o.tile ? o.tile : kAdjStageCap;
    if (o.precision != PSR_FP64 && (rc = check_tile(h, a.stage_cap))) return rc;
    if (o.precision != PSR_FP64 &&
        adj_f32_smem(o.precision, o.interp, o.table_n, o.warps, a.stage_cap) > kSmemPerBlock)
        return fail(PSR_E_ARG, "adjoint table and staging buffers exceed shared memory; "
                               "use fewer warps or a smaller table");
    a.out = d_grad_pos;
    a.out_m = d_grad_mass;
    if ((rc = grid_blocks(h, o, 1, &a.blocks))) return rc;
    int e = (o.precision == PSR_FP64) ? launch_adj_f64(a, st) : launch_adj_f32(a, o.precision, st);
    if (e) return cuda_fail((cudaError_t)e, "adjoint kernel launch");
    return PSR_OK;
}

int psr_autotune(psr_leaves* hh, const psr_opts* base, void* d_acc, void* stream, int reps,
                 int timeout_ms, psr_opts* best, float* best_ms)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h || !d_acc || !best) return fail(PSR_E_ARG, "null argument");
    if (!h->uploaded) return fail(PSR_E_STATE, "psr_upload has not been called");
    if (reps < 1) return fail(PSR_E_ARG, "reps must be >= 1");
    psr_opts b{};
    if (base) b = *base;
    else b.precision = PSR_FP32_TABLE;
    Opts chk;
    int rc = check_opts(&b, &chk);
    if (rc) return rc;
    if (b.precision == PSR_FP64) return fail(PSR_E_ARG, "the autotuner covers the FP32 kernels");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce;
    if ((ce = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(ce, "cudaEventCreate");
    if ((ce = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    float best_t = -1.0f;
    psr_opts best_o = b;
    const int kernels[2] = {PSR_KERNEL_SCALAR, PSR_KERNEL_PACKED};
    const int warps[2] = {4, 8};
    const int tiles[3] = {64, 128, 256};
    for (int ki = 0; ki < 2 && rc == PSR_OK; ++ki)
        for (int wi = 0; wi < 2 && rc == PSR_OK; ++wi)
            for (int ti = 0; ti < 3 && rc == PSR_OK; ++ti) {
                psr_opts c = b;
                c.kernel = kernels[ki];
                c.warps_per_block = warps[wi];
                c.source_tile = tiles[ti];
                c.count_pairs = 0;
                if (tiles[ti] < h->max_leaf) continue;
                Opts oc;
                if (check_opts(&c, &oc) != PSR_OK) continue;
                if (fwd_f32_smem(oc.precision, oc.interp, oc.table_n, warps[wi], tiles[ti]) >
                    kSmemPerBlock)
                    continue;
                if ((rc = psr_p2p_forces(hh, &c, d_acc, stream))) break;  // warm-up
                float tmin = -1.0f;
                for (int r = 0; r < reps && rc == PSR_OK; ++r) {
                    if ((ce = cudaEventRecord(e0, st)) != cudaSuccess) { rc = cuda_fail(ce, "cudaEventRecord"); break; }
                    if ((rc = psr_p2p_forces(hh, &c, d_acc, stream))) break;
                    if ((ce = cudaEventRecord(e1, st)) != cudaSuccess) { rc = cuda_fail(ce, "cudaEventRecord"); break; }
                    if ((rc = wait_stream(st, timeout_ms))) break;
                    float ms = 0.0f;
                    if ((ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) { rc = cuda_fail(ce, "cudaEventElapsedTime"); break; }
                    if (tmin < 0.0f || ms < tmin) tmin = ms;
                }
                if (rc == PSR_OK && tmin >= 0.0f && (best_t < 0.0f || tmin < best_t)) {
                    best_t = tmin;
                    best_o = c;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best_t < 0.0f) return fail(PSR_E_ARG, "no candidate tile shape fits this leaf set");
    *best = best_o;
    if (best_ms) *best_ms = best_t;
    return PSR_OK;
}

// ------------------------------------------------------- FP32 FMA rate --
// Every thread runs kPeakChains independent chains x <- x a + b for iters x
// kPeakUnroll steps and stores their sum; with a just below one the chains
// settle near b / (1 - a) and stay normal.
namespace {
constexpr int kPeakChains = 8, kPeakUnroll = 8, kPeakThreads = 256, kPeakBlocksPerSm = 4;
}

__global__ void __launch_bounds__(kPeakThreads) fp32_peak_kernel(float* __restrict__ sink, int iters,
                                                                 float a, float b)
{
    float x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = 1.0f + 1e-3f * (float)(c + (threadIdx.x & 7));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int psr_fp32_peak(void* d_sink, size_t sink_bytes, int iters, int launches, void* stream,
                  int timeout_ms, double* flops_per_s)
{
    if (!d_sink || !flops_per_s) return fail(PSR_E_ARG, "null argument");
    if (iters < 1 || launches < 1) return fail(PSR_E_ARG, "iters and launches must be >= 1");
    int dev = 0, sms = 0;
    cudaError_t ce;
    if ((ce = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    if ((ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(ce, "cudaDeviceGetAttribute");
    const int blocks = sms * kPeakBlocksPerSm;
    const size_t need = (size_t)blocks * kPeakThreads * sizeof(float);
    if (sink_bytes < need)
        return fail(PSR_E_ARG, "the sink must hold " + std::to_string(need) + " bytes on this device");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((ce = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(ce, "cudaEventCreate");
    if ((ce = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    int rc = PSR_OK;
    float best = -1.0f;
    for (int l = 0; l < launches && rc == PSR_OK; ++l) {
        if ((ce = cudaEventRecord(e0, st)) != cudaSuccess) { rc = cuda_fail(ce, "cudaEventRecord"); break; }
        fp32_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(reinterpret_cast<float*>(d_sink), iters,
                                                           0.9999f, 1.0e-4f);
        if ((ce = cudaGetLastError()) != cudaSuccess) { rc = cuda_fail(ce, "FP32 peak kernel launch"); break; }
        if ((ce = cudaEventRecord(e1, st)) != cudaSuccess) { rc = cuda_fail(ce, "cudaEventRecord"); break; }
        if ((rc = wait_stream(st, timeout_ms))) break;
        float ms = 0.0f;
        if ((ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) { rc = cuda_fail(ce, "cudaEventElapsedTime"); break; }
        if (best < 0.0f || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *flops_per_s = 2.0 * kPeakChains * kPeakUnroll * (double)iters * (double)blocks * kPeakThreads /
                   ((double)best * 1e-3);
    return PSR_OK;
}

static int read_counter(psr_leaves* hh, void* stream, int timeout_ms, int word, int64_t* count)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h || !count) return fail(PSR_E_ARG, "null argument");
    if (!h->uploaded) return fail(PSR_E_STATE, "psr_upload has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = wait_stream(st, timeout_ms);
    if (rc) return rc;
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->d_ws + h->lay.ctrl + word * 4, 8,
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (pair counter)");
    if ((rc = wait_stream(st, timeout_ms))) return rc;
    *count = (int64_t)v;
    return PSR_OK;
}

int psr_pair_count(psr_leaves* hh, void* stream, int timeout_ms, int64_t* count)
{
    return read_counter(hh, stream, timeout_ms, kCtrlPairsLo, count);
}

int psr_evaluated_count(psr_leaves* hh, void* stream, int timeout_ms, int64_t* count)
{
    return read_counter(hh, stream, timeout_ms, kCtrlEvalLo, count);
}

int psr_check(psr_leaves* hh, void* stream, int timeout_ms)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h) return fail(PSR_E_ARG, "null handle");
    if (!h->uploaded) return fail(PSR_E_STATE, "psr_upload has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = wait_stream(st, timeout_ms);
    if (rc) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    unsigned v = 0;
    e = cudaMemcpyAsync(&v, h->d_ws + h->lay.ctrl + kCtrlError * 4, 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (error word)");
    if ((rc = wait_stream(st, timeout_ms))) return rc;
    if (v) {
        e = cudaMemsetAsync(h->d_ws + h->lay.ctrl + kCtrlError * 4, 0, 4, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (error word)");
        if ((rc = wait_stream(st, timeout_ms))) return rc;
        return fail(PSR_E_DEVICE, "device bounds check failed, error bits 0x" + std::to_string(v));
    }
    return PSR_OK;
}

int psr_table(int table_n, int interp, double x_c, void* d_out, void* stream)
{
    if (!d_out) return fail(PSR_E_ARG, "null output");
    if (interp < PSR_LINEAR || interp > PSR_TAYLOR4) return fail(PSR_E_ARG, "interp out of range");
    if (interp >= PSR_TAYLOR2 && (table_n < 64 || table_n > kMaxTaylorN))
        return fail(PSR_E_ARG, "table_n must be in [64, 2048] for the Taylor tables");
    if (interp < PSR_TAYLOR2 && (table_n < 64 || table_n > kMaxTableN || (table_n & (table_n - 1))))
        return fail(PSR_E_ARG, "table_n must be a power of two in [64, 8192]");
    if (!(x_c > 0) || !std::isfinite(x_c)) return fail(PSR_E_ARG, "x_c must be positive");
    int e = launch_table(table_n, interp, x_c, d_out, nullptr, stream);
    if (e) return cuda_fail((cudaError_t)e, "table kernel launch");
    return PSR_OK;
}

int psr_leaves_host_arrays(const psr_leaves* hh, psr_host_arrays* out)
{
    const Leaves* h = reinterpret_cast<const Leaves*>(hh);
    if (!h || !out) return fail(PSR_E_ARG, "null argument");
    if (h->device_built) return fail(PSR_E_STATE, "a device-built handle has no host arrays");
    out->pf = h->pf.data();
    out->pd = !h->has_pd ? nullptr : h->pd.data();
    out->leaf = h->leaf.data();
    out->lcen = h->lcen.data();
    out->rowptr = h->rowptr.data();
    out->pairs = h->pairs.data();
    out->items = h->items.data();
    return PSR_OK;
}

int psr_leaves_regions(const psr_leaves* hh, psr_regions* out)
{
    const Leaves* h = reinterpret_cast<const Leaves*>(hh);
    if (!h || !out) return fail(PSR_E_ARG, "null argument");
    const Layout& L = h->lay;
    out->pf = L.pf;
    out->pd = L.pd;
    out->perm = L.perm;
    out->leaf = L.leaf;
    out->lcen = L.lcen;
    out->rowptr = L.rowptr;
    out->pairs = L.pairs;
    out->items = L.items;
    out->frow = L.frow;
    out->fpairs = L.fpairs;
    out->fcen = L.fcen;
    out->fofs = L.fofs;
    out->total = L.total;
    return PSR_OK;
}

void psr_free_leaves(psr_leaves* hh) { delete reinterpret_cast<Leaves*>(hh); }

}  // extern "C"
