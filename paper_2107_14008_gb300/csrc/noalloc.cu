// psr_p2p_forces_noalloc: the forward P2P launch of psr_p2p_forces for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc, or any routine that allocates: code
// running inside a memory pool or arena owned by a host framework, inside a
// real-time or interrupt-like context where allocation may block, or under a
// policy that forbids allocations after start-up.  They can still pass device
// buffers that already exist: the leaf set uploaded with psr_upload (the
// inputs) and the acceleration array (the output).  This entry point takes
// exactly those; the kernel's scratch memory - the persistent scheduler's work
// counters and error word, and the interpolation table - lives in one
// file-scope __device__ array of fixed size instead of in the caller's
// workspace.  No call allocates through the runtime (no cudaMalloc, no
// allocating library routine).  The first call on each device is the set-up:
// it looks up the array's address (scratch_address below), and under CUDA's
// default lazy module loading that look-up loads the module holding the array,
// whose storage the driver allocates then; callers that cannot allow that
// make one call per device at start-up, before any stream capture.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "psr_internal.h"

namespace psr {
void set_last_error(const std::string& msg);
int prepare_forward(Leaves* h, const psr_opts* opts, FwdArgs* a, int* precision);
}  // namespace psr

using namespace psr;

namespace {

// Largest table the scratch array holds: 4096 intervals (cubic entries are
// 16 bytes, plus the zero sentinel).
constexpr int kNoAllocMaxTableN = 4096;
constexpr size_t kTableBytes = (((size_t)kNoAllocMaxTableN + 1) * 16 + 255) & ~(size_t)255;
constexpr size_t kCtrlBytes = (size_t)kCtrlWords * 4;
constexpr size_t kScratchBytes = kTableBytes + kCtrlBytes;  // 66,048 bytes

// The scratch array: one copy per device that loads the library, kept until
// the process exits.  Every call on a device shares it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host code cannot use g_scratch's name as a device address (in host code it
// names a host-side stand-in).  The address is looked up once per device,
// with that device current, and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return PSR_E_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("device index out of range for the scratch address cache");
        return PSR_E_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error(std::string("cudaGetSymbolAddress (scratch): ") + cudaGetErrorString(e));
            return PSR_E_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PSR_OK;
}

}  // namespace

extern "C" int psr_p2p_forces_noalloc(psr_leaves* hh, const psr_opts* opts, void* d_acc,
                                      void* stream)
{
    Leaves* h = reinterpret_cast<Leaves*>(hh);
    if (!h || !d_acc) {
        set_last_error("null argument");
        return PSR_E_ARG;
    }
    FwdArgs a;
    int precision = 0;
    int rc = prepare_forward(h, opts, &a, &precision);
    if (rc) return rc;
    if (precision == PSR_FP64 && (a.interp == PSR_TAYLOR2 || a.interp == PSR_TAYLOR4)) {
        set_last_error("psr_p2p_forces_noalloc: the FP64 Taylor table path needs the workspace's "
                       "table (use psr_p2p_forces)");
        return PSR_E_ARG;
    }
    if (precision == PSR_FP32_TABLE &&
        (size_t)(a.table_n + 1) * (a.interp == PSR_LINEAR || a.interp == PSR_CUBIC ? 16 : 32) >
            kTableBytes) {
        set_last_error("psr_p2p_forces_noalloc: a table of " + std::to_string(a.table_n) +
                       " intervals exceeds its fixed scratch array (4096 intervals; every "
                       "Taylor table fits)");
        return PSR_E_ARG;
    }
    void* scratch = nullptr;
    if ((rc = scratch_address(&scratch))) return rc;
    unsigned char* base = static_cast<unsigned char*>(scratch);
    cudaStream_t st = (cudaStream_t)stream;
    a.table = base;
    a.ctrl = reinterpret_cast<unsigned*>(base + kTableBytes);
    a.out = d_acc;
    // the work counters must start at zero; the array keeps the last call's values
    cudaError_t e = cudaMemsetAsync(a.ctrl, 0, kCtrlBytes, st);
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaMemsetAsync (scratch counters): ") + cudaGetErrorString(e));
        return PSR_E_CUDA;
    }
    if (precision == PSR_FP32_TABLE) {
        const double x_c = h->boxes[0].r_c / (2.0 * h->boxes[0].r_s);
        int le = launch_table(a.table_n, a.interp, x_c, base, nullptr, st);
        if (le) {
            set_last_error(std::string("table kernel launch: ") + cudaGetErrorString((cudaError_t)le));
            return PSR_E_CUDA;
        }
    }
    int le = precision == PSR_FP64              ? launch_fwd_f64(a, st)
             : a.variant == PSR_KERNEL_PAPER ? launch_fwd_blk(a, precision, st)
                                             : launch_fwd_f32(a, precision, st);
    if (le) {
        set_last_error(std::string("forward kernel launch: ") + cudaGetErrorString((cudaError_t)le));
        return PSR_E_CUDA;
    }
    return PSR_OK;
}
