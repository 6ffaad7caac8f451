// Internal declarations shared by the host builder, the C ABI and the CUDA
// kernels of libpsr.  Not part of the public ABI (see include/psr.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "psr.h"

namespace psr {

// Positions are quantised to 21 bits per axis for the Morton order; leaf-cell
// centres are integers in units of L / 2^22 (a cell of level l and index i has
// its centre at (2i + 1) 2^(21 - l)), so centre differences, with a periodic
// shift of n * 2^22, are integers below 2^24 in magnitude and convert to FP32
// exactly.
constexpr int kMortonBits = 21;
constexpr int kCentreShift = 22;
constexpr int kMaxLeaf = 64;
constexpr int kShiftCodes = 27;  // (nx+1)*9 + (ny+1)*3 + (nz+1)
constexpr int kMaxTableN = 8192;
constexpr int kMaxTaylorN = 2048;    // Taylor tables: 32-byte entries
constexpr int kTaylorPaperN = 384;   // x_c / 384 = 3 / 512 at x_c = 2.25, the paper's spacing

// Per-box constants as the kernels see them (plain old data, 16B aligned).
struct alignas(16) BoxDev {
    double L, r_s, r_c, G;      // FP64 path
    double rc2, inv_2rs, pad0, pad1;
    float unit;     // (L / 2^22) / (2 r_s): centre units -> FP32 coordinate units
    float x_c;      // r_c / (2 r_s): cutoff in FP32 coordinate units (= x)
    float x_c2;     // x_c^2
    float g_acc;    // G / (2 r_s)^2: FP32 coordinate sums -> acceleration
    float g_adj;    // G / (8 r_s^3): adjoint position gradient factor
    float g_adjm;   // G / (4 r_s^2): adjoint mass gradient factor
    float m_eq;     // the mass every particle of the box has (as FP32), 0 if they differ
    float pad3;
};
static_assert(sizeof(BoxDev) == 96, "BoxDev layout");

// Byte offsets of the regions of the device workspace (256-byte aligned).
struct Layout {
    size_t pf;       // float4[n]    FP32 leaf-local coords / (2 r_s), mass
    size_t pd;       // double4[n]   FP64 wrapped coords, mass (optional)
    size_t perm;     // int32[n]     sorted -> original
    size_t leaf;     // int4[nl]     first, count, box, pad
    size_t lcen;     // int4[nl]     centre x, y, z (units L/2^22), level
    size_t rowptr;   // int64[nl+1]  CSR of pair entries by target leaf
    size_t pairs;    // uint32[np]   (source leaf << 5) | shift code
    size_t items;    // int32[nl]    target leaves in schedule order
    size_t boxes;    // BoxDev[nbox]
    size_t table;    // float4[2 * (kMaxTableN + 1)]: T table, then exp(-x^2)
    size_t cotf;     // float4[n] / double4[n] adjoint source payload scratch
    size_t ctrl;     // uint32[64]  scheduler tickets, error word, counters
    // multipole split (device builds with an acceptance parameter only)
    size_t frow;     // int64[nl+1]  CSR of well-separated (M2L) entries by target leaf
    size_t fpairs;   // uint32[nf]   (source leaf << 5) | shift code
    size_t fcen;     // double4[nl]  expansion centre (particle box centre), radius
    size_t fofs;     // float4[nl]   that centre minus the cell centre (lcen), radius
    size_t total;
};

// ctrl word indices
enum : int {
    kCtrlTicketFwd = 0,
    kCtrlDoneFwd = 1,
    kCtrlTicketAdj = 2,
    kCtrlDoneAdj = 3,
    kCtrlError = 8,
    kCtrlPairsLo = 16,  // uint64 at words 16..17: pairs within the cutoff
    kCtrlEvalLo = 18,   // uint64 at words 18..19: pairs evaluated
    kCtrlWords = 64,
};
// error bits
enum : unsigned {
    kErrLeafIndex = 1u,
    kErrParticleRange = 2u,
    kErrItemIndex = 4u,
    kErrShiftCode = 8u,
};

struct Leaves {
    int nbox = 0;
    std::vector<psr_box> boxes;
    std::vector<BoxDev> boxdev;
    std::vector<int64_t> box_first;  // first particle of each box (original numbering)
    int64_t n = 0;
    int max_leaf_req = 0;
    int flags = 0;
    double build_seconds = 0.0;
    // sorted particles
    std::vector<float> pf;     // 4 per particle
    std::vector<double> pd;    // 4 per particle
    std::vector<int32_t> perm32;
    std::vector<int64_t> perm;
    // leaves
    std::vector<int32_t> leaf;  // 4 per leaf
    std::vector<int32_t> lcen;  // 4 per leaf
    std::vector<int64_t> rowptr;
    std::vector<uint32_t> pairs;
    std::vector<int32_t> items;
    int64_t evaluated = 0;
    int max_leaf = 0;
    int max_row = 0;
    // counts (set by both builders; a device-built handle has no host arrays)
    int64_t n_leaves = 0;
    int64_t n_pairs = 0;
    bool has_pd = false;        // FP64 payload present in the workspace
    bool device_built = false;  // arrays were built on the device
    bool equal_mass = false;    // in every box all particles share one mass (BoxDev::m_eq)
    bool has_far = false;       // pair list split into P2P (near) and M2L (far) entries
    double theta = 0.0;         //   multipole acceptance parameter of that split
    int64_t n_far = 0;          //   far entries
    char* db_scratch = nullptr; // device build between its two calls: the caller's scratch
    int64_t db_maxcost = 0;     //   and the largest per-leaf cost (schedule sort width)
    int db_kslot = 0;           //   runs per row in the pair cache (0: not used)
    int db_interleave = 0;      //   whether the walks take rows interleaved over warps
    int64_t db_uncached = 0;    //   and the rows it could not hold
    // device state
    Layout lay{};
    char* d_ws = nullptr;
    size_t ws_bytes = 0;
    bool uploaded = false;
    int table_key = -1;       // cached forward table (n, interp) encoding
    double table_xc = -1.0;
    int adj_table_key = -1;
    int sm_count = 0;
    int device = -1;
};

// builder.cpp
int build_batch(int nbox, const double* const* pos, const double* const* mass, const int64_t* n,
                const psr_box* boxes, int max_leaf, int flags, Leaves** out, std::string* err);
Layout make_layout(const Leaves& h);
size_t table_entry_bytes(int interp);  // p2p_fwd_f32.cu
BoxDev box_constants(const psr_box& b);  // per-box kernel constants

// kernels (launchers defined in the .cu files; return cudaError_t as int)
struct FwdArgs {
    const void* pf;
    const void* pd;
    const int32_t* perm;
    const int32_t* leaf;
    const int32_t* lcen;
    const int64_t* rowptr;
    const uint32_t* pairs;
    const int32_t* items;
    const BoxDev* boxes;
    const void* table;   // float4[(table_n + 1)] forward, then Q table
    unsigned* ctrl;
    const void* cot;     // adjoint: cotangent, original order
    void* cot_sorted;    // adjoint: sorted payload scratch
    void* out;           // forward: acc; adjoint: grad pos
    void* out_m;         // adjoint: grad mass (may be null)
    int64_t n;
    int64_t n_leaves;
    int64_t n_pairs;
    int n_items;
    int nbox;
    int table_n;
    int interp;
    int accum;
    int fold_every;
    int count_pairs;
    int warps_per_block;
    int blocks;
    int max_leaf;
    int variant;     // FP32 forward: PSR_KERNEL_SCALAR, _PACKED or _PAPER
    int stage_cap;   // FP32 kernels: staged particles per warp
    int item_stride; // this launch takes schedule entries ticket * stride + offset
    int item_offset;
    int equal_mass;  // every box has one particle mass: the FP32 kernels take it out of the sums
};

int launch_table(int table_n, int interp, double x_c, void* d_out, void* d_q_out, void* stream);
int launch_fwd_f32(const FwdArgs& a, int precision, void* stream);
int launch_fwd_f64(const FwdArgs& a, void* stream);
int launch_adj_f32(const FwdArgs& a, int precision, void* stream);
int launch_adj_f64(const FwdArgs& a, void* stream);
int fwd_f32_occupancy(int precision, int interp, int accum, int warps, int max_leaf, int table_n,
                      int cap, int variant, int* out);
size_t fwd_f32_smem(int precision, int interp, int table_n, int warps, int cap);
constexpr size_t kSmemPerBlock = 227 * 1024;  // opt-in dynamic shared memory per block
int fwd_f64_occupancy(int warps, int max_leaf, int interp, int table_n, int* out);
int launch_table64(int table_n, int interp, double x_c, void* d_out, void* stream);  // p2p_fwd_f64.cu
size_t fwd_f64_smem(int interp, int table_n);
int launch_fwd_blk(const FwdArgs& a, int precision, void* stream);  // p2p_fwd_blk.cu
int fwd_blk_occupancy(int precision, int interp, int accum, int max_leaf, int table_n, int* out);
int adj_occupancy(int precision, int interp, int accum, int warps, int max_leaf, int table_n,
                  int cap, int variant, int* out);
size_t adj_f32_smem(int precision, int interp, int table_n, int warps, int cap);

}  // namespace psr
