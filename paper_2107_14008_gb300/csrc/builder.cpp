// Host leaf and leaf-pair builder of libpsr.
//
// Paper, Section 2: particles of a domain are organised in a tree whose
// finest cells point to contiguous particle packs (leaves) of at most
// MAXLEAF particles.  Section 3.1: after the tree reorder, particle
// components are laid out as arrays (SoA) for coalesced loads.  Section 3.2:
// the P2P task list of <i-leaf, j-leaf> pairs is regrouped by i-leaf
// (TaskGroup) with an index of start and length per i-leaf (GroupIdx).
//
// This builder uses an octree cut along a 63-bit Morton order (21 bits per
// axis) by default, its leaves packed (consecutive sibling leaves share one
// leaf up to MAXLEAF particles); with PSR_BUILD_ORB it builds the paper's ORB tree (each
// cell's particles split into two halves of equal count along the longest
// axis of their box).  The sum it feeds is tree-independent up to rounding
// order.  The near-field list holds, for every target leaf,
// every (source leaf, periodic image) whose tight bounding boxes come closer
// than r_c, so no pair within the cutoff is missed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>

#include "psr_internal.h"

namespace psr {
namespace {

int host_threads()
{
    const char* env = std::getenv("PSR_THREADS");
    if (env && std::atoi(env) > 0) return std::atoi(env);
    unsigned t = std::thread::hardware_concurrency();
    return t ? (int)t : 1;
}

// Runs f(begin, end) over [0, n) in chunks of `grain` on all host threads.
template <class F>
void parallel_for(int64_t n, int64_t grain, F f)
{
    if (n <= 0) return;
    int64_t chunks = (n + grain - 1) / grain;
    int nt = (int)std::min<int64_t>(host_threads(), chunks);
    if (nt <= 1) {
        f((int64_t)0, n);
        return;
    }
    std::atomic<int64_t> next{0};
    auto work = [&]() {
        for (;;) {
            int64_t b = next.fetch_add(grain);
            if (b >= n) break;
            f(b, std::min(n, b + grain));
        }
    };
    std::vector<std::thread> th;
    th.reserve(nt - 1);
    for (int i = 1; i < nt; ++i) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
}

// Spread the low 21 bits of v so that bit k lands on bit 3k.
inline uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

struct KeyIdx {
    uint64_t key;
    int64_t idx;
};

// Stable LSD radix sort on the 63-bit key (8 passes of 8 bits).
void radix_sort(std::vector<KeyIdx>& a)
{
    const int64_t n = (int64_t)a.size();
    if (n < (1 << 16)) {
        std::sort(a.begin(), a.end(), [](const KeyIdx& x, const KeyIdx& y) {
            return x.key < y.key || (x.key == y.key && x.idx < y.idx);
        });
        return;
    }
    std::vector<KeyIdx> tmp(n);
    int nt = std::max(1, std::min(host_threads(), 64));
    int64_t per = (n + nt - 1) / nt;
    std::vector<int64_t> hist((size_t)nt * 256);
    KeyIdx* src = a.data();
    KeyIdx* dst = tmp.data();
    for (int pass = 0; pass < 8; ++pass) {
        int sh = 8 * pass;
        std::fill(hist.begin(), hist.end(), 0);
        std::vector<std::thread> th;
        auto count = [&](int t) {
            int64_t b = t * per, e = std::min(n, b + per);
            int64_t* h = &hist[(size_t)t * 256];
            for (int64_t i = b; i < e; ++i) h[(src[i].key >> sh) & 255]++;
        };
        for (int t = 1; t < nt; ++t) th.emplace_back(count, t);
        count(0);
        for (auto& x : th) x.join();
        th.clear();
        int64_t sum = 0;
        for (int d = 0; d < 256; ++d)
            for (int t = 0; t < nt; ++t) {
                int64_t c = hist[(size_t)t * 256 + d];
                hist[(size_t)t * 256 + d] = sum;
                sum += c;
            }
        auto scatter = [&](int t) {
            int64_t b = t * per, e = std::min(n, b + per);
            int64_t* h = &hist[(size_t)t * 256];
            for (int64_t i = b; i < e; ++i) dst[h[(src[i].key >> sh) & 255]++] = src[i];
        };
        for (int t = 1; t < nt; ++t) th.emplace_back(scatter, t);
        scatter(0);
        for (auto& x : th) x.join();
        std::swap(src, dst);
    }
    // 8 passes: result is back in a
}

struct Node {
    double lo[3], hi[3];
    int32_t first_child;  // into children[], or -1
    int32_t nchild;
    int32_t leaf;         // global leaf index, or -1 for an internal node
};

struct LeafRec {
    int64_t first;  // global sorted index
    int32_t count;
    int32_t level;
    uint32_t ix, iy, iz;  // octree cell (octree leaves)
    int32_t cen[3];       // reference point in units of L / 2^22 (ORB leaves), or -1
    double lo[3], hi[3];
};

// Octree of one box over its sorted keys.
struct Tree {
    const uint64_t* key = nullptr;  // sorted keys of this box (local index)
    const double* xs = nullptr;     // sorted wrapped positions of this box (3 per particle)
    int64_t base = 0;               // global sorted index of local particle 0
    int max_leaf = 32;
    bool pack = false;              // pack sibling leaves (see build)
    int32_t leaf_base = 0;          // global index of this box's first leaf
    std::vector<Node> nodes;
    std::vector<int32_t> children;
    std::vector<LeafRec> leaves;
    int32_t root = -1;

    void leaf_box(LeafRec& lf) const
    {
        for (int a = 0; a < 3; ++a) {
            lf.lo[a] = INFINITY;
            lf.hi[a] = -INFINITY;
        }
        for (int64_t i = lf.first - base; i < lf.first - base + lf.count; ++i)
            for (int a = 0; a < 3; ++a) {
                double v = xs[3 * i + a];
                lf.lo[a] = std::min(lf.lo[a], v);
                lf.hi[a] = std::max(lf.hi[a], v);
            }
    }

    int32_t make_leaf(int64_t b, int64_t e, int level, uint32_t ix, uint32_t iy, uint32_t iz)
    {
        LeafRec lf;
        lf.first = base + b;
        lf.count = (int32_t)(e - b);
        lf.level = level;
        lf.ix = ix;
        lf.iy = iy;
        lf.iz = iz;
        lf.cen[0] = lf.cen[1] = lf.cen[2] = -1;
        leaf_box(lf);
        Node nd;
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = lf.lo[a];
            nd.hi[a] = lf.hi[a];
        }
        nd.first_child = -1;
        nd.nchild = 0;
        nd.leaf = leaf_base + (int32_t)leaves.size();
        leaves.push_back(lf);
        nodes.push_back(nd);
        return (int32_t)nodes.size() - 1;
    }

    int32_t build(int64_t b, int64_t e, int level, uint32_t ix, uint32_t iy, uint32_t iz)
    {
        std::vector<int32_t> kids;
        if (e - b <= max_leaf) return make_leaf(b, e, level, ix, iy, iz);
        if (level == kMortonBits) {
            // Coincident quantised positions: split the pack into chunks of
            // max_leaf particles that share the cell centre.
            for (int64_t s = b; s < e; s += max_leaf)
                kids.push_back(make_leaf(s, std::min(e, s + max_leaf), level, ix, iy, iz));
        } else {
            int sh = 3 * (kMortonBits - 1 - level);
            uint64_t prefix = key[b] & ~((sh + 3 >= 64) ? ~0ULL : ((1ULL << (sh + 3)) - 1));
            int64_t s = b;
            // packing: consecutive children that would be leaves share one
            // leaf (this cell's) while their total stays within max_leaf; a
            // pack of one child keeps the child's own cell
            int64_t pb = -1, pe = -1;  // open pack [pb, pe)
            int pc = 0, pk = 0;        // its single child's octant, children in it
            auto close_pack = [&]() {
                if (pk == 1)
                    kids.push_back(make_leaf(pb, pe, level + 1, 2 * ix + ((pc >> 2) & 1),
                                             2 * iy + ((pc >> 1) & 1), 2 * iz + (pc & 1)));
                else if (pk > 1)
                    kids.push_back(make_leaf(pb, pe, level, ix, iy, iz));
                pk = 0;
            };
            for (int c = 0; c < 8; ++c) {
                uint64_t hi = prefix | ((uint64_t)(c + 1) << sh);
                int64_t t = (c == 7) ? e : (int64_t)(std::lower_bound(key + s, key + e, hi) - key);
                if (t > s) {
                    if (pack && t - s <= max_leaf) {
                        if (pk > 0 && (pe - pb) + (t - s) <= max_leaf) {
                            pe = t;
                            ++pk;
                        } else {
                            close_pack();
                            pb = s;
                            pe = t;
                            pc = c;
                            pk = 1;
                        }
                    } else {
                        close_pack();
                        kids.push_back(build(s, t, level + 1, 2 * ix + ((c >> 2) & 1),
                                             2 * iy + ((c >> 1) & 1), 2 * iz + (c & 1)));
                    }
                }
                s = t;
            }
            close_pack();
        }
        Node nd;
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = INFINITY;
            nd.hi[a] = -INFINITY;
        }
        for (int32_t k : kids)
            for (int a = 0; a < 3; ++a) {
                nd.lo[a] = std::min(nd.lo[a], nodes[k].lo[a]);
                nd.hi[a] = std::max(nd.hi[a], nodes[k].hi[a]);
            }
        nd.first_child = (int32_t)children.size();
        nd.nchild = (int32_t)kids.size();
        nd.leaf = -1;
        children.insert(children.end(), kids.begin(), kids.end());
        nodes.push_back(nd);
        return (int32_t)nodes.size() - 1;
    }

    // ---- ORB (paper, Section 2) over the local particles in `ord` order:
    // a cell's particles go in equal halves (the second one larger by one
    // for an odd count) to two children, split at the median of the longest
    // axis of their box (ties by index), until at most max_leaf remain.
    // ord[k] is the local index of the particle at ORB position k.
    std::vector<int32_t> ord;
    double unit = 1.0;  // L / 2^22

    int32_t make_orb_leaf(int64_t b, int64_t e, int level)
    {
        LeafRec lf;
        lf.first = base + b;
        lf.count = (int32_t)(e - b);
        lf.level = level;
        lf.ix = lf.iy = lf.iz = 0;
        for (int a = 0; a < 3; ++a) {
            lf.lo[a] = INFINITY;
            lf.hi[a] = -INFINITY;
        }
        for (int64_t k = b; k < e; ++k)
            for (int a = 0; a < 3; ++a) {
                const double v = xs[3 * (int64_t)ord[k] + a];
                lf.lo[a] = std::min(lf.lo[a], v);
                lf.hi[a] = std::max(lf.hi[a], v);
            }
        // reference point: the box centre rounded to the integer grid
        for (int a = 0; a < 3; ++a) {
            double c = std::floor(0.5 * (lf.lo[a] + lf.hi[a]) / unit + 0.5);
            c = std::min(std::max(c, 0.0), (double)((1 << kCentreShift) - 1));
            lf.cen[a] = (int32_t)c;
        }
        Node nd;
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = lf.lo[a];
            nd.hi[a] = lf.hi[a];
        }
        nd.first_child = -1;
        nd.nchild = 0;
        nd.leaf = leaf_base + (int32_t)leaves.size();
        leaves.push_back(lf);
        nodes.push_back(nd);
        return (int32_t)nodes.size() - 1;
    }

    int32_t build_orb(int64_t b, int64_t e, int level)
    {
        if (e - b <= max_leaf) return make_orb_leaf(b, e, level);
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t k = b; k < e; ++k)
            for (int a = 0; a < 3; ++a) {
                const double v = xs[3 * (int64_t)ord[k] + a];
                lo[a] = std::min(lo[a], v);
                hi[a] = std::max(hi[a], v);
            }
        int ax = 0;
        for (int a = 1; a < 3; ++a)
            if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
        std::vector<int32_t> kids;
        if (!(hi[ax] > lo[ax])) {
            // coincident positions: chunks of max_leaf particles
            for (int64_t s = b; s < e; s += max_leaf)
                kids.push_back(make_orb_leaf(s, std::min(e, s + max_leaf), level + 1));
        } else {
            const int64_t mid = b + (e - b) / 2;
            const double* x = xs;
            std::nth_element(ord.begin() + b, ord.begin() + mid, ord.begin() + e,
                             [x, ax](int32_t i, int32_t j) {
                                 const double u = x[3 * (int64_t)i + ax], v = x[3 * (int64_t)j + ax];
                                 return u < v || (u == v && i < j);
                             });
            kids.push_back(build_orb(b, mid, level + 1));
            kids.push_back(build_orb(mid, e, level + 1));
        }
        Node nd;
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = INFINITY;
            nd.hi[a] = -INFINITY;
        }
        for (int32_t k : kids)
            for (int a = 0; a < 3; ++a) {
                nd.lo[a] = std::min(nd.lo[a], nodes[k].lo[a]);
                nd.hi[a] = std::max(nd.hi[a], nodes[k].hi[a]);
            }
        nd.first_child = (int32_t)children.size();
        nd.nchild = (int32_t)kids.size();
        nd.leaf = -1;
        children.insert(children.end(), kids.begin(), kids.end());
        nodes.push_back(nd);
        return (int32_t)nodes.size() - 1;
    }
};

inline double gap2(const double alo[3], const double ahi[3], const double blo[3],
                   const double bhi[3], const double sh[3])
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double l = blo[a] + sh[a], h = bhi[a] + sh[a];
        double g = std::max(0.0, std::max(l - ahi[a], alo[a] - h));
        s += g * g;
    }
    return s;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

BoxDev box_constants(const psr_box& bx)
{
    BoxDev d{};
    d.L = bx.L;
    d.r_s = bx.r_s;
    d.r_c = bx.r_c;
    d.G = bx.G;
    d.rc2 = bx.r_c * bx.r_c;
    d.inv_2rs = 1.0 / (2.0 * bx.r_s);
    d.unit = (float)(std::ldexp(bx.L, -kCentreShift) / (2.0 * bx.r_s));
    d.x_c = (float)(bx.r_c / (2.0 * bx.r_s));
    d.x_c2 = d.x_c * d.x_c;
    d.g_acc = (float)(bx.G / (4.0 * bx.r_s * bx.r_s));
    d.g_adj = (float)(bx.G / (8.0 * bx.r_s * bx.r_s * bx.r_s));
    d.g_adjm = (float)(bx.G / (4.0 * bx.r_s * bx.r_s));
    return d;
}

Layout make_layout(const Leaves& h)
{
    Layout L{};
    size_t o = 0;
    const size_t n = (size_t)h.n, nl = (size_t)h.n_leaves, np = (size_t)h.n_pairs;
    L.pf = o;        o = align256(o + n * 16);
    L.pd = o;        o = align256(o + ((h.flags & PSR_BUILD_NO_FP64) ? 0 : n * 32));
    L.perm = o;      o = align256(o + n * 4);
    L.leaf = o;      o = align256(o + nl * 16);
    L.lcen = o;      o = align256(o + nl * 16);
    L.rowptr = o;    o = align256(o + (nl + 1) * 8);
    L.pairs = o;     o = align256(o + np * 4);
    L.items = o;     o = align256(o + nl * 4);
    L.boxes = o;     o = align256(o + h.boxdev.size() * sizeof(BoxDev));
    L.table = o;     o = align256(o + 2 * (size_t)(kMaxTableN + 1) * 16);
    L.cotf = o;      o = align256(o + n * ((h.flags & PSR_BUILD_NO_FP64) ? 16 : 32));
    L.ctrl = o;      o = align256(o + kCtrlWords * 4);
    L.frow = o;      o = align256(o + (h.has_far ? (nl + 1) * 8 : 0));
    L.fpairs = o;    o = align256(o + (h.has_far ? (size_t)h.n_far * 4 : 0));
    L.fcen = o;      o = align256(o + (h.has_far ? nl * 32 : 0));
    L.fofs = o;      o = align256(o + (h.has_far ? nl * 16 : 0));
    L.total = o;
    return L;
}

int build_batch(int nbox, const double* const* pos, const double* const* mass, const int64_t* n,
                const psr_box* boxes, int max_leaf, int flags, Leaves** out, std::string* err)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!out || !pos || !n || !boxes || nbox < 1) {
        *err = "null argument or nbox < 1";
        return PSR_E_ARG;
    }
    *out = nullptr;
    if (max_leaf < 1 || max_leaf > kMaxLeaf) {
        *err = "max_leaf must be in [1, 64]";
        return PSR_E_ARG;
    }
    if (flags & ~(PSR_BUILD_NO_FP64 | PSR_BUILD_ORB | PSR_BUILD_UNPACKED)) {
        *err = "unknown build flags";
        return PSR_E_ARG;
    }
    int64_t ntot = 0;
    double ratio = -1.0;
    for (int b = 0; b < nbox; ++b) {
        const psr_box& bx = boxes[b];
        if (n[b] < 0 || (n[b] > 0 && !pos[b])) {
            *err = "box " + std::to_string(b) + ": null positions or n < 0";
            return PSR_E_ARG;
        }
        if (!(std::isfinite(bx.L) && bx.L > 0) || !(std::isfinite(bx.r_s) && bx.r_s > 0) ||
            !std::isfinite(bx.G)) {
            *err = "box " + std::to_string(b) + ": L, r_s must be finite and positive";
            return PSR_E_ARG;
        }
        if (!(bx.r_c > 0) || !(bx.r_c < bx.L)) {
            *err = "box " + std::to_string(b) + ": need 0 < r_c < L";
            return PSR_E_CUTOFF;
        }
        double r = bx.r_c / bx.r_s;
        if (ratio < 0) ratio = r;
        if (std::fabs(r - ratio) > 1e-12 * ratio) {
            *err = "all boxes of a batch must share r_c / r_s";
            return PSR_E_ARG;
        }
        ntot += n[b];
    }
    if (ntot >= ((int64_t)1 << 31)) {
        *err = "at most 2^31 - 1 particles";
        return PSR_E_ARG;
    }
    Leaves* h = new (std::nothrow) Leaves();
    if (!h) {
        *err = "out of host memory";
        return PSR_E_NOMEM;
    }
    try {
        h->nbox = nbox;
        h->boxes.assign(boxes, boxes + nbox);
        h->n = ntot;
        h->max_leaf_req = max_leaf;
        h->flags = flags;
        h->box_first.resize(nbox + 1);
        h->box_first[0] = 0;
        for (int b = 0; b < nbox; ++b) h->box_first[b + 1] = h->box_first[b] + n[b];

        // ---- wrap and key -------------------------------------------------
        std::vector<double> wrapped((size_t)ntot * 3);
        std::vector<double> m((size_t)ntot);
        std::vector<KeyIdx> keys((size_t)ntot);
        std::atomic<int> bad{0};
        for (int b = 0; b < nbox; ++b) {
            const double L = boxes[b].L;
            const double* p = pos[b];
            const double* mb = mass ? mass[b] : nullptr;
            const int64_t off = h->box_first[b];
            const double scale = std::ldexp(1.0, kMortonBits) / L;
            parallel_for(n[b], 1 << 16, [&](int64_t s, int64_t e) {
                for (int64_t i = s; i < e; ++i) {
                    uint64_t q[3];
                    for (int a = 0; a < 3; ++a) {
                        double v = p[3 * i + a];
                        if (!std::isfinite(v)) {
                            bad = 1;
                            v = 0.0;
                        }
                        v = std::fmod(v, L);
                        if (v < 0) v += L;
                        if (!(v < L)) v = 0.0;
                        wrapped[3 * (off + i) + a] = v;
                        double qq = std::floor(v * scale);
                        if (qq < 0) qq = 0;
                        if (qq > (double)((1u << kMortonBits) - 1)) qq = (double)((1u << kMortonBits) - 1);
                        q[a] = (uint64_t)qq;
                    }
                    double mi = mb ? mb[i] : 1.0 / (double)n[b];
                    if (!std::isfinite(mi)) {
                        bad = 1;
                        mi = 0.0;
                    }
                    m[off + i] = mi;
                    // box id in the top bits keeps boxes contiguous
                    keys[off + i].key = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
                    keys[off + i].idx = off + i;
                }
            });
        }
        if (bad) {
            delete h;
            *err = "non-finite position or mass";
            return PSR_E_ARG;
        }
        // sort each box separately (boxes stay contiguous, box 0 first)
        for (int b = 0; b < nbox; ++b) {
            std::vector<KeyIdx> part(keys.begin() + h->box_first[b], keys.begin() + h->box_first[b + 1]);
            radix_sort(part);
            std::copy(part.begin(), part.end(), keys.begin() + h->box_first[b]);
        }
        std::vector<uint64_t> skey((size_t)ntot);
        std::vector<double> sx((size_t)ntot * 3);
        h->perm.resize(ntot);
        h->perm32.resize(ntot);
        parallel_for(ntot, 1 << 16, [&](int64_t s, int64_t e) {
            for (int64_t k = s; k < e; ++k) {
                skey[k] = keys[k].key;
                int64_t i = keys[k].idx;
                h->perm[k] = i;
                h->perm32[k] = (int32_t)i;
                for (int a = 0; a < 3; ++a) sx[3 * k + a] = wrapped[3 * i + a];
            }
        });
        std::vector<KeyIdx>().swap(keys);

        // ---- octrees ------------------------------------------------------
        std::vector<Tree> trees(nbox);
        int32_t leaf_total = 0;
        for (int b = 0; b < nbox; ++b) {
            Tree& t = trees[b];
            t.key = skey.data() + h->box_first[b];
            t.xs = sx.data() + 3 * h->box_first[b];
            t.base = h->box_first[b];
            t.max_leaf = max_leaf;
            t.pack = !(flags & PSR_BUILD_UNPACKED);
            t.leaf_base = leaf_total;
            if (n[b] == 0) continue;  // an empty box has no leaves
            if (flags & PSR_BUILD_ORB) {
                t.unit = std::ldexp(boxes[b].L, -kCentreShift);
                t.ord.resize(n[b]);
                for (int64_t k = 0; k < n[b]; ++k) t.ord[k] = (int32_t)k;  // from Morton order
                t.root = t.build_orb(0, n[b], 0);
            } else {
                t.root = t.build(0, n[b], 0, 0, 0, 0);
            }
            leaf_total += (int32_t)t.leaves.size();
            if (leaf_total >= (1 << 27)) {
                delete h;
                *err = "more than 2^27 leaves";
                return PSR_E_ARG;
            }
        }
        if (flags & PSR_BUILD_ORB) {
            // particles into ORB order, box by box
            std::vector<double> sx2(sx.size());
            std::vector<int64_t> perm2(h->perm.size());
            for (int b = 0; b < nbox; ++b) {
                const Tree& t = trees[b];
                const int64_t base = h->box_first[b];
                for (int64_t k = 0; k < n[b]; ++k) {
                    const int64_t o = base + t.ord[k];
                    for (int a = 0; a < 3; ++a) sx2[3 * (base + k) + a] = sx[3 * o + a];
                    perm2[base + k] = h->perm[o];
                }
            }
            sx.swap(sx2);
            h->perm.swap(perm2);
            for (Tree& t : trees) t.xs = nullptr;  // the trees' boxes are final
            for (int64_t k = 0; k < ntot; ++k) h->perm32[k] = (int32_t)h->perm[k];
        }
        const int64_t nl = leaf_total;
        h->leaf.resize(nl * 4);
        h->lcen.resize(nl * 4);
        std::vector<const LeafRec*> lrec(nl);
        std::vector<int> lbox(nl);
        for (int b = 0; b < nbox; ++b)
            for (size_t k = 0; k < trees[b].leaves.size(); ++k) {
                int64_t g = trees[b].leaf_base + (int64_t)k;
                lrec[g] = &trees[b].leaves[k];
                lbox[g] = b;
            }
        int maxl = 0;
        for (int64_t g = 0; g < nl; ++g) {
            const LeafRec& lf = *lrec[g];
            h->leaf[4 * g + 0] = (int32_t)lf.first;
            h->leaf[4 * g + 1] = lf.count;
            h->leaf[4 * g + 2] = lbox[g];
            h->leaf[4 * g + 3] = 0;
            if (lf.cen[0] >= 0) {  // ORB leaf: its box centre on the integer grid
                for (int a = 0; a < 3; ++a) h->lcen[4 * g + a] = lf.cen[a];
            } else {
                uint32_t sc = 1u << (kMortonBits - lf.level);  // 2^(21-l)
                h->lcen[4 * g + 0] = (int32_t)((2 * lf.ix + 1) * sc);
                h->lcen[4 * g + 1] = (int32_t)((2 * lf.iy + 1) * sc);
                h->lcen[4 * g + 2] = (int32_t)((2 * lf.iz + 1) * sc);
            }
            h->lcen[4 * g + 3] = lf.level;
            maxl = std::max(maxl, lf.count);
        }
        h->max_leaf = maxl;

        // ---- per-box constants -------------------------------------------
        h->boxdev.resize(nbox);
        h->equal_mass = true;
        for (int b = 0; b < nbox; ++b) {
            h->boxdev[b] = box_constants(boxes[b]);
            // one mass for the whole box: the FP32 kernels then apply it once
            // per target instead of once per pair
            const int64_t f = h->box_first[b], e = h->box_first[b + 1];
            bool eq = true;
            for (int64_t i = f + 1; i < e && eq; ++i) eq = m[i] == m[f];
            h->boxdev[b].m_eq = (eq && e > f) ? (float)m[f] : 0.0f;
            if (!eq) h->equal_mass = false;
        }

        // ---- sorted payloads ----------------------------------------------
        h->pf.resize((size_t)ntot * 4);
        if (!(flags & PSR_BUILD_NO_FP64)) h->pd.resize((size_t)ntot * 4);
        parallel_for(nl, 1024, [&](int64_t s, int64_t e) {
            for (int64_t g = s; g < e; ++g) {
                const psr_box& bx = boxes[lbox[g]];
                const double unit = std::ldexp(bx.L, -kCentreShift);
                const double inv = 1.0 / (2.0 * bx.r_s);
                double c[3] = {h->lcen[4 * g] * unit, h->lcen[4 * g + 1] * unit,
                               h->lcen[4 * g + 2] * unit};
                int64_t f = h->leaf[4 * g], cnt = h->leaf[4 * g + 1];
                for (int64_t k = f; k < f + cnt; ++k) {
                    for (int a = 0; a < 3; ++a)
                        h->pf[4 * k + a] = (float)((sx[3 * k + a] - c[a]) * inv);
                    double mk = m[h->perm[k]];
                    h->pf[4 * k + 3] = (float)mk;
                    if (!h->pd.empty()) {
                        for (int a = 0; a < 3; ++a) h->pd[4 * k + a] = sx[3 * k + a];
                        h->pd[4 * k + 3] = mk;
                    }
                }
            }
        });

        // ---- near-field leaf-pair list ------------------------------------
        // rows in leaf order; each task handles a chunk of target leaves
        const int64_t grain = 256;
        const int64_t nchunks = (nl + grain - 1) / grain;
        std::vector<std::vector<uint32_t>> cpairs(nchunks);
        std::vector<std::vector<int64_t>> crow(nchunks);
        std::vector<int64_t> cost(nl, 0);
        parallel_for(nl, grain, [&](int64_t s, int64_t e) {
            int64_t ci = s / grain;
            std::vector<uint32_t>& out = cpairs[ci];
            std::vector<int64_t>& rows = crow[ci];
            std::vector<int32_t> stack;
            stack.reserve(256);
            for (int64_t g = s; g < e; ++g) {
                rows.push_back((int64_t)out.size());
                const LeafRec& A = *lrec[g];
                const Tree& t = trees[lbox[g]];
                const psr_box& bx = boxes[lbox[g]];
                const double rc2 = bx.r_c * bx.r_c * (1.0 + 1e-5);
                int64_t src = 0;
                for (int code = 0; code < kShiftCodes; ++code) {
                    double sh[3] = {(code / 9 - 1) * bx.L, ((code / 3) % 3 - 1) * bx.L,
                                    (code % 3 - 1) * bx.L};
                    const Node& R = t.nodes[t.root];
                    if (gap2(A.lo, A.hi, R.lo, R.hi, sh) >= rc2) continue;
                    stack.clear();
                    stack.push_back(t.root);
                    while (!stack.empty()) {
                        int32_t k = stack.back();
                        stack.pop_back();
                        const Node& N = t.nodes[k];
                        if (gap2(A.lo, A.hi, N.lo, N.hi, sh) >= rc2) continue;
                        if (N.leaf >= 0) {
                            out.push_back(((uint32_t)N.leaf << 5) | (uint32_t)code);
                            src += h->leaf[4 * (int64_t)N.leaf + 1];
                        } else {
                            // push in reverse so children pop in Morton order
                            for (int c = N.nchild - 1; c >= 0; --c)
                                stack.push_back(t.children[N.first_child + c]);
                        }
                    }
                }
                cost[g] = src * (int64_t)A.count;
            }
        });
        std::vector<int64_t> cbase(nchunks + 1, 0);
        for (int64_t c = 0; c < nchunks; ++c) cbase[c + 1] = cbase[c] + (int64_t)cpairs[c].size();
        h->pairs.resize(cbase[nchunks]);
        h->rowptr.resize(nl + 1);
        parallel_for(nchunks, 1, [&](int64_t s, int64_t e) {
            for (int64_t c = s; c < e; ++c) {
                std::copy(cpairs[c].begin(), cpairs[c].end(), h->pairs.begin() + cbase[c]);
                for (size_t r = 0; r < crow[c].size(); ++r)
                    h->rowptr[c * grain + (int64_t)r] = cbase[c] + crow[c][r];
                std::vector<uint32_t>().swap(cpairs[c]);
            }
        });
        h->rowptr[nl] = cbase[nchunks];
        int maxrow = 0;
        int64_t evaluated = 0;
        for (int64_t g = 0; g < nl; ++g) {
            maxrow = std::max<int64_t>(maxrow, h->rowptr[g + 1] - h->rowptr[g]);
            evaluated += cost[g];
        }
        h->max_row = maxrow;
        h->evaluated = evaluated;

        // ---- schedule: largest work first (stable in Morton order) --------
        h->items.resize(nl);
        for (int64_t g = 0; g < nl; ++g) h->items[g] = (int32_t)g;
        std::stable_sort(h->items.begin(), h->items.end(),
                         [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
        h->n_leaves = nl;
        h->n_pairs = (int64_t)h->pairs.size();
        h->has_pd = !(flags & PSR_BUILD_NO_FP64);
        h->lay = make_layout(*h);
    } catch (const std::bad_alloc&) {
        delete h;
        *err = "out of host memory";
        return PSR_E_NOMEM;
    }
    h->build_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return PSR_OK;
}

}  // namespace psr
