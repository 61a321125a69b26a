// world.cpp -- the C ABI of include/dem.h: world and pile management, host
// set-up of aggregates in FP64, device layout (every pile contiguous in every
// array, pile-local indices inside), the per-step launch sequence captured
// once into a CUDA graph, readout and error reporting.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dem_internal.h"

using namespace dem;

namespace {

// NVTX range over a host call (visible in Nsight Systems; a no-op without a tool)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

enum Cls { C_SPH, C_ENT, C_CTILE, C_AGG, C_CELL, C_TILE, C_CHUNK, C_PILE, C_GITEM, C_GPART, C_TNODE,
           C_TLEAF, C_TSPH, C_NCLS };

struct Field {
    void **ptr;
    Cls cls;
    size_t el;
    bool keep;   // preserved (per-pile ranges copied) when the layout changes
};

struct PileHost {
    int32_t id;
    int64_t ns, na, nc, nch, nt;
    int64_t ne;            // candidate-list entries (never shrinks)
    int nx, ny, nz;
    double cell, smax, smin;
    double ext[3];         // extent of the wrapped grid at creation (cell x dims)
    dem_params P;
    double M_total;
    bool reported;
    bool watch_on;         // a radius-growth watch is armed (evaluated in the step graph)
};

}  // namespace

struct dem_world {
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    dem_alloc_fn alloc = nullptr;
    dem_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    std::string err = "";
    int precision = -1;
    int K = -1;
    std::vector<PileHost> piles;   // in layout order
    int32_t next_id = 0;
    Arrays A{};
    Sizes Z{};
    int64_t cap[C_NCLS] = {0};
    std::vector<Field> fields;
    void *slab = nullptr;             // every field's device memory, one allocation
    size_t held = 0;
    // graph
    cudaGraphExec_t exec = nullptr;
    bool graph_valid = false;
    // tuning
    int grav_block = 128, grav_ib = 4;
    int64_t grav_jchunk = 0;          // > 0: fixed j-range length per work item
    double grav_item = 1048576.0;     // else: target interactions per work item
    bool grav_pack = false;           // packed f32x2 pair terms (even grav_ib)
    bool grav_sym = true;             // mixed path: symmetric tile-pair form
    int grav_tile = 0;                // symmetric form's tile: 0 = automatic, 128 or 512
    double grav_theta = 0.0;          // > 0 (mixed path): tree gravity with this opening angle
    int grav_order = 4;               // tree gravity: highest multipole rank (4 or 2)
    int tree_maxD = 0;                // deepest tree of the current layout
    int sm_count = 0;
    double cell_factor = 1.0;
    double skin_frac = 0.1;           // neighbour-list skin / largest radius
    int contact_inbox = kInboxCap;    // contact inbox entries per tile range (testing: smaller splits more)
    int contact_mode = 0;             // 0: one thread per sphere, 1: tiles with a shared-memory inbox
    // flags readback
    PileDyn *h_dyn = nullptr;   // pinned
    int64_t h_dyn_cap = 0;
    // host staging of dem_add_aggregates, kept between calls (pinned if possible)
    char *h_stage = nullptr;
    size_t h_stage_cap = 0;
    bool h_stage_pinned = false;
    cudaEvent_t ev_flags = nullptr;
    // asynchronous reads: destination, doubles, whether they are float-float slots, event after the copy
    struct AsyncRead { double *out; int64_t n; bool ff; };
    std::vector<AsyncRead> reads;
    cudaEvent_t rev[DEM_MAX_ASYNC_READS] = {};
    bool pending = false;
    int64_t pending_n = 0;
    bool own_stream = false;
    // timing inside the graph
    int timed_kernel = -1;
    cudaEvent_t kev[2] = {nullptr, nullptr};
    cudaEvent_t sev[2] = {nullptr, nullptr};
    int32_t graph_kernels = 0;
};

namespace {

dem_status fail(dem_world *w, dem_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (w) w->err = buf;
    return s;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(w, DEM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

void *dev_alloc(dem_world *w, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (w->alloc) {
        p = w->alloc(bytes, (void *)w->stream, w->ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(dem_world *w, void *p)
{
    if (!p) return;
    if (w->free_fn) w->free_fn(p, w->ctx);
    else cudaFree(p);
}

// Contact range of a pile's cells: the largest radii sum, and that plus the
// neighbour-list skin.
double min_cell(const PileHost &q) { return 2.0 * q.smax * (1.0 + 1e-6); }

// Skin actually used by a pile: the requested fraction of its largest radius,
// limited by what its cell edge leaves beyond the radii sum.
double skin_of(const dem_world *w, const PileHost &q)
{
    double want = w->skin_frac * q.smax;
    double room = q.cell - min_cell(q);
    return std::max(0.0, std::min(want, room));
}

// Candidate-list entries of a pile: kEntPerSphere per sphere at the default
// skin (0.1 of the largest radius), scaled by the candidate volume
// ((2 + skin) / 2.1)^3 for larger skins; a pile's capacity never shrinks, so
// offsets of lists built earlier stay inside it.
void size_lists(const dem_world *w, PileHost &q)
{
    const double f = std::max(1.0, std::pow((2.0 + w->skin_frac) / 2.1, 3.0));
    const int64_t per = (int64_t)std::ceil(kEntPerSphere * f);
    q.ne = std::max<int64_t>(q.ne, q.ns * per);
}

void build_fields(dem_world *w)
{
    Arrays &a = w->A;
    bool d = w->precision == DEM_FP64;
    auto add = [&](void **p, Cls c, size_t el, bool keep) { w->fields.push_back({p, c, el, keep}); };
    w->fields.clear();
    add((void **)&a.sph_agg, C_SPH, 4, true);
    add((void **)&a.sph_pile, C_SPH, 4, false);
    add((void **)&a.b64, C_SPH, 24, true);
    add((void **)&a.s64, C_SPH, 8, true);
    add((void **)&a.m64, C_SPH, 8, true);
    add((void **)&a.key, C_SPH, 4, false);
    add((void **)&a.rank, C_SPH, 4, false);
    add((void **)&a.sorted, C_SPH, 4, false);
    add((void **)&a.sagg, C_SPH, 4, false);
    add((void **)&a.fg, C_SPH, 32, true);
    // candidate lists (both buffers: a rebuild after a layout change reads the
    // previous ones) and contact tiles
    for (int b = 0; b < 2; ++b) {
        add((void **)&a.ccnt[b], C_SPH, 4, true);
        add((void **)&a.coff[b], C_SPH, 4, true);
        add((void **)&a.cand[b], C_ENT, 8, true);
        add((void **)&a.cand_id[b], C_ENT, 4, true);
    }
    add((void **)&a.ctile, C_CTILE, 16, false);
    add((void **)&a.ctile_cnt, C_CTILE, 4, false);
    add((void **)&a.ctile_base, C_CTILE, 4, false);
    add((void **)&a.pos_of_home[0], C_SPH, 4, true);
    add((void **)&a.pos_of_home[1], C_SPH, 4, true);
    if (d) {
        add((void **)&a.dp_, C_SPH, 32, false);
        add((void **)&a.dv_, C_SPH, 32, false);
        add((void **)&a.dw_, C_SPH, 32, false);
        add((void **)&a.gpos64, C_SPH, 32, false);
        add((void **)&a.ftc64, C_SPH, 64, true);
        add((void **)&a.hist64[0], C_ENT, 32, true);
        add((void **)&a.hist64[1], C_ENT, 32, true);
        add((void **)&a.hist64_rm, C_ENT, 32, false);
        add((void **)&a.rec64, C_AGG, sizeof(AggRec64), false);
    } else {
        add((void **)&a.bh, C_SPH, 16, true);
        add((void **)&a.bl, C_SPH, 16, true);
        add((void **)&a.xqr, C_SPH, 32, false);
        add((void **)&a.sph_, C_SPH, 16, false);
        add((void **)&a.svw, C_SPH, 32, false);
        add((void **)&a.gpos32, C_SPH, 16, false);
        add((void **)&a.ftc32, C_SPH, 32, true);
        add((void **)&a.hist32[0], C_ENT, 16, true);
        add((void **)&a.hist32[1], C_ENT, 16, true);
        add((void **)&a.hist32_rm, C_ENT, 16, false);
        add((void **)&a.rec32, C_AGG, sizeof(AggRecMixed), false);
        add((void **)&a.I32, C_AGG, 36, true);
        add((void **)&a.Iinv32, C_AGG, 36, true);
        add((void **)&a.gacc, C_SPH, 32, false);
    }
    add((void **)&a.agg_first, C_AGG, 4, true);
    add((void **)&a.agg_count, C_AGG, 4, true);
    add((void **)&a.agg_pile, C_AGG, 4, false);
    add((void **)&a.M, C_AGG, 8, true);
    add((void **)&a.I, C_AGG, 72, true);
    add((void **)&a.Iinv, C_AGG, 72, true);
    add((void **)&a.r, C_AGG, 24, true);
    add((void **)&a.v, C_AGG, 24, true);
    add((void **)&a.q, C_AGG, 32, true);
    add((void **)&a.wb, C_AGG, 24, true);
    add((void **)&a.acc, C_AGG, 24, true);
    add((void **)&a.torque, C_AGG, 24, true);
    for (int k = 0; k < 3; ++k) add((void **)&a.out[k], C_AGG, 48, true);
    add((void **)&a.invM, C_AGG, 8, true);
    a.out_ff = d ? 0 : 1;
    add((void **)&a.aref, C_AGG, 32, true);
    add((void **)&a.ccount, C_CELL, 4, false);
    add((void **)&a.cstart, C_CELL, 4, false);
    add((void **)&a.tile_sum, C_TILE, 4, false);
    add((void **)&a.chunk_part, C_CHUNK, 8 * kPartialDoubles, false);
    add((void **)&a.chunk_pile, C_CHUNK, 4, false);
    add((void **)&a.bulk_part, C_CHUNK, 8 * 32, false);
    add((void **)&a.pile_arrive, C_PILE, 4, false);
    add((void **)&a.watch, C_PILE, sizeof(PileWatch), true);
    add((void **)&a.ps, C_PILE, sizeof(PileStatic), false);
    add((void **)&a.pd, C_PILE, sizeof(PileDyn), true);
    add((void **)&a.enabled, C_PILE, 4, false);
    add((void **)&a.gpart_base, C_PILE, 8, false);
    add((void **)&a.gnchunk, C_PILE, 4, false);
    add((void **)&a.gcounter, C_PILE, 4, false);
    add((void **)&a.gitems, C_GITEM, 16, false);
    add((void **)&a.gpart, C_GPART, d ? 32 : 16, false);
    add((void **)&a.tkey, C_TSPH, 4, false);
    add((void **)&a.trank, C_TSPH, 4, false);
    add((void **)&a.tsorted, C_TSPH, 4, false);
    add((void **)&a.tpos, C_TSPH, 16, false);
    add((void **)&a.tagg, C_TSPH, 4, false);
    add((void **)&a.tpart, C_TSPH, 64 * 16, false);
    add((void **)&a.tbox, C_PILE, 32, false);
    add((void **)&a.tnode, C_TNODE, 144, false);
    add((void **)&a.traw, C_TNODE, 128, false);
    add((void **)&a.tnode_pile, C_TNODE, 4, false);
    add((void **)&a.tleaf, C_TLEAF, 8, false);
    add((void **)&a.tleaf_pile, C_TLEAF, 4, false);
}

// Tree depth of a pile under tree gravity (0 = direct sum): leaves of ~4
// spheres, 2..6 levels below the root.
int tree_depth(const dem_world *w, const PileHost &q)
{
    if (!(w->grav_theta > 0) || w->precision != DEM_MIXED || q.P.G == 0.0) return 0;
    int D = 2;   // the walk starts at the 64 cells of level 2
    while (D < 6 && ((int64_t)1 << (3 * D)) * 4 < q.ns) ++D;
    return D;
}

// Elements of class c that pile q occupies (and its per-element multiplier).
int64_t pile_count(const dem_world *w, const PileHost &q, Cls c)
{
    switch (c) {
    case C_SPH: return q.ns;
    case C_ENT: return q.ne;
    case C_CTILE: return (q.ns + kCTile - 1) / kCTile;
    case C_AGG: return q.na;
    case C_CELL: return q.nc;
    case C_TILE: return q.nt;
    case C_CHUNK: return q.nch;
    case C_PILE: return 1;
    case C_TNODE: { int D = tree_depth(w, q); return D ? (((int64_t)1 << (3 * (D + 1))) - 1) / 7 : 0; }
    case C_TLEAF: { int D = tree_depth(w, q); return D ? (int64_t)1 << (3 * D) : 0; }
    // per-sphere tree arrays, indexed like the sphere arrays: every pile gets
    // them while tree gravity is on, none otherwise
    case C_TSPH: return (w->grav_theta > 0 && w->precision == DEM_MIXED) ? q.ns : 0;
    default: return 0;
    }
}

struct GravPlan {
    int tile = kGravSymTile;   // symmetric form: spheres per tile
    std::vector<int4> items;
    std::vector<int64_t> base;
    std::vector<int32_t> nch;
    int64_t gp = 0;
};

bool use_sym(const dem_world *w) { return w->grav_sym; }

// Tile of the symmetric form.  512-sphere tiles unless the mixed path's
// 512-tile pairs of all piles would not fill one wave of the persistent grid
// and no pile exceeds 8,192 spheres: then 128-sphere tiles, 16 times the work
// items for the same pairs (their partial rows, 2 T x N, stay <= 17 MB).
// Measured per step, 512 -> 128: 1,000 spheres 89 -> 75 us, 5,000 97 -> 91,
// 8,000 118 -> 108.  Piles of at most 2,048 spheres use 64-sphere tiles
// (512 -> 128 -> 64: 500 spheres 93 -> 79 -> 68 us, 2,000 101 -> 83 -> 81;
// at 4,000 the two small tiles are even).
int sym_tile(dem_world *w)
{
    if (w->precision != DEM_MIXED) return kGravSymTile;
    int64_t items = 0, nmax = 0;
    for (auto &q : w->piles) {
        if (q.P.G == 0.0) continue;
        const int64_t T = (q.ns + kGravSymTile - 1) / kGravSymTile;
        items += T * (T + 1) / 2;
        nmax = std::max(nmax, q.ns);
    }
    if (nmax == 0 || nmax > kSmallTileMaxN) return kGravSymTile;
    if (w->grav_tile == kGravSymTileTiny && nmax > kTinyTileMaxN) return kGravSymTileSmall;
    if (w->grav_tile) return w->grav_tile;
    if (w->sm_count == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&w->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return kGravSymTile;
        }
    }
    const int bps = gravity_blocks_per_sm(false, 128, 4, false, true, kGravSymTile);
    cudaGetLastError();
    if (items >= (int64_t)std::max(1, bps) * w->sm_count) return kGravSymTile;
    return nmax <= kTinyTileMaxN ? kGravSymTileTiny : kGravSymTileSmall;
}

// Work items in decreasing cost, ties in generation order (a stable sort by
// cost).  Most items share the largest cost (whole tiles or j-ranges): those
// are taken first in order, and only the rest is sorted.
struct GravItem { int4 v; int64_t cost; };
void order_items(const std::vector<GravItem> &its, std::vector<int4> &out)
{
    int64_t top = 0;
    for (const auto &x : its) top = std::max(top, x.cost);
    out.reserve(out.size() + its.size());
    std::vector<GravItem> rest;
    for (const auto &x : its) {
        if (x.cost == top) out.push_back(x.v);
        else rest.push_back(x);
    }
    std::stable_sort(rest.begin(), rest.end(), [](const GravItem &x, const GravItem &y) { return x.cost > y.cost; });
    for (const auto &x : rest) out.push_back(x.v);
}

GravPlan plan_gravity(dem_world *w)
{
    GravPlan g;
    if (w->grav_theta > 0 && w->precision == DEM_MIXED) {   // tree gravity: no direct items
        for (size_t p = 0; p < w->piles.size(); ++p) { g.nch.push_back(1); g.base.push_back(-1); }
        return g;
    }
    if (use_sym(w)) {
        const int64_t tile = g.tile = sym_tile(w);
        // items: every pair of tiles (a, b), a <= b; partial rows
        // [b][i] and [T + a][j] (2 T rows of ns) for piles with more than one tile
        std::vector<GravItem> its;
        for (size_t p = 0; p < w->piles.size(); ++p) {
            const PileHost &q = w->piles[p];
            const int64_t T = (q.ns + tile - 1) / tile;
            if (q.P.G == 0.0) {
                g.nch.push_back(1);
                g.base.push_back(-1);
                continue;
            }
            g.nch.push_back((int32_t)T);
            if (T > 1 && w->precision == DEM_FP64) {
                g.base.push_back(g.gp);
                g.gp += 2 * T * q.ns;
            } else {   // one tile, or the mixed path's integer accumulators
                g.base.push_back(-1);
            }
            for (int64_t ta = 0; ta < T; ++ta)
                for (int64_t tb = ta; tb < T; ++tb) {
                    int64_t nb = std::min<int64_t>(tile, q.ns - tb * tile);
                    its.push_back({make_int4((int)p, (int)ta, (int)tb, 0), nb});
                }
        }
        order_items(its, g.items);
        return g;
    }
    int BI = w->grav_block * w->grav_ib;
    std::vector<GravItem> its;
    for (size_t p = 0; p < w->piles.size(); ++p) {
        const PileHost &q = w->piles[p];
        int64_t ns = q.ns;
        int64_t nch = 1;
        int64_t jlen = w->grav_jchunk;
        if (jlen <= 0) jlen = std::max<int64_t>(w->grav_block, (int64_t)(w->grav_item / BI));
        if (ns > jlen) nch = (ns + jlen - 1) / jlen;
        int64_t jc = (ns + nch - 1) / nch;
        if (q.P.G == 0.0) {   // no self-gravity: no work items; fg stays zero from set-up
            g.nch.push_back(1);
            g.base.push_back(-1);
            continue;
        }
        g.nch.push_back((int32_t)nch);
        if (nch > 1) {
            g.base.push_back(g.gp);
            g.gp += nch * ns;
        } else {
            g.base.push_back(-1);
        }
        for (int64_t i0 = 0; i0 < ns; i0 += BI)
            for (int64_t c = 0; c < nch; ++c) {
                int64_t j0 = c * jc, j1 = std::min(ns, (c + 1) * jc);
                its.push_back({make_int4((int)p, (int)i0, (int)j0, (int)j1), j1 - j0});
            }
    }
    order_items(its, g.items);
    return g;
}

int64_t need_of(const dem_world *w, Cls c, const std::vector<PileHost> &piles, const GravPlan *gp)
{
    if (c == C_GITEM) return gp ? (int64_t)gp->items.size() : 0;
    if (c == C_GPART) return gp ? gp->gp : 0;
    int64_t n = 0;
    for (auto &q : piles) n += pile_count(w, q, c);
    return n;
}

// Move to a new layout: `newp` is the new pile list (a subset of the old one
// in the same order, possibly plus piles appended at the end).  Preserved
// fields of surviving piles are copied range by range.  Capacities grow by
// 1.5x when exceeded; a shrinking layout reuses the capacity.
dem_status relayout(dem_world *w, const std::vector<PileHost> &newp, const GravPlan *gp)
{
    int64_t need[C_NCLS], ncap[C_NCLS];
    bool grow = false;
    for (int c = 0; c < C_NCLS; ++c) {
        need[c] = need_of(w, (Cls)c, newp, gp);
        ncap[c] = w->cap[c];
        if (need[c] > w->cap[c]) {
            ncap[c] = std::max<int64_t>(need[c], (int64_t)(1.5 * (double)w->cap[c]));
            grow = true;
        }
    }
    // bytes after the change (each field 256-byte aligned in one slab)
    size_t total = 0;
    for (auto &f : w->fields) total += (f.el * (size_t)ncap[f.cls] + 255) / 256 * 256;
    if (w->budget && total > w->budget)
        return fail(w, DEM_ERR_OOM, "HBM budget exceeded: need %zu bytes, budget %zu", total, w->budget);
    // old and new offsets of the surviving piles
    std::vector<int64_t> old_off[C_NCLS];
    for (int c = 0; c < C_NCLS; ++c) {
        int64_t o = 0;
        for (auto &q : w->piles) { old_off[c].push_back(o); o += pile_count(w, q, (Cls)c); }
    }
    // map each new pile to its old slot (-1 = new)
    std::vector<int> from(newp.size(), -1);
    for (size_t k = 0; k < newp.size(); ++k)
        for (size_t o = 0; o < w->piles.size(); ++o)
            if (w->piles[o].id == newp[k].id) from[k] = (int)o;
    bool moved = grow || newp.size() < w->piles.size();
    for (size_t k = 0; k < newp.size() && !moved; ++k)
        if (from[k] >= 0 && (from[k] != (int)k || newp[k].ne != w->piles[from[k]].ne)) moved = true;
    if (!moved) {
        // only the transient classes may need new capacity (none grew)
        return DEM_OK;
    }
    // one slab for every field (offsets 256-byte aligned): one allocator call per layout
    std::vector<void *> fresh(w->fields.size(), nullptr);
    const size_t slab_bytes = total;
    char *slab = (char *)dev_alloc(w, slab_bytes);
    if (!slab) return fail(w, DEM_ERR_OOM, "device allocation of %zu bytes failed", slab_bytes);
    for (size_t f = 0, o = 0; f < w->fields.size(); ++f) {
        fresh[f] = slab + o;
        o += (w->fields[f].el * (size_t)ncap[w->fields[f].cls] + 255) / 256 * 256;
    }
    for (size_t f = 0; f < w->fields.size(); ++f) {
        const Field &fd = w->fields[f];
        if (!fd.keep || *fd.ptr == nullptr) continue;
        int64_t o = 0;
        for (size_t k = 0; k < newp.size(); ++k) {
            int64_t n = pile_count(w, newp[k], fd.cls);
            if (from[k] >= 0 && n > 0) {
                // a class may grow for a surviving pile (its list entries): copy what it had
                const int64_t nold = pile_count(w, w->piles[from[k]], fd.cls);
                size_t src = (size_t)old_off[fd.cls][from[k]] * fd.el;
                CU(cudaMemcpyAsync((char *)fresh[f] + (size_t)o * fd.el, (char *)*fd.ptr + src,
                                   (size_t)std::min(n, nold) * fd.el, cudaMemcpyDeviceToDevice, w->stream));
            }
            o += n;
        }
    }
    CU(cudaStreamSynchronize(w->stream));
    dev_free(w, w->slab);
    w->slab = slab;
    for (size_t f = 0; f < w->fields.size(); ++f) *w->fields[f].ptr = fresh[f];
    for (int c = 0; c < C_NCLS; ++c) w->cap[c] = ncap[c];
    w->held = slab_bytes;
    return DEM_OK;
}

void split(double x, float &hi, float &lo);

// Rebuild the device pile table, ids and the gravity plan; capture the graph.
dem_status upload_tables(dem_world *w, const GravPlan &gp)
{
    std::vector<PileStatic> ps;
    std::vector<int4> ctiles;
    int64_t s0 = 0, a0 = 0, c0 = 0, ch0 = 0, tn0 = 0, tl0 = 0, tg0 = 0, e0 = 0;
    std::vector<int32_t> tnode_pile, tleaf_pile;
    w->tree_maxD = 0;
    for (auto &q : w->piles) {
        PileStatic S{};
        S.tD = tree_depth(w, q);
        S.theta = (float)w->grav_theta;
        S.tnode0 = tn0;
        S.tleaf0 = tl0;
        S.tg0 = tg0;
        tg0 += (q.ns + 31) / 32;
        const int64_t nn = pile_count(w, q, C_TNODE), nl = pile_count(w, q, C_TLEAF);
        tnode_pile.insert(tnode_pile.end(), nn, (int32_t)ps.size());
        tleaf_pile.insert(tleaf_pile.end(), nl, (int32_t)ps.size());
        tn0 += nn;
        tl0 += nl;
        w->tree_maxD = std::max(w->tree_maxD, S.tD);
        S.s0 = s0; S.ns = q.ns; S.a0 = a0; S.na = q.na; S.c0 = c0; S.nc = q.nc;
        S.ch0 = ch0; S.nch = q.nch; S.t0 = c0 / kScanTile; S.nt = q.nt;
        S.nx = q.nx; S.ny = q.ny; S.nz = q.nz; S.K = w->K;
        S.cell = q.cell; S.inv_cell = 1.0 / q.cell;
        S.skin = skin_of(w, q);
        // contact lists and tiles; fixed-point quantum q = 2^qexp with
        // 2^31 q >= 10.5 x the largest radius (depends on nothing else, so
        // results do not depend on the cell size or the skin)
        S.e0 = e0;
        S.ne = pile_count(w, q, C_ENT);
        S.ct0 = (int64_t)ctiles.size();
        S.nct = pile_count(w, q, C_CTILE);
        for (int64_t t = 0; t < S.nct; ++t)
            ctiles.push_back(make_int4((int)ps.size(), (int)(t * kCTile),
                                       (int)std::min<int64_t>(kCTile, q.ns - t * kCTile), 0));
        e0 += S.ne;
        S.qexp = (int32_t)std::ceil(std::log2(10.5 * q.smax)) - 31;
        S.skin_q = (int64_t)std::llround(S.skin / std::ldexp(1.0, S.qexp));
        const dem_params &P = q.P;
        S.G = P.G; S.h = P.dt; S.kn = P.kn; S.kt = P.kt; S.cn = P.cn; S.ct = P.ct;
        {
            const double law[9] = {P.kn, P.kt, P.cn, P.ct, P.mu_s, P.mu_r, P.mu_t, P.w0, P.dt};
            for (int c = 0; c < 9; ++c) S.lawf[c] = (float)law[c];
            split(P.dt, S.hff[0], S.hff[1]);
            for (int c = 0; c < 3; ++c) S.spin_f[c] = (float)P.spin_inc[c];
            S.yorp = (P.spin_inc[0] != 0.0 || P.spin_inc[1] != 0.0 || P.spin_inc[2] != 0.0) ? 1 : 0;
        }
        S.mu_s = P.mu_s; S.mu_r = P.mu_r; S.mu_t = P.mu_t; S.w0 = P.w0;
        S.eps2 = P.eps_soft * P.eps_soft;
        S.ext_mass = P.ext_mass; S.M_total = q.M_total;
        {
            // a pair term of the gravity sum is at most m_j x 0.385 / eps^2
            // (the maximum of d / (d^2 + eps^2)^1.5), and at most m_j x 4 / s_min^2
            // while spheres of different aggregates stay > s_min / 2 apart, so a
            // sphere's sum of |terms| is below B = M x min(...); margin for the
            // FP32 masses and rounding
            double b = 4.0 / (q.smin * q.smin);
            if (S.eps2 > 0) b = std::min(b, 0.3849 / S.eps2);
            const double B = q.M_total * b * 1.01;
            int k = (B > 0 && std::isfinite(B)) ? (int)std::floor(61.0 - std::log2(B)) : 0;
            k = std::max(-120, std::min(120, k));   // a normal FP32 power of two
            S.gscale_f = std::ldexp(1.0f, k);
            S.ginv = std::ldexp(1.0, -k);
        }
        for (int c = 0; c < 3; ++c) S.spin_inc[c] = P.spin_inc[c];
        S.rot_tol = P.rot_tol;
        ps.push_back(S);
        s0 += q.ns; a0 += q.na; c0 += q.nc; ch0 += q.nch;
    }
    w->Z.N = s0; w->Z.A = a0; w->Z.C = c0; w->Z.T = c0 / kScanTile; w->Z.CH = ch0;
    w->Z.CT = (int64_t)ctiles.size();
    w->Z.E = e0;
    w->Z.P = (int64_t)w->piles.size();
    w->Z.GI = (int64_t)gp.items.size();
    w->Z.GP = gp.gp;
    w->Z.K = w->K;
    w->Z.TN = tn0;
    w->Z.TL = tl0;
    w->Z.TG = tg0;
    w->Z.adapt = 0;
    w->Z.grav = 0;
    for (auto &q : w->piles) {
        if (q.P.rot_tol > 0) w->Z.adapt = 1;
        if (q.P.G != 0.0) w->Z.grav = 1;
    }
    if (w->sm_count == 0) {
        int dev = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&w->sm_count, cudaDevAttrMultiProcessorCount, dev));
    }
    w->Z.gtile = gp.tile;
    w->Z.icap = w->contact_inbox;
    w->Z.gacc_on = (w->precision == DEM_MIXED && use_sym(w) && !(w->grav_theta > 0)) ? 1 : 0;
    w->Z.cmode = w->contact_mode;
    int bps = gravity_blocks_per_sm(w->precision == DEM_FP64, w->grav_block, w->grav_ib, w->grav_pack,
                                    use_sym(w), gp.tile);
    CU(cudaGetLastError());
    CU(contact_setup(w->precision == DEM_FP64, w->K));
    w->Z.GB = (int64_t)std::max(1, bps) * w->sm_count;
    if (!ps.empty()) {
        CU(cudaMemcpyAsync(w->A.ps, ps.data(), sizeof(PileStatic) * ps.size(),
                           cudaMemcpyHostToDevice, w->stream));
        CU(cudaMemcpyAsync(w->A.gpart_base, gp.base.data(), 8 * gp.base.size(),
                           cudaMemcpyHostToDevice, w->stream));
        CU(cudaMemcpyAsync(w->A.gnchunk, gp.nch.data(), 4 * gp.nch.size(),
                           cudaMemcpyHostToDevice, w->stream));
    }
    if (!gp.items.empty())
        CU(cudaMemcpyAsync(w->A.gitems, gp.items.data(), 16 * gp.items.size(),
                           cudaMemcpyHostToDevice, w->stream));
    if (!ctiles.empty()) {
        CU(cudaMemcpyAsync(w->A.ctile, ctiles.data(), 16 * ctiles.size(), cudaMemcpyHostToDevice, w->stream));
        CU(cudaStreamSynchronize(w->stream));   // the host vector goes out of scope
    }
    if (tn0 > 0) {
        CU(cudaMemcpyAsync(w->A.tnode_pile, tnode_pile.data(), 4 * tnode_pile.size(),
                           cudaMemcpyHostToDevice, w->stream));
        CU(cudaMemcpyAsync(w->A.tleaf_pile, tleaf_pile.data(), 4 * tleaf_pile.size(),
                           cudaMemcpyHostToDevice, w->stream));
        CU(cudaStreamSynchronize(w->stream));   // host vectors go out of scope
    }
    // the persistent gravity grid's work counter (it resets itself after each launch)
    CU(cudaMemsetAsync(w->A.gcounter, 0, sizeof(int32_t), w->stream));
    // the mixed path's gravity accumulators (each step's conversion leaves them at zero)
    if (w->A.gacc && w->Z.N > 0) CU(cudaMemsetAsync(w->A.gacc, 0, 32 * (size_t)w->Z.N, w->stream));
    // arrival counters of the pile reductions (each reduction leaves them at zero)
    if (w->Z.P > 0) CU(cudaMemsetAsync(w->A.pile_arrive, 0, sizeof(int32_t) * (size_t)w->Z.P, w->stream));
    launch_fill_ids(w->A, w->Z, w->stream);
    // a new layout leaves the transient sort and hit lists undefined
    launch_force_rebuild(w->A, w->Z, -1, w->stream);
    CU(cudaGetLastError());
    return DEM_OK;
}

bool any_watch(const dem_world *w)
{
    for (auto &q : w->piles)
        if (q.watch_on) return true;
    return false;
}

// Radius-growth watches: evaluated after the step's last phase.
void enqueue_watch(dem_world *w)
{
    if (any_watch(w)) launch_bulk(w->A, w->Z, 1, -1, w->stream);
}

void enqueue_phase(dem_world *w, int ph)
{
    set_launch_pdl(w->Z.N);
    const Arrays &a = w->A;
    const Sizes &z = w->Z;
    bool d = w->precision == DEM_FP64;
    cudaStream_t st = w->stream;
    switch (ph) {
    case DEM_K_AGG_BEGIN: launch_agg_begin(a, z, d, st); break;
    case DEM_K_PILE_BEGIN: launch_pile_begin(a, z, st); break;
    case DEM_K_KEYS: launch_keys(a, z, d, st); break;
    case DEM_K_SCAN: launch_scan(a, z, st); break;
    case DEM_K_SCATTER: launch_scatter(a, z, st); break;
    case DEM_K_CELL_ORDER: launch_cell_order(a, z, st); break;
    case DEM_K_GATHER: launch_gather(a, z, d, st); break;
    case DEM_K_CONTACT: launch_contact(a, z, d, w->K, st); break;
    case DEM_K_GRAVITY:
        if (z.TN > 0) launch_tree_gravity(a, z, w->tree_maxD, w->grav_order, st);
        else launch_gravity(a, z, d, w->grav_block, w->grav_ib, w->grav_pack, use_sym(w), st);
        break;
    case DEM_K_AGG_END: launch_agg_end(a, z, d, st); break;
    case DEM_K_PILE_END: launch_pile_end(a, z, st); break;
    default: break;
    }
}

dem_status prepare(dem_world *w)
{
    if (w->graph_valid) return DEM_OK;
    Range range("dem: layout and step graph");
    GravPlan gp = plan_gravity(w);
    dem_status s = relayout(w, w->piles, &gp);
    if (s != DEM_OK) return s;
    s = upload_tables(w, gp);
    if (s != DEM_OK) return s;
    if (w->exec) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
    }
    if (w->piles.empty()) {
        w->graph_valid = true;
        return DEM_OK;
    }
    CU(cudaStreamSynchronize(w->stream));
    cudaGraph_t g = nullptr;
    if (w->timed_kernel >= 0 && !w->kev[0]) {
        CU(cudaEventCreate(&w->kev[0]));
        CU(cudaEventCreate(&w->kev[1]));
    }
    CU(cudaStreamBeginCapture(w->stream, cudaStreamCaptureModeThreadLocal));
    for (int ph = 0; ph < DEM_K_COUNT; ++ph) {
        if (ph == w->timed_kernel) cudaEventRecordWithFlags(w->kev[0], w->stream, cudaEventRecordExternal);
        enqueue_phase(w, ph);
        if (ph == w->timed_kernel) cudaEventRecordWithFlags(w->kev[1], w->stream, cudaEventRecordExternal);
    }
    enqueue_watch(w);
    cudaError_t e = cudaStreamEndCapture(w->stream, &g);
    if (e != cudaSuccess) return fail(w, DEM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    int32_t nk = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    w->graph_kernels = nk;
    e = cudaGraphInstantiate(&w->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(w, DEM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    w->graph_valid = true;
    return DEM_OK;
}

int find_pile(const dem_world *w, int32_t id)
{
    for (size_t k = 0; k < w->piles.size(); ++k)
        if (w->piles[k].id == id) return (int)k;
    return -1;
}

// Wait for the flag words of the last dem_step and turn newly failed piles
// into a status.
dem_status collect_flags(dem_world *w)
{
    if (!w->pending) return DEM_OK;
    w->pending = false;
    CU(cudaEventSynchronize(w->ev_flags));
    dem_status st = DEM_OK;
    for (size_t k = 0; k < w->piles.size() && (int64_t)k < w->pending_n; ++k) {
        PileHost &q = w->piles[k];
        const PileDyn &D = w->h_dyn[k];
        if (!q.reported && D.failed) {
            q.reported = true;
            if (D.flags & DEM_FLAG_NONFINITE) {
                st = DEM_ERR_NONFINITE;
                fail(w, st, "pile %d: state became non-finite; pile frozen", q.id);
            } else if (D.flags & DEM_FLAG_GRAV_RANGE) {
                st = DEM_ERR_NONFINITE;
                fail(w, st, "pile %d: gravity sum beyond the range of its accumulators; pile frozen", q.id);
            } else if (st == DEM_OK) {
                st = DEM_ERR_SLOTS;
                fail(w, st, "pile %d: more contacts than %d history slots; pile frozen", q.id, w->K);
            }
        }
    }
    return st;
}

dem_status issue_flags_readback(dem_world *w)
{
    int64_t P = (int64_t)w->piles.size();
    if (P == 0) return DEM_OK;
    if (P > w->h_dyn_cap) {
        if (w->h_dyn) cudaFreeHost(w->h_dyn);
        w->h_dyn = nullptr;
        CU(cudaMallocHost((void **)&w->h_dyn, sizeof(PileDyn) * (size_t)P * 2));
        w->h_dyn_cap = P * 2;
    }
    CU(cudaMemcpyAsync(w->h_dyn, w->A.pd, sizeof(PileDyn) * (size_t)P, cudaMemcpyDeviceToHost,
                       w->stream));
    CU(cudaEventRecord(w->ev_flags, w->stream));
    w->pending = true;
    w->pending_n = P;
    return DEM_OK;
}

dem_status set_enabled(dem_world *w, const int32_t *ids, int32_t n)
{
    std::vector<int32_t> en(w->piles.size(), ids ? 0 : 1);
    if (ids) {
        for (int32_t k = 0; k < n; ++k) {
            int s = find_pile(w, ids[k]);
            if (s < 0) return fail(w, DEM_ERR_ARG, "unknown pile id %d", ids[k]);
            en[s] = 1;
        }
    }
    if (!en.empty())
        CU(cudaMemcpyAsync(w->A.enabled, en.data(), 4 * en.size(), cudaMemcpyHostToDevice, w->stream));
    return DEM_OK;
}

bool finite_all(const double *x, int64_t n)
{
    for (int64_t k = 0; k < n; ++k)
        if (!std::isfinite(x[k])) return false;
    return true;
}

void split(double x, float &hi, float &lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Mixed path: each FP64 slot of the aggregate state (r, v, q, w_body, a, N)
// and of 1/M holds the float-float pair (hi, lo) of its value.  hi is the
// value rounded to FP32 and lo the rounded remainder, so hi = fl(hi + lo):
// a value read out and written back gives the same pair.
double pack_ff(double x)
{
    float2 f;
    split(x, f.x, f.y);
    double d;
    std::memcpy(&d, &f, sizeof d);
    return d;
}
double unpack_ff(double d)
{
    float2 f;
    std::memcpy(&f, &d, sizeof f);
    return (double)f.x + (double)f.y;
}
void unpack_all(const dem_world *w, double *x, int64_t n)
{
    if (w->precision == DEM_MIXED)
        for (int64_t k = 0; k < n; ++k) x[k] = unpack_ff(x[k]);
}
std::vector<double> packed(const dem_world *w, const double *x, int64_t n)
{
    std::vector<double> out(x, x + n);
    if (w->precision == DEM_MIXED)
        for (auto &d : out) d = pack_ff(d);
    return out;
}

void rotmat(const double *q, double *R)
{
    double w0 = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w0 * z);    R[2] = 2 * (x * z + w0 * y);
    R[3] = 2 * (x * y + w0 * z);    R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w0 * x);
    R[6] = 2 * (x * z - w0 * y);    R[7] = 2 * (y * z + w0 * x);    R[8] = 1 - 2 * (x * x + y * y);
}

// Wrapped grid for one pile: cell >= 2 x largest radius (times the tuning
// factor), dims >= 3 so the 27 neighbour cells are distinct, total cells
// capped near 4 x spheres by enlarging the cell.
// Cell edge and wrapped grid dims for an extent `ext` (plus `pad` cells per
// axis): cell = base x cell_factor, at least the radii sum plus the skin,
// enlarged until the grid holds at most max(4 N, 27) cells.
void set_grid(const dem_world *w, PileHost &q, const double *ext, int pad)
{
    double cell = (q.P.cell_size > 0 ? q.P.cell_size : min_cell(q)) * w->cell_factor;
    cell = std::max(cell, min_cell(q) + w->skin_frac * q.smax);
    int64_t cap = std::max<int64_t>(4 * q.ns, 27);
    int dims[3];
    for (int it = 0; it < 200; ++it) {
        int64_t tot = 1;
        for (int c = 0; c < 3; ++c) {
            int64_t n = (int64_t)std::ceil(ext[c] / cell) + pad;
            n = std::max<int64_t>(3, std::min<int64_t>(n, 1 << 20));
            dims[c] = (int)n;
            tot *= n;
        }
        if (tot <= cap) break;
        cell *= std::cbrt((double)tot / (double)cap) * 1.01;
    }
    q.cell = cell;
    q.nx = dims[0]; q.ny = dims[1]; q.nz = dims[2];
    const int64_t cells = cell_count(q.nx, q.ny, q.nz);
    q.nc = (cells + kScanTile - 1) / kScanTile * kScanTile;
    q.nt = q.nc / kScanTile;
}

// New grids for every pile (cells, candidate lists and the sort are rebuilt at
// every pile's next step; the history is carried over by partner index).
dem_status regrid(dem_world *w);

// lo, hi: the box of the sphere centres relative to the pile's COM (the grid
// spans it and the origin).
void choose_grid(const dem_world *w, PileHost &q, const double (&lo_rel)[3], const double (&hi_rel)[3])
{
    double lo[3], hi[3];
    for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(0.0, lo_rel[c]);
        hi[c] = std::max(0.0, hi_rel[c]);
    }
    double ext[3];
    for (int c = 0; c < 3; ++c) ext[c] = hi[c] - lo[c] + 2.0 * q.smax;
    set_grid(w, q, ext, 2);
    for (int c = 0; c < 3; ++c) q.ext[c] = q.cell * (c == 0 ? q.nx : c == 1 ? q.ny : q.nz);
}

dem_status regrid(dem_world *w)
{
    std::vector<PileHost> newp = w->piles;
    for (auto &q : newp) {
        set_grid(w, q, q.ext, 0);
        size_lists(w, q);
    }
    dem_status s = relayout(w, newp, nullptr);
    if (s != DEM_OK) return s;
    w->piles = newp;
    return DEM_OK;
}

}  // namespace

// =====================================================================
extern "C" {

dem_status dem_create(void *cuda_stream, size_t hbm_budget_bytes, dem_world **out)
{
    if (!out) return DEM_ERR_ARG;
    dem_world *w = new dem_world();
    w->stream = (cudaStream_t)cuda_stream;
    w->budget = hbm_budget_bytes;
    if (w->stream == nullptr) {   // graphs cannot be captured on the legacy stream
        if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete w;
            return DEM_ERR_CUDA;
        }
        w->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&w->ev_flags, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete w;
        return DEM_ERR_CUDA;
    }
    *out = w;
    return DEM_OK;
}

dem_status dem_set_allocator(dem_world *w, dem_alloc_fn alloc, dem_free_fn free_fn, void *ctx)
{
    if (!w) return DEM_ERR_ARG;
    if (w->held > 0) return fail(w, DEM_ERR_STATE, "allocator must be set before adding piles");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(w, DEM_ERR_ARG, "alloc and free must both be set or both NULL");
    w->alloc = alloc;
    w->free_fn = free_fn;
    w->ctx = ctx;
    return DEM_OK;
}

dem_status dem_add_aggregates(dem_world *w, const dem_params *p, int64_t n_agg,
                              const int32_t *spa, const double *pos, const double *rad,
                              const double *dens, const double *agg_vel, const double *agg_omega,
                              int32_t *out_pile_id)
{
    Range range("dem_add_aggregates");
    if (!w) return DEM_ERR_ARG;
    if (!p || !spa || !pos || !rad || !dens || !out_pile_id || n_agg <= 0)
        return fail(w, DEM_ERR_ARG, "NULL argument or n_agg <= 0");
    if (n_agg > (int64_t)1 << 30) return fail(w, DEM_ERR_ARG, "too many aggregates");
    if (p->precision != DEM_FP64 && p->precision != DEM_MIXED)
        return fail(w, DEM_ERR_ARG, "precision must be DEM_FP64 or DEM_MIXED");
    if (w->precision >= 0 && p->precision != w->precision)
        return fail(w, DEM_ERR_ARG, "all piles of a world must use the same precision");
    if (p->max_contacts < 1 || p->max_contacts > kMaxK)
        return fail(w, DEM_ERR_ARG, "max_contacts must be in 1..%d", kMaxK);
    if (w->K >= 0 && p->max_contacts != w->K)
        return fail(w, DEM_ERR_ARG, "all piles of a world must use the same max_contacts");
    const double scal[] = {p->G, p->dt, p->kn, p->kt, p->cn, p->ct, p->mu_s, p->mu_r, p->mu_t,
                           p->w0, p->eps_soft, p->cell_size, p->ext_mass, p->rot_tol};
    if (!finite_all(scal, 14) || !finite_all(p->ext_pos, 3) || !finite_all(p->ext_vel, 3) ||
        !finite_all(p->spin_inc, 3))
        return fail(w, DEM_ERR_ARG, "non-finite parameter");
    if (!(p->dt > 0) || p->kn < 0 || p->kt < 0 || p->cn < 0 || p->ct < 0 || p->mu_s < 0 ||
        p->mu_r < 0 || p->mu_t < 0 || !(p->w0 > 0) || p->eps_soft < 0 || p->G < 0 ||
        p->ext_mass < 0 || p->cell_size < 0 || p->rot_tol < 0)
        return fail(w, DEM_ERR_ARG, "parameter out of range (dt > 0, w0 > 0, others >= 0)");
    int64_t N = 0;
    for (int64_t a = 0; a < n_agg; ++a) {
        if (spa[a] < 1) return fail(w, DEM_ERR_ARG, "aggregate %lld has %d spheres", (long long)a, spa[a]);
        N += spa[a];
    }
    if (N > ((int64_t)1 << 30)) return fail(w, DEM_ERR_ARG, "too many spheres");

    // ---- host set-up in FP64 (Sec. 2.2.1) ----
    // Aggregates are set up in 16 fixed ranges (on up to 16 host threads for
    // large piles), each range also checking its inputs, putting its part of
    // the state into the world's formats and boxing its sphere centres; the
    // pile sums are added range by range in order, so the result does not
    // depend on the number of threads.
    const int A = (int)n_agg;
    // Host arrays of the set-up, carved from one staging buffer that the
    // world keeps between calls (pinned when possible): no allocation, page
    // faults or zero fill per call, and the uploads below run asynchronously
    // from it.  Every array is fully written before it is read or uploaded.
    int32_t *first, *sph_agg, *iota;
    double *m, *b, *M, *I, *Iinv, *q, *r, *v, *wb, *pk_invM, *pk_r, *pk_v, *pk_q, *pk_wb;
    float4 *bh, *bl;
    float *I32, *Iinv32, *aref;
    auto carve = [&](char *base) -> size_t {
        size_t off = 0;
        auto take = [&](auto *&ptr, int64_t n) {
            off = (off + 255) & ~(size_t)255;
            ptr = reinterpret_cast<std::remove_reference_t<decltype(ptr)>>(reinterpret_cast<uintptr_t>(base) + off);
            off += (size_t)n * sizeof(*ptr);
        };
        take(first, A); take(sph_agg, N); take(iota, N);
        take(m, N); take(b, 3 * N); take(M, A); take(I, 9 * A); take(Iinv, 9 * A);
        take(q, 4 * A); take(r, 3 * A); take(v, 3 * A); take(wb, 3 * A);
        take(pk_invM, A); take(pk_r, 3 * A); take(pk_v, 3 * A); take(pk_q, 4 * A); take(pk_wb, 3 * A);
        take(bh, N); take(bl, N); take(I32, 9 * A); take(Iinv32, 9 * A); take(aref, 8 * A);
        return off;
    };
    {
        const size_t need = carve(nullptr);
        if (need > w->h_stage_cap) {
            if (w->h_stage) {
                if (w->h_stage_pinned) cudaFreeHost(w->h_stage);
                else std::free(w->h_stage);
            }
            w->h_stage = nullptr;
            w->h_stage_cap = 0;
            const size_t cap = need + need / 4;
            void *hp = nullptr;
            // pinned up to 1 GiB; pageable above that or if pinning fails
            if (cap <= ((size_t)1 << 30) && cudaMallocHost(&hp, cap) == cudaSuccess) {
                w->h_stage_pinned = true;
            } else {
                cudaGetLastError();
                hp = std::malloc(cap);
                w->h_stage_pinned = false;
            }
            if (!hp) return fail(w, DEM_ERR_OOM, "host staging of %zu bytes failed", cap);
            w->h_stage = (char *)hp;
            w->h_stage_cap = cap;
        }
        carve(w->h_stage);
    }
    {
        int64_t k = 0;
        for (int a = 0; a < A; ++a) { first[a] = (int32_t)k; k += spa[a]; }
    }
    struct Part {
        double smax = 0, smin = HUGE_VAL, Mtot = 0, Rp[3] = {0, 0, 0}, Vp[3] = {0, 0, 0};
        double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
        bool nonfinite = false, nonpositive = false;
        int bad = -1;   // first aggregate of the range with a singular inertia tensor
    };
    const bool mixed = p->precision == DEM_MIXED;
    constexpr int kRanges = 16;
    Part part[kRanges];
    auto setup_range = [&](int rg) {
        Part &P = part[rg];
        const int a_lo = (int)((int64_t)A * rg / kRanges), a_hi = (int)((int64_t)A * (rg + 1) / kRanges);
        {
            // inputs of the range: finite, radius and density > 0; box of the centres
            const int64_t i_lo = first[a_lo], i_hi = a_hi < A ? (int64_t)first[a_hi] : N;
            for (int64_t i = i_lo; i < i_hi; ++i) {
                for (int c = 0; c < 3; ++c) {
                    const double x = pos[3 * i + c];
                    if (!std::isfinite(x)) P.nonfinite = true;
                    P.lo[c] = std::min(P.lo[c], x);
                    P.hi[c] = std::max(P.hi[c], x);
                }
                if (!std::isfinite(rad[i]) || !std::isfinite(dens[i])) P.nonfinite = true;
                else if (!(rad[i] > 0) || !(dens[i] > 0)) P.nonpositive = true;
            }
            for (int a = a_lo; a < a_hi; ++a)
                for (int c = 0; c < 3; ++c)
                    if ((agg_vel && !std::isfinite(agg_vel[3 * a + c])) ||
                        (agg_omega && !std::isfinite(agg_omega[3 * a + c])))
                        P.nonfinite = true;
            if (P.nonfinite || P.nonpositive) return;
        }
        for (int a = a_lo; a < a_hi; ++a) {
            int64_t k = first[a];
            // mass-weighted mean about the first member: a one-sphere aggregate
            // gets its COM exactly at the sphere (zero offset, zero lever)
            double Ma = 0, c[3] = {0, 0, 0}, x0[3] = {pos[3 * k], pos[3 * k + 1], pos[3 * k + 2]};
            for (int t = 0; t < spa[a]; ++t, ++k) {
                m[k] = dens[k] * (4.0 / 3.0) * M_PI * rad[k] * rad[k] * rad[k];
                sph_agg[k] = a;
                Ma += m[k];
                for (int d = 0; d < 3; ++d) c[d] += m[k] * (pos[3 * k + d] - x0[d]);
                P.smax = std::max(P.smax, rad[k]);
                P.smin = std::min(P.smin, rad[k]);
            }
            for (int d = 0; d < 3; ++d) c[d] = x0[d] + c[d] / Ma;
            M[a] = Ma;
            double T[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int64_t i = first[a]; i < first[a] + spa[a]; ++i) {
                double bi[3];
                for (int d = 0; d < 3; ++d) bi[d] = b[3 * i + d] = pos[3 * i + d] - c[d];
                double bb = bi[0] * bi[0] + bi[1] * bi[1] + bi[2] * bi[2];
                double sph = 0.4 * m[i] * rad[i] * rad[i];
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y)
                        T[3 * x + y] += (x == y ? sph + m[i] * bb : 0.0) - m[i] * bi[x] * bi[y];
            }
            // inverse by cofactors
            double c00 = T[4] * T[8] - T[5] * T[7], c01 = T[5] * T[6] - T[3] * T[8],
                   c02 = T[3] * T[7] - T[4] * T[6];
            double det = T[0] * c00 + T[1] * c01 + T[2] * c02;
            if (!(std::fabs(det) > 0) || !std::isfinite(det)) {
                if (P.bad < 0) P.bad = a;
                continue;
            }
            double inv[9] = {c00, T[2] * T[7] - T[1] * T[8], T[1] * T[5] - T[2] * T[4],
                             c01, T[0] * T[8] - T[2] * T[6], T[2] * T[3] - T[0] * T[5],
                             c02, T[1] * T[6] - T[0] * T[7], T[0] * T[4] - T[1] * T[3]};
            for (int e = 0; e < 9; ++e) {
                I[9 * a + e] = T[e];
                Iinv[9 * a + e] = inv[e] / det;
            }
            for (int d = 0; d < 3; ++d) {
                r[3 * a + d] = c[d];
                v[3 * a + d] = agg_vel ? agg_vel[3 * a + d] : 0.0;
                wb[3 * a + d] = agg_omega ? agg_omega[3 * a + d] : 0.0;
            }
            q[4 * a] = 1.0;
            q[4 * a + 1] = q[4 * a + 2] = q[4 * a + 3] = 0.0;
            P.Mtot += Ma;
            for (int d = 0; d < 3; ++d) { P.Rp[d] += Ma * c[d]; P.Vp[d] += Ma * v[3 * a + d]; }
            // the device formats of this aggregate: state slots (float-float
            // pairs in the mixed path), FP32 inertia copies, the list
            // reference, and its members' float-float offsets
            auto slot = [&](double x) { return mixed ? pack_ff(x) : x; };
            pk_invM[a] = slot(1.0 / Ma);
            for (int d = 0; d < 3; ++d) {
                pk_r[3 * a + d] = slot(r[3 * a + d]);
                pk_v[3 * a + d] = slot(v[3 * a + d]);
                pk_wb[3 * a + d] = slot(wb[3 * a + d]);
            }
            for (int d = 0; d < 4; ++d) pk_q[4 * a + d] = slot(q[4 * a + d]);
            for (int e = 0; e < 9; ++e) {
                I32[9 * a + e] = (float)I[9 * a + e];
                Iinv32[9 * a + e] = (float)Iinv[9 * a + e];
            }
            double bm = 0;
            for (int64_t i = first[a]; i < first[a] + spa[a]; ++i) {
                iota[i] = (int32_t)i;
                bm = std::max(bm, std::sqrt(b[3 * i] * b[3 * i] + b[3 * i + 1] * b[3 * i + 1] +
                                            b[3 * i + 2] * b[3 * i + 2]));
                if (mixed) {
                    split(b[3 * i], bh[i].x, bl[i].x);
                    split(b[3 * i + 1], bh[i].y, bl[i].y);
                    split(b[3 * i + 2], bh[i].z, bl[i].z);
                    split(rad[i], bh[i].w, bl[i].w);
                }
            }
            for (int e = 0; e < 7; ++e) aref[8 * a + e] = 0.0f;
            aref[8 * a + 7] = (float)bm * (1.0f + 1e-6f);
        }
    };
    {
        // ranges a thread could not be started for run here (no exception leaves the ABI)
        // threads: one per ~4,096 aggregates, at most one per range and per
        // host core; thread t takes ranges t, t + nt, ...
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)kRanges, (int64_t)hw, A / 4096}));
        auto run = [&](int t) {
            for (int rg = t; rg < kRanges; rg += nt) setup_range(rg);
        };
        std::vector<std::thread> pool;
        int started = 1;
        try {
            for (; started < nt; ++started) pool.emplace_back(run, started);
        } catch (...) {
        }
        run(0);
        for (int t = started; t < nt; ++t) run(t);
        for (auto &t : pool) t.join();
    }
    for (int rg = 0; rg < kRanges; ++rg)
        if (part[rg].nonfinite) return fail(w, DEM_ERR_ARG, "non-finite input");
    for (int rg = 0; rg < kRanges; ++rg)
        if (part[rg].nonpositive) return fail(w, DEM_ERR_ARG, "radius and density must be > 0");
    double smax = 0, smin = HUGE_VAL, Mtot = 0, Rp[3] = {0, 0, 0}, Vp[3] = {0, 0, 0};
    double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int rg = 0; rg < kRanges; ++rg) {
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], part[rg].lo[c]);
            hi[c] = std::max(hi[c], part[rg].hi[c]);
        }
        if (part[rg].bad >= 0)
            return fail(w, DEM_ERR_ARG, "aggregate %d has a singular inertia tensor", part[rg].bad);
        smax = std::max(smax, part[rg].smax);
        smin = std::min(smin, part[rg].smin);
        Mtot += part[rg].Mtot;
        for (int d = 0; d < 3; ++d) { Rp[d] += part[rg].Rp[d]; Vp[d] += part[rg].Vp[d]; }
    }
    for (int d = 0; d < 3; ++d) { Rp[d] /= Mtot; Vp[d] /= Mtot; }

    PileHost ph{};
    ph.id = w->next_id;
    ph.ns = N;
    ph.na = A;
    ph.nch = (A + kAggChunk - 1) / kAggChunk;
    ph.smax = smax;
    ph.smin = smin;
    ph.P = *p;
    ph.M_total = Mtot;
    {
        // the box relative to the COM (subtracting a constant keeps the order:
        // the same as the box of the differences)
        if (p->cell_size > 0 && p->cell_size < 2.0 * smax)
            return fail(w, DEM_ERR_ARG, "cell_size must be >= 2 x the largest radius");
        double lo_rel[3], hi_rel[3];
        for (int c = 0; c < 3; ++c) { lo_rel[c] = lo[c] - Rp[c]; hi_rel[c] = hi[c] - Rp[c]; }
        choose_grid(w, ph, lo_rel, hi_rel);
    }
    size_lists(w, ph);

    // ---- first pile fixes the world's precision and slot count ----
    bool first_pile = w->precision < 0;
    if (first_pile) {
        w->precision = p->precision;
        w->K = p->max_contacts;
        build_fields(w);
    }
    std::vector<PileHost> newp = w->piles;
    newp.push_back(ph);
    dem_status s = relayout(w, newp, nullptr);
    if (s != DEM_OK) {
        if (first_pile && w->piles.empty()) { w->precision = -1; w->K = -1; }
        return s;
    }
    w->piles = newp;
    w->next_id++;
    w->graph_valid = false;

    // ---- upload the new pile's ranges ----
    int64_t s0 = 0, a0 = 0;
    for (size_t t = 0; t + 1 < w->piles.size(); ++t) { s0 += w->piles[t].ns; a0 += w->piles[t].na; }
    const int slot = (int)w->piles.size() - 1;
    Arrays &D = w->A;
    cudaStream_t st = w->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) -> dem_status {
        CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
        return DEM_OK;
    };
#define UP(dst, src, bytes)                         \
    do {                                            \
        dem_status s_ = up((dst), (src), (bytes));  \
        if (s_ != DEM_OK) return s_;                \
    } while (0)
    UP(D.sph_agg + s0, sph_agg, 4 * N);
    UP(D.b64 + 3 * s0, b, 24 * N);
    UP(D.s64 + s0, rad, 8 * N);
    UP(D.m64 + s0, m, 8 * N);
    // no previous candidate lists: nothing to carry over at the first rebuild
    CU(cudaMemsetAsync(D.ccnt[0] + s0, 0, 4 * N, st));
    CU(cudaMemsetAsync(D.ccnt[1] + s0, 0, 4 * N, st));
    CU(cudaMemsetAsync(D.coff[0] + s0, 0, 4 * N, st));
    CU(cudaMemsetAsync(D.coff[1] + s0, 0, 4 * N, st));
    UP(D.pos_of_home[0] + s0, iota, 4 * N);
    UP(D.pos_of_home[1] + s0, iota, 4 * N);
    CU(cudaMemsetAsync(D.fg + s0, 0, 32 * N, st));
    if (w->precision == DEM_MIXED) {
        UP(D.bh + s0, bh, 16 * N);
        UP(D.bl + s0, bl, 16 * N);
        CU(cudaMemsetAsync(D.ftc32 + 2 * s0, 0, 32 * N, st));
    } else {
        CU(cudaMemsetAsync(D.ftc64 + 2 * s0, 0, 64 * N, st));
    }
    UP(D.agg_first + a0, first, 4 * A);
    UP(D.agg_count + a0, spa, 4 * A);
    UP(D.M + a0, M, 8 * A);
    UP(D.invM + a0, pk_invM, 8 * A);
    UP(D.I + 9 * a0, I, 72 * A);
    UP(D.Iinv + 9 * a0, Iinv, 72 * A);
    if (w->precision == DEM_MIXED) {
        UP(D.I32 + 9 * a0, I32, 36 * A);
        UP(D.Iinv32 + 9 * a0, Iinv32, 36 * A);
    }
    UP(D.r + 3 * a0, pk_r, 24 * A);
    UP(D.v + 3 * a0, pk_v, 24 * A);
    UP(D.q + 4 * a0, pk_q, 32 * A);
    UP(D.wb + 3 * a0, pk_wb, 24 * A);
    CU(cudaMemsetAsync(D.acc + 3 * a0, 0, 24 * A, st));
    CU(cudaMemsetAsync(D.torque + 3 * a0, 0, 24 * A, st));
    for (int k = 0; k < 3; ++k) CU(cudaMemsetAsync(D.out[k] + 6 * a0, 0, 48 * A, st));
    UP(D.aref + 8 * a0, aref, 32 * A);
    PileDyn dyn{};
    dyn.rebuild = 1;
    dyn.rebuilt_prev = 1;
    for (int d = 0; d < 3; ++d) {
        dyn.O[d] = Rp[d]; dyn.V[d] = Vp[d]; dyn.Rc[d] = Rp[d]; dyn.Vc[d] = Vp[d];
        dyn.hVf[d] = (float)(p->dt * Vp[d]);
        split(Rp[d], dyn.Of[d].x, dyn.Of[d].y);
        split(Vp[d], dyn.Vf[d].x, dyn.Vf[d].y);
        dyn.Rcf[d] = dyn.Of[d];
        dyn.P_pos[d] = p->ext_pos[d]; dyn.P_vel[d] = p->ext_vel[d]; dyn.P_acc[d] = 0.0;
    }
    UP(D.pd + slot, &dyn, sizeof dyn);
    PileWatch wat{};
    wat.every = 1;
    wat.fired = -1;
    UP(D.watch + slot, &wat, sizeof wat);
#undef UP
    CU(cudaStreamSynchronize(st));   // the staging buffer is free for the next call
    *out_pile_id = ph.id;
    return DEM_OK;
}

dem_status dem_step(dem_world *w, const int32_t *pile_ids, int32_t n_piles, int64_t n_steps)
{
    Range range("dem_step");
    if (!w) return DEM_ERR_ARG;
    if (n_steps < 0 || (pile_ids && n_piles < 0)) return fail(w, DEM_ERR_ARG, "negative count");
    dem_status prev = collect_flags(w);
    if (n_steps == 0 || w->piles.empty()) return prev;
    dem_status s = prepare(w);
    if (s != DEM_OK) return s;
    s = set_enabled(w, pile_ids, n_piles);
    if (s != DEM_OK) return s;
    for (int64_t t = 0; t < n_steps; ++t) CU(cudaGraphLaunch(w->exec, w->stream));
    s = issue_flags_readback(w);
    if (s != DEM_OK) return s;
    return prev;
}

dem_status dem_sync(dem_world *w)
{
    if (!w) return DEM_ERR_ARG;
    CU(cudaStreamSynchronize(w->stream));
    return collect_flags(w);
}

dem_status dem_step_profiled(dem_world *w, int64_t n_steps, int32_t which, float *ms_out)
{
    Range range("dem_step_profiled");
    if (!w) return DEM_ERR_ARG;
    if (n_steps < 0 || which < 0 || which >= DEM_K_COUNT || (n_steps > 0 && !ms_out))
        return fail(w, DEM_ERR_ARG, "bad arguments");
    dem_status prev = collect_flags(w);
    if (n_steps == 0 || w->piles.empty()) return prev;
    dem_status s = prepare(w);
    if (s != DEM_OK) return s;
    s = set_enabled(w, nullptr, 0);
    if (s != DEM_OK) return s;
    std::vector<cudaEvent_t> ev(2 * (size_t)n_steps, nullptr);
    for (auto &e : ev) CU(cudaEventCreate(&e));
    for (int64_t t = 0; t < n_steps; ++t) {
        for (int ph = 0; ph < DEM_K_COUNT; ++ph) {
            static const char *names[DEM_K_COUNT] = {"agg_begin", "pile_begin", "keys", "scan", "scatter",
                                                     "cell_order", "gather", "contact", "gravity", "agg_end",
                                                     "pile_end"};
            Range phase(names[ph]);
            if (ph == which) CU(cudaEventRecord(ev[2 * t], w->stream));
            enqueue_phase(w, ph);
            if (ph == which) CU(cudaEventRecord(ev[2 * t + 1], w->stream));
        }
        enqueue_watch(w);
    }
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(w->stream));
    for (int64_t t = 0; t < n_steps; ++t) CU(cudaEventElapsedTime(ms_out + t, ev[2 * t], ev[2 * t + 1]));
    for (auto &e : ev) cudaEventDestroy(e);
    s = issue_flags_readback(w);
    if (s != DEM_OK) return s;
    return prev;
}

dem_status dem_set_timed_kernel(dem_world *w, int32_t which)
{
    if (!w) return DEM_ERR_ARG;
    if (which < -1 || which >= DEM_K_COUNT) return fail(w, DEM_ERR_ARG, "unknown kernel %d", which);
    if (w->timed_kernel != which) {
        w->timed_kernel = which;
        w->graph_valid = false;
    }
    return DEM_OK;
}

dem_status dem_step_timed(dem_world *w, float *step_ms, float *kernel_ms)
{
    if (!w || !step_ms) return DEM_ERR_ARG;
    dem_status prev = collect_flags(w);
    if (w->piles.empty()) return fail(w, DEM_ERR_STATE, "no piles");
    dem_status s = prepare(w);
    if (s != DEM_OK) return s;
    s = set_enabled(w, nullptr, 0);
    if (s != DEM_OK) return s;
    if (!w->sev[0]) {
        CU(cudaEventCreate(&w->sev[0]));
        CU(cudaEventCreate(&w->sev[1]));
    }
    CU(cudaEventRecord(w->sev[0], w->stream));
    CU(cudaGraphLaunch(w->exec, w->stream));
    CU(cudaEventRecord(w->sev[1], w->stream));
    CU(cudaEventSynchronize(w->sev[1]));
    CU(cudaEventElapsedTime(step_ms, w->sev[0], w->sev[1]));
    if (kernel_ms) {
        *kernel_ms = 0.f;
        if (w->timed_kernel >= 0) CU(cudaEventElapsedTime(kernel_ms, w->kev[0], w->kev[1]));
    }
    s = issue_flags_readback(w);
    if (s != DEM_OK) return s;
    return prev;
}

dem_status dem_graph_kernel_count(dem_world *w, int32_t *n_out)
{
    if (!w || !n_out) return DEM_ERR_ARG;
    dem_status s = prepare(w);
    if (s != DEM_OK) return s;
    *n_out = w->graph_kernels;
    return DEM_OK;
}

dem_status dem_read_state(dem_world *w, int32_t pile_id, int32_t field, double *out, int64_t n_out)
{
    Range range("dem_read_state");
    if (!w) return DEM_ERR_ARG;
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile id %d", pile_id);
    if (!out) return fail(w, DEM_ERR_ARG, "NULL output");
    CU(cudaStreamSynchronize(w->stream));
    const PileHost &q = w->piles[slot];
    int64_t s0 = 0, a0 = 0;
    for (int t = 0; t < slot; ++t) { s0 += w->piles[t].ns; a0 += w->piles[t].na; }
    const int64_t N = q.ns, A = q.na;
    const Arrays &D = w->A;
    auto get = [&](void *dst, const void *src, size_t bytes) -> dem_status {
        CU(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        return DEM_OK;
    };
    auto need = [&](int64_t n) -> dem_status {
        if (n_out < n) return fail(w, DEM_ERR_ARG, "output too small: need %lld doubles", (long long)n);
        return DEM_OK;
    };
    dem_status s;
#define CHK(x) do { s = (x); if (s != DEM_OK) return s; } while (0)
    PileDyn dyn{};   // the pile's device record: read only for the fields that use it
    if (field == DEM_FIELD_FRAME || field == DEM_FIELD_CONTACTS || field == DEM_FIELD_PLANET ||
        field == DEM_FIELD_INFO)
        CHK(get(&dyn, D.pd + slot, sizeof dyn));
    switch (field) {
    case DEM_FIELD_COM: CHK(need(3 * A)); CHK(get(out, D.r + 3 * a0, 24 * A)); unpack_all(w, out, 3 * A); break;
    case DEM_FIELD_VEL: CHK(need(3 * A)); CHK(get(out, D.v + 3 * a0, 24 * A)); unpack_all(w, out, 3 * A); break;
    case DEM_FIELD_QUAT: CHK(need(4 * A)); CHK(get(out, D.q + 4 * a0, 32 * A)); unpack_all(w, out, 4 * A); break;
    case DEM_FIELD_OMEGA_BODY:
        CHK(need(3 * A)); CHK(get(out, D.wb + 3 * a0, 24 * A)); unpack_all(w, out, 3 * A); break;
    case DEM_FIELD_ACC: CHK(need(3 * A)); CHK(get(out, D.acc + 3 * a0, 24 * A)); unpack_all(w, out, 3 * A); break;
    case DEM_FIELD_TORQUE_STORED:
        CHK(need(3 * A)); CHK(get(out, D.torque + 3 * a0, 24 * A)); unpack_all(w, out, 3 * A); break;
    case DEM_FIELD_FRAME:
        CHK(need(6));
        for (int c = 0; c < 3; ++c) { out[c] = dyn.O[c]; out[3 + c] = dyn.V[c]; }
        break;
    case DEM_FIELD_MASS: CHK(need(A)); CHK(get(out, D.M + a0, 8 * A)); break;
    case DEM_FIELD_BODY_OFFSETS: CHK(need(3 * N)); CHK(get(out, D.b64 + 3 * s0, 24 * N)); break;
    case DEM_FIELD_OMEGA: {
        CHK(need(3 * A));
        std::vector<double> qq(4 * A), ww(3 * A);
        CHK(get(qq.data(), D.q + 4 * a0, 32 * A));
        CHK(get(ww.data(), D.wb + 3 * a0, 24 * A));
        unpack_all(w, qq.data(), 4 * A);
        unpack_all(w, ww.data(), 3 * A);
        for (int64_t a = 0; a < A; ++a) {
            double R[9];
            rotmat(&qq[4 * a], R);
            for (int c = 0; c < 3; ++c)
                out[3 * a + c] = R[3 * c] * ww[3 * a] + R[3 * c + 1] * ww[3 * a + 1] + R[3 * c + 2] * ww[3 * a + 2];
        }
        break;
    }
    case DEM_FIELD_SPHERE_POS: {
        CHK(need(3 * N));
        std::vector<double> qq(4 * A), rr(3 * A), bb(3 * N);
        std::vector<int32_t> ag(N);
        CHK(get(qq.data(), D.q + 4 * a0, 32 * A));
        CHK(get(rr.data(), D.r + 3 * a0, 24 * A));
        unpack_all(w, qq.data(), 4 * A);
        unpack_all(w, rr.data(), 3 * A);
        CHK(get(bb.data(), D.b64 + 3 * s0, 24 * N));
        CHK(get(ag.data(), D.sph_agg + s0, 4 * N));
        for (int64_t i = 0; i < N; ++i) {
            int a = ag[i];
            double R[9];
            rotmat(&qq[4 * a], R);
            for (int c = 0; c < 3; ++c)
                out[3 * i + c] = rr[3 * a + c] + R[3 * c] * bb[3 * i] + R[3 * c + 1] * bb[3 * i + 1] +
                                 R[3 * c + 2] * bb[3 * i + 2];
        }
        break;
    }
    case DEM_FIELD_FORCE: case DEM_FIELD_TORQUE:
    case DEM_FIELD_FORCE_CONTACT: case DEM_FIELD_TORQUE_CONTACT:
    case DEM_FIELD_FORCE_GRAV: case DEM_FIELD_TORQUE_GRAV:
    case DEM_FIELD_FORCE_EXT: case DEM_FIELD_TORQUE_EXT: {
        CHK(need(3 * A));
        // the three parts (contact, gravity, planet), each [A][6]: F then N
        std::vector<double> o(18 * A);
        for (int k = 0; k < 3; ++k) CHK(get(o.data() + 6 * A * k, D.out[k] + 6 * a0, 48 * A));
        if (w->precision == DEM_MIXED) {   // float-float pairs
            std::vector<float> f(36 * A);
            std::memcpy(f.data(), o.data(), 144 * A);
            for (int64_t k = 0; k < 18 * A; ++k) o[k] = (double)f[2 * k] + (double)f[2 * k + 1];
        }
        for (int64_t a = 0; a < A; ++a)
            for (int c = 0; c < 3; ++c) {
                const double *xc = &o[6 * a], *xg = &o[6 * (A + a)], *xe = &o[6 * (2 * A + a)];
                double val = 0;
                switch (field) {
                case DEM_FIELD_FORCE: val = xc[c] + xg[c] + xe[c]; break;
                case DEM_FIELD_TORQUE: val = xc[3 + c] + xg[3 + c] + xe[3 + c]; break;
                case DEM_FIELD_FORCE_CONTACT: val = xc[c]; break;
                case DEM_FIELD_TORQUE_CONTACT: val = xc[3 + c]; break;
                case DEM_FIELD_FORCE_GRAV: val = xg[c]; break;
                case DEM_FIELD_TORQUE_GRAV: val = xg[3 + c]; break;
                case DEM_FIELD_FORCE_EXT: val = xe[c]; break;
                default: val = xe[3 + c]; break;
                }
                out[3 * a + c] = val;
            }
        break;
    }
    case DEM_FIELD_SPHERE_FC: case DEM_FIELD_SPHERE_TC: case DEM_FIELD_SPHERE_FG: {
        CHK(need(3 * N));
        if (field == DEM_FIELD_SPHERE_FG) {
            std::vector<dbl4> f(N);
            CHK(get(f.data(), D.fg + s0, 32 * N));
            for (int64_t i = 0; i < N; ++i) { out[3 * i] = f[i].x; out[3 * i + 1] = f[i].y; out[3 * i + 2] = f[i].z; }
            break;
        }
        // (stored at home indices)
        const int sel = field == DEM_FIELD_SPHERE_FC ? 0 : 1;
        if (w->precision == DEM_FP64) {
            std::vector<dbl4> f(2 * N);
            CHK(get(f.data(), D.ftc64 + 2 * s0, 64 * N));
            for (int64_t i = 0; i < N; ++i) {
                const dbl4 &e = f[2 * i + sel];
                out[3 * i] = e.x; out[3 * i + 1] = e.y; out[3 * i + 2] = e.z;
            }
        } else {
            std::vector<float4> f(2 * N);
            CHK(get(f.data(), D.ftc32 + 2 * s0, 32 * N));
            for (int64_t i = 0; i < N; ++i) {
                const float4 &e = f[2 * i + sel];
                out[3 * i] = e.x; out[3 * i + 1] = e.y; out[3 * i + 2] = e.z;
            }
        }
        break;
    }
    case DEM_FIELD_CONTACTS: {
        // the current candidate lists (entries in partner order) and the
        // history at each pair's owner entry (S from the lower-index sphere)
        const int K = w->K;
        CHK(need(N * (1 + 4 * (int64_t)K)));
        const int par = dyn.parity, cp = dyn.cpar;
        int64_t e0 = 0;
        for (int t = 0; t < slot; ++t) e0 += pile_count(w, w->piles[t], C_ENT);
        std::vector<int32_t> cnt(N), off(N), pos(N);
        CHK(get(cnt.data(), D.ccnt[cp] + s0, 4 * N));
        CHK(get(off.data(), D.coff[cp] + s0, 4 * N));
        CHK(get(pos.data(), D.pos_of_home[par] + s0, 4 * N));
        // sliced layout: entry e of sorted sphere k at off[k] + 32 e
        int64_t E = 0;
        for (int64_t k = 0; k < N; ++k)
            if (cnt[k] > 0) E = std::max<int64_t>(E, (int64_t)off[k] + 32 * ((int64_t)cnt[k] - 1) + 1);
        E = std::min<int64_t>(E, pile_count(w, q, C_ENT));
        std::vector<int32_t> ids(E);
        std::vector<int2> cd(E);
        std::vector<double> hs(4 * E);
        if (E > 0) {
            CHK(get(ids.data(), D.cand_id[cp] + e0, 4 * E));
            CHK(get(cd.data(), D.cand[cp] + e0, 8 * E));
            if (w->precision == DEM_FP64) {
                std::vector<dbl4> h(E);
                CHK(get(h.data(), D.hist64[par] + e0, 32 * E));
                for (int64_t f = 0; f < E; ++f) { hs[4 * f] = h[f].x; hs[4 * f + 1] = h[f].y; hs[4 * f + 2] = h[f].z; hs[4 * f + 3] = h[f].w; }
            } else {
                std::vector<float4> h(E);
                CHK(get(h.data(), D.hist32[par] + e0, 16 * E));
                for (int64_t f = 0; f < E; ++f) { hs[4 * f] = h[f].x; hs[4 * f + 1] = h[f].y; hs[4 * f + 2] = h[f].z; hs[4 * f + 3] = h[f].w; }
            }
        }
        std::fill(out, out + N * (1 + 4 * (int64_t)K), 0.0);
        for (int64_t i = 0; i < N; ++i) {
            double *o = out + i * (1 + 4 * K);
            const int64_t k = pos[i];
            int n = 0;
            for (int e = 0; e < cnt[k]; ++e) {
                const int64_t f = (int64_t)off[k] + 32 * (int64_t)e;
                if (f < 0 || f >= E) break;
                const int64_t h = cd[f].x < 0 ? f : (int64_t)cd[f].y;
                if (h < 0 || h >= E || hs[4 * h + 3] == 0.0) continue;
                if (n < K) {
                    o[1 + 4 * n] = ids[f];
                    o[2 + 4 * n] = hs[4 * h]; o[3 + 4 * n] = hs[4 * h + 1]; o[4 + 4 * n] = hs[4 * h + 2];
                }
                ++n;
            }
            o[0] = std::min(n, K);
        }
        break;
    }
    case DEM_FIELD_PLANET:
        CHK(need(9));
        for (int c = 0; c < 3; ++c) { out[c] = dyn.P_pos[c]; out[3 + c] = dyn.P_vel[c]; out[6 + c] = dyn.P_acc[c]; }
        break;
    case DEM_FIELD_INFO: {
        CHK(need(20));
        double info[20] = {(double)A, (double)N, (double)dyn.steps, (double)dyn.flags,
                           (double)q.nx, (double)q.ny, (double)q.nz, q.cell,
                           (double)w->K, (double)w->precision, dyn.O[0], dyn.O[1], dyn.O[2],
                           (double)dyn.failed, (double)dyn.parity, q.M_total,
                           (double)dyn.rebuilds, skin_of(w, q), (double)dyn.rebuild, 0.0};
        std::memcpy(out, info, sizeof info);
        break;
    }
    default:
        return fail(w, DEM_ERR_ARG, "unknown field %d", field);
    }
#undef CHK
    return DEM_OK;
}

dem_status dem_read_state_async(dem_world *w, int32_t pile_id, int32_t field, double *out, int64_t n_out)
{
    Range range("dem_read_state_async");
    if (!w) return DEM_ERR_ARG;
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile id %d", pile_id);
    if (!out) return fail(w, DEM_ERR_ARG, "NULL output");
    if ((int)w->reads.size() >= DEM_MAX_ASYNC_READS)
        return fail(w, DEM_ERR_ARG, "%d asynchronous reads pending: call dem_read_wait", DEM_MAX_ASYNC_READS);
    int64_t a0 = 0;
    for (int t = 0; t < slot; ++t) a0 += w->piles[t].na;
    const int64_t A = w->piles[slot].na;
    const Arrays &D = w->A;
    const double *src = nullptr;
    int64_t n = 3 * A;
    bool ff = w->precision == DEM_MIXED;
    switch (field) {
    case DEM_FIELD_COM: src = D.r + 3 * a0; break;
    case DEM_FIELD_VEL: src = D.v + 3 * a0; break;
    case DEM_FIELD_QUAT: src = D.q + 4 * a0; n = 4 * A; break;
    case DEM_FIELD_OMEGA_BODY: src = D.wb + 3 * a0; break;
    case DEM_FIELD_ACC: src = D.acc + 3 * a0; break;
    case DEM_FIELD_TORQUE_STORED: src = D.torque + 3 * a0; break;
    case DEM_FIELD_MASS: src = D.M + a0; n = A; ff = false; break;
    default: return fail(w, DEM_ERR_ARG, "field %d cannot be read asynchronously", field);
    }
    if (n_out < n) return fail(w, DEM_ERR_ARG, "output too small: need %lld doubles", (long long)n);
    const size_t k = w->reads.size();
    if (!w->rev[k]) CU(cudaEventCreateWithFlags(&w->rev[k], cudaEventDisableTiming));
    CU(cudaMemcpyAsync(out, src, 8 * (size_t)n, cudaMemcpyDeviceToHost, w->stream));
    CU(cudaEventRecord(w->rev[k], w->stream));
    w->reads.push_back({out, n, ff});
    return DEM_OK;
}

dem_status dem_read_wait(dem_world *w)
{
    Range range("dem_read_wait");
    if (!w) return DEM_ERR_ARG;
    dem_status st = DEM_OK;
    for (size_t k = 0; k < w->reads.size(); ++k) {
        if (cudaEventSynchronize(w->rev[k]) != cudaSuccess) {
            cudaGetLastError();
            st = fail(w, DEM_ERR_CUDA, "asynchronous read failed");
            continue;
        }
        const auto &r = w->reads[k];
        if (r.ff)
            for (int64_t i = 0; i < r.n; ++i) r.out[i] = unpack_ff(r.out[i]);
    }
    w->reads.clear();
    return st;
}

dem_status dem_write_state(dem_world *w, int32_t pile_id, int32_t field, const double *in,
                           int64_t n_in)
{
    Range range("dem_write_state");
    if (!w) return DEM_ERR_ARG;
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile id %d", pile_id);
    if (!in) return fail(w, DEM_ERR_ARG, "NULL input");
    CU(cudaStreamSynchronize(w->stream));
    const PileHost &q = w->piles[slot];
    int64_t s0 = 0, a0 = 0;
    for (int t = 0; t < slot; ++t) { s0 += w->piles[t].ns; a0 += w->piles[t].na; }
    const int64_t N = q.ns, A = q.na;
    const Arrays &D = w->A;
    auto put = [&](void *dst, const void *src, size_t bytes) -> dem_status {
        CU(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
        return DEM_OK;
    };
    auto need = [&](int64_t n) -> dem_status {
        if (n_in < n) return fail(w, DEM_ERR_ARG, "input too small: need %lld doubles", (long long)n);
        if (!finite_all(in, n)) return fail(w, DEM_ERR_ARG, "non-finite input");
        return DEM_OK;
    };
    dem_status s;
#define CHK(x) do { s = (x); if (s != DEM_OK) return s; } while (0)
    PileDyn dyn;
    CU(cudaMemcpy(&dyn, D.pd + slot, sizeof dyn, cudaMemcpyDeviceToHost));
    switch (field) {
    case DEM_FIELD_COM: CHK(need(3 * A)); CHK(put(D.r + 3 * a0, packed(w, in, 3 * A).data(), 24 * A)); break;
    case DEM_FIELD_VEL: CHK(need(3 * A)); CHK(put(D.v + 3 * a0, packed(w, in, 3 * A).data(), 24 * A)); break;
    case DEM_FIELD_QUAT: CHK(need(4 * A)); CHK(put(D.q + 4 * a0, packed(w, in, 4 * A).data(), 32 * A)); break;
    case DEM_FIELD_OMEGA_BODY:
        CHK(need(3 * A)); CHK(put(D.wb + 3 * a0, packed(w, in, 3 * A).data(), 24 * A)); break;
    case DEM_FIELD_ACC: CHK(need(3 * A)); CHK(put(D.acc + 3 * a0, packed(w, in, 3 * A).data(), 24 * A)); break;
    case DEM_FIELD_TORQUE_STORED:
        CHK(need(3 * A)); CHK(put(D.torque + 3 * a0, packed(w, in, 3 * A).data(), 24 * A)); break;
    case DEM_FIELD_PLANET:
    case DEM_FIELD_FRAME: {
        CHK(need(field == DEM_FIELD_PLANET ? 9 : 6));
        for (int c = 0; c < 3; ++c) {
            if (field == DEM_FIELD_PLANET) {
                dyn.P_pos[c] = in[c]; dyn.P_vel[c] = in[3 + c]; dyn.P_acc[c] = in[6 + c];
            } else {
                dyn.O[c] = in[c]; dyn.V[c] = in[3 + c];
                dyn.hVf[c] = (float)(q.P.dt * in[3 + c]);
                split(in[c], dyn.Of[c].x, dyn.Of[c].y);
                split(in[3 + c], dyn.Vf[c].x, dyn.Vf[c].y);
            }
        }
        CHK(put(D.pd + slot, &dyn, sizeof dyn));
        break;
    }
    case DEM_FIELD_CONTACTS: {
        // written as the pile's current candidate lists (one entry per
        // contact, both spheres of a pair listing each other, partner order)
        // with the history at the owner entries; the next step rebuilds the
        // lists and carries S over by partner index
        const int K = w->K;
        const int64_t row = 1 + 4 * (int64_t)K;
        if (n_in < N * row) return fail(w, DEM_ERR_ARG, "input too small: need %lld doubles", (long long)(N * row));
        const int par = dyn.parity, cp = dyn.cpar;
        int64_t e0 = 0;
        for (int t = 0; t < slot; ++t) e0 += pile_count(w, w->piles[t], C_ENT);
        const int64_t cap = pile_count(w, q, C_ENT);
        std::vector<int32_t> pos(N), home(N);
        CU(cudaMemcpy(pos.data(), D.pos_of_home[par] + s0, 4 * N, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < N; ++i) {
            if (pos[i] < 0 || pos[i] >= N) return fail(w, DEM_ERR_STATE, "sorted order unavailable");
            home[pos[i]] = (int32_t)i;
        }
        // rows sorted by partner
        std::vector<std::vector<std::pair<int32_t, int>>> rows(N);   // (partner, input slot)
        for (int64_t i = 0; i < N; ++i) {
            const double *e = in + i * row;
            const int n = (int)e[0];
            if (!(e[0] >= 0) || n > K || (double)n != e[0])
                return fail(w, DEM_ERR_ARG, "sphere %lld: bad contact count", (long long)i);
            for (int t = 0; t < n; ++t) {
                const double *sl = e + 1 + 4 * t;
                if (!(sl[0] >= 0 && sl[0] < (double)N) || (double)(int64_t)sl[0] != sl[0] || sl[0] == (double)i ||
                    !finite_all(sl + 1, 3))
                    return fail(w, DEM_ERR_ARG, "sphere %lld: bad contact entry", (long long)i);
                rows[i].push_back({(int32_t)sl[0], t});
            }
            std::sort(rows[i].begin(), rows[i].end());
            for (size_t t = 1; t < rows[i].size(); ++t)
                if (rows[i][t].first == rows[i][t - 1].first)
                    return fail(w, DEM_ERR_ARG, "sphere %lld: partner listed twice", (long long)i);
        }
        // sliced layout as the library builds it: slices of 32 sorted
        // positions, each as wide as its longest list, entry e of sphere k at
        // off[k] + 32 e
        std::vector<int32_t> cnt(N), off(N);
        int64_t E = 0;
        for (int64_t k0 = 0; k0 < N; k0 += 32) {
            int64_t wmax = 0;
            for (int64_t k = k0; k < std::min<int64_t>(N, k0 + 32); ++k) {
                cnt[k] = (int32_t)rows[home[k]].size();
                wmax = std::max<int64_t>(wmax, cnt[k]);
                off[k] = (int32_t)(E + (k - k0));
            }
            E += 32 * wmax;
        }
        if (E > cap) return fail(w, DEM_ERR_ARG, "too many contacts for the pile's candidate lists");
        std::vector<int32_t> ids(E);
        std::vector<int2> cd(E);
        std::vector<double> hs(4 * E, 0.0);
        for (int64_t k = 0; k < N; ++k) {
            const int32_t i = home[k];
            for (int e = 0; e < cnt[k]; ++e) {
                const int64_t f = off[k] + 32 * (int64_t)e;
                const int32_t J = rows[i][e].first;
                // this pair in J's row
                const auto &rj = rows[J];
                auto it = std::lower_bound(rj.begin(), rj.end(), std::make_pair(i, -1));
                if (it == rj.end() || it->first != i)
                    return fail(w, DEM_ERR_ARG, "contact %d-%d listed by one sphere only", i, J);
                const int64_t mir = off[pos[J]] + 32 * (int64_t)(it - rj.begin());
                ids[f] = J;
                const bool owned = i < J;
                cd[f] = make_int2(pos[J] | (owned ? (int)0x80000000u : 0), (int)mir);
                if (owned) {
                    const double *sl = in + (int64_t)i * row + 1 + 4 * rows[i][e].second;
                    hs[4 * f] = sl[1]; hs[4 * f + 1] = sl[2]; hs[4 * f + 2] = sl[3]; hs[4 * f + 3] = 1.0;
                }
            }
        }
        CHK(put(D.ccnt[cp] + s0, cnt.data(), 4 * N));
        CHK(put(D.coff[cp] + s0, off.data(), 4 * N));
        if (E > 0) {
            CHK(put(D.cand_id[cp] + e0, ids.data(), 4 * E));
            CHK(put(D.cand[cp] + e0, cd.data(), 8 * E));
            if (w->precision == DEM_FP64) {
                std::vector<dbl4> h(E);
                for (int64_t f = 0; f < E; ++f) h[f] = make_dbl4(hs[4 * f], hs[4 * f + 1], hs[4 * f + 2], hs[4 * f + 3]);
                CHK(put(D.hist64[par] + e0, h.data(), 32 * E));
            } else {
                std::vector<float4> h(E);
                for (int64_t f = 0; f < E; ++f)
                    h[f] = make_float4((float)hs[4 * f], (float)hs[4 * f + 1], (float)hs[4 * f + 2], (float)hs[4 * f + 3]);
                CHK(put(D.hist32[par] + e0, h.data(), 16 * E));
            }
        }
        break;
    }
    default:
        return fail(w, DEM_ERR_ARG, "field %d is not writable", field);
    }
#undef CHK
    // positions, orientations or contacts may have changed: rebuild the
    // neighbour lists of this pile at its next step
    launch_force_rebuild(w->A, w->Z, slot, w->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(w->stream));
    return DEM_OK;
}

dem_status dem_pile_flags(dem_world *w, int32_t pile_id, int32_t *flags_out)
{
    if (!w || !flags_out) return DEM_ERR_ARG;
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile id %d", pile_id);
    CU(cudaStreamSynchronize(w->stream));
    PileDyn dyn;
    CU(cudaMemcpy(&dyn, w->A.pd + slot, sizeof dyn, cudaMemcpyDeviceToHost));
    *flags_out = dyn.flags;
    return DEM_OK;
}

dem_status dem_remove_pile(dem_world *w, int32_t pile_id)
{
    Range range("dem_remove_pile");
    if (!w) return DEM_ERR_ARG;
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile id %d", pile_id);
    CU(cudaStreamSynchronize(w->stream));
    w->pending = false;
    std::vector<PileHost> newp = w->piles;
    newp.erase(newp.begin() + slot);
    dem_status s = relayout(w, newp, nullptr);
    if (s != DEM_OK) return s;
    w->piles = newp;
    w->graph_valid = false;
    return DEM_OK;
}

dem_status dem_set_tuning(dem_world *w, const char *key, double value)
{
    if (!w || !key) return DEM_ERR_ARG;
    std::string k = key;
    if (k == "grav_block") {
        int b = (int)value;
        if (b != 64 && b != 128 && b != 256) return fail(w, DEM_ERR_ARG, "grav_block must be 64, 128 or 256");
        w->grav_block = b;
    } else if (k == "grav_ib") {
        int b = (int)value;
        if (b != 1 && b != 2 && b != 4) return fail(w, DEM_ERR_ARG, "grav_ib must be 1, 2 or 4");
        w->grav_ib = b;
    } else if (k == "grav_jchunk") {
        if (value < 0) return fail(w, DEM_ERR_ARG, "grav_jchunk must be >= 0");
        w->grav_jchunk = (int64_t)value;
    } else if (k == "grav_pack") {
        w->grav_pack = value != 0.0;
    } else if (k == "grav_sym") {
        w->grav_sym = value != 0.0;
    } else if (k == "grav_tile") {
        const int t = (int)value;
        if (t != 0 && t != 64 && t != 128 && t != 256 && t != 512)
            return fail(w, DEM_ERR_ARG, "grav_tile must be 0, 64, 128, 256 or 512");
        w->grav_tile = t;
    } else if (k == "grav_theta") {
        if (!(value >= 0.0) || !(value < 1.0)) return fail(w, DEM_ERR_ARG, "grav_theta must be in [0, 1)");
        const double old = w->grav_theta;
        w->grav_theta = value;
        dem_status s = relayout(w, w->piles, nullptr);   // tree arrays change size
        if (s != DEM_OK) { w->grav_theta = old; return s; }
    } else if (k == "grav_order") {
        const int o = (int)value;
        if (o != 2 && o != 4) return fail(w, DEM_ERR_ARG, "grav_order must be 2 or 4");
        w->grav_order = o;
    } else if (k == "grav_item") {
        if (!(value >= 1024.0)) return fail(w, DEM_ERR_ARG, "grav_item must be >= 1024");
        w->grav_item = value;
    } else if (k == "contact_mode") {
        if (value != 0.0 && value != 1.0) return fail(w, DEM_ERR_ARG, "contact_mode must be 0 or 1");
        w->contact_mode = (int)value;
    } else if (k == "contact_inbox") {
        if (!(value >= 1.0) || value > kInboxCap)
            return fail(w, DEM_ERR_ARG, "contact_inbox must be in [1, %d]", kInboxCap);
        w->contact_inbox = (int)value;
    } else if (k == "cell_factor" || k == "skin") {
        if (k == "cell_factor" && (!(value >= 1.0) || value > 16.0))
            return fail(w, DEM_ERR_ARG, "cell_factor must be in [1, 16]");
        if (k == "skin" && (!(value >= 0.0) || value > 4.0))
            return fail(w, DEM_ERR_ARG, "skin must be in [0, 4] (fraction of the largest radius)");
        double &knob = k == "skin" ? w->skin_frac : w->cell_factor;
        if (knob != value) {
            double old = knob;
            knob = value;
            dem_status s = regrid(w);
            if (s != DEM_OK) { knob = old; return s; }
        }
    } else {
        return fail(w, DEM_ERR_ARG, "unknown tuning key '%s'", key);
    }
    w->graph_valid = false;
    return DEM_OK;
}

dem_status dem_get_tuning(dem_world *w, const char *key, double *value_out)
{
    if (!w || !key || !value_out) return DEM_ERR_ARG;
    const std::string k = key;
    if (k == "grav_block") *value_out = w->grav_block;
    else if (k == "grav_ib") *value_out = w->grav_ib;
    else if (k == "grav_jchunk") *value_out = (double)w->grav_jchunk;
    else if (k == "grav_pack") *value_out = w->grav_pack ? 1.0 : 0.0;
    else if (k == "grav_sym") *value_out = w->grav_sym ? 1.0 : 0.0;
    else if (k == "grav_tile") *value_out = w->grav_tile;
    else if (k == "grav_theta") *value_out = w->grav_theta;
    else if (k == "grav_order") *value_out = w->grav_order;
    else if (k == "grav_item") *value_out = w->grav_item;
    else if (k == "cell_factor") *value_out = w->cell_factor;
    else if (k == "skin") *value_out = w->skin_frac;
    else if (k == "contact_inbox") *value_out = w->contact_inbox;
    else if (k == "contact_mode") *value_out = w->contact_mode;
    else return fail(w, DEM_ERR_ARG, "unknown tuning key '%s'", key);
    return DEM_OK;
}

dem_status dem_autotune(dem_world *w, int32_t trial_steps, double *best_ms_out)
{
    Range range("dem_autotune");
    if (!w || trial_steps < 1) return DEM_ERR_ARG;
    if (w->piles.empty()) return DEM_OK;
    dem_status s = collect_flags(w);
    if (s != DEM_OK) return s;
    struct Knobs { int blk, ib; double item; bool pack, sym; int tile; double cell; int cmode; };
    const Knobs orig = {w->grav_block, w->grav_ib, w->grav_item, w->grav_pack, w->grav_sym, w->grav_tile,
                        w->cell_factor, w->contact_mode};
    const int64_t orig_jchunk = w->grav_jchunk;
    std::vector<Knobs> cands;
    cands.push_back({128, 4, 1048576.0, false, true, 512, 0, orig.cmode});
    if (w->precision == DEM_MIXED)
        for (int tile : {64, 128, 256}) cands.push_back({128, 4, 1048576.0, false, true, tile, 0, orig.cmode});
    for (int blk : {64, 128, 256})
        for (int ib : {1, 2, 4})
            for (double item : {262144.0, 1048576.0, 4194304.0}) {
                cands.push_back({blk, ib, item, false, false, 0, 0, orig.cmode});
                if (ib % 2 == 0) cands.push_back({blk, ib, item, true, false, 0, 0, orig.cmode});
            }
    // The trials step the live piles.  Snapshot every field that carries state
    // from step to step (the fields a layout change preserves) and put it back
    // afterwards, so the piles leave the tuner exactly as they entered it.
    std::vector<std::pair<size_t, size_t>> snap_of;   // field index -> (offset, bytes)
    size_t snap_bytes = 0;
    for (size_t f = 0; f < w->fields.size(); ++f) {
        const Field &fd = w->fields[f];
        if (!fd.keep || *fd.ptr == nullptr) continue;
        int64_t n = 0;
        for (auto &q : w->piles) n += pile_count(w, q, fd.cls);
        const size_t bytes = (size_t)n * fd.el;
        snap_of.push_back({f, bytes});
        snap_bytes += (bytes + 255) / 256 * 256;
    }
    char *snap = snap_bytes ? (char *)dev_alloc(w, snap_bytes) : nullptr;
    if (snap_bytes && !snap) return fail(w, DEM_ERR_OOM, "autotune: snapshot of %zu bytes failed", snap_bytes);
    {
        size_t o = 0;
        for (auto &fb : snap_of) {
            cudaError_t e = cudaMemcpyAsync(snap + o, *w->fields[fb.first].ptr, fb.second,
                                            cudaMemcpyDeviceToDevice, w->stream);
            if (e != cudaSuccess) {
                dev_free(w, snap);
                return fail(w, DEM_ERR_CUDA, "autotune snapshot: %s", cudaGetErrorString(e));
            }
            o += (fb.second + 255) / 256 * 256;
        }
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto set_knobs = [&](const Knobs &k) -> dem_status {
        w->grav_block = k.blk; w->grav_ib = k.ib; w->grav_item = k.item; w->grav_pack = k.pack;
        w->grav_sym = k.sym; w->grav_tile = k.tile; w->contact_mode = k.cmode;
        w->graph_valid = false;
        if (k.cell > 0 && k.cell != w->cell_factor) return dem_set_tuning(w, "cell_factor", k.cell);
        return DEM_OK;
    };
    // time trial_steps graph launches after one warm launch
    auto trial = [&](double &per) -> dem_status {
        dem_status t = prepare(w);
        if (t == DEM_OK) t = set_enabled(w, nullptr, 0);
        if (t != DEM_OK) return t;
        CU(cudaGraphLaunch(w->exec, w->stream));
        CU(cudaEventRecord(ev[0], w->stream));
        for (int i = 0; i < trial_steps; ++i) CU(cudaGraphLaunch(w->exec, w->stream));
        CU(cudaEventRecord(ev[1], w->stream));
        CU(cudaEventSynchronize(ev[1]));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        per = ms / trial_steps;
        return DEM_OK;
    };
    // restore the state (and, on failure, the original knobs) on every way out
    auto finish = [&](dem_status st, const Knobs &k) -> dem_status {
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        std::string err = st == DEM_OK ? std::string() : w->err;
        w->grav_jchunk = st == DEM_OK ? 0 : orig_jchunk;
        dem_status r = set_knobs(st == DEM_OK ? k : orig);
        if (r == DEM_OK) r = prepare(w);
        if (r == DEM_OK && snap) {
            size_t o = 0;
            for (auto &fb : snap_of) {
                if (cudaMemcpyAsync(*w->fields[fb.first].ptr, snap + o, fb.second, cudaMemcpyDeviceToDevice,
                                    w->stream) != cudaSuccess) {
                    r = fail(w, DEM_ERR_CUDA, "autotune: restoring the pile state failed");
                    break;
                }
                o += (fb.second + 255) / 256 * 256;
            }
            // the transient sort and candidate lists belong to the trials' state
            if (r == DEM_OK) launch_force_rebuild(w->A, w->Z, -1, w->stream);
            if (r == DEM_OK && cudaStreamSynchronize(w->stream) != cudaSuccess)
                r = fail(w, DEM_ERR_CUDA, "autotune: restoring the pile state failed");
        }
        if (snap) dev_free(w, snap);
        if (st != DEM_OK) {
            w->err = err;
            return st;
        }
        return r;
    };
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)
        return finish(fail(w, DEM_ERR_CUDA, "autotune: cudaEventCreate failed"), orig);
    w->grav_jchunk = 0;
    double best = 1e300;
    Knobs bk = orig;
    for (auto c : cands) {
        c.cell = orig.cell;
        s = set_knobs(c);
        double per = 0.0;
        if (s == DEM_OK) s = trial(per);
        if (s != DEM_OK) return finish(s, orig);
        if (per < best) { best = per; bk = c; }
    }
    // then the cell edge (contact search), with the chosen gravity shape
    for (double f : {1.0, 1.25, 1.5, 2.0}) {
        Knobs c = bk;
        c.cell = f;
        s = set_knobs(c);
        double per = 0.0;
        if (s == DEM_OK) s = trial(per);
        if (s != DEM_OK) return finish(s, orig);
        if (per < best) { best = per; bk = c; }
    }
    // then the contact pass's form (one thread per sphere, or 128-sphere tile
    // blocks with a shared-memory inbox; both give bitwise the same results)
    for (int m : {0, 1}) {
        if (m == bk.cmode) continue;
        Knobs c = bk;
        c.cmode = m;
        s = set_knobs(c);
        double per = 0.0;
        if (s == DEM_OK) s = trial(per);
        if (s != DEM_OK) return finish(s, orig);
        if (per < best) { best = per; bk = c; }
    }
    if (best_ms_out) *best_ms_out = best;
    return finish(DEM_OK, bk);
}

dem_status dem_pile_bulk(dem_world *w, int32_t pile_id, double *out, int64_t n_out)
{
    Range range("dem_pile_bulk");
    if (!w) return DEM_ERR_ARG;
    if (!out || n_out < DEM_BULK_LEN) return fail(w, DEM_ERR_ARG, "output needs %d doubles", DEM_BULK_LEN);
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile %d", pile_id);
    dem_status s = prepare(w);
    if (s != DEM_OK) return s;
    slot = find_pile(w, pile_id);
    launch_bulk(w->A, w->Z, 0, slot, w->stream);
    CU(cudaGetLastError());
    const char *src = (const char *)(w->A.watch + slot) + offsetof(PileWatch, now);
    CU(cudaMemcpyAsync(out, src, 8 * DEM_BULK_LEN, cudaMemcpyDeviceToHost, w->stream));
    CU(cudaStreamSynchronize(w->stream));
    return DEM_OK;
}

dem_status dem_watch(dem_world *w, int32_t pile_id, double growth, int64_t every)
{
    if (!w) return DEM_ERR_ARG;
    if (!(growth >= 0.0) || !std::isfinite(growth) || every < 1)
        return fail(w, DEM_ERR_ARG, "bad watch (growth %g, every %lld)", growth, (long long)every);
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile %d", pile_id);
    dem_status s = prepare(w);
    if (s != DEM_OK) return s;
    slot = find_pile(w, pile_id);
    PileWatch wat{};
    wat.growth = growth;
    wat.every = every;
    wat.fired = -1;
    wat.arm = growth > 0.0 ? 1 : 0;
    CU(cudaMemcpyAsync(w->A.watch + slot, &wat, sizeof wat, cudaMemcpyHostToDevice, w->stream));
    if (growth > 0.0) launch_bulk(w->A, w->Z, 0, slot, w->stream);   // takes R_b0
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(w->stream));   // wat goes out of scope
    const bool on = growth > 0.0;
    if (w->piles[slot].watch_on != on) {
        w->piles[slot].watch_on = on;
        w->graph_valid = false;   // the watch phase joins or leaves the graph
    }
    return DEM_OK;
}

dem_status dem_watch_result(dem_world *w, int32_t pile_id, double *out, int64_t n_out)
{
    if (!w) return DEM_ERR_ARG;
    if (!out || n_out < DEM_WATCH_LEN) return fail(w, DEM_ERR_ARG, "output needs %d doubles", DEM_WATCH_LEN);
    int slot = find_pile(w, pile_id);
    if (slot < 0) return fail(w, DEM_ERR_ARG, "unknown pile %d", pile_id);
    dem_status s = prepare(w);
    if (s != DEM_OK) return s;
    slot = find_pile(w, pile_id);
    PileWatch wat;
    CU(cudaMemcpyAsync(&wat, w->A.watch + slot, sizeof wat, cudaMemcpyDeviceToHost, w->stream));
    CU(cudaStreamSynchronize(w->stream));
    out[0] = (double)wat.fired;
    out[1] = wat.growth;
    out[2] = (double)wat.every;
    out[3] = wat.growth > 0.0 ? 1.0 : 0.0;
    for (int k = 0; k < DEM_BULK_LEN; ++k) {
        out[4 + k] = wat.at_arm[k];
        out[4 + DEM_BULK_LEN + k] = wat.fired >= 0 ? wat.at_fire[k] : 0.0;
    }
    return DEM_OK;
}

size_t dem_footprint_bytes(int64_t n_spheres, int64_t n_agg, int32_t max_contacts, int32_t precision)
{
    if (n_spheres < 0 || n_agg < 0 || max_contacts < 1) return 0;
    bool d = precision == DEM_FP64;
    size_t sph = 4 + 4 + 24 + 8 + 8 + 4 + 4 + 4 + 4 + 32;
    sph += 8;        // pos_of_home, both parities
    sph += 2 * 8;    // candidate counts and offsets, both buffers
    sph += d ? (32 * 3 + 32 + 64) : (16 * 2 + 16 * 5 + 16 + 32);
    // candidate-list entries: partner and mirror, partner index (both
    // buffers), history (both parities) and the carried-over history
    size_t ent = 2 * (8 + 4) + 3 * (d ? 32 : 16);
    size_t agg = 4 * 3 + 8 + 72 * 2 + 24 * 2 + 32 + 24 * 3 + 144 + 64 +
                 (d ? sizeof(AggRec64) : sizeof(AggRecMixed) + 72);
    int64_t cells = std::max<int64_t>(4 * n_spheres, 27) + kScanTile;
    size_t bytes = sph * (size_t)n_spheres + ent * (size_t)n_spheres * (size_t)kEntPerSphere +
                   24 * (size_t)((n_spheres + kCTile - 1) / kCTile) +
                   agg * (size_t)n_agg + 8 * (size_t)cells + 4 * (size_t)(cells / kScanTile + 1) +
                   (size_t)(n_agg / kAggChunk + 1) * (8 * kPartialDoubles + 4 + 8 * 32) +
                   sizeof(PileStatic) + sizeof(PileDyn) + sizeof(PileWatch) + 20 + 16 * (size_t)(n_spheres / 64 + 1);
    // direct-sum gravity: partial sums of the 512-sphere tile pairs (2 T rows of
    // n spheres) and the work items (T (T + 1) / 2)
    // (up to 8,192 spheres the mixed path may use 128-sphere tiles, up to
    // 2,048 spheres 64-sphere tiles: count those)
    const int64_t tile = d ? kGravSymTile
                           : n_spheres <= kTinyTileMaxN ? kGravSymTileTiny
                           : n_spheres <= kSmallTileMaxN ? kGravSymTileSmall : kGravSymTile;
    const int64_t T = (n_spheres + tile - 1) / tile;
    if (T > 1) bytes += (size_t)(2 * T) * (size_t)n_spheres * (d ? 32 : 16);
    bytes += 16 * (size_t)(T * (T + 1) / 2);
    bytes += 256 * 80;   // each of the world's arrays starts on a 256-byte boundary of one slab
    return bytes;
}

size_t dem_world_bytes(const dem_world *w) { return w ? w->held : 0; }

const char *dem_last_error(const dem_world *w)
{
    if (!w) return "NULL world";
    return w->err.c_str();
}

void dem_destroy(dem_world *w)
{
    if (!w) return;
    cudaStreamSynchronize(w->stream);
    if (w->exec) cudaGraphExecDestroy(w->exec);
    dev_free(w, w->slab);
    if (w->h_dyn) cudaFreeHost(w->h_dyn);
    if (w->h_stage) {
        if (w->h_stage_pinned) cudaFreeHost(w->h_stage);
        else std::free(w->h_stage);
    }
    if (w->ev_flags) cudaEventDestroy(w->ev_flags);
    for (auto &e : w->rev)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (w->kev[k]) cudaEventDestroy(w->kev[k]);
        if (w->sev[k]) cudaEventDestroy(w->sev[k]);
    }
    if (w->own_stream) cudaStreamDestroy(w->stream);
    delete w;
}

}  // extern "C"
