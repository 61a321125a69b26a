// dem_internal.h -- device data layout and kernel entry points of the GB300
// DEM library (bonded-sphere aggregates, arXiv 2311.11322).  Internal: the
// public boundary is include/dem.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dem.h"

namespace dem {

// 32-byte aligned double vector (CUDA 13 spelling); loads as one 256-bit access.
typedef double4_32a dbl4;
__host__ __device__ __forceinline__ dbl4 make_dbl4(double x, double y, double z, double w)
{
    return make_double4_32a(x, y, z, w);
}

constexpr int kMaxK = 64;          // largest max_contacts
constexpr int kScanTile = 2048;    // cells per scan block (256 threads x 8)
constexpr int kAggChunk = 512;     // aggregates per pile-reduction block
constexpr int kPartialDoubles = 16;
// Contact pass: tiles of consecutive sorted spheres, one block each; the
// candidate lists of a pile hold kEntPerSphere entries per sphere on average
// at the default skin (more for larger skins, in proportion to the candidate
// volume; a pile whose lists need more is flagged DEM_FLAG_SLOTS and frozen);
// a tile with at most kInboxCap list entries evaluates each of its inner pairs
// once and passes the partner's share through shared memory.
constexpr int kCTile = 128;
constexpr int kEntPerSphere = 32;
constexpr int kInboxCap = 1280;

// Cell index of wrapped cell coordinates (cx, cy, cz) on an nx x ny x nz grid:
// bricks of 4 x 4 x 4 cells in row-major brick order, row-major inside a brick
// (x fastest).  Consecutive sorted spheres then fill compact blocks of space,
// and the three x-neighbours of a cell are consecutive unless a brick
// boundary falls between them.  The grid has ceil(n/4)*4 cells per axis.
__host__ __device__ __forceinline__ int64_t cell_id(int cx, int cy, int cz, int nx, int ny)
{
    const int64_t nbx = (nx + 3) >> 2, nby = (ny + 3) >> 2;
    const int64_t brick = ((int64_t)(cz >> 2) * nby + (cy >> 2)) * nbx + (cx >> 2);
    return (brick << 6) | (((cz & 3) << 4) | ((cy & 3) << 2) | (cx & 3));
}
__host__ __device__ __forceinline__ int64_t cell_count(int nx, int ny, int nz)
{
    return (int64_t)((nx + 3) >> 2) * ((ny + 3) >> 2) * ((nz + 3) >> 2) * 64;
}

// Static description of one pile (host-owned; re-uploaded on membership change).
struct PileStatic {
    int64_t s0, ns;        // sphere range [s0, s0+ns) (home order == sorted range)
    int64_t a0, na;        // aggregate range
    int64_t c0, nc;        // cell range (nc padded to a multiple of kScanTile)
    int64_t ch0, nch;      // aggregate-chunk range (pile reductions)
    int64_t t0, nt;        // scan-tile range
    int32_t nx, ny, nz, K; // wrapped grid dims (>= 3 each), history slots
    double cell, inv_cell; // cell edge and its inverse
    double skin;           // neighbour-list skin (>= 0; 0 = search every step)
    double G, h, kn, kt, cn, ct, mu_s, mu_r, mu_t, w0, eps2;
    double ext_mass, M_total;
    double spin_inc[3];
    double rot_tol;        // 0: RK4 rotation; > 0: adaptive RK5(4) tolerance
    // contact lists: entry range [e0, e0 + ne) and tile range [ct0, ct0 + nct);
    // mixed path: fixed-point position quantum q = 2^qexp (m) and the skin in
    // quanta (the exact integer candidate test)
    int64_t e0, ne, ct0, nct;
    int32_t qexp;
    int32_t pad_q;
    int64_t skin_q;
    // tree gravity (0 levels = direct sum): depth, opening angle, node and leaf ranges
    int32_t tD;
    float theta;
    int64_t tnode0, tleaf0, tg0;   // first node, leaf and 32-sphere group of the pile
    // mixed symmetric gravity: tile sums enter 64-bit integer accumulators
    // scaled by gscale = 2^k (the largest power of two with gscale x (bound on
    // a sphere's sum of |terms|) <= 2^61, |k| <= 120); ginv = 1 / gscale
    double ginv;
    float gscale_f;
    int32_t pad_g;
    // the contact law's constants in FP32 for the mixed path (kn, kt, cn, ct,
    // mu_s, mu_r, mu_t, w0, h), rounded once on the host
    float lawf[9];
    // mixed path: h as a float-float pair, the spin increment in FP32 and
    // whether it is nonzero
    float hff[2];
    float spin_f[3];
    int32_t yorp;
};

// Dynamic per-pile state (device-owned; written by kernels).
struct PileDyn {
    double O[3], V[3];        // frame of positions / velocities used this step
    float hVf[3];             // h V in FP32 (the neighbour-list test)
    int32_t pad_dyn;
    // mixed path: O, V and Rc as float-float pairs (hi, lo)
    float2 Of[3], Vf[3], Rcf[3];
    float2 pad_dyn2;
    double Rc[3], Vc[3];      // pile COM after the drift, mean velocity after the first kick
    double P_pos[3], P_vel[3], P_acc[3];   // planet
    int64_t steps;
    int32_t flags;            // DEM_FLAG_* bits
    int32_t parity;           // history buffer holding the previous contacts
    int32_t failed;           // frozen after a fatal flag
    int32_t rebuild;          // this step rebuilds the cell list and candidate lists
    int32_t cpar;             // candidate-list buffer of the current lists
    int32_t rebuilds;         // number of rebuilds so far
    int32_t rebuilt_prev;     // the previous step rebuilt (its sorted order is new)
    int32_t pad_dyn3;
};

// Bulk shape and spin of a pile (record laid out as enum dem_bulk) and its
// radius-growth watch (device-owned; the host writes it only to arm).
constexpr int kBulkParts = 25;   // doubles summed per aggregate chunk
struct PileWatch {
    double growth;               // > 0: armed; trigger at R_b >= (1 + growth) R_b0
    int64_t every;               // evaluate when steps % every == 0
    int64_t fired;               // step count at the latch, -1 = not yet
    int32_t arm;                 // 1: the next evaluation takes R_b0 (arming)
    int32_t pad;
    double now[DEM_BULK_LEN];    // last evaluation
    double at_arm[DEM_BULK_LEN]; // evaluation when armed
    double at_fire[DEM_BULK_LEN];// latched evaluation
};

// Per-aggregate quantities the sphere kernels need, mixed precision.
// R and c are float-float (hi + lo) so that sphere positions relative to the
// pile frame keep ~48 bits; velocity and spin are plain FP32, relative to the
// pile frame velocity.
struct __align__(16) AggRecMixed {
    float Rh[9], Rl[9];   // rotation body -> space
    float ch[3], cl[3];   // r_A - O
    float vb[3];          // v_A,n+1/2 + h/2 a_A,n - V
    float w[3];           // predicted spin (space frame)
    float pad[2];
};

struct __align__(16) AggRec64 {
    double R[9];
    double c[3];
    double vb[3];
    double w[3];
};

// Device pointers of every array (global, pile-contiguous, pile-local indices).
struct Arrays {
    // spheres, home order
    int32_t *sph_agg;    // aggregate index within the pile
    int32_t *sph_pile;   // pile slot
    double *b64;         // [N][3] body offsets (master copy, never rewritten)
    double *s64, *m64;   // radius, mass
    float4 *bh, *bl;     // mixed: body offset hi/lo with radius hi/lo in .w
    int32_t *key;        // cell index within the pile
    int32_t *rank;       // rank among spheres counted into the same cell
    int32_t *sorted;     // sorted position (pile-local) -> home index (pile-local)
    // sorted copies for the contact pass
    // mixed: per sphere two 16-byte halves of one 32-byte sector each:
    // xqr[2k] = low 32 bits of round((r_i - O) / q) per axis and round(radius / q),
    // xqr[2k+1] = what those roundings left (FP32 bits, in quanta, |.| <= 1/2);
    // svw[2k] = velocity (+agg), svw[2k+1] = spin (+home id)
    int4 *xqr;
    float4 *svw;
    float4 *sph_;                   // mixed: pos hi (+s hi; rebuild steps only)
    dbl4 *dp_, *dv_, *dw_;          // fp64: pos (+s), vel (+agg), spin (+home id)
    int32_t *sagg;                  // aggregate (pile-local) of each sorted position
    // candidate lists (compressed rows per sorted sphere, entries in the
    // order of the partners' home indices), double-buffered by PileDyn::cpar
    // so that a rebuild can carry the history over from the previous lists:
    // ccnt/coff per sorted position (coff pile-local into the pile's entries),
    // cand per entry (partner sorted position | owner bit << 31, entry of this
    // sphere in the partner's list), cand_id per entry (partner home index)
    int32_t *ccnt[2], *coff[2];
    int2 *cand[2];
    int32_t *cand_id[2];
    // contact tiles: (pile slot, first sorted position, spheres, 0); entries
    // of each tile and their pile-local base (rebuild steps)
    int4 *ctile;
    int32_t *ctile_cnt, *ctile_base;
    // gravity inputs / outputs
    float4 *gpos32;      // mixed: pos hi (+mass)
    dbl4 *gpos64;     // fp64: pos (+mass)
    dbl4 *fg;         // gravity on each sphere (from other aggregates)
    // contact outputs at each sphere's home index, interleaved: [2i] = force, [2i+1] = torque
    float4 *ftc32;
    dbl4 *ftc64;
    // sorted position (pile-local) of each home sphere, double-buffered by parity
    int32_t *pos_of_home[2];
    // contact history per candidate-list entry of the pair's owner (its lower
    // home index): S from the owner's side and 1 in .w while the pair is in
    // contact, double-buffered by pile parity; *_rm: the previous history
    // carried over to new lists at a rebuild
    float4 *hist32[2], *hist32_rm;
    dbl4 *hist64[2], *hist64_rm;
    // aggregates
    int32_t *agg_first, *agg_count, *agg_pile;
    double *M, *I, *Iinv;          // [A], [A][9], [A][9]
    float *I32, *Iinv32;           // mixed: [A][9] FP32 copies of I and of I^-1
    double *r, *v, *q, *wb, *acc, *torque;   // [A][3], q [A][4]
    AggRecMixed *rec32;
    AggRec64 *rec64;
    // per-aggregate force and torque by part: out[0] contact, out[1] sphere
    // gravity, out[2] planet, each [A][6] = F then N (FP64 path; in the mixed
    // path the same 48 bytes hold 6 float-float pairs).  One array per part,
    // so that a step that writes only the contact part writes whole sectors.
    double *out[3];
    // 1 in the mixed path: out holds float-float pairs, and so does each FP64
    // slot of the aggregate state (r, v, q, w_body, a, N) and of 1/M: a pair
    // (hi, lo) with hi = fl(hi + lo) in the 8 bytes of one double
    int32_t out_ff;
    double *invM;                  // [A] 1 / M
    // neighbour-list reference per aggregate: position relative to the
    // extrapolated pile frame and orientation at the last rebuild, and the
    // largest member offset |b| (fixed): [A][8] = c_ref[3], q_ref[4], bmax
    float *aref;
    // cells
    int32_t *ccount, *cstart, *tile_sum;
    // pile reductions
    double *chunk_part;            // [chunks][kPartialDoubles]
    int32_t *chunk_pile;           // [chunks] pile slot of each chunk
    int32_t *pile_arrive;          // [piles] chunk blocks of a reduction finished so far (0 between launches)
    double *bulk_part;             // [chunks][32] bulk-shape sums (kBulkParts used)
    PileWatch *watch;              // [piles]
    // gravity work list and j-chunk partial sums
    int4 *gitems;                  // (pile, i0 local, j0 local, j1 local)
    void *gpart;                   // partial sum of one j-range per sphere (scratch):
                                   // float4 in the mixed path, dbl4 in the FP64 path
    int64_t *gpart_base;           // per pile: first slot in gpart (or -1 = direct)
    int32_t *gnchunk;              // per pile: number of j-chunks
    int32_t *gcounter;             // [0]: next work item of the persistent gravity grid
    unsigned long long *gacc;      // mixed symmetric form: per sphere 4 x int64 (x, y, z, 0)
                                   // fixed-point sums of the tile items (zero between steps)
    // tree gravity: per sphere leaf key, rank in its leaf, leaf-ordered home
    // index; per pile cube (ordered-int min/max, 8 ints); nodes (3 float4 each:
    // COM + mass, quadrupole, opening radius^2) level by level, Morton order
    // inside a level; leaves (start, count); node and leaf owner piles
    int32_t *tkey, *trank, *tsorted;
    float4 *tpos;        // leaf-ordered positions (+mass)
    int32_t *tagg;       // leaf-ordered aggregates
    float4 *tpart;       // [64][N] partial sums of the 64 subtrees at level 2
    int *tbox;
    float4 *tnode;       // per node 9 float4: COM, M, opening radius^2, traceless moments of ranks 2-4
    float4 *traw;        // per node 8 float4: raw moments of ranks 2-4 about the COM (upward pass)
    int2 *tleaf;
    int32_t *tnode_pile, *tleaf_pile;
    // piles
    PileStatic *ps;
    PileDyn *pd;
    int32_t *enabled;
};

struct Sizes {
    int64_t N, A, C, T, CH, P, GI, GP;
    int64_t CT, E;   // contact tiles and candidate-list entries of all piles
    int64_t GB;   // blocks of the persistent gravity grid (0 = one block per item)
    int64_t TN, TL, TG;   // tree nodes, leaves and 32-sphere groups of all piles (TN = 0: direct sum)
    int32_t K;    // history slots per sphere (world-wide)
    int32_t adapt;   // some pile integrates rotation with the adaptive RK5(4)
    int32_t gtile;   // spheres per tile of the symmetric gravity form (512, or 128 in the mixed path)
    int32_t icap;    // contact inbox entries used per tile range (<= the kernel's capacity)
    int32_t cmode;   // contact pass: 0 = one thread per sphere, 1 = tiles with a shared-memory inbox
    int32_t gacc_on; // mixed symmetric gravity: piles of more than one tile leave their sums in gacc,
                     // which k_grav_acc_to_force turns into forces
    int32_t grav;    // some pile has self-gravity (G > 0)
};

// ---- kernel launchers (kernels_*.cu) -------------------------------------
void launch_agg_begin(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st);
void launch_pile_begin(const Arrays &a, const Sizes &z, cudaStream_t st);
void launch_keys(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st);
void launch_scan(const Arrays &a, const Sizes &z, cudaStream_t st);
void launch_scatter(const Arrays &a, const Sizes &z, cudaStream_t st);
void launch_cell_order(const Arrays &a, const Sizes &z, cudaStream_t st);
void launch_gather(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st);
void launch_contact(const Arrays &a, const Sizes &z, bool fp64, int K, cudaStream_t st);
cudaError_t contact_setup(bool fp64, int K);
// sym: symmetric tile-pair form (items are (pile, tile a, tile b), gnchunk =
// tiles per pile); tiles of 512 spheres, or of 128 (mixed path, small piles)
constexpr int kGravSymTile = 512, kGravSymTileSmall = 128, kGravSymTileTiny = 64;
constexpr int64_t kTinyTileMaxN = 2048;   // largest pile that may use 64-sphere tiles
// largest pile (spheres) of a world that may use tiles smaller than 512
#ifndef DEM_SMALL_TILE_MAX
#define DEM_SMALL_TILE_MAX 8192
#endif
constexpr int64_t kSmallTileMaxN = DEM_SMALL_TILE_MAX;
void launch_gravity(const Arrays &a, const Sizes &z, bool fp64, int block, int ib, bool pack,
                    bool sym, cudaStream_t st);
int gravity_blocks_per_sm(bool fp64, int block, int ib, bool pack, bool sym, int tile);
void launch_agg_end(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st);
void launch_pile_end(const Arrays &a, const Sizes &z, cudaStream_t st);
void launch_fill_ids(const Arrays &a, const Sizes &z, cudaStream_t st);
// order: highest multipole rank of accepted cells (2 or 4)
void launch_tree_gravity(const Arrays &a, const Sizes &z, int max_depth, int order, cudaStream_t st);
void launch_force_rebuild(const Arrays &a, const Sizes &z, int slot, cudaStream_t st);
// programmatic dependent launch for the launches that follow on this host
// thread: on for worlds of at most kPdlMaxSpheres spheres (launch.cuh)
void set_launch_pdl(int64_t n_spheres);
// bulk record of piles into watch.now (mode 0: every pile, or only slot
// `only` when >= 0; mode 1: the watch evaluation inside the step graph, armed
// piles whose step is due)
void launch_bulk(const Arrays &a, const Sizes &z, int mode, int only, cudaStream_t st);

}  // namespace dem
