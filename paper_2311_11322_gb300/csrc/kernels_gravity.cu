// kernels_gravity.cu -- softened self-gravity of every pile by a tiled direct
// sum (Sec. 2.2.3, Eq. particle_gravity with Plummer softening):
//   F_i = G m_i sum_j m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2},
// over the spheres j of the same pile that belong to other aggregates.
// Internal pairs of a rigid aggregate cancel in its total force and torque
// (Eq. agg_gravity, Eq. gravity_torque), so leaving them out changes no
// aggregate total; in FP32 it also removes their rounding noise.
//
// Work item = (pile, block of i-spheres, range of j-spheres).  j-tiles are
// staged in shared memory (one float4 / dbl4 per sphere: position relative
// to the pile frame and mass) and broadcast to the whole block; each thread
// keeps IB i-spheres in registers.  Members of an aggregate are contiguous, so
// the spheres to skip for a block lie in one short index range: only the one
// or two tiles that overlap it take the masked inner loop.
// Mixed: FP32 pair terms, FP32 partial sums flushed into FP64 every kFlush
// j-spheres.  FP64: double throughout.
// A pile with several j-ranges writes one partial per (range, sphere), the
// range's FP64 sum rounded to FP32 (one more rounding of a sum of ~2,000
// terms), and k_grav_combine adds them in FP64 in range order (deterministic).
//
// Symmetric form (default; packed FP32 in the mixed path, scalar FP64 in the
// FP64 path).  The pair term is antisymmetric
// (Newton's third law): F_ij = -F_ji.  The pile is cut into tiles of 512
// spheres; a work item is a pair of tiles (a, b), a < b, and evaluates each of
// its 512 x 512 pairs once, adding the term to sphere i of tile a and its
// negative to sphere j of tile b.  Each warp keeps 128 i-spheres in registers
// (4 per lane) and passes 32 j-spheres round the warp by register shuffles,
// each j carrying its own running sum, so a j-sphere visits all 128 i-spheres
// of the warp in 32 steps; per pair this costs 16 FP32 instructions and one
// reciprocal square root where the one-sided form needs 24 and two.  Items
// (a, a) take the one-sided form.  Mixed path: every item adds its FP32
// i-sums and j-sums, scaled by a power of two and rounded once, to 64-bit
// integer accumulators per sphere (atomic integer adds, which give the same
// result in any order, so nothing depends on the schedule);
// k_grav_acc_to_force turns them into forces.  FP64 path: every item writes
// its i-sums (one per b) and j-sums (one per a) as FP64 partials, and
// k_grav_combine_sym64 adds a sphere's partials in tile order.
#include "dem_internal.h"
#include "devmath.cuh"
#include "launch.cuh"

namespace dem {

constexpr int kFlush = 1024;

// Packed FP32 pairs (two lanes of one 64-bit register) for the sm_100-family
// f32x2 instructions: one instruction does the same operation on two
// i-spheres, halving the issue slots of the FP32 part of the pair term.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// One work item of the mixed-precision kernel (see the file comment).
template <int BS, int IB>
__device__ __forceinline__ void gravity32_item(const Arrays &a, const int4 it, float4 *sp, int *sag,
                                               int *excl)
{
    const int p = it.x;
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int i0 = it.y, j0 = it.z, j1 = it.w;
    const float eps2 = (float)S.eps2;
    const float4 far = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f);
    if (threadIdx.x == 0) {
        int ilast = min(i0 + BS * IB, ns) - 1;
        int alo = a.sph_agg[s0 + i0], ahi = a.sph_agg[s0 + ilast];
        int64_t g0 = S.a0;
        excl[0] = a.agg_first[g0 + alo];
        excl[1] = a.agg_first[g0 + ahi] + a.agg_count[g0 + ahi];
    }
    float4 xi[IB];
    int ai[IB];
    float ax[IB], ay[IB], az[IB];
    double dx_[IB], dy_[IB], dz_[IB];
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        int il = i0 + threadIdx.x + k * BS;
        bool ok = il < ns;
        xi[k] = ok ? a.gpos32[s0 + il] : make_float4(0.f, 0.f, 0.f, 0.f);
        ai[k] = ok ? a.sph_agg[s0 + il] : -2;
        ax[k] = ay[k] = az[k] = 0.f;
        dx_[k] = dy_[k] = dz_[k] = 0.0;
    }
    __syncthreads();
    const int elo = excl[0], ehi = excl[1];
    // register prefetch of the next tile overlaps its L2 latency with compute
    int j = j0 + threadIdx.x;
    float4 nxt = j < j1 ? a.gpos32[s0 + j] : far;
    int nxa = (j0 < ehi && j0 + BS > elo && j < j1) ? a.sph_agg[s0 + j] : -1;
    int since = 0;
    for (int jt = j0; jt < j1; jt += BS) {
        const bool masked = jt < ehi && jt + BS > elo;
        __syncthreads();
        sp[threadIdx.x] = nxt;
        sag[threadIdx.x] = nxa;
        __syncthreads();
        const int jn = jt + BS;
        j = jn + threadIdx.x;
        nxt = j < j1 ? a.gpos32[s0 + j] : far;
        nxa = (jn < ehi && jn + BS > elo && j < j1) ? a.sph_agg[s0 + j] : -1;
        if (masked) {
            for (int jj = 0; jj < BS; ++jj) {
                float4 pj = sp[jj];
                int aj = sag[jj];
#pragma unroll
                for (int k = 0; k < IB; ++k) {
                    float ddx = pj.x - xi[k].x, ddy = pj.y - xi[k].y, ddz = pj.z - xi[k].z;
                    float r2 = fmaf(ddz, ddz, fmaf(ddy, ddy, fmaf(ddx, ddx, eps2)));
                    float inv = rsqrtf(r2);
                    float s = (pj.w * inv) * (inv * inv);
                    s = (aj == ai[k]) ? 0.f : s;
                    ax[k] = fmaf(ddx, s, ax[k]);
                    ay[k] = fmaf(ddy, s, ay[k]);
                    az[k] = fmaf(ddz, s, az[k]);
                }
            }
        } else {
#pragma unroll 8
            for (int jj = 0; jj < BS; ++jj) {
                float4 pj = sp[jj];
#pragma unroll
                for (int k = 0; k < IB; ++k) {
                    float ddx = pj.x - xi[k].x, ddy = pj.y - xi[k].y, ddz = pj.z - xi[k].z;
                    float r2 = fmaf(ddz, ddz, fmaf(ddy, ddy, fmaf(ddx, ddx, eps2)));
                    float inv = rsqrtf(r2);
                    float s = (pj.w * inv) * (inv * inv);
                    ax[k] = fmaf(ddx, s, ax[k]);
                    ay[k] = fmaf(ddy, s, ay[k]);
                    az[k] = fmaf(ddz, s, az[k]);
                }
            }
        }
        since += BS;
        if (since >= kFlush) {
            since = 0;
#pragma unroll
            for (int k = 0; k < IB; ++k) {
                dx_[k] += ax[k]; dy_[k] += ay[k]; dz_[k] += az[k];
                ax[k] = ay[k] = az[k] = 0.f;
            }
        }
    }
    const int nch = a.gnchunk[p];
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        int il = i0 + threadIdx.x + k * BS;
        if (il >= ns) continue;
        double sx = dx_[k] + ax[k], sy = dy_[k] + ay[k], sz = dz_[k] + az[k];
        if (nch == 1) {
            double gm = S.G * a.m64[s0 + il];
            a.fg[s0 + il] = make_dbl4(gm * sx, gm * sy, gm * sz, 0.0);
        } else {
            int64_t slot = a.gpart_base[p] + (int64_t)(j0 / ((ns + nch - 1) / nch)) * ns + il;
            ((float4 *)a.gpart)[slot] = make_float4((float)sx, (float)sy, (float)sz, 0.f);
        }
    }
}


// Packed variant: each thread keeps NP pairs of i-spheres in f32x2 registers
// for the whole work item (masked tiles included); the FP64 flush targets sit
// in shared memory, which keeps the register count, and so the number of
// resident warps, up.  Same terms and order of summation per sphere as the
// scalar kernel up to the FP32 rounding of packed vs scalar lanes.
template <int BS, int NP>
__device__ __forceinline__ void gravity32p_item(const Arrays &a, const int4 it, float4 *sp, int *sag,
                                                int *excl, double *sacc)
{
    constexpr int IB = 2 * NP;
    const int p = it.x;
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int i0 = it.y, j0 = it.z, j1 = it.w;
    const float eps2 = (float)S.eps2;
    const float4 far = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f);
    const int t = threadIdx.x;
    if (t == 0) {
        int ilast = min(i0 + BS * IB, ns) - 1;
        int alo = a.sph_agg[s0 + i0], ahi = a.sph_agg[s0 + ilast];
        int64_t g0 = S.a0;
        excl[0] = a.agg_first[g0 + alo];
        excl[1] = a.agg_first[g0 + ahi] + a.agg_count[g0 + ahi];
    }
    f2_t px[NP], py[NP], pz[NP], qx[NP], qy[NP], qz[NP];
    int ai[IB];
    const f2_t zero2 = f2_pack(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float4 u, v;
        int ila = i0 + t + (2 * q) * BS, ilb = i0 + t + (2 * q + 1) * BS;
        u = ila < ns ? a.gpos32[s0 + ila] : make_float4(0.f, 0.f, 0.f, 0.f);
        v = ilb < ns ? a.gpos32[s0 + ilb] : make_float4(0.f, 0.f, 0.f, 0.f);
        ai[2 * q] = ila < ns ? a.sph_agg[s0 + ila] : -2;
        ai[2 * q + 1] = ilb < ns ? a.sph_agg[s0 + ilb] : -2;
        px[q] = f2_pack(u.x, v.x);
        py[q] = f2_pack(u.y, v.y);
        pz[q] = f2_pack(u.z, v.z);
        qx[q] = qy[q] = qz[q] = zero2;
    }
#pragma unroll
    for (int c = 0; c < 6 * NP; ++c) sacc[c * BS + t] = 0.0;
    __syncthreads();
    const int elo = excl[0], ehi = excl[1];
    const f2_t e2 = f2_pack(eps2, eps2);
    int j = j0 + t;
    float4 nxt = j < j1 ? a.gpos32[s0 + j] : far;
    int nxa = (j0 < ehi && j0 + BS > elo && j < j1) ? a.sph_agg[s0 + j] : -1;
    int since = 0;
    const ulonglong2 *dup = reinterpret_cast<const ulonglong2 *>(sp);
    for (int jt = j0; jt < j1; jt += BS) {
        const bool masked = jt < ehi && jt + BS > elo;
        __syncthreads();
        sp[2 * t] = make_float4(nxt.x, nxt.x, nxt.y, nxt.y);
        sp[2 * t + 1] = make_float4(nxt.z, nxt.z, nxt.w, nxt.w);
        sag[t] = nxa;
        __syncthreads();
        const int jn = jt + BS;
        j = jn + t;
        nxt = j < j1 ? a.gpos32[s0 + j] : far;
        nxa = (jn < ehi && jn + BS > elo && j < j1) ? a.sph_agg[s0 + j] : -1;
        if (masked) {
            for (int jj = 0; jj < BS; ++jj) {
                const ulonglong2 xy = dup[2 * jj], zm = dup[2 * jj + 1];
                const int aj = sag[jj];
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    f2_t ddx = f2_sub(xy.x, px[q]), ddy = f2_sub(xy.y, py[q]), ddz = f2_sub(zm.x, pz[q]);
                    f2_t r2 = f2_fma(ddz, ddz, f2_fma(ddy, ddy, f2_fma(ddx, ddx, e2)));
                    float r2a, r2b;
                    f2_unpack(r2, r2a, r2b);
                    f2_t inv = f2_pack(rsqrtf(r2a), rsqrtf(r2b));
                    f2_t sv = f2_mul(f2_mul(zm.y, inv), f2_mul(inv, inv));
                    float sa, sb;
                    f2_unpack(sv, sa, sb);
                    sa = (aj == ai[2 * q]) ? 0.f : sa;
                    sb = (aj == ai[2 * q + 1]) ? 0.f : sb;
                    sv = f2_pack(sa, sb);
                    qx[q] = f2_fma(ddx, sv, qx[q]);
                    qy[q] = f2_fma(ddy, sv, qy[q]);
                    qz[q] = f2_fma(ddz, sv, qz[q]);
                }
            }
        } else {
#pragma unroll 4
            for (int jj = 0; jj < BS; ++jj) {
                const ulonglong2 xy = dup[2 * jj], zm = dup[2 * jj + 1];
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    f2_t ddx = f2_sub(xy.x, px[q]), ddy = f2_sub(xy.y, py[q]), ddz = f2_sub(zm.x, pz[q]);
                    f2_t r2 = f2_fma(ddz, ddz, f2_fma(ddy, ddy, f2_fma(ddx, ddx, e2)));
                    float r2a, r2b;
                    f2_unpack(r2, r2a, r2b);
                    f2_t inv = f2_pack(rsqrtf(r2a), rsqrtf(r2b));
                    f2_t sv = f2_mul(f2_mul(zm.y, inv), f2_mul(inv, inv));
                    qx[q] = f2_fma(ddx, sv, qx[q]);
                    qy[q] = f2_fma(ddy, sv, qy[q]);
                    qz[q] = f2_fma(ddz, sv, qz[q]);
                }
            }
        }
        since += BS;
        if (since >= kFlush || jt + BS >= j1) {
            since = 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float lo, hi;
                f2_unpack(qx[q], lo, hi);
                sacc[(6 * q + 0) * BS + t] += lo;
                sacc[(6 * q + 1) * BS + t] += hi;
                f2_unpack(qy[q], lo, hi);
                sacc[(6 * q + 2) * BS + t] += lo;
                sacc[(6 * q + 3) * BS + t] += hi;
                f2_unpack(qz[q], lo, hi);
                sacc[(6 * q + 4) * BS + t] += lo;
                sacc[(6 * q + 5) * BS + t] += hi;
                qx[q] = qy[q] = qz[q] = zero2;
            }
        }
    }
    const int nch = a.gnchunk[p];
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int il = i0 + t + (2 * q + h) * BS;
            if (il >= ns) continue;
            double sx = sacc[(6 * q + 0 + h) * BS + t], sy = sacc[(6 * q + 2 + h) * BS + t],
                   sz = sacc[(6 * q + 4 + h) * BS + t];
            if (nch == 1) {
                double gm = S.G * a.m64[s0 + il];
                a.fg[s0 + il] = make_dbl4(gm * sx, gm * sy, gm * sz, 0.0);
            } else {
                int64_t slot = a.gpart_base[p] + (int64_t)(j0 / ((ns + nch - 1) / nch)) * ns + il;
                ((float4 *)a.gpart)[slot] = make_float4((float)sx, (float)sy, (float)sz, 0.f);
            }
        }
}

// Next work item of a persistent grid.  Every block takes items until it
// draws one past the end, so a launch makes exactly GI + gridDim.x draws; the
// last draw puts the counter back to zero for the next launch (the counter
// is zeroed once when the layout is uploaded), so no memset node is needed
// between the kernels of a step.
__device__ __forceinline__ int grab_item(int32_t *counter, int64_t GI)
{
    const int v = atomicAdd(counter, 1);
    if ((int64_t)v == GI + (int64_t)gridDim.x - 1) atomicExch(counter, 0);
    return v;
}

template <int BS, int NP>
__global__ void __launch_bounds__(BS) k_gravity32p(Arrays a, Sizes z)
{
    pdl_enter();
    __shared__ float4 sp[2 * BS];
    __shared__ int sag[BS];
    __shared__ int excl[2];
    __shared__ double sacc[6 * NP * BS];
    __shared__ int next;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) next = grab_item(a.gcounter, z.GI);
        __syncthreads();
        const int item = next;
        if (item >= z.GI) return;
        gravity32p_item<BS, NP>(a, a.gitems[item], sp, sag, excl, sacc);
    }
}

// Persistent grid: each block takes the next item from a counter (see
// grab_item) until the list is exhausted.  Items are listed largest first;
// which block runs an item does not change its result, so the sums stay
// deterministic.
template <int BS, int IB>
__global__ void __launch_bounds__(BS) k_gravity32(Arrays a, Sizes z)
{
    pdl_enter();
    __shared__ float4 sp[BS];
    __shared__ int sag[BS];
    __shared__ int excl[2];
    __shared__ int next;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) next = grab_item(a.gcounter, z.GI);
        __syncthreads();
        const int item = next;
        if (item >= z.GI) return;
        gravity32_item<BS, IB>(a, a.gitems[item], sp, sag, excl);
    }
}

template <int BS, int IB>
__global__ void __launch_bounds__(BS) k_gravity64(Arrays a, Sizes z)
{
    pdl_enter();
    __shared__ dbl4 sp[BS];
    __shared__ int sag[BS];
    __shared__ int excl[2];
    const int4 it = a.gitems[blockIdx.x];
    const int p = it.x;
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int i0 = it.y, j0 = it.z, j1 = it.w;
    const double eps2 = S.eps2;
    if (threadIdx.x == 0) {
        int ilast = min(i0 + BS * IB, ns) - 1;
        int alo = a.sph_agg[s0 + i0], ahi = a.sph_agg[s0 + ilast];
        int64_t g0 = S.a0;
        excl[0] = a.agg_first[g0 + alo];
        excl[1] = a.agg_first[g0 + ahi] + a.agg_count[g0 + ahi];
    }
    dbl4 xi[IB];
    int ai[IB];
    double ax[IB], ay[IB], az[IB];
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        int il = i0 + threadIdx.x + k * BS;
        bool ok = il < ns;
        xi[k] = ok ? a.gpos64[s0 + il] : make_dbl4(0, 0, 0, 0);
        ai[k] = ok ? a.sph_agg[s0 + il] : -2;
        ax[k] = ay[k] = az[k] = 0.0;
    }
    __syncthreads();
    const int elo = excl[0], ehi = excl[1];
    for (int jt = j0; jt < j1; jt += BS) {
        __syncthreads();
        int j = jt + threadIdx.x;
        if (j < j1) {
            sp[threadIdx.x] = a.gpos64[s0 + j];
            sag[threadIdx.x] = a.sph_agg[s0 + j];
        } else {
            sp[threadIdx.x] = make_dbl4(1.0e150, 1.0e150, 1.0e150, 0.0);
            sag[threadIdx.x] = -1;
        }
        __syncthreads();
        const bool masked = jt < ehi && jt + BS > elo;
        for (int jj = 0; jj < BS; ++jj) {
            dbl4 pj = sp[jj];
            int aj = sag[jj];
#pragma unroll
            for (int k = 0; k < IB; ++k) {
                double ddx = pj.x - xi[k].x, ddy = pj.y - xi[k].y, ddz = pj.z - xi[k].z;
                double r2 = ddx * ddx + ddy * ddy + ddz * ddz + eps2;
                double inv = rsqrt(r2);
                double s = pj.w * inv * inv * inv;
                if (masked && aj == ai[k]) s = 0.0;
                ax[k] += ddx * s;
                ay[k] += ddy * s;
                az[k] += ddz * s;
            }
        }
    }
    const int nch = a.gnchunk[p];
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        int il = i0 + threadIdx.x + k * BS;
        if (il >= ns) continue;
        if (nch == 1) {
            double gm = S.G * a.m64[s0 + il];
            a.fg[s0 + il] = make_dbl4(gm * ax[k], gm * ay[k], gm * az[k], 0.0);
        } else {
            int64_t slot = a.gpart_base[p] + (int64_t)(j0 / ((ns + nch - 1) / nch)) * ns + il;
            ((dbl4 *)a.gpart)[slot] = make_dbl4(ax[k], ay[k], az[k], 0.0);
        }
    }
}

// ---------------------------------------------------------------- symmetric form
constexpr int kSymBS = 128, kSymIB = 4, kSymTile = kSymBS * kSymIB;   // 512 spheres per tile
// shape of the mixed path's 512-sphere tiles: warps per block x i-spheres per lane
#ifndef DEM_SYM_WPB
#define DEM_SYM_WPB 4
#endif
constexpr int kBigWPB = DEM_SYM_WPB, kBigIB = 512 / (32 * DEM_SYM_WPB);
static_assert(32 * kBigWPB * kBigIB == kSymTile, "512-sphere tiles");
// launch bounds of the symmetric kernel (optionally with a minimum number of
// resident blocks per SM, which caps its registers)
#ifdef DEM_GSYM_MINB
#define DEM_GSYM_BOUNDS __launch_bounds__(32 * WPB, DEM_GSYM_MINB)
#else
#define DEM_GSYM_BOUNDS __launch_bounds__(32 * WPB)
#endif

// Mixed symmetric form: add one tile item's FP32 sum on home sphere s to its
// 64-bit integer accumulators.  The sum is scaled by the pile's power of two
// (exact) and rounded to the nearest integer once; integer additions are
// exact, so the accumulated value does not depend on the order in which the
// items finish, and the result is the same in any schedule or batch.  A sum
// outside the accumulators' range (or NaN) adds nothing and returns the
// pile flag to raise.
__device__ __forceinline__ void grav_accumulate(const Arrays &a, int64_t s, float x, float y, float z,
                                                float scale, int *bad)
{
    // x * 2^k is exact in FP32 (a power-of-two scale; results below the
    // normal range flush to zero, far below half a quantum)
    const float vx = x * scale, vy = y * scale, vz = z * scale;
    const float lim = 2305843009213693952.0f;   // 2^61
    const bool ok = fabsf(vx) < lim && fabsf(vy) < lim && fabsf(vz) < lim;
    unsigned long long *g = a.gacc + 4 * s;
    atomicAdd(g, (unsigned long long)(ok ? __float2ll_rn(vx) : 0ll));
    atomicAdd(g + 1, (unsigned long long)(ok ? __float2ll_rn(vy) : 0ll));
    atomicAdd(g + 2, (unsigned long long)(ok ? __float2ll_rn(vz) : 0ll));
    if (!ok) atomicOr(bad, (vx != vx || vy != vy || vz != vz) ? DEM_FLAG_NONFINITE : DEM_FLAG_GRAV_RANGE);
}

// Partial slots of pile p: i-sums of tile pair (a, b) at [b][i], j-sums at
// [T + a][j], rows of ns spheres from gpart_base[p].
__device__ __forceinline__ int64_t sym_slot(const Arrays &a, int p, int64_t ns, int64_t row, int64_t i)
{
    return a.gpart_base[p] + row * ns + i;
}

// One step of the ring: the lane's IB i-spheres against the j-sphere it holds.
template <bool MASK, int IB>
__device__ __forceinline__ void sym_pairs(const float4 &pj, int aj, const float4 (&xi)[IB],
                                          const float (&nm)[IB], const int (&ai)[IB],
                                          float (&ax)[IB], float (&ay)[IB],
                                          float (&az)[IB], float &fx, float &fy, float &fz,
                                          float eps2)
{
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        const float dx = pj.x - xi[k].x, dy = pj.y - xi[k].y, dz = pj.z - xi[k].z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        const float inv = rsqrtf(r2);
        const float inv3 = (inv * inv) * inv;
        float si = pj.w * inv3, sj = nm[k] * inv3;
        if (MASK && aj == ai[k]) si = sj = 0.f;
        ax[k] = fmaf(dx, si, ax[k]);
        ay[k] = fmaf(dy, si, ay[k]);
        az[k] = fmaf(dz, si, az[k]);
        fx = fmaf(dx, sj, fx);
        fy = fmaf(dy, sj, fy);
        fz = fmaf(dz, sj, fz);
    }
}

// 32 ring steps over one chunk of 32 j-spheres (one per lane at the start,
// back in its lane at the end with the sum over the warp's 128 i-spheres).
template <bool MASK, int IB>
__device__ __forceinline__ float4 sym_ring(float4 pj, int aj, const float4 (&xi)[IB],
                                           const float (&nm)[IB], const int (&ai)[IB],
                                           float (&ax)[IB], float (&ay)[IB],
                                           float (&az)[IB], float eps2)
{
    const int src = (threadIdx.x + 1) & 31;
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll 4
    for (int s = 0; s < 32; ++s) {
        sym_pairs<MASK, IB>(pj, aj, xi, nm, ai, ax, ay, az, fx, fy, fz, eps2);
        pj.x = __shfl_sync(0xffffffffu, pj.x, src);
        pj.y = __shfl_sync(0xffffffffu, pj.y, src);
        pj.z = __shfl_sync(0xffffffffu, pj.z, src);
        pj.w = __shfl_sync(0xffffffffu, pj.w, src);
        fx = __shfl_sync(0xffffffffu, fx, src);
        fy = __shfl_sync(0xffffffffu, fy, src);
        fz = __shfl_sync(0xffffffffu, fz, src);
        if (MASK) aj = __shfl_sync(0xffffffffu, aj, src);
    }
    return make_float4(fx, fy, fz, 0.f);
}

// ring steps unrolled per loop iteration (a tuning constant)
#ifndef DEM_RING_UNROLL
#define DEM_RING_UNROLL 16
#endif
constexpr int kRingUnroll = DEM_RING_UNROLL;

// Packed ring (unmasked tile pairs): each lane holds two j-spheres, packed
// into the two halves of 64-bit registers, and its 4 i-spheres duplicated into
// both halves, so one f32x2 instruction evaluates the same step of two pairs.
// A chunk is 64 j-spheres (j and j + 32 in lane l).  The i-sums are kept per
// half and added at the end of the item; the j-sums travel with their j.
template <int IB>
__device__ __forceinline__ void sym_ring2(const float4 &pa, const float4 &pb,
                                          const f2_t (&xx)[IB], const f2_t (&xy)[IB],
                                          const f2_t (&xz)[IB], const f2_t (&nm2)[IB],
                                          f2_t (&qx)[IB], f2_t (&qy)[IB], f2_t (&qz)[IB],
                                          f2_t e2, float4 &fa, float4 &fb)
{
    const int src = (threadIdx.x + 1) & 31;
    f2_t jx = f2_pack(pa.x, pb.x), jy = f2_pack(pa.y, pb.y), jz = f2_pack(pa.z, pb.z),
         jm = f2_pack(pa.w, pb.w);
    f2_t fx = f2_pack(0.f, 0.f), fy = fx, fz = fx;
#pragma unroll kRingUnroll
    for (int s = 0; s < 32; ++s) {
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const f2_t dx = f2_sub(jx, xx[k]), dy = f2_sub(jy, xy[k]), dz = f2_sub(jz, xz[k]);
            const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_fma(dx, dx, e2)));
            float ra, rb;
            f2_unpack(r2, ra, rb);
            const f2_t inv = f2_pack(rsqrtf(ra), rsqrtf(rb));
            const f2_t inv3 = f2_mul(f2_mul(inv, inv), inv);
            const f2_t si = f2_mul(jm, inv3), sj = f2_mul(nm2[k], inv3);
            qx[k] = f2_fma(dx, si, qx[k]);
            qy[k] = f2_fma(dy, si, qy[k]);
            qz[k] = f2_fma(dz, si, qz[k]);
            fx = f2_fma(dx, sj, fx);
            fy = f2_fma(dy, sj, fy);
            fz = f2_fma(dz, sj, fz);
        }
        jx = __shfl_sync(0xffffffffu, jx, src);
        jy = __shfl_sync(0xffffffffu, jy, src);
        jz = __shfl_sync(0xffffffffu, jz, src);
        jm = __shfl_sync(0xffffffffu, jm, src);
        fx = __shfl_sync(0xffffffffu, fx, src);
        fy = __shfl_sync(0xffffffffu, fy, src);
        fz = __shfl_sync(0xffffffffu, fz, src);
    }
    float ax, bx, ay, by, az, bz;
    f2_unpack(fx, ax, bx);
    f2_unpack(fy, ay, by);
    f2_unpack(fz, az, bz);
    fa = make_float4(ax, ay, az, 0.f);
    fb = make_float4(bx, by, bz, 0.f);
}

// Work item (pile, tile a, tile b): the symmetric pass for a < b, the
// one-sided pass over the tile itself for a == b.  sp/sag: tile b staged in
// shared memory; sj: per-warp j-sums.  WPB warps per block, each with
// 32 x IB i-spheres: tiles of 32 WPB IB spheres (512 for the large-pile
// form, 128 for small piles whose 512-sphere tile pairs would not fill the GPU).
template <int WPB, int IB>
__device__ __forceinline__ void gravity32s_item(const Arrays &a, const int4 it, float4 *sp, int *sag,
                                                float4 *sj, int *bad)
{
    constexpr int kSymBS = 32 * WPB, kSymTile = kSymBS * IB;
    const int p = it.x;
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int T = a.gnchunk[p];
    const int ta = it.y, tb = it.z;
    const bool diag = ta == tb;
    const float eps2 = (float)S.eps2;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int jb0 = tb * kSymTile;
    const int nj = min(kSymTile, ns - jb0);
    for (int m = threadIdx.x; m < kSymTile; m += kSymBS) {
        const int j = jb0 + m;
        sp[m] = j < ns ? a.gpos32[s0 + j] : make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f);
        sag[m] = j < ns ? a.sph_agg[s0 + j] : -1;
    }
    float4 xi[IB];
    float nm[IB];
    int ai[IB];
    float ax[IB], ay[IB], az[IB];
    const int i0 = ta * kSymTile + w * (32 * IB) + l;
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        const int i = i0 + 32 * k;
        const bool ok = i < ns;
        xi[k] = ok ? a.gpos32[s0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        ai[k] = ok ? a.sph_agg[s0 + i] : -2;
        nm[k] = -xi[k].w;
        ax[k] = ay[k] = az[k] = 0.f;
    }
    // an aggregate can span the two tiles only if it spans their boundary
    const bool masked = diag || a.sph_agg[s0 + (int64_t)ta * kSymTile + kSymTile - 1] == a.sph_agg[s0 + jb0];
    __syncthreads();
    if (diag) {
        for (int jj = 0; jj < nj; ++jj) {
            const float4 pj = sp[jj];
            const int aj = sag[jj];
#pragma unroll
            for (int k = 0; k < IB; ++k) {
                const float dx = pj.x - xi[k].x, dy = pj.y - xi[k].y, dz = pj.z - xi[k].z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
                const float inv = rsqrtf(r2);
                float si = (pj.w * inv) * (inv * inv);
                si = aj == ai[k] ? 0.f : si;
                ax[k] = fmaf(dx, si, ax[k]);
                ay[k] = fmaf(dy, si, ay[k]);
                az[k] = fmaf(dz, si, az[k]);
            }
        }
    } else if (masked) {
        for (int c = 0; c * 32 < nj; ++c) {
            const float4 pj = sp[c * 32 + l];
            const int aj = sag[c * 32 + l];
            sj[w * kSymTile + c * 32 + l] = sym_ring<true, IB>(pj, aj, xi, nm, ai, ax, ay, az, eps2);
        }
    } else {
        f2_t xx[IB], xy[IB], xz[IB], nm2[IB], qx[IB], qy[IB], qz[IB];
        const f2_t zero2 = f2_pack(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            xx[k] = f2_pack(xi[k].x, xi[k].x);
            xy[k] = f2_pack(xi[k].y, xi[k].y);
            xz[k] = f2_pack(xi[k].z, xi[k].z);
            nm2[k] = f2_pack(nm[k], nm[k]);
            qx[k] = qy[k] = qz[k] = zero2;
        }
        const f2_t e2 = f2_pack(eps2, eps2);
        for (int c = 0; c * 64 < nj; ++c) {
            float4 fa, fb;
            sym_ring2<IB>(sp[c * 64 + l], sp[c * 64 + 32 + l], xx, xy, xz, nm2, qx, qy, qz, e2, fa, fb);
            sj[w * kSymTile + c * 64 + l] = fa;
            sj[w * kSymTile + c * 64 + 32 + l] = fb;
        }
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            float lo, hi;
            f2_unpack(qx[k], lo, hi);
            ax[k] = lo + hi;
            f2_unpack(qy[k], lo, hi);
            ay[k] = lo + hi;
            f2_unpack(qz[k], lo, hi);
            az[k] = lo + hi;
        }
    }
    if (!diag) {
        __syncthreads();
        for (int m = threadIdx.x; m < nj; m += kSymBS) {
            float4 u = sj[m];
#pragma unroll
            for (int v = 1; v < WPB; ++v) {
                const float4 t = sj[v * kSymTile + m];
                u.x += t.x;
                u.y += t.y;
                u.z += t.z;
            }
            grav_accumulate(a, s0 + jb0 + m, u.x, u.y, u.z, S.gscale_f, bad);
        }
    }
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        const int i = i0 + 32 * k;
        if (i >= ns) continue;
        if (T == 1) {
            const double gm = S.G * a.m64[s0 + i];
            a.fg[s0 + i] = make_dbl4(gm * ax[k], gm * ay[k], gm * az[k], 0.0);
        } else {
            grav_accumulate(a, s0 + i, ax[k], ay[k], az[k], S.gscale_f, bad);
        }
    }
}

template <int WPB, int IB>
__global__ void DEM_GSYM_BOUNDS k_gravity32s(Arrays a, Sizes z)
{
    pdl_enter();
    constexpr int kTile = 32 * WPB * IB;
    __shared__ float4 sp[kTile];
    __shared__ int sag[kTile];
    __shared__ float4 sj[WPB * kTile];
    __shared__ int next, bad, bad_pile;   // flags raised by the block's last item, and its pile
    if (threadIdx.x == 0) bad = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            if (bad) {
                atomicOr(&a.pd[bad_pile].flags, bad);
                bad = 0;
            }
            next = grab_item(a.gcounter, z.GI);
            if (next < z.GI) bad_pile = a.gitems[next].x;
        }
        __syncthreads();
        const int item = next;
        if (item >= z.GI) return;
        gravity32s_item<WPB, IB>(a, a.gitems[item], sp, sag, sj, &bad);
    }
}

// FP64 path, symmetric form: the same tile pairs and ring as the mixed path
// in double precision (scalar: no packed FP64 instructions), partial sums in
// FP64 and combined in FP64.  Shared memory: tile b (32 B per sphere), its
// aggregates and the per-warp j-sums (4 x 512 x 32 B): 82 KB per block.
template <bool MASK>
__device__ __forceinline__ dbl4 sym_ring64(dbl4 pj, int aj, const dbl4 (&xi)[kSymIB], const int (&ai)[kSymIB],
                                           double (&ax)[kSymIB], double (&ay)[kSymIB], double (&az)[kSymIB],
                                           double eps2)
{
    const int src = (threadIdx.x + 1) & 31;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int s = 0; s < 32; ++s) {
#pragma unroll
        for (int k = 0; k < kSymIB; ++k) {
            const double dx = pj.x - xi[k].x, dy = pj.y - xi[k].y, dz = pj.z - xi[k].z;
            const double r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
            const double inv = rsqrt(r2);
            const double inv3 = (inv * inv) * inv;
            double si = pj.w * inv3, sj = -xi[k].w * inv3;
            if (MASK && aj == ai[k]) si = sj = 0.0;
            ax[k] = fma(dx, si, ax[k]);
            ay[k] = fma(dy, si, ay[k]);
            az[k] = fma(dz, si, az[k]);
            fx = fma(dx, sj, fx);
            fy = fma(dy, sj, fy);
            fz = fma(dz, sj, fz);
        }
        pj.x = __shfl_sync(0xffffffffu, pj.x, src);
        pj.y = __shfl_sync(0xffffffffu, pj.y, src);
        pj.z = __shfl_sync(0xffffffffu, pj.z, src);
        pj.w = __shfl_sync(0xffffffffu, pj.w, src);
        fx = __shfl_sync(0xffffffffu, fx, src);
        fy = __shfl_sync(0xffffffffu, fy, src);
        fz = __shfl_sync(0xffffffffu, fz, src);
        if (MASK) aj = __shfl_sync(0xffffffffu, aj, src);
    }
    return make_dbl4(fx, fy, fz, 0.0);
}

__device__ __forceinline__ void gravity64s_item(const Arrays &a, const int4 it, dbl4 *sp, int *sag, dbl4 *sj)
{
    const int p = it.x;
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int T = a.gnchunk[p];
    const int ta = it.y, tb = it.z;
    const bool diag = ta == tb;
    const double eps2 = S.eps2;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int jb0 = tb * kSymTile;
    const int nj = min(kSymTile, ns - jb0);
    for (int m = threadIdx.x; m < kSymTile; m += kSymBS) {
        const int j = jb0 + m;
        sp[m] = j < ns ? a.gpos64[s0 + j] : make_dbl4(1.0e150, 1.0e150, 1.0e150, 0.0);
        sag[m] = j < ns ? a.sph_agg[s0 + j] : -1;
    }
    dbl4 xi[kSymIB];
    int ai[kSymIB];
    double ax[kSymIB], ay[kSymIB], az[kSymIB];
    const int i0 = ta * kSymTile + w * (32 * kSymIB) + l;
#pragma unroll
    for (int k = 0; k < kSymIB; ++k) {
        const int i = i0 + 32 * k;
        const bool ok = i < ns;
        xi[k] = ok ? a.gpos64[s0 + i] : make_dbl4(0.0, 0.0, 0.0, 0.0);
        ai[k] = ok ? a.sph_agg[s0 + i] : -2;
        ax[k] = ay[k] = az[k] = 0.0;
    }
    const bool masked = diag || a.sph_agg[s0 + (int64_t)ta * kSymTile + kSymTile - 1] == a.sph_agg[s0 + jb0];
    __syncthreads();
    if (diag) {
        for (int jj = 0; jj < nj; ++jj) {
            const dbl4 pj = sp[jj];
            const int aj = sag[jj];
#pragma unroll
            for (int k = 0; k < kSymIB; ++k) {
                const double dx = pj.x - xi[k].x, dy = pj.y - xi[k].y, dz = pj.z - xi[k].z;
                const double r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
                const double inv = rsqrt(r2);
                double si = (pj.w * inv) * (inv * inv);
                si = aj == ai[k] ? 0.0 : si;
                ax[k] = fma(dx, si, ax[k]);
                ay[k] = fma(dy, si, ay[k]);
                az[k] = fma(dz, si, az[k]);
            }
        }
    } else {
        for (int c = 0; c * 32 < nj; ++c) {
            const dbl4 pj = sp[c * 32 + l];
            const int aj = sag[c * 32 + l];
            sj[w * kSymTile + c * 32 + l] = masked ? sym_ring64<true>(pj, aj, xi, ai, ax, ay, az, eps2)
                                                   : sym_ring64<false>(pj, aj, xi, ai, ax, ay, az, eps2);
        }
        __syncthreads();
        for (int m = threadIdx.x; m < nj; m += kSymBS) {
            const dbl4 u0 = sj[m], u1 = sj[kSymTile + m], u2 = sj[2 * kSymTile + m], u3 = sj[3 * kSymTile + m];
            ((dbl4 *)a.gpart)[sym_slot(a, p, ns, T + ta, jb0 + m)] =
                make_dbl4(((u0.x + u1.x) + u2.x) + u3.x, ((u0.y + u1.y) + u2.y) + u3.y,
                          ((u0.z + u1.z) + u2.z) + u3.z, 0.0);
        }
    }
#pragma unroll
    for (int k = 0; k < kSymIB; ++k) {
        const int i = i0 + 32 * k;
        if (i >= ns) continue;
        if (T == 1) {
            const double gm = S.G * a.m64[s0 + i];
            a.fg[s0 + i] = make_dbl4(gm * ax[k], gm * ay[k], gm * az[k], 0.0);
        } else {
            ((dbl4 *)a.gpart)[sym_slot(a, p, ns, tb, i)] = make_dbl4(ax[k], ay[k], az[k], 0.0);
        }
    }
}

constexpr size_t kSym64Smem = sizeof(dbl4) * kSymTile * 5 + sizeof(int) * kSymTile;

__global__ void __launch_bounds__(kSymBS) k_gravity64s(Arrays a, Sizes z)
{
    pdl_enter();
    extern __shared__ __align__(32) unsigned char sm64[];
    dbl4 *sp = (dbl4 *)sm64;
    dbl4 *sj = sp + kSymTile;
    int *sag = (int *)(sj + 4 * kSymTile);
    __shared__ int next;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) next = grab_item(a.gcounter, z.GI);
        __syncthreads();
        const int item = next;
        if (item >= z.GI) return;
        gravity64s_item(a, a.gitems[item], sp, sag, sj);
    }
}

__global__ void k_grav_combine_sym64(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.N) return;
    int p = a.sph_pile[i];
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const int T = a.gnchunk[p];
    if (T <= 1) return;
    const PileStatic &S = a.ps[p];
    const int64_t il = i - S.s0;
    const int t = (int)(il / kSymTile);
    const dbl4 *gp = (const dbl4 *)a.gpart;
    double sx = 0, sy = 0, sz = 0;
    for (int b = t; b < T; ++b) {
        const dbl4 v = gp[sym_slot(a, p, S.ns, b, il)];
        sx += v.x; sy += v.y; sz += v.z;
    }
    for (int r = 0; r < t; ++r) {
        const dbl4 v = gp[sym_slot(a, p, S.ns, T + r, il)];
        sx += v.x; sy += v.y; sz += v.z;
    }
    const double gm = S.G * a.m64[i];
    a.fg[i] = make_dbl4(gm * sx, gm * sy, gm * sz, 0.0);
}

// Sum the j-range partials of piles that were split, in range order.
template <bool FP64>
__global__ void k_grav_combine(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.N) return;
    int p = a.sph_pile[i];
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    int nch = a.gnchunk[p];
    if (nch <= 1) return;
    const PileStatic &S = a.ps[p];
    int64_t il = i - S.s0;
    double sx = 0, sy = 0, sz = 0;
    for (int c = 0; c < nch; ++c) {
        const int64_t slot = a.gpart_base[p] + (int64_t)c * S.ns + il;
        if (FP64) {
            const dbl4 v = ((const dbl4 *)a.gpart)[slot];
            sx += v.x; sy += v.y; sz += v.z;
        } else {
            const float4 v = ((const float4 *)a.gpart)[slot];
            sx += v.x; sy += v.y; sz += v.z;
        }
    }
    double gm = S.G * a.m64[i];
    a.fg[i] = make_dbl4(gm * sx, gm * sy, gm * sz, 0.0);
}

template <int BS, int IB>
static void launch_g(const Arrays &a, const Sizes &z, bool fp64, bool pack, cudaStream_t st)
{
    if (fp64) {
        launch_pdl(k_gravity64<BS, IB>, (unsigned)z.GI, BS, 0, st, a, z);
    } else {
        int64_t nb = z.GB > 0 && z.GB < z.GI ? z.GB : z.GI;
        if constexpr (IB % 2 == 0) {
            if (pack) {
                launch_pdl(k_gravity32p<BS, IB / 2>, (unsigned)nb, BS, 0, st, a, z);
                return;
            }
        }
        launch_pdl(k_gravity32<BS, IB>, (unsigned)nb, BS, 0, st, a, z);
    }
}

template <int BS, int IB>
static int occ(bool fp64, bool pack)
{
    int n = 0;
    if (fp64) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity64<BS, IB>, BS, 0);
    } else {
        if constexpr (IB % 2 == 0) {
            if (pack) {
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity32p<BS, IB / 2>, BS, 0);
                return n;
            }
        }
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity32<BS, IB>, BS, 0);
    }
    return n;
}

int gravity_blocks_per_sm(bool fp64, int block, int ib, bool pack, bool sym, int tile)
{
    if (sym) {
        int n = 0;
        if (fp64) {
            cudaFuncSetAttribute(k_gravity64s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSym64Smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity64s, kSymBS, kSym64Smem);
        } else {
            if (tile == 64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity32s<1, 2>, 32, 0);
            else if (tile == 128) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity32s<1, 4>, 32, 0);
            else if (tile == 256) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity32s<2, 4>, 64, 0);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gravity32s<kBigWPB, kBigIB>, 32 * kBigWPB, 0);
        }
        return n;
    }
    if (block == 64) return ib == 1 ? occ<64, 1>(fp64, pack) : ib == 2 ? occ<64, 2>(fp64, pack) : occ<64, 4>(fp64, pack);
    if (block == 128) return ib == 1 ? occ<128, 1>(fp64, pack) : ib == 2 ? occ<128, 2>(fp64, pack) : occ<128, 4>(fp64, pack);
    return ib == 1 ? occ<256, 1>(fp64, pack) : ib == 2 ? occ<256, 2>(fp64, pack) : occ<256, 4>(fp64, pack);
}

// Mixed symmetric form: turn the integer sums of piles with more than one
// tile into F_i = G m_i sum 2^-k and clear the accumulators for the next step
// (one thread per sphere: the accumulators are read once, coalesced, with
// every sphere in flight; done inside the per-aggregate pass instead, one
// thread walking an aggregate's members, it was 4x slower on 256 small piles).
__global__ void k_grav_acc_to_force(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.N) return;
    int p = a.sph_pile[i];
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    if (a.gnchunk[p] <= 1) return;
    const PileStatic &S = a.ps[p];
    longlong2 *g = (longlong2 *)(a.gacc + 4 * i);
    const longlong2 xy = g[0], zw = g[1];
    g[0] = make_longlong2(0, 0);
    g[1] = make_longlong2(0, 0);
    const double gm = S.G * a.m64[i] * S.ginv;
    a.fg[i] = make_dbl4(gm * (double)xy.x, gm * (double)xy.y, gm * (double)zw.x, 0.0);
}

void launch_gravity(const Arrays &a, const Sizes &z, bool fp64, int block, int ib, bool pack,
                    bool sym, cudaStream_t st)
{
    if (z.GI == 0) return;
    if (sym) {
        int64_t nb = z.GB > 0 && z.GB < z.GI ? z.GB : z.GI;
        if (fp64) {
            launch_pdl(k_gravity64s, (unsigned)nb, kSymBS, kSym64Smem, st, a, z);
            if (z.GP > 0) launch_pdl(k_grav_combine_sym64, (unsigned)((z.N + 255) / 256), 256, 0, st, a, z);
        } else {
            if (z.gtile == 64) launch_pdl(k_gravity32s<1, 2>, (unsigned)nb, 32, 0, st, a, z);
            else if (z.gtile == 128) launch_pdl(k_gravity32s<1, 4>, (unsigned)nb, 32, 0, st, a, z);
            else if (z.gtile == 256) launch_pdl(k_gravity32s<2, 4>, (unsigned)nb, 64, 0, st, a, z);
            else launch_pdl(k_gravity32s<kBigWPB, kBigIB>, (unsigned)nb, 32 * kBigWPB, 0, st, a, z);
            if (z.gacc_on) launch_pdl(k_grav_acc_to_force, (unsigned)((z.N + 255) / 256), 256, 0, st, a, z);
        }
        return;
    }
    if (block == 64 && ib == 1) launch_g<64, 1>(a, z, fp64, pack, st);
    else if (block == 64 && ib == 2) launch_g<64, 2>(a, z, fp64, pack, st);
    else if (block == 64 && ib == 4) launch_g<64, 4>(a, z, fp64, pack, st);
    else if (block == 128 && ib == 1) launch_g<128, 1>(a, z, fp64, pack, st);
    else if (block == 128 && ib == 2) launch_g<128, 2>(a, z, fp64, pack, st);
    else if (block == 128 && ib == 4) launch_g<128, 4>(a, z, fp64, pack, st);
    else if (block == 256 && ib == 1) launch_g<256, 1>(a, z, fp64, pack, st);
    else if (block == 256 && ib == 2) launch_g<256, 2>(a, z, fp64, pack, st);
    else launch_g<256, 4>(a, z, fp64, pack, st);
    if (z.GP > 0) {
        if (fp64) launch_pdl(k_grav_combine<true>, (unsigned)((z.N + 255) / 256), 256, 0, st, a, z);
        else launch_pdl(k_grav_combine<false>, (unsigned)((z.N + 255) / 256), 256, 0, st, a, z);
    }
}

}  // namespace dem
