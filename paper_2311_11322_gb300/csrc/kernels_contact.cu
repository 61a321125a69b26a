// kernels_contact.cu -- the contact pass: one thread per sphere in cell
// order, 27 neighbour cells of a wrapped uniform grid, pairs inside one
// aggregate skipped (Sec. 2.2: members are rigidly bonded), linear
// spring-dashpot normal force, tangential spring with history and Coulomb
// cap, rolling and twisting couples (Sec. 2.1, Sec. 2.2.5), applied at the
// contact point at the centre of the intersection circle (Sec. 2.2.4,
// Eq. lever_arm).
//
// Each pair is evaluated by both of its spheres, each taking itself as sphere
// a.  Every step of the law maps exactly onto its negative or onto itself when
// a and b swap (differences and products of negated operands round to the
// negated or the same result, TwoSum's error term is exact, and l_a, l_b are
// formed as |d|/2 +- (s_a^2 - s_b^2)/(2|d|)), so the two evaluations give
// bitwise opposite forces and couples and the tangential displacements S_b =
// -S_a each sphere keeps in its own history.  Nothing is written with atomics
// except error flags; each sphere sums its contacts in partner order, so the
// pass is deterministic.
//
// Two kernels.  k_contact_filter (one thread per sphere in sorted order, few
// registers, many resident warps) walks the 27 neighbour cells -- the three
// x-adjacent cells of each (dy, dz) row are consecutive in the sorted order, so
// they are read as 9 index ranges -- and writes the candidates that pass a
// bounding test (other aggregate, centres closer than the radii sum plus the
// skin plus the FP32 rounding margin) to a per-sphere hit list, ordered by the
// partner's pile-local index.  It runs only in steps that rebuild the cell
// list: in between, the lists stay complete as long as no sphere has moved
// more than half the skin (checked per aggregate at the drift).  k_contact
// evaluates the listed pairs every step; its lanes stay converged because
// every lane works through a short list of candidates.  A sphere whose list
// overflowed searches its cells again inside k_contact (its pile then
// rebuilds every step, so the cells are current).
// Every sphere sums its contacts in the order of the partners' indices, so
// forces, torques and history do not depend on the cell size, the skin or
// the steps at which the lists were rebuilt: the trajectory is bitwise the
// same for any of them.
// History slots are stored in sorted order (slot-major inside each pile) and
// read at the position the sphere had in the previous step; the previous
// partners' ids are staged in shared memory and matched with a cursor, since
// slots and hits are both in partner order.  Force and torque are written in
// sorted order, interleaved, so that the aggregate reduction gathers one
// 32-byte sector per sphere.
//
// Force law (the paper defers the constants and form to earlier work):
//   d = r_b - r_a, n = d/|d|, x = s_a + s_b - |d| > 0 (overlap),
//   l_a = (s_a^2 - s_b^2 + |d|^2) / (2|d|), l_b = |d| - l_a,
//   u = (v_b + w_b x (-l_b n)) - (v_a + w_a x (l_a n)), u_n = (u.n) n, u_t = u - u_n,
//   F_N = -kn x n + cn u_n,
//   S = (S_prev projected on the tangent plane, rescaled to |S_prev|) + u_t h,
//   F_T = kt S + ct u_t, capped at mu_s |F_N| (then S = (F_T - ct u_t)/kt),
//   M = -mu_r |F_N| R w_r / max(|w_r|, w0) - mu_t |F_N| R w_t / max(|w_t|, w0),
//     w = w_a - w_b, w_t = (w.n) n, w_r = w - w_t, R = s_a s_b / (s_a + s_b);
//   sphere a: F = F_N + F_T, tau = (l_a n) x F + M;
//   sphere b: -F,            tau = (l_b n) x F - M.
#include "dem_internal.h"
#include "devmath.cuh"
#include "launch.cuh"

namespace dem {

struct ParamsF {
    float kn, kt, cn, ct, mu_s, mu_r, mu_t, w0, h;
};
struct ParamsD {
    double kn, kt, cn, ct, mu_s, mu_r, mu_t, w0, h;
};

template <typename T, typename V>
struct PairOut {
    V F, M, S, n;
    T la, lb, x;
};

// Division and square root of the force law: fast hardware approximations in
// FP32 (relative error ~1e-7, far inside the FP32 path's tolerance; both
// spheres of a pair run the same instructions, so they still agree bitwise),
// IEEE in FP64.
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qsqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }

// Tangential spring, Coulomb cap and rolling/twisting couples, shared by
// both precisions (T = float or double).
template <typename T, typename V, typename P>
__device__ __forceinline__ void force_law(V n, T x, T la, T lb, V va, V wa, V vb, V wb, T sa,
                                          T sb, V Sprev, const P &prm, PairOut<T, V> &o)
{
    V ca = la * n, cb = (-lb) * n;
    V u = (vb + cross(wb, cb)) - (va + cross(wa, ca));
    T uns = dot(u, n);
    V un = uns * n;
    V ut = u - un;
    // F_N is along n: its signed magnitude is -kn x + cn (u.n)
    const T fn = prm.cn * uns - prm.kn * x;
    V FN = fn * n;
    T FNm = fabs(fn);
    T sn = dot(Sprev, n);
    V Sp = Sprev - sn * n;
    T Spm = qsqrt(dot(Sp, Sp)), Sprevm = qsqrt(dot(Sprev, Sprev));
    Sp = Spm > T(0) ? qdiv(Sprevm, Spm) * Sp : T(0) * Sp;
    V S = Sp + prm.h * ut;
    V FT = prm.kt * S + prm.ct * ut;
    T FTm = qsqrt(dot(FT, FT)), cap = prm.mu_s * FNm;
    if (FTm > cap) {
        FT = qdiv(cap, FTm) * FT;
        S = prm.kt > T(0) ? qdiv(T(1), prm.kt) * (FT - prm.ct * ut) : T(0) * S;
    }
    V w = wa - wb;
    T wn = dot(w, n);
    V wt = wn * n;
    V wr = w - wt;
    T Rred = qdiv(sa * sb, sa + sb);
    V M = T(0) * n;
    if (prm.mu_r > T(0)) {
        T wrm = qsqrt(dot(wr, wr));
        if (wrm > T(0)) M = M + qdiv(-prm.mu_r * FNm * Rred, fmax(wrm, prm.w0)) * wr;
    }
    if (prm.mu_t > T(0)) {
        T wtm = qsqrt(dot(wt, wt));
        if (wtm > T(0)) M = M + qdiv(-prm.mu_t * FNm * Rred, fmax(wtm, prm.w0)) * wt;
    }
    o.F = FN + FT;
    o.M = M;
    o.S = S;
    o.n = n;
    o.la = la;
    o.lb = lb;
    o.x = x;
}

// Mixed precision pair: the overlap x = s_a + s_b - |d| is formed from
// float-float positions and radii (exact differences by TwoSum, |d|^2 with
// TwoProduct terms, one Newton correction of the hardware square root), so x
// keeps ~24 significant bits even when x << |d|; the rest of the law is FP32.
__device__ __forceinline__ bool pair_mixed(float4 ah, float4 al, float4 av, float4 aw, float4 bh,
                                           float4 bl, float4 bv, float4 bw, float3 Sprev,
                                           const ParamsF &prm, PairOut<float, float3> &o)
{
    float sx, ex, sy, ey, sz, ez;
    two_sum(bh.x, -ah.x, sx, ex);
    two_sum(bh.y, -ah.y, sy, ey);
    two_sum(bh.z, -ah.z, sz, ez);
    ex = __fadd_rn(ex, __fsub_rn(bl.x, al.x));
    ey = __fadd_rn(ey, __fsub_rn(bl.y, al.y));
    ez = __fadd_rn(ez, __fsub_rn(bl.z, al.z));
    float dhx, dlx, dhy, dly, dhz, dlz;
    fast_two_sum(sx, ex, dhx, dlx);
    fast_two_sum(sy, ey, dhy, dly);
    fast_two_sum(sz, ez, dhz, dlz);
    float px, epx, py, epy, pz, epz;
    two_prod(dhx, dhx, px, epx);
    two_prod(dhy, dhy, py, epy);
    two_prod(dhz, dhz, pz, epz);
    float s1, t1, Dh, t2;
    two_sum(px, py, s1, t1);
    two_sum(s1, pz, Dh, t2);
    float cr = __fmul_rn(dhx, dlx);
    cr = __fmaf_rn(dhy, dly, cr);
    cr = __fmaf_rn(dhz, dlz, cr);
    float Dl = __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(__fadd_rn(epx, epy), epz));
    Dl = __fmaf_rn(2.0f, cr, Dl);
    // |d| = r + delta: r from the hardware reciprocal square root (a few ulp),
    // delta its Newton correction from the exact remainder Dh - r^2 (one FMA)
    // and the low part Dl, so the overlap below keeps ~24 bits of its own.
    if (!(Dh > 0.0f)) return false;
    const float inv = rsqrtf(Dh);
    const float r = __fmul_rn(Dh, inv);
    float delta = __fmul_rn(__fadd_rn(__fmaf_rn(-r, r, Dh), Dl), __fmul_rn(0.5f, inv));
    float Sh, e;
    two_sum(ah.w, bh.w, Sh, e);
    float Sl = __fadd_rn(e, __fadd_rn(al.w, bl.w));
    float x = __fadd_rn(__fsub_rn(Sh, r), __fsub_rn(Sl, delta));
    if (!(x > 0.0f)) return false;
    float dist = __fadd_rn(r, delta);
    float3 n = f3(__fmul_rn(dhx, inv), __fmul_rn(dhy, inv), __fmul_rn(dhz, inv));
    float sa = ah.w, sb = bh.w;
    // l_a, l_b = |d|/2 +- (s_a^2 - s_b^2)/(2|d|): swapping a and b swaps them exactly
    const float hd = __fmul_rn(0.5f, dist);
    const float g = __fmul_rn(__fmul_rn(__fsub_rn(sa, sb), __fadd_rn(sa, sb)), __fmul_rn(0.5f, inv));
    float la = __fadd_rn(hd, g);
    float lb = __fsub_rn(hd, g);
    force_law<float, float3, ParamsF>(n, x, la, lb, f3(av.x, av.y, av.z), f3(aw.x, aw.y, aw.z),
                                      f3(bv.x, bv.y, bv.z), f3(bw.x, bw.y, bw.z), sa, sb, Sprev,
                                      prm, o);
    return true;
}

__device__ __forceinline__ bool pair_64(dbl4 ap, dbl4 av, dbl4 aw, dbl4 bp, dbl4 bv, dbl4 bw,
                                        double3 Sprev, const ParamsD &prm,
                                        PairOut<double, double3> &o)
{
    double3 d = d3(bp.x - ap.x, bp.y - ap.y, bp.z - ap.z);
    double dist = sqrt(dot(d, d));
    double x = ap.w + bp.w - dist;
    if (!(x > 0.0) || !(dist > 0.0)) return false;
    const double inv = 1.0 / dist;
    double3 n = inv * d;
    const double hd = __dmul_rn(0.5, dist);
    const double g = __dmul_rn(__dmul_rn(__dsub_rn(ap.w, bp.w), __dadd_rn(ap.w, bp.w)), __dmul_rn(0.5, inv));
    double la = __dadd_rn(hd, g);
    double lb = __dsub_rn(hd, g);
    force_law<double, double3, ParamsD>(n, x, la, lb, d3(av.x, av.y, av.z), d3(aw.x, aw.y, aw.z),
                                        d3(bv.x, bv.y, bv.z), d3(bw.x, bw.y, bw.z), ap.w, bp.w,
                                        Sprev, prm, o);
    return true;
}

__device__ __forceinline__ int wrapc(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

__device__ __forceinline__ int cellc_f(float x, float inv_cell, int n)
{
    float f = floorf(__fmul_rn(x, inv_cell));
    f = fminf(fmaxf(f, -1.0e9f), 1.0e9f);
    int m = ((int)f) % n;
    return m < 0 ? m + n : m;
}

__device__ __forceinline__ int cellc_d(double x, double inv_cell, int n)
{
    double f = floor(__dmul_rn(x, inv_cell));
    f = fmin(fmax(f, -1.0e9), 1.0e9);
    int m = ((int)f) % n;
    return m < 0 ? m + n : m;
}

// The (up to 3) sorted index ranges of the x-neighbour cells cx-1..cx+1 of
// one (y, z) row: one range when no wrap-around splits them.
struct Strip {
    int beg[3], end[3], n;
};

__device__ __forceinline__ void strip_ranges(const int32_t *cstart, const int32_t *ccount,
                                             int rowbase, int cx, int nx, Strip &s)
{
    if (cx >= 1 && cx + 1 < nx) {
        int c0 = rowbase + cx - 1, c2 = rowbase + cx + 1;
        s.beg[0] = cstart[c0];
        s.end[0] = cstart[c2] + ccount[c2];
        s.n = 1;
    } else {
        s.n = 0;
        for (int dx = -1; dx <= 1; ++dx) {
            int c = rowbase + wrapc(cx + dx, nx);
            s.beg[s.n] = cstart[c];
            s.end[s.n] = cstart[c] + ccount[c];
            ++s.n;
        }
    }
}

constexpr int kContactBlock = 128;


// launch bounds of the pair kernel (optionally with a minimum number of
// resident blocks per SM, which caps its registers)
// partner data of the next hit loaded one hit ahead (1), plus the S of the
// slot the next hit most likely matches (2)
#ifndef DEM_CONTACT_PREFETCH
#define DEM_CONTACT_PREFETCH 0
#endif
#ifdef DEM_CONTACT_MINB
#define DEM_CONTACT_BOUNDS __launch_bounds__(kContactBlock, DEM_CONTACT_MINB)
#else
#define DEM_CONTACT_BOUNDS __launch_bounds__(kContactBlock)
#endif


template <bool FP64> struct CT;
template <> struct CT<false> {
    typedef float T;
    typedef float3 V;
    typedef float4 P4;
    typedef ParamsF Prm;
};
template <> struct CT<true> {
    typedef double T;
    typedef double3 V;
    typedef dbl4 P4;
    typedef ParamsD Prm;
};

// Per-sphere state of the thread's own sphere and its running sums.
template <bool FP64>
struct Me {
    typename CT<FP64>::P4 p, v, w;   // position(+radius hi), velocity(+agg), spin(+gid)
    float4 l;                        // mixed: position lo (+radius lo)
    int agg, hl, nprev, nn, cursor, flags;
    float tol;                       // mixed: pre-filter margin
    typename CT<FP64>::T skin;       // filter: neighbour-list skin (0 in k_contact)
    typename CT<FP64>::V F, T;
};

// Candidate filter: overlap possible (bounding test with the FP32 rounding
// margin in mixed precision), not the sphere itself, other aggregate.
template <bool FP64>
__device__ __forceinline__ bool candidate(int64_t k, int64_t kk, const typename CT<FP64>::P4 &nh,
                                          int nagg, const Me<FP64> &m)
{
    if constexpr (FP64) {
        const double ddx = nh.x - m.p.x, ddy = nh.y - m.p.y, ddz = nh.z - m.p.z;
        const double sr2 = nh.w + m.p.w + m.skin;
        return ddx * ddx + ddy * ddy + ddz * ddz < sr2 * sr2 && kk != k && nagg != m.agg;
    } else {
        const float ddx = nh.x - m.p.x, ddy = nh.y - m.p.y, ddz = nh.z - m.p.z;
        const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        const float srt = nh.w + m.p.w + m.tol + m.skin;
        return r2 <= srt * srt && kk != k && nagg != m.agg;
    }
}

// Partner data of one candidate (sorted SoA entries).
template <bool FP64>
struct Nb {
    typename CT<FP64>::P4 h, v, w;   // position (+radius), velocity (+agg), spin (+index)
    float4 l;                        // mixed: position lo (+radius lo)
};

template <bool FP64>
__device__ __forceinline__ void load_nb(const Arrays &a, int64_t kk, Nb<FP64> &nb)
{
    if constexpr (FP64) {
        nb.h = a.dp_[kk];
        nb.v = a.dv_[kk];
        nb.w = a.dw_[kk];
    } else {
        nb.h = a.sph_[kk];
        nb.l = a.spl_[kk];
        nb.v = a.sv_[kk];
        nb.w = a.sw_[kk];
    }
}

// One candidate that passed the filter: history lookup, canonical pair
// evaluation, accumulation and slot write.  `spec`/`Sspec`: the previous slot
// guessed for this partner and its S, loaded ahead (spec < 0: none).
template <bool FP64>
__device__ __forceinline__ void process(const Arrays &a, const Nb<FP64> &nb, Me<FP64> &m,
                                        const int *myprev, const void *hprev_v, void *hnew_v, int ns,
                                        int K, const typename CT<FP64>::Prm &prm, int spec,
                                        const typename CT<FP64>::V &Sspec)
{
    typedef typename CT<FP64>::V V;
    const typename CT<FP64>::P4 &nh = nb.h, &nv = nb.v, &nw = nb.w;
    int ngid;
    if constexpr (FP64) ngid = (int)nw.w;
    else ngid = __float_as_int(nw.w);
    int slot = -1;
    if (m.cursor < m.nprev && myprev[m.cursor * kContactBlock] == ngid) slot = m.cursor;
    else
        for (int h = 0; h < m.nprev; ++h)
            if (myprev[h * kContactBlock] == ngid) { slot = h; break; }
    V Sprev;
    if constexpr (FP64) Sprev = d3(0, 0, 0);
    else Sprev = f3(0, 0, 0);
    if (slot >= 0) {
        if (slot == spec) {
            Sprev = Sspec;
        } else if constexpr (FP64) {
            const dbl4 sl = ((const dbl4 *)hprev_v)[(int64_t)slot * ns];
            Sprev = d3(sl.x, sl.y, sl.z);
        } else {
            const float4 sl = ((const float4 *)hprev_v)[(int64_t)slot * ns];
            Sprev = f3(sl.x, sl.y, sl.z);
        }
        m.cursor = slot + 1;
    }
    // this sphere is sphere a of the law
    PairOut<typename CT<FP64>::T, V> o;
    bool hit;
    if constexpr (FP64) hit = pair_64(m.p, m.v, m.w, nh, nv, nw, Sprev, prm, o);
    else hit = pair_mixed(m.p, m.l, m.v, m.w, nh, nb.l, nv, nw, Sprev, prm, o);
    if (!hit) return;
    // sphere a: F, (l_a n) x F + M
    m.F = m.F + o.F;
    m.T = m.T + cross(o.la * o.n, o.F) + o.M;
    if (m.nn < K) {
        if constexpr (FP64)
            ((dbl4 *)hnew_v)[(int64_t)m.nn * ns] = make_dbl4(o.S.x, o.S.y, o.S.z, (double)ngid);
        else
            ((float4 *)hnew_v)[(int64_t)m.nn * ns] = make_float4(o.S.x, o.S.y, o.S.z, __int_as_float(ngid));
    } else {
        m.flags |= DEM_FLAG_SLOTS;
    }
    ++m.nn;
    if (o.x > typename CT<FP64>::T(0.1) * fmin(m.p.w, nh.w)) m.flags |= DEM_FLAG_OVERLAP;
}

// Pile, sorted-position and cell set-up shared by both kernels.
template <bool FP64>
__device__ __forceinline__ void own_cell(const PileStatic &S, const typename CT<FP64>::P4 &p, int &cx,
                                         int &cy, int &cz)
{
    if constexpr (FP64) {
        cx = cellc_d(p.x, S.inv_cell, S.nx);
        cy = cellc_d(p.y, S.inv_cell, S.ny);
        cz = cellc_d(p.z, S.inv_cell, S.nz);
    } else {
        const float icell = (float)S.inv_cell;
        cx = cellc_f(p.x, icell, S.nx);
        cy = cellc_f(p.y, icell, S.ny);
        cz = cellc_f(p.z, icell, S.nz);
    }
}

// Rounding of the hi position parts is at most ulp(|p|)/2 per coordinate and
// every neighbour lies within 2 cells, so one margin serves all candidates.
__device__ __forceinline__ float filter_tol(const PileStatic &S, float4 p)
{
    const float my_abs = fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z)));
    return 4.0e-7f * (2.0f * my_abs + 3.0f * (float)S.cell) + 4.0e-6f * p.w;
}

template <bool FP64>
__global__ void __launch_bounds__(kContactBlock) k_contact_filter(Arrays a, Sizes z)
{
    pdl_enter();
    typedef typename CT<FP64>::P4 P4;
    // per thread: the hits found so far, (partner index << 32 | sorted
    // position), kept in increasing order by insertion
    __shared__ unsigned long long s_list[kHitCap][kContactBlock];
    const int64_t k = (int64_t)blockIdx.x * kContactBlock + threadIdx.x;
    if (k >= z.N) return;
    const int p = a.sph_pile[k];
    if (a.enabled[p] == 0 || a.pd[p].failed || !a.pd[p].rebuild) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const int kl = (int)(k - s0);
    Me<FP64> m;
    if constexpr (FP64) {
        m.p = a.dp_[k];
        m.tol = 0.f;
        m.skin = S.skin;
    } else {
        m.p = a.sph_[k];
        m.tol = filter_tol(S, m.p);
        m.skin = (float)S.skin;
    }
    m.agg = a.sagg[k];
    int cx, cy, cz;
    own_cell<FP64>(S, m.p, cx, cy, cz);
    const int32_t *cstart = a.cstart + S.c0, *ccount = a.ccount + S.c0;
    const int32_t *srt = a.sorted + s0;
    unsigned long long *list = &s_list[0][threadIdx.x];
    int n = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
            Strip sr;
            strip_ranges(cstart, ccount, (wrapc(cz + dz, nz) * ny + wrapc(cy + dy, ny)) * nx, cx, nx, sr);
            for (int r = 0; r < sr.n; ++r) {
#pragma unroll 4
                for (int t = sr.beg[r]; t < sr.end[r]; ++t) {
                    const int64_t kk = s0 + t;
                    P4 nh;
                    if constexpr (FP64) nh = a.dp_[kk];
                    else nh = a.sph_[kk];
                    if (candidate<FP64>(k, kk, nh, a.sagg[kk], m)) {
                        if (n < kHitCap) {
                            const unsigned long long e =
                                ((unsigned long long)(unsigned)srt[t] << 32) | (unsigned)t;
                            int j = n;
                            while (j > 0 && list[(j - 1) * kContactBlock] > e) {
                                list[j * kContactBlock] = list[(j - 1) * kContactBlock];
                                --j;
                            }
                            list[j * kContactBlock] = e;
                        }
                        ++n;
                    }
                }
            }
        }
    int32_t *hl = a.hits + s0 * kHitCap + kl;
    const int nw = n < kHitCap ? n : kHitCap;
    for (int e = 0; e < nw; ++e) hl[(int64_t)e * ns] = (int32_t)(unsigned)list[e * kContactBlock];
    a.hitn[k] = n;
    if (n > kHitCap) atomicOr(&a.pd[p].hit_overflow, 1);
}

// A sphere whose hit list overflowed (its pile rebuilt the cells this step:
// an overflow forces a rebuild every step) searches its neighbour cells
// again: the candidate with the smallest partner index above `last`, or -1.
// Kept out of line, so that the rare path costs the pair kernel no registers.
template <bool FP64>
__device__ __noinline__ int64_t overflow_next(const Arrays &a, const PileStatic &S, int64_t k,
                                              typename CT<FP64>::P4 p, int agg, float tol, int last)
{
    typedef typename CT<FP64>::P4 P4;
    Me<FP64> m;
    m.p = p;
    m.agg = agg;
    m.tol = tol;
    m.skin = 0;
    const int64_t s0 = S.s0;
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    int cx, cy, cz;
    own_cell<FP64>(S, m.p, cx, cy, cz);
    const int32_t *cstart = a.cstart + S.c0, *ccount = a.ccount + S.c0;
    const int32_t *srt = a.sorted + s0;
    int best = 0x7fffffff;
    int64_t bk = -1;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
            Strip sr;
            strip_ranges(cstart, ccount, (wrapc(cz + dz, nz) * ny + wrapc(cy + dy, ny)) * nx, cx, nx, sr);
            for (int r = 0; r < sr.n; ++r)
                for (int t = sr.beg[r]; t < sr.end[r]; ++t) {
                    const int id = srt[t];
                    if (id <= last || id >= best) continue;
                    const int64_t kk = s0 + t;
                    P4 q;
                    if constexpr (FP64) q = a.dp_[kk];
                    else q = a.sph_[kk];
                    if (candidate<FP64>(k, kk, q, a.sagg[kk], m)) {
                        best = id;
                        bk = kk;
                    }
                }
        }
    return bk;
}

template <bool FP64>
__global__ void DEM_CONTACT_BOUNDS k_contact(Arrays a, Sizes z)
{
    pdl_enter();
    typedef typename CT<FP64>::P4 P4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = z.K;
    // shared memory: [hit list, kHitCap x block] [partner ids of the previous
    // slots, K x block]
    int *s_hit = (int *)smem_raw;
    int *s_prev = s_hit + kHitCap * kContactBlock;
    const int64_t k = (int64_t)blockIdx.x * kContactBlock + threadIdx.x;
    if (k >= z.N) return;
    const int p = a.sph_pile[k];
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int par = a.pd[p].parity;
    const int kl = (int)(k - s0);
    Me<FP64> m;
    // own sorted state first (independent loads); the home index is in the
    // spin record's fourth word
    if constexpr (FP64) {
        m.p = a.dp_[k];
        m.v = a.dv_[k];
        m.w = a.dw_[k];
        m.hl = (int)m.w.w;
    } else {
        m.p = a.sph_[k];
        m.l = a.spl_[k];
        m.v = a.sv_[k];
        m.w = a.sw_[k];
        m.hl = __float_as_int(m.w.w);
    }
    const int nh = a.hitn[k];
    // the previous step's sorted position: unchanged unless this step re-sorted
    const int prevk = a.pd[p].rebuild ? a.pos_of_home[par][s0 + m.hl] : kl;
    m.nprev = a.hist_n[par][s0 + prevk];
    m.nn = 0;
    m.cursor = 0;
    m.flags = 0;
    int *myprev = s_prev + threadIdx.x;
    const void *hprev;
    void *hnew;
    typename CT<FP64>::Prm prm;
    if constexpr (FP64) {
        prm = {S.kn, S.kt, S.cn, S.ct, S.mu_s, S.mu_r, S.mu_t, S.w0, S.h};
        const dbl4 *hp = a.hist64[par] + s0 * K + prevk;
        for (int t = 0; t < m.nprev; ++t) myprev[t * kContactBlock] = (int)hp[(int64_t)t * ns].w;
        hprev = hp;
        hnew = a.hist64[par ^ 1] + s0 * K + kl;
        m.agg = (int)m.v.w;
        m.tol = 0.f;
        m.skin = 0.0;
        m.F = d3(0, 0, 0);
        m.T = d3(0, 0, 0);
    } else {
        prm = {(float)S.kn, (float)S.kt, (float)S.cn, (float)S.ct, (float)S.mu_s,
               (float)S.mu_r, (float)S.mu_t, (float)S.w0, (float)S.h};
        const float4 *hp = a.hist32[par] + s0 * K + prevk;
        for (int t = 0; t < m.nprev; ++t) myprev[t * kContactBlock] = __float_as_int(hp[(int64_t)t * ns].w);
        hprev = hp;
        hnew = a.hist32[par ^ 1] + s0 * K + kl;
        m.agg = __float_as_int(m.v.w);
        m.tol = filter_tol(S, m.p);
        m.skin = 0.f;
        m.F = f3(0, 0, 0);
        m.T = f3(0, 0, 0);
    }
    const bool listed = nh <= kHitCap;
    int *myhit = s_hit + threadIdx.x;
    if (listed) {   // all hit indices first (independent loads), then the pairs
        const int32_t *hl = a.hits + s0 * kHitCap + kl;
        for (int e = 0; e < nh; ++e) myhit[e * kContactBlock] = hl[(int64_t)e * ns];
    }
    typedef typename CT<FP64>::V V;
    V Snone;
    if constexpr (FP64) Snone = d3(0, 0, 0);
    else Snone = f3(0, 0, 0);
    if (listed) {
#if DEM_CONTACT_PREFETCH
        // partner data one hit ahead, and the S of the slot the next hit most
        // likely matches (hits and slots are both in partner order)
        Nb<FP64> cur, nxt;
        if (nh > 0) load_nb<FP64>(a, s0 + myhit[0], cur);
        for (int e = 0; e < nh; ++e) {
            if (e + 1 < nh) load_nb<FP64>(a, s0 + myhit[(e + 1) * kContactBlock], nxt);
            int spec = -1;
            V Sspec = Snone;
#if DEM_CONTACT_PREFETCH > 1
            if (m.cursor < m.nprev) {
                spec = m.cursor;
                if constexpr (FP64) {
                    const dbl4 sl = ((const dbl4 *)hprev)[(int64_t)spec * ns];
                    Sspec = d3(sl.x, sl.y, sl.z);
                } else {
                    const float4 sl = ((const float4 *)hprev)[(int64_t)spec * ns];
                    Sspec = f3(sl.x, sl.y, sl.z);
                }
            }
#endif
            process<FP64>(a, cur, m, myprev, hprev, hnew, ns, K, prm, spec, Sspec);
            cur = nxt;
        }
#else
        for (int e = 0; e < nh; ++e) {
            Nb<FP64> nb;
            load_nb<FP64>(a, s0 + myhit[e * kContactBlock], nb);
            process<FP64>(a, nb, m, myprev, hprev, hnew, ns, K, prm, -1, Snone);
        }
#endif
    } else {
        for (int last = -1;;) {
            const int64_t kk = overflow_next<FP64>(a, S, k, m.p, m.agg, m.tol, last);
            if (kk < 0) break;
            last = a.sorted[kk];
            Nb<FP64> nb;
            load_nb<FP64>(a, kk, nb);
            process<FP64>(a, nb, m, myprev, hprev, hnew, ns, K, prm, -1, Snone);
        }
    }
    if constexpr (FP64) {
        a.ftc64[2 * k] = make_dbl4(m.F.x, m.F.y, m.F.z, 0.0);
        a.ftc64[2 * k + 1] = make_dbl4(m.T.x, m.T.y, m.T.z, 0.0);
    } else {
        a.ftc32[2 * k] = make_float4(m.F.x, m.F.y, m.F.z, 0.f);
        a.ftc32[2 * k + 1] = make_float4(m.T.x, m.T.y, m.T.z, 0.f);
    }
    a.hist_n[par ^ 1][k] = m.nn < K ? m.nn : K;
    if (m.flags) atomicOr(&a.pd[p].flags, m.flags);
}

static size_t contact_smem(bool, int K)
{
    return sizeof(int) * (size_t)(K + kHitCap) * kContactBlock;
}

cudaError_t contact_setup(bool fp64, int K)
{
    int smem = (int)contact_smem(fp64, K);
    if (fp64) return cudaFuncSetAttribute(k_contact<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return cudaFuncSetAttribute(k_contact<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

void launch_contact(const Arrays &a, const Sizes &z, bool fp64, int K, cudaStream_t st)
{
    if (z.N == 0) return;
    unsigned nb = (unsigned)((z.N + kContactBlock - 1) / kContactBlock);
    size_t smem = contact_smem(fp64, K);
    if (fp64) {
        launch_pdl(k_contact_filter<true>, nb, kContactBlock, 0, st, a, z);
        launch_pdl(k_contact<true>, nb, kContactBlock, smem, st, a, z);
    } else {
        launch_pdl(k_contact_filter<false>, nb, kContactBlock, 0, st, a, z);
        launch_pdl(k_contact<false>, nb, kContactBlock, smem, st, a, z);
    }
}

}  // namespace dem
