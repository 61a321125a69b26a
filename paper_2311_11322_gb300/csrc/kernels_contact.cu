// kernels_contact.cu -- the contact pass: uniform cells of a wrapped grid,
// pairs inside one aggregate skipped (Sec. 2.2: members are rigidly bonded),
// linear spring-dashpot normal force, tangential spring with history and
// Coulomb cap, rolling and twisting couples (Sec. 2.1, Sec. 2.2.5), applied at
// the contact point at the centre of the intersection circle (Sec. 2.2.4,
// Eq. lever_arm).
//
// Candidate lists.  At a rebuild (a new cell sort) every sphere lists the
// spheres of other aggregates whose centres are closer than the radii sum
// plus the skin, in the order of their home indices, in compressed rows per
// sorted sphere (k_cand_count, k_cand_scan, k_cand_fill); k_cand_link then
// gives every entry the position of the same pair in the partner's list and
// marks the entries whose sphere owns the pair (the lower home index).  The
// lists stay complete until some aggregate may have moved half the skin
// (checked at the drift).  The candidate test is exact and symmetric, so
// both spheres of a pair always list each other.
//
// Shares of a pair.  Both spheres' shares come from one evaluation with the
// owner as sphere a:
//   a:  F,  tau_a = (l_a n) x F + M;   b:  -F,  tau_b = (l_b n) x F - M.
// The law is written with every operation's rounding pinned, and each of its
// steps maps exactly onto its negative or onto itself when the two spheres
// swap, so an evaluation with b as sphere a gives b's share bit for bit.
// Two forms of the pass, with bitwise the same results:
//   k_contact_sphere (the default): one thread per sorted sphere evaluates
//     every entry of its list with itself as sphere a (each pair twice, once
//     per sphere) and sums its shares in list order; the owner's thread
//     writes the history;
//   k_contact (contact_mode 1): tiles of kCTile consecutive sorted spheres,
//     which fill compact blocks of space (cells are numbered brick by brick);
//     a pair inside a tile is evaluated once, by the thread that drew it from
//     the tile's work queue, and both shares go to the spheres' slots in a
//     shared-memory inbox; a pair that crosses tiles is evaluated by both
//     tiles, each keeping its own sphere's share.
// Every sphere sums its shares in list order, i.e. in the order of its
// partners' home indices, so forces, torques and history are bitwise the same
// whatever the form, the tiles, the cell size, the skin or the steps at which
// the lists were rebuilt.  Nothing is written with atomics except error flags.
//
// History (Sec. 2.1: the tangential displacement is tracked while the two
// spheres stay in contact) lives at the owner's list entry, from the owner's
// side, with .w = 1 while in contact; the evaluation reads the owner's entry
// and the owner's tile writes it.  A rebuild carries it over to the new lists
// by partner index.
//
// Mixed precision positions.  The overlap x = s_a + s_b - |d| of two nearby
// spheres needs more than FP32's 24 bits of |d|.  Each sphere's position
// relative to the pile frame is held as the low 32 bits of round(r / q) per
// axis, q = 2^qexp with 2^31 q >= 10.5 x the largest radius (so that a
// candidate pair's difference fits in int32 after any allowed motion), its
// radius as round(s / q), and the four rounding remainders in FP32.  The
// integer difference is exact and the large cancellation in
// (s_a + s_b)^2 - |d|^2 happens exactly in int64; the remainders add small
// FP32 corrections, so x = ((s_a + s_b)^2 - |d|^2) / (s_a + s_b + |d|) keeps
// FP32 relative accuracy; the rest of the law is FP32.
//
// Force law (the paper defers the constants and form to earlier work):
//   d = r_b - r_a, n = d/|d|, x = s_a + s_b - |d| > 0 (overlap),
//   l_a = (s_a^2 - s_b^2 + |d|^2) / (2|d|), l_b = |d| - l_a,
//   u = (v_b + w_b x (-l_b n)) - (v_a + w_a x (l_a n)), u_n = (u.n) n, u_t = u - u_n,
//   F_N = -kn x n + cn u_n,
//   S = (S_prev projected on the tangent plane, rescaled to |S_prev|) + u_t h,
//   F_T = kt S + ct u_t, capped at mu_s |F_N| (then S = (F_T - ct u_t)/kt),
//   M = -mu_r |F_N| R w_r / max(|w_r|, w0) - mu_t |F_N| R w_t / max(|w_t|, w0),
//     w = w_a - w_b, w_t = (w.n) n, w_r = w - w_t, R = s_a s_b / (s_a + s_b).
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
    T la, lb, x, rmin;
};

// Division and square root of the force law: fast hardware approximations in
// FP32 (relative error ~1e-7, far inside the FP32 path's tolerance), IEEE in FP64.
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qsqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }

// Correctly rounded operations for the force law: every product, sum and
// fused multiply-add is written out, so the compiler neither contracts nor
// reassociates anything and the law gives the same bits in every kernel
// that inlines it (the pair kernels rely on that for bitwise results).
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T, typename V> __device__ __forceinline__ V vmk(T x, T y, T z);
template <> __device__ __forceinline__ float3 vmk<float, float3>(float x, float y, float z) { return f3(x, y, z); }
template <> __device__ __forceinline__ double3 vmk<double, double3>(double x, double y, double z) { return d3(x, y, z); }
template <typename T, typename V> __device__ __forceinline__ V vscale(T s, V a)
{ return vmk<T, V>(rmul(s, a.x), rmul(s, a.y), rmul(s, a.z)); }
template <typename T, typename V> __device__ __forceinline__ V vadd(V a, V b)
{ return vmk<T, V>(radd(a.x, b.x), radd(a.y, b.y), radd(a.z, b.z)); }
template <typename T, typename V> __device__ __forceinline__ V vsub(V a, V b)
{ return vmk<T, V>(rsub(a.x, b.x), rsub(a.y, b.y), rsub(a.z, b.z)); }
template <typename T, typename V> __device__ __forceinline__ V vaxpy(T s, V a, V b)   // s a + b
{ return vmk<T, V>(rfma(s, a.x, b.x), rfma(s, a.y, b.y), rfma(s, a.z, b.z)); }
template <typename T, typename V> __device__ __forceinline__ T vdot(V a, V b)
{ return rfma(a.z, b.z, rfma(a.y, b.y, rmul(a.x, b.x))); }
template <typename T, typename V> __device__ __forceinline__ V vcross(V a, V b)
{
    return vmk<T, V>(rfma(a.y, b.z, -rmul(a.z, b.y)), rfma(a.z, b.x, -rmul(a.x, b.z)),
                     rfma(a.x, b.y, -rmul(a.y, b.x)));
}
__device__ __forceinline__ float rdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rnorm(float x) { return x > 0.f ? rmul(x, rsqrtf(x)) : 0.f; }
__device__ __forceinline__ double rnorm(double x) { return __dsqrt_rn(x); }

// Tangential spring, Coulomb cap and rolling/twisting couples, shared by
// both precisions (T = float or double).
template <typename T, typename V, typename P>
__device__ __forceinline__ void force_law(V n, T x, T la, T lb, V va, V wa, V vb, V wb, T sa,
                                          T sb, V Sprev, const P &prm, PairOut<T, V> &o)
{
    // relative velocity of b's contact point with respect to a's
    const V ca = vscale<T, V>(la, n), cb = vscale<T, V>(-lb, n);
    const V u = vsub<T, V>(vadd<T, V>(vb, vcross<T, V>(wb, cb)), vadd<T, V>(va, vcross<T, V>(wa, ca)));
    const T uns = vdot<T, V>(u, n);
    const V ut = vaxpy<T, V>(-uns, n, u);                 // u - (u.n) n
    // F_N is along n: its signed magnitude is -kn x + cn (u.n)
    const T fn = rfma(prm.cn, uns, -rmul(prm.kn, x));
    const T FNm = fabs(fn);
    // tangential spring: S_prev on the new tangent plane, rescaled to |S_prev|
    V Sp = vaxpy<T, V>(-vdot<T, V>(Sprev, n), n, Sprev);
    const T Spm = rnorm(vdot<T, V>(Sp, Sp)), Sprevm = rnorm(vdot<T, V>(Sprev, Sprev));
    Sp = Spm > T(0) ? vscale<T, V>(rdiv(Sprevm, Spm), Sp) : vmk<T, V>(T(0), T(0), T(0));
    V S = vaxpy<T, V>(prm.h, ut, Sp);
    V FT = vaxpy<T, V>(prm.ct, ut, vscale<T, V>(prm.kt, S));
    const T FTm = rnorm(vdot<T, V>(FT, FT)), cap = rmul(prm.mu_s, FNm);
    if (FTm > cap) {
        FT = vscale<T, V>(rdiv(cap, FTm), FT);
        S = prm.kt > T(0) ? vscale<T, V>(rdiv(T(1), prm.kt), vaxpy<T, V>(-prm.ct, ut, FT))
                          : vmk<T, V>(T(0), T(0), T(0));
    }
    // rolling and twisting couples
    const V w = vsub<T, V>(wa, wb);
    const T wn = vdot<T, V>(w, n);
    const V wt = vscale<T, V>(wn, n);
    const V wr = vsub<T, V>(w, wt);
    const T Rred = rdiv(rmul(sa, sb), radd(sa, sb));
    V M = vmk<T, V>(T(0), T(0), T(0));
    if (prm.mu_r > T(0)) {
        const T wrm = rnorm(vdot<T, V>(wr, wr));
        if (wrm > T(0)) M = vscale<T, V>(rdiv(-rmul(rmul(prm.mu_r, FNm), Rred), fmax(wrm, prm.w0)), wr);
    }
    if (prm.mu_t > T(0)) {
        const T wtm = rnorm(vdot<T, V>(wt, wt));
        if (wtm > T(0)) M = vaxpy<T, V>(rdiv(-rmul(rmul(prm.mu_t, FNm), Rred), fmax(wtm, prm.w0)), wt, M);
    }
    o.F = vaxpy<T, V>(fn, n, FT);                         // F_N + F_T
    o.M = M;
    o.S = S;
    o.n = n;
    o.la = la;
    o.lb = lb;
    o.x = x;
}

// Mixed-precision pair from fixed-point positions (see the file comment).
// A, B: (x, y, z low 32 bits, radius) in quanta q; RA, RB: the remainders of
// those roundings (in quanta).  In quanta, with d = D_i + dd_i per axis (D_i
// the exact integer difference, |dd_i| <= 1) and s = S + rho (S the integer
// radii sum):
//   (s_a + s_b)^2 - |d|^2 = (S^2 - sum D_i^2) + 2 S rho + rho^2
//                           - 2 sum D_i dd_i - sum dd_i^2,
// the first bracket exact in int64 (the large cancellation), the small terms
// in FP32; x = that / (s + |d|).
__device__ __forceinline__ bool pair_mixed(int4 A, float4 RA, int4 B, float4 RB, float q, float4 av,
                                           float4 aw, float4 bv, float4 bw, float3 Sprev,
                                           const ParamsF &prm, PairOut<float, float3> &o)
{
    const int dx = (int)((unsigned)B.x - (unsigned)A.x);
    const int dy = (int)((unsigned)B.y - (unsigned)A.y);
    const int dz = (int)((unsigned)B.z - (unsigned)A.z);
    const long long D = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
    const int Ss = A.w + B.w;
    const long long num_i = (long long)Ss * Ss - D;
    const float ex = __fsub_rn(RB.x, RA.x), ey = __fsub_rn(RB.y, RA.y), ez = __fsub_rn(RB.z, RA.z);
    const float rho = __fadd_rn(RA.w, RB.w);
    const float fx = __int2float_rn(dx), fy = __int2float_rn(dy), fz = __int2float_rn(dz);
    const float Ssf = __int2float_rn(Ss);
    const float cr = __fmaf_rn(fz, ez, __fmaf_rn(fy, ey, __fmul_rn(fx, ex)));
    const float ee = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
    const float corr = __fsub_rn(__fsub_rn(__fmaf_rn(__fmul_rn(2.0f, Ssf), rho, __fmul_rn(rho, rho)),
                                           __fmul_rn(2.0f, cr)), ee);
    // the int64 bracket to FP32 from its 32-bit halves (two 32-bit conversions
    // and one FMA, off the FP64 unit that a 64-bit conversion would use;
    // within 2 ulp of the correctly rounded value and symmetric in a, b)
    const float numi = __fmaf_rn(__int2float_rn((int)(num_i >> 32)), 4294967296.0f,
                                 __uint2float_rn((unsigned)(num_i & 0xffffffffll)));
    const float num = __fadd_rn(numi, corr);
    if (!(num > 0.0f)) return false;
    const float3 d = f3(__fadd_rn(fx, ex), __fadd_rn(fy, ey), __fadd_rn(fz, ez));
    const float Df = __fmaf_rn(d.z, d.z, __fmaf_rn(d.y, d.y, __fmul_rn(d.x, d.x)));
    if (!(Df > 0.0f)) return false;
    const float inv = rsqrtf(Df);
    const float dist = __fmul_rn(Df, inv);
    const float3 n = f3(__fmul_rn(d.x, inv), __fmul_rn(d.y, inv), __fmul_rn(d.z, inv));
    const float sqa = __fadd_rn(__int2float_rn(A.w), RA.w), sqb = __fadd_rn(__int2float_rn(B.w), RB.w);
    const float ssum = __fadd_rn(sqa, sqb);
    const float x = __fmul_rn(__fdividef(num, __fadd_rn(ssum, dist)), q);
    // l_a, l_b = |d|/2 +- (s_a - s_b)(s_a + s_b)/(2|d|)
    const float hd = __fmul_rn(0.5f, dist);
    const float g = __fmul_rn(__fmul_rn(0.5f, __fsub_rn(sqa, sqb)), __fmul_rn(ssum, inv));
    const float la = __fmul_rn(__fadd_rn(hd, g), q);
    const float lb = __fmul_rn(__fsub_rn(hd, g), q);
    const float sa = __fmul_rn(sqa, q), sb = __fmul_rn(sqb, q);
    o.rmin = fminf(sa, sb);
    force_law<float, float3, ParamsF>(n, x, la, lb, f3(av.x, av.y, av.z), f3(aw.x, aw.y, aw.z),
                                      f3(bv.x, bv.y, bv.z), f3(bw.x, bw.y, bw.z), sa, sb, Sprev, prm, o);
    return true;
}

__device__ __forceinline__ bool pair_64(dbl4 ap, dbl4 av, dbl4 aw, dbl4 bp, dbl4 bv, dbl4 bw,
                                        double3 Sprev, const ParamsD &prm, PairOut<double, double3> &o)
{
    const double3 d = d3(__dsub_rn(bp.x, ap.x), __dsub_rn(bp.y, ap.y), __dsub_rn(bp.z, ap.z));
    const double dist = __dsqrt_rn(vdot<double, double3>(d, d));
    const double x = __dsub_rn(__dadd_rn(ap.w, bp.w), dist);
    if (!(x > 0.0) || !(dist > 0.0)) return false;
    const double inv = __ddiv_rn(1.0, dist);
    const double3 n = vscale<double, double3>(inv, d);
    const double hd = __dmul_rn(0.5, dist);
    const double g = __dmul_rn(__dmul_rn(__dsub_rn(ap.w, bp.w), __dadd_rn(ap.w, bp.w)), __dmul_rn(0.5, inv));
    double la = __dadd_rn(hd, g);
    double lb = __dsub_rn(hd, g);
    o.rmin = fmin(ap.w, bp.w);
    force_law<double, double3, ParamsD>(n, x, la, lb, d3(av.x, av.y, av.z), d3(aw.x, aw.y, aw.z),
                                        d3(bv.x, bv.y, bv.z), d3(bw.x, bw.y, bw.z), ap.w, bp.w, Sprev, prm, o);
    return true;
}

// The two spheres' shares of one evaluation, every operation pinned to its
// rounding (no contraction), so a share is the same bits wherever it is formed.
__device__ __forceinline__ float3 lever_x_force(float l, float3 n, float3 F)
{
    const float3 c = f3(__fmul_rn(l, n.x), __fmul_rn(l, n.y), __fmul_rn(l, n.z));
    return f3(__fmaf_rn(c.y, F.z, __fmul_rn(-c.z, F.y)), __fmaf_rn(c.z, F.x, __fmul_rn(-c.x, F.z)),
              __fmaf_rn(c.x, F.y, __fmul_rn(-c.y, F.x)));
}
__device__ __forceinline__ double3 lever_x_force(double l, double3 n, double3 F)
{
    const double3 c = d3(__dmul_rn(l, n.x), __dmul_rn(l, n.y), __dmul_rn(l, n.z));
    return d3(__fma_rn(c.y, F.z, __dmul_rn(-c.z, F.y)), __fma_rn(c.z, F.x, __dmul_rn(-c.x, F.z)),
              __fma_rn(c.x, F.y, __dmul_rn(-c.y, F.x)));
}
__device__ __forceinline__ float addr(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double addr(double a, double b) { return __dadd_rn(a, b); }

// One sphere's share of an evaluation: sphere a (side_a) gets F and
// (l_a n) x F + M, sphere b gets -F and (l_b n) x F - M.
template <typename T, typename V>
__device__ __forceinline__ void share(const PairOut<T, V> &o, bool side_a, V &F, V &Tq)
{
    const T sg = side_a ? T(1) : T(-1);
    const V c = lever_x_force(side_a ? o.la : o.lb, o.n, o.F);
    F = vmk<T, V>(sg * o.F.x, sg * o.F.y, sg * o.F.z);
    Tq = vmk<T, V>(addr(c.x, sg * o.M.x), addr(c.y, sg * o.M.y), addr(c.z, sg * o.M.z));
}

template <bool FP64> struct CT;
template <> struct CT<false> {
    typedef float T;
    typedef float3 V;
    typedef ParamsF Prm;
    typedef float4 H;                      // history record
    typedef int4 P;                        // position record
    typedef float4 VR;                     // velocity / spin record
    static constexpr int kCap = kInboxCap; // inbox entries per block
};
template <> struct CT<true> {
    typedef double T;
    typedef double3 V;
    typedef ParamsD Prm;
    typedef dbl4 H;
    typedef dbl4 P;
    typedef dbl4 VR;
    static constexpr int kCap = kInboxCap / 2;
};

__device__ __forceinline__ bool pile_live(const Arrays &a, int p)
{
    return a.enabled[p] != 0 && a.pd[p].failed == 0;
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

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ float4 as_f4(int4 v)
{
    return make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w));
}

// Candidate test of sphere k (own data) against sorted position kk.  Exact and
// symmetric: swapping the spheres gives the same answer.
struct CandMe {
    int4 xq;        // mixed
    float4 ph;      // mixed: position hi, radius hi
    dbl4 p;         // fp64
    int agg;
};

template <bool FP64>
__device__ __forceinline__ bool cand_test(const Arrays &a, const PileStatic &S, const CandMe &m, int64_t kk)
{
    if constexpr (FP64) {
        const dbl4 q = a.dp_[kk];
        const double dx = q.x - m.p.x, dy = q.y - m.p.y, dz = q.z - m.p.z;
        const double t = m.p.w + q.w + S.skin;
        return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx))) < __dmul_rn(t, t);
    } else {
        // FP32 test first (it rejects the spheres of other wraps of the grid,
        // whose 32-bit fixed-point difference would alias): the FP32 centres
        // are the rounded float-float positions, so a margin of a few units in
        // the last place of both keeps every candidate; the margin depends on
        // both spheres alike, so the test stays symmetric
        const float4 q = a.sph_[kk];
        const float dx = __fsub_rn(q.x, m.ph.x), dy = __fsub_rn(q.y, m.ph.y), dz = __fsub_rn(q.z, m.ph.z);
        const float big = __fadd_rn(fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z))),
                                    fmaxf(fabsf(m.ph.x), fmaxf(fabsf(m.ph.y), fabsf(m.ph.z))));
        const float sr = __fadd_rn(q.w, m.ph.w);
        const float tc = __fadd_rn(__fadd_rn(sr, (float)S.skin), __fmaf_rn(1e-6f, big, __fmul_rn(1e-5f, sr)));
        if (!(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < __fmul_rn(tc, tc))) return false;
        const int4 B = a.xqr[2 * kk];
        const int ex = (int)((unsigned)B.x - (unsigned)m.xq.x);
        const int ey = (int)((unsigned)B.y - (unsigned)m.xq.y);
        const int ez = (int)((unsigned)B.z - (unsigned)m.xq.z);
        const long long D = (long long)ex * ex + (long long)ey * ey + (long long)ez * ez;
        // two quanta more than the skin: the rounding remainders cannot hide a contact
        const long long t = (long long)m.xq.w + B.w + S.skin_q + 2;
        return D < t * t;
    }
}

// Visit every sphere of the 27 neighbour cells of sorted position k (the
// three x-neighbours of a (y, z) row as one index range when they are
// consecutive), calling f(kk) for the candidates.
template <bool FP64, typename Fn>
__device__ __forceinline__ void for_candidates(const Arrays &a, const PileStatic &S, int64_t k,
                                               const CandMe &m, Fn f)
{
    int cx, cy, cz;
    if constexpr (FP64) {
        cx = cellc_d(m.p.x, S.inv_cell, S.nx);
        cy = cellc_d(m.p.y, S.inv_cell, S.ny);
        cz = cellc_d(m.p.z, S.inv_cell, S.nz);
    } else {
        const float ic = (float)S.inv_cell;
        cx = cellc_f(m.ph.x, ic, S.nx);
        cy = cellc_f(m.ph.y, ic, S.ny);
        cz = cellc_f(m.ph.z, ic, S.nz);
    }
    const int32_t *cstart = a.cstart + S.c0, *ccount = a.ccount + S.c0;
    const int64_t s0 = S.s0;
    // without wrap-around the three x-neighbours are consecutive cell ids
    // except across a brick boundary: one or two index ranges
    const bool nowrap = cx >= 1 && cx + 1 < S.nx;
    const int split = (cx & 3) == 0 ? 1 : (cx & 3) == 3 ? 2 : 3;   // first cell of the second range
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrapc(cy + dy, S.ny), zz = wrapc(cz + dz, S.nz);
            int beg[3], end[3], nr;
            if (nowrap) {
                const int64_t cl = cell_id(cx - 1, yy, zz, S.nx, S.ny);
                const int64_t cs = cell_id(cx - 1 + split, yy, zz, S.nx, S.ny);
                const int64_t ce = cell_id(cx + 1, yy, zz, S.nx, S.ny);
                if (split == 3) {
                    beg[0] = cstart[cl];
                    end[0] = cstart[ce] + ccount[ce];
                    nr = 1;
                } else {
                    const int64_t cm = split == 1 ? cl : cell_id(cx, yy, zz, S.nx, S.ny);
                    beg[0] = cstart[cl];
                    end[0] = cstart[cm] + ccount[cm];
                    beg[1] = cstart[cs];
                    end[1] = cstart[ce] + ccount[ce];
                    nr = 2;
                }
            } else {
                nr = 0;
                for (int ddx = -1; ddx <= 1; ++ddx) {
                    const int64_t c = cell_id(wrapc(cx + ddx, S.nx), yy, zz, S.nx, S.ny);
                    beg[nr] = cstart[c];
                    end[nr] = cstart[c] + ccount[c];
                    ++nr;
                }
            }
            for (int r = 0; r < nr; ++r)
                for (int t = beg[r]; t < end[r]; ++t) {
                    const int64_t kk = s0 + t;
                    if (kk == k || a.sagg[kk] == m.agg) continue;
                    if (cand_test<FP64>(a, S, m, kk)) f(t);
                }
        }
}

template <bool FP64>
__device__ __forceinline__ void load_me(const Arrays &a, int64_t k, CandMe &m)
{
    if constexpr (FP64) m.p = a.dp_[k];
    else {
        m.xq = a.xqr[2 * k];
        m.ph = a.sph_[k];
    }
    m.agg = a.sagg[k];
}

// ---------------------------------------------------------------- rebuild
__device__ __forceinline__ bool tile_rebuilds(const Arrays &a, int4 tl)
{
    return pile_live(a, tl.x) && a.pd[tl.x].rebuild;
}

// Whether any pile rebuilds this step (the block's threads read the piles'
// flags together): in most steps no pile does, and the rebuild kernels end here.
__device__ __forceinline__ bool any_rebuild(const Arrays &a, const Sizes &z)
{
    int mine = 0;
    for (int p = threadIdx.x; p < z.P; p += blockDim.x) mine |= pile_live(a, p) && a.pd[p].rebuild;
    return __syncthreads_or(mine) != 0;
}

// Candidates per sphere (new list buffer) and per tile.
template <bool FP64>
__global__ void __launch_bounds__(kCTile) k_cand_count(Arrays a, Sizes z)
{
    pdl_enter();
    __shared__ int red[kCTile / 32];
    if (!any_rebuild(a, z)) return;
    for (int64_t tile = blockIdx.x; tile < z.CT; tile += gridDim.x) {
    const int4 tl = a.ctile[tile];
    if (!tile_rebuilds(a, tl)) continue;
    const int p = tl.x;
    const PileStatic &S = a.ps[p];
    const int lp = a.pd[p].cpar ^ 1;
    int n = 0;
    if ((int)threadIdx.x < tl.z) {
        const int64_t k = S.s0 + tl.y + threadIdx.x;
        CandMe m;
        load_me<FP64>(a, k, m);
        for_candidates<FP64>(a, S, k, m, [&](int) { ++n; });
        a.ccnt[lp][k] = n;
    }
    // entries of the tile: every slice of 32 spheres (a warp) is as wide as
    // its longest list
    const int wmax = __reduce_max_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = 32 * wmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kCTile / 32; ++w) s += red[w];
        a.ctile_cnt[tile] = s;
    }
    __syncthreads();   // red[] is reused by the next tile
    }
}

// One block per pile: exclusive scan of the tiles' entry counts.  Lists that
// do not fit the pile's entries flag the pile (frozen at the end of the step).
__global__ void __launch_bounds__(1024) k_cand_scan(Arrays a, Sizes z)
{
    pdl_enter();
    const int p = blockIdx.x;
    if (!pile_live(a, p) || !a.pd[p].rebuild) return;
    const PileStatic &S = a.ps[p];
    __shared__ long long buf[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < S.nct; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const long long v = t < S.nct ? a.ctile_cnt[S.ct0 + t] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const long long add = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += add;
            __syncthreads();
        }
        const long long incl = buf[threadIdx.x];
        if (t < S.nct) a.ctile_base[S.ct0 + t] = (int32_t)(carry + incl - v);
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0 && carry > S.ne) {
        atomicOr(&a.pd[p].flags, DEM_FLAG_SLOTS);
        for (int64_t t = 0; t < S.nct; ++t) a.ctile_base[S.ct0 + t] = -1;
    }
}

// Offsets, then the candidates themselves, sorted by partner home index.
// Sliced layout: the 32 spheres of a slice (a warp) store entry e of their
// lists side by side, so sphere k's entry e is at coff[k] + 32 e (coalesced
// when a warp walks its lists together).
constexpr int kFillCap = 20;   // candidates sorted in shared memory per sphere (more: in place)

template <bool FP64>
__device__ __forceinline__ void cand_fill_tile(const Arrays &a, int4 tl, int base, int *sw,
                                               int2 (*s_list)[kCTile])
{
    const int p = tl.x;
    const PileStatic &S = a.ps[p];
    const int lp = a.pd[p].cpar ^ 1;
    const bool mine = (int)threadIdx.x < tl.z;
    const int64_t k = S.s0 + tl.y + threadIdx.x;
    const int n = mine ? a.ccnt[lp][k] : 0;
    const int wmax = __reduce_max_sync(0xffffffffu, n);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sw[wid] = 32 * wmax;
    __syncthreads();
    int sb = base;
    for (int w = 0; w < wid; ++w) sb += sw[w];
    if (!mine) return;
    const int off = sb + lane;
    a.coff[lp][k] = off;
    int32_t *ids = a.cand_id[lp] + S.e0 + off;
    int2 *cd = a.cand[lp] + S.e0 + off;
    const int32_t *srt = a.sorted + S.s0;
    CandMe m;
    load_me<FP64>(a, k, m);
    int j = 0;
    if (n <= kFillCap) {
        // insertion by partner home index in shared memory, then one write
        int2 *l = &s_list[0][threadIdx.x];
        for_candidates<FP64>(a, S, k, m, [&](int t) {
            if (j >= n) return;   // (the count pass visited the same candidates)
            const int id = srt[t];
            int y = j++;
            while (y > 0 && l[(y - 1) * kCTile].x > id) {
                l[y * kCTile] = l[(y - 1) * kCTile];
                --y;
            }
            l[y * kCTile] = make_int2(id, t);
        });
        for (int y = 0; y < j; ++y) {
            const int2 v = l[y * kCTile];
            ids[32 * y] = v.x;
            cd[32 * y] = make_int2(v.y, 0);
        }
        return;
    }
    for_candidates<FP64>(a, S, k, m, [&](int t) {
        if (j >= n) return;
        // long list: insertion by partner home index in place
        const int id = srt[t];
        int y = j++;
        while (y > 0 && ids[32 * (y - 1)] > id) {
            ids[32 * y] = ids[32 * (y - 1)];
            cd[32 * y] = cd[32 * (y - 1)];
            --y;
        }
        ids[32 * y] = id;
        cd[32 * y] = make_int2(t, 0);
    });
}

template <bool FP64>
__global__ void __launch_bounds__(kCTile) k_cand_fill(Arrays a, Sizes z)
{
    pdl_enter();
    __shared__ int sw[kCTile / 32];
    __shared__ int2 s_list[kFillCap][kCTile];   // (partner home index, sorted position)
    if (!any_rebuild(a, z)) return;
    for (int64_t tile = blockIdx.x; tile < z.CT; tile += gridDim.x) {
        __syncthreads();   // sw[] of the previous tile
        const int4 tl = a.ctile[tile];
        if (!tile_rebuilds(a, tl)) continue;
        const int base = a.ctile_base[tile];
        if (base < 0) continue;
        cand_fill_tile<FP64>(a, tl, base, sw, s_list);
    }
}


// Owner bit and mirror entry of every list entry; history carried from the
// previous lists (by the home indices of both spheres) into hist_rm.
template <bool FP64>
__device__ __forceinline__ void cand_link_sphere(const Arrays &a, int4 tl)
{
    typedef typename CT<FP64>::H H;
    const int p = tl.x;
    const PileStatic &S = a.ps[p];
    const PileDyn &D = a.pd[p];
    const int lp = D.cpar ^ 1, op = D.cpar, par = D.parity;
    const int64_t s0 = S.s0, e0 = S.e0;
    const int kl = tl.y + threadIdx.x;
    const int me = a.sorted[s0 + kl];
    const int n = a.ccnt[lp][s0 + kl], off = a.coff[lp][s0 + kl];
    // the previous list of this home sphere
    const int kprev = a.pos_of_home[par][s0 + me];
    const int pn = a.ccnt[op][s0 + kprev], poff = a.coff[op][s0 + kprev];
    const int32_t *pids = a.cand_id[op] + e0 + poff;
    const H *hprev;
    H *hrm;
    if constexpr (FP64) { hprev = a.hist64[par] + e0; hrm = a.hist64_rm + e0; }
    else { hprev = a.hist32[par] + e0; hrm = a.hist32_rm + e0; }
    int cursor = 0;
    for (int e = 0; e < n; ++e) {
        const int f = off + 32 * e;
        const int2 c = a.cand[lp][e0 + f];
        const int kk = c.x;
        const int id = a.cand_id[lp][e0 + f];
        // my entry in the partner's list: binary search by home index
        const int pn2 = a.ccnt[lp][s0 + kk], po2 = a.coff[lp][s0 + kk];
        const int32_t *ids2 = a.cand_id[lp] + e0 + po2;
        int lo = 0, hi = pn2 - 1, mir = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int v = ids2[32 * mid];
            if (v == me) { mir = po2 + 32 * mid; break; }
            if (v < me) lo = mid + 1; else hi = mid - 1;
        }
        if (mir < 0) atomicOr(&a.pd[p].flags, DEM_FLAG_SLOTS);   // lists not symmetric: cannot happen
        const bool owned = me < id;
        a.cand[lp][e0 + f] = make_int2(kk | (owned ? (int)0x80000000u : 0), mir < 0 ? 0 : mir);
        if (!owned) continue;
        // carried history: the same partner in the previous list (both lists
        // are in partner order, so one forward cursor finds it)
        H h;
        if constexpr (FP64) h = make_dbl4(0.0, 0.0, 0.0, 0.0);
        else h = make_float4(0.f, 0.f, 0.f, 0.f);
        while (cursor < pn && pids[32 * cursor] < id) ++cursor;
        if (cursor < pn && pids[32 * cursor] == id) {
            const H g = hprev[poff + 32 * cursor];
            if (g.w != 0) h = g;
        }
        hrm[f] = h;
    }
}

template <bool FP64>
__global__ void __launch_bounds__(kCTile) k_cand_link(Arrays a, Sizes z)
{
    pdl_enter();
    if (!any_rebuild(a, z)) return;
    for (int64_t tile = blockIdx.x; tile < z.CT; tile += gridDim.x) {
        const int4 tl = a.ctile[tile];
        if (!tile_rebuilds(a, tl) || a.ctile_base[tile] < 0 || (int)threadIdx.x >= tl.z) continue;
        cand_link_sphere<FP64>(a, tl);
    }
}

// ---------------------------------------------------------------- step
// One sorted sphere k: every entry of its list is evaluated in the canonical
// orientation (owner as sphere a, the same evaluation the tiles make) and the
// sphere keeps its own share, summed in list order; the owner's side writes
// the pair's history.  Each pair is evaluated twice (once per sphere), with
// bitwise the same result both times, so the forces equal the tile form's bit
// for bit.  s_x / s_v: the sorted spheres [kb0, kb0 + 128) staged in shared
// memory (mixed path), or null.
template <bool FP64>
__device__ __forceinline__ void sphere_contacts(const Arrays &a, const PileStatic &S, int lp,
                                                const typename CT<FP64>::H *hread,
                                                typename CT<FP64>::H *hwrite,
                                                const typename CT<FP64>::Prm &prm, float q, int64_t k,
                                                int64_t kb0, const int4 *s_x, const float4 *s_v, int &flags)
{
    typedef typename CT<FP64>::T T;
    typedef typename CT<FP64>::V V;
    typedef typename CT<FP64>::H H;
    const int64_t s0 = S.s0, e0 = S.e0;
    const int2 *cand = a.cand[lp] + e0;
    const int off = a.coff[lp][k], n = a.ccnt[lp][k];
    // own data
    typename CT<FP64>::P mp;
    float4 mr;
    typename CT<FP64>::VR mv, mw;
    if constexpr (FP64) { mp = a.dp_[k]; mv = a.dv_[k]; mw = a.dw_[k]; }
    else if (s_x) {
        const int64_t lk = k - kb0;
        mp = s_x[2 * lk]; mr = as_f4(s_x[2 * lk + 1]);
        mv = s_v[2 * lk]; mw = s_v[2 * lk + 1];
    } else {
        mp = a.xqr[2 * k]; mr = as_f4(a.xqr[2 * k + 1]);
        mv = a.svw[2 * k]; mw = a.svw[2 * k + 1];
    }
    V F, Tq;
    if constexpr (FP64) { F = d3(0, 0, 0); Tq = d3(0, 0, 0); }
    else { F = f3(0.f, 0.f, 0.f); Tq = f3(0.f, 0.f, 0.f); }
    int nc = 0;
    // One entry: this sphere as sphere a.  Every step of the law maps exactly
    // onto its negative or onto itself when the spheres swap (differences and
    // products of negated operands round to the negated or the same value),
    // so this evaluation's share a is bit for bit the share of this side of
    // the owner's evaluation; the owner's S is seen from this side with the
    // opposite sign.  The owner's side writes the history.
    auto entry = [&](int f, bool owned, bool ok, const H &hp, const typename CT<FP64>::P &pp,
                     const float4 &pr, const typename CT<FP64>::VR &pv, const typename CT<FP64>::VR &pw) {
        PairOut<T, V> o;
        bool hit = false;
        const T sgn = owned ? T(1) : T(-1);
        if (ok) {
            if constexpr (FP64) {
                const double3 Sprev = hp.w != 0 ? d3(sgn * hp.x, sgn * hp.y, sgn * hp.z) : d3(0, 0, 0);
                hit = pair_64(mp, mv, mw, pp, pv, pw, Sprev, prm, o);
            } else {
                const float3 Sprev = hp.w != 0.f ? f3(sgn * hp.x, sgn * hp.y, sgn * hp.z) : f3(0.f, 0.f, 0.f);
                hit = pair_mixed(mp, mr, pp, pr, q, mv, mw, pv, pw, Sprev, prm, o);
            }
        }
        if (owned && ok) {
            H h;
            if constexpr (FP64) h = hit ? make_dbl4(o.S.x, o.S.y, o.S.z, 1.0) : make_dbl4(0, 0, 0, 0);
            else h = hit ? make_float4(o.S.x, o.S.y, o.S.z, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
            hwrite[f] = h;
        }
        if (!hit) return;
        if (o.x > T(0.1) * o.rmin) flags |= DEM_FLAG_OVERLAP;
        V sF, sT;
        share<T, V>(o, true, sF, sT);
        F.x = addr(F.x, sF.x); F.y = addr(F.y, sF.y); F.z = addr(F.z, sF.z);
        Tq.x = addr(Tq.x, sT.x); Tq.y = addr(Tq.y, sT.y); Tq.z = addr(Tq.z, sT.z);
        ++nc;
    };
    // an entry's partner and history indices (clamped: the checks never fail)
    auto where = [&](int2 c, int f, int64_t &g, int &hidx, bool &ok) {
        const int kk = c.x & 0x7fffffff;
        hidx = c.x < 0 ? f : c.y;
        ok = (unsigned)kk < (unsigned)S.ns && (unsigned)hidx < (unsigned)S.ne;
        g = s0 + (ok ? kk : 0);
        if (!ok) hidx = 0;
    };
    if constexpr (FP64) {
        for (int e = 0; e < n; ++e) {
            const int f = off + 32 * e;
            const int2 c = cand[f];
            int64_t g;
            int hidx;
            bool ok;
            where(c, f, g, hidx, ok);
            entry(f, c.x < 0, ok, hread[hidx], a.dp_[g], make_float4(0.f, 0.f, 0.f, 0.f), a.dv_[g], a.dw_[g]);
        }
    } else {
        // partner data from the staged block when it is there, else from global memory
        auto fetch = [&](int64_t g, int4 &x, int4 &r, float4 &v, float4 &w) {
            const int64_t lk = g - kb0;
            if (s_x && (uint64_t)lk < 128) {
                x = s_x[2 * lk]; r = s_x[2 * lk + 1]; v = s_v[2 * lk]; w = s_v[2 * lk + 1];
            } else {
                x = a.xqr[2 * g]; r = a.xqr[2 * g + 1]; v = a.svw[2 * g]; w = a.svw[2 * g + 1];
            }
        };
        // software pipeline: the list entry two ahead and the partner data and
        // history one ahead are in flight while an entry is evaluated
        int2 c1 = make_int2(0, 0);
        if (n > 1) c1 = cand[off + 32];
        int2 cc = make_int2(0, 0);
        int4 px = make_int4(0, 0, 0, 0), pr = px;
        float4 pv = make_float4(0.f, 0.f, 0.f, 0.f), pw = pv;
        H hp = make_float4(0.f, 0.f, 0.f, 0.f);
        bool ok = false;
        if (n > 0) {
            cc = cand[off];
            int64_t g;
            int hidx;
            where(cc, off, g, hidx, ok);
            fetch(g, px, pr, pv, pw);
            hp = hread[hidx];
        }
        for (int e = 0; e < n; ++e) {
            const int f = off + 32 * e;
            int4 nx = px, nr = pr;
            float4 nv = pv, nw = pw;
            H nh = hp;
            bool nok = false;
            if (e + 1 < n) {
                int64_t g;
                int hidx;
                where(c1, f + 32, g, hidx, nok);
                fetch(g, nx, nr, nv, nw);
                nh = hread[hidx];
            }
            const int2 c2 = e + 2 < n ? cand[f + 64] : make_int2(0, 0);
            entry(f, cc.x < 0, ok, hp, px, as_f4(pr), pv, pw);
            cc = c1; c1 = c2;
            px = nx; pr = nr; pv = nv; pw = nw; hp = nh; ok = nok;
        }
    }
    // stored at the sphere's home index (its aggregate's members are then
    // contiguous for k_agg_end); the gathered spin record carries that index
    // (checked against the pile's range: the check never fails)
    if constexpr (FP64) {
        const int hl = (int)mw.w;
        if ((unsigned)hl < (unsigned)S.ns) {
            a.ftc64[2 * (s0 + hl)] = make_dbl4(F.x, F.y, F.z, 0.0);
            a.ftc64[2 * (s0 + hl) + 1] = make_dbl4(Tq.x, Tq.y, Tq.z, 0.0);
        }
    } else {
        const int hl = __float_as_int(mw.w);
        if ((unsigned)hl < (unsigned)S.ns)
            st_f4x2(a.ftc32 + 2 * (s0 + hl), make_float4(F.x, F.y, F.z, 0.f), make_float4(Tq.x, Tq.y, Tq.z, 0.f));
    }
    if (nc > S.K) flags |= DEM_FLAG_SLOTS;
}

// Shared memory of k_contact (dynamic): list offsets and lengths of the
// tile's spheres and its slice bases, staged sphere data, the inbox (each
// entry's share: F and tau as six arrays, and a contact flag) and the work
// queue.
template <bool FP64>
struct Smem {
    typedef typename CT<FP64>::T T;
    static constexpr int kCap = CT<FP64>::kCap;
    static constexpr size_t off_bytes = sizeof(int) * (2 * kCTile + 32);   // keeps what follows 32-byte aligned
    static constexpr size_t stage_bytes = (FP64 ? 3 * sizeof(dbl4) : 4 * sizeof(float4)) * kCTile;
    static constexpr size_t inbox_bytes = 6 * sizeof(T) * kCap;
    static constexpr size_t flag_bytes = kCap;
    static constexpr size_t queue_bytes = sizeof(int) * kCap;
    static constexpr size_t scan_bytes = sizeof(int) * (kCTile / 32 + 8);
    static constexpr size_t total = off_bytes + stage_bytes + inbox_bytes + flag_bytes + queue_bytes + scan_bytes;
};

// Exclusive prefix sum over the block (kCTile threads); *total gets the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int *ws, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < kCTile / 32 ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kCTile / 32) ws[lane] = t;
        if (lane == kCTile / 32 - 1) ws[kCTile / 32] = t;
    }
    __syncthreads();
    const int r = (wid ? ws[wid - 1] : 0) + x - v;
    *total = ws[kCTile / 32];
    __syncthreads();
    return r;
}

template <bool FP64>
__global__ void __launch_bounds__(kCTile, FP64 ? 2 : 4) k_contact(Arrays a, Sizes z)
{
    pdl_enter();
    typedef typename CT<FP64>::T T;
    typedef typename CT<FP64>::V V;
    typedef typename CT<FP64>::H H;
    typedef Smem<FP64> SM;
    const int kCap = min(SM::kCap, max(32, z.icap));
    extern __shared__ __align__(32) unsigned char smem[];
    int *s_off = (int *)smem;                 // [kCTile] list offsets (pile-local entries)
    int *s_cnt = s_off + kCTile;              // [kCTile] list lengths
    int *s_sb = s_cnt + kCTile;               // [kSl + 1] slice bases, then the tile's end
    unsigned char *stage = smem + SM::off_bytes;
    T *inbox = (T *)(stage + SM::stage_bytes);   // [6][SM::kCap]
    unsigned char *flag = (unsigned char *)(inbox + 6 * SM::kCap);
    int *queue = (int *)(flag + SM::kCap);
    int *ws = (int *)((unsigned char *)queue + SM::queue_bytes);
    __shared__ int pile_flags;

    const int4 tl = a.ctile[blockIdx.x];
    const int p = tl.x;
    if (!pile_live(a, p)) return;
    const PileStatic &S = a.ps[p];
    const PileDyn &D = a.pd[p];
    if (D.flags & DEM_FLAG_SLOTS) return;          // lists could not be built: frozen this step
    const bool rb = D.rebuild != 0;
    const int lp = rb ? D.cpar ^ 1 : D.cpar, par = D.parity;
    const int64_t s0 = S.s0, e0 = S.e0;
    const int first = tl.y, nt = tl.z;
    const int K = S.K;
    typename CT<FP64>::Prm prm;
    const H *hread;
    H *hwrite;
    if constexpr (FP64) {
        prm = {S.kn, S.kt, S.cn, S.ct, S.mu_s, S.mu_r, S.mu_t, S.w0, S.h};
        hread = (rb ? a.hist64_rm : a.hist64[par]) + e0;
        hwrite = a.hist64[par ^ 1] + e0;
    } else {
        prm = {S.lawf[0], S.lawf[1], S.lawf[2], S.lawf[3], S.lawf[4], S.lawf[5], S.lawf[6], S.lawf[7],
               S.lawf[8]};
        hread = (rb ? a.hist32_rm : a.hist32[par]) + e0;
        hwrite = a.hist32[par ^ 1] + e0;
    }
    const float q = pow2f(S.qexp);
    const int2 *cand = a.cand[lp] + e0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nsl = (nt + 31) >> 5;
    if (tid == 0) pile_flags = 0;
    {
        int off = 0, n = 0;
        if (tid < nt) {
            const int64_t k = s0 + first + tid;
            off = a.coff[lp][k];
            n = a.ccnt[lp][k];
            if constexpr (FP64) {
                dbl4 *st = (dbl4 *)stage;
                st[tid] = a.dp_[k];
                st[kCTile + tid] = a.dv_[k];
                st[2 * kCTile + tid] = a.dw_[k];
            } else {
                int4 *sx = (int4 *)stage;
                float4 *sv = (float4 *)(sx + kCTile);
                const int4 xr = a.xqr[2 * k + 1];
                sx[tid] = a.xqr[2 * k];
                sv[tid] = a.svw[2 * k];
                sv[kCTile + tid] = a.svw[2 * k + 1];
                sv[2 * kCTile + tid] = make_float4(__int_as_float(xr.x), __int_as_float(xr.y),
                                                   __int_as_float(xr.z), __int_as_float(xr.w));
            }
        }
        s_off[tid] = off;
        s_cnt[tid] = n;
        const int wmax = __reduce_max_sync(0xffffffffu, n);
        if (lane == 0 && wid < nsl) s_sb[wid] = off;               // lane 0 sits at its slice's base
        if (lane == 0 && wid == nsl - 1) s_sb[nsl] = off + 32 * wmax;
    }
    __syncthreads();
    int myflags = 0;
    // slice ranges [r0, r1) of the tile whose list entries fit the inbox
    for (int r0 = 0; r0 < nsl;) {
        int r1 = nsl;
        while (s_sb[r1] - s_sb[r0] > kCap && r1 - r0 > 1) r1 = r0 + (r1 - r0 + 1) / 2;
        const int E0 = s_sb[r0], nE = s_sb[r1] - E0;
        if (nE > SM::kCap) {
            // one slice with more list entries than the inbox holds: its
            // spheres evaluate their own lists (bitwise the same results)
            if (tid >= 32 * r0 && tid < min(32 * r1, nt))
                sphere_contacts<FP64>(a, S, lp, hread, hwrite, prm, q, s0 + first + tid, 0, nullptr, nullptr,
                                      myflags);
            r0 = r1;
            continue;
        }
        const int i0 = 32 * r0, i1 = min(32 * r1, nt);
        // work queue in (sphere, entry) order: pairs this range owns, and
        // pairs that leave the range (from this sphere's side)
        const unsigned lo = (unsigned)(first + i0), span = (unsigned)(i1 - i0);
        const bool inr = tid >= i0 && tid < i1;
        const int off = s_off[tid], n = inr ? s_cnt[tid] : 0;
        int cnt = 0;
        for (int e = 0; e < n; ++e) {
            const int2 c = cand[off + 32 * e];
            const unsigned kk = (unsigned)c.x & 0x7fffffffu;
            cnt += (c.x < 0 || kk - lo >= span) ? 1 : 0;
        }
        int nq;
        int pos = block_exclusive_scan(cnt, ws, &nq);
        for (int e = 0; e < n; ++e) {
            const int2 c = cand[off + 32 * e];
            const unsigned kk = (unsigned)c.x & 0x7fffffffu;
            if (c.x < 0 || kk - lo >= span) queue[pos++] = (tid << 12) | e;
        }
        __syncthreads();
        for (int r = tid; r < nq; r += kCTile) {
            const int rec = queue[r];
            const int i = rec >> 12, e = rec & 0xfff;
            const int f = s_off[i] + 32 * e;
            const int2 c = cand[f];
            const int kk = c.x & 0x7fffffff;
            const bool owned = c.x < 0;
            const bool inner = (unsigned)kk - lo < span;
            // sphere a is the owner
            const int ia = owned ? i : kk - first, ib = owned ? kk - first : i;
            const bool a_loc = owned || inner, b_loc = !owned || inner;
            const int hidx = owned ? f : c.y;
            if ((unsigned)kk >= (unsigned)S.ns || (unsigned)hidx >= (unsigned)S.ne) continue;   // (never taken)
            const H hp = hread[hidx];
            PairOut<T, V> o;
            bool hit;
            if constexpr (FP64) {
                const dbl4 *st = (const dbl4 *)stage;
                const int64_t ga = s0 + (owned ? first + i : kk), gb = s0 + (owned ? kk : first + i);
                const dbl4 ap = a_loc ? st[ia] : a.dp_[ga], av = a_loc ? st[kCTile + ia] : a.dv_[ga],
                           aw = a_loc ? st[2 * kCTile + ia] : a.dw_[ga];
                const dbl4 bp = b_loc ? st[ib] : a.dp_[gb], bv = b_loc ? st[kCTile + ib] : a.dv_[gb],
                           bw = b_loc ? st[2 * kCTile + ib] : a.dw_[gb];
                const double3 Sprev = hp.w != 0 ? d3(hp.x, hp.y, hp.z) : d3(0, 0, 0);
                hit = pair_64(ap, av, aw, bp, bv, bw, Sprev, prm, o);
            } else {
                const int4 *sx = (const int4 *)stage;
                const float4 *sv = (const float4 *)(sx + kCTile);
                const int64_t ga = s0 + (owned ? first + i : kk), gb = s0 + (owned ? kk : first + i);
                const int4 A = a_loc ? sx[ia] : a.xqr[2 * ga], B = b_loc ? sx[ib] : a.xqr[2 * gb];
                const float4 RA = a_loc ? sv[2 * kCTile + ia] : as_f4(a.xqr[2 * ga + 1]);
                const float4 RB = b_loc ? sv[2 * kCTile + ib] : as_f4(a.xqr[2 * gb + 1]);
                const float4 av = a_loc ? sv[ia] : a.svw[2 * ga], aw = a_loc ? sv[kCTile + ia] : a.svw[2 * ga + 1];
                const float4 bv = b_loc ? sv[ib] : a.svw[2 * gb], bw = b_loc ? sv[kCTile + ib] : a.svw[2 * gb + 1];
                const float3 Sprev = hp.w != 0.f ? f3(hp.x, hp.y, hp.z) : f3(0.f, 0.f, 0.f);
                hit = pair_mixed(A, RA, B, RB, q, av, aw, bv, bw, Sprev, prm, o);
            }
            if (owned) {
                H h;
                if constexpr (FP64) h = hit ? make_dbl4(o.S.x, o.S.y, o.S.z, 1.0) : make_dbl4(0, 0, 0, 0);
                else h = hit ? make_float4(o.S.x, o.S.y, o.S.z, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
                hwrite[f] = h;
            }
            if (hit && o.x > T(0.1) * o.rmin) myflags |= DEM_FLAG_OVERLAP;
            V F, Tq;
            if (a_loc) {
                const int slot = (owned ? f : c.y) - E0;
                if ((unsigned)slot >= (unsigned)nE) continue;   // (lists are symmetric: never taken)
                if (hit) {
                    share<T, V>(o, true, F, Tq);
                    inbox[slot] = F.x; inbox[SM::kCap + slot] = F.y; inbox[2 * SM::kCap + slot] = F.z;
                    inbox[3 * SM::kCap + slot] = Tq.x; inbox[4 * SM::kCap + slot] = Tq.y;
                    inbox[5 * SM::kCap + slot] = Tq.z;
                }
                flag[slot] = hit ? 1 : 0;
            }
            if (b_loc) {
                const int slot = (owned ? c.y : f) - E0;
                if ((unsigned)slot >= (unsigned)nE) continue;
                if (hit) {
                    share<T, V>(o, false, F, Tq);
                    inbox[slot] = F.x; inbox[SM::kCap + slot] = F.y; inbox[2 * SM::kCap + slot] = F.z;
                    inbox[3 * SM::kCap + slot] = Tq.x; inbox[4 * SM::kCap + slot] = Tq.y;
                    inbox[5 * SM::kCap + slot] = Tq.z;
                }
                flag[slot] = hit ? 1 : 0;
            }
        }
        __syncthreads();
        // every sphere of the range sums its slots in list order
        if (inr) {
            V F, Tq;
            if constexpr (FP64) { F = d3(0, 0, 0); Tq = d3(0, 0, 0); }
            else { F = f3(0.f, 0.f, 0.f); Tq = f3(0.f, 0.f, 0.f); }
            int nc = 0;
            for (int e = 0; e < n; ++e) {
                const int slot = off - E0 + 32 * e;
                if (!flag[slot]) continue;
                F.x = addr(F.x, inbox[slot]); F.y = addr(F.y, inbox[SM::kCap + slot]);
                F.z = addr(F.z, inbox[2 * SM::kCap + slot]);
                Tq.x = addr(Tq.x, inbox[3 * SM::kCap + slot]); Tq.y = addr(Tq.y, inbox[4 * SM::kCap + slot]);
                Tq.z = addr(Tq.z, inbox[5 * SM::kCap + slot]);
                ++nc;
            }
            // at the sphere's home index (from the staged spin record; checked
            // against the pile's range, which it never leaves)
            if constexpr (FP64) {
                const int hl = (int)((const dbl4 *)stage)[2 * kCTile + tid].w;
                if ((unsigned)hl < (unsigned)S.ns) {
                    a.ftc64[2 * (s0 + hl)] = make_dbl4(F.x, F.y, F.z, 0.0);
                    a.ftc64[2 * (s0 + hl) + 1] = make_dbl4(Tq.x, Tq.y, Tq.z, 0.0);
                }
            } else {
                const float4 *sv = (const float4 *)((const int4 *)stage + kCTile);
                const int hl = __float_as_int(sv[kCTile + tid].w);
                if ((unsigned)hl < (unsigned)S.ns)
                    st_f4x2(a.ftc32 + 2 * (s0 + hl), make_float4(F.x, F.y, F.z, 0.f),
                            make_float4(Tq.x, Tq.y, Tq.z, 0.f));
            }
            if (nc > K) myflags |= DEM_FLAG_SLOTS;
        }
        __syncthreads();
        r0 = r1;
    }
    if (myflags) atomicOr(&pile_flags, myflags);
    __syncthreads();
    if (tid == 0 && pile_flags) atomicOr(&a.pd[p].flags, pile_flags);
}

// One thread per sorted sphere (sphere_contacts); the block's own 128 sorted
// spheres are staged in shared memory in the mixed path (consecutive sorted
// spheres fill a compact block of space, so most partners are among them).
template <bool FP64>
__global__ void __launch_bounds__(128) k_contact_sphere(Arrays a, Sizes z)
{
    pdl_enter();
    typedef typename CT<FP64>::H H;
    const int64_t kb0 = (int64_t)blockIdx.x * 128;
    const int64_t k = kb0 + threadIdx.x;
    __shared__ int4 s_x[FP64 ? 1 : 2 * 128];
    __shared__ float4 s_v[FP64 ? 1 : 2 * 128];
    if constexpr (!FP64) {
        if (k < z.N) {
            s_x[2 * threadIdx.x] = a.xqr[2 * k];
            s_x[2 * threadIdx.x + 1] = a.xqr[2 * k + 1];
            s_v[2 * threadIdx.x] = a.svw[2 * k];
            s_v[2 * threadIdx.x + 1] = a.svw[2 * k + 1];
        }
        __syncthreads();
    }
    if (k >= z.N) return;
    const int p = a.sph_pile[k];
    if (!pile_live(a, p)) return;
    const PileStatic &S = a.ps[p];
    const PileDyn &D = a.pd[p];
    if (D.flags & DEM_FLAG_SLOTS) return;
    const bool rb = D.rebuild != 0;
    const int lp = rb ? D.cpar ^ 1 : D.cpar, par = D.parity;
    typename CT<FP64>::Prm prm;
    const H *hread;
    H *hwrite;
    if constexpr (FP64) {
        prm = {S.kn, S.kt, S.cn, S.ct, S.mu_s, S.mu_r, S.mu_t, S.w0, S.h};
        hread = (rb ? a.hist64_rm : a.hist64[par]) + S.e0;
        hwrite = a.hist64[par ^ 1] + S.e0;
    } else {
        prm = {S.lawf[0], S.lawf[1], S.lawf[2], S.lawf[3], S.lawf[4], S.lawf[5], S.lawf[6], S.lawf[7],
               S.lawf[8]};
        hread = (rb ? a.hist32_rm : a.hist32[par]) + S.e0;
        hwrite = a.hist32[par ^ 1] + S.e0;
    }
    int flags = 0;
    sphere_contacts<FP64>(a, S, lp, hread, hwrite, prm, pow2f(S.qexp), k, kb0, FP64 ? nullptr : s_x,
                          FP64 ? nullptr : s_v, flags);
    if (flags) atomicOr(&a.pd[p].flags, flags);
}

cudaError_t contact_setup(bool fp64, int)
{
    if (fp64)
        return cudaFuncSetAttribute(k_contact<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Smem<true>::total);
    return cudaFuncSetAttribute(k_contact<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Smem<false>::total);
}

void launch_contact(const Arrays &a, const Sizes &z, bool fp64, int, cudaStream_t st)
{
    if (z.N == 0 || z.CT == 0) return;
    const unsigned nt = (unsigned)z.CT;
    // the rebuild kernels walk the tiles with a grid of a few blocks per SM:
    // in steps without a rebuild they only read each tile's pile flags
    const unsigned ng = (unsigned)(z.CT < 512 ? z.CT : 512);
    if (fp64) {
        launch_pdl(k_cand_count<true>, ng, kCTile, 0, st, a, z);
        launch_pdl(k_cand_scan, (unsigned)z.P, 1024, 0, st, a, z);
        launch_pdl(k_cand_fill<true>, ng, kCTile, 0, st, a, z);
        launch_pdl(k_cand_link<true>, ng, kCTile, 0, st, a, z);
        if (z.cmode == 1) launch_pdl(k_contact<true>, nt, kCTile, Smem<true>::total, st, a, z);
        else launch_pdl(k_contact_sphere<true>, (unsigned)((z.N + 127) / 128), 128, 0, st, a, z);
    } else {
        launch_pdl(k_cand_count<false>, ng, kCTile, 0, st, a, z);
        launch_pdl(k_cand_scan, (unsigned)z.P, 1024, 0, st, a, z);
        launch_pdl(k_cand_fill<false>, ng, kCTile, 0, st, a, z);
        launch_pdl(k_cand_link<false>, ng, kCTile, 0, st, a, z);
        if (z.cmode == 1) launch_pdl(k_contact<false>, nt, kCTile, Smem<false>::total, st, a, z);
        else launch_pdl(k_contact_sphere<false>, (unsigned)((z.N + 127) / 128), 128, 0, st, a, z);
    }
}

}  // namespace dem
