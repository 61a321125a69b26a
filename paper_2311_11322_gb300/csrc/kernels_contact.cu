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
// One evaluation per pair.  The law is evaluated with the owner as sphere a
// (canonical orientation), so both spheres' shares come from one evaluation:
//   a:  F,  tau_a = (l_a n) x F + M;   b:  -F,  tau_b = (l_b n) x F - M.
// k_contact works on tiles of kCTile consecutive sorted spheres, which fill
// compact blocks of space (cells are numbered brick by brick).  A pair inside
// a tile is evaluated once, by the thread that drew it from the tile's work
// queue, and both shares go to the spheres' slots in a shared-memory inbox; a
// pair that crosses tiles is evaluated by both tiles, each keeping its own
// sphere's share.  Every sphere then sums its inbox slots in list order, i.e.
// in the order of its partners' home indices, so forces, torques and history
// are bitwise the same whatever the tiles, the cell size, the skin or the
// steps at which the lists were rebuilt.  Nothing is written with atomics
// except error flags and the work-queue counter.
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
    const float num = __fadd_rn(__ll2float_rn(num_i), corr);
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

template <typename T, typename V>
__device__ __forceinline__ void share_a(const PairOut<T, V> &o, V &F, V &Tq)
{
    F = o.F;
    const V c = lever_x_force(o.la, o.n, o.F);
    Tq.x = addr(c.x, o.M.x); Tq.y = addr(c.y, o.M.y); Tq.z = addr(c.z, o.M.z);
}
template <typename T, typename V>
__device__ __forceinline__ void share_b(const PairOut<T, V> &o, V &F, V &Tq)
{
    F.x = -o.F.x; F.y = -o.F.y; F.z = -o.F.z;
    const V c = lever_x_force(o.lb, o.n, o.F);
    Tq.x = addr(c.x, -o.M.x); Tq.y = addr(c.y, -o.M.y); Tq.z = addr(c.z, -o.M.z);
}

template <bool FP64> struct CT;
template <> struct CT<false> {
    typedef float T;
    typedef float3 V;
    typedef ParamsF Prm;
    typedef float4 H;                      // history record
    typedef int4 P;                        // position record
    static constexpr int kCap = kInboxCap; // inbox entries per block
};
template <> struct CT<true> {
    typedef double T;
    typedef double3 V;
    typedef ParamsD Prm;
    typedef dbl4 H;
    typedef dbl4 P;
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
        // coarse FP32 test first: rejects spheres of another wrap of the grid,
        // whose 32-bit fixed-point difference would alias
        const float4 q = a.sph_[kk];
        const float dx = __fsub_rn(q.x, m.ph.x), dy = __fsub_rn(q.y, m.ph.y), dz = __fsub_rn(q.z, m.ph.z);
        const float tc = __fmul_rn(2.0f, __fadd_rn(__fadd_rn(q.w, m.ph.w), (float)S.skin)) + 1e-30f;
        if (!(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < __fmul_rn(tc, tc))) return false;
        const int4 B = a.xq[kk];
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
    const bool one = cx >= 1 && cx + 1 < S.nx && ((cx - 1) >> 2) == ((cx + 1) >> 2);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrapc(cy + dy, S.ny), zz = wrapc(cz + dz, S.nz);
            int beg[3], end[3], nr;
            if (one) {
                const int64_t c0 = cell_id(cx - 1, yy, zz, S.nx, S.ny);
                beg[0] = cstart[c0];
                end[0] = cstart[c0 + 2] + ccount[c0 + 2];
                nr = 1;
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
        m.xq = a.xq[k];
        m.ph = a.sph_[k];
    }
    m.agg = a.sagg[k];
}

// ---------------------------------------------------------------- rebuild
__device__ __forceinline__ bool tile_rebuilds(const Arrays &a, int4 tl)
{
    return pile_live(a, tl.x) && a.pd[tl.x].rebuild;
}

// Candidates per sphere (new list buffer) and per tile.
template <bool FP64>
__global__ void __launch_bounds__(kCTile) k_cand_count(Arrays a, Sizes z)
{
    pdl_enter();
    __shared__ int red[kCTile / 32];
    const int4 tl = a.ctile[blockIdx.x];
    if (!tile_rebuilds(a, tl)) return;
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
    int v = n;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kCTile / 32; ++w) s += red[w];
        a.ctile_cnt[blockIdx.x] = s;
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
template <bool FP64>
__global__ void __launch_bounds__(kCTile) k_cand_fill(Arrays a, Sizes z)
{
    pdl_enter();
    __shared__ int pre[kCTile];
    const int4 tl = a.ctile[blockIdx.x];
    if (!tile_rebuilds(a, tl)) return;
    const int base = a.ctile_base[blockIdx.x];
    if (base < 0) return;
    const int p = tl.x;
    const PileStatic &S = a.ps[p];
    const int lp = a.pd[p].cpar ^ 1;
    const bool mine = (int)threadIdx.x < tl.z;
    const int64_t k = S.s0 + tl.y + threadIdx.x;
    const int n = mine ? a.ccnt[lp][k] : 0;
    pre[threadIdx.x] = n;
    __syncthreads();
    for (int o = 1; o < kCTile; o <<= 1) {
        const int add = threadIdx.x >= (unsigned)o ? pre[threadIdx.x - o] : 0;
        __syncthreads();
        pre[threadIdx.x] += add;
        __syncthreads();
    }
    if (!mine) return;
    const int off = base + pre[threadIdx.x] - n;
    a.coff[lp][k] = off;
    int32_t *ids = a.cand_id[lp] + S.e0 + off;
    int2 *cd = a.cand[lp] + S.e0 + off;
    const int32_t *srt = a.sorted + S.s0;
    CandMe m;
    load_me<FP64>(a, k, m);
    int j = 0;
    for_candidates<FP64>(a, S, k, m, [&](int t) {
        if (j >= n) return;   // (the count pass visited the same candidates)
        // insertion by partner home index (lists are short)
        const int id = srt[t];
        int y = j++;
        while (y > 0 && ids[y - 1] > id) {
            ids[y] = ids[y - 1];
            cd[y] = cd[y - 1];
            --y;
        }
        ids[y] = id;
        cd[y] = make_int2(t, 0);
    });
}

// Owner bit and mirror entry of every list entry; history carried from the
// previous lists (by the home indices of both spheres) into hist_rm.
template <bool FP64>
__global__ void __launch_bounds__(kCTile) k_cand_link(Arrays a, Sizes z)
{
    pdl_enter();
    typedef typename CT<FP64>::H H;
    const int4 tl = a.ctile[blockIdx.x];
    if (!tile_rebuilds(a, tl)) return;
    if (a.ctile_base[blockIdx.x] < 0) return;
    if ((int)threadIdx.x >= tl.z) return;
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
        const int f = off + e;
        const int2 c = a.cand[lp][e0 + f];
        const int kk = c.x;
        const int id = a.cand_id[lp][e0 + f];
        // my entry in the partner's list: binary search by home index
        const int pn2 = a.ccnt[lp][s0 + kk], po2 = a.coff[lp][s0 + kk];
        const int32_t *ids2 = a.cand_id[lp] + e0 + po2;
        int lo = 0, hi = pn2 - 1, mir = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int v = ids2[mid];
            if (v == me) { mir = po2 + mid; break; }
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
        while (cursor < pn && pids[cursor] < id) ++cursor;
        if (cursor < pn && pids[cursor] == id) {
            const H g = hprev[poff + cursor];
            if (g.w != 0) h = g;
        }
        hrm[f] = h;
    }
}

// ---------------------------------------------------------------- step
// Shared memory of k_contact (dynamic): list offsets of the tile's spheres,
// staged sphere data, the inbox (each entry's share: F, tau) with contact
// flags, and the work queue.
template <bool FP64>
struct Smem {
    typedef typename CT<FP64>::T T;
    static constexpr int kCap = CT<FP64>::kCap;
    static constexpr size_t off_bytes = sizeof(int) * (kCTile + 8);   // keeps what follows 32-byte aligned
    static constexpr size_t stage_bytes = (FP64 ? 3 * sizeof(dbl4) : 4 * sizeof(float4)) * kCTile;
    static constexpr size_t inbox_bytes = 6 * sizeof(T) * kCap;
    static constexpr size_t flag_bytes = kCap;
    static constexpr size_t queue_bytes = sizeof(int) * kCap;
    static constexpr size_t total = off_bytes + stage_bytes + inbox_bytes + flag_bytes + queue_bytes + 16;
};

template <bool FP64>
__global__ void __launch_bounds__(kCTile, FP64 ? 1 : 2) k_contact(Arrays a, Sizes z)
{
    pdl_enter();
    typedef typename CT<FP64>::T T;
    typedef typename CT<FP64>::V V;
    typedef typename CT<FP64>::H H;
    typedef Smem<FP64> SM;
    const int kCap = min(SM::kCap, max(1, z.icap));
    extern __shared__ __align__(32) unsigned char smem[];
    int *s_off = (int *)smem;
    unsigned char *stage = smem + SM::off_bytes;
    T *inbox = (T *)(stage + SM::stage_bytes);
    unsigned char *flag = (unsigned char *)(inbox + 6 * SM::kCap);
    int *queue = (int *)(flag + SM::kCap);
    __shared__ int qn, pile_flags;

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
        prm = {(float)S.kn, (float)S.kt, (float)S.cn, (float)S.ct, (float)S.mu_s, (float)S.mu_r,
               (float)S.mu_t, (float)S.w0, (float)S.h};
        hread = (rb ? a.hist32_rm : a.hist32[par]) + e0;
        hwrite = a.hist32[par ^ 1] + e0;
    }
    const float q = pow2f(S.qexp);
    const int2 *cand = a.cand[lp] + e0;
    const int tid = threadIdx.x;
    if (tid == 0) pile_flags = 0;
    if (tid < nt) {
        const int64_t k = s0 + first + tid;
        const int off = a.coff[lp][k];
        s_off[tid] = off;
        if (tid == nt - 1) s_off[nt] = off + a.ccnt[lp][k];
        if constexpr (FP64) {
            dbl4 *st = (dbl4 *)stage;
            st[tid] = a.dp_[k];
            st[kCTile + tid] = a.dv_[k];
            st[2 * kCTile + tid] = a.dw_[k];
        } else {
            int4 *sx = (int4 *)stage;
            float4 *sv = (float4 *)(sx + kCTile);
            sx[tid] = a.xq[k];
            sv[tid] = a.sv_[k];
            sv[kCTile + tid] = a.sw_[k];
            sv[2 * kCTile + tid] = a.xr[k];
        }
    }
    __syncthreads();
    int myflags = 0;
    // sphere ranges [r0, r1) of the tile whose list entries fit the inbox
    for (int r0 = 0; r0 < nt;) {
        int r1 = nt;
        while (s_off[r1] - s_off[r0] > kCap && r1 - r0 > 1) r1 = r0 + (r1 - r0 + 1) / 2;
        const int E0 = s_off[r0];
        if (s_off[r1] - E0 > SM::kCap) {   // one sphere with more candidates than the inbox holds
            if (tid == 0) atomicOr(&pile_flags, DEM_FLAG_SLOTS);
            r0 = r1;
            continue;
        }
        if (tid == 0) qn = 0;
        __syncthreads();
        // work queue: entries this range evaluates -- pairs it owns, and pairs
        // that leave the range (from this sphere's side)
        const unsigned lo = (unsigned)(first + r0), span = (unsigned)(r1 - r0);
        if (tid >= r0 && tid < r1) {
            const int off = s_off[tid], n = s_off[tid + 1] - off;
            for (int e = 0; e < n; ++e) {
                const int2 c = cand[off + e];
                const unsigned kk = (unsigned)c.x & 0x7fffffffu;
                const bool owned = c.x < 0, inner = kk - lo < span;
                if (owned || !inner) queue[atomicAdd(&qn, 1)] = (tid << 12) | e;
            }
        }
        __syncthreads();
        const int nq = qn;
        for (int r = tid; r < nq; r += kCTile) {
            const int rec = queue[r];
            const int i = rec >> 12, e = rec & 0xfff;
            const int f = s_off[i] + e;
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
            V Sprev;
            PairOut<T, V> o;
            bool hit;
            if constexpr (FP64) {
                const dbl4 *st = (const dbl4 *)stage;
                const int64_t ga = s0 + (owned ? first + i : kk), gb = s0 + (owned ? kk : first + i);
                const dbl4 ap = a_loc ? st[ia] : a.dp_[ga], av = a_loc ? st[kCTile + ia] : a.dv_[ga],
                           aw = a_loc ? st[2 * kCTile + ia] : a.dw_[ga];
                const dbl4 bp = b_loc ? st[ib] : a.dp_[gb], bv = b_loc ? st[kCTile + ib] : a.dv_[gb],
                           bw = b_loc ? st[2 * kCTile + ib] : a.dw_[gb];
                Sprev = hp.w != 0 ? d3(hp.x, hp.y, hp.z) : d3(0, 0, 0);
                hit = pair_64(ap, av, aw, bp, bv, bw, Sprev, prm, o);
            } else {
                const int4 *sx = (const int4 *)stage;
                const float4 *sv = (const float4 *)(sx + kCTile);
                const int64_t ga = s0 + (owned ? first + i : kk), gb = s0 + (owned ? kk : first + i);
                const int4 A = a_loc ? sx[ia] : a.xq[ga], B = b_loc ? sx[ib] : a.xq[gb];
                const float4 RA = a_loc ? sv[2 * kCTile + ia] : a.xr[ga], RB = b_loc ? sv[2 * kCTile + ib] : a.xr[gb];
                const float4 av = a_loc ? sv[ia] : a.sv_[ga], aw = a_loc ? sv[kCTile + ia] : a.sw_[ga];
                const float4 bv = b_loc ? sv[ib] : a.sv_[gb], bw = b_loc ? sv[kCTile + ib] : a.sw_[gb];
                Sprev = hp.w != 0.f ? f3(hp.x, hp.y, hp.z) : f3(0.f, 0.f, 0.f);
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
            const unsigned nE = (unsigned)(s_off[r1] - E0);
            if (a_loc) {
                const int slot = (owned ? f : c.y) - E0;
                if ((unsigned)slot >= nE) continue;   // (lists are symmetric: never taken)
                if (hit) {
                    share_a<T, V>(o, F, Tq);
                    T *ib_ = inbox + 6 * slot;
                    ib_[0] = F.x; ib_[1] = F.y; ib_[2] = F.z; ib_[3] = Tq.x; ib_[4] = Tq.y; ib_[5] = Tq.z;
                }
                flag[slot] = hit ? 1 : 0;
            }
            if (b_loc) {
                const int slot = (owned ? c.y : f) - E0;
                if ((unsigned)slot >= nE) continue;
                if (hit) {
                    share_b<T, V>(o, F, Tq);
                    T *ib_ = inbox + 6 * slot;
                    ib_[0] = F.x; ib_[1] = F.y; ib_[2] = F.z; ib_[3] = Tq.x; ib_[4] = Tq.y; ib_[5] = Tq.z;
                }
                flag[slot] = hit ? 1 : 0;
            }
        }
        __syncthreads();
        // every sphere of the range sums its slots in list order
        if (tid >= r0 && tid < r1) {
            const int off = s_off[tid], n = s_off[tid + 1] - off;
            V F, Tq;
            if constexpr (FP64) { F = d3(0, 0, 0); Tq = d3(0, 0, 0); }
            else { F = f3(0.f, 0.f, 0.f); Tq = f3(0.f, 0.f, 0.f); }
            int nc = 0;
            for (int e = 0; e < n; ++e) {
                const int slot = off + e - E0;
                if (!flag[slot]) continue;
                const T *ib_ = inbox + 6 * slot;
                F.x = addr(F.x, ib_[0]); F.y = addr(F.y, ib_[1]); F.z = addr(F.z, ib_[2]);
                Tq.x = addr(Tq.x, ib_[3]); Tq.y = addr(Tq.y, ib_[4]); Tq.z = addr(Tq.z, ib_[5]);
                ++nc;
            }
            const int64_t k = s0 + first + tid;
            if constexpr (FP64) {
                a.ftc64[2 * k] = make_dbl4(F.x, F.y, F.z, 0.0);
                a.ftc64[2 * k + 1] = make_dbl4(Tq.x, Tq.y, Tq.z, 0.0);
            } else {
                a.ftc32[2 * k] = make_float4(F.x, F.y, F.z, __int_as_float(nc));
                a.ftc32[2 * k + 1] = make_float4(Tq.x, Tq.y, Tq.z, 0.f);
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
    if (fp64) {
        launch_pdl(k_cand_count<true>, nt, kCTile, 0, st, a, z);
        launch_pdl(k_cand_scan, (unsigned)z.P, 1024, 0, st, a, z);
        launch_pdl(k_cand_fill<true>, nt, kCTile, 0, st, a, z);
        launch_pdl(k_cand_link<true>, nt, kCTile, 0, st, a, z);
        launch_pdl(k_contact<true>, nt, kCTile, Smem<true>::total, st, a, z);
    } else {
        launch_pdl(k_cand_count<false>, nt, kCTile, 0, st, a, z);
        launch_pdl(k_cand_scan, (unsigned)z.P, 1024, 0, st, a, z);
        launch_pdl(k_cand_fill<false>, nt, kCTile, 0, st, a, z);
        launch_pdl(k_cand_link<false>, nt, kCTile, 0, st, a, z);
        launch_pdl(k_contact<false>, nt, kCTile, Smem<false>::total, st, a, z);
    }
}

}  // namespace dem
