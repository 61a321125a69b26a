// kernels_step.cu -- per-step kernels other than the contact pass and gravity:
// rigid-body kick/drift/rotation, pile reductions, sphere expansion and cell
// keys, the counting sort into cells, the sorted gather, and the reduction of
// sphere forces onto aggregates with the closing kick.
//
// Paper references: leapfrog with predicted velocities (Sec. 2.1), aggregate
// mass and COM (Sec. 2.2.1, Eq. agg_mass, Eq. agg_position), Euler's equations
// for spin (Sec. 2.2.1), predicted sphere velocity (Sec. 2.2.2, Eq. pred-vel),
// aggregate force and torque sums (Sec. 2.2.3-2.2.4, Eq. agg_gravity,
// Eq. gravity_torque, Eq. agg_contact_accel, contact torque at the contact
// point), YORP increment (Sec. 4.1), point-mass planet (Sec. 4.2).
#include "dem_internal.h"
#include "devmath.cuh"
#include "launch.cuh"

namespace dem {

__device__ __forceinline__ bool pile_active(const Arrays &a, int p)
{
    return a.enabled[p] != 0 && a.pd[p].failed == 0;
}

// ---------------------------------------------------------------- ids
__device__ int find_slot(const PileStatic *ps, int P, int64_t idx, int which)
{
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int64_t b = which == 0 ? ps[mid].s0 : which == 1 ? ps[mid].a0 : which == 2 ? ps[mid].t0 : ps[mid].ch0;
        if (b <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_fill_ids(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int P = (int)z.P;
    if (t < z.N) a.sph_pile[t] = find_slot(a.ps, P, t, 0);
    if (t < z.A) a.agg_pile[t] = find_slot(a.ps, P, t, 1);
    if (t < z.CH) a.chunk_pile[t] = find_slot(a.ps, P, t, 3);
}

void launch_fill_ids(const Arrays &a, const Sizes &z, cudaStream_t st)
{
    int64_t n = z.N > z.A ? z.N : z.A;
    if (z.CH > n) n = z.CH;
    if (n == 0 || z.P == 0) return;
    launch_pdl(k_fill_ids, (unsigned)((n + 255) / 256), 256, 0, st, a, z);
}

// ---------------------------------------------------------------- rotation
// Torque-free Euler equations in the body frame (Sec. 2.2.1):
//   dq/dt = 1/2 q (x) (0, w),  dw/dt = I^-1 (-w x (I w)).
__device__ __forceinline__ void rot_rhs(const double *y, const double *I, const double *Iinv,
                                        double *dy)
{
    const double *q = y, *w = y + 4;
    dy[0] = -0.5 * (q[1] * w[0] + q[2] * w[1] + q[3] * w[2]);
    dy[1] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    dy[2] = 0.5 * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
    dy[3] = 0.5 * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
    double3 wv = d3(w[0], w[1], w[2]);
    double3 Iw = mat_mul(I, wv);
    double3 g = -cross(wv, Iw);
    double3 dw = mat_mul(Iinv, g);
    dy[4] = dw.x; dy[5] = dw.y; dy[6] = dw.z;
}

// One classical RK4 step of the free rotor over h, q renormalised.
__device__ void free_rotate(double *q, double3 &wb, const double *I, const double *Iinv, double h)
{
    double y[7] = {q[0], q[1], q[2], q[3], wb.x, wb.y, wb.z};
    double k1[7], k2[7], k3[7], k4[7], t[7];
    rot_rhs(y, I, Iinv, k1);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + 0.5 * h * k1[c];
    rot_rhs(t, I, Iinv, k2);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + 0.5 * h * k2[c];
    rot_rhs(t, I, Iinv, k3);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + h * k3[c];
    rot_rhs(t, I, Iinv, k4);
    for (int c = 0; c < 7; ++c) y[c] += h / 6.0 * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
    double n = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
    q[0] = y[0] / n; q[1] = y[1] / n; q[2] = y[2] / n; q[3] = y[3] / n;
    wb = d3(y[4], y[5], y[6]);
}

// Stage derivatives of the torque-free rotor in FP32 (mixed path).
__device__ __forceinline__ void rot_rhs_f(const float *y, const float *I, const float *Iinv, float *dy)
{
    const float *q = y, *w = y + 4;
    dy[0] = -0.5f * (q[1] * w[0] + q[2] * w[1] + q[3] * w[2]);
    dy[1] = 0.5f * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    dy[2] = 0.5f * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
    dy[3] = 0.5f * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
    const float3 wv = f3(w[0], w[1], w[2]);
    const float3 dw = mat_mulf(Iinv, -cross(wv, mat_mulf(I, wv)));
    dy[4] = dw.x; dy[5] = dw.y; dy[6] = dw.z;
}

// The paper's rotation integrator (Sec. 2.2.1): time-adaptive fifth-order
// Runge-Kutta.  The torque-free rotation over h is taken in substeps of the
// embedded Cash-Karp RK5(4) pair; a substep is accepted when the difference
// of its fifth- and fourth-order results (q absolute, w relative to |w|) is
// within tol, the next one is scaled by 0.9 (tol/err)^(1/5) (at most x5), a
// rejected one retried at 0.9 (tol/err)^(1/4) of it (at least x0.1); the first
// trial is the whole step, and a substep below h / 2^20 is accepted whatever
// its error, so the loop ends.  FP64 in both precisions; q renormalised at the
// end as after RK4.
__device__ void free_rotate_adaptive(double *q, double3 &wb, const double *I, const double *Iinv,
                                     double h, double tol)
{
    // Cash-Karp coefficients
    const double A21 = 1.0 / 5.0;
    const double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
    const double A41 = 3.0 / 10.0, A42 = -9.0 / 10.0, A43 = 6.0 / 5.0;
    const double A51 = -11.0 / 54.0, A52 = 5.0 / 2.0, A53 = -70.0 / 27.0, A54 = 35.0 / 27.0;
    const double A61 = 1631.0 / 55296.0, A62 = 175.0 / 512.0, A63 = 575.0 / 13824.0,
                 A64 = 44275.0 / 110592.0, A65 = 253.0 / 4096.0;
    const double B1 = 37.0 / 378.0, B3 = 250.0 / 621.0, B4 = 125.0 / 594.0, B6 = 512.0 / 1771.0;
    const double E1 = B1 - 2825.0 / 27648.0, E3 = B3 - 18575.0 / 48384.0,
                 E4 = B4 - 13525.0 / 55296.0, E5 = -277.0 / 14336.0, E6 = B6 - 1.0 / 4.0;
    double y[7] = {q[0], q[1], q[2], q[3], wb.x, wb.y, wb.z};
    double t = 0.0, dt = h;
    const double dt_min = h * 0x1p-20;
    while (t < h) {
        if (t + dt > h) dt = h - t;
        double k1[7], k2[7], k3[7], k4[7], k5[7], k6[7], z[7];
        rot_rhs(y, I, Iinv, k1);
        for (int c = 0; c < 7; ++c) z[c] = y[c] + dt * (A21 * k1[c]);
        rot_rhs(z, I, Iinv, k2);
        for (int c = 0; c < 7; ++c) z[c] = y[c] + dt * (A31 * k1[c] + A32 * k2[c]);
        rot_rhs(z, I, Iinv, k3);
        for (int c = 0; c < 7; ++c) z[c] = y[c] + dt * (A41 * k1[c] + A42 * k2[c] + A43 * k3[c]);
        rot_rhs(z, I, Iinv, k4);
        for (int c = 0; c < 7; ++c)
            z[c] = y[c] + dt * (A51 * k1[c] + A52 * k2[c] + A53 * k3[c] + A54 * k4[c]);
        rot_rhs(z, I, Iinv, k5);
        for (int c = 0; c < 7; ++c)
            z[c] = y[c] + dt * (A61 * k1[c] + A62 * k2[c] + A63 * k3[c] + A64 * k4[c] + A65 * k5[c]);
        rot_rhs(z, I, Iinv, k6);
        const double wn = sqrt(y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
        double err = 0.0;
        for (int c = 0; c < 7; ++c) {
            double e = fabs(dt * (E1 * k1[c] + E3 * k3[c] + E4 * k4[c] + E5 * k5[c] + E6 * k6[c]));
            if (c >= 4 && wn > 0.0) e /= wn;
            err = fmax(err, e);
        }
        const double ratio = err / tol;
        if (ratio <= 1.0 || dt <= dt_min) {
            for (int c = 0; c < 7; ++c)
                y[c] += dt * (B1 * k1[c] + B3 * k3[c] + B4 * k4[c] + B6 * k6[c]);
            t += dt;
            dt *= ratio > 0.0 ? fmin(5.0, 0.9 * pow(ratio, -0.2)) : 5.0;
        } else {
            dt *= fmax(0.1, 0.9 * pow(ratio, -0.25));
        }
    }
    double n = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
    q[0] = y[0] / n; q[1] = y[1] / n; q[2] = y[2] / n; q[3] = y[3] / n;
    wb = d3(y[4], y[5], y[6]);
}

// ---------------------------------------------------------------- step begin
// Neighbour-list validity.  Every sphere of the aggregate moved, relative to
// the pile frame extrapolated by one step (O + h V), by at most
// |c' - c'_ref| + |(R - R_ref) b| <= |c' - c'_ref| + 2 |b|max min|q -+ q_ref|
// since the last rebuild.  The candidate lists hold every pair closer than the
// radii sum plus the skin at the rebuild, so they stay complete while no
// sphere has moved more than half the skin.  The bound is taken in FP32
// (positions relative to the pile frame, reference stored in FP32) with a
// margin of a few units in the last place of the positions and 1e-4
// relative, far above its rounding.  c: COM relative to the frame (hi parts),
// qn: the new orientation in FP32.
__device__ __forceinline__ void rebuild_test(const Arrays &a, int p, int64_t g, const float (&c)[3],
                                             const float (&qn)[4])
{
    const double skin = a.ps[p].skin;
    if (!(skin > 0.0)) return;
    const float *ar = a.aref + 8 * g;
    const float *hv = a.pd[p].hVf;
    const float3 dcf = f3(c[0] - hv[0] - ar[0], c[1] - hv[1] - ar[1], c[2] - hv[2] - ar[2]);
    float dm = 0.f, dp = 0.f;
    for (int k = 0; k < 4; ++k) {
        const float m = qn[k] - ar[3 + k], s_ = qn[k] + ar[3 + k];
        dm = fmaf(m, m, dm);
        dp = fmaf(s_, s_, dp);
    }
    const float big = fmaxf(fabsf(c[0]), fmaxf(fabsf(c[1]), fabsf(c[2]))) +
                      fmaxf(fabsf(ar[0]), fmaxf(fabsf(ar[1]), fabsf(ar[2])));
    const float disp = sqrtf(dot(dcf, dcf)) + 2.0f * ar[7] * sqrtf(fminf(dm, dp)) + 1e-6f * (big + ar[7]);
    if (!(disp * 1.0001f <= 0.5f * (float)skin)) atomicOr(&a.pd[p].rebuild, 1);
}

// FP64 path.  Per aggregate: half kick of COM and spin with the stored
// a_A,n / N_A,n, drift, torque-free rotation, then the record the sphere
// kernels read: rotation, COM relative to the pile frame, predicted COM
// velocity v_A,n+1/2 + h/2 a_A,n (Eq. pred-vel) and predicted spin w_A,n+1
// (the drifted spin plus the second half kick of the old torque).
template <bool ADAPT>
__device__ __forceinline__ void agg_begin_64(const Arrays &a, int64_t g, int p)
{
    const double h = a.ps[p].h;
    const double *I = a.I + 9 * g, *Iinv = a.Iinv + 9 * g;
    double q[4] = {a.q[4 * g], a.q[4 * g + 1], a.q[4 * g + 2], a.q[4 * g + 3]};
    double3 r = ld3(a.r + 3 * g), v = ld3(a.v + 3 * g), wb = ld3(a.wb + 3 * g);
    const double3 acc = ld3(a.acc + 3 * g), N = ld3(a.torque + 3 * g);
    double R[9];
    quat_to_R(q, R);
    v = v + (0.5 * h) * acc;
    wb = wb + (0.5 * h) * mat_mul(Iinv, mat_tmul(R, N));
    r = r + h * v;
    if (ADAPT && a.ps[p].rot_tol > 0.0) free_rotate_adaptive(q, wb, I, Iinv, h, a.ps[p].rot_tol);
    else free_rotate(q, wb, I, Iinv, h);
    quat_to_R(q, R);
    const double3 wpred_b = wb + (0.5 * h) * mat_mul(Iinv, mat_tmul(R, N));
    const double3 ws = mat_mul(R, wpred_b);
    st3(a.r + 3 * g, r);
    st3(a.v + 3 * g, v);
    st3(a.wb + 3 * g, wb);
    a.q[4 * g] = q[0]; a.q[4 * g + 1] = q[1]; a.q[4 * g + 2] = q[2]; a.q[4 * g + 3] = q[3];
    const PileDyn &D = a.pd[p];
    const double3 c = r - ld3(D.O);
    const double3 vb = v + (0.5 * h) * acc - ld3(D.V);
    const float cf[3] = {(float)c.x, (float)c.y, (float)c.z};
    const float qn[4] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
    rebuild_test(a, p, g, cf, qn);
    AggRec64 rec;
    for (int k = 0; k < 9; ++k) rec.R[k] = R[k];
    st3(rec.c, c);
    st3(rec.vb, vb);
    st3(rec.w, ws);
    a.rec64[g] = rec;
}

// Mixed path: the torque-free RK4 step with the stage derivatives evaluated
// in FP32 (from FP32 copies of q, w and the inertia tensor) and the step's
// increment added to the float-float state; q is then renormalised in
// float-float by the series 1/|q| = 1 - e/2 + 3e^2/8 - ..., e = |q|^2 - 1
// ~ |increment|^2 (the increment is tangent to the unit sphere; the dropped
// terms are O(e^3)).  The increment is O(h |w|), so its FP32 rounding is
// ~1e-7 of the change per step, far below the FP32 error of the forces that
// drive it.
__device__ __forceinline__ void free_rotate_ff(ff (&q)[4], ff (&wb)[3], const float *qf, const float *I,
                                               const float *Iinv, float h)
{
    float y[7] = {qf[0], qf[1], qf[2], qf[3], wb[0].hi, wb[1].hi, wb[2].hi};
    float k1[7], k2[7], k3[7], k4[7], t[7];
    rot_rhs_f(y, I, Iinv, k1);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + 0.5f * h * k1[c];
    rot_rhs_f(t, I, Iinv, k2);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + 0.5f * h * k2[c];
    rot_rhs_f(t, I, Iinv, k3);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + h * k3[c];
    rot_rhs_f(t, I, Iinv, k4);
    float d[7];
    for (int c = 0; c < 7; ++c) d[c] = (h / 6.0f) * (k1[c] + 2.0f * k2[c] + 2.0f * k3[c] + k4[c]);
    for (int c = 0; c < 4; ++c) q[c] = ff_addf(q[c], d[c]);
    ff n2 = ff_mul(q[0], q[0]);
    for (int c = 1; c < 4; ++c) n2 = ff_add(n2, ff_mul(q[c], q[c]));
    const ff em = ff_addf(n2, -1.0f);
    const float e = __fadd_rn(em.hi, em.lo);
    const ff inv = {1.0f, e * (-0.5f + 0.375f * e)};
    for (int c = 0; c < 4; ++c) q[c] = ff_mul(q[c], inv);
    for (int c = 0; c < 3; ++c) wb[c] = ff_addf(wb[c], d[4 + c]);
}

// Mixed path: the same step with the aggregate state in float-float pairs
// and every operation on the FP32 units (no FP64 instruction on this path
// unless the pile asks for the adaptive rotor, which runs in FP64).
template <bool ADAPT>
__device__ __forceinline__ void agg_begin_mixed(const Arrays &a, int64_t g, int p)
{
    const PileStatic &S = a.ps[p];
    const PileDyn &D = a.pd[p];
    const float hf = S.lawf[8];
    const ff hh = {0.5f * S.hff[0], 0.5f * S.hff[1]}, hfull = {S.hff[0], S.hff[1]};
    ff q[4], r[3], v[3], wb[3], acc[3];
    float3 Nf;
    for (int c = 0; c < 4; ++c) q[c] = ldff(a.q + 4 * g + c);
    for (int c = 0; c < 3; ++c) {
        r[c] = ldff(a.r + 3 * g + c);
        v[c] = ldff(a.v + 3 * g + c);
        wb[c] = ldff(a.wb + 3 * g + c);
        acc[c] = ldff(a.acc + 3 * g + c);
    }
    Nf = f3(ldff(a.torque + 3 * g).hi, ldff(a.torque + 3 * g + 1).hi, ldff(a.torque + 3 * g + 2).hi);
    // spin kicks and the rotor's stage derivatives are increments: FP32
    const float *I32 = a.I32 + 9 * g, *Iinv32 = a.Iinv32 + 9 * g;
    float qf[4] = {q[0].hi, q[1].hi, q[2].hi, q[3].hi};
    float Rf[9], Rlo[9];
    quat_to_Rf(qf, Rf);
    const float3 dw = (0.5f * hf) * mat_mulf(Iinv32, mat_tmulf(Rf, Nf));
    for (int c = 0; c < 3; ++c) v[c] = ff_add(v[c], ff_mul(hh, acc[c]));
    wb[0] = ff_addf(wb[0], dw.x); wb[1] = ff_addf(wb[1], dw.y); wb[2] = ff_addf(wb[2], dw.z);
    for (int c = 0; c < 3; ++c) r[c] = ff_add(r[c], ff_mul(hfull, v[c]));
    if (ADAPT && S.rot_tol > 0.0) {
        double qd[4] = {ff_value(q[0]), ff_value(q[1]), ff_value(q[2]), ff_value(q[3])};
        double3 wd = d3(ff_value(wb[0]), ff_value(wb[1]), ff_value(wb[2]));
        free_rotate_adaptive(qd, wd, a.I + 9 * g, a.Iinv + 9 * g, S.h, S.rot_tol);
        for (int c = 0; c < 4; ++c) q[c] = ff_of(qd[c]);
        wb[0] = ff_of(wd.x); wb[1] = ff_of(wd.y); wb[2] = ff_of(wd.z);
    } else {
        free_rotate_ff(q, wb, qf, I32, Iinv32, hf);
    }
    // rotation matrix in float-float from the float-float quaternion
    quat_ff_to_R_ff(q, Rf, Rlo);
    for (int c = 0; c < 4; ++c) qf[c] = q[c].hi;
    const float3 wpred = f3(wb[0].hi, wb[1].hi, wb[2].hi) + (0.5f * hf) * mat_mulf(Iinv32, mat_tmulf(Rf, Nf));
    const float3 wsf = mat_mulf(Rf, wpred);
    for (int c = 0; c < 4; ++c) stff(a.q + 4 * g + c, q[c]);
    for (int c = 0; c < 3; ++c) {
        stff(a.r + 3 * g + c, r[c]);
        stff(a.v + 3 * g + c, v[c]);
        stff(a.wb + 3 * g + c, wb[c]);
    }
    if (!(isfinite(r[0].hi) && isfinite(r[1].hi) && isfinite(r[2].hi)))
        atomicOr(&a.pd[p].flags, DEM_FLAG_NONFINITE);
    ff cc[3];
    float vb[3];
    for (int c = 0; c < 3; ++c) {
        cc[c] = ff_sub(r[c], ff_of2(D.Of[c]));
        vb[c] = ff_sub(ff_add(v[c], ff_mul(hh, acc[c])), ff_of2(D.Vf[c])).hi;
    }
    const float cf[3] = {cc[0].hi, cc[1].hi, cc[2].hi};
    rebuild_test(a, p, g, cf, qf);
    AggRecMixed rec;
    for (int k = 0; k < 9; ++k) { rec.Rh[k] = Rf[k]; rec.Rl[k] = Rlo[k]; }
    for (int c = 0; c < 3; ++c) { rec.ch[c] = cc[c].hi; rec.cl[c] = cc[c].lo; rec.vb[c] = vb[c]; }
    rec.w[0] = wsf.x; rec.w[1] = wsf.y; rec.w[2] = wsf.z;
    rec.pad[0] = rec.pad[1] = 0.f;
    a.rec32[g] = rec;
}

template <bool FP64, bool ADAPT>
__global__ void k_agg_begin(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= z.A) return;
    int p = a.agg_pile[g];
    if (!pile_active(a, p)) return;
    if constexpr (FP64) agg_begin_64<ADAPT>(a, g, p);
    else agg_begin_mixed<ADAPT>(a, g, p);
}

void launch_agg_begin(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st)
{
    if (z.A == 0) return;
    unsigned nb = (unsigned)((z.A + 127) / 128);
    // the adaptive rotor needs many more registers: its variant runs only when
    // some pile asks for it
    if (z.adapt) {
        if (fp64) launch_pdl(k_agg_begin<true, true>, nb, 128, 0, st, a, z);
        else launch_pdl(k_agg_begin<false, true>, nb, 128, 0, st, a, z);
    } else {
        if (fp64) launch_pdl(k_agg_begin<true, false>, nb, 128, 0, st, a, z);
        else launch_pdl(k_agg_begin<false, false>, nb, 128, 0, st, a, z);
    }
}

// ---------------------------------------------------------------- pile reductions
// Block b sums kAggChunk aggregates of one pile.  Mode 0 (after the drift):
// sum M, sum M r, sum M v.  Mode 1 (after the closing kick): sum of the planet
// force on the pile.  The last of a pile's chunk blocks to finish (counted in
// pile_arrive, which it puts back to zero) then adds the pile's chunk sums and
// updates the pile: thread t adds chunks t, t+128, ... in order and
// block_sum7 combines the threads in a fixed order, so the result does not
// depend on which block came last.  Fixed orders throughout: deterministic.
// Without a planet the closing pass has nothing to sum: the pile's first
// chunk block alone updates it.
// Sum of v over the block's 128 threads in a fixed order (each warp by
// shuffles, then the four warp sums in warp order); the result is in
// thread 0.  ws: 4 x 7 scratch doubles.
__device__ __forceinline__ void block_sum7(double (&v)[7], double *ws)
{
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 7; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 7; ++k) ws[7 * wid + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) v[k] = (ws[k] + ws[7 + k]) + (ws[14 + k] + ws[21 + k]);
}

// The same in float-float (mixed path: FP32 units only).
__device__ __forceinline__ void block_sum7(ff (&v)[7], ff *ws)
{
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 7; ++k) {
            const ff t = {__shfl_down_sync(0xffffffffu, v[k].hi, o), __shfl_down_sync(0xffffffffu, v[k].lo, o)};
            v[k] = ff_add(v[k], t);
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 7; ++k) ws[7 * wid + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) v[k] = ff_add(ff_add(ws[k], ws[7 + k]), ff_add(ws[14 + k], ws[21 + k]));
}

template <int MODE>
__device__ void pile_finalize_block(const Arrays &a, int p, double (&sh)[7][128])
{
    const PileStatic &S = a.ps[p];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    if (MODE == 0 || S.ext_mass > 0) {   // the closing pass sums only the planet's reaction
        for (int64_t ch = S.ch0 + threadIdx.x; ch < S.ch0 + S.nch; ch += blockDim.x)
            for (int k = 0; k < 7; ++k) s[k] += __ldcg(a.chunk_part + ch * kPartialDoubles + k);
        __syncthreads();   // sh is free again
        block_sum7(s, &sh[0][0]);
    }
    if (threadIdx.x != 0) return;
    PileDyn &D = a.pd[p];
    const double h = S.h;
    if (MODE == 0) {
        for (int c = 0; c < 3; ++c) {
            D.Rc[c] = s[1 + c] / s[0];
            D.Vc[c] = s[4 + c] / s[0];
            const ff rc = ff_of(D.Rc[c]);
            D.Rcf[c] = make_float2(rc.hi, rc.lo);
        }
        if (S.ext_mass > 0) {   // planet: kick with the stored acceleration, drift
            for (int c = 0; c < 3; ++c) {
                D.P_vel[c] += 0.5 * h * D.P_acc[c];
                D.P_pos[c] += h * D.P_vel[c];
            }
        }
    } else {
        if (S.ext_mass > 0) {   // planet: reaction of the pile, closing kick
            for (int c = 0; c < 3; ++c) {
                D.P_acc[c] = -s[c] / S.ext_mass;
                D.P_vel[c] += 0.5 * h * D.P_acc[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            D.O[c] = D.Rc[c];
            D.V[c] = D.Vc[c];
            D.hVf[c] = (float)(h * D.Vc[c]);
            D.Of[c] = D.Rcf[c];
            const ff vc = ff_of(D.Vc[c]);
            D.Vf[c] = make_float2(vc.hi, vc.lo);
        }
        D.steps += 1;
        D.parity ^= 1;
        if (D.flags & (DEM_FLAG_SLOTS | DEM_FLAG_NONFINITE | DEM_FLAG_GRAV_RANGE)) D.failed = 1;
        if (D.rebuild) {
            D.rebuilds += 1;
            D.cpar ^= 1;   // the lists built this step become the current ones
        }
        D.rebuilt_prev = D.rebuild;
        D.rebuild = S.skin <= 0.0 ? 1 : 0;
    }
}

template <int MODE>
__global__ void __launch_bounds__(128) k_pile_reduce(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t ch = blockIdx.x;
    if (ch >= z.CH) return;
    int p = a.chunk_pile[ch];
    __shared__ double sh[7][128];
    __shared__ int last;
    if (MODE == 1 && !(a.ps[p].ext_mass > 0)) {
        // no planet: nothing to sum, the pile's first chunk block finishes it
        if (ch != a.ps[p].ch0 || !pile_active(a, p)) return;
        pile_finalize_block<MODE>(a, p, sh);
        return;
    }
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    ff accf[7];
    for (int k = 0; k < 7; ++k) accf[k] = ff{0.f, 0.f};
    const bool act = pile_active(a, p);
    if (act) {
        const PileStatic &S = a.ps[p];
        int64_t beg = S.a0 + (ch - S.ch0) * kAggChunk;
        int64_t end = beg + kAggChunk;
        if (end > S.a0 + S.na) end = S.a0 + S.na;
        if (MODE == 0 && a.out_ff) {
            // mixed path: float-float state, M as FP32 (the sums fix the
            // frame origin and velocity, whose exact values do not enter any
            // result: positions and velocities are taken relative to them
            // exactly).  The thread's kAggChunk / 128 aggregates are loaded
            // together, then added in index order.
            constexpr int kPer = kAggChunk / 128;
            static_assert(kAggChunk % 128 == 0, "k_pile_reduce runs 128 threads per chunk");
            const PileDyn &D = a.pd[p];
            float Mf[kPer];
            ff rr[kPer][3], vv[kPer][3];
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int64_t g = beg + threadIdx.x + 128 * t;
                const bool in = g < end;
                Mf[t] = in ? (float)a.M[g] : 0.f;
                for (int c = 0; c < 3; ++c) {
                    rr[t][c] = in ? ldff(a.r + 3 * g + c) : ff{0.f, 0.f};
                    vv[t][c] = in ? ldff(a.v + 3 * g + c) : ff{0.f, 0.f};
                }
            }
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int64_t g = beg + threadIdx.x + 128 * t;
                if (g >= end) break;
                if (D.rebuild) {   // new neighbour-list reference, as the test forms it
                    float *ar = a.aref + 8 * g;
                    for (int c = 0; c < 3; ++c) ar[c] = ff_sub(rr[t][c], ff_of2(D.Of[c])).hi - D.hVf[c];
                    for (int c = 0; c < 4; ++c) ar[3 + c] = ldff(a.q + 4 * g + c).hi;
                }
                accf[0] = ff_addf(accf[0], Mf[t]);
                for (int c = 0; c < 3; ++c) {
                    accf[1 + c] = ff_add(accf[1 + c], ff_mul(ff{Mf[t], 0.f}, rr[t][c]));
                    accf[4 + c] = ff_add(accf[4 + c], ff_mul(ff{Mf[t], 0.f}, vv[t][c]));
                }
            }
        } else
        for (int64_t g = beg + threadIdx.x; g < end; g += blockDim.x) {
            if (MODE == 0) {
                if (a.pd[p].rebuild) {   // new neighbour-list reference
                    const PileDyn &D = a.pd[p];
                    float *ar = a.aref + 8 * g;
                    for (int c = 0; c < 3; ++c) ar[c] = (float)(a.r[3 * g + c] - D.O[c] - S.h * D.V[c]);
                    for (int c = 0; c < 4; ++c) ar[3 + c] = (float)a.q[4 * g + c];
                }
                double M = a.M[g];
                acc[0] += M;
                for (int c = 0; c < 3; ++c) {
                    acc[1 + c] += M * a.r[3 * g + c];
                    acc[4 + c] += M * a.v[3 * g + c];
                }
            } else if (a.out_ff) {   // mixed path: the parts are float-float pairs
                const float2 *o32 = (const float2 *)(a.out[2] + 6 * g);
                for (int c = 0; c < 3; ++c) accf[c] = ff_add(accf[c], ff_of2(o32[c]));
            } else {
                for (int c = 0; c < 3; ++c) acc[c] += a.out[2][6 * g + c];
            }
        }
    }
    if (a.out_ff) {
        // mixed path: the block's sum in float-float on the FP32 units (the
        // FP64 units of this part are ~75 times slower), one conversion
        block_sum7(accf, reinterpret_cast<ff *>(&sh[0][0]));
        if (threadIdx.x == 0)
            for (int k = 0; k < 7; ++k) acc[k] = ff_value(accf[k]);
    } else {
        block_sum7(acc, &sh[0][0]);
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 7; ++k) a.chunk_part[ch * kPartialDoubles + k] = acc[k];
        __threadfence();   // the sums are visible before this block is counted
        last = atomicAdd(a.pile_arrive + p, 1) == (int)a.ps[p].nch - 1;
        if (last) a.pile_arrive[p] = 0;
    }
    __syncthreads();
    if (!last || !act) return;
    __threadfence();
    pile_finalize_block<MODE>(a, p, sh);
}

void launch_pile_begin(const Arrays &a, const Sizes &z, cudaStream_t st)
{
    if (z.CH == 0) return;
    launch_pdl(k_pile_reduce<0>, (unsigned)z.CH, 128, 0, st, a, z);
}

void launch_pile_end(const Arrays &a, const Sizes &z, cudaStream_t st)
{
    if (z.CH == 0) return;
    launch_pdl(k_pile_reduce<1>, (unsigned)z.CH, 128, 0, st, a, z);
}

// ---------------------------------------------------------------- expansion
// Sphere centre relative to the pile frame, r_i - O = (r_A - O) + R(q_A) b_i.
// Mixed: float-float, bitwise identical wherever it is inlined.
__device__ __forceinline__ void expand_mixed(const AggRecMixed &rec, float4 bh, float4 bl,
                                             ff &px, ff &py, ff &pz)
{
    ff rx = ff_dot3(rec.Rh + 0, rec.Rl + 0, bh.x, bh.y, bh.z, bl.x, bl.y, bl.z);
    ff ry = ff_dot3(rec.Rh + 3, rec.Rl + 3, bh.x, bh.y, bh.z, bl.x, bl.y, bl.z);
    ff rz = ff_dot3(rec.Rh + 6, rec.Rl + 6, bh.x, bh.y, bh.z, bl.x, bl.y, bl.z);
    ff cx = {rec.ch[0], rec.cl[0]}, cy = {rec.ch[1], rec.cl[1]}, cz = {rec.ch[2], rec.cl[2]};
    px = ff_add(cx, rx);
    py = ff_add(cy, ry);
    pz = ff_add(cz, rz);
}

__device__ __forceinline__ double3 expand_64(const AggRec64 &rec, const double *b)
{
    const double *R = rec.R;
    double x = __fma_rn(R[2], b[2], __fma_rn(R[1], b[1], __dmul_rn(R[0], b[0])));
    double y = __fma_rn(R[5], b[2], __fma_rn(R[4], b[1], __dmul_rn(R[3], b[0])));
    double zz = __fma_rn(R[8], b[2], __fma_rn(R[7], b[1], __dmul_rn(R[6], b[0])));
    return d3(__dadd_rn(rec.c[0], x), __dadd_rn(rec.c[1], y), __dadd_rn(rec.c[2], zz));
}

__device__ __forceinline__ int wrap_cell(int c, int n)
{
    int m = c % n;
    return m < 0 ? m + n : m;
}

__device__ __forceinline__ int cell_coord_f(float x, float inv_cell, int n)
{
    float f = floorf(__fmul_rn(x, inv_cell));
    f = fminf(fmaxf(f, -1.0e9f), 1.0e9f);
    return wrap_cell((int)f, n);
}

__device__ __forceinline__ int cell_coord_d(double x, double inv_cell, int n)
{
    double f = floor(__dmul_rn(x, inv_cell));
    f = fmin(fmax(f, -1.0e9), 1.0e9);
    return wrap_cell((int)f, n);
}

// Per sphere (home order): expand, cell key, atomic count into the cell (the
// returned rank is made deterministic later by ordering each cell), gravity
// input (position relative to the pile frame, mass).  A pile without
// self-gravity needs no gravity input: in its steps without a rebuild there
// is nothing to do.
template <bool FP64>
__global__ void k_keys(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.N) return;
    int p = a.sph_pile[i];
    if (!pile_active(a, p)) return;
    const PileStatic &S = a.ps[p];
    const bool grav = S.G != 0.0;
    if (!grav && !a.pd[p].rebuild) return;
    int64_t g = S.a0 + a.sph_agg[i];
    int cx, cy, cz;
    if (FP64) {
        double3 pos = expand_64(a.rec64[g], a.b64 + 3 * i);
        cx = cell_coord_d(pos.x, S.inv_cell, S.nx);
        cy = cell_coord_d(pos.y, S.inv_cell, S.ny);
        cz = cell_coord_d(pos.z, S.inv_cell, S.nz);
        if (grav) a.gpos64[i] = make_dbl4(pos.x, pos.y, pos.z, a.m64[i]);
    } else {
        ff px, py, pz;
        expand_mixed(a.rec32[g], a.bh[i], a.bl[i], px, py, pz);
        float ic = (float)S.inv_cell;
        cx = cell_coord_f(px.hi, ic, S.nx);
        cy = cell_coord_f(py.hi, ic, S.ny);
        cz = cell_coord_f(pz.hi, ic, S.nz);
        if (grav) a.gpos32[i] = make_float4(px.hi, py.hi, pz.hi, (float)a.m64[i]);
    }
    if (!a.pd[p].rebuild) return;   // cell list kept from the last rebuild
    const int key = (int)cell_id(cx, cy, cz, S.nx, S.ny);
    a.key[i] = key;
    a.rank[i] = atomicAdd(a.ccount + S.c0 + key, 1);
}

__device__ int tile_pile(const Arrays &a, const Sizes &z, int64_t t);

// Zero the cell counts of the piles that rebuild this step.
__global__ void k_clear_cells(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= z.C) return;
    int p = tile_pile(a, z, c / kScanTile);
    if (pile_active(a, p) && a.pd[p].rebuild) a.ccount[c] = 0;
}

void launch_keys(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st)
{
    if (z.N == 0) return;
    launch_pdl(k_clear_cells, (unsigned)((z.C + 255) / 256), 256, 0, st, a, z);
    unsigned nb = (unsigned)((z.N + 255) / 256);
    if (fp64) launch_pdl(k_keys<true>, nb, 256, 0, st, a, z);
    else launch_pdl(k_keys<false>, nb, 256, 0, st, a, z);
}

// Host request (after a state write or a new layout): the next step rebuilds
// the cell list and hit lists of pile `slot` (all piles for slot < 0).
__global__ void k_force_rebuild(Arrays a, Sizes z, int slot)
{
    pdl_enter();
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= z.P || (slot >= 0 && p != slot)) return;
    a.pd[p].rebuild = 1;
}

void set_launch_pdl(int64_t n_spheres) { tl_pdl = n_spheres <= kPdlMaxSpheres; }

void launch_force_rebuild(const Arrays &a, const Sizes &z, int slot, cudaStream_t st)
{
    if (z.P == 0) return;
    launch_pdl(k_force_rebuild, (unsigned)((z.P + 127) / 128), 128, 0, st, a, z, slot);
}

// ---------------------------------------------------------------- scan of cell counts
// Tiles of kScanTile cells never straddle piles (cell ranges are padded).
__device__ int tile_pile(const Arrays &a, const Sizes &z, int64_t t)
{
    int lo = 0, hi = (int)z.P - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.ps[mid].t0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_scan_tiles(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t t = blockIdx.x;
    int p = tile_pile(a, z, t);
    if (!pile_active(a, p) || !a.pd[p].rebuild) return;
    const int32_t *c = a.ccount + t * kScanTile;
    int s = 0;
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) s += c[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ int ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += ws[k];
        a.tile_sum[t] = tot;
    }
}

// One block per pile: exclusive scan of its tile sums (in place).
__global__ void k_scan_piles(Arrays a, Sizes z)
{
    pdl_enter();
    int p = blockIdx.x;
    if (!pile_active(a, p) || !a.pd[p].rebuild) return;
    const PileStatic &S = a.ps[p];
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < S.nt; base += 1024) {
        int64_t t = base + threadIdx.x;
        int v = t < S.nt ? a.tile_sum[S.t0 + t] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int add = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += add;
            __syncthreads();
        }
        int incl = buf[threadIdx.x];
        if (t < S.nt) a.tile_sum[S.t0 + t] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
}

// One block (256 threads x 8 cells) per tile: exclusive scan plus tile offset.
__global__ void k_scan_cells(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t t = blockIdx.x;
    int p = tile_pile(a, z, t);
    if (!pile_active(a, p) || !a.pd[p].rebuild) return;
    const int32_t *c = a.ccount + t * kScanTile;
    int32_t *o = a.cstart + t * kScanTile;
    int v[8];
    int loc = 0;
    for (int k = 0; k < 8; ++k) {
        v[k] = c[threadIdx.x * 8 + k];
        loc += v[k];
    }
    __shared__ int buf[256];
    buf[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        int add = threadIdx.x >= (unsigned)off ? buf[threadIdx.x - off] : 0;
        __syncthreads();
        buf[threadIdx.x] += add;
        __syncthreads();
    }
    int run = a.tile_sum[t] + buf[threadIdx.x] - loc;
    for (int k = 0; k < 8; ++k) {
        o[threadIdx.x * 8 + k] = run;
        run += v[k];
    }
}

void launch_scan(const Arrays &a, const Sizes &z, cudaStream_t st)
{
    if (z.T == 0) return;
    launch_pdl(k_scan_tiles, (unsigned)z.T, 256, 0, st, a, z);
    launch_pdl(k_scan_piles, (unsigned)z.P, 1024, 0, st, a, z);
    launch_pdl(k_scan_cells, (unsigned)z.T, 256, 0, st, a, z);
}

// ---------------------------------------------------------------- scatter and cell order
__global__ void k_scatter(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.N) return;
    int p = a.sph_pile[i];
    if (!pile_active(a, p) || !a.pd[p].rebuild) return;
    const PileStatic &S = a.ps[p];
    int slot = a.cstart[S.c0 + a.key[i]] + a.rank[i];
    a.sorted[S.s0 + slot] = (int32_t)(i - S.s0);
}

void launch_scatter(const Arrays &a, const Sizes &z, cudaStream_t st)
{
    if (z.N == 0) return;
    launch_pdl(k_scatter, (unsigned)((z.N + 255) / 256), 256, 0, st, a, z);
}

// The thread at the first position of each cell sorts that cell's entries by
// home index (insertion sort; cells hold a handful of spheres), which makes
// the order of neighbours, and so every contact sum, deterministic.
__global__ void k_cell_order(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z.N) return;
    int p = a.sph_pile[k];
    if (!pile_active(a, p) || !a.pd[p].rebuild) return;
    const PileStatic &S = a.ps[p];
    int32_t *srt = a.sorted + S.s0;
    int kl = (int)(k - S.s0);
    int key = a.key[S.s0 + srt[kl]];
    int start = a.cstart[S.c0 + key];
    if (kl != start) return;
    int n = a.ccount[S.c0 + key];
    for (int x = 1; x < n; ++x) {
        int v = srt[start + x];
        int y = x - 1;
        while (y >= 0 && srt[start + y] > v) {
            srt[start + y + 1] = srt[start + y];
            --y;
        }
        srt[start + y + 1] = v;
    }
}

void launch_cell_order(const Arrays &a, const Sizes &z, cudaStream_t st)
{
    if (z.N == 0) return;
    launch_pdl(k_cell_order, (unsigned)((z.N + 255) / 256), 256, 0, st, a, z);
}

// ---------------------------------------------------------------- gather
// Sorted copies for the contact pass: position (float-float in mixed), predicted
// velocity v_i = [v_A + h/2 a_A] + w_A x (r_i - r_A) (Eq. pred-vel), spin, ids.
template <bool FP64>
__global__ void k_gather(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z.N) return;
    int p = a.sph_pile[k];
    if (!pile_active(a, p)) return;
    const PileStatic &S = a.ps[p];
    int hl = a.sorted[k];
    int64_t i = S.s0 + hl;
    // the sorted order changes only at rebuilds: the sorted aggregate ids are
    // written in a rebuild step (and read here otherwise); the home -> sorted
    // map, which k_cand_link reads at the next rebuild to find each sphere's
    // previous list, is double-buffered by parity and written in a rebuild
    // step and the step after it
    const PileDyn &D = a.pd[p];
    const bool fresh = D.rebuild != 0, refresh = fresh || D.rebuilt_prev != 0;
    const int al = fresh ? a.sph_agg[i] : a.sagg[k];
    int64_t g = S.a0 + al;
    if (refresh) a.pos_of_home[D.parity ^ 1][i] = (int32_t)(k - S.s0);
    if (fresh) a.sagg[k] = al;
    if (FP64) {
        const AggRec64 &rec = a.rec64[g];
        const double *b = a.b64 + 3 * i;
        double3 pos = expand_64(rec, b);
        double3 rb = mat_mul(rec.R, d3(b[0], b[1], b[2]));
        double3 w = ld3(rec.w);
        double3 v = ld3(rec.vb) + cross(w, rb);
        a.dp_[k] = make_dbl4(pos.x, pos.y, pos.z, a.s64[i]);
        a.dv_[k] = make_dbl4(v.x, v.y, v.z, (double)al);
        a.dw_[k] = make_dbl4(w.x, w.y, w.z, (double)hl);
    } else {
        const AggRecMixed &rec = a.rec32[g];
        float4 bh = a.bh[i], bl = a.bl[i];
        ff px, py, pz;
        expand_mixed(rec, bh, bl, px, py, pz);
        float3 rb = f3(rec.Rh[0] * bh.x + rec.Rh[1] * bh.y + rec.Rh[2] * bh.z,
                       rec.Rh[3] * bh.x + rec.Rh[4] * bh.y + rec.Rh[5] * bh.z,
                       rec.Rh[6] * bh.x + rec.Rh[7] * bh.y + rec.Rh[8] * bh.z);
        float3 w = f3(rec.w[0], rec.w[1], rec.w[2]);
        float3 v = f3(rec.vb[0], rec.vb[1], rec.vb[2]) + cross(w, rb);
        // fixed point in quanta q = 2^qexp: low 32 bits of round((r_i - O) / q)
        // per axis (differences of nearby spheres are exact int32) and
        // round(radius / q), with what the rounding left in FP32
        const int e = -S.qexp;
        float4 rm;
        const int X = ff_to_fixed(px, e, rm.x), Y = ff_to_fixed(py, e, rm.y), Z = ff_to_fixed(pz, e, rm.z);
        const int Sr = ff_to_fixed(ff{bh.w, bl.w}, e, rm.w);
        a.xqr[2 * k] = make_int4(X, Y, Z, Sr);
        a.xqr[2 * k + 1] = make_int4(__float_as_int(rm.x), __float_as_int(rm.y), __float_as_int(rm.z),
                                     __float_as_int(rm.w));
        if (fresh) a.sph_[k] = make_float4(px.hi, py.hi, pz.hi, bh.w);
        a.svw[2 * k] = make_float4(v.x, v.y, v.z, __int_as_float(al));
        a.svw[2 * k + 1] = make_float4(w.x, w.y, w.z, __int_as_float(hl));
    }
}

void launch_gather(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st)
{
    if (z.N == 0) return;
    unsigned nb = (unsigned)((z.N + 255) / 256);
    if (fp64) launch_pdl(k_gather<true>, nb, 256, 0, st, a, z);
    else launch_pdl(k_gather<false>, nb, 256, 0, st, a, z);
}

// ---------------------------------------------------------------- step end
// Per aggregate: F_A = sum_i (F_c,i + F_g,i + F_e,i) and
// N_A = sum_i [(r_i - r_A) x F_i + tau_i], kept separately for contact,
// gravity and planet; a_A = F_A / M; closing half kick of COM and spin; YORP
// increment dw: v_A += dw x (r_A - R_pile), w_A += dw (rigid rotation of the
// whole pile).  Members are contiguous (spheres stored in aggregate order).
// GRAV = false: no pile of the world has self-gravity (the gravity sums are
// left out, and with them their registers).
template <bool FP64, bool GRAV>
__global__ void __launch_bounds__(128) k_agg_end(Arrays a, Sizes z)
{
    pdl_enter();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= z.A) return;
    int p = a.agg_pile[g];
    if (!pile_active(a, p)) return;
    const PileStatic &S = a.ps[p];
    const PileDyn &D = a.pd[p];
    const double h = S.h;
    int64_t i0 = S.s0 + a.agg_first[g];
    int n = a.agg_count[g];
    double3 Fc, Nc, Fg, Ng;
    double3 Fe = d3(0, 0, 0), Ne = d3(0, 0, 0);
    const bool planet = S.ext_mass > 0;
    double3 Pp = planet ? ld3(D.P_pos) : d3(0, 0, 0);
    double3 O = ld3(D.O);
    if constexpr (FP64) {
        Fc = Nc = Fg = Ng = d3(0, 0, 0);
        const AggRec64 &rec = a.rec64[g];
        for (int t = 0; t < n; ++t) {
            int64_t i = i0 + t;
            const double *b = a.b64 + 3 * i;
            const double3 lever = mat_mul(rec.R, d3(b[0], b[1], b[2]));
            const dbl4 f = a.ftc64[2 * i], tq = a.ftc64[2 * i + 1];
            const double3 fc = d3(f.x, f.y, f.z), tc = d3(tq.x, tq.y, tq.z);
            const dbl4 gg = GRAV ? a.fg[i] : make_dbl4(0.0, 0.0, 0.0, 0.0);
            const double3 fg = d3(gg.x, gg.y, gg.z);
            Fc = Fc + fc;
            Nc = Nc + cross(lever, fc) + tc;
            Fg = Fg + fg;
            Ng = Ng + cross(lever, fg);
            if (planet) {
                const double3 d = Pp - (O + expand_64(rec, b));
                const double inv = 1.0 / sqrt(dot(d, d));
                const double3 fe = (S.G * S.ext_mass * a.m64[i] * inv * inv * inv) * d;
                Fe = Fe + fe;
                Ne = Ne + cross(lever, fe);
            }
        }
    } else {
        // per-sphere terms in FP32 (their inputs are FP32), sums float-float
        FFSum s[12];
        const AggRecMixed &rec = a.rec32[g];
        float Rh[9];
        for (int k = 0; k < 9; ++k) Rh[k] = rec.Rh[k];
        // members in order (without self-gravity the gravity sums stay zero)
        auto term = [&](float4 bh, float4 f, float4 tq, dbl4 gg) {
            const float3 lever = mat_mulf(Rh, f3(bh.x, bh.y, bh.z));
            const float3 fc = f3(f.x, f.y, f.z);
            const float3 nc = cross(lever, fc) + f3(tq.x, tq.y, tq.z);
            s[0].add(fc.x); s[1].add(fc.y); s[2].add(fc.z);
            s[3].add(nc.x); s[4].add(nc.y); s[5].add(nc.z);
            if (GRAV) {
                const float3 fg = f3((float)gg.x, (float)gg.y, (float)gg.z);
                const float3 ng = cross(lever, fg);
                s[6].add(fg.x); s[7].add(fg.y); s[8].add(fg.z);
                s[9].add(ng.x); s[10].add(ng.y); s[11].add(ng.z);
            }
        };
        // a pile without self-gravity has zero sphere gravity: not read
        const bool grav = GRAV && S.G != 0.0;
        const dbl4 g0 = make_dbl4(0.0, 0.0, 0.0, 0.0);
        auto gravity_of = [&](int64_t i) -> dbl4 { return grav ? a.fg[i] : g0; };
        int t2 = 0;
        if (!planet) {   // the loads of two members issued together
            for (; t2 + 1 < n; t2 += 2) {
                const int64_t i = i0 + t2;
                const float4 bha = a.bh[i], bhb = a.bh[i + 1];
                float4 fa, ta, fb, tb;
                ld_f4x2(a.ftc32 + 2 * i, fa, ta);
                ld_f4x2(a.ftc32 + 2 * i + 2, fb, tb);
                const dbl4 ga = gravity_of(i), gb = gravity_of(i + 1);
                term(bha, fa, ta, ga);
                term(bhb, fb, tb, gb);
            }
        }
        for (int t = t2; t < n; ++t) {
            int64_t i = i0 + t;
            const float4 bh = a.bh[i];
            float4 fc, tc;
            ld_f4x2(a.ftc32 + 2 * i, fc, tc);
            term(bh, fc, tc, gravity_of(i));
            if (planet) {
                const float3 lever = mat_mulf(Rh, f3(bh.x, bh.y, bh.z));
                ff px, py, pz;
                expand_mixed(rec, bh, a.bl[i], px, py, pz);
                const double3 pos = O + d3((double)px.hi + (double)px.lo, (double)py.hi + (double)py.lo,
                                           (double)pz.hi + (double)pz.lo);
                const double3 d = Pp - pos;
                const double inv = 1.0 / sqrt(dot(d, d));
                const double3 fe = (S.G * S.ext_mass * a.m64[i] * inv * inv * inv) * d;
                const double3 lv = d3(lever.x, lever.y, lever.z);
                Fe = Fe + fe;
                Ne = Ne + cross(lv, fe);
            }
        }
        // the parts as float-float pairs (readout only), the totals formed in
        // float-float and converted once (FP64 instructions are ~60 times
        // slower than FP32 ones here)
        ff part[18];
        for (int k = 0; k < 12; ++k) part[k] = ff{s[k].hi, s[k].lo};
        if (planet) {
            part[12] = ff_of(Fe.x); part[13] = ff_of(Fe.y); part[14] = ff_of(Fe.z);
            part[15] = ff_of(Ne.x); part[16] = ff_of(Ne.y); part[17] = ff_of(Ne.z);
        } else {
            for (int k = 12; k < 18; ++k) part[k] = ff{0.f, 0.f};
        }
        // the gravity and planet parts of a pile without them stay zero (as
        // set when the pile was added): not rewritten
        for (int k = 0; k < 18; ++k)
            if (k < 6 || (k < 12 && grav) || (k >= 12 && planet))
                reinterpret_cast<float2 *>(a.out[k / 6] + 6 * g)[k % 6] = make_float2(part[k].hi, part[k].lo);
        // totals, a_A = F_A / M and the closing kick in float-float (the
        // state is float-float pairs: no FP64 instruction here)
        const ff hh = {0.5f * S.hff[0], 0.5f * S.hff[1]};
        const ff iM = ldff(a.invM + g);
        ff Ft[3], Nt[3], accf[3], v[3], wb[3];
        for (int c = 0; c < 3; ++c) {
            Ft[c] = ff_add(ff_add(part[c], part[6 + c]), part[12 + c]);
            Nt[c] = ff_add(ff_add(part[3 + c], part[9 + c]), part[15 + c]);
            accf[c] = ff_mul(Ft[c], iM);
            v[c] = ff_add(ldff(a.v + 3 * g + c), ff_mul(hh, accf[c]));
            wb[c] = ldff(a.wb + 3 * g + c);
        }
        // closing spin kick: an increment, FP32, with the step's rotation
        // matrix (the record's FP32 part)
        const float3 Nf = f3(Nt[0].hi, Nt[1].hi, Nt[2].hi);
        const float3 dw = (0.5f * S.lawf[8]) * mat_mulf(a.Iinv32 + 9 * g, mat_tmulf(Rh, Nf));
        wb[0] = ff_addf(wb[0], dw.x); wb[1] = ff_addf(wb[1], dw.y); wb[2] = ff_addf(wb[2], dw.z);
        if (S.yorp) {   // rigid-rotation increment of the whole pile: increments in FP32
            const float3 dwy = f3(S.spin_f[0], S.spin_f[1], S.spin_f[2]);
            const float3 lev = f3(ff_sub(ldff(a.r + 3 * g), ff_of2(D.Rcf[0])).hi,
                                  ff_sub(ldff(a.r + 3 * g + 1), ff_of2(D.Rcf[1])).hi,
                                  ff_sub(ldff(a.r + 3 * g + 2), ff_of2(D.Rcf[2])).hi);
            const float3 dv = cross(dwy, lev), dwb = mat_tmulf(Rh, dwy);
            v[0] = ff_addf(v[0], dv.x); v[1] = ff_addf(v[1], dv.y); v[2] = ff_addf(v[2], dv.z);
            wb[0] = ff_addf(wb[0], dwb.x); wb[1] = ff_addf(wb[1], dwb.y); wb[2] = ff_addf(wb[2], dwb.z);
        }
        bool fin = true;
        for (int c = 0; c < 3; ++c) {
            stff(a.acc + 3 * g + c, accf[c]);
            stff(a.torque + 3 * g + c, Nt[c]);
            stff(a.v + 3 * g + c, v[c]);
            stff(a.wb + 3 * g + c, wb[c]);
            fin = fin && isfinite(v[c].hi) && isfinite(wb[c].hi) && isfinite(Nt[c].hi);
        }
        if (!fin) atomicOr(&a.pd[p].flags, DEM_FLAG_NONFINITE);
    }
    if constexpr (FP64) {
        st3(a.out[0] + 6 * g, Fc); st3(a.out[0] + 6 * g + 3, Nc);
        st3(a.out[1] + 6 * g, Fg); st3(a.out[1] + 6 * g + 3, Ng);
        st3(a.out[2] + 6 * g, Fe); st3(a.out[2] + 6 * g + 3, Ne);
        const double3 F = Fc + Fg + Fe, N = Nc + Ng + Ne;
        const double3 acc = a.invM[g] * F;
        const double q[4] = {a.q[4 * g], a.q[4 * g + 1], a.q[4 * g + 2], a.q[4 * g + 3]};
        double3 v = ld3(a.v + 3 * g) + (0.5 * h) * acc;
        double3 wb = ld3(a.wb + 3 * g);
        const double3 dwy = ld3(S.spin_inc);
        double R[9];
        quat_to_R(q, R);
        wb = wb + (0.5 * h) * mat_mul(a.Iinv + 9 * g, mat_tmul(R, N));
        if (dwy.x != 0.0 || dwy.y != 0.0 || dwy.z != 0.0) {
            v = v + cross(dwy, ld3(a.r + 3 * g) - ld3(D.Rc));
            wb = wb + mat_tmul(R, dwy);
        }
        st3(a.acc + 3 * g, acc);
        st3(a.torque + 3 * g, N);
        st3(a.v + 3 * g, v);
        st3(a.wb + 3 * g, wb);
        if (!finite3(v) || !finite3(wb) || !finite3(N) || !finite3(ld3(a.r + 3 * g)))
            atomicOr(&a.pd[p].flags, DEM_FLAG_NONFINITE);
    }
}

void launch_agg_end(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st)
{
    if (z.A == 0) return;
    unsigned nb = (unsigned)((z.A + 127) / 128);
    if (fp64) {
        if (z.grav) launch_pdl(k_agg_end<true, true>, nb, 128, 0, st, a, z);
        else launch_pdl(k_agg_end<true, false>, nb, 128, 0, st, a, z);
    } else {
        if (z.grav) launch_pdl(k_agg_end<false, true>, nb, 128, 0, st, a, z);
        else launch_pdl(k_agg_end<false, false>, nb, 128, 0, st, a, z);
    }
}

}  // namespace dem
