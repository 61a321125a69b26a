/*
 * dem_oracle.c -- plain FP64 CPU oracle for bonded-sphere aggregates in
 * soft-sphere DEM with self-gravity (Marohnic et al., arXiv 2311.11322).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library
 * against a slow, obviously correct restatement of the method.  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is double precision.  Pair search is brute force O(N^2);
 * gravity is a plain O(N^2) double loop.  OpenMP only splits independent
 * rows; every sum that feeds a result is taken in one fixed serial order.
 *
 * Citations are to sections and equations of the paper:
 *   Sec. 2.1    spring-dashpot SSDEM contacts, fixed-step leapfrog with
 *               predicted velocities;
 *   Sec. 2.2.1  Eq. (agg_mass), Eq. (agg_position);
 *   Sec. 2.2.2  Eq. (pred-vel), the predicted particle velocity;
 *   Sec. 2.2.3  Eq. (particle_gravity), Eq. (agg_gravity), Eq. (gravity_torque);
 *   Sec. 2.2.4  Eq. (agg_contact_accel), Eq. (lever_arm), the contact torque;
 *   Sec. 2.2.5  rolling and twisting friction;
 *   Sec. 4.1    YORP spin-up by a constant per-step increment;
 *   Sec. 4.2    tidal encounter with a point-mass planet.
 * Where the paper defers to work that is not reproduced in it (the force-law
 * constants, the rotation integrator, the rolling law), the reading adopted
 * is stated beside the code that implements it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* parameters                                                          */
/* ------------------------------------------------------------------ */
typedef struct {
    double G;          /* gravitational constant */
    double dt;         /* fixed step h */
    double kn, kt;     /* normal / tangential spring constants */
    double cn, ct;     /* normal / tangential dashpot constants */
    double mu_s;       /* static (= dynamic) friction coefficient */
    double mu_r;       /* rolling friction coefficient */
    double mu_t;       /* twisting friction coefficient */
    double w0;         /* rolling/twisting regularisation rate (rad/s) */
    double eps;        /* Plummer softening length */
    double ext_mass;   /* planet mass, 0 = no planet */
    double spin_inc[3];/* YORP spin increment per step (rad/s, space frame) */
    double rot_tol;    /* 0: one classical RK4 step per rotation; > 0: adaptive
                          embedded RK5(4) (Cash-Karp) to this tolerance */
} ora_params;

/* One rubble pile.  Arrays are owned by the caller. */
typedef struct {
    int64_t n_agg, n_sph;
    int32_t hcap;               /* history capacity per sphere (canonical owner) */
    /* aggregates */
    const int32_t *first, *count;
    const double *M, *I, *Iinv; /* I, Iinv: 9 per aggregate, row major */
    double *r, *v, *q, *wb;     /* 3, 3, 4 (w,x,y,z), 3 (body-frame spin) */
    double *acc, *torque;       /* stored a_A,n and N_A,n (space frame), 3 each */
    /* spheres */
    const int32_t *agg_of;
    const double *m, *s, *b;    /* mass, radius, body offset (3) */
    /* contact history, canonical owner = lower sphere index */
    int32_t *h_n, *h_partner;   /* [n_sph], [n_sph*hcap] */
    double *h_S;                /* [n_sph*hcap*3] */
    /* per-sphere results of the last force evaluation */
    double *sph_pos, *sph_vel, *sph_w;   /* 3 each */
    double *Fc, *Tc, *Fg, *Fe;           /* 3 each */
    /* per-aggregate results of the last force evaluation */
    double *FA_c, *NA_c, *FA_g, *NA_g, *FA_e, *NA_e;   /* 3 each */
    /* planet state: pos[3], vel[3], acc[3] */
    double *planet;
    /* optional: condition scales (sum of magnitudes of summed terms) */
    double *scaleF, *scaleN;    /* per aggregate, may be NULL */
    /* optional: pair list of the last contact evaluation (i, j) and overlap */
    int32_t *pairs; double *pair_x; int64_t pair_cap; int64_t n_pairs;
    /* optional per-sphere scales: contact |F| sum, contact torque-term sum,
       gravity |F_ij| sum */
    double *sph_Fmc, *sph_Tmc, *sph_Fmg;
} ora_sim;

int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* small vector helpers (FP64)                                         */
/* ------------------------------------------------------------------ */
static void v_cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double v_dot(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static double v_norm(const double a[3]) { return sqrt(v_dot(a, a)); }

static void mat_vec(const double A[9], const double x[3], double y[3])
{
    for (int r = 0; r < 3; ++r)
        y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}
static void mat_tvec(const double A[9], const double x[3], double y[3])
{
    for (int c = 0; c < 3; ++c)
        y[c] = A[c] * x[0] + A[3 + c] * x[1] + A[6 + c] * x[2];
}

/* Rotation matrix (body -> space) of the unit quaternion q = (w, x, y, z). */
void ora_rotmat(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------ */
/* aggregate construction                                              */
/* ------------------------------------------------------------------ */
/*
 * Sec. 2.2.1: M = sum m_i (Eq. agg_mass), r_A = sum m_i r_i / M
 * (Eq. agg_position).  Sphere mass m = rho * 4/3 pi s^3.  The inertia tensor
 * about the COM is sum [ 2/5 m s^2 1 + m (|b|^2 1 - b b^T) ] with b = r_i - r_A
 * (touching spheres: no overlap volume is removed).  The body frame is the
 * space frame at creation (q = identity), so body offsets are b_i = r_i - r_A
 * and the full tensor is kept (no diagonalisation).
 * Returns 0, or -1 on invalid input, -2 on a singular inertia tensor.
 */
int ora_build(int64_t n_agg, const int32_t *count, const double *pos,
              const double *radius, const double *density,
              int32_t *first, int32_t *agg_of, double *m, double *b,
              double *M, double *com, double *I, double *Iinv)
{
    int64_t k = 0;
    for (int64_t a = 0; a < n_agg; ++a) {
        if (count[a] <= 0) return -1;
        first[a] = (int32_t)k;
        /* Eq. agg_position, the mass-weighted mean, taken about the first
         * member: a one-sphere aggregate then has its COM exactly at the
         * sphere and a zero offset. */
        double Ma = 0, c[3] = {0, 0, 0}, x0[3];
        for (int d = 0; d < 3; ++d) x0[d] = pos[3 * k + d];
        for (int32_t t = 0; t < count[a]; ++t, ++k) {
            double s = radius[k], rho = density[k];
            if (!(s > 0) || !(rho > 0) || !isfinite(s) || !isfinite(rho)) return -1;
            for (int d = 0; d < 3; ++d) if (!isfinite(pos[3 * k + d])) return -1;
            m[k] = rho * 4.0 / 3.0 * M_PI * s * s * s;
            agg_of[k] = (int32_t)a;
            Ma += m[k];
            for (int d = 0; d < 3; ++d) c[d] += m[k] * (pos[3 * k + d] - x0[d]);
        }
        for (int d = 0; d < 3; ++d) c[d] = x0[d] + c[d] / Ma;
        M[a] = Ma;
        for (int d = 0; d < 3; ++d) com[3 * a + d] = c[d];
        double T[9] = {0};
        for (int64_t i = first[a]; i < first[a] + count[a]; ++i) {
            double bi[3];
            for (int d = 0; d < 3; ++d) { bi[d] = pos[3 * i + d] - c[d]; b[3 * i + d] = bi[d]; }
            double bb = v_dot(bi, bi), sph = 0.4 * m[i] * radius[i] * radius[i];
            for (int r = 0; r < 3; ++r)
                for (int cc = 0; cc < 3; ++cc)
                    T[3 * r + cc] += (r == cc ? sph + m[i] * bb : 0.0) - m[i] * bi[r] * bi[cc];
        }
        /* inverse by the adjugate */
        double A = T[0], B = T[1], C = T[2], D = T[3], E = T[4], F = T[5], G = T[6], H = T[7], J = T[8];
        double c00 = E * J - F * H, c01 = -(D * J - F * G), c02 = D * H - E * G;
        double det = A * c00 + B * c01 + C * c02;
        if (!(fabs(det) > 0) || !isfinite(det)) return -2;
        double inv[9] = {
            c00 / det, -(B * J - C * H) / det, (B * F - C * E) / det,
            c01 / det, (A * J - C * G) / det, -(A * F - C * D) / det,
            c02 / det, -(A * H - B * G) / det, (A * E - B * D) / det};
        memcpy(I + 9 * a, T, sizeof T);
        memcpy(Iinv + 9 * a, inv, sizeof inv);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* contact law for one canonical pair                                  */
/* ------------------------------------------------------------------ */
/*
 * Pair (i, j) with i the lower sphere index.  Sec. 2.1 (linear spring-dashpot
 * normal and tangential forces with contact history, static friction cap,
 * rolling and twisting friction) and Sec. 2.2.4 (contact point at the centre
 * of the intersection circle, lever arm Eq. lever_arm).
 *
 * Readings (the force law itself is deferred by the paper to earlier work):
 *   d = r_j - r_i, n = d/|d|, overlap x = s_i + s_j - |d|;
 *   l_i from Eq. lever_arm, l_j = |d| - l_i (both spheres share the point);
 *   u = (v_j + w_j x (-l_j n)) - (v_i + w_i x (l_i n)), u_n = (u.n) n, u_t = u - u_n;
 *   F_N = -kn x n + cn u_n                                 (force on i);
 *   S  = S_prev projected on the plane normal to n, rescaled to |S_prev|,
 *        plus u_t h;  F_T = kt S + ct u_t;
 *   |F_T| > mu_s |F_N|  =>  F_T scaled to mu_s |F_N|, S = (F_T - ct u_t)/kt;
 *   w = w_i - w_j, w_r = w - (w.n) n, w_t = (w.n) n, R = s_i s_j/(s_i + s_j);
 *   M_roll = -mu_r |F_N| R w_r / max(|w_r|, w0),
 *   M_tw   = -mu_t |F_N| R w_t / max(|w_t|, w0)            (couple on i);
 *   i gets F = F_N + F_T and tau_i = (l_i n) x F + M; j gets -F and
 *   tau_j = (-l_j n) x (-F) - M.
 * Outputs: F (on i), tau_i, tau_j, S_new, x, plus magnitudes for the scales.
 */
typedef struct {
    double F[3], ti[3], tj[3], S[3], x, li, lj, Fmag, Mmag;
} ora_pair;

static void ora_contact_pair(const double ri[3], const double rj[3],
                             const double vi[3], const double vj[3],
                             const double wi[3], const double wj[3],
                             double si, double sj, const double Sprev[3],
                             const ora_params *P, ora_pair *o)
{
    double d[3] = {rj[0] - ri[0], rj[1] - ri[1], rj[2] - ri[2]};
    double dist = v_norm(d);
    double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
    double x = si + sj - dist;
    double li = (si * si - sj * sj + dist * dist) / (2.0 * dist);
    double lj = dist - li;
    double ai[3] = {li * n[0], li * n[1], li * n[2]};
    double aj[3] = {-lj * n[0], -lj * n[1], -lj * n[2]};
    double wxa_i[3], wxa_j[3];
    v_cross(wi, ai, wxa_i);
    v_cross(wj, aj, wxa_j);
    double u[3];
    for (int k = 0; k < 3; ++k) u[k] = (vj[k] + wxa_j[k]) - (vi[k] + wxa_i[k]);
    double un_s = v_dot(u, n);
    double un[3] = {un_s * n[0], un_s * n[1], un_s * n[2]};
    double ut[3] = {u[0] - un[0], u[1] - un[1], u[2] - un[2]};
    double FN[3];
    for (int k = 0; k < 3; ++k) FN[k] = -P->kn * x * n[k] + P->cn * un[k];
    double FNmag = v_norm(FN);
    /* tangential spring: rotate the old displacement into the new tangent plane */
    double Sp[3];
    double sn = v_dot(Sprev, n);
    for (int k = 0; k < 3; ++k) Sp[k] = Sprev[k] - sn * n[k];
    double Sp_mag = v_norm(Sp), Sprev_mag = v_norm(Sprev);
    if (Sp_mag > 0) {
        double f = Sprev_mag / Sp_mag;
        for (int k = 0; k < 3; ++k) Sp[k] *= f;
    } else {
        Sp[0] = Sp[1] = Sp[2] = 0;
    }
    double S[3], FT[3];
    for (int k = 0; k < 3; ++k) {
        S[k] = Sp[k] + ut[k] * P->dt;
        FT[k] = P->kt * S[k] + P->ct * ut[k];
    }
    double FTmag = v_norm(FT), cap = P->mu_s * FNmag;
    if (FTmag > cap) {
        double f = cap / FTmag;
        for (int k = 0; k < 3; ++k) {
            FT[k] *= f;
            S[k] = (FT[k] - P->ct * ut[k]) / P->kt;
        }
    }
    /* rolling and twisting couples on i */
    double w[3] = {wi[0] - wj[0], wi[1] - wj[1], wi[2] - wj[2]};
    double wn = v_dot(w, n);
    double wt[3] = {wn * n[0], wn * n[1], wn * n[2]};
    double wr[3] = {w[0] - wt[0], w[1] - wt[1], w[2] - wt[2]};
    double Rred = si * sj / (si + sj);
    double M[3] = {0, 0, 0};
    double wr_mag = v_norm(wr), wt_mag = v_norm(wt);
    if (wr_mag > 0 && P->mu_r > 0) {
        double f = -P->mu_r * FNmag * Rred / fmax(wr_mag, P->w0);
        for (int k = 0; k < 3; ++k) M[k] += f * wr[k];
    }
    if (wt_mag > 0 && P->mu_t > 0) {
        double f = -P->mu_t * FNmag * Rred / fmax(wt_mag, P->w0);
        for (int k = 0; k < 3; ++k) M[k] += f * wt[k];
    }
    double F[3] = {FN[0] + FT[0], FN[1] + FT[1], FN[2] + FT[2]};
    double Fneg[3] = {-F[0], -F[1], -F[2]};
    double ti[3], tj[3];
    v_cross(ai, F, ti);
    v_cross(aj, Fneg, tj);
    for (int k = 0; k < 3; ++k) {
        ti[k] += M[k];
        tj[k] -= M[k];
        o->F[k] = F[k];
        o->ti[k] = ti[k];
        o->tj[k] = tj[k];
        o->S[k] = S[k];
    }
    o->x = x;
    o->li = li;
    o->lj = lj;
    o->Fmag = v_norm(F);
    o->Mmag = v_norm(M);
}

/* ------------------------------------------------------------------ */
/* contact pass                                                        */
/* ------------------------------------------------------------------ */
/*
 * Brute-force contact pass over all sphere pairs i < j that belong to
 * different aggregates and overlap (x > 0).  Pairs inside one aggregate are
 * skipped: its members are rigidly bonded (Sec. 2.2).  History is looked up
 * in the previous list of the canonical owner (i) by partner index and a new
 * list is written (Sec. 2.1: overlaps are tracked while contact lasts).
 * Forces are accumulated per sphere in ascending (i, j) order.
 * Fmag_i/Tmag_i (optional) receive per-sphere sums of |F| and of
 * (l |F| + |M|) over the sphere's contacts.
 * Returns the number of contacting pairs, or -1 on history overflow.
 */
int64_t ora_contacts(int64_t n, const double *pos, const double *vel, const double *w,
                     const double *radius, const int32_t *agg_of, const ora_params *P,
                     int32_t hcap, const int32_t *hn_prev, const int32_t *hp_prev,
                     const double *hS_prev, int32_t *hn_new, int32_t *hp_new, double *hS_new,
                     double *Fc, double *Tc, double *Fmag_i, double *Tmag_i,
                     int32_t *pairs, double *pair_x, int64_t pair_cap)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    /* pass 1: count overlapping pairs owned by each i */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = i + 1; j < n; ++j) {
            if (agg_of[j] == agg_of[i]) continue;
            double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                           pos[3 * j + 2] - pos[3 * i + 2]};
            if (radius[i] + radius[j] - v_norm(d) > 0) ++c;
        }
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int64_t np = cnt[n];
    int64_t *pj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    if (!pj) { free(cnt); return -1; }
    /* pass 2: fill partners in ascending j */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cnt[i];
        for (int64_t j = i + 1; j < n; ++j) {
            if (agg_of[j] == agg_of[i]) continue;
            double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                           pos[3 * j + 2] - pos[3 * i + 2]};
            if (radius[i] + radius[j] - v_norm(d) > 0) pj[c++] = j;
        }
    }
    memset(Fc, 0, sizeof(double) * 3 * (size_t)n);
    memset(Tc, 0, sizeof(double) * 3 * (size_t)n);
    if (Fmag_i) memset(Fmag_i, 0, sizeof(double) * (size_t)n);
    if (Tmag_i) memset(Tmag_i, 0, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) hn_new[i] = 0;
    int overflow = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = cnt[i]; k < cnt[i + 1]; ++k) {
            int64_t j = pj[k];
            double Sprev[3] = {0, 0, 0};
            for (int32_t h = 0; h < hn_prev[i]; ++h) {
                if (hp_prev[(int64_t)i * hcap + h] == (int32_t)j) {
                    for (int d = 0; d < 3; ++d) Sprev[d] = hS_prev[((int64_t)i * hcap + h) * 3 + d];
                    break;
                }
            }
            ora_pair o;
            ora_contact_pair(pos + 3 * i, pos + 3 * j, vel + 3 * i, vel + 3 * j, w + 3 * i,
                             w + 3 * j, radius[i], radius[j], Sprev, P, &o);
            for (int d = 0; d < 3; ++d) {
                Fc[3 * i + d] += o.F[d];
                Fc[3 * j + d] -= o.F[d];
                Tc[3 * i + d] += o.ti[d];
                Tc[3 * j + d] += o.tj[d];
            }
            if (Fmag_i) { Fmag_i[i] += o.Fmag; Fmag_i[j] += o.Fmag; }
            if (Tmag_i) {
                Tmag_i[i] += fabs(o.li) * o.Fmag + o.Mmag;
                Tmag_i[j] += fabs(o.lj) * o.Fmag + o.Mmag;
            }
            if (hn_new[i] < hcap) {
                int64_t slot = (int64_t)i * hcap + hn_new[i];
                hp_new[slot] = (int32_t)j;
                for (int d = 0; d < 3; ++d) hS_new[slot * 3 + d] = o.S[d];
                hn_new[i]++;
            } else {
                overflow = 1;
            }
            if (pairs && k < pair_cap) {
                pairs[2 * k] = (int32_t)i;
                pairs[2 * k + 1] = (int32_t)j;
                if (pair_x) pair_x[k] = o.x;
            }
        }
    }
    free(pj);
    free(cnt);
    return overflow ? -1 : np;
}

/* ------------------------------------------------------------------ */
/* gravity                                                             */
/* ------------------------------------------------------------------ */
/*
 * Eq. (particle_gravity), softened (Plummer, length eps):
 *   F_i = sum_{j != i} G m_i m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}.
 * exclude_same_agg = 0 sums every j != i of the pile, as the equation is
 * written.  The step uses exclude_same_agg = 1, which drops the members of
 * i's own aggregate: inside a rigid body those central pair forces cancel in
 * both the aggregate force and torque (Eq. agg_gravity, Eq. gravity_torque),
 * so every aggregate total is the same in exact arithmetic, and the per-sphere
 * force F_i is then the force from the other aggregates only.
 * rows == NULL computes every sphere; otherwise only the n_rows listed ones,
 * written to F[3*k] for the k-th listed sphere.  Fmag (optional) receives
 * sum_j |F_ij|.
 */
void ora_gravity(int64_t n, const double *pos, const double *m, const int32_t *agg_of,
                 double G, double eps, int exclude_same_agg, int64_t n_rows,
                 const int64_t *rows, double *F, double *Fmag)
{
    int64_t nr = rows ? n_rows : n;
    double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nr; ++k) {
        int64_t i = rows ? rows[k] : k;
        double f[3] = {0, 0, 0}, fm = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (exclude_same_agg && agg_of[j] == agg_of[i]) continue;
            double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                           pos[3 * j + 2] - pos[3 * i + 2]};
            double r2 = v_dot(d, d) + e2;
            double g = G * m[i] * m[j] / (r2 * sqrt(r2));
            for (int c = 0; c < 3; ++c) f[c] += g * d[c];
            if (Fmag) fm += g * sqrt(v_dot(d, d));
        }
        for (int c = 0; c < 3; ++c) F[3 * k + c] = f[c];
        if (Fmag) Fmag[k] = fm;
    }
}

/* Point-mass planet (Sec. 4.2): F_i = G M_P m_i (r_P - r_i)/|r_P - r_i|^3. */
static void ora_planet_force(const double rP[3], double MP, double G, const double ri[3],
                             double mi, double F[3])
{
    double d[3] = {rP[0] - ri[0], rP[1] - ri[1], rP[2] - ri[2]};
    double r = v_norm(d);
    double g = G * MP * mi / (r * r * r);
    for (int c = 0; c < 3; ++c) F[c] = g * d[c];
}

/* ------------------------------------------------------------------ */
/* rotation: Euler's equations                                          */
/* ------------------------------------------------------------------ */
/*
 * Sec. 2.2.1: orientation and spin obey Euler's rigid-body equations.  The
 * paper integrates them with an adaptive 5th-order Runge-Kutta scheme next to
 * its kick-drift-kick leapfrog for the COM (Sec. 2.1).  The reading here splits
 * the spin the same way as the COM: a half kick of the space-frame angular
 * momentum by h/2 N (ora_spin_kick), a torque-free rotation over h by one
 * classical RK4 step on y = (q, w_body) with
 *   dq/dt = 1/2 q (x) (0, w_body),
 *   dw/dt = I^-1 (N_body - w x (I w))      (N_body = 0 in the drift),
 * q renormalised afterwards, then the second half kick with the new torque.
 * Kicks of orbital and spin momentum then happen together with balanced
 * torques, so the total angular momentum is conserved to round-off plus the
 * RK4 error of the free rotor.  ora_rotate accepts a body-frame torque held
 * over the step (R(q_n)^T N) for use as a plain integrator.
 */
static void ora_rot_deriv(const double y[7], const double *I, const double *Iinv,
                          const double Nb[3], double dy[7])
{
    const double *q = y, *w = y + 4;
    dy[0] = -0.5 * (q[1] * w[0] + q[2] * w[1] + q[3] * w[2]);
    dy[1] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
    dy[2] = 0.5 * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
    dy[3] = 0.5 * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
    double Iw[3], wxIw[3], rhs[3];
    mat_vec(I, w, Iw);
    v_cross(w, Iw, wxIw);
    for (int k = 0; k < 3; ++k) rhs[k] = Nb[k] - wxIw[k];
    mat_vec(Iinv, rhs, dy + 4);
}

void ora_rotate(double q[4], double wb[3], const double *I, const double *Iinv,
                const double N_space[3], double h)
{
    double R[9], Nb[3];
    ora_rotmat(q, R);
    mat_tvec(R, N_space, Nb);
    double y[7] = {q[0], q[1], q[2], q[3], wb[0], wb[1], wb[2]};
    double k1[7], k2[7], k3[7], k4[7], t[7];
    ora_rot_deriv(y, I, Iinv, Nb, k1);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + 0.5 * h * k1[c];
    ora_rot_deriv(t, I, Iinv, Nb, k2);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + 0.5 * h * k2[c];
    ora_rot_deriv(t, I, Iinv, Nb, k3);
    for (int c = 0; c < 7; ++c) t[c] = y[c] + h * k3[c];
    ora_rot_deriv(t, I, Iinv, Nb, k4);
    for (int c = 0; c < 7; ++c) y[c] += h / 6.0 * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
    double qn = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
    for (int c = 0; c < 4; ++c) q[c] = y[c] / qn;
    for (int c = 0; c < 3; ++c) wb[c] = y[4 + c];
}

/*
 * The paper's rotation integrator (Sec. 2.2.1): a time-adaptive fifth-order
 * Runge-Kutta scheme.  The torque-free rotation over h is taken in substeps of
 * the embedded Runge-Kutta pair of Cash and Karp (6 stages: a fifth-order
 * solution and a fourth-order one whose difference estimates the error).  A
 * substep is accepted when its error, measured in q absolutely and in w
 * relative to |w|, is at most tol; the next substep is the present one times
 * 0.9 (tol/err)^(1/5) (at most 5 times larger), a rejected one is retried
 * with 0.9 (tol/err)^(1/4) of it (at least a tenth).  The first trial is the
 * whole step.  A substep shorter than h / 2^20 is accepted whatever its error,
 * so the loop always ends.  q is renormalised at the end of the step, as in
 * the RK4 reading.  Returns the number of accepted substeps.
 */
static const double ck_c[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double ck_a[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
static const double ck_b5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static const double ck_b4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                                277.0 / 14336.0, 1.0 / 4.0};

int ora_rotate_adaptive(double q[4], double wb[3], const double *I, const double *Iinv,
                        double h, double tol)
{
    const double zero[3] = {0, 0, 0};
    double y[7] = {q[0], q[1], q[2], q[3], wb[0], wb[1], wb[2]};
    double t = 0.0, dt = h;
    int accepted = 0;
    (void)ck_c;   /* autonomous equations: the stage times are not needed */
    while (t < h) {
        if (t + dt > h) dt = h - t;
        double k[6][7], z[7];
        ora_rot_deriv(y, I, Iinv, zero, k[0]);
        for (int st = 1; st < 6; ++st) {
            for (int c = 0; c < 7; ++c) {
                double acc = 0.0;
                for (int j = 0; j < st; ++j) acc += ck_a[st][j] * k[j][c];
                z[c] = y[c] + dt * acc;
            }
            ora_rot_deriv(z, I, Iinv, zero, k[st]);
        }
        double y5[7], err = 0.0;
        double wn = sqrt(y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
        for (int c = 0; c < 7; ++c) {
            double s5 = 0.0, s4 = 0.0;
            for (int j = 0; j < 6; ++j) { s5 += ck_b5[j] * k[j][c]; s4 += ck_b4[j] * k[j][c]; }
            y5[c] = y[c] + dt * s5;
            double e = fabs(dt * (s5 - s4));
            if (c >= 4) e /= (wn > 0 ? wn : 1.0);
            if (e > err) err = e;
        }
        double ratio = err / tol;
        if (ratio <= 1.0 || dt <= h * 0x1p-20) {
            memcpy(y, y5, sizeof y);
            t += dt;
            ++accepted;
            double grow = ratio > 0 ? 0.9 * pow(ratio, -0.2) : 5.0;
            dt *= grow < 5.0 ? grow : 5.0;
        } else {
            double shrink = 0.9 * pow(ratio, -0.25);
            dt *= shrink > 0.1 ? shrink : 0.1;
        }
    }
    double qn = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
    for (int c = 0; c < 4; ++c) q[c] = y[c] / qn;
    for (int c = 0; c < 3; ++c) wb[c] = y[4 + c];
    return accepted;
}

/* Half kick of the spin: L_space += dt N  <=>  w_body += dt I^-1 R(q)^T N. */
void ora_spin_kick(const double q[4], double wb[3], const double *Iinv, const double N_space[3],
                   double dt)
{
    double R[9], Nb[3], dw[3];
    ora_rotmat(q, R);
    mat_tvec(R, N_space, Nb);
    mat_vec(Iinv, Nb, dw);
    for (int c = 0; c < 3; ++c) wb[c] += dt * dw[c];
}

/* ------------------------------------------------------------------ */
/* one step                                                            */
/* ------------------------------------------------------------------ */
/* Sphere positions, predicted velocities and spins (Sec. 2.2.2, Eq. pred-vel):
 *   r_i = r_A + R(q_A) b_i,
 *   v_i = [v_A,n+1/2 + h/2 a_A,n] + w_A,n+1 x (r_i - r_A),   w_i = w_A,n+1,
 * where w_A,n+1 is the spin the full step would reach under N_A,n: the drifted
 * spin plus the second half kick with the old torque (the spin analogue of the
 * bracketed COM term). */
static void ora_expand(ora_sim *S, double h)
{
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < S->n_agg; ++a) {
        double R[9], ws[3], wpred[3];
        for (int c = 0; c < 3; ++c) wpred[c] = S->wb[3 * a + c];
        ora_spin_kick(S->q + 4 * a, wpred, S->Iinv + 9 * a, S->torque + 3 * a, 0.5 * h);
        ora_rotmat(S->q + 4 * a, R);
        mat_vec(R, wpred, ws);
        for (int64_t i = S->first[a]; i < S->first[a] + S->count[a]; ++i) {
            double rb[3], wxr[3];
            mat_vec(R, S->b + 3 * i, rb);
            v_cross(ws, rb, wxr);
            for (int c = 0; c < 3; ++c) {
                S->sph_pos[3 * i + c] = S->r[3 * a + c] + rb[c];
                S->sph_vel[3 * i + c] = S->v[3 * a + c] + 0.5 * h * S->acc[3 * a + c] + wxr[c];
                S->sph_w[3 * i + c] = ws[c];
            }
        }
    }
}

/* Sec. 2.2.3 and 2.2.4: per-aggregate totals.
 *   F_A = sum_i (F_c,i + F_g,i + F_e,i)       (Eq. agg_gravity, Eq. agg_contact_accel, times M)
 *   N_A = sum_i [(r_i - r_A) x F_i] + tau_i   (Eq. gravity_torque; the contact torque
 *         read as (r_i + l n - r_A) x F, i.e. lever about the sphere centre plus
 *         (r_i - r_A) x F; the printed form drops r_i). */
static void ora_reduce(ora_sim *S, const double *Fmag_c, const double *Tmag_c,
                       const double *Fmag_g)
{
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < S->n_agg; ++a) {
        double Fc[3] = {0, 0, 0}, Nc[3] = {0, 0, 0}, Fg[3] = {0, 0, 0}, Ng[3] = {0, 0, 0};
        double Fe[3] = {0, 0, 0}, Ne[3] = {0, 0, 0};
        double sF = 0, sN = 0;
        for (int64_t i = S->first[a]; i < S->first[a] + S->count[a]; ++i) {
            double rel[3], t[3];
            for (int c = 0; c < 3; ++c) rel[c] = S->sph_pos[3 * i + c] - S->r[3 * a + c];
            v_cross(rel, S->Fc + 3 * i, t);
            for (int c = 0; c < 3; ++c) { Fc[c] += S->Fc[3 * i + c]; Nc[c] += t[c] + S->Tc[3 * i + c]; }
            v_cross(rel, S->Fg + 3 * i, t);
            for (int c = 0; c < 3; ++c) { Fg[c] += S->Fg[3 * i + c]; Ng[c] += t[c]; }
            v_cross(rel, S->Fe + 3 * i, t);
            for (int c = 0; c < 3; ++c) { Fe[c] += S->Fe[3 * i + c]; Ne[c] += t[c]; }
            double mag = (Fmag_c ? Fmag_c[i] : 0) + (Fmag_g ? Fmag_g[i] : 0) + v_norm(S->Fe + 3 * i);
            sF += mag;
            sN += v_norm(rel) * mag + (Tmag_c ? Tmag_c[i] : 0);
        }
        for (int c = 0; c < 3; ++c) {
            S->FA_c[3 * a + c] = Fc[c]; S->NA_c[3 * a + c] = Nc[c];
            S->FA_g[3 * a + c] = Fg[c]; S->NA_g[3 * a + c] = Ng[c];
            S->FA_e[3 * a + c] = Fe[c]; S->NA_e[3 * a + c] = Ne[c];
        }
        if (S->scaleF) S->scaleF[a] = sF;
        if (S->scaleN) S->scaleN[a] = sN;
    }
}

/*
 * Force evaluation at the current sphere positions/velocities: contacts,
 * gravity, planet, aggregate totals.  want_scales != 0 also fills the
 * condition scales (costs one more square root per gravity pair).
 * History is read from the h_* arrays and the new list written back.
 */
static int ora_forces(ora_sim *S, const ora_params *P, int want_scales)
{
    int64_t n = S->n_sph;
    int32_t *hn_new = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *hp_new = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * S->hcap);
    double *hS_new = (double *)malloc(sizeof(double) * (size_t)n * S->hcap * 3);
    double *Fmc = want_scales ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    double *Tmc = want_scales ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    double *Fmg = want_scales ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    if (!hn_new || !hp_new || !hS_new) return -1;
    int64_t np = ora_contacts(n, S->sph_pos, S->sph_vel, S->sph_w, S->s, S->agg_of, P, S->hcap,
                              S->h_n, S->h_partner, S->h_S, hn_new, hp_new, hS_new, S->Fc, S->Tc,
                              Fmc, Tmc, S->pairs, S->pair_x, S->pair_cap);
    S->n_pairs = np;
    memcpy(S->h_n, hn_new, sizeof(int32_t) * (size_t)n);
    memcpy(S->h_partner, hp_new, sizeof(int32_t) * (size_t)n * S->hcap);
    memcpy(S->h_S, hS_new, sizeof(double) * (size_t)n * S->hcap * 3);
    free(hn_new); free(hp_new); free(hS_new);
    ora_gravity(n, S->sph_pos, S->m, S->agg_of, P->G, P->eps, 1, 0, NULL, S->Fg, Fmg);
    for (int64_t i = 0; i < n; ++i) {
        if (P->ext_mass > 0)
            ora_planet_force(S->planet, P->ext_mass, P->G, S->sph_pos + 3 * i, S->m[i], S->Fe + 3 * i);
        else
            S->Fe[3 * i] = S->Fe[3 * i + 1] = S->Fe[3 * i + 2] = 0;
    }
    ora_reduce(S, Fmc, Tmc, Fmg);
    if (want_scales) {
        if (S->sph_Fmc) memcpy(S->sph_Fmc, Fmc, sizeof(double) * (size_t)n);
        if (S->sph_Tmc) memcpy(S->sph_Tmc, Tmc, sizeof(double) * (size_t)n);
        if (S->sph_Fmg) memcpy(S->sph_Fmg, Fmg, sizeof(double) * (size_t)n);
    }
    free(Fmc); free(Tmc); free(Fmg);
    return np < 0 ? -2 : 0;
}

/*
 * One fixed step h of the leapfrog (Sec. 2.1) for a pile of aggregates:
 *   1. v_A += h/2 a_A,n;  spin half kick by h/2 N_A,n;  r_A += h v_A;
 *      torque-free RK4 rotation of (q, w_body) over h            (Sec. 2.1, 2.2.1)
 *      planet: same kick-drift with its stored acceleration
 *   2. sphere positions, predicted velocities, spins             (Eq. pred-vel)
 *   3. contacts, gravity, planet force, aggregate totals          (Sec. 2.2.3-2.2.4)
 *   4. a_A = F_A / M;  v_A += h/2 a_A;  spin half kick by h/2 N_A;  a_A, N_A
 *      stored for the next step
 *      planet: a_P = -(sum of planet forces on the spheres)/M_P; v_P += h/2 a_P
 *   5. YORP (Sec. 4.1): constant spin increment dw about a fixed axis applied
 *      to the whole pile as a rigid rotation increment: for every aggregate
 *      w_A += dw and v_A += dw x (r_A - R_pile), R_pile = pile COM.
 * The stored a_A and N_A of a new pile are zero.
 * Returns 0, -2 on history overflow.
 */
static void ora_kick_drift(ora_sim *S, const ora_params *P, double h)
{
    const double zero[3] = {0, 0, 0};
    for (int64_t a = 0; a < S->n_agg; ++a) {
        for (int c = 0; c < 3; ++c) {
            S->v[3 * a + c] += 0.5 * h * S->acc[3 * a + c];
            S->r[3 * a + c] += h * S->v[3 * a + c];
        }
        ora_spin_kick(S->q + 4 * a, S->wb + 3 * a, S->Iinv + 9 * a, S->torque + 3 * a, 0.5 * h);
        if (P->rot_tol > 0)
            ora_rotate_adaptive(S->q + 4 * a, S->wb + 3 * a, S->I + 9 * a, S->Iinv + 9 * a, h,
                                P->rot_tol);
        else
            ora_rotate(S->q + 4 * a, S->wb + 3 * a, S->I + 9 * a, S->Iinv + 9 * a, zero, h);
    }
}

int ora_step(ora_sim *S, const ora_params *P, int want_scales)
{
    double h = P->dt;
    ora_kick_drift(S, P, h);
    if (P->ext_mass > 0) {
        for (int c = 0; c < 3; ++c) {
            S->planet[3 + c] += 0.5 * h * S->planet[6 + c];
            S->planet[c] += h * S->planet[3 + c];
        }
    }
    ora_expand(S, h);
    int rc = ora_forces(S, P, want_scales);
    double Fe_tot[3] = {0, 0, 0};
    for (int64_t a = 0; a < S->n_agg; ++a) {
        double Ma = S->M[a];
        for (int c = 0; c < 3; ++c) {
            double F = S->FA_c[3 * a + c] + S->FA_g[3 * a + c] + S->FA_e[3 * a + c];
            S->acc[3 * a + c] = F / Ma;
            S->torque[3 * a + c] = S->NA_c[3 * a + c] + S->NA_g[3 * a + c] + S->NA_e[3 * a + c];
            S->v[3 * a + c] += 0.5 * h * S->acc[3 * a + c];
            Fe_tot[c] += S->FA_e[3 * a + c];
        }
        ora_spin_kick(S->q + 4 * a, S->wb + 3 * a, S->Iinv + 9 * a, S->torque + 3 * a, 0.5 * h);
    }
    if (P->ext_mass > 0) {
        for (int c = 0; c < 3; ++c) {
            S->planet[6 + c] = -Fe_tot[c] / P->ext_mass;
            S->planet[3 + c] += 0.5 * h * S->planet[6 + c];
        }
    }
    if (P->spin_inc[0] != 0 || P->spin_inc[1] != 0 || P->spin_inc[2] != 0) {
        double Mt = 0, Rp[3] = {0, 0, 0};
        for (int64_t a = 0; a < S->n_agg; ++a) {
            Mt += S->M[a];
            for (int c = 0; c < 3; ++c) Rp[c] += S->M[a] * S->r[3 * a + c];
        }
        for (int c = 0; c < 3; ++c) Rp[c] /= Mt;
        for (int64_t a = 0; a < S->n_agg; ++a) {
            double rel[3], dv[3], R[9], dwb[3];
            for (int c = 0; c < 3; ++c) rel[c] = S->r[3 * a + c] - Rp[c];
            v_cross(P->spin_inc, rel, dv);
            ora_rotmat(S->q + 4 * a, R);
            mat_tvec(R, P->spin_inc, dwb);
            for (int c = 0; c < 3; ++c) {
                S->v[3 * a + c] += dv[c];
                S->wb[3 * a + c] += dwb[c];
            }
        }
    }
    return rc;
}

/*
 * Steps 1-3 of ora_step for the whole pile, then forces for the listed
 * spheres only (contacts by brute force against every sphere, gravity
 * rows, planet), with empty contact history.  Used to check large piles on
 * sampled outputs after their first step.  Outputs per listed sphere k:
 * Fc, Tc, Fg, Fe (3 each) and, if non-NULL, the scales Fmag (contact + gravity
 * magnitude sums) and Tmag (contact lever magnitude sums).
 * State arrays of S are advanced through the drift (positions, rotation).
 */
int ora_step_sampled(ora_sim *S, const ora_params *P, int64_t n_rows, const int64_t *rows,
                     double *Fc, double *Tc, double *Fg, double *Fe, double *Fmag, double *Tmag)
{
    double h = P->dt;
    ora_kick_drift(S, P, h);
    double planet_pos[3] = {0, 0, 0};
    if (P->ext_mass > 0) {
        for (int c = 0; c < 3; ++c) {
            S->planet[3 + c] += 0.5 * h * S->planet[6 + c];
            S->planet[c] += h * S->planet[3 + c];
            planet_pos[c] = S->planet[c];
        }
    }
    ora_expand(S, h);
    int64_t n = S->n_sph;
    double *Fgm = Fmag ? (double *)malloc(sizeof(double) * (size_t)n_rows) : NULL;
    ora_gravity(n, S->sph_pos, S->m, S->agg_of, P->G, P->eps, 1, n_rows, rows, Fg, Fgm);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < n_rows; ++k) {
        int64_t i = rows[k];
        double f[3] = {0, 0, 0}, t[3] = {0, 0, 0}, fm = 0, tm = 0;
        const double zero[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i || S->agg_of[j] == S->agg_of[i]) continue;
            const double *pi = S->sph_pos + 3 * i, *pj = S->sph_pos + 3 * j;
            double d[3] = {pj[0] - pi[0], pj[1] - pi[1], pj[2] - pi[2]};
            if (S->s[i] + S->s[j] - v_norm(d) <= 0) continue;
            ora_pair o;
            int64_t lo = i < j ? i : j, hi = i < j ? j : i;
            ora_contact_pair(S->sph_pos + 3 * lo, S->sph_pos + 3 * hi, S->sph_vel + 3 * lo,
                             S->sph_vel + 3 * hi, S->sph_w + 3 * lo, S->sph_w + 3 * hi, S->s[lo],
                             S->s[hi], zero, P, &o);
            for (int c = 0; c < 3; ++c) {
                f[c] += (i == lo) ? o.F[c] : -o.F[c];
                t[c] += (i == lo) ? o.ti[c] : o.tj[c];
            }
            fm += o.Fmag;
            tm += fabs(i == lo ? o.li : o.lj) * o.Fmag + o.Mmag;
        }
        for (int c = 0; c < 3; ++c) { Fc[3 * k + c] = f[c]; Tc[3 * k + c] = t[c]; }
        if (P->ext_mass > 0)
            ora_planet_force(planet_pos, P->ext_mass, P->G, S->sph_pos + 3 * i, S->m[i], Fe + 3 * k);
        else
            Fe[3 * k] = Fe[3 * k + 1] = Fe[3 * k + 2] = 0;
        if (Fmag) Fmag[k] = fm + Fgm[k] + v_norm(Fe + 3 * k);
        if (Tmag) Tmag[k] = tm;
    }
    free(Fgm);
    return 0;
}
