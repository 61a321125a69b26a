// kernels_analysis.cu -- bulk shape and spin of each pile, and the
// radius-growth watch evaluated inside the step graph.
//
// Paper references: the critical spin ratio measures the spin period at which
// a pile's radius has grown by 5% against the nominal period
// sqrt(3 pi / (G rho)) of a rigid sphere of the pile's bulk density
// (Sec. 4.1); the disruption ratio measures the planet distance at which the
// bulk radius has grown by 0.5% against the Roche distance (Sec. 4.2).  The
// paper does not say how it measures a pile's radius; here it is the radius
// (a b c)^(1/3) of the uniform ellipsoid with the pile's mass and principal
// moments of inertia, which also gives the bulk density.
//
// One kernel, like the pile reductions of the step: blocks of kAggChunk
// aggregates sum 25 moments about the pile frame (fixed tree order), then the
// pile's last block to finish adds the chunks in order and its first thread
// finishes the record in FP64 (parallel-axis shift, 3x3 Jacobi eigenvalues,
// Cramer solve).
#include <math_constants.h>

#include "dem_internal.h"
#include "devmath.cuh"
#include "launch.cuh"

namespace dem {

namespace {

constexpr int kBulkBlock = 128;

// Whether pile p is evaluated by this launch.  Mode 0: every pile (or only
// `only`).  Mode 1 (step graph): armed, not yet latched, stepping piles whose
// step counter is a multiple of the watch period.
__device__ __forceinline__ bool bulk_due(const Arrays &a, int p, int mode, int only)
{
    if (mode == 0) return only < 0 || p == only;
    if (a.enabled[p] == 0 || a.pd[p].failed) return false;
    const PileWatch &W = a.watch[p];
    if (!(W.growth > 0.0) || W.fired >= 0) return false;
    return a.pd[p].steps % W.every == 0;
}

// Moments of aggregate g about the pile frame (x = r - O, u = v - V):
// [0] M, [1..3] M x, [4..6] M u, [7..12] M x x^T (xx yy zz xy xz yz),
// [13..18] R I R^T (same order), [19..21] M x cross u, [22..24] R I w_body.
__device__ __forceinline__ void agg_moments(const Arrays &a, int64_t g, const PileDyn &D, double *m)
{
    const double M = a.M[g];
    // the state as doubles (the mixed path stores float-float pairs)
    auto st = [&](const double *s, int k) { return a.out_ff ? ff_value(ldff(s + k)) : s[k]; };
    const double x[3] = {st(a.r, 3 * g) - D.O[0], st(a.r, 3 * g + 1) - D.O[1], st(a.r, 3 * g + 2) - D.O[2]};
    const double u[3] = {st(a.v, 3 * g) - D.V[0], st(a.v, 3 * g + 1) - D.V[1], st(a.v, 3 * g + 2) - D.V[2]};
    const double qd[4] = {st(a.q, 4 * g), st(a.q, 4 * g + 1), st(a.q, 4 * g + 2), st(a.q, 4 * g + 3)};
    double R[9];
    quat_to_R(qd, R);
    const double *Ib = a.I + 9 * g;
    double T[9];   // R I_body
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = R[3 * i] * Ib[j] + R[3 * i + 1] * Ib[3 + j] + R[3 * i + 2] * Ib[6 + j];
    // (R I R^T)_ij = sum_k T_ik R_jk
    auto rirt = [&](int i, int j) {
        return T[3 * i] * R[3 * j] + T[3 * i + 1] * R[3 * j + 1] + T[3 * i + 2] * R[3 * j + 2];
    };
    const double wb[3] = {st(a.wb, 3 * g), st(a.wb, 3 * g + 1), st(a.wb, 3 * g + 2)};
    m[0] = M;
    for (int c = 0; c < 3; ++c) {
        m[1 + c] = M * x[c];
        m[4 + c] = M * u[c];
    }
    m[7] = M * x[0] * x[0];
    m[8] = M * x[1] * x[1];
    m[9] = M * x[2] * x[2];
    m[10] = M * x[0] * x[1];
    m[11] = M * x[0] * x[2];
    m[12] = M * x[1] * x[2];
    m[13] = rirt(0, 0);
    m[14] = rirt(1, 1);
    m[15] = rirt(2, 2);
    m[16] = rirt(0, 1);
    m[17] = rirt(0, 2);
    m[18] = rirt(1, 2);
    m[19] = M * (x[1] * u[2] - x[2] * u[1]);
    m[20] = M * (x[2] * u[0] - x[0] * u[2]);
    m[21] = M * (x[0] * u[1] - x[1] * u[0]);
    for (int c = 0; c < 3; ++c) m[22 + c] = T[3 * c] * wb[0] + T[3 * c + 1] * wb[1] + T[3 * c + 2] * wb[2];
}

__device__ void bulk_finalize(const Arrays &a, int p, int mode, double (&sh)[kBulkParts][kBulkBlock]);

__global__ void __launch_bounds__(kBulkBlock) k_bulk_partials(Arrays a, Sizes z, int mode, int only)
{
    pdl_enter();
    const int64_t ch = blockIdx.x;
    if (ch >= z.CH) return;
    const int p = a.chunk_pile[ch];
    if (!bulk_due(a, p, mode, only)) return;
    const PileStatic &S = a.ps[p];
    const PileDyn &D = a.pd[p];
    __shared__ double sh[kBulkParts][kBulkBlock];
    double acc[kBulkParts];
    for (int k = 0; k < kBulkParts; ++k) acc[k] = 0.0;
    const int64_t beg = S.a0 + (ch - S.ch0) * kAggChunk;
    const int64_t end = min(beg + kAggChunk, S.a0 + S.na);
    for (int64_t g = beg + threadIdx.x; g < end; g += kBulkBlock) {
        double m[kBulkParts];
        agg_moments(a, g, D, m);
        for (int k = 0; k < kBulkParts; ++k) acc[k] += m[k];
    }
    for (int k = 0; k < kBulkParts; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kBulkBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < kBulkParts; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    // the pile's last chunk block to finish adds up the pile (see bulk_finalize)
    __shared__ int last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kBulkParts; ++k) a.bulk_part[ch * 32 + k] = sh[k][0];
        __threadfence();   // the sums are visible before this block is counted
        last = atomicAdd(a.pile_arrive + p, 1) == (int)S.nch - 1;
        if (last) a.pile_arrive[p] = 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    bulk_finalize(a, p, mode, sh);
}

// Eigenvalues of the symmetric 3x3 matrix (xx yy zz xy xz yz), ascending, by
// cyclic Jacobi rotations (Golub and Van Loan, Sec. 8.5); at most 32 sweeps.
__device__ void sym3_eigenvalues(const double *s, double *ev)
{
    double A[3][3] = {{s[0], s[3], s[4]}, {s[3], s[1], s[5]}, {s[4], s[5], s[2]}};
    for (int sweep = 0; sweep < 32; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (!(off > 1e-34 * dia)) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A[p][q];
                if (apq == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                // A <- J^T A J with J the rotation in the (p, q) plane
                for (int k = 0; k < 3; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                A[p][q] = A[q][p] = 0.0;
            }
    }
    double e0 = A[0][0], e1 = A[1][1], e2 = A[2][2], t;
    if (e0 > e1) { t = e0; e0 = e1; e1 = t; }
    if (e1 > e2) { t = e1; e1 = e2; e2 = t; }
    if (e0 > e1) { t = e0; e0 = e1; e1 = t; }
    ev[0] = e0;
    ev[1] = e1;
    ev[2] = e2;
}

// The record of enum dem_bulk from the 25 summed moments.
__device__ void bulk_record(const double *s, const PileStatic &S, const PileDyn &D, double *out)
{
    const double M = s[0];
    const double c[3] = {s[1] / M, s[2] / M, s[3] / M};      // COM - O
    const double uc[3] = {s[4] / M, s[5] / M, s[6] / M};     // v_c - V
    // second moment about the COM, then the orbital inertia plus the
    // aggregates' own
    const double Sxx = s[7] - M * c[0] * c[0], Syy = s[8] - M * c[1] * c[1], Szz = s[9] - M * c[2] * c[2];
    const double Sxy = s[10] - M * c[0] * c[1], Sxz = s[11] - M * c[0] * c[2], Syz = s[12] - M * c[1] * c[2];
    const double tr = Sxx + Syy + Szz;
    const double I6[6] = {tr - Sxx + s[13], tr - Syy + s[14], tr - Szz + s[15],
                          -Sxy + s[16], -Sxz + s[17], -Syz + s[18]};
    const double L[3] = {s[19] - M * (c[1] * uc[2] - c[2] * uc[1]) + s[22],
                         s[20] - M * (c[2] * uc[0] - c[0] * uc[2]) + s[23],
                         s[21] - M * (c[0] * uc[1] - c[1] * uc[0]) + s[24]};
    double ev[3];
    sym3_eigenvalues(I6, ev);
    const double k = 5.0 / (2.0 * M);
    const double a2 = fmax(0.0, k * (ev[1] + ev[2] - ev[0]));
    const double b2 = fmax(0.0, k * (ev[0] + ev[2] - ev[1]));
    const double c2 = fmax(0.0, k * (ev[0] + ev[1] - ev[2]));
    const double ax = sqrt(a2), bx = sqrt(b2), cx = sqrt(c2);
    const double vol = ax * bx * cx;
    const double rho = vol > 0.0 ? 3.0 * M / (4.0 * CUDART_PI * vol) : CUDART_INF;
    // w = I^-1 L by Cramer's rule
    const double xx = I6[0], yy = I6[1], zz = I6[2], xy = I6[3], xz = I6[4], yz = I6[5];
    const double c00 = yy * zz - yz * yz, c01 = xz * yz - xy * zz, c02 = xy * yz - xz * yy;
    const double c11 = xx * zz - xz * xz, c12 = xy * xz - xx * yz, c22 = xx * yy - xy * xy;
    const double det = xx * c00 + xy * c01 + xz * c02;
    double w[3] = {0.0, 0.0, 0.0};
    if (det > 0.0) {
        w[0] = (c00 * L[0] + c01 * L[1] + c02 * L[2]) / det;
        w[1] = (c01 * L[0] + c11 * L[1] + c12 * L[2]) / det;
        w[2] = (c02 * L[0] + c12 * L[1] + c22 * L[2]) / det;
    }
    const double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    out[DEM_BULK_MASS] = M;
    for (int d = 0; d < 3; ++d) {
        out[DEM_BULK_COM + d] = D.O[d] + c[d];
        out[DEM_BULK_VCOM + d] = D.V[d] + uc[d];
        out[DEM_BULK_SPIN + d] = w[d];
        out[DEM_BULK_L + d] = L[d];
        out[DEM_BULK_MOMENTS + d] = ev[d];
    }
    out[DEM_BULK_AXES] = ax;
    out[DEM_BULK_AXES + 1] = bx;
    out[DEM_BULK_AXES + 2] = cx;
    out[DEM_BULK_RADIUS] = cbrt(vol);
    out[DEM_BULK_DENSITY] = rho;
    out[DEM_BULK_PERIOD] = wn > 0.0 ? 2.0 * CUDART_PI / wn : CUDART_INF;
    out[DEM_BULK_PCRIT] = (S.G > 0.0 && rho > 0.0 && rho < CUDART_INF) ? sqrt(3.0 * CUDART_PI / (S.G * rho))
                                                                       : CUDART_INF;
    double dist = 0.0;
    if (S.ext_mass > 0.0) {
        double d2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double e = D.P_pos[d] - out[DEM_BULK_COM + d];
            d2 += e * e;
        }
        dist = sqrt(d2);
    }
    out[DEM_BULK_PLANET_DIST] = dist;
}

// Run by the last chunk block of pile p: thread t adds chunks t, t+128, ... in
// order, a fixed tree combines the threads (deterministic whichever block is
// last), thread 0 forms the record and updates the watch.
__device__ void bulk_finalize(const Arrays &a, int p, int mode, double (&sh)[kBulkParts][kBulkBlock])
{
    const PileStatic &S = a.ps[p];
    double s[kBulkParts];
    for (int k = 0; k < kBulkParts; ++k) s[k] = 0.0;
    for (int64_t ch = S.ch0 + threadIdx.x; ch < S.ch0 + S.nch; ch += kBulkBlock)
        for (int k = 0; k < kBulkParts; ++k) s[k] += __ldcg(a.bulk_part + ch * 32 + k);
    __syncthreads();   // sh is free again
    for (int k = 0; k < kBulkParts; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int o = kBulkBlock / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < kBulkParts; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    for (int k = 0; k < kBulkParts; ++k) s[k] = sh[k][0];
    PileWatch &W = a.watch[p];
    bulk_record(s, S, a.pd[p], W.now);
    if (!(W.growth > 0.0) || W.fired >= 0) return;
    if (W.arm) {
        for (int k = 0; k < DEM_BULK_LEN; ++k) W.at_arm[k] = W.now[k];
        W.arm = 0;
    } else if (mode == 1 && W.now[DEM_BULK_RADIUS] >= (1.0 + W.growth) * W.at_arm[DEM_BULK_RADIUS]) {
        for (int k = 0; k < DEM_BULK_LEN; ++k) W.at_fire[k] = W.now[k];
        W.fired = a.pd[p].steps;
    }
}

}  // namespace

void launch_bulk(const Arrays &a, const Sizes &z, int mode, int only, cudaStream_t st)
{
    if (z.CH == 0 || z.P == 0) return;
    launch_pdl(k_bulk_partials, (unsigned)z.CH, kBulkBlock, 0, st, a, z, mode, only);
}

}  // namespace dem
