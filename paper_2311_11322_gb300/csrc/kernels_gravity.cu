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
// A pile with several j-ranges writes one FP64 partial per (range, sphere)
// and k_grav_combine adds them in range order (deterministic).
#include "dem_internal.h"
#include "devmath.cuh"

namespace dem {

constexpr int kFlush = 1024;

template <int BS, int IB>
__global__ void __launch_bounds__(BS) k_gravity32(Arrays a, Sizes z)
{
    __shared__ float4 sp[BS];
    __shared__ int sag[BS];
    __shared__ int excl[2];
    const int4 it = a.gitems[blockIdx.x];
    const int p = it.x;
    if (a.enabled[p] == 0 || a.pd[p].failed) return;
    const PileStatic &S = a.ps[p];
    const int64_t s0 = S.s0;
    const int ns = (int)S.ns;
    const int i0 = it.y, j0 = it.z, j1 = it.w;
    const float eps2 = (float)S.eps2;
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
    int since = 0;
    for (int jt = j0; jt < j1; jt += BS) {
        __syncthreads();
        int j = jt + threadIdx.x;
        if (j < j1) {
            sp[threadIdx.x] = a.gpos32[s0 + j];
            sag[threadIdx.x] = a.sph_agg[s0 + j];
        } else {
            sp[threadIdx.x] = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f);
            sag[threadIdx.x] = -1;
        }
        __syncthreads();
        if (jt < ehi && jt + BS > elo) {
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
            a.gpart[slot] = make_dbl4(sx, sy, sz, 0.0);
        }
    }
}

template <int BS, int IB>
__global__ void __launch_bounds__(BS) k_gravity64(Arrays a, Sizes z)
{
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
            a.gpart[slot] = make_dbl4(ax[k], ay[k], az[k], 0.0);
        }
    }
}

// Sum the j-range partials of piles that were split, in range order.
__global__ void k_grav_combine(Arrays a, Sizes z)
{
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
        dbl4 v = a.gpart[a.gpart_base[p] + (int64_t)c * S.ns + il];
        sx += v.x; sy += v.y; sz += v.z;
    }
    double gm = S.G * a.m64[i];
    a.fg[i] = make_dbl4(gm * sx, gm * sy, gm * sz, 0.0);
}

template <int BS, int IB>
static void launch_g(const Arrays &a, const Sizes &z, bool fp64, cudaStream_t st)
{
    if (fp64) k_gravity64<BS, IB><<<(unsigned)z.GI, BS, 0, st>>>(a, z);
    else k_gravity32<BS, IB><<<(unsigned)z.GI, BS, 0, st>>>(a, z);
}

void launch_gravity(const Arrays &a, const Sizes &z, bool fp64, int block, int ib, cudaStream_t st)
{
    if (z.GI == 0) return;
    if (block == 64 && ib == 1) launch_g<64, 1>(a, z, fp64, st);
    else if (block == 64 && ib == 2) launch_g<64, 2>(a, z, fp64, st);
    else if (block == 128 && ib == 1) launch_g<128, 1>(a, z, fp64, st);
    else if (block == 128 && ib == 2) launch_g<128, 2>(a, z, fp64, st);
    else if (block == 256 && ib == 1) launch_g<256, 1>(a, z, fp64, st);
    else launch_g<256, 2>(a, z, fp64, st);
    if (z.GP > 0) k_grav_combine<<<(unsigned)((z.N + 255) / 256), 256, 0, st>>>(a, z);
}

}  // namespace dem
