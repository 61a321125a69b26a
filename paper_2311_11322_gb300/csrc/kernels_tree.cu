// kernels_tree.cu -- tree gravity (the paper's gravity method, Sec. 2.1: a
// tree code with multipole expansions), as an option beside the direct sum.
//
// Per pile and step: a cubic box around the pile (min/max of the sphere
// centres), an implicit octree of depth D over it (level L has 8^L cells in
// Morton order, so the parent of cell m is m >> 3), spheres counted into the
// leaf cells and ordered by leaf (counting sort, each leaf ordered by home
// index, deterministic), leaf moments from their spheres and upper moments
// from 8 children: mass, centre of mass and the raw moments of ranks 2-4
// about the COM (shifted exactly from child to parent), kept for evaluation
// as their traceless parts -- quadrupole, octupole and hexadecapole, the
// expansion order of the paper's tree code (Sec. 2.1) -- then each warp
// walks the tree depth-first for 32 spheres at once.  A cell is accepted when
// the group of spheres is farther from its COM than size/theta +
// |COM - centre| (so no sphere is inside an accepted cell) and contributes
// the gradient of its multipole potential up to rank 4 (or rank 2, the
// cheaper option); an opened leaf is summed directly
// with Plummer softening, skipping the sphere itself and its aggregate mates
// (pairs inside one aggregate cancel in its totals, Sec. 2.2.3).  Mates that
// fall in an accepted distant cell are not removed: their share cancels in
// the aggregate totals to the accuracy of the expansion.  FP32 throughout
// (positions relative to the pile frame); the result is written to the same
// per-sphere gravity array as the direct sum.
#include "dem_internal.h"
#include "devmath.cuh"
#include "launch.cuh"

namespace dem {

// order-preserving map of floats to ints (min/max by integer atomics)
__device__ __forceinline__ int f2o(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ bool tree_pile(const Arrays &a, int p)
{
    return a.enabled[p] != 0 && a.pd[p].failed == 0 && a.ps[p].tD > 0;
}

// level offset inside a pile's node block: sum_{k<L} 8^k
__host__ __device__ __forceinline__ int64_t lvl_off(int L) { return ((int64_t)1 << (3 * L)) / 7; }

__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ff;
    v = (v | (v << 16)) & 0x030000ff;
    v = (v | (v << 8)) & 0x0300f00f;
    v = (v | (v << 4)) & 0x030c30c3;
    v = (v | (v << 2)) & 0x09249249;
    return v;
}

// One block per pile: reset the box and the leaf counts.
__global__ void k_tree_init(Arrays a, Sizes z)
{
    pdl_enter();
    const int p = blockIdx.x;
    if (p >= z.P || !tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    if (threadIdx.x < 3) {
        a.tbox[8 * p + threadIdx.x] = f2o(3.0e38f);
        a.tbox[8 * p + 3 + threadIdx.x] = f2o(-3.0e38f);
    }
    const int64_t nl = (int64_t)1 << (3 * S.tD);
    for (int64_t c = threadIdx.x; c < nl; c += blockDim.x) a.tleaf[S.tleaf0 + c] = make_int2(0, 0);
}

// Box of each pile: per warp, lanes of the same pile reduce their min/max
// first (piles are contiguous, so a warp holds one or two), then one atomic
// per warp and pile (min/max do not depend on the order).
__global__ void k_tree_box(Arrays a, Sizes z)
{
    pdl_enter();
    const unsigned FULL = 0xffffffffu;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = i < z.N ? a.sph_pile[i] : -1;
    const bool act = p >= 0 && tree_pile(a, p);
    const float4 x = act ? a.gpos32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned todo = __ballot_sync(FULL, act);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int pp = __shfl_sync(FULL, p, leader);
        const bool mine = act && p == pp;
        todo &= ~__ballot_sync(FULL, mine);
        int v[6] = {f2o(x.x), f2o(x.y), f2o(x.z), f2o(x.x), f2o(x.y), f2o(x.z)};
        if (!mine) {
            v[0] = v[1] = v[2] = 0x7fffffff;
            v[3] = v[4] = v[5] = (int)0x80000000;
        }
        for (int o = 16; o > 0; o >>= 1)
            for (int c = 0; c < 6; ++c) {
                const int u = __shfl_xor_sync(FULL, v[c], o);
                v[c] = c < 3 ? min(v[c], u) : max(v[c], u);
            }
        if ((threadIdx.x & 31) == leader)
            for (int c = 0; c < 6; ++c) {
                if (c < 3) atomicMin(&a.tbox[8 * pp + c], v[c]);
                else atomicMax(&a.tbox[8 * pp + c], v[c]);
            }
    }
}

// cube of the pile: lower corner and edge
__device__ __forceinline__ void tree_cube(const Arrays &a, int p, float3 &lo, float &edge)
{
    const int *b = a.tbox + 8 * p;
    lo = f3(o2f(b[0]), o2f(b[1]), o2f(b[2]));
    const float ex = o2f(b[3]) - lo.x, ey = o2f(b[4]) - lo.y, ez = o2f(b[5]) - lo.z;
    edge = fmaxf(fmaxf(ex, ey), fmaxf(ez, 1e-6f)) * 1.0001f;
}

__global__ void k_tree_keys(Arrays a, Sizes z)
{
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.N) return;
    const int p = a.sph_pile[i];
    if (!tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    float3 lo;
    float edge;
    tree_cube(a, p, lo, edge);
    const int n1 = 1 << S.tD;
    const float sc = (float)n1 / edge;
    const float4 x = a.gpos32[i];
    const int cx = min(max((int)((x.x - lo.x) * sc), 0), n1 - 1);
    const int cy = min(max((int)((x.y - lo.y) * sc), 0), n1 - 1);
    const int cz = min(max((int)((x.z - lo.z) * sc), 0), n1 - 1);
    const int key = (int)(spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2));
    a.tkey[i] = key;
    a.trank[i] = atomicAdd(&a.tleaf[S.tleaf0 + key].y, 1);
}

// One block of 1024 threads per pile: exclusive scan of the leaf counts.
__global__ void k_tree_scan(Arrays a, Sizes z)
{
    pdl_enter();
    const int p = blockIdx.x;
    if (p >= z.P || !tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    const int64_t nl = (int64_t)1 << (3 * S.tD);
    const int64_t per = (nl + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * per, b1 = min(nl, b0 + per);
    int loc = 0;
    for (int64_t c = b0; c < b1; ++c) loc += a.tleaf[S.tleaf0 + c].y;
    __shared__ int buf[1024];
    buf[threadIdx.x] = loc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int add = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += add;
        __syncthreads();
    }
    int run = buf[threadIdx.x] - loc;
    for (int64_t c = b0; c < b1; ++c) {
        int2 &L = a.tleaf[S.tleaf0 + c];
        L.x = run;
        run += L.y;
    }
}

__global__ void k_tree_scatter(Arrays a, Sizes z)
{
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.N) return;
    const int p = a.sph_pile[i];
    if (!tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    a.tsorted[S.s0 + a.tleaf[S.tleaf0 + a.tkey[i]].x + a.trank[i]] = (int32_t)(i - S.s0);
}

// The first position of each leaf orders the leaf by home index (insertion
// sort; leaves hold a handful of spheres): deterministic sums.
__global__ void k_tree_leaf_order(Arrays a, Sizes z)
{
    pdl_enter();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z.N) return;
    const int p = a.sph_pile[k];
    if (!tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    int32_t *srt = a.tsorted + S.s0;
    const int kl = (int)(k - S.s0);
    const int2 L = a.tleaf[S.tleaf0 + a.tkey[S.s0 + srt[kl]]];
    if (kl != L.x) return;
    for (int x = 1; x < L.y; ++x) {
        const int v = srt[L.x + x];
        int y = x - 1;
        while (y >= 0 && srt[L.x + y] > v) {
            srt[L.x + y + 1] = srt[L.x + y];
            --y;
        }
        srt[L.x + y + 1] = v;
    }
}

// Leaf-ordered copies of the spheres' positions (+mass) and aggregates, so
// that a leaf's spheres are contiguous for the moments and the walk.
__global__ void k_tree_gather(Arrays a, Sizes z)
{
    pdl_enter();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z.N) return;
    const int p = a.sph_pile[k];
    if (!tree_pile(a, p)) return;
    const int64_t s0 = a.ps[p].s0;
    const int i = a.tsorted[k];
    a.tpos[k] = a.gpos32[s0 + i];
    a.tagg[k] = a.sph_agg[s0 + i];
}

// ---- multipole moments up to the hexadecapole
// A symmetric tensor of rank n is kept as its (n+1)(n+2)/2 distinct
// components, component (a, b, c) having a x-, b y- and c z-indices, in the
// order of mono_idx.  Raw moments of a node about its COM, R_abc = sum m x^a
// y^b z^c (rank 1 vanishes), ranks 2..4 at offsets 0, 6, 16 (31 floats,
// traw: 8 float4 per node).  Node record (tnode: 9 float4 = 36 floats): COM
// 0..2, M 3, opening radius^2 4, then the evaluation tensors T_n = c_n
// detrace(R_n) of ranks 2, 3, 4 at 5, 11, 21 with c_n = (2n-1)!!/n!
// (3/2, 5/2, 35/8), so that the potential of the node at offset x from its
// COM is -G (M / r + sum_n T_n . x^n / r^(2n+1)).
constexpr int kNodeF4 = 9, kRawF4 = 8;
__host__ __device__ constexpr int mono_idx(int a, int b, int c)
{
    int n = a + b + c, i = 0;
    for (int aa = n; aa > a; --aa) i += n - aa + 1;
    return i + (n - a) - b;
}
__host__ __device__ constexpr int raw_off(int n) { return n == 2 ? 0 : n == 3 ? 6 : 16; }
__host__ __device__ constexpr int node_off(int n) { return n == 2 ? 5 : n == 3 ? 11 : 21; }
__host__ __device__ constexpr float binomf(int n, int k)
{
    return (k < 0 || k > n) ? 0.f : (k == 0 || k == n) ? 1.f : (n == 2 ? 2.f : n == 3 ? 3.f : (k == 2 ? 6.f : 4.f));
}
__host__ __device__ constexpr float factf(int n) { return n <= 1 ? 1.f : n == 2 ? 2.f : n == 3 ? 6.f : 24.f; }
// number of ways to pair up 4 indices so that both pairs have equal axes
__host__ __device__ constexpr float pairings4(int a, int b, int c)
{
    return ((a & 1) || (b & 1) || (c & 1)) ? 0.f : (a == 4 || b == 4 || c == 4) ? 3.f : 1.f;
}

__device__ __forceinline__ void powers4(float x, float *p)
{
    p[0] = 1.f;
    p[1] = x;
    p[2] = x * x;
    p[3] = p[2] * x;
    p[4] = p[2] * p[2];
}

// trace over one index pair of the rank-n raw moment, component f (rank n - 2)
template <int N>
__device__ __forceinline__ float trace1(const float *R, int fa, int fb, int fc)
{
    return R[raw_off(N) + mono_idx(fa + 2, fb, fc)] + R[raw_off(N) + mono_idx(fa, fb + 2, fc)] +
           R[raw_off(N) + mono_idx(fa, fb, fc + 2)];
}

// Evaluation tensors from raw moments: the traceless part of each rank
// (subtract the symmetrised traces: 1/(2n-1) of single traces, plus 1/35 of
// the double trace at rank 4), scaled by (2n-1)!!/n!.
template <int N>
__device__ __forceinline__ void detrace_scaled(const float *R, float *T)
{
    constexpr float cn = N == 2 ? 1.5f : N == 3 ? 2.5f : 4.375f;
    float W = 0.f;
    if (N == 4) W = trace1<4>(R, 2, 0, 0) + trace1<4>(R, 0, 2, 0) + trace1<4>(R, 0, 0, 2);
#pragma unroll
    for (int a = N; a >= 0; --a)
#pragma unroll
        for (int b = N - a; b >= 0; --b) {
            const int c = N - a - b;
            float tr = 0.f;
            if (a >= 2) tr += binomf(a, 2) * trace1<N>(R, a - 2, b, c);
            if (b >= 2) tr += binomf(b, 2) * trace1<N>(R, a, b - 2, c);
            if (c >= 2) tr += binomf(c, 2) * trace1<N>(R, a, b, c - 2);
            float v = R[raw_off(N) + mono_idx(a, b, c)] - tr * (1.f / (2 * N - 1));
            if (N == 4) v += pairings4(a, b, c) * W * (1.f / 35.f);
            T[node_off(N) - 5 + mono_idx(a, b, c)] = cn * v;
        }
}

__device__ __forceinline__ void put_node(const Arrays &a, int64_t n, float3 c, float M, const float *R,
                                         float ropen2)
{
    float nd[4 * kNodeF4];
    nd[0] = c.x; nd[1] = c.y; nd[2] = c.z; nd[3] = M; nd[4] = ropen2;
    detrace_scaled<2>(R, nd + 5);
    detrace_scaled<3>(R, nd + 5);
    detrace_scaled<4>(R, nd + 5);
    float4 *o = a.tnode + kNodeF4 * n;
#pragma unroll
    for (int k = 0; k < kNodeF4; ++k) o[k] = make_float4(nd[4 * k], nd[4 * k + 1], nd[4 * k + 2], nd[4 * k + 3]);
    float4 *r = a.traw + kRawF4 * n;
#pragma unroll
    for (int k = 0; k < kRawF4; ++k)
        r[k] = make_float4(R[4 * k], R[4 * k + 1], R[4 * k + 2], k == kRawF4 - 1 ? 0.f : R[4 * k + 3]);
}

// centre of cell m (Morton) at level L of pile p's cube
__device__ __forceinline__ float3 cell_centre(float3 lo, float edge, int L, uint32_t m)
{
    uint32_t x = 0, y = 0, zz = 0;
    for (int b = 0; b < L; ++b) {
        x |= ((m >> (3 * b)) & 1u) << b;
        y |= ((m >> (3 * b + 1)) & 1u) << b;
        zz |= ((m >> (3 * b + 2)) & 1u) << b;
    }
    const float s = edge / (float)(1 << L);
    return f3(lo.x + (x + 0.5f) * s, lo.y + (y + 0.5f) * s, lo.z + (zz + 0.5f) * s);
}

__device__ __forceinline__ float opening2(float3 com, float3 ctr, float size, float theta)
{
    const float dx = com.x - ctr.x, dy = com.y - ctr.y, dz = com.z - ctr.z;
    const float r = size / theta + sqrtf(dx * dx + dy * dy + dz * dz);
    return r * r;
}

// Leaf moments: one thread per leaf of every tree pile.
__global__ void k_tree_leaves(Arrays a, Sizes z)
{
    pdl_enter();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= z.TL) return;
    const int p = a.tleaf_pile[g];
    if (p < 0 || !tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    const uint32_t m = (uint32_t)(g - S.tleaf0);
    const int2 L = a.tleaf[g];
    const int64_t n = S.tnode0 + lvl_off(S.tD) + m;
    float R[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) R[k] = 0.f;
    if (L.y == 0) {
        put_node(a, n, f3(0, 0, 0), 0.f, R, 0.f);
        return;
    }
    const float4 *tp = a.tpos + S.s0;
    float M = 0.f;
    float3 c = f3(0, 0, 0);
    const float4 x0 = tp[L.x];
    for (int k = 0; k < L.y; ++k) {   // COM about the first sphere
        const float4 x = tp[L.x + k];
        M += x.w;
        c = c + x.w * f3(x.x - x0.x, x.y - x0.y, x.z - x0.z);
    }
    c = f3(x0.x, x0.y, x0.z) + (1.0f / M) * c;
    for (int k = 0; k < L.y; ++k) {
        const float4 x = tp[L.x + k];
        float px[5], py[5], pz[5];
        powers4(x.x - c.x, px);
        powers4(x.y - c.y, py);
        powers4(x.z - c.z, pz);
#pragma unroll
        for (int r = 2; r <= 4; ++r)
#pragma unroll
            for (int ea = r; ea >= 0; --ea)
#pragma unroll
                for (int eb = r - ea; eb >= 0; --eb) {
                    const int ec = r - ea - eb;
                    R[raw_off(r) + mono_idx(ea, eb, ec)] += x.w * (px[ea] * py[eb] * pz[ec]);
                }
    }
    float3 lo;
    float edge;
    tree_cube(a, p, lo, edge);
    const float size = edge / (float)(1 << S.tD);
    put_node(a, n, c, M, R, opening2(c, cell_centre(lo, edge, S.tD, m), size, S.theta));
}

// Moments of level L from the 8 children: raw moments shifted from each
// child's COM to the parent's, R_e += sum_{f <= e} C(e, f) R_child,f s^(e-f)
// with s = child COM - parent COM (rank-1 terms vanish about a COM), one
// thread per node of every tree pile deep enough.
__global__ void k_tree_up(Arrays a, Sizes z, int L)
{
    pdl_enter();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= z.TN) return;
    const int p = a.tnode_pile[g];
    if (p < 0 || !tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    if (L >= S.tD) return;
    const int64_t local = g - S.tnode0;
    const int64_t o = lvl_off(L);
    if (local < o || local >= o + ((int64_t)1 << (3 * L))) return;
    const uint32_t m = (uint32_t)(local - o);
    const int64_t c0 = S.tnode0 + lvl_off(L + 1) + 8 * (int64_t)m;
    float M = 0.f;
    float3 c = f3(0, 0, 0);
    for (int k = 0; k < 8; ++k) {
        const float4 A = a.tnode[kNodeF4 * (c0 + k)];
        M += A.w;
        c = c + A.w * f3(A.x, A.y, A.z);
    }
    float R[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) R[k] = 0.f;
    if (M == 0.f) {
        put_node(a, g, f3(0, 0, 0), 0.f, R, 0.f);
        return;
    }
    c = (1.0f / M) * c;
    for (int k = 0; k < 8; ++k) {
        const float4 A = a.tnode[kNodeF4 * (c0 + k)];
        if (A.w == 0.f) continue;
        float Rc[32];
        const float4 *r = a.traw + kRawF4 * (c0 + k);
#pragma unroll
        for (int q = 0; q < kRawF4; ++q) {
            const float4 v = r[q];
            Rc[4 * q] = v.x; Rc[4 * q + 1] = v.y; Rc[4 * q + 2] = v.z; Rc[4 * q + 3] = v.w;
        }
        float sx[5], sy[5], sz[5];
        powers4(A.x - c.x, sx);
        powers4(A.y - c.y, sy);
        powers4(A.z - c.z, sz);
#pragma unroll
        for (int n = 2; n <= 4; ++n)
#pragma unroll
            for (int ea = n; ea >= 0; --ea)
#pragma unroll
                for (int eb = n - ea; eb >= 0; --eb) {
                    const int ec = n - ea - eb;
                    float v = 0.f;
#pragma unroll
                    for (int fa = 0; fa <= ea; ++fa)
#pragma unroll
                        for (int fb = 0; fb <= eb; ++fb)
#pragma unroll
                            for (int fc = 0; fc <= ec; ++fc) {
                                const int deg = fa + fb + fc;
                                if (deg == 1) continue;
                                const float Rf = deg == 0 ? A.w : Rc[raw_off(deg) + mono_idx(fa, fb, fc)];
                                v += (binomf(ea, fa) * binomf(eb, fb) * binomf(ec, fc)) * Rf *
                                     (sx[ea - fa] * sy[eb - fb] * sz[ec - fc]);
                            }
                    R[raw_off(n) + mono_idx(ea, eb, ec)] += v;
                }
    }
    float3 lo;
    float edge;
    tree_cube(a, p, lo, edge);
    put_node(a, g, c, M, R, opening2(c, cell_centre(lo, edge, L, m), edge / (float)(1 << L), S.theta));
}

// traversal stack per warp: each round pops up to 32 cells and pushes at most
// 8 children of each, and cells of one level are all popped before their
// parents' remaining siblings, so at most 8 x 32 cells of each level below
// the walk's start wait on the stack: 256 x 4 = 1,024 for the deepest tree
#ifndef DEM_TREE_STACK
#define DEM_TREE_STACK 1024
#endif
constexpr int kTreeStack = DEM_TREE_STACK;
// the walk of each group of spheres is split over the subtrees at this level
#ifndef DEM_TREE_SPLIT_LEVEL
#define DEM_TREE_SPLIT_LEVEL 2
#endif
constexpr int kSplitL = DEM_TREE_SPLIT_LEVEL, kSplit = 1 << (3 * kSplitL);

// The node's multipoles up to rank ORDER on the sphere at x: a / G.  With u
// the unit vector from the node's COM to x and r the distance,
//   a / G = -M u / r^2 + sum_n (n T_n . u^(n-1) - (2n+1) (T_n . u^n) u) / r^(n+2),
// the gradient of the potential -G (M / r + sum_n T_n . x^n / r^(2n+1))
// (unit-vector form: no power of r above the sixth is formed).
template <int ORDER>
__device__ __forceinline__ void node_force(const float *nd, const float4 &x, float &ax, float &ay, float &az)
{
    const float dx = x.x - nd[0], dy = x.y - nd[1], dz = x.z - nd[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    const float ux = dx * inv, uy = dy * inv, uz = dz * inv;
    float px[5], py[5], pz[5];
    powers4(ux, px);
    powers4(uy, py);
    powers4(uz, pz);
    float tx = 0.f, ty = 0.f, tz = 0.f;   // sum_n t_n / r^(n-2), Horner in 1/r from the top rank
#pragma unroll
    for (int n = ORDER; n >= 2; --n) {
        const float *T = nd + node_off(n);
        float vx = 0.f, vy = 0.f, vz = 0.f;   // T_n . u^(n-1)
#pragma unroll
        for (int fa = n - 1; fa >= 0; --fa)
#pragma unroll
            for (int fb = n - 1 - fa; fb >= 0; --fb) {
                const int fc = n - 1 - fa - fb;
                const float w = (factf(n - 1) / (factf(fa) * factf(fb) * factf(fc))) * (px[fa] * py[fb] * pz[fc]);
                vx = fmaf(w, T[mono_idx(fa + 1, fb, fc)], vx);
                vy = fmaf(w, T[mono_idx(fa, fb + 1, fc)], vy);
                vz = fmaf(w, T[mono_idx(fa, fb, fc + 1)], vz);
            }
        const float sn = vx * ux + vy * uy + vz * uz;   // T_n . u^n
        const float k1 = (float)n, k2 = (float)(2 * n + 1);
        tx = tx * inv + (k1 * vx - k2 * sn * ux);
        ty = ty * inv + (k1 * vy - k2 * sn * uy);
        tz = tz * inv + (k1 * vz - k2 * sn * uz);
    }
    const float inv2 = inv * inv, M = nd[3];
    ax += inv2 * (tx * inv2 - M * ux);
    ay += inv2 * (ty * inv2 - M * uy);
    az += inv2 * (tz * inv2 - M * uz);
}

// One warp walks the tree for a group of 32 consecutive spheres in leaf order.  Each round takes up to 32 nodes off the warp's stack, one per lane,
// and tests them in parallel against the group's bounding box: a cell is
// accepted when the box is farther from its COM than its opening radius (so
// the test holds for every sphere of the group), an opened leaf is summed
// directly, any other opened cell pushes its 8 children.  Every lane then
// adds its own sphere's interaction with each accepted cell (cell data passed
// by shuffles) and with the spheres of each opened leaf, so the arithmetic
// has no divergence and the node loads of a round overlap.  Should the stack
// ever fill, the cell is taken as accepted and the pile gets DEM_FLAG_TREE.
// Groups are 32 consecutive spheres of one pile in leaf order, counted from
// the pile's first sphere, so a pile's result does not depend on the other
// piles of the batch.  The walk of each group is split over the kSplit
// subtrees at level kSplitL (one warp each, grid dimension y), so that many
// more warps hide the latency of the rounds; each writes its partial sum,
// k_tree_combine adds them in order.
#ifdef DEM_TREE_MINB
#define DEM_TREE_BOUNDS __launch_bounds__(32, DEM_TREE_MINB)
#else
#define DEM_TREE_BOUNDS __launch_bounds__(32)
#endif
template <int ORDER>
__global__ void DEM_TREE_BOUNDS k_tree_force(Arrays a, Sizes z)
{
    pdl_enter();
    // one warp per block: walks of very different lengths do not hold one
    // another's block resident
    __shared__ int st[kTreeStack];
    // accepted cells of a round (ranks above 2), then the spheres of its
    // opened leaves, staged for every lane
    constexpr int kStage = ORDER > 2 ? 32 * kNodeF4 : 128;
    __shared__ float4 stage[kStage];
    __shared__ int sagg[kStage];
    __shared__ int lbase[32], lfirst[32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int sub = blockIdx.y;   // subtree: cell sub at level kSplitL
    const int64_t wg = blockIdx.x;   // group
    if (wg >= z.TG) return;
    int lo = 0, hi = (int)z.P - 1;   // pile of the group
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.ps[mid].tg0 <= wg) lo = mid; else hi = mid - 1;
    }
    const int pp = lo;
    if (!tree_pile(a, pp)) return;   // uniform over the warp
    const PileStatic &S = a.ps[pp];
    const int64_t s0 = S.s0;
    const int ti = (int)(32 * (wg - S.tg0)) + lane;   // leaf-order position in the pile
    const bool mine = ti < S.ns;
    const int64_t k = s0 + ti;
    const float4 xi = mine ? a.tpos[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ai = mine ? a.tagg[k] : -2;
    // group box (lanes past the pile's end take lane 0's position)
    const float lx = __shfl_sync(FULL, xi.x, 0), ly = __shfl_sync(FULL, xi.y, 0),
                lz = __shfl_sync(FULL, xi.z, 0);
    float bx0 = mine ? xi.x : lx, by0 = mine ? xi.y : ly, bz0 = mine ? xi.z : lz;
    float bx1 = bx0, by1 = by0, bz1 = bz0;
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fminf(bx0, __shfl_xor_sync(FULL, bx0, o));
        by0 = fminf(by0, __shfl_xor_sync(FULL, by0, o));
        bz0 = fminf(bz0, __shfl_xor_sync(FULL, bz0, o));
        bx1 = fmaxf(bx1, __shfl_xor_sync(FULL, bx1, o));
        by1 = fmaxf(by1, __shfl_xor_sync(FULL, by1, o));
        bz1 = fmaxf(bz1, __shfl_xor_sync(FULL, bz1, o));
    }
    const float eps2 = (float)S.eps2;
    const int D = S.tD;
    const float4 *nodes = a.tnode + kNodeF4 * S.tnode0;
    const int2 *leaves = a.tleaf + S.tleaf0;
    const float4 *tp = a.tpos + s0;
    const int32_t *tg = a.tagg + s0;
    float ax = 0.f, ay = 0.f, az = 0.f;
    bool full = false;
    int sp = 1;
    if (lane == 0) st[0] = ((int)(lvl_off(kSplitL) + sub) << 3) | kSplitL;   // this warp's subtree
    __syncwarp();
    while (sp > 0) {
        const int cnt = min(sp, 32);
        const int e = lane < cnt ? st[sp - 1 - lane] : -1;
        sp -= cnt;
        __syncwarp();
        // test this lane's node
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A, C = A;
        bool acc = false, leaf = false, open = false;
        int2 lf = make_int2(0, 0);
        if (e >= 0) {
            const int n = e >> 3, L = e & 7;
            A = nodes[kNodeF4 * n];
            if (A.w != 0.f) {
                B = nodes[kNodeF4 * n + 1];   // opening radius^2, T2
                const float gx = fmaxf(fmaxf(bx0 - A.x, A.x - bx1), 0.f);
                const float gy = fmaxf(fmaxf(by0 - A.y, A.y - by1), 0.f);
                const float gz = fmaxf(fmaxf(bz0 - A.z, A.z - bz1), 0.f);
                acc = gx * gx + gy * gy + gz * gz > B.x;
                leaf = !acc && L == D;
                open = !acc && L < D;
                if (acc) C = nodes[kNodeF4 * n + 2];
                if (leaf) lf = leaves[n - lvl_off(D)];
            }
        }
        // push the children of opened cells (compacted); a full stack
        // turns the cell into an accepted one
        const unsigned om = __ballot_sync(FULL, open);
        const int need = 8 * __popc(om);
        if (sp + need > kTreeStack) {
            if (open) {
                acc = true;
                open = false;
                C = nodes[kNodeF4 * (e >> 3) + 2];
            }
            full = true;
        } else if (open) {
            const int n = e >> 3, L = e & 7;
            const int c0 = (int)(lvl_off(L + 1) + 8 * (n - lvl_off(L)));
            const int at = sp + 8 * __popc(om & below);
            for (int c = 0; c < 8; ++c) st[at + c] = ((c0 + 7 - c) << 3) | (L + 1);
        }
        if (sp + need <= kTreeStack) sp += need;
        __syncwarp();
        // accepted cells: every lane adds each of them (rank 2: the cell's 3
        // float4 passed by shuffles; higher ranks: its 9 float4 staged in
        // shared memory by the lane that accepted it)
        unsigned am = __ballot_sync(FULL, acc);
        if (ORDER > 2) {
            if (acc) {
                const float4 *nd = nodes + kNodeF4 * (e >> 3);
                stage[kNodeF4 * lane] = A;
                stage[kNodeF4 * lane + 1] = B;
                stage[kNodeF4 * lane + 2] = C;
#pragma unroll
                for (int q = 3; q < kNodeF4; ++q) stage[kNodeF4 * lane + q] = nd[q];
            }
            __syncwarp();
        }
        while (am) {
            const int b = __ffs(am) - 1;
            am &= am - 1;
            if (ORDER > 2) {
                float nd[4 * kNodeF4];
#pragma unroll
                for (int q = 0; q < kNodeF4; ++q) {
                    const float4 v = stage[kNodeF4 * b + q];
                    nd[4 * q] = v.x; nd[4 * q + 1] = v.y; nd[4 * q + 2] = v.z; nd[4 * q + 3] = v.w;
                }
                if (mine) node_force<ORDER>(nd, xi, ax, ay, az);
            } else {
                float nd[12];
                nd[0] = __shfl_sync(FULL, A.x, b); nd[1] = __shfl_sync(FULL, A.y, b);
                nd[2] = __shfl_sync(FULL, A.z, b); nd[3] = __shfl_sync(FULL, A.w, b);
                nd[4] = 0.f;
                nd[5] = __shfl_sync(FULL, B.y, b); nd[6] = __shfl_sync(FULL, B.z, b);
                nd[7] = __shfl_sync(FULL, B.w, b); nd[8] = __shfl_sync(FULL, C.x, b);
                nd[9] = __shfl_sync(FULL, C.y, b); nd[10] = __shfl_sync(FULL, C.z, b);
                nd[11] = 0.f;
                if (mine) node_force<2>(nd, xi, ax, ay, az);
            }
        }
        if (ORDER > 2) __syncwarp();
        // opened leaves: the spheres of all of them (leaves in lane order,
        // spheres in leaf order) are staged in shared memory kStage at a
        // time, one round of loads for the whole round's leaves, then every
        // lane adds each of them.  A sphere's own aggregate is skipped, and
        // with it the sphere itself.
        const int lcnt = leaf ? lf.y : 0;
        int incl = lcnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        if (total > 0) {
            lbase[lane] = incl - lcnt;   // first staged position of this lane's leaf
            lfirst[lane] = lf.x;        // first sphere of the leaf (leaf order)
            __syncwarp();
            for (int c0 = 0; c0 < total; c0 += kStage) {
                const int nb = min(kStage, total - c0);
                for (int t = lane; t < nb; t += 32) {
                    // the leaf holding staged position c0 + t: the last lane whose
                    // first staged position is not after it
                    const int g = c0 + t;
                    int lo2 = 0, hi2 = 31;
                    while (lo2 < hi2) {
                        const int mid = (lo2 + hi2 + 1) >> 1;
                        if (lbase[mid] <= g) lo2 = mid; else hi2 = mid - 1;
                    }
                    const int idx = lfirst[lo2] + (g - lbase[lo2]);
                    stage[t] = tp[idx];
                    sagg[t] = tg[idx];
                }
                __syncwarp();
                for (int u = 0; u < nb; ++u) {
                    const float4 xj = stage[u];
                    if (mine && sagg[u] != ai) {
                        const float ex = xj.x - xi.x, ey = xj.y - xi.y, ez = xj.z - xi.z;
                        const float q2 = fmaf(ez, ez, fmaf(ey, ey, fmaf(ex, ex, eps2)));
                        const float iv = rsqrtf(q2);
                        const float sj = xj.w * iv * iv * iv;
                        ax = fmaf(ex, sj, ax);
                        ay = fmaf(ey, sj, ay);
                        az = fmaf(ez, sj, az);
                    }
                }
                __syncwarp();
            }
        }
    }
    if (mine) a.tpart[(int64_t)sub * z.N + k] = make_float4(ax, ay, az, 0.f);
    if (full && lane == 0) atomicOr(&a.pd[pp].flags, DEM_FLAG_TREE);
}

// Sum the subtree partials of each sphere (float-float, fixed order).
__global__ void k_tree_combine(Arrays a, Sizes z)
{
    pdl_enter();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z.N) return;
    const int p = a.sph_pile[k];
    if (!tree_pile(a, p)) return;
    const PileStatic &S = a.ps[p];
    FFSum sx, sy, sz;
    for (int s = 0; s < kSplit; ++s) {
        const float4 v = a.tpart[(int64_t)s * z.N + k];
        sx.add(v.x); sy.add(v.y); sz.add(v.z);
    }
    const int i = a.tsorted[k];
    const double gm = S.G * a.m64[S.s0 + i];
    a.fg[S.s0 + i] = make_dbl4(gm * sx.value(), gm * sy.value(), gm * sz.value(), 0.0);
}

void launch_tree_gravity(const Arrays &a, const Sizes &z, int max_depth, int order, cudaStream_t st)
{
    if (z.N == 0 || z.TN == 0) return;
    const unsigned nb = (unsigned)((z.N + 255) / 256);
    launch_pdl(k_tree_init, (unsigned)z.P, 256, 0, st, a, z);
    launch_pdl(k_tree_box, nb, 256, 0, st, a, z);
    launch_pdl(k_tree_keys, nb, 256, 0, st, a, z);
    launch_pdl(k_tree_scan, (unsigned)z.P, 1024, 0, st, a, z);
    launch_pdl(k_tree_scatter, nb, 256, 0, st, a, z);
    launch_pdl(k_tree_leaf_order, nb, 256, 0, st, a, z);
    launch_pdl(k_tree_gather, nb, 256, 0, st, a, z);
    launch_pdl(k_tree_leaves, (unsigned)((z.TL + 127) / 128), 128, 0, st, a, z);
    for (int L = max_depth - 1; L >= 0; --L)
        launch_pdl(k_tree_up, (unsigned)((z.TN + 255) / 256), 256, 0, st, a, z, L);
    if (order == 2) launch_pdl(k_tree_force<2>, dim3((unsigned)z.TG, kSplit), 32, 0, st, a, z);
    else launch_pdl(k_tree_force<4>, dim3((unsigned)z.TG, kSplit), 32, 0, st, a, z);
    launch_pdl(k_tree_combine, nb, 256, 0, st, a, z);
}

}  // namespace dem
