// devmath.cuh -- small device helpers: float3/double3 vectors and
// float-float ("double-float") arithmetic built only from correctly rounded
// FP32 operations.
//
// Float-float values are unevaluated sums hi + lo with |lo| <= ulp(hi)/2.
// The error-free transformations are the classical ones: Knuth's TwoSum
// (six additions), Dekker's FastTwoSum (for |a| >= |b|) and the FMA-based
// TwoProduct (p = a*b rounded, e = fma(a, b, -p) exact).  All steps use the
// _rn intrinsics so that the compiler never contracts or reorders them; the
// results are therefore bitwise reproducible in every kernel that inlines
// them, which the cell-list build relies on.
#pragma once

#include <cuda_runtime.h>

namespace dem {

// ---------------------------------------------------------------- float-float
struct ff {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    ff r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ ff ff_sub(ff a, ff b)
{
    ff nb = {-b.hi, -b.lo};
    return ff_add(a, nb);
}

// (R_hi + R_lo) . (b_hi + b_lo) for one row, to ~2^-44 relative.
__device__ __forceinline__ ff ff_dot3(const float *Rh, const float *Rl, float bx_h, float by_h,
                                      float bz_h, float bx_l, float by_l, float bz_l)
{
    float p0, e0, p1, e1, p2, e2;
    two_prod(Rh[0], bx_h, p0, e0);
    two_prod(Rh[1], by_h, p1, e1);
    two_prod(Rh[2], bz_h, p2, e2);
    float s, t1, t2;
    two_sum(p0, p1, s, t1);
    two_sum(s, p2, s, t2);
    float lo = __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(__fadd_rn(e0, e1), e2));
    float cross = __fmul_rn(Rh[0], bx_l);
    cross = __fmaf_rn(Rh[1], by_l, cross);
    cross = __fmaf_rn(Rh[2], bz_l, cross);
    cross = __fmaf_rn(Rl[0], bx_h, cross);
    cross = __fmaf_rn(Rl[1], by_h, cross);
    cross = __fmaf_rn(Rl[2], bz_h, cross);
    lo = __fadd_rn(lo, cross);
    ff r;
    fast_two_sum(s, lo, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    ff r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ ff ff_of(double x)
{
    ff r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - (double)r.hi);
    return r;
}

__device__ __forceinline__ double ff_value(ff v) { return (double)v.hi + (double)v.lo; }

// a + b for a float b
__device__ __forceinline__ ff ff_addf(ff a, float b)
{
    float s, e;
    two_sum(a.hi, b, s, e);
    e = __fadd_rn(e, a.lo);
    ff r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// The pair with lo cut (towards zero) to the bits an FP64 number holds below
// hi: multiples of 2^(e - 52), e the exponent of hi (lo = 0 when hi is below
// 2^-74).  Then hi + lo is exactly a double and splitting that double gives
// the same pair back, so a state read out as doubles and written back is
// bitwise the state it was.
__device__ __forceinline__ ff ff_canon(ff v)
{
    const int e = ((__float_as_int(v.hi) >> 23) & 255) - 127;
    if (e < -74) return ff{v.hi, 0.f};
    const float up = __int_as_float((52 - e + 127) << 23);   // 2^(52 - e)
    const float dn = __int_as_float((e - 52 + 127) << 23);   // 2^(e - 52)
    return ff{v.hi, __fmul_rn(truncf(__fmul_rn(v.lo, up)), dn)};
}

// A float-float pair stored in the 8 bytes of one FP64 slot (the mixed
// path's aggregate state), stored in the canonical form above.
__device__ __forceinline__ ff ldff(const double *p)
{
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return ff{v.x, v.y};
}
__device__ __forceinline__ void stff(double *p, ff v)
{
    const ff c = ff_canon(v);
    *reinterpret_cast<float2 *>(p) = make_float2(c.hi, c.lo);
}
__device__ __forceinline__ ff ff_of2(float2 v) { return ff{v.x, v.y}; }

// Rotation matrix (body -> space) of the unit quaternion q = (w, x, y, z) in
// float-float, to ~2^-44: the FP64 quaternion is split once and every product
// and sum is an error-free FP32 transformation (FP64 instructions are ~60
// times slower than FP32 ones on this part).
__device__ __forceinline__ void quat_to_R_ff(const double *q, float *Rh, float *Rl, float *qhi)
{
    const ff w = ff_of(q[0]), x = ff_of(q[1]), y = ff_of(q[2]), z = ff_of(q[3]);
    qhi[0] = w.hi; qhi[1] = x.hi; qhi[2] = y.hi; qhi[3] = z.hi;
    const ff xx = ff_mul(x, x), yy = ff_mul(y, y), zz = ff_mul(z, z);
    const ff xy = ff_mul(x, y), xz = ff_mul(x, z), yz = ff_mul(y, z);
    const ff wx = ff_mul(w, x), wy = ff_mul(w, y), wz = ff_mul(w, z);
    const ff one = {1.0f, 0.0f};
    auto twice = [](ff a) { return ff{2.0f * a.hi, 2.0f * a.lo}; };
    const ff R[9] = {ff_sub(one, twice(ff_add(yy, zz))), twice(ff_sub(xy, wz)), twice(ff_add(xz, wy)),
                     twice(ff_add(xy, wz)), ff_sub(one, twice(ff_add(xx, zz))), twice(ff_sub(yz, wx)),
                     twice(ff_sub(xz, wy)), twice(ff_add(yz, wx)), ff_sub(one, twice(ff_add(xx, yy)))};
    for (int k = 0; k < 9; ++k) { Rh[k] = R[k].hi; Rl[k] = R[k].lo; }
}

// The same from a float-float quaternion (no FP64 instruction at all).
__device__ __forceinline__ void quat_ff_to_R_ff(const ff *q, float *Rh, float *Rl)
{
    const ff w = q[0], x = q[1], y = q[2], z = q[3];
    const ff xx = ff_mul(x, x), yy = ff_mul(y, y), zz = ff_mul(z, z);
    const ff xy = ff_mul(x, y), xz = ff_mul(x, z), yz = ff_mul(y, z);
    const ff wx = ff_mul(w, x), wy = ff_mul(w, y), wz = ff_mul(w, z);
    const ff one = {1.0f, 0.0f};
    auto twice = [](ff a) { return ff{2.0f * a.hi, 2.0f * a.lo}; };
    const ff R[9] = {ff_sub(one, twice(ff_add(yy, zz))), twice(ff_sub(xy, wz)), twice(ff_add(xz, wy)),
                     twice(ff_add(xy, wz)), ff_sub(one, twice(ff_add(xx, zz))), twice(ff_sub(yz, wx)),
                     twice(ff_sub(xz, wy)), twice(ff_add(yz, wx)), ff_sub(one, twice(ff_add(xx, yy)))};
    for (int k = 0; k < 9; ++k) { Rh[k] = R[k].hi; Rl[k] = R[k].lo; }
}

// Running float-float sum (TwoSum of each term, rounding errors collected in
// the low word): FP32 terms added with ~FP64 accuracy on the FP32 units (the
// FP64 units of this part are ~60 times slower).
struct FFSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float s, e;
        two_sum(hi, v, s, e);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Low 32 bits of round((hi + lo) x 2^e), the float-float value scaled by a
// power of two (exact) and rounded to an integer: hi is rounded first (exact
// in 64-bit integers below 2^63), the remainder (hi - round(hi)) + lo is
// rounded second.  Two's-complement wrap-around keeps differences of nearby
// values exact.
// The remainder (hi + lo) x 2^e - round(...) goes to rem (|rem| <= 1/2).
__device__ __forceinline__ int ff_to_fixed(ff v, int e, float &rem)
{
    const float sc = __int_as_float((e + 127) << 23);   // 2^e
    const float h = __fmul_rn(v.hi, sc), l = __fmul_rn(v.lo, sc);
    const float hr = rintf(h);
    const long long i1 = __float2ll_rn(hr);
    const float t = __fadd_rn(__fsub_rn(h, hr), l);
    const float tr = rintf(t);
    rem = __fsub_rn(t, tr);
    const int i2 = __float2int_rn(tr);
    return (int)(unsigned)((unsigned long long)i1 + (unsigned long long)(long long)i2);
}

// Split a double into hi + lo floats.
__host__ __device__ __forceinline__ void split_d(double x, float &hi, float &lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// ---------------------------------------------------------------- vectors
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ double3 d3(double x, double y, double z) { return make_double3(x, y, z); }
__device__ __forceinline__ double3 operator+(double3 a, double3 b) { return d3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ double3 operator-(double3 a, double3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double3 operator-(double3 a) { return d3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ double3 operator*(double s, double3 a) { return d3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 cross(double3 a, double3 b)
{
    return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ double3 ld3(const double *p) { return d3(p[0], p[1], p[2]); }
__device__ __forceinline__ void st3(double *p, double3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }

// Rotation matrix (body -> space) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_R(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

__device__ __forceinline__ double3 mat_mul(const double *A, double3 x)
{
    return d3(A[0] * x.x + A[1] * x.y + A[2] * x.z, A[3] * x.x + A[4] * x.y + A[5] * x.z,
              A[6] * x.x + A[7] * x.y + A[8] * x.z);
}
__device__ __forceinline__ double3 mat_tmul(const double *A, double3 x)
{
    return d3(A[0] * x.x + A[3] * x.y + A[6] * x.z, A[1] * x.x + A[4] * x.y + A[7] * x.z,
              A[2] * x.x + A[5] * x.y + A[8] * x.z);
}

// FP32 copies of the above (increments and derivatives of the mixed path).
__device__ __forceinline__ void quat_to_Rf(const float *q, float *R)
{
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
__device__ __forceinline__ float3 mat_mulf(const float *A, float3 x)
{
    return f3(A[0] * x.x + A[1] * x.y + A[2] * x.z, A[3] * x.x + A[4] * x.y + A[5] * x.z,
              A[6] * x.x + A[7] * x.y + A[8] * x.z);
}
__device__ __forceinline__ float3 mat_tmulf(const float *A, float3 x)
{
    return f3(A[0] * x.x + A[3] * x.y + A[6] * x.z, A[1] * x.x + A[4] * x.y + A[7] * x.z,
              A[2] * x.x + A[5] * x.y + A[8] * x.z);
}

// Two float4 as one 32-byte store (256-bit global stores exist from sm_100 on);
// p must be 32-byte aligned.  One request per thread where two 16-byte
// stores would be two, for stores that scatter across a warp.
__device__ __forceinline__ void st_f4x2(float4 *p, float4 a, float4 b)
{
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "f"(a.x), "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// Two float4 from one 32-byte load; p must be 32-byte aligned.
__device__ __forceinline__ void ld_f4x2(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

__device__ __forceinline__ bool finite3(double3 v)
{
    return isfinite(v.x) && isfinite(v.y) && isfinite(v.z);
}

}  // namespace dem
