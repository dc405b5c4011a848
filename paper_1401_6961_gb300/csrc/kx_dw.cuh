// kx_dw.cuh -- double-word FP32 arithmetic ("dw"): a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant
// bits, computed entirely on the FP32 pipe.  On GB300 the FP32 pipe issues
// one warp-wide FMA per cycle and sub-partition while a warp-wide FP64 FMA
// occupies the FP64 pipe for about 64 cycles, so a double-word multiply-add
// of about 15 FP32 instructions is several times faster than an FP64 one.
//
// Building blocks (error-free transformations):
//   TwoSum(a, b)     s + t = a + b exactly (Knuth; 6 operations)
//   Fast2Sum(a, b)   the same when |a| >= |b| or a == 0 (Dekker; 3 operations)
//   TwoProd(a, b)    p + e = a * b exactly, e = fma(a, b, -p)
// Double-word operations after Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44 (2017): the "sloppy" sum (absolute error of
// order 2^-47 (|x| + |y|)), the product with the lo*lo term dropped
// (relative error below 5 * 2^-48), and products by a float.  The fused
// x * y + z used by the accumulations keeps the product unnormalised:
//   ph + pl = x * y (lo terms by FMA), then the sloppy sum with z.
// Reciprocal and square root take the FP32 result and one Newton step in
// double-word arithmetic (residual exact by FMA), about 2^-46 relative.
//
// `x * y` returns a lazy product; it becomes a dw when assigned, and `acc +=
// x * y`, `acc -= x * y`, `z + x * y` use the fused form.  So templated
// kernels written for float and double compile unchanged for dw.
#pragma once

#include <cuda_runtime.h>

namespace kx {

struct dw {
    float hi, lo;
    dw() = default;
    __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dw(int n) : hi((float)n), lo(0.f) {}
    // split of a double: hi = nearest float, lo = the rounded remainder
    __host__ __device__ dw(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = a + b;
    const float ap = s - b;
    const float bp = s - ap;
    return dw(s, (a - ap) + (b - bp));
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = a + b;
    return dw(s, b - (s - a));
}

// sloppy double-word sum
__device__ __forceinline__ dw dw_add(dw x, dw y) {
    const dw s = two_sum(x.hi, y.hi);
    const float w = s.lo + (x.lo + y.lo);
    return fast_two_sum(s.hi, w);
}
// x * y with the lo * lo term dropped
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    const float ch = x.hi * y.hi;
    const float cl1 = fmaf(x.hi, y.hi, -ch);
    const float cl2 = fmaf(x.lo, y.hi, x.hi * y.lo);
    return fast_two_sum(ch, cl1 + cl2);
}
__device__ __forceinline__ dw dw_mulf(dw x, float y) {
    const float ch = x.hi * y;
    const float cl = fmaf(x.lo, y, fmaf(x.hi, y, -ch));
    return fast_two_sum(ch, cl);
}
// x * y + z (product unnormalised, then the sloppy sum)
__device__ __forceinline__ dw dw_fma(dw x, dw y, dw z) {
    const float ph = x.hi * y.hi;
    const float pl = fmaf(x.lo, y.hi, fmaf(x.hi, y.lo, fmaf(x.hi, y.hi, -ph)));
    const dw s = two_sum(ph, z.hi);
    const float w = s.lo + (pl + z.lo);
    return fast_two_sum(s.hi, w);
}
__device__ __forceinline__ dw dw_neg(dw x) { return dw(-x.hi, -x.lo); }

// 1/x: y0 = 1/hi, one Newton step y0 + y0 (1 - x y0), residual by FMA
__device__ __forceinline__ dw dw_recip(dw x) {
    const float y = 1.0f / x.hi;
    const float e = fmaf(-x.lo, y, fmaf(-x.hi, y, 1.0f));
    return fast_two_sum(y, y * e);
}
// sqrt(x) for x > 0: y0 = sqrtf(hi), correction (x - y0^2) / (2 y0)
__device__ __forceinline__ dw dw_sqrt(dw x) {
    const float y = sqrtf(x.hi);
    if (!(y > 0.f)) return dw(y, 0.f);
    const float r = fmaf(-y, y, x.hi) + x.lo;
    return fast_two_sum(y, r * (0.5f / y));
}

// lazy product
struct dw_prod {
    dw x, y;
    __device__ __forceinline__ operator dw() const { return dw_mul(x, y); }
};

__device__ __forceinline__ dw_prod operator*(dw x, dw y) { return dw_prod{x, y}; }
__device__ __forceinline__ dw_prod operator*(dw_prod p, dw y) { return dw_prod{dw(p), y}; }
__device__ __forceinline__ dw_prod operator*(dw x, dw_prod p) { return dw_prod{x, dw(p)}; }
__device__ __forceinline__ dw_prod operator*(dw_prod p, dw_prod q) { return dw_prod{dw(p), dw(q)}; }
__device__ __forceinline__ dw operator+(dw x, dw y) { return dw_add(x, y); }
__device__ __forceinline__ dw operator+(dw z, dw_prod p) { return dw_fma(p.x, p.y, z); }
__device__ __forceinline__ dw operator+(dw_prod p, dw z) { return dw_fma(p.x, p.y, z); }
__device__ __forceinline__ dw operator+(dw_prod p, dw_prod q) { return dw_fma(p.x, p.y, dw(q)); }
__device__ __forceinline__ dw operator-(dw x) { return dw_neg(x); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ dw operator-(dw z, dw_prod p) { return dw_fma(dw_neg(p.x), p.y, z); }
__device__ __forceinline__ dw operator-(dw_prod p, dw z) { return dw_fma(p.x, p.y, dw_neg(z)); }
__device__ __forceinline__ dw operator/(dw x, dw y) { return dw_mul(x, dw_recip(y)); }
__device__ __forceinline__ dw& operator+=(dw& z, dw x) { return z = dw_add(z, x); }
__device__ __forceinline__ dw& operator+=(dw& z, dw_prod p) { return z = dw_fma(p.x, p.y, z); }
__device__ __forceinline__ dw& operator-=(dw& z, dw x) { return z = dw_add(z, dw_neg(x)); }
__device__ __forceinline__ dw& operator-=(dw& z, dw_prod p) { return z = dw_fma(dw_neg(p.x), p.y, z); }
__device__ __forceinline__ dw& operator*=(dw& z, dw x) { return z = dw_mul(z, x); }
__device__ __forceinline__ bool operator<(dw x, dw y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

// FP64 value of a double-word number (exact: both parts convert exactly)
__device__ __forceinline__ double dw_to_f64(dw x) { return (double)x.hi + (double)x.lo; }

// shuffle of both words
__device__ __forceinline__ dw shfl_up(unsigned mask, dw v, int d) {
    return dw(__shfl_up_sync(mask, v.hi, d), __shfl_up_sync(mask, v.lo, d));
}

}  // namespace kx
