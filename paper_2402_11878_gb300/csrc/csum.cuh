// Compensated FP32 sums for the reductions of the complex64 kernels.
//
// A running sum is carried as an unevaluated pair hi + lo of floats and each
// addition uses Knuth's TwoSum (The Art of Computer Programming, Vol. 2,
// Sec. 4.2.2), which returns the rounded sum and its exact rounding error:
//     s = a + b,  b' = s - a,  err = (a - (s - b')) + (b - b').
// The error terms are collected in lo, so the pair keeps about 48 bits of the
// running sum (the accuracy of an FP64 accumulation of FP32 values to within
// a few units of 2^-48) while every operation runs on the FP32 pipe, which on
// this GPU issues 64 times the FP64 rate.  The pair is widened to FP64 once,
// for the fixed-order reductions across blocks.
#pragma once

namespace vqe {

struct F32c {
    float hi, lo;
};

__device__ __forceinline__ F32c f32c_zero() { return F32c{0.f, 0.f}; }

// Exact: a + b = s + err.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// acc += v
__device__ __forceinline__ void f32c_add(F32c &acc, float v) {
    float s, e;
    two_sum(acc.hi, v, s, e);
    acc.hi = s;
    acc.lo += e;
}

// a + b of two pairs, renormalised so that |lo| stays below an ulp of hi.
__device__ __forceinline__ F32c f32c_add(F32c a, F32c b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    float s2, e2;
    two_sum(s, e, s2, e2);
    return F32c{s2, e2};
}

// a + b of two pairs without the final renormalisation (the tree levels of
// a block sum): the rounding error of hi joins lo, which stays a few ulps of
// hi over the five levels of a warp tree.
__device__ __forceinline__ F32c f32c_add_lazy(F32c a, F32c b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return F32c{s, e + (a.lo + b.lo)};
}

__device__ __forceinline__ F32c f32c_shfl_xor(unsigned mask, F32c v, int o) {
    return F32c{__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o)};
}

// Sum over the `lanes` (a power of two, <= 32) lanes of the warp, in a fixed
// butterfly order; every lane ends with the total.
__device__ __forceinline__ F32c f32c_warp_sum(F32c v, unsigned mask, int lanes) {
    for (int o = lanes >> 1; o > 0; o >>= 1) v = f32c_add(v, f32c_shfl_xor(mask, v, o));
    return v;
}

__device__ __forceinline__ double f32c_value(F32c v) { return (double)v.hi + (double)v.lo; }

}  // namespace vqe
