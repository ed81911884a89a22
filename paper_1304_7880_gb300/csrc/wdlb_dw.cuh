// Double-word arithmetic on the FP32 units ("float-float"): a value is the
// unevaluated sum hi + lo of two floats, about 48 significant bits.  Built
// from the error-free transformations of Knuth's two-sum, Dekker's fast
// two-sum (|a| >= |b|) and the product error that one fused multiply-add
// gives exactly.  Results are left unnormalised (|lo| may exceed ulp(hi)/2
// by a few ulps of lo): the next two-sum takes hi exactly and the final
// rounding (dw_round) adds lo back, so the pair keeps ~2^-44 of the larger
// operand, while skipping the fast two-sum after every operation saves three
// instructions each.  Addition is the short form, whose error is bounded
// relative to the larger operand: what a sum that cancels down to a small
// difference needs here.  Every sum and product is a round-to-nearest
// intrinsic, so contraction cannot change the error-free steps and a checked
// build computes the same bits.
//
// GB300 issues FP64 at 1/64 of its FP32 rate; each operation below costs 2 to
// 8 FP32 instructions (the division 12).
#pragma once

#include <cuda_runtime.h>

namespace wdlb {

struct dwf {
    float hi, lo;
};

// whether a collision arithmetic type is the double-word one
template <class A>
struct is_dw {
    static constexpr bool value = false;
};
template <>
struct is_dw<dwf> {
    static constexpr bool value = true;
};

__device__ __forceinline__ dwf dw_from(float a) { return dwf{a, 0.f}; }

// split of a double known at compile time (weights, small rationals): the
// compiler folds the FP64 arithmetic
__device__ __forceinline__ dwf dw_const(double a)
{
    const float h = float(a);
    return dwf{h, float(a - double(h))};
}

// host split of a run-time double into a pair of floats
inline void dw_split(double a, float out[2])
{
    out[0] = float(a);
    out[1] = float(a - double(out[0]));
}

__device__ __forceinline__ dwf dw_load(const float v[2]) { return dwf{v[0], v[1]}; }

__device__ __forceinline__ float dw_round(dwf a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ dwf fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return dwf{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dwf two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dwf{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dwf operator-(dwf a) { return dwf{-a.hi, -a.lo}; }

__device__ __forceinline__ dwf operator+(dwf a, dwf b)
{
    const dwf s = two_sum(a.hi, b.hi);
    return dwf{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ dwf operator+(dwf a, float b)
{
    const dwf s = two_sum(a.hi, b);
    return dwf{s.hi, __fadd_rn(s.lo, a.lo)};
}

__device__ __forceinline__ dwf operator+(float a, dwf b) { return b + a; }
__device__ __forceinline__ dwf operator-(dwf a, dwf b) { return a + (-b); }
__device__ __forceinline__ dwf operator-(dwf a, float b) { return a + (-b); }
__device__ __forceinline__ dwf operator-(float a, dwf b) { return (-b) + a; }

__device__ __forceinline__ dwf operator*(dwf a, dwf b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    const float t = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return dwf{p, __fadd_rn(e, t)};
}

__device__ __forceinline__ dwf operator*(dwf a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    return dwf{p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p))};
}

// a times a power of two (exact, away from underflow)
__device__ __forceinline__ dwf dw_scale2(dwf a, float s) { return dwf{__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)}; }

__device__ __forceinline__ dwf operator*(float a, dwf b) { return b * a; }

// product of two floats, exact
__device__ __forceinline__ dwf two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return dwf{p, __fmaf_rn(a, b, -p)};
}

// a / b: one correction of the float quotient (the remainder's two parts
// added first: unnormalised, its hi need not lead)
__device__ __forceinline__ dwf operator/(dwf a, dwf b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dwf r = a - b * q1;
    return fast_two_sum(q1, __fdiv_rn(__fadd_rn(r.hi, r.lo), b.hi));
}

__device__ __forceinline__ dwf &operator+=(dwf &a, dwf b) { return a = a + b; }
__device__ __forceinline__ dwf &operator+=(dwf &a, float b) { return a = a + b; }
__device__ __forceinline__ dwf &operator-=(dwf &a, float b) { return a = a - b; }

}  // namespace wdlb
