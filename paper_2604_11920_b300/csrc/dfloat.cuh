// dfloat.cuh -- double-float ("df64") numbers for the FP64-accurate sweeps.
//
// A dfl holds the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2:
// about 48 significant bits (relative rounding ~2^-47), against FP64's 53.  On
// B300 the FP64 pipe is narrow (the plain FP64 sweeps are bound by it, not by
// HBM); dfl arithmetic runs on the FP32 pipe.  The operations are built from
// the classic error-free transforms:
//   two-sum      s + e = a + b exactly          (Knuth, TAOCP vol. 2, 4.2.2)
//   fast-two-sum s + e = a + b, |a| >= |b|      (Dekker 1971)
//   exact product p + e = a * b, e = fma(a, b, -p)
// combined as in the double-double arithmetic of Hida, Li and Bailey (2001),
// in the "sloppy" add (one two-sum on the high parts).  Every step uses the
// round-to-nearest intrinsics, so the compiler cannot contract or reorder it.
#pragma once

#include "common.cuh"

namespace pdst {

// keep the built-in overloads visible next to the dfl ones below
using ::__ldcg;
using ::__ldcs;
using ::__ldg;
using ::__shfl_sync;
using ::__shfl_xor_sync;

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfl(s, e);
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const dfl s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl &operator-=(dfl &a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl &operator*=(dfl &a, dfl b) { return a = a * b; }

// loads and shuffles of both halves
__device__ __forceinline__ dfl __ldg(const dfl *p) {
    const float2 t = ::__ldg(reinterpret_cast<const float2 *>(p));
    return dfl(t.x, t.y);
}
__device__ __forceinline__ dfl __ldcs(const dfl *p) {
    const float2 t = ::__ldcs(reinterpret_cast<const float2 *>(p));
    return dfl(t.x, t.y);
}
__device__ __forceinline__ dfl __ldcg(const dfl *p) {
    const float2 t = ::__ldcg(reinterpret_cast<const float2 *>(p));
    return dfl(t.x, t.y);
}
__device__ __forceinline__ dfl __shfl_xor_sync(unsigned mask, dfl v, int o) {
    return dfl(::__shfl_xor_sync(mask, v.hi, o), ::__shfl_xor_sync(mask, v.lo, o));
}
__device__ __forceinline__ dfl __shfl_sync(unsigned mask, dfl v, int src) {
    return dfl(::__shfl_sync(mask, v.hi, src), ::__shfl_sync(mask, v.lo, src));
}

}  // namespace pdst

// beside the other widen() overloads (global namespace)
__device__ __forceinline__ pdst::dfl widen(pdst::dfl v) { return v; }
