// Float-float ("double-single") arithmetic for the accuracy-critical parts of
// the Kron-STAP path: the temporal factor B, its leading eigenvectors U_B and
// the projection X F_B^T.  At 30-40 dB clutter-to-noise the projected residual
// is ~1e-2 of the clutter amplitude, so single-precision rounding of B or U_B
// alone moves T_v by ~1e-3 (Sec. 5 filter; measured against the FP64 oracle).
//
// A value is hi + lo with |lo| <= ulp(hi)/2.  The building blocks are the
// error-free transformations of Dekker (1971) and Knuth: two_prod via fused
// multiply-add and two_sum.  Every operation uses an explicit __f*_rn
// intrinsic so the compiler can neither contract nor reassociate it.
#pragma once
#include <cuda_runtime.h>

namespace kstap {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  // requires |a| >= |b| (or a == 0)
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ ff ff_make(float s, float c) {
  ff r;
  two_sum(s, c, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  ff r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  ff r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  float p, e;
  two_prod(a.hi, b, p, e);
  e = __fmaf_rn(a.lo, b, e);
  ff r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

// Long division with one correction step (Dekker): q1 = a/b, r = a - q1 b.
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = ff_sub(a, ff_mul_f(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  ff out;
  quick_two_sum(q1, q2, out.hi, out.lo);
  return out;
}

// One Newton correction on the single-precision square root (Dekker).
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (a.hi <= 0.f) return ff{0.f, 0.f};
  const float x = __fsqrt_rn(a.hi);
  float p, e;
  two_prod(x, x, p, e);
  const ff r = ff_sub(a, ff{p, e});
  const float c = __fdiv_rn(r.hi, __fmul_rn(2.f, x));
  ff out;
  quick_two_sum(x, c, out.hi, out.lo);
  return out;
}

// Running sum s + c of exact products: adds a * b (a, b single) exactly up to
// the final rounding of c.
__device__ __forceinline__ void acc_prod(float& s, float& c, float a, float b) {
  float p, e, t, f;
  two_prod(a, b, p, e);
  two_sum(s, p, t, f);
  s = t;
  c = __fadd_rn(c, __fadd_rn(f, e));
}

// s + c += (xh + xl) * y
__device__ __forceinline__ void acc_ffxf(float& s, float& c, float xh, float xl, float y) {
  acc_prod(s, c, xh, y);
  c = __fmaf_rn(xl, y, c);
}

// s + c += (xh + xl) * (yh + yl), dropping the lo*lo term
__device__ __forceinline__ void acc_ffxff(float& s, float& c, float xh, float xl, float yh,
                                          float yl) {
  acc_prod(s, c, xh, yh);
  c = __fmaf_rn(xh, yl, c);
  c = __fmaf_rn(xl, yh, c);
}

// ------------------------------------------------------- packed pairs ------
// Two independent single-precision lanes per instruction (f32x2, sm_100 and
// later).  Each lane is rounded exactly as the scalar __f*_rn operation.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  unsigned long long A, B, D;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(B));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(D));
  return r;
}

// acc_ffxf on a pair of lanes: S + C += (XH + XL) * Y per lane, with
// NXH = -XH.  The product error comes as -e = p - XH Y (exact), so no lane
// needs a separate negation; every lane's result equals the scalar acc_ffxf
// bit for bit.
__device__ __forceinline__ void acc_ffxf2(float2& S, float2& C, float2 XH, float2 NXH,
                                          float2 XL, float2 Y) {
  const float2 p = f2_mul(XH, Y);
  const float2 ne = f2_fma(NXH, Y, p);            // p - XH Y
  const float2 t = f2_add(S, p);                  // two_sum(S, p)
  const float2 bb = f2_sub(t, S);
  const float2 f = f2_add(f2_sub(S, f2_sub(t, bb)), f2_sub(p, bb));
  S = t;
  C = f2_add(C, f2_sub(f, ne));
  C = f2_fma(XL, Y, C);
}

// ------------------------------------------------------------ complex ------
struct cff {
  ff re, im;
};

__device__ __forceinline__ cff cff_zero() { return cff{{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ cff cff_add(cff a, cff b) {
  return cff{ff_add(a.re, b.re), ff_add(a.im, b.im)};
}
__device__ __forceinline__ cff cff_sub(cff a, cff b) {
  return cff{ff_sub(a.re, b.re), ff_sub(a.im, b.im)};
}
// a * b
__device__ __forceinline__ cff cff_mul(cff a, cff b) {
  return cff{ff_sub(ff_mul(a.re, b.re), ff_mul(a.im, b.im)),
             ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
// conj(a) * b
__device__ __forceinline__ cff cff_cmul(cff a, cff b) {
  return cff{ff_add(ff_mul(a.re, b.re), ff_mul(a.im, b.im)),
             ff_sub(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
__device__ __forceinline__ cff cff_scale(cff a, ff s) { return cff{ff_mul(a.re, s), ff_mul(a.im, s)}; }

// Warp all-reduce (sum) of a float-float value across the lanes of `mask`
// (full warp); every lane ends with the same result.
__device__ __forceinline__ ff ff_warp_sum(ff v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ff w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_add(v, w);
  }
  return v;
}

}  // namespace kstap
