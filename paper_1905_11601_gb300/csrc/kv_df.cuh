// Double-float arithmetic for the mixed-precision path: a value is an unevaluated pair of FP32
// numbers h + l, and every operation runs on the FP32 pipe (GB300's FP64 pipe runs at 1/64 of
// the FP32 rate and cannot keep up with HBM in the streaming kernels of the Krylov step).
//
// An FP64 value is split with integer operations only: the head is its leading 24 significant
// bits (exact), the remaining 29 bits rounded to 23 (half up), so the pair carries the value to
// within 2^-48 of its magnitude without a systematic bias (a truncated tail would scale every
// value by 1 - O(2^-47), and those errors add up over a long inner product instead of averaging
// out). Values below 2^-103 in magnitude become 0 (an absolute change of at most
// 2^-103); values at or above 2^128, Inf and NaN are outside the pair's range and become a NaN
// pair, so that a non-finite input shows up as a non-finite result instead of vanishing.
// Products are formed as head*head (exact, with the FMA error term) plus the two cross terms,
// and sums with an exact TwoSum on the leading words, so each operation carries a relative
// error of about 2^-46 of the magnitudes involved.
#pragma once

#include <cuda_runtime.h>

struct DF {
  float h, l;
};

__device__ __forceinline__ DF df_split(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  const unsigned int ex = (hi >> 20) & 0x7FFu;  // biased FP64 exponent
  DF r{0.0f, 0.0f};
  // 2^-103 <= |x| < 2^128: the head's FP32 exponent ex-896 and the tail's ex-919 are both normal
  if (ex - 920u <= 230u) {
    // head: FP32 exponent rebiased in place, then 23 fraction bits (20 from hi, 3 from lo)
    const unsigned int hb = __funnelshift_l(lo, hi - (896u << 20), 3) | (hi & 0x80000000u);
    // tail: lo bits 28..0 rounded (half up) to the 23 bits 28..6, m, as 2^k (1 + m 2^-23) - 2^k,
    // k the weight of lo bit 28 plus one (m = 2^23 after rounding up carries into the exponent:
    // 2^(k+1) - 2^k); the subtraction is exact
    const unsigned int eb = (hb & 0xFF800000u) - (23u << 23);
    const unsigned int m = ((lo & 0x1FFFFFFFu) + 0x20u) >> 6;
    r.h = __uint_as_float(hb);
    r.l = __fsub_rn(__uint_as_float(eb + m), __uint_as_float(eb));
  } else if (ex >= 1151u) {  // |x| >= 2^128, Inf, NaN
    r.h = __uint_as_float(0x7FC00000u);
    r.l = r.h;
  }
  return r;
}

// exact FP32 -> FP64 by bit manipulation (no FP64 instruction); FP32 denormals map to 0, Inf
// and NaN to Inf and NaN
__device__ __forceinline__ double df_f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int fe = (b >> 23) & 0xFFu;
  if (fe == 0u) return 0.0;
  const unsigned int eb = fe == 0xFFu ? 0x7FFu : fe - 127u + 1023u;
  const unsigned int hi = (b & 0x80000000u) | (eb << 20) | ((b & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)((b & 0x7u) << 29));
}

// the pair rounded to FP64 (one FP64 addition)
__device__ __forceinline__ double df_value(const DF a) { return df_f2d(a.h) + df_f2d(a.l); }

__device__ __forceinline__ DF df_neg(const DF a) { return DF{-a.h, -a.l}; }

// a + b: TwoSum of the heads, the tails added to the error, renormalised (Fast2Sum)
__device__ __forceinline__ DF df_add(const DF a, const DF b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bp = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bp)), __fsub_rn(b.h, bp));
  const float t = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, t);
  return DF{h, __fsub_rn(t, __fsub_rn(h, s))};
}

__device__ __forceinline__ DF df_sub(const DF a, const DF b) { return df_add(a, df_neg(b)); }

// a + b left unnormalised: the head is fl(a.h + b.h), the tail carries the exact TwoSum error of
// the heads plus both tails (|tail| may exceed ulp(head)/2 by a few ulps; the pair still holds
// the sum to about 2^-47 of |a| + |b|). For operands of products (DFAcc::fma takes such pairs).
__device__ __forceinline__ DF df_add_lazy(const DF a, const DF b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bp = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bp)), __fsub_rn(b.h, bp));
  return DF{s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

// a * c for an FP32 constant c (exact head product via FMA, tail product rounded)
__device__ __forceinline__ DF df_mul_f(const DF a, float c) {
  const float p = __fmul_rn(a.h, c);
  const float e = __fmaf_rn(a.h, c, -p);
  const float t = __fmaf_rn(a.l, c, e);
  const float h = __fadd_rn(p, t);
  return DF{h, __fsub_rn(t, __fsub_rn(h, p))};
}

// a * b (the a.l*b.l term, below 2^-46 of the product, is dropped)
__device__ __forceinline__ DF df_mul(const DF a, const DF b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.h, -p);
  const float t = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  const float h = __fadd_rn(p, t);
  return DF{h, __fsub_rn(t, __fsub_rn(h, p))};
}

// Running sum of products: S carries the exact running sum of the leading product words
// (TwoSum), C the FP32 sum of every error and tail term.
struct DFAcc {
  float S = 0.0f, C = 0.0f;
  __device__ __forceinline__ void start(const DF a) {
    S = a.h;
    C = a.l;
  }
  // += a*b (the a.l*b.l term is dropped)
  __device__ __forceinline__ void fma(const DF a, const DF b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.h, -p);
    const float t = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    const float s = __fadd_rn(S, p);
    const float bp = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    S = s;
    C = __fadd_rn(C, __fadd_rn(err, t));
  }
  __device__ __forceinline__ void fma(const float2 c, const DF x) { fma(DF{c.x, c.y}, x); }
  // the pair renormalised (TwoSum), so that |l| <= ulp(h)/2
  __device__ __forceinline__ DF pair() const {
    const float s = __fadd_rn(S, C);
    const float bp = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(C, bp));
    return DF{s, err};
  }
  __device__ __forceinline__ double value() const { return df_f2d(S) + df_f2d(C); }
};
