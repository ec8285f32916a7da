// Fixed-point arithmetic for the mixed path's linearised operator (kv_fixed.cu): every value is
// an integer multiple of a power of two, held as a pair of 32-bit integers, and every product
// is formed with 32 x 32 -> 64-bit integer multiply-adds into 64-bit accumulators. Integer sums
// are exact, so the only rounding is the conversion of each input to its grid of 2^-49 of the
// largest value (inputs, base state and the constant factors each on their own grid) and the
// final conversion to FP64. The functions are host-and-device so that the same arithmetic can be
// checked on the host.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define KV_HD __host__ __device__ __forceinline__
#else
#define KV_HD inline
#endif

// value = h * 2^24 + l. A converted value has 0 <= l < 2^24 and |h| <= 2^25; sums and small
// integer multiples of such pairs stay exact as long as both words fit 32 bits.
struct FX {
  int h, l;
};

constexpr int FX_BITS = 49;   // converted values: |v| < 2^49 units
constexpr int FX_SPLIT = 24;  // low word bits
// fx_of's shift base for a bound |x| < 2^e: r0 = fx_r0(e) (1075 = FP64 exponent bias + 52)
KV_HD constexpr int fx_r0(int e) { return 1075 - FX_BITS + e; }

KV_HD FX fx_add(FX a, FX b) { return FX{a.h + b.h, a.l + b.l}; }
KV_HD FX fx_sub(FX a, FX b) { return FX{a.h - b.h, a.l - b.l}; }
KV_HD FX fx_mul(FX a, int w) { return FX{a.h * w, a.l * w}; }
KV_HD FX fx_sum4(FX a, FX b, FX c, FX d) { return FX{a.h + b.h + c.h + d.h, a.l + b.l + c.l + d.l}; }
// w.m a + w.c b + w.p c for small integer weights
struct W3i {
  int m, c, p;
};
KV_HD FX fx_w3(W3i w, FX a, FX b, FX c) {
  return FX{w.m * a.h + w.c * b.h + w.p * c.h, w.m * a.l + w.c * b.l + w.p * c.l};
}

// Sum of products: H collects the high-word products (weight 2^48), M1 both cross products
// (weight 2^24); the low-word product (weight 1, below 2^-40 of one high-word unit per term) is
// left out. Two chains of multiply-adds; the equations below use two such accumulators in turn,
// so that the chains stay short.
struct FXAcc {
  long long H = 0, M1 = 0;
  KV_HD void mac(FX a, FX b) {
    H += (long long)a.h * b.h;
    M1 += (long long)a.h * b.l;
    M1 += (long long)a.l * b.h;
  }
};
// the sum of two accumulators in units of 2^48, the cross part rounded down
KV_HD long long fx_total(const FXAcc& a, const FXAcc& b) {
  return a.H + b.H + ((a.M1 + b.M1) >> FX_SPLIT);
}

KV_HD unsigned long long fx_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

KV_HD double fx_from_bits(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

// x on the grid of 2^(e - 49), for |x| < 2^e: round(x 2^(49 - e)) as a pair; r0 = fx_r0(e).
// With b the biased exponent of x, the value is its 53-bit significand shifted right by
// r = r0 - b >= 4, rounded half away from zero. Zero, subnormal values and values below half a
// unit give 0. (Non-finite inputs are caught before: the caller's bound e is then meaningless.)
KV_HD FX fx_of(double x, int r0) {
  const unsigned long long b = fx_bits(x);
  const int eb = (int)((b >> 52) & 0x7FF);
  const int r = r0 - eb;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long a = (eb == 0 || r < 1 || r > 60) ? 0ull : ((m >> (r - 1)) + 1ull) >> 1;
  const long long s = (b >> 63) ? -(long long)a : (long long)a;
  return FX{(int)(s >> FX_SPLIT), (int)(s & ((1ll << FX_SPLIT) - 1))};
}

// An integer (|t| < 2^63) as FP64, rounded to nearest
KV_HD double fx_to_double(long long t) {
#if defined(__CUDA_ARCH__)
  return __ll2double_rn(t);
#else
  return (double)t;
#endif
}

// Derivative weights as small integers. First derivative in units of 1/(6h): interior or face
// (-3, 0, 3), first cell next to a wall (-8, 6, 2), last cell (-2, -6, 8); second derivative in
// units of 1/h^2: (1, -2, 1), (2, -3, 1), (1, -3, 2) (wall nodes at h/2 from the cell centres).
KV_HD W3i fx_d1(int cls) { return cls == 0 ? W3i{-3, 0, 3} : (cls == 1 ? W3i{-8, 6, 2} : W3i{-2, -6, 8}); }
// First-order upwind (same units): the one-sided difference towards the upstream node over the
// node gap, backward where the selecting velocity is >= 0 (back), else forward; the gap to a wall
// node is h/2 (first cell backward, last cell forward).
KV_HD W3i fx_u1(int cls, bool back) {
  if (back) return cls == 1 ? W3i{-12, 12, 0} : W3i{-6, 6, 0};
  return cls == 2 ? W3i{0, -12, 12} : W3i{0, -6, 6};
}
// The face axis' weights of a velocity equation carry 4 (see the equations below): central
// 4 x (-3, 0, 3) as the multiplier of a difference, upwind 4 x the one-sided weights (faces are
// h apart everywhere).
KV_HD W3i fx_u1_face(bool back) { return back ? W3i{-24, 24, 0} : W3i{0, -24, 24}; }
KV_HD FX fx_face(int face, FX m, FX, FX p) { return fx_mul(fx_sub(p, m), face); }
KV_HD FX fx_face(W3i w, FX m, FX c, FX p) { return fx_w3(w, m, c, p); }
KV_HD W3i fx_d2(int cls) { return cls == 0 ? W3i{1, -2, 1} : (cls == 1 ? W3i{2, -3, 1} : W3i{1, -3, 2}); }
KV_HD int fx_class(int t, int n) { return t == 1 ? 1 : (t == n ? 2 : 0); }

// ---- the four equations of J P_BC x at one cell, in fixed point ------------------------------
//
// On a uniform cubic grid (h = 1/n on every axis) every term of the linearised operator (the
// discretisation of the FP64 kernels: diffusion in flux form, advection in advective form with
// 2- or 4-point averaged advecting velocities, buoyancy on the w-faces) is a product of a
// base-state quantity and an input quantity, each an exact integer combination of staged values,
// times a common factor -n/24:
//   u:  4U D1x(u) + S4V D1y(u) + S4W D1z(u) + 4u D1x(U) + S4v D1y(U) + S4w D1z(U) + Kd_m L(u)
//   v, w alike (w adds Kb (T + T_k+1)); T:  2 S2U D1x(T) + ... + 2 s2u D1x(Theta) + ... + Kd_e L(T)
// with D1 the first-derivative weights in units of 1/(6h), S4 / S2 the 4- / 2-point sums of the
// averaged velocities, L the second-derivative weights (units 1/h^2) summed over the axes, and
// the constants Kd_m = -24 nu n, Kd_e = -24 kappa n, Kb = -12/n on the base state's grid (K).
// Accessors: X(f, di, dj, dk) the projected input of field f (u, v, w, T) at the offset,
// B(f, di, dj, dk) the base state (U, V, W, Theta). face: the face axis' first derivative, 4 x its
// weights: central, an int multiplier of the difference (12, or 4 with the constants K divided by
// 3); upwind, a W3i (fx_u1_face). d1a, d2a: the derivative weights along axis a at the cell
// (fx_d1 / fx_d2 of its wall class, or fx_u1 with upwinding; constants for interior cells, so
// that the weighted sums reduce to differences). With upwinding, each axis' one-sided choice is
// the base velocity's, shared by the two advection terms that differentiate along that axis.
struct FxK {
  FX kd_m, kd_e, kb;  // on the base state's grid
};
// k1: the constants above. k3: the same divided by 3, for cells whose first-derivative weights
// are all the interior ones, which then run as (-1, 0, 1) (the factor 3 moves to the output).
struct FxConst {
  FxK k1, k3;
  double f0;  // -n/24 x 2^(E - 50): the result of a unit total for x on the grid 2^-49 (k1)
  int e;      // base state grid: |values| < 2^E
};

template <class XA, class BA, class FW>
KV_HD long long fx_eq_u(const XA& X, const BA& B, W3i d1y, W3i d2y, W3i d1z, W3i d2z, const FxK& K, FW face) {
  const FX u0 = X(0, 0, 0, 0), uxm = X(0, -1, 0, 0), uxp = X(0, 1, 0, 0), uym = X(0, 0, -1, 0),
           uyp = X(0, 0, 1, 0), uzm = X(0, 0, 0, -1), uzp = X(0, 0, 0, 1);
  const FX U0 = B(0, 0, 0, 0);
  FXAcc a, b;
  // x is the face axis: D1 = (-3, 0, 3); the own velocity carries 4 (the others are 4-point sums)
  a.mac(U0, fx_face(face, uxm, u0, uxp));
  b.mac(fx_sum4(B(1, 0, -1, 0), B(1, 0, 0, 0), B(1, 1, -1, 0), B(1, 1, 0, 0)), fx_w3(d1y, uym, u0, uyp));
  a.mac(fx_sum4(B(2, 0, 0, -1), B(2, 0, 0, 0), B(2, 1, 0, -1), B(2, 1, 0, 0)), fx_w3(d1z, uzm, u0, uzp));
  b.mac(u0, fx_face(face, B(0, -1, 0, 0), U0, B(0, 1, 0, 0)));
  a.mac(fx_sum4(X(1, 0, -1, 0), X(1, 0, 0, 0), X(1, 1, -1, 0), X(1, 1, 0, 0)),
        fx_w3(d1y, B(0, 0, -1, 0), U0, B(0, 0, 1, 0)));
  b.mac(fx_sum4(X(2, 0, 0, -1), X(2, 0, 0, 0), X(2, 1, 0, -1), X(2, 1, 0, 0)),
        fx_w3(d1z, B(0, 0, 0, -1), U0, B(0, 0, 0, 1)));
  const W3i d2x{1, -2, 1};
  a.mac(K.kd_m, fx_add(fx_add(fx_w3(d2x, uxm, u0, uxp), fx_w3(d2y, uym, u0, uyp)), fx_w3(d2z, uzm, u0, uzp)));
  return fx_total(a, b);
}

template <class XA, class BA, class FW>
KV_HD long long fx_eq_v(const XA& X, const BA& B, W3i d1x, W3i d2x, W3i d1z, W3i d2z, const FxK& K, FW face) {
  const FX v0 = X(1, 0, 0, 0), vxm = X(1, -1, 0, 0), vxp = X(1, 1, 0, 0), vym = X(1, 0, -1, 0),
           vyp = X(1, 0, 1, 0), vzm = X(1, 0, 0, -1), vzp = X(1, 0, 0, 1);
  const FX V0 = B(1, 0, 0, 0);
  FXAcc a, b;
  a.mac(fx_sum4(B(0, -1, 0, 0), B(0, 0, 0, 0), B(0, -1, 1, 0), B(0, 0, 1, 0)), fx_w3(d1x, vxm, v0, vxp));
  b.mac(V0, fx_face(face, vym, v0, vyp));
  a.mac(fx_sum4(B(2, 0, 0, -1), B(2, 0, 0, 0), B(2, 0, 1, -1), B(2, 0, 1, 0)), fx_w3(d1z, vzm, v0, vzp));
  b.mac(fx_sum4(X(0, -1, 0, 0), X(0, 0, 0, 0), X(0, -1, 1, 0), X(0, 0, 1, 0)),
        fx_w3(d1x, B(1, -1, 0, 0), V0, B(1, 1, 0, 0)));
  a.mac(v0, fx_face(face, B(1, 0, -1, 0), V0, B(1, 0, 1, 0)));
  b.mac(fx_sum4(X(2, 0, 0, -1), X(2, 0, 0, 0), X(2, 0, 1, -1), X(2, 0, 1, 0)),
        fx_w3(d1z, B(1, 0, 0, -1), V0, B(1, 0, 0, 1)));
  const W3i d2y{1, -2, 1};
  a.mac(K.kd_m, fx_add(fx_add(fx_w3(d2x, vxm, v0, vxp), fx_w3(d2y, vym, v0, vyp)), fx_w3(d2z, vzm, v0, vzp)));
  return fx_total(a, b);
}

template <class XA, class BA, class FW>
KV_HD long long fx_eq_w(const XA& X, const BA& B, W3i d1x, W3i d2x, W3i d1y, W3i d2y, const FxK& K, FW face) {
  const FX w0 = X(2, 0, 0, 0), wxm = X(2, -1, 0, 0), wxp = X(2, 1, 0, 0), wym = X(2, 0, -1, 0),
           wyp = X(2, 0, 1, 0), wzm = X(2, 0, 0, -1), wzp = X(2, 0, 0, 1);
  const FX W0 = B(2, 0, 0, 0);
  FXAcc a, b;
  a.mac(fx_sum4(B(0, -1, 0, 0), B(0, 0, 0, 0), B(0, -1, 0, 1), B(0, 0, 0, 1)), fx_w3(d1x, wxm, w0, wxp));
  b.mac(fx_sum4(B(1, 0, -1, 0), B(1, 0, 0, 0), B(1, 0, -1, 1), B(1, 0, 0, 1)), fx_w3(d1y, wym, w0, wyp));
  a.mac(W0, fx_face(face, wzm, w0, wzp));
  b.mac(fx_sum4(X(0, -1, 0, 0), X(0, 0, 0, 0), X(0, -1, 0, 1), X(0, 0, 0, 1)),
        fx_w3(d1x, B(2, -1, 0, 0), W0, B(2, 1, 0, 0)));
  a.mac(fx_sum4(X(1, 0, -1, 0), X(1, 0, 0, 0), X(1, 0, -1, 1), X(1, 0, 0, 1)),
        fx_w3(d1y, B(2, 0, -1, 0), W0, B(2, 0, 1, 0)));
  b.mac(w0, fx_face(face, B(2, 0, 0, -1), W0, B(2, 0, 0, 1)));
  const W3i d2z{1, -2, 1};
  a.mac(K.kd_m, fx_add(fx_add(fx_w3(d2x, wxm, w0, wxp), fx_w3(d2y, wym, w0, wyp)), fx_w3(d2z, wzm, w0, wzp)));
  b.mac(K.kb, fx_add(X(3, 0, 0, 0), X(3, 0, 0, 1)));  // buoyancy (T_k + T_k+1) / 2
  return fx_total(a, b);
}

template <class XA, class BA>
KV_HD long long fx_eq_t(const XA& X, const BA& B, W3i d1x, W3i d2x, W3i d1y, W3i d2y, W3i d1z, W3i d2z,
                        const FxK& K, int face) {
  const FX t0 = X(3, 0, 0, 0), txm = X(3, -1, 0, 0), txp = X(3, 1, 0, 0), tym = X(3, 0, -1, 0),
           typ = X(3, 0, 1, 0), tzm = X(3, 0, 0, -1), tzp = X(3, 0, 0, 1);
  const FX th0 = B(3, 0, 0, 0);
  FXAcc a, b;
  // 2-point averages: the sums carry 2 to share the factor -n/24 with the momentum equations
  a.mac(fx_mul(fx_add(B(0, -1, 0, 0), B(0, 0, 0, 0)), 2), fx_w3(d1x, txm, t0, txp));
  b.mac(fx_mul(fx_add(B(1, 0, -1, 0), B(1, 0, 0, 0)), 2), fx_w3(d1y, tym, t0, typ));
  a.mac(fx_mul(fx_add(B(2, 0, 0, -1), B(2, 0, 0, 0)), 2), fx_w3(d1z, tzm, t0, tzp));
  b.mac(fx_mul(fx_add(X(0, -1, 0, 0), X(0, 0, 0, 0)), 2), fx_w3(d1x, B(3, -1, 0, 0), th0, B(3, 1, 0, 0)));
  a.mac(fx_mul(fx_add(X(1, 0, -1, 0), X(1, 0, 0, 0)), 2), fx_w3(d1y, B(3, 0, -1, 0), th0, B(3, 0, 1, 0)));
  b.mac(fx_mul(fx_add(X(2, 0, 0, -1), X(2, 0, 0, 0)), 2), fx_w3(d1z, B(3, 0, 0, -1), th0, B(3, 0, 0, 1)));
  a.mac(K.kd_e, fx_add(fx_add(fx_w3(d2x, txm, t0, txp), fx_w3(d2y, tym, t0, typ)), fx_w3(d2z, tzm, t0, tzp)));
  return fx_total(a, b);
}
