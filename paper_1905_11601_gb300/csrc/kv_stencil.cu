// The linearised Boussinesq operator of Eqs (8)-(9) as used by Eqs (11)-(12), and the
// steady residual of Eqs (1)-(2), on the MAC grid (FP64), uniform or stretched by Eq (22).
//
// Discrete operators (the paper defers its schemes to its reference [11]; these are the
// readings this library implements):
//   diffusion  flux form ((f+ - f)/(x+ - x) - (f - f-)/(x - x-)) / w, w the control-volume
//              width (h on the uniform grid; the cell width at a cell-like node and the
//              distance between the adjacent cell centres at a face-like node when stretched);
//              wall nodes on the walls, cell centres at the midpoints of their faces;
//   advection  (a . grad) b in advective form: 3-point central derivative of b at b's node
//              (non-uniform next to a wall node), times a averaged (2 or 4 points) there;
//   buoyancy   T e_z on a w-face: mean of the two adjacent cell temperatures.
// One thread per padded index (i, j, k) writes the u, v and w entries at that index (the
// momentum right-hand side on interior faces, 0 elsewhere) and the projected temperature.
#include "kv_df.cuh"
#include "kv_internal.cuh"

namespace {

struct W3 {
  double m, c, p;
};

// first / second derivative weights at a cell-like index t = 1..n (wall nodes at h/2)
__device__ __forceinline__ W3 d1_cell(int t, int n, double ih) {
  if (t == 1) return {-4.0 / 3.0 * ih, ih, 1.0 / 3.0 * ih};
  if (t == n) return {-1.0 / 3.0 * ih, -ih, 4.0 / 3.0 * ih};
  return {-0.5 * ih, 0.0, 0.5 * ih};
}
__device__ __forceinline__ W3 d2_cell(int t, int n, double ih2) {
  if (t == 1) return {2.0 * ih2, -3.0 * ih2, ih2};
  if (t == n) return {ih2, -3.0 * ih2, 2.0 * ih2};
  return {ih2, -2.0 * ih2, ih2};
}
__device__ __forceinline__ W3 d1_face(double ih) { return {-0.5 * ih, 0.0, 0.5 * ih}; }
__device__ __forceinline__ W3 d2_face(double ih2) { return {ih2, -2.0 * ih2, ih2}; }

// Weights at padded index t along axis A: the stretched grid's tables (Eq 22) when STR, else the
// uniform formulas above.
template <int A>
__device__ __forceinline__ int ax_n(const KvGeom& g) {
  return A == 0 ? g.nx : (A == 1 ? g.ny : g.nz);
}
template <int A>
__device__ __forceinline__ double ax_ih(const KvGeom& g) {
  return A == 0 ? g.ihx : (A == 1 ? g.ihy : g.ihz);
}
template <int A>
__device__ __forceinline__ double ax_ih2(const KvGeom& g) {
  return ax_ih<A>(g) * ax_ih<A>(g);  // as the host's ihx2 etc.; formed here it keeps k_stencil unspilled
}
template <int A>
__device__ __forceinline__ W3 sw3(const KvGeom& g, const KvStretch& S, int row, int t) {
  const int L = ax_n<A>(g) + 2;
  const double* p = S.sw + S.swo[A] + row * L + t;
  return {__ldg(p), __ldg(p + L), __ldg(p + 2 * L)};
}
template <int A, bool STR>
__device__ __forceinline__ W3 wc1(const KvGeom& g, const KvStretch& S, int t) {
  return STR ? sw3<A>(g, S, KV_SW_C1, t) : d1_cell(t, ax_n<A>(g), ax_ih<A>(g));
}
template <int A, bool STR>
__device__ __forceinline__ W3 wc2(const KvGeom& g, const KvStretch& S, int t) {
  return STR ? sw3<A>(g, S, KV_SW_C2, t) : d2_cell(t, ax_n<A>(g), ax_ih2<A>(g));
}
template <int A, bool STR>
__device__ __forceinline__ W3 wf1(const KvGeom& g, const KvStretch& S, int t) {
  return STR ? sw3<A>(g, S, KV_SW_F1, t) : d1_face(ax_ih<A>(g));
}
template <int A, bool STR>
__device__ __forceinline__ W3 wf2(const KvGeom& g, const KvStretch& S, int t) {
  return STR ? sw3<A>(g, S, KV_SW_F2, t) : d2_face(ax_ih2<A>(g));
}

// First-order upwind weights on the uniform grid (KvGeom::adv): the one-sided difference towards
// the upstream node, backward where the selecting velocity s >= 0, over the node gap (h/2 between
// the first or last cell centre and its wall node, h elsewhere and between faces).
__device__ __forceinline__ W3 up_cell(int t, int n, double ih, double s) {
  if (s >= 0.0) {
    const double w = t == 1 ? 2.0 * ih : ih;
    return {-w, w, 0.0};
  }
  const double w = t == n ? 2.0 * ih : ih;
  return {0.0, -w, w};
}
__device__ __forceinline__ W3 up_face(double ih, double s) {
  return s >= 0.0 ? W3{-ih, ih, 0.0} : W3{0.0, -ih, ih};
}
// The selecting sum of a 4-point average, in a fixed order: the two entries at t-1 along the
// velocity's own axis, then the two at t (each pair: t, t+1 along the node's face axis). Only its
// sign is used.
__device__ __forceinline__ double sel4(double a, double b, double c, double d) { return ((a + b) + c) + d; }
// First-derivative weights of an advection term along axis A at a cell-like / face-like index t:
// central, or upwind by the selecting velocity s.
template <int A, bool STR>
__device__ __forceinline__ W3 adv_c(const KvGeom& g, const KvStretch& S, int t, double s) {
  if (!STR && g.adv) return up_cell(t, ax_n<A>(g), ax_ih<A>(g), s);
  return wc1<A, STR>(g, S, t);
}
template <int A, bool STR>
__device__ __forceinline__ W3 adv_f(const KvGeom& g, const KvStretch& S, int t, double s) {
  if (!STR && g.adv) return up_face(ax_ih<A>(g), s);
  return wf1<A, STR>(g, S, t);
}

__device__ __forceinline__ double ap(const W3& w, double fm, double f0, double fp) {
  return fma(w.m, fm, fma(w.c, f0, w.p * fp));
}

struct Grid {
  KvGeom g;
  __device__ __forceinline__ int at(int i, int j, int k) const { return i + g.X * (j + g.Y * k); }
  __device__ __forceinline__ bool dof_u(int i, int j, int k) const {
    return i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
  }
  __device__ __forceinline__ bool dof_v(int i, int j, int k) const {
    return i >= 1 && i <= g.nx && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz;
  }
  __device__ __forceinline__ bool dof_w(int i, int j, int k) const {
    return i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz - 1;
  }
};

// Loads of the input vector. PROJ: apply P_BC on the fly (velocity zero outside the interior
// faces; temperature projected onto the homogeneous BCs); otherwise raw.
template <bool PROJ>
struct Loader {
  Grid G;
  const double* __restrict__ u;
  const double* __restrict__ v;
  const double* __restrict__ w;
  const double* __restrict__ T;
  __device__ __forceinline__ double lu(int i, int j, int k) const {
    if (PROJ && !G.dof_u(i, j, k)) return 0.0;
    return __ldg(u + G.at(i, j, k));
  }
  __device__ __forceinline__ double lv(int i, int j, int k) const {
    if (PROJ && !G.dof_v(i, j, k)) return 0.0;
    return __ldg(v + G.at(i, j, k));
  }
  __device__ __forceinline__ double lw(int i, int j, int k) const {
    if (PROJ && !G.dof_w(i, j, k)) return 0.0;
    return __ldg(w + G.at(i, j, k));
  }
  __device__ __forceinline__ double lT(int i, int j, int k) const {
    if (!PROJ) return __ldg(T + G.at(i, j, k));
    const KvGeom& g = G.g;
    if (i < 1 || i > g.nx || k < 1 || k > g.nz) return 0.0;
    if (g.bc == KV_BC_CC) {
      if (j < 1 || j > g.ny) return 0.0;
      return __ldg(T + G.at(i, j, k));
    }
    int jw, jn;  // wall node and its interior neighbour
    if (j <= 1) {
      jw = 0;
      jn = 1;
    } else if (j >= g.ny) {
      jw = g.ny + 1;
      jn = g.ny;
    } else {
      return __ldg(T + G.at(i, j, k));
    }
    double tn = __ldg(T + G.at(i, jn, k));
    if (g.tproj == KV_TPROJ_OBLIQUE) return tn;
    return 0.5 * (tn + __ldg(T + G.at(i, jw, k)));
  }
};

// MODE 0: J P_BC x with (U, Theta) = base. MODE 1: steady residual F(S), S = base = x.
template <int MODE, bool STR>
__global__ void __launch_bounds__(256) k_stencil(KvGeom g, KvStretch S, const double* __restrict__ base,
                                                 const double* __restrict__ x, size_t P,
                                                 double* __restrict__ vstar, double* __restrict__ tout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  constexpr bool PROJ = (MODE == 0);
  Grid G{g};
  const int e = G.at(i, j, k);
  // base flow (raw) and input (projected in MODE 0)
  Loader<false> B{G, base, base + P, base + 2 * P, base + 3 * P};
  Loader<PROJ> Xl{G, x, x + P, x + 2 * P, x + 3 * P};

  // ---- u on the x-face (i, j, k) ----
  double ru = 0.0;
  if (G.dof_u(i, j, k)) {
    const W3 dx2 = wf2<0, STR>(g, S, i), dy2 = wc2<1, STR>(g, S, j), dz2 = wc2<2, STR>(g, S, k);
    const W3 dx1 = adv_f<0, STR>(g, S, i, B.lu(i, j, k));
    const W3 dy1 = adv_c<1, STR>(g, S, j, sel4(B.lv(i, j - 1, k), B.lv(i + 1, j - 1, k), B.lv(i, j, k), B.lv(i + 1, j, k)));
    const W3 dz1 = adv_c<2, STR>(g, S, k, sel4(B.lw(i, j, k - 1), B.lw(i + 1, j, k - 1), B.lw(i, j, k), B.lw(i + 1, j, k)));
    const double c = Xl.lu(i, j, k);
    const double xm = Xl.lu(i - 1, j, k), xp = Xl.lu(i + 1, j, k);
    const double ym = Xl.lu(i, j - 1, k), yp = Xl.lu(i, j + 1, k);
    const double zm = Xl.lu(i, j, k - 1), zp = Xl.lu(i, j, k + 1);
    const double lap = ap(dx2, xm, c, xp) + ap(dy2, ym, c, yp) + ap(dz2, zm, c, zp);
    const double Ua = B.lu(i, j, k);
    const double Va = 0.25 * (B.lv(i, j - 1, k) + B.lv(i, j, k) + B.lv(i + 1, j - 1, k) + B.lv(i + 1, j, k));
    const double Wa = 0.25 * (B.lw(i, j, k - 1) + B.lw(i, j, k) + B.lw(i + 1, j, k - 1) + B.lw(i + 1, j, k));
    double r = g.nu * lap - (Ua * ap(dx1, xm, c, xp) + Va * ap(dy1, ym, c, yp) + Wa * ap(dz1, zm, c, zp));
    if (MODE == 0) {
      const double va = 0.25 * (Xl.lv(i, j - 1, k) + Xl.lv(i, j, k) + Xl.lv(i + 1, j - 1, k) + Xl.lv(i + 1, j, k));
      const double wa = 0.25 * (Xl.lw(i, j, k - 1) + Xl.lw(i, j, k) + Xl.lw(i + 1, j, k - 1) + Xl.lw(i + 1, j, k));
      const double gx = ap(dx1, B.lu(i - 1, j, k), Ua, B.lu(i + 1, j, k));
      const double gy = ap(dy1, B.lu(i, j - 1, k), Ua, B.lu(i, j + 1, k));
      const double gz = ap(dz1, B.lu(i, j, k - 1), Ua, B.lu(i, j, k + 1));
      r -= c * gx + va * gy + wa * gz;
    }
    ru = r;
  }
  vstar[e] = ru;

  // ---- v on the y-face (i, j, k) ----
  double rv = 0.0;
  if (G.dof_v(i, j, k)) {
    const W3 dx2 = wc2<0, STR>(g, S, i), dy2 = wf2<1, STR>(g, S, j), dz2 = wc2<2, STR>(g, S, k);
    const W3 dx1 = adv_c<0, STR>(g, S, i, sel4(B.lu(i - 1, j, k), B.lu(i - 1, j + 1, k), B.lu(i, j, k), B.lu(i, j + 1, k)));
    const W3 dy1 = adv_f<1, STR>(g, S, j, B.lv(i, j, k));
    const W3 dz1 = adv_c<2, STR>(g, S, k, sel4(B.lw(i, j, k - 1), B.lw(i, j + 1, k - 1), B.lw(i, j, k), B.lw(i, j + 1, k)));
    const double c = Xl.lv(i, j, k);
    const double xm = Xl.lv(i - 1, j, k), xp = Xl.lv(i + 1, j, k);
    const double ym = Xl.lv(i, j - 1, k), yp = Xl.lv(i, j + 1, k);
    const double zm = Xl.lv(i, j, k - 1), zp = Xl.lv(i, j, k + 1);
    const double lap = ap(dx2, xm, c, xp) + ap(dy2, ym, c, yp) + ap(dz2, zm, c, zp);
    const double Ua = 0.25 * (B.lu(i - 1, j, k) + B.lu(i, j, k) + B.lu(i - 1, j + 1, k) + B.lu(i, j + 1, k));
    const double Va = B.lv(i, j, k);
    const double Wa = 0.25 * (B.lw(i, j, k - 1) + B.lw(i, j, k) + B.lw(i, j + 1, k - 1) + B.lw(i, j + 1, k));
    double r = g.nu * lap - (Ua * ap(dx1, xm, c, xp) + Va * ap(dy1, ym, c, yp) + Wa * ap(dz1, zm, c, zp));
    if (MODE == 0) {
      const double ua = 0.25 * (Xl.lu(i - 1, j, k) + Xl.lu(i, j, k) + Xl.lu(i - 1, j + 1, k) + Xl.lu(i, j + 1, k));
      const double wa = 0.25 * (Xl.lw(i, j, k - 1) + Xl.lw(i, j, k) + Xl.lw(i, j + 1, k - 1) + Xl.lw(i, j + 1, k));
      const double gx = ap(dx1, B.lv(i - 1, j, k), Va, B.lv(i + 1, j, k));
      const double gy = ap(dy1, B.lv(i, j - 1, k), Va, B.lv(i, j + 1, k));
      const double gz = ap(dz1, B.lv(i, j, k - 1), Va, B.lv(i, j, k + 1));
      r -= ua * gx + c * gy + wa * gz;
    }
    rv = r;
  }
  vstar[P + e] = rv;

  // ---- w on the z-face (i, j, k), with the buoyancy term T e_z ----
  double rw = 0.0;
  if (G.dof_w(i, j, k)) {
    const W3 dx2 = wc2<0, STR>(g, S, i), dy2 = wc2<1, STR>(g, S, j), dz2 = wf2<2, STR>(g, S, k);
    const W3 dx1 = adv_c<0, STR>(g, S, i, sel4(B.lu(i - 1, j, k), B.lu(i - 1, j, k + 1), B.lu(i, j, k), B.lu(i, j, k + 1)));
    const W3 dy1 = adv_c<1, STR>(g, S, j, sel4(B.lv(i, j - 1, k), B.lv(i, j - 1, k + 1), B.lv(i, j, k), B.lv(i, j, k + 1)));
    const W3 dz1 = adv_f<2, STR>(g, S, k, B.lw(i, j, k));
    const double c = Xl.lw(i, j, k);
    const double xm = Xl.lw(i - 1, j, k), xp = Xl.lw(i + 1, j, k);
    const double ym = Xl.lw(i, j - 1, k), yp = Xl.lw(i, j + 1, k);
    const double zm = Xl.lw(i, j, k - 1), zp = Xl.lw(i, j, k + 1);
    const double lap = ap(dx2, xm, c, xp) + ap(dy2, ym, c, yp) + ap(dz2, zm, c, zp);
    const double Ua = 0.25 * (B.lu(i - 1, j, k) + B.lu(i, j, k) + B.lu(i - 1, j, k + 1) + B.lu(i, j, k + 1));
    const double Va = 0.25 * (B.lv(i, j - 1, k) + B.lv(i, j, k) + B.lv(i, j - 1, k + 1) + B.lv(i, j, k + 1));
    const double Wa = B.lw(i, j, k);
    double r = g.nu * lap - (Ua * ap(dx1, xm, c, xp) + Va * ap(dy1, ym, c, yp) + Wa * ap(dz1, zm, c, zp));
    if (MODE == 0) {
      const double ua = 0.25 * (Xl.lu(i - 1, j, k) + Xl.lu(i, j, k) + Xl.lu(i - 1, j, k + 1) + Xl.lu(i, j, k + 1));
      const double va = 0.25 * (Xl.lv(i, j - 1, k) + Xl.lv(i, j, k) + Xl.lv(i, j - 1, k + 1) + Xl.lv(i, j, k + 1));
      const double gx = ap(dx1, B.lw(i - 1, j, k), Wa, B.lw(i + 1, j, k));
      const double gy = ap(dy1, B.lw(i, j - 1, k), Wa, B.lw(i, j + 1, k));
      const double gz = ap(dz1, B.lw(i, j, k - 1), Wa, B.lw(i, j, k + 1));
      r -= ua * gx + va * gy + c * gz;
      r += 0.5 * (Xl.lT(i, j, k) + Xl.lT(i, j, k + 1));
    } else {
      r += 0.5 * (B.lT(i, j, k) + B.lT(i, j, k + 1));
    }
    rw = r;
  }
  vstar[2 * P + e] = rw;

  // ---- T at the cell (i, j, k), then the temperature projection of Eq (21) ----
  const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
  if (cell) {
    const W3 dx2 = wc2<0, STR>(g, S, i), dy2 = wc2<1, STR>(g, S, j), dz2 = wc2<2, STR>(g, S, k);
    const W3 dx1 = adv_c<0, STR>(g, S, i, B.lu(i - 1, j, k) + B.lu(i, j, k));
    const W3 dy1 = adv_c<1, STR>(g, S, j, B.lv(i, j - 1, k) + B.lv(i, j, k));
    const W3 dz1 = adv_c<2, STR>(g, S, k, B.lw(i, j, k - 1) + B.lw(i, j, k));
    const double c = Xl.lT(i, j, k);
    const double xm = Xl.lT(i - 1, j, k), xp = Xl.lT(i + 1, j, k);
    const double ym = Xl.lT(i, j - 1, k), yp = Xl.lT(i, j + 1, k);
    const double zm = Xl.lT(i, j, k - 1), zp = Xl.lT(i, j, k + 1);
    const double lap = ap(dx2, xm, c, xp) + ap(dy2, ym, c, yp) + ap(dz2, zm, c, zp);
    const double Ua = 0.5 * (B.lu(i - 1, j, k) + B.lu(i, j, k));
    const double Va = 0.5 * (B.lv(i, j - 1, k) + B.lv(i, j, k));
    const double Wa = 0.5 * (B.lw(i, j, k - 1) + B.lw(i, j, k));
    double r = g.kappa * lap - (Ua * ap(dx1, xm, c, xp) + Va * ap(dy1, ym, c, yp) + Wa * ap(dz1, zm, c, zp));
    if (MODE == 0) {
      const double ua = 0.5 * (Xl.lu(i - 1, j, k) + Xl.lu(i, j, k));
      const double va = 0.5 * (Xl.lv(i, j - 1, k) + Xl.lv(i, j, k));
      const double wa = 0.5 * (Xl.lw(i, j, k - 1) + Xl.lw(i, j, k));
      const double th = B.lT(i, j, k);
      const double gx = ap(dx1, B.lT(i - 1, j, k), th, B.lT(i + 1, j, k));
      const double gy = ap(dy1, B.lT(i, j - 1, k), th, B.lT(i, j + 1, k));
      const double gz = ap(dz1, B.lT(i, j, k - 1), th, B.lT(i, j, k + 1));
      r -= ua * gx + va * gy + wa * gz;
    }
    if (g.bc == KV_BC_AA && (j == 1 || j == g.ny)) {
      // insulated wall pair: the wall node carries no equation (0 before the projection)
      const double t = (g.tproj == KV_TPROJ_OBLIQUE) ? r : 0.5 * r;
      tout[e] = t;
      tout[G.at(i, j == 1 ? 0 : g.ny + 1, k)] = t;
    } else {
      tout[e] = r;
    }
  } else {
    // walls, edges and corners: zero, except insulated wall nodes written by their neighbour
    const bool aa_wall = g.bc == KV_BC_AA && (j == 0 || j == g.ny + 1) && i >= 1 && i <= g.nx && k >= 1 &&
                         k <= g.nz;
    if (!aa_wall) tout[e] = 0.0;
  }
}

// ---- the linearised operator in assembled-coefficient form -----------------------------
//
// J is linear in x and its coefficients depend only on the base flow, so they are formed once
// per base flow (k_assemble) and every Krylov vector is a 15-point (velocity faces) / 13-point
// (cells) product (k_apply): 60 FP64 multiply-adds per cell instead of recomputing the
// interpolated velocities, base gradients and wall weights every time. Coefficient array q
// (KV_NCOEF of them, each a padded field) at entry e:
//   u-face  q = 0..6   own-field points (c, x-, x+, y-, y+, z-, z+)
//           q = 7, 8   factors of the 4-point sums of v and w around the face
//   v-face  q = 9..15, 16 (sum of u), 17 (sum of w)
//   w-face  q = 18..24, 25 (sum of u), 26 (sum of v); plus 0.5 (T_k + T_k+1) buoyancy
//   T-cell  q = 27..33, 34, 35, 36 (factors of the 2-point sums of u, v, w)
template <bool STR>
__global__ void __launch_bounds__(256) k_assemble(KvGeom g, KvStretch S, const double* __restrict__ base, size_t P,
                                                  double* __restrict__ coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  Grid G{g};
  const int e = G.at(i, j, k);
  Loader<false> B{G, base, base + P, base + 2 * P, base + 3 * P};
  double c[KV_NCOEF];
#pragma unroll
  for (int q = 0; q < KV_NCOEF; ++q) c[q] = 0.0;
  // own-field coefficients of nu Lap f - (a . grad) f - f_self * g_self
  auto own = [&](double* o, double diff, const W3& x1, const W3& x2, const W3& y1, const W3& y2, const W3& z1,
                 const W3& z2, double ax, double ay, double az, double gself) {
    o[1] = diff * x2.m - ax * x1.m;
    o[2] = diff * x2.p - ax * x1.p;
    o[3] = diff * y2.m - ay * y1.m;
    o[4] = diff * y2.p - ay * y1.p;
    o[5] = diff * z2.m - az * z1.m;
    o[6] = diff * z2.p - az * z1.p;
    o[0] = diff * (x2.c + y2.c + z2.c) - (ax * x1.c + ay * y1.c + az * z1.c) - gself;
  };
  if (G.dof_u(i, j, k)) {
    const W3 dx2 = wf2<0, STR>(g, S, i), dy2 = wc2<1, STR>(g, S, j), dz2 = wc2<2, STR>(g, S, k);
    const W3 dx1 = adv_f<0, STR>(g, S, i, B.lu(i, j, k));
    const W3 dy1 = adv_c<1, STR>(g, S, j, sel4(B.lv(i, j - 1, k), B.lv(i + 1, j - 1, k), B.lv(i, j, k), B.lv(i + 1, j, k)));
    const W3 dz1 = adv_c<2, STR>(g, S, k, sel4(B.lw(i, j, k - 1), B.lw(i + 1, j, k - 1), B.lw(i, j, k), B.lw(i + 1, j, k)));
    const double Ua = B.lu(i, j, k);
    const double Va = 0.25 * (B.lv(i, j - 1, k) + B.lv(i, j, k) + B.lv(i + 1, j - 1, k) + B.lv(i + 1, j, k));
    const double Wa = 0.25 * (B.lw(i, j, k - 1) + B.lw(i, j, k) + B.lw(i + 1, j, k - 1) + B.lw(i + 1, j, k));
    const double gx = ap(dx1, B.lu(i - 1, j, k), Ua, B.lu(i + 1, j, k));
    const double gy = ap(dy1, B.lu(i, j - 1, k), Ua, B.lu(i, j + 1, k));
    const double gz = ap(dz1, B.lu(i, j, k - 1), Ua, B.lu(i, j, k + 1));
    own(c + 0, g.nu, dx1, dx2, dy1, dy2, dz1, dz2, Ua, Va, Wa, gx);
    c[7] = -0.25 * gy;
    c[8] = -0.25 * gz;
  }
  if (G.dof_v(i, j, k)) {
    const W3 dx2 = wc2<0, STR>(g, S, i), dy2 = wf2<1, STR>(g, S, j), dz2 = wc2<2, STR>(g, S, k);
    const W3 dx1 = adv_c<0, STR>(g, S, i, sel4(B.lu(i - 1, j, k), B.lu(i - 1, j + 1, k), B.lu(i, j, k), B.lu(i, j + 1, k)));
    const W3 dy1 = adv_f<1, STR>(g, S, j, B.lv(i, j, k));
    const W3 dz1 = adv_c<2, STR>(g, S, k, sel4(B.lw(i, j, k - 1), B.lw(i, j + 1, k - 1), B.lw(i, j, k), B.lw(i, j + 1, k)));
    const double Ua = 0.25 * (B.lu(i - 1, j, k) + B.lu(i, j, k) + B.lu(i - 1, j + 1, k) + B.lu(i, j + 1, k));
    const double Va = B.lv(i, j, k);
    const double Wa = 0.25 * (B.lw(i, j, k - 1) + B.lw(i, j, k) + B.lw(i, j + 1, k - 1) + B.lw(i, j + 1, k));
    const double gx = ap(dx1, B.lv(i - 1, j, k), Va, B.lv(i + 1, j, k));
    const double gy = ap(dy1, B.lv(i, j - 1, k), Va, B.lv(i, j + 1, k));
    const double gz = ap(dz1, B.lv(i, j, k - 1), Va, B.lv(i, j, k + 1));
    own(c + 9, g.nu, dx1, dx2, dy1, dy2, dz1, dz2, Ua, Va, Wa, gy);
    c[16] = -0.25 * gx;
    c[17] = -0.25 * gz;
  }
  if (G.dof_w(i, j, k)) {
    const W3 dx2 = wc2<0, STR>(g, S, i), dy2 = wc2<1, STR>(g, S, j), dz2 = wf2<2, STR>(g, S, k);
    const W3 dx1 = adv_c<0, STR>(g, S, i, sel4(B.lu(i - 1, j, k), B.lu(i - 1, j, k + 1), B.lu(i, j, k), B.lu(i, j, k + 1)));
    const W3 dy1 = adv_c<1, STR>(g, S, j, sel4(B.lv(i, j - 1, k), B.lv(i, j - 1, k + 1), B.lv(i, j, k), B.lv(i, j, k + 1)));
    const W3 dz1 = adv_f<2, STR>(g, S, k, B.lw(i, j, k));
    const double Ua = 0.25 * (B.lu(i - 1, j, k) + B.lu(i, j, k) + B.lu(i - 1, j, k + 1) + B.lu(i, j, k + 1));
    const double Va = 0.25 * (B.lv(i, j - 1, k) + B.lv(i, j, k) + B.lv(i, j - 1, k + 1) + B.lv(i, j, k + 1));
    const double Wa = B.lw(i, j, k);
    const double gx = ap(dx1, B.lw(i - 1, j, k), Wa, B.lw(i + 1, j, k));
    const double gy = ap(dy1, B.lw(i, j - 1, k), Wa, B.lw(i, j + 1, k));
    const double gz = ap(dz1, B.lw(i, j, k - 1), Wa, B.lw(i, j, k + 1));
    own(c + 18, g.nu, dx1, dx2, dy1, dy2, dz1, dz2, Ua, Va, Wa, gz);
    c[25] = -0.25 * gx;
    c[26] = -0.25 * gy;
  }
  if (i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz) {
    const W3 dx2 = wc2<0, STR>(g, S, i), dy2 = wc2<1, STR>(g, S, j), dz2 = wc2<2, STR>(g, S, k);
    const W3 dx1 = adv_c<0, STR>(g, S, i, B.lu(i - 1, j, k) + B.lu(i, j, k));
    const W3 dy1 = adv_c<1, STR>(g, S, j, B.lv(i, j - 1, k) + B.lv(i, j, k));
    const W3 dz1 = adv_c<2, STR>(g, S, k, B.lw(i, j, k - 1) + B.lw(i, j, k));
    const double Ua = 0.5 * (B.lu(i - 1, j, k) + B.lu(i, j, k));
    const double Va = 0.5 * (B.lv(i, j - 1, k) + B.lv(i, j, k));
    const double Wa = 0.5 * (B.lw(i, j, k - 1) + B.lw(i, j, k));
    const double th = B.lT(i, j, k);
    const double gx = ap(dx1, B.lT(i - 1, j, k), th, B.lT(i + 1, j, k));
    const double gy = ap(dy1, B.lT(i, j - 1, k), th, B.lT(i, j + 1, k));
    const double gz = ap(dz1, B.lT(i, j, k - 1), th, B.lT(i, j, k + 1));
    own(c + 27, g.kappa, dx1, dx2, dy1, dy2, dz1, dz2, Ua, Va, Wa, 0.0);
    c[34] = -0.5 * gx;
    c[35] = -0.5 * gy;
    c[36] = -0.5 * gz;
  }
#pragma unroll
  for (int q = 0; q < KV_NCOEF; ++q) coef[(size_t)q * P + e] = c[q];
}

__device__ __forceinline__ double cf(const double* __restrict__ coef, size_t P, int q, int e) {
  return __ldg(coef + (size_t)q * P + e);
}

// y* = J P_BC x with the assembled coefficients; output as k_stencil<0, STR>.
__global__ void __launch_bounds__(256) k_apply(KvGeom g, const double* __restrict__ coef,
                                               const double* __restrict__ x, size_t P, double* __restrict__ vstar,
                                               double* __restrict__ tout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  Grid G{g};
  const int e = G.at(i, j, k);
  Loader<true> X{G, x, x + P, x + 2 * P, x + 3 * P};
  double ru = 0.0, rv = 0.0, rw = 0.0;
  if (G.dof_u(i, j, k)) {
    ru = cf(coef, P, 0, e) * X.lu(i, j, k) + cf(coef, P, 1, e) * X.lu(i - 1, j, k) +
         cf(coef, P, 2, e) * X.lu(i + 1, j, k) + cf(coef, P, 3, e) * X.lu(i, j - 1, k) +
         cf(coef, P, 4, e) * X.lu(i, j + 1, k) + cf(coef, P, 5, e) * X.lu(i, j, k - 1) +
         cf(coef, P, 6, e) * X.lu(i, j, k + 1) +
         cf(coef, P, 7, e) * (X.lv(i, j - 1, k) + X.lv(i, j, k) + X.lv(i + 1, j - 1, k) + X.lv(i + 1, j, k)) +
         cf(coef, P, 8, e) * (X.lw(i, j, k - 1) + X.lw(i, j, k) + X.lw(i + 1, j, k - 1) + X.lw(i + 1, j, k));
  }
  vstar[e] = ru;
  if (G.dof_v(i, j, k)) {
    rv = cf(coef, P, 9, e) * X.lv(i, j, k) + cf(coef, P, 10, e) * X.lv(i - 1, j, k) +
         cf(coef, P, 11, e) * X.lv(i + 1, j, k) + cf(coef, P, 12, e) * X.lv(i, j - 1, k) +
         cf(coef, P, 13, e) * X.lv(i, j + 1, k) + cf(coef, P, 14, e) * X.lv(i, j, k - 1) +
         cf(coef, P, 15, e) * X.lv(i, j, k + 1) +
         cf(coef, P, 16, e) * (X.lu(i - 1, j, k) + X.lu(i, j, k) + X.lu(i - 1, j + 1, k) + X.lu(i, j + 1, k)) +
         cf(coef, P, 17, e) * (X.lw(i, j, k - 1) + X.lw(i, j, k) + X.lw(i, j + 1, k - 1) + X.lw(i, j + 1, k));
  }
  vstar[P + e] = rv;
  if (G.dof_w(i, j, k)) {
    rw = cf(coef, P, 18, e) * X.lw(i, j, k) + cf(coef, P, 19, e) * X.lw(i - 1, j, k) +
         cf(coef, P, 20, e) * X.lw(i + 1, j, k) + cf(coef, P, 21, e) * X.lw(i, j - 1, k) +
         cf(coef, P, 22, e) * X.lw(i, j + 1, k) + cf(coef, P, 23, e) * X.lw(i, j, k - 1) +
         cf(coef, P, 24, e) * X.lw(i, j, k + 1) +
         cf(coef, P, 25, e) * (X.lu(i - 1, j, k) + X.lu(i, j, k) + X.lu(i - 1, j, k + 1) + X.lu(i, j, k + 1)) +
         cf(coef, P, 26, e) * (X.lv(i, j - 1, k) + X.lv(i, j, k) + X.lv(i, j - 1, k + 1) + X.lv(i, j, k + 1)) +
         0.5 * (X.lT(i, j, k) + X.lT(i, j, k + 1));
  }
  vstar[2 * P + e] = rw;
  const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
  if (cell) {
    const double r = cf(coef, P, 27, e) * X.lT(i, j, k) + cf(coef, P, 28, e) * X.lT(i - 1, j, k) +
                     cf(coef, P, 29, e) * X.lT(i + 1, j, k) + cf(coef, P, 30, e) * X.lT(i, j - 1, k) +
                     cf(coef, P, 31, e) * X.lT(i, j + 1, k) + cf(coef, P, 32, e) * X.lT(i, j, k - 1) +
                     cf(coef, P, 33, e) * X.lT(i, j, k + 1) + cf(coef, P, 34, e) * (X.lu(i - 1, j, k) + X.lu(i, j, k)) +
                     cf(coef, P, 35, e) * (X.lv(i, j - 1, k) + X.lv(i, j, k)) +
                     cf(coef, P, 36, e) * (X.lw(i, j, k - 1) + X.lw(i, j, k));
    if (g.bc == KV_BC_AA && (j == 1 || j == g.ny)) {
      const double t = (g.tproj == KV_TPROJ_OBLIQUE) ? r : 0.5 * r;
      tout[e] = t;
      tout[G.at(i, j == 1 ? 0 : g.ny + 1, k)] = t;
    } else {
      tout[e] = r;
    }
  } else {
    const bool aa_wall = g.bc == KV_BC_AA && (j == 0 || j == g.ny + 1) && i >= 1 && i <= g.nx && k >= 1 &&
                         k <= g.nz;
    if (!aa_wall) tout[e] = 0.0;
  }
}

// ---- the same operator on the FP32 pipe (mixed precision) ----------------------------------
//
// GB300's FP64 pipe runs at 1/64 of its FP32 rate, so the mixed path evaluates J x in
// double-float arithmetic (kv_df.cuh): every coefficient is stored as an FP32 pair, the
// projected input is split into pairs once per evaluation, and each product is accumulated with
// an exact FP32 product (FMA error term), an exact running sum (TwoSum) and a small FP32
// correction. The result carries about 2^-44 of the sum of the term magnitudes; the only FP64
// instruction per output is the final addition of the two FP32 halves.

// P_BC x (the input projection of Eq (13)) at every stored entry, split into FP32 pairs: the
// operator below then loads each input value as a ready pair, with no masks and no splitting.
__global__ void __launch_bounds__(256) k_split_input(KvGeom g, const double* __restrict__ x, size_t P,
                                                     float2* __restrict__ xs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  Grid G{g};
  const Loader<true> L{G, x, x + P, x + 2 * P, x + 3 * P};
  const int e = G.at(i, j, k);
  const DF u = df_split(L.lu(i, j, k)), v = df_split(L.lv(i, j, k)), w = df_split(L.lw(i, j, k)),
           t = df_split(L.lT(i, j, k));
  xs[e] = make_float2(u.h, u.l);
  xs[P + e] = make_float2(v.h, v.l);
  xs[2 * P + e] = make_float2(w.h, w.l);
  xs[3 * P + e] = make_float2(t.h, t.l);
}

// Own-field coefficients in pairs: along one axis, the "plus" coefficient of an equation is an
// affine function of its "minus" coefficient, c+ = alpha + beta c-, with beta = -1 (interior),
// -1/4 (first cell next to a wall) or -4 (last cell) and alpha = 2, 3/2 or 6 times diff / h^2
// (diff = nu for the momentum equations, kappa for the energy equation): both come from the same
// advecting velocity a through the derivative weights of d1_cell / d2_cell / d1_face / d2_face,
// c- = diff d2.m - a d1.m and c+ = diff d2.p - a d1.p. So the double-float operator stores c-
// only and forms c- x- + c+ x+ = c- (x- + beta x+) + alpha x+ (beta is a power of two: the
// scaled pair is exact). alpha[d][axis][class]: d = 0 momentum, 1 energy; class 0 interior or
// face axis, 1 first cell, 2 last cell.
struct DfAlpha {
  float2 a[2][3][3];
};

__device__ __forceinline__ int wall_class(int t, int n) { return t == 1 ? 1 : (t == n ? 2 : 0); }

__device__ __forceinline__ float2 alpha_of(const DfAlpha& al, int d, int axis, int cls) {
  const float2 a0 = al.a[d][axis][0], a1 = al.a[d][axis][1], a2 = al.a[d][axis][2];
  return cls == 0 ? a0 : (cls == 1 ? a1 : a2);
}

__device__ __forceinline__ float beta_of(int cls) { return cls == 0 ? -1.0f : (cls == 1 ? -0.25f : -4.0f); }

// a += c- x- + c+ x+ along one axis (see DfAlpha)
__device__ __forceinline__ void own_axis(DFAcc& a, const float2 cm, const DF xm, const DF xp, const float2 alpha,
                                         const float beta) {
  a.fma(cm, df_add_lazy(xm, DF{beta * xp.h, beta * xp.l}));
  a.fma(alpha, xp);
}

// Inputs that share a coefficient (the cross terms' 2- and 4-point sums, the buoyancy average)
// are summed before the one product.
__device__ __forceinline__ DF sum4(const DF a, const DF b, const DF c, const DF d) {
  return df_add_lazy(df_add_lazy(df_add_lazy(a, b), c), d);
}

// Double-float coefficient q (KV_NCOEF_DF of them) = assembled coefficient kDfFromFull[q]: per
// equation the centre, the three minus coefficients and the cross-term factors.
__constant__ int kDfFromFull[KV_NCOEF_DF] = {0,  1,  3,  5,  7,  8,  9,  10, 12, 14, 16, 17, 18,
                                             19, 21, 23, 25, 26, 27, 28, 30, 32, 34, 35, 36};

// Assembled coefficient of each plus neighbour (x+, y+, z+ of u, v, w, T), which the operator of a
// stretched grid reads directly (there beta is not a power of two, so c+ is not rebuilt from c-),
// and so does the operator with upwind advection (its c+ is not alpha + beta c- either).
__constant__ int kPlusFromFull[KV_NCOEF_DFP] = {2, 4, 6, 11, 13, 15, 20, 22, 24, 29, 31, 33};

// y* = J P_BC x with the FP32-pair coefficients and the split projected input xs (output as
// k_apply). STR (stretched grid, or upwind advection): the plus coefficients come from cplus (KV_NCOEF_DFP pairs per
// point) instead of alpha + beta c-. One thread per (cell, equation): threadIdx.y = 4 row + eq, eq = 0..3 for u, v, w,
// T, so each warp forms one equation for consecutive cells (no divergence) and keeps only that
// equation's inputs (15-17 pairs) and coefficients (6-7 pairs) live; the inputs shared between
// equations come from L1. Cells are 1 <= i <= nx, ... (every input they read is inside the
// padded array, projected); outputs that are not unknowns at a position are written as 0.
template <bool STR>
__global__ void __launch_bounds__(512) k_apply_df(KvGeom g, const float2* __restrict__ coef,
                                                  const float2* __restrict__ cplus, const float2* __restrict__ xs,
                                                  size_t P, double* __restrict__ vstar, double* __restrict__ tout,
                                                  DfAlpha al) {
  const int eq = threadIdx.y & 3;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * (blockDim.y >> 2) + (threadIdx.y >> 2);
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  const int sx = 1, sy = g.X, sz = g.X * g.Y;
  const int e = i + sy * j + sz * k;
  if (!(i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz)) {
    if (eq < 3) {
      vstar[(size_t)eq * P + e] = 0.0;
    } else {
      // the insulated walls' temperature nodes are written by their neighbouring cells
      const bool aa_wall = g.bc == KV_BC_AA && (j == 0 || j == g.ny + 1) && i >= 1 && i <= g.nx && k >= 1 &&
                           k <= g.nz;
      if (!aa_wall) tout[e] = 0.0;
    }
    return;
  }
  const float2* __restrict__ xu = xs;
  const float2* __restrict__ xv = xs + P;
  const float2* __restrict__ xw = xs + 2 * P;
  const float2* __restrict__ xT = xs + 3 * P;
  auto L = [&](const float2* __restrict__ f, int off) {
    const float2 t = __ldg(f + e + off);
    return DF{t.x, t.y};
  };
  auto C = [&](int q) { return __ldg(coef + (size_t)q * P + e); };
  // wall classes of this cell along the cell-type axes
  const int ci = wall_class(i, g.nx), cj = wall_class(j, g.ny), ck = wall_class(k, g.nz);
  DFAcc a;
  // c- x- + c+ x+ along one axis; q = the plus coefficient's index in cplus
  auto own_axis = [&](DFAcc& acc, const float2 cm, const DF xm, const DF xp, const float2 alpha, const float beta,
                      int q) {
    if (STR) {
      acc.fma(cm, xm);
      acc.fma(__ldg(cplus + (size_t)q * P + e), xp);
    } else {
      ::own_axis(acc, cm, xm, xp, alpha, beta);
    }
  };
  if (eq == 0) {  // u on x-faces (x is the face axis); cross terms: 4-point sums of v and w
    const float2 c0 = C(0), cx = C(1), cy = C(2), cz = C(3), c7 = C(4), c8 = C(5);
    a.fma(c0, L(xu, 0));
    own_axis(a, cx, L(xu, -sx), L(xu, sx), alpha_of(al, 0, 0, 0), -1.0f, 0);
    own_axis(a, cy, L(xu, -sy), L(xu, sy), alpha_of(al, 0, 1, cj), beta_of(cj), 1);
    own_axis(a, cz, L(xu, -sz), L(xu, sz), alpha_of(al, 0, 2, ck), beta_of(ck), 2);
    // v(i, j-1), v(i, j), v(i+1, j-1), v(i+1, j); w(i, k-1), w(i, k), w(i+1, k-1), w(i+1, k)
    a.fma(c7, sum4(L(xv, -sy), L(xv, 0), L(xv, sx - sy), L(xv, sx)));
    a.fma(c8, sum4(L(xw, -sz), L(xw, 0), L(xw, sx - sz), L(xw, sx)));
    vstar[e] = i <= g.nx - 1 ? a.value() : 0.0;
  } else if (eq == 1) {  // v on y-faces
    const float2 c0 = C(6), cx = C(7), cy = C(8), cz = C(9), c16 = C(10), c17 = C(11);
    a.fma(c0, L(xv, 0));
    own_axis(a, cx, L(xv, -sx), L(xv, sx), alpha_of(al, 0, 0, ci), beta_of(ci), 3);
    own_axis(a, cy, L(xv, -sy), L(xv, sy), alpha_of(al, 0, 1, 0), -1.0f, 4);
    own_axis(a, cz, L(xv, -sz), L(xv, sz), alpha_of(al, 0, 2, ck), beta_of(ck), 5);
    // u(i-1, j), u(i, j), u(i-1, j+1), u(i, j+1); w(j, k-1), w(j, k), w(j+1, k-1), w(j+1, k)
    a.fma(c16, sum4(L(xu, -sx), L(xu, 0), L(xu, -sx + sy), L(xu, sy)));
    a.fma(c17, sum4(L(xw, -sz), L(xw, 0), L(xw, sy - sz), L(xw, sy)));
    vstar[P + e] = j <= g.ny - 1 ? a.value() : 0.0;
  } else if (eq == 2) {  // w on z-faces, with the buoyancy 0.5 (T_k + T_k+1)
    const float2 c0 = C(12), cx = C(13), cy = C(14), cz = C(15), c25 = C(16), c26 = C(17);
    a.fma(c0, L(xw, 0));
    own_axis(a, cx, L(xw, -sx), L(xw, sx), alpha_of(al, 0, 0, ci), beta_of(ci), 6);
    own_axis(a, cy, L(xw, -sy), L(xw, sy), alpha_of(al, 0, 1, cj), beta_of(cj), 7);
    own_axis(a, cz, L(xw, -sz), L(xw, sz), alpha_of(al, 0, 2, 0), -1.0f, 8);
    // u(i-1, k), u(i, k), u(i-1, k+1), u(i, k+1); v(j-1, k), v(j, k), v(j-1, k+1), v(j, k+1)
    a.fma(c25, sum4(L(xu, -sx), L(xu, 0), L(xu, -sx + sz), L(xu, sz)));
    a.fma(c26, sum4(L(xv, -sy), L(xv, 0), L(xv, -sy + sz), L(xv, sz)));
    a.fma(make_float2(0.5f, 0.0f), df_add_lazy(L(xT, 0), L(xT, sz)));
    vstar[2 * P + e] = k <= g.nz - 1 ? a.value() : 0.0;
  } else {  // T on cells
    const float2 c0 = C(18), cx = C(19), cy = C(20), cz = C(21), c34 = C(22), c35 = C(23), c36 = C(24);
    a.fma(c0, L(xT, 0));
    own_axis(a, cx, L(xT, -sx), L(xT, sx), alpha_of(al, 1, 0, ci), beta_of(ci), 9);
    own_axis(a, cy, L(xT, -sy), L(xT, sy), alpha_of(al, 1, 1, cj), beta_of(cj), 10);
    own_axis(a, cz, L(xT, -sz), L(xT, sz), alpha_of(al, 1, 2, ck), beta_of(ck), 11);
    a.fma(c34, df_add_lazy(L(xu, -sx), L(xu, 0)));
    a.fma(c35, df_add_lazy(L(xv, -sy), L(xv, 0)));
    a.fma(c36, df_add_lazy(L(xw, -sz), L(xw, 0)));
    const double r = a.value();
    if (g.bc == KV_BC_AA && (j == 1 || j == g.ny)) {
      const double t = (g.tproj == KV_TPROJ_OBLIQUE) ? r : 0.5 * r;
      tout[e] = t;
      tout[i + sy * (j == 1 ? 0 : g.ny + 1) + sz * k] = t;
    } else {
      tout[e] = r;
    }
  }
}

// ---- the same operator as a 2.5D march (no separate split pass) -----------------------------
//
// A block owns a tile of MB_X x MB_Y cells and walks a chunk of kc z-planes. It keeps four
// planes of the projected input (P_BC x, split into FP32 pairs, with a one-cell halo) in shared
// memory: at step k it issues the FP64 loads of plane k+2, forms the equations of plane k from
// planes k-1..k+1 (one thread per cell and equation, as k_apply_df), then projects, splits and
// stores plane k+2 into the slot plane k-2 used, and synchronises once. Each input value is thus
// read from HBM once per block (plus a two-plane halo per chunk) and split once, and the
// coefficients of plane k+1 are prefetched into registers while plane k is computed.
constexpr int MB_X = 32, MB_Y = 4;
constexpr int MT_X = MB_X + 2, MT_Y = MB_Y + 2, MPTS = MT_X * MT_Y;
constexpr int MTHREADS = MB_X * MB_Y * 4;
static_assert((MTHREADS & (MTHREADS - 1)) == 0, "the staging order below rotates thread indices mod MTHREADS");
constexpr int MVALS = 4 * MPTS;                                 // values per plane (4 fields)
constexpr int MPER = (MVALS + MTHREADS - 1) / MTHREADS;         // values per thread per plane

__device__ __forceinline__ double proj_value(const Loader<true>& L, int f, int i, int j, int k) {
  return f == 0 ? L.lu(i, j, k) : (f == 1 ? L.lv(i, j, k) : (f == 2 ? L.lw(i, j, k) : L.lT(i, j, k)));
}

template <bool STR>
__device__ __forceinline__ void march_body(const KvGeom& g, const float2* __restrict__ coef,
                                           const float2* __restrict__ cplus, const double* __restrict__ x, size_t P,
                                           double* __restrict__ vstar, double* __restrict__ tout, const DfAlpha& al,
                                           int kc) {
  __shared__ float2 xt[4][4][MPTS];  // [slot][field][point]
  float2* const xflat = &xt[0][0][0];
  const int tid = threadIdx.x;
  const int tx = tid & 31, warp = tid >> 5;
  const int ty = warp % MB_Y, eq = warp / MB_Y;
  const int i = 1 + blockIdx.x * MB_X + tx, j = 1 + blockIdx.y * MB_Y + ty;
  const int k0 = 1 + blockIdx.z * kc;
  const int k1 = min(k0 + kc, g.nz + 1);  // planes k0 .. k1-1
  const bool active = i <= g.nx && j <= g.ny;
  const int sy = g.X, sz = g.X * g.Y;
  Grid G{g};
  const Loader<true> LD{G, x, x + P, x + 2 * P, x + 3 * P};
  // Staging order: ft = (tid + 128) mod 512, so the 304 threads that stage a second value per
  // plane are the temperature warps (the fewest products) and the first momentum warps; the
  // w warps (buoyancy terms) stage one.
  const int ft = (tid + 128) & (MTHREADS - 1);
  // The values this thread stages for every plane: value v = ft + r MTHREADS of a plane is
  // field f = v / MPTS at tile point v % MPTS, stored at xt[slot][0][v]. P_BC x there is
  // x_f(i, j, k) for 1 <= k <= lim[r] and 0 for other planes (col[r]: the (f, i, j) column of x;
  // lim[r] = 0: always 0), except the temperature rows next to insulated walls (lim[r] < 0),
  // which proj_value projects (the wall node and its neighbour combine). Offsets into the packed
  // vector fit 32 bits (the variant is taken only for 4 P < 2^31).
  unsigned int col[MPER];
  int lim[MPER];
#pragma unroll
  for (int r = 0; r < MPER; ++r) {
    const int v = ft + r * MTHREADS;
    col[r] = 0;
    lim[r] = 0;
    if (v < MVALS) {
      const int f = v / MPTS, pt = v - f * MPTS;
      const int ii = blockIdx.x * MB_X + pt % MT_X, jj = blockIdx.y * MB_Y + pt / MT_X;
      if (ii <= g.nx + 1 && jj <= g.ny + 1) {
        col[r] = (unsigned int)((size_t)f * P + ii + (size_t)sy * jj);
        const bool in_i = ii >= 1 && ii <= g.nx, in_j = jj >= 1 && jj <= g.ny;
        if (f == 0)
          lim[r] = (ii >= 1 && ii <= g.nx - 1 && in_j) ? g.nz : 0;
        else if (f == 1)
          lim[r] = (in_i && jj >= 1 && jj <= g.ny - 1) ? g.nz : 0;
        else if (f == 2)
          lim[r] = (in_i && in_j) ? g.nz - 1 : 0;
        else if (g.bc == KV_BC_CC)
          lim[r] = (in_i && in_j) ? g.nz : 0;
        else
          lim[r] = !in_i ? 0 : ((jj >= 2 && jj <= g.ny - 1) ? g.nz : -1);
      }
    }
  }
  auto fetch = [&](int kk, double (&val)[MPER]) {
#pragma unroll
    for (int r = 0; r < MPER; ++r) {
      // lim < 0 compares as a large unsigned limit: the load stays inside the column
      val[r] = (unsigned)(kk - 1) < (unsigned)lim[r] ? __ldg(x + (col[r] + (unsigned int)(sz * kk))) : 0.0;
      if (lim[r] < 0) {
        const int pt = ft + r * MTHREADS - 3 * MPTS;
        val[r] = proj_value(LD, 3, blockIdx.x * MB_X + pt % MT_X, blockIdx.y * MB_Y + pt / MT_X, kk);
      }
    }
  };
  auto put = [&](int slot, const double (&val)[MPER]) {
#pragma unroll
    for (int r = 0; r < MPER; ++r) {
      const int v = ft + r * MTHREADS;
      if (v < MVALS) {
        const DF d = df_split(val[r]);
        xflat[slot * MVALS + v] = make_float2(d.h, d.l);
      }
    }
  };
  {
    double val[MPER];
    for (int kk = k0 - 1; kk <= k0 + 1; ++kk) {
      fetch(kk, val);
      put(kk & 3, val);
    }
  }
  __syncthreads();
  const int ci = wall_class(i, g.nx), cj = wall_class(j, g.ny);
  const int q0 = eq == 0 ? 0 : (eq == 1 ? 6 : (eq == 2 ? 12 : 18));
  const int nqe = eq == 3 ? 7 : 6;
  // coefficient column of this thread's cell (clamped into the grid for threads past its edge)
  const float2* const ccol =
      coef + (size_t)q0 * P + (size_t)min(i, g.nx) + (size_t)sy * min(j, g.ny);
  float2 cn[7];
  auto coefs = [&](int kk, float2 (&c)[7]) {
    const float2* const cp = ccol + (size_t)sz * kk;
#pragma unroll
    for (int q = 0; q < 7; ++q) c[q] = q < nqe ? __ldg(cp + (size_t)q * P) : make_float2(0.f, 0.f);
  };
  coefs(k0, cn);
  const int pc = (ty + 1) * MT_X + (tx + 1);  // this cell's point in the tile
  for (int k = k0; k < k1; ++k) {
    const bool more = k + 1 < k1;
    double nxt[MPER];
    if (more) fetch(k + 2, nxt);
    float2 c[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) c[q] = cn[q];
    if (more) coefs(k + 1, cn);
    if (active) {
      const int sm = (k - 1) & 3, s0 = k & 3, sp = (k + 1) & 3;
      // input value of field f at offset (di, dj) in plane slot sl
      auto X = [&](int sl, int f, int di, int dj) {
        const float2 t = xt[sl][f][pc + di + MT_X * dj];
        return DF{t.x, t.y};
      };
      const int ck = wall_class(k, g.nz);
      const size_t e = (size_t)i + (size_t)sy * j + (size_t)sz * k;
      DFAcc a;
      // c- x- + c+ x+ along one axis; on a stretched grid or with upwinding (STR) c+ is read from cplus (entry
      // 3 eq + axis), else rebuilt as alpha + beta c-
      auto own_axis = [&](DFAcc& acc, const float2 cm, const DF xm, const DF xp, const float2 alpha, const float beta,
                          int axis) {
        if (STR) {
          acc.fma(cm, xm);
          acc.fma(__ldg(cplus + (size_t)(3 * eq + axis) * P + e), xp);
        } else {
          ::own_axis(acc, cm, xm, xp, alpha, beta);
        }
      };
      if (eq == 0) {
        a.fma(c[0], X(s0, 0, 0, 0));
        own_axis(a, c[1], X(s0, 0, -1, 0), X(s0, 0, 1, 0), alpha_of(al, 0, 0, 0), -1.0f, 0);
        own_axis(a, c[2], X(s0, 0, 0, -1), X(s0, 0, 0, 1), alpha_of(al, 0, 1, cj), beta_of(cj), 1);
        own_axis(a, c[3], X(sm, 0, 0, 0), X(sp, 0, 0, 0), alpha_of(al, 0, 2, ck), beta_of(ck), 2);
        // v(i, j-1), v(i, j), v(i+1, j-1), v(i+1, j); w(i, k-1), w(i, k), w(i+1, k-1), w(i+1, k)
        a.fma(c[4], sum4(X(s0, 1, 0, -1), X(s0, 1, 0, 0), X(s0, 1, 1, -1), X(s0, 1, 1, 0)));
        a.fma(c[5], sum4(X(sm, 2, 0, 0), X(s0, 2, 0, 0), X(sm, 2, 1, 0), X(s0, 2, 1, 0)));
        vstar[e] = i <= g.nx - 1 ? a.value() : 0.0;
      } else if (eq == 1) {
        a.fma(c[0], X(s0, 1, 0, 0));
        own_axis(a, c[1], X(s0, 1, -1, 0), X(s0, 1, 1, 0), alpha_of(al, 0, 0, ci), beta_of(ci), 0);
        own_axis(a, c[2], X(s0, 1, 0, -1), X(s0, 1, 0, 1), alpha_of(al, 0, 1, 0), -1.0f, 1);
        own_axis(a, c[3], X(sm, 1, 0, 0), X(sp, 1, 0, 0), alpha_of(al, 0, 2, ck), beta_of(ck), 2);
        // u(i-1, j), u(i, j), u(i-1, j+1), u(i, j+1); w(j, k-1), w(j, k), w(j+1, k-1), w(j+1, k)
        a.fma(c[4], sum4(X(s0, 0, -1, 0), X(s0, 0, 0, 0), X(s0, 0, -1, 1), X(s0, 0, 0, 1)));
        a.fma(c[5], sum4(X(sm, 2, 0, 0), X(s0, 2, 0, 0), X(sm, 2, 0, 1), X(s0, 2, 0, 1)));
        vstar[P + e] = j <= g.ny - 1 ? a.value() : 0.0;
      } else if (eq == 2) {
        a.fma(c[0], X(s0, 2, 0, 0));
        own_axis(a, c[1], X(s0, 2, -1, 0), X(s0, 2, 1, 0), alpha_of(al, 0, 0, ci), beta_of(ci), 0);
        own_axis(a, c[2], X(s0, 2, 0, -1), X(s0, 2, 0, 1), alpha_of(al, 0, 1, cj), beta_of(cj), 1);
        own_axis(a, c[3], X(sm, 2, 0, 0), X(sp, 2, 0, 0), alpha_of(al, 0, 2, 0), -1.0f, 2);
        // u(i-1, k), u(i, k), u(i-1, k+1), u(i, k+1); v(j-1, k), v(j, k), v(j-1, k+1), v(j, k+1)
        a.fma(c[4], sum4(X(s0, 0, -1, 0), X(s0, 0, 0, 0), X(sp, 0, -1, 0), X(sp, 0, 0, 0)));
        a.fma(c[5], sum4(X(s0, 1, 0, -1), X(s0, 1, 0, 0), X(sp, 1, 0, -1), X(sp, 1, 0, 0)));
        a.fma(make_float2(0.5f, 0.0f), df_add_lazy(X(s0, 3, 0, 0), X(sp, 3, 0, 0)));
        vstar[2 * P + e] = k <= g.nz - 1 ? a.value() : 0.0;
      } else {
        a.fma(c[0], X(s0, 3, 0, 0));
        own_axis(a, c[1], X(s0, 3, -1, 0), X(s0, 3, 1, 0), alpha_of(al, 1, 0, ci), beta_of(ci), 0);
        own_axis(a, c[2], X(s0, 3, 0, -1), X(s0, 3, 0, 1), alpha_of(al, 1, 1, cj), beta_of(cj), 1);
        own_axis(a, c[3], X(sm, 3, 0, 0), X(sp, 3, 0, 0), alpha_of(al, 1, 2, ck), beta_of(ck), 2);
        a.fma(c[4], df_add_lazy(X(s0, 0, -1, 0), X(s0, 0, 0, 0)));
        a.fma(c[5], df_add_lazy(X(s0, 1, 0, -1), X(s0, 1, 0, 0)));
        a.fma(c[6], df_add_lazy(X(sm, 2, 0, 0), X(s0, 2, 0, 0)));
        const double r = a.value();
        if (g.bc == KV_BC_AA && (j == 1 || j == g.ny)) {
          const double t = (g.tproj == KV_TPROJ_OBLIQUE) ? r : 0.5 * r;
          tout[e] = t;
          tout[(size_t)i + (size_t)sy * (j == 1 ? 0 : g.ny + 1) + (size_t)sz * k] = t;
        } else {
          tout[e] = r;
        }
      }
    }
    if (more) put((k + 2) & 3, nxt);
    __syncthreads();
  }
}

// The uniform grid's march: two blocks of 512 threads per SM (64 registers a thread).
__global__ void __launch_bounds__(MTHREADS, 2) k_apply_df_march(KvGeom g, const float2* __restrict__ coef,
                                                                const double* __restrict__ x, size_t P,
                                                                double* __restrict__ vstar,
                                                                double* __restrict__ tout, DfAlpha al, int kc) {
  march_body<false>(g, coef, nullptr, x, P, vstar, tout, al, kc);
}

// The march of a stretched grid (Eq 22) or of upwind advection: the three plus coefficients per
// equation come from cplus, which needs more registers than two blocks per SM leave.
__global__ void __launch_bounds__(MTHREADS, 1) k_apply_df_march_str(KvGeom g, const float2* __restrict__ coef,
                                                                    const float2* __restrict__ cplus,
                                                                    const double* __restrict__ x, size_t P,
                                                                    double* __restrict__ vstar,
                                                                    double* __restrict__ tout, DfAlpha al, int kc) {
  march_body<true>(g, coef, cplus, x, P, vstar, tout, al, kc);
}

// The padded-boundary entries of v* and T* (walls, edges, corners: 0; the insulated walls'
// temperature nodes are written by their neighbouring cells), which the march does not visit.
__global__ void __launch_bounds__(256) k_zero_boundary(KvGeom g, size_t P, double* __restrict__ vstar,
                                                       double* __restrict__ tout) {
  // the six boundary planes in turn: k = 0, Z-1 (X*Y each), j = 0, Y-1 (X*(Z-2)), i = 0, X-1 ((Y-2)*(Z-2))
  const long long nk = (long long)g.X * g.Y, nj = (long long)g.X * (g.Z - 2), ni = (long long)(g.Y - 2) * (g.Z - 2);
  const long long n = 2 * (nk + nj + ni);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    long long r = t;
    int i, j, k;
    if (r < 2 * nk) {
      k = r < nk ? 0 : g.Z - 1;
      r %= nk;
      i = (int)(r % g.X);
      j = (int)(r / g.X);
    } else if ((r -= 2 * nk) < 2 * nj) {
      j = r < nj ? 0 : g.Y - 1;
      r %= nj;
      i = (int)(r % g.X);
      k = 1 + (int)(r / g.X);
    } else {
      r -= 2 * nj;
      i = r < ni ? 0 : g.X - 1;
      r %= ni;
      j = 1 + (int)(r % (g.Y - 2));
      k = 1 + (int)(r / (g.Y - 2));
    }
    const size_t e = (size_t)i + (size_t)g.X * ((size_t)j + (size_t)g.Y * k);
    vstar[e] = 0.0;
    vstar[P + e] = 0.0;
    vstar[2 * P + e] = 0.0;
    const bool aa_wall = g.bc == KV_BC_AA && (j == 0 || j == g.ny + 1) && i >= 1 && i <= g.nx && k >= 1 &&
                         k <= g.nz;
    if (!aa_wall) tout[e] = 0.0;
  }
}

// FP32-pair copy of the assembled coefficients the double-float operator reads
// (kDfFromFull): ch = fp32(c), cl = fp32(c - ch).
__global__ void __launch_bounds__(256) k_coef_df(const double* __restrict__ coef, float2* __restrict__ cdf, size_t P) {
  const size_t n = (size_t)KV_NCOEF_DF * P;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t q = t / P, e = t - q * P;
    const double c = coef[(size_t)kDfFromFull[q] * P + e];
    const float h = __double2float_rn(c);
    cdf[t] = make_float2(h, __double2float_rn(c - (double)h));
  }
}

// The plus coefficients of a stretched grid or of upwind advection as FP32 pairs (KV_NCOEF_DFP of them).
__global__ void __launch_bounds__(256) k_coef_df_plus(const double* __restrict__ coef, float2* __restrict__ cdf,
                                                      size_t P) {
  const size_t n = (size_t)KV_NCOEF_DFP * P;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t q = t / P, e = t - q * P;
    const double c = coef[(size_t)kPlusFromFull[q] * P + e];
    const float h = __double2float_rn(c);
    cdf[t] = make_float2(h, __double2float_rn(c - (double)h));
  }
}

// x as an FP32 pair (host side)
float2 host_pair(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

}  // namespace

void kv_launch_stencil(const kv_grid* h, int mode, const double* base, const double* x, double* vstar,
                       double* tout, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1);
  dim3 grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  const bool str = h->str.sw != nullptr;
  if (mode == 0 && str)
    k_stencil<0, true><<<grid, block, 0, s>>>(g, h->str, base, x, h->P, vstar, tout);
  else if (mode == 0)
    k_stencil<0, false><<<grid, block, 0, s>>>(g, h->str, base, x, h->P, vstar, tout);
  else if (str)
    k_stencil<1, true><<<grid, block, 0, s>>>(g, h->str, base, x, h->P, vstar, tout);
  else
    k_stencil<1, false><<<grid, block, 0, s>>>(g, h->str, base, x, h->P, vstar, tout);
}

void kv_launch_assemble(const kv_grid* h, const double* base, double* coef, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  if (h->str.sw)
    k_assemble<true><<<grid, block, 0, s>>>(g, h->str, base, h->P, coef);
  else
    k_assemble<false><<<grid, block, 0, s>>>(g, h->str, base, h->P, coef);
}

void kv_launch_apply(const kv_grid* h, const double* coef, const double* x, double* vstar, double* tout,
                     cudaStream_t s) {
  const KvGeom& g = h->g;
  const int bx = h->apply_bx, by = h->apply_by;
  dim3 block(bx, by, 1), grid((g.X + bx - 1) / bx, (g.Y + by - 1) / by, g.Z);
  k_apply<<<grid, block, 0, s>>>(g, coef, x, h->P, vstar, tout);
}

void kv_launch_zero_boundary(const kv_grid* h, double* vstar, double* tout, cudaStream_t s) {
  k_zero_boundary<<<2 * 152, 256, 0, s>>>(h->g, h->P, vstar, tout);
}

void kv_launch_coef_df(const kv_grid* h, const double* coef, float2* cdf, cudaStream_t s) {
  k_coef_df<<<4 * 152, 256, 0, s>>>(coef, cdf, h->P);
  if (h->str.sw || h->g.adv) k_coef_df_plus<<<4 * 152, 256, 0, s>>>(coef, h->coef_dfp, h->P);
}

void kv_launch_apply_df(const kv_grid* h, const float2* cdf, const double* x, double* vstar, double* tout,
                        cudaStream_t s) {
  const KvGeom& g = h->g;
  // alpha = {2, 3/2, 6} diff / h^2 per axis (interior, first cell, last cell)
  DfAlpha al;
  const double diff[2] = {g.nu, g.kappa}, ih2[3] = {g.ihx * g.ihx, g.ihy * g.ihy, g.ihz * g.ihz};
  const double fac[3] = {2.0, 1.5, 6.0};
  for (int d = 0; d < 2; ++d)
    for (int ax = 0; ax < 3; ++ax)
      for (int c = 0; c < 3; ++c) al.a[d][ax][c] = host_pair(fac[c] * diff[d] * ih2[ax]);
  if (h->df_variant == 2 && h->fx_ok) {  // fixed point, df_by planes per block (kv_fixed.cu)
    kv_launch_apply_fx(h, x, vstar, tout, h->df_by, s);
    return;
  }
  // variant 2 on a base state the fixed-point form does not take (non-finite): the march
  if (h->df_variant == 1 || h->df_variant == 2) {
    // the 2.5D march: df_by planes per block
    k_zero_boundary<<<2 * 152, 256, 0, s>>>(g, h->P, vstar, tout);
    const int kc = h->df_by;
    dim3 grid((g.nx + MB_X - 1) / MB_X, (g.ny + MB_Y - 1) / MB_Y, (g.nz + kc - 1) / kc);
    if (h->str.sw || g.adv)  // plus coefficients stored: stretched or upwind
      k_apply_df_march_str<<<grid, MTHREADS, 0, s>>>(g, cdf, h->coef_dfp, x, h->P, vstar, tout, al, kc);
    else
      k_apply_df_march<<<grid, MTHREADS, 0, s>>>(g, cdf, x, h->P, vstar, tout, al, kc);
    return;
  }
  {
    dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
    k_split_input<<<grid, block, 0, s>>>(g, x, h->P, h->xsplit);
  }
  // df_by rows of cells per block, four equation warps-rows each
  const int bx = h->df_bx, rows = h->df_by;
  dim3 block(bx, 4 * rows, 1), grid((g.X + bx - 1) / bx, (g.Y + rows - 1) / rows, g.Z);
  if (h->str.sw || g.adv)
    k_apply_df<true><<<grid, block, 0, s>>>(g, cdf, h->coef_dfp, h->xsplit, h->P, vstar, tout, al);
  else
    k_apply_df<false><<<grid, block, 0, s>>>(g, cdf, nullptr, h->xsplit, h->P, vstar, tout, al);
}
