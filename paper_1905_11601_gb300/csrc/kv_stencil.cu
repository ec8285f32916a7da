// The linearised Boussinesq operator of Eqs (8)-(9) as used by Eqs (11)-(12), and the
// steady residual of Eqs (1)-(2), on the uniform MAC grid (FP64).
//
// Discrete operators (the paper defers its schemes to its reference [11]; these are the
// readings this library implements):
//   diffusion  flux form ((f+ - f)/(x+ - x) - (f - f-)/(x - x-)) / h, wall nodes at h/2;
//   advection  (a . grad) b in advective form: 3-point central derivative of b at b's node
//              (non-uniform next to a wall node), times a averaged (2 or 4 points) there;
//   buoyancy   T e_z on a w-face: mean of the two adjacent cell temperatures.
// One thread per padded index (i, j, k) writes the u, v and w entries at that index (the
// momentum right-hand side on interior faces, 0 elsewhere) and the projected temperature.
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
template <int MODE>
__global__ void __launch_bounds__(256) k_stencil(KvGeom g, const double* __restrict__ base,
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
  const double ihx = g.ihx, ihy = g.ihy, ihz = g.ihz;
  const double ihx2 = ihx * ihx, ihy2 = ihy * ihy, ihz2 = ihz * ihz;

  // ---- u on the x-face (i, j, k) ----
  double ru = 0.0;
  if (G.dof_u(i, j, k)) {
    const W3 dx1 = d1_face(ihx), dx2 = d2_face(ihx2);
    const W3 dy1 = d1_cell(j, g.ny, ihy), dy2 = d2_cell(j, g.ny, ihy2);
    const W3 dz1 = d1_cell(k, g.nz, ihz), dz2 = d2_cell(k, g.nz, ihz2);
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
    const W3 dx1 = d1_cell(i, g.nx, ihx), dx2 = d2_cell(i, g.nx, ihx2);
    const W3 dy1 = d1_face(ihy), dy2 = d2_face(ihy2);
    const W3 dz1 = d1_cell(k, g.nz, ihz), dz2 = d2_cell(k, g.nz, ihz2);
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
    const W3 dx1 = d1_cell(i, g.nx, ihx), dx2 = d2_cell(i, g.nx, ihx2);
    const W3 dy1 = d1_cell(j, g.ny, ihy), dy2 = d2_cell(j, g.ny, ihy2);
    const W3 dz1 = d1_face(ihz), dz2 = d2_face(ihz2);
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
    const W3 dx1 = d1_cell(i, g.nx, ihx), dx2 = d2_cell(i, g.nx, ihx2);
    const W3 dy1 = d1_cell(j, g.ny, ihy), dy2 = d2_cell(j, g.ny, ihy2);
    const W3 dz1 = d1_cell(k, g.nz, ihz), dz2 = d2_cell(k, g.nz, ihz2);
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
__global__ void __launch_bounds__(256) k_assemble(KvGeom g, const double* __restrict__ base, size_t P,
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
  const double ihx2 = g.ihx * g.ihx, ihy2 = g.ihy * g.ihy, ihz2 = g.ihz * g.ihz;
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
    const W3 dx1 = d1_face(g.ihx), dx2 = d2_face(ihx2);
    const W3 dy1 = d1_cell(j, g.ny, g.ihy), dy2 = d2_cell(j, g.ny, ihy2);
    const W3 dz1 = d1_cell(k, g.nz, g.ihz), dz2 = d2_cell(k, g.nz, ihz2);
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
    const W3 dx1 = d1_cell(i, g.nx, g.ihx), dx2 = d2_cell(i, g.nx, ihx2);
    const W3 dy1 = d1_face(g.ihy), dy2 = d2_face(ihy2);
    const W3 dz1 = d1_cell(k, g.nz, g.ihz), dz2 = d2_cell(k, g.nz, ihz2);
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
    const W3 dx1 = d1_cell(i, g.nx, g.ihx), dx2 = d2_cell(i, g.nx, ihx2);
    const W3 dy1 = d1_cell(j, g.ny, g.ihy), dy2 = d2_cell(j, g.ny, ihy2);
    const W3 dz1 = d1_face(g.ihz), dz2 = d2_face(ihz2);
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
    const W3 dx1 = d1_cell(i, g.nx, g.ihx), dx2 = d2_cell(i, g.nx, ihx2);
    const W3 dy1 = d1_cell(j, g.ny, g.ihy), dy2 = d2_cell(j, g.ny, ihy2);
    const W3 dz1 = d1_cell(k, g.nz, g.ihz), dz2 = d2_cell(k, g.nz, ihz2);
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

// y* = J P_BC x with the assembled coefficients; output as k_stencil<0>.
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
// GB300's FP64 pipe runs at 1/60 of its FP32 rate, so the mixed path evaluates J x in
// double-float arithmetic: every coefficient is stored as an FP32 pair c = ch + cl (|cl| <=
// 2^-24 |ch|), every FP64 input is split into xh (its leading 21 bits, exact) and xl (the rest,
// rounded to FP32) with integer operations only, and each product is accumulated as an exact
// FP32 product ch*xh (FMA error term), an exact running sum (TwoSum) and a small FP32
// correction. The result carries about 2^-44 of the sum of the term magnitudes; the only FP64
// instruction per output is the final addition of the two FP32 halves.

struct DF {
  float h, l;
};

// x = xh + xl: xh from the high word (sign, exponent, 20 mantissa bits), xl = the low 32
// mantissa bits times 2^(e-52), converted with two exact 16-bit pieces. |x| < 2^-74 maps to 0.
__device__ __forceinline__ DF split_d(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7FFu);
  const unsigned int sign = hi & 0x80000000u;
  DF r{0.0f, 0.0f};
  if (E - 1023 + 127 <= 0) return r;
  r.h = __uint_as_float(sign | ((unsigned int)(E - 1023 + 127) << 23) | ((hi & 0xFFFFFu) << 3));
  if (E - 948 <= 0 || lo == 0u) return r;
  const float fa = __fsub_rn(__uint_as_float(0x4B000000u | (lo >> 16)), 8388608.0f);      // exact
  const float fb = __fsub_rn(__uint_as_float(0x4B000000u | (lo & 0xFFFFu)), 8388608.0f);  // exact
  const float lf = __fmaf_rn(fa, 65536.0f, fb);                                           // one rounding
  const float sc = __uint_as_float((unsigned int)(E - 948) << 23);                        // 2^(E-1075)
  r.l = __uint_as_float(__float_as_uint(__fmul_rn(lf, sc)) ^ sign);
  return r;
}

// exact FP32 -> FP64 by bit manipulation (no FP64 instruction); denormals map to 0
__device__ __forceinline__ double f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int fe = (b >> 23) & 0xFFu;
  if (fe == 0u) return 0.0;
  const unsigned int hi = (b & 0x80000000u) | ((fe - 127u + 1023u) << 20) | ((b & 0x7FFFFFu) >> 3);
  const unsigned int lo = (b & 0x7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}

struct Acc {
  float S = 0.0f, C = 0.0f;
  __device__ __forceinline__ void add(const float2 c, const DF x) {
    const float p = __fmul_rn(c.x, x.h);
    const float e = __fmaf_rn(c.x, x.h, -p);
    const float small = __fmaf_rn(c.x, x.l, __fmaf_rn(c.y, x.h, e));
    const float s = __fadd_rn(S, p);
    const float bp = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    S = s;
    C = __fadd_rn(C, __fadd_rn(err, small));
  }
  __device__ __forceinline__ double value() const { return f2d(S) + f2d(C); }
};

template <bool PROJ>
struct DFLoader {
  Loader<PROJ> L;
  __device__ __forceinline__ DF u(int i, int j, int k) const { return split_d(L.lu(i, j, k)); }
  __device__ __forceinline__ DF v(int i, int j, int k) const { return split_d(L.lv(i, j, k)); }
  __device__ __forceinline__ DF w(int i, int j, int k) const { return split_d(L.lw(i, j, k)); }
  __device__ __forceinline__ DF T(int i, int j, int k) const { return split_d(L.lT(i, j, k)); }
};

__device__ __forceinline__ float2 cf2(const float2* __restrict__ coef, size_t P, int q, int e) {
  return __ldg(coef + (size_t)q * P + e);
}

// The interior case of k_apply_df (see there): unmasked loads, each value split once.
__device__ __forceinline__ void apply_df_interior(const KvGeom& g, const float2* __restrict__ coef,
                                                  const double* __restrict__ x, size_t P, double* __restrict__ vstar,
                                                  double* __restrict__ tout, int i, int j, int k) {
  const int sx = 1, sy = g.X, sz = g.X * g.Y;
  const int e = i + sy * j + sz * k;
  const double* __restrict__ xu = x;
  const double* __restrict__ xv = x + P;
  const double* __restrict__ xw = x + 2 * P;
  const double* __restrict__ xT = x + 3 * P;
  auto L = [&](const double* __restrict__ f, int off) { return split_d(__ldg(f + e + off)); };
  // u: own 7 + (i-1, j+1) + (i-1, k+1)
  const DF u0 = L(xu, 0), uxm = L(xu, -sx), uxp = L(xu, sx), uym = L(xu, -sy), uyp = L(xu, sy), uzm = L(xu, -sz),
           uzp = L(xu, sz), uxmyp = L(xu, -sx + sy), uxmzp = L(xu, -sx + sz);
  // v: own 7 + (i+1, j-1) + (j-1, k+1)
  const DF v0 = L(xv, 0), vxm = L(xv, -sx), vxp = L(xv, sx), vym = L(xv, -sy), vyp = L(xv, sy), vzm = L(xv, -sz),
           vzp = L(xv, sz), vxpym = L(xv, sx - sy), vymzp = L(xv, -sy + sz);
  // w: own 7 + (i+1, k-1) + (j+1, k-1)
  const DF w0 = L(xw, 0), wxm = L(xw, -sx), wxp = L(xw, sx), wym = L(xw, -sy), wyp = L(xw, sy), wzm = L(xw, -sz),
           wzp = L(xw, sz), wxpzm = L(xw, sx - sz), wypzm = L(xw, sy - sz);
  // T: own 7 (the buoyancy reads T(k) and T(k+1))
  const DF t0 = L(xT, 0), txm = L(xT, -sx), txp = L(xT, sx), tym = L(xT, -sy), typ = L(xT, sy), tzm = L(xT, -sz),
           tzp = L(xT, sz);
  {
    Acc a;
    a.add(cf2(coef, P, 0, e), u0);
    a.add(cf2(coef, P, 1, e), uxm);
    a.add(cf2(coef, P, 2, e), uxp);
    a.add(cf2(coef, P, 3, e), uym);
    a.add(cf2(coef, P, 4, e), uyp);
    a.add(cf2(coef, P, 5, e), uzm);
    a.add(cf2(coef, P, 6, e), uzp);
    const float2 c7 = cf2(coef, P, 7, e), c8 = cf2(coef, P, 8, e);
    a.add(c7, vym);    // v(i, j-1)
    a.add(c7, v0);     // v(i, j)
    a.add(c7, vxpym);  // v(i+1, j-1)
    a.add(c7, vxp);    // v(i+1, j)
    a.add(c8, wzm);    // w(i, k-1)
    a.add(c8, w0);     // w(i, k)
    a.add(c8, wxpzm);  // w(i+1, k-1)
    a.add(c8, wxp);    // w(i+1, k)
    vstar[e] = a.value();
  }
  {
    Acc a;
    a.add(cf2(coef, P, 9, e), v0);
    a.add(cf2(coef, P, 10, e), vxm);
    a.add(cf2(coef, P, 11, e), vxp);
    a.add(cf2(coef, P, 12, e), vym);
    a.add(cf2(coef, P, 13, e), vyp);
    a.add(cf2(coef, P, 14, e), vzm);
    a.add(cf2(coef, P, 15, e), vzp);
    const float2 c16 = cf2(coef, P, 16, e), c17 = cf2(coef, P, 17, e);
    a.add(c16, uxm);    // u(i-1, j)
    a.add(c16, u0);     // u(i, j)
    a.add(c16, uxmyp);  // u(i-1, j+1)
    a.add(c16, uyp);    // u(i, j+1)
    a.add(c17, wzm);    // w(j, k-1)
    a.add(c17, w0);     // w(j, k)
    a.add(c17, wypzm);  // w(j+1, k-1)
    a.add(c17, wyp);    // w(j+1, k)
    vstar[P + e] = a.value();
  }
  {
    Acc a;
    a.add(cf2(coef, P, 18, e), w0);
    a.add(cf2(coef, P, 19, e), wxm);
    a.add(cf2(coef, P, 20, e), wxp);
    a.add(cf2(coef, P, 21, e), wym);
    a.add(cf2(coef, P, 22, e), wyp);
    a.add(cf2(coef, P, 23, e), wzm);
    a.add(cf2(coef, P, 24, e), wzp);
    const float2 c25 = cf2(coef, P, 25, e), c26 = cf2(coef, P, 26, e);
    a.add(c25, uxm);    // u(i-1, k)
    a.add(c25, u0);     // u(i, k)
    a.add(c25, uxmzp);  // u(i-1, k+1)
    a.add(c25, uzp);    // u(i, k+1)
    a.add(c26, vym);    // v(j-1, k)
    a.add(c26, v0);     // v(j, k)
    a.add(c26, vymzp);  // v(j-1, k+1)
    a.add(c26, vzp);    // v(j, k+1)
    const float2 half = make_float2(0.5f, 0.0f);
    a.add(half, t0);
    a.add(half, tzp);
    vstar[2 * P + e] = a.value();
  }
  {
    Acc a;
    a.add(cf2(coef, P, 27, e), t0);
    a.add(cf2(coef, P, 28, e), txm);
    a.add(cf2(coef, P, 29, e), txp);
    a.add(cf2(coef, P, 30, e), tym);
    a.add(cf2(coef, P, 31, e), typ);
    a.add(cf2(coef, P, 32, e), tzm);
    a.add(cf2(coef, P, 33, e), tzp);
    const float2 c34 = cf2(coef, P, 34, e), c35 = cf2(coef, P, 35, e), c36 = cf2(coef, P, 36, e);
    a.add(c34, uxm);
    a.add(c34, u0);
    a.add(c35, vym);
    a.add(c35, v0);
    a.add(c36, wzm);
    a.add(c36, w0);
    tout[e] = a.value();
  }
}

// y* = J P_BC x with the FP32-pair coefficients (output as k_apply). MINB: the launch bound's
// minimum resident blocks, which sets the register budget (more registers, more independent
// loads in flight; fewer, more resident warps); the autotuner picks the faster.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_apply_df(KvGeom g, const float2* __restrict__ coef,
                                                        const double* __restrict__ x, size_t P,
                                                        double* __restrict__ vstar, double* __restrict__ tout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  // Blocks three or more cells away from every wall: every output is an interior unknown and
  // every input it reads is one too (and no temperature it reads belongs to an insulated wall
  // pair), so the loads need no masking; each distinct input value (34 per cell) is loaded and
  // split once.
  {
    const int i0 = blockIdx.x * blockDim.x, j0 = blockIdx.y * blockDim.y;
    if (i0 >= 3 && i0 + (int)blockDim.x - 1 <= g.nx - 3 && j0 >= 3 && j0 + (int)blockDim.y - 1 <= g.ny - 3 &&
        k >= 3 && k <= g.nz - 3) {
      apply_df_interior(g, coef, x, P, vstar, tout, i, j, k);
      return;
    }
  }
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  Grid G{g};
  const int e = G.at(i, j, k);
  DFLoader<true> X{Loader<true>{G, x, x + P, x + 2 * P, x + 3 * P}};
  double ru = 0.0, rv = 0.0, rw = 0.0;
  if (G.dof_u(i, j, k)) {
    Acc a;
    a.add(cf2(coef, P, 0, e), X.u(i, j, k));
    a.add(cf2(coef, P, 1, e), X.u(i - 1, j, k));
    a.add(cf2(coef, P, 2, e), X.u(i + 1, j, k));
    a.add(cf2(coef, P, 3, e), X.u(i, j - 1, k));
    a.add(cf2(coef, P, 4, e), X.u(i, j + 1, k));
    a.add(cf2(coef, P, 5, e), X.u(i, j, k - 1));
    a.add(cf2(coef, P, 6, e), X.u(i, j, k + 1));
    const float2 c7 = cf2(coef, P, 7, e), c8 = cf2(coef, P, 8, e);
    a.add(c7, X.v(i, j - 1, k));
    a.add(c7, X.v(i, j, k));
    a.add(c7, X.v(i + 1, j - 1, k));
    a.add(c7, X.v(i + 1, j, k));
    a.add(c8, X.w(i, j, k - 1));
    a.add(c8, X.w(i, j, k));
    a.add(c8, X.w(i + 1, j, k - 1));
    a.add(c8, X.w(i + 1, j, k));
    ru = a.value();
  }
  vstar[e] = ru;
  if (G.dof_v(i, j, k)) {
    Acc a;
    a.add(cf2(coef, P, 9, e), X.v(i, j, k));
    a.add(cf2(coef, P, 10, e), X.v(i - 1, j, k));
    a.add(cf2(coef, P, 11, e), X.v(i + 1, j, k));
    a.add(cf2(coef, P, 12, e), X.v(i, j - 1, k));
    a.add(cf2(coef, P, 13, e), X.v(i, j + 1, k));
    a.add(cf2(coef, P, 14, e), X.v(i, j, k - 1));
    a.add(cf2(coef, P, 15, e), X.v(i, j, k + 1));
    const float2 c16 = cf2(coef, P, 16, e), c17 = cf2(coef, P, 17, e);
    a.add(c16, X.u(i - 1, j, k));
    a.add(c16, X.u(i, j, k));
    a.add(c16, X.u(i - 1, j + 1, k));
    a.add(c16, X.u(i, j + 1, k));
    a.add(c17, X.w(i, j, k - 1));
    a.add(c17, X.w(i, j, k));
    a.add(c17, X.w(i, j + 1, k - 1));
    a.add(c17, X.w(i, j + 1, k));
    rv = a.value();
  }
  vstar[P + e] = rv;
  if (G.dof_w(i, j, k)) {
    Acc a;
    a.add(cf2(coef, P, 18, e), X.w(i, j, k));
    a.add(cf2(coef, P, 19, e), X.w(i - 1, j, k));
    a.add(cf2(coef, P, 20, e), X.w(i + 1, j, k));
    a.add(cf2(coef, P, 21, e), X.w(i, j - 1, k));
    a.add(cf2(coef, P, 22, e), X.w(i, j + 1, k));
    a.add(cf2(coef, P, 23, e), X.w(i, j, k - 1));
    a.add(cf2(coef, P, 24, e), X.w(i, j, k + 1));
    const float2 c25 = cf2(coef, P, 25, e), c26 = cf2(coef, P, 26, e);
    a.add(c25, X.u(i - 1, j, k));
    a.add(c25, X.u(i, j, k));
    a.add(c25, X.u(i - 1, j, k + 1));
    a.add(c25, X.u(i, j, k + 1));
    a.add(c26, X.v(i, j - 1, k));
    a.add(c26, X.v(i, j, k));
    a.add(c26, X.v(i, j - 1, k + 1));
    a.add(c26, X.v(i, j, k + 1));
    const float2 half = make_float2(0.5f, 0.0f);
    a.add(half, X.T(i, j, k));
    a.add(half, X.T(i, j, k + 1));
    rw = a.value();
  }
  vstar[2 * P + e] = rw;
  const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
  if (cell) {
    Acc a;
    a.add(cf2(coef, P, 27, e), X.T(i, j, k));
    a.add(cf2(coef, P, 28, e), X.T(i - 1, j, k));
    a.add(cf2(coef, P, 29, e), X.T(i + 1, j, k));
    a.add(cf2(coef, P, 30, e), X.T(i, j - 1, k));
    a.add(cf2(coef, P, 31, e), X.T(i, j + 1, k));
    a.add(cf2(coef, P, 32, e), X.T(i, j, k - 1));
    a.add(cf2(coef, P, 33, e), X.T(i, j, k + 1));
    const float2 c34 = cf2(coef, P, 34, e), c35 = cf2(coef, P, 35, e), c36 = cf2(coef, P, 36, e);
    a.add(c34, X.u(i - 1, j, k));
    a.add(c34, X.u(i, j, k));
    a.add(c35, X.v(i, j - 1, k));
    a.add(c35, X.v(i, j, k));
    a.add(c36, X.w(i, j, k - 1));
    a.add(c36, X.w(i, j, k));
    const double r = a.value();
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

// FP32-pair copy of the FP64 coefficients: ch = fp32(c), cl = fp32(c - ch).
__global__ void __launch_bounds__(256) k_coef_df(const double* __restrict__ coef, float2* __restrict__ cdf, size_t n) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double c = coef[t];
    const float h = __double2float_rn(c);
    cdf[t] = make_float2(h, __double2float_rn(c - (double)h));
  }
}

}  // namespace

void kv_launch_stencil(const kv_grid* h, int mode, const double* base, const double* x, double* vstar,
                       double* tout, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1);
  dim3 grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  if (mode == 0)
    k_stencil<0><<<grid, block, 0, s>>>(g, base, x, h->P, vstar, tout);
  else
    k_stencil<1><<<grid, block, 0, s>>>(g, base, x, h->P, vstar, tout);
}

void kv_launch_assemble(const kv_grid* h, const double* base, double* coef, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  k_assemble<<<grid, block, 0, s>>>(g, base, h->P, coef);
}

void kv_launch_apply(const kv_grid* h, const double* coef, const double* x, double* vstar, double* tout,
                     cudaStream_t s) {
  const KvGeom& g = h->g;
  const int bx = h->apply_bx, by = h->apply_by;
  dim3 block(bx, by, 1), grid((g.X + bx - 1) / bx, (g.Y + by - 1) / by, g.Z);
  k_apply<<<grid, block, 0, s>>>(g, coef, x, h->P, vstar, tout);
}

void kv_launch_coef_df(const kv_grid* h, const double* coef, float2* cdf, cudaStream_t s) {
  k_coef_df<<<4 * 152, 256, 0, s>>>(coef, cdf, (size_t)KV_NCOEF * h->P);
}

void kv_launch_apply_df(const kv_grid* h, const float2* cdf, const double* x, double* vstar, double* tout,
                        cudaStream_t s) {
  const KvGeom& g = h->g;
  const int bx = h->df_bx, by = h->df_by;
  dim3 block(bx, by, 1), grid((g.X + bx - 1) / bx, (g.Y + by - 1) / by, g.Z);
  if (h->df_variant == 0)
    k_apply_df<3><<<grid, block, 0, s>>>(g, cdf, x, h->P, vstar, tout);
  else
    k_apply_df<1><<<grid, block, 0, s>>>(g, cdf, x, h->P, vstar, tout);
}
