// Transpose of the Krylov map and the gradient of <y, A x> with respect to the base state.
//
// With the orthogonal reading of the temperature projection Eq (21), P_BC, Pi_v and P_T are all
// symmetric, so A^T = P_BC J^T (Pi_v (+) P_T). J^T is applied from the same assembled
// coefficients as J (kv_stencil.cu): each input entry gathers coefficient x output products
// from the outputs whose stencils read it. The base-state sensitivity of <y, A x> (adjoint
// eigenvector y and eigenvector x give the eigenvalue sensitivity) only involves the term
// -(v . grad) Theta of the energy equation for Theta and the viscous / conductive scalings for
// Gr (Eqs (8)-(9)).
#include "kv_internal.cuh"

namespace {

struct AdjGrid {
  KvGeom g;
  size_t P;
  __device__ __forceinline__ bool in(int i, int j, int k) const {
    return i >= 0 && i < g.X && j >= 0 && j < g.Y && k >= 0 && k < g.Z;
  }
  __device__ __forceinline__ int at(int i, int j, int k) const { return i + g.X * (j + g.Y * k); }
  // coefficient q of the output at (i, j, k) times field f there; 0 outside the padded box
  __device__ __forceinline__ double cy(const double* __restrict__ coef, int q, const double* __restrict__ f, int i,
                                       int j, int k) const {
    if (!in(i, j, k)) return 0.0;
    const int o = at(i, j, k);
    return __ldg(coef + (size_t)q * P + o) * __ldg(f + o);
  }
};

// Raw transpose of the temperature part at input entry (i, j, k): gathers the cell outputs'
// own-field coefficients, and the buoyancy weights of the two w-faces next to the cell.
__device__ __forceinline__ double gather_T(const AdjGrid& A, const double* __restrict__ coef,
                                           const double* __restrict__ yw, const double* __restrict__ yT, int i, int j,
                                           int k) {
  double r = A.cy(coef, 27, yT, i, j, k) + A.cy(coef, 28, yT, i + 1, j, k) + A.cy(coef, 29, yT, i - 1, j, k) +
             A.cy(coef, 30, yT, i, j + 1, k) + A.cy(coef, 31, yT, i, j - 1, k) + A.cy(coef, 32, yT, i, j, k + 1) +
             A.cy(coef, 33, yT, i, j, k - 1);
  // w-face (i, j, k) reads T(k) and T(k+1); w-face (i, j, k-1) reads T(k-1) and T(k)
  if (A.in(i, j, k)) r += 0.5 * __ldg(yw + A.at(i, j, k));
  if (A.in(i, j, k - 1)) r += 0.5 * __ldg(yw + A.at(i, j, k - 1));
  return r;
}

// z = P_BC J^T yh, yh = (Pi_v (+) P_T) y already projected (zero outside the output entries).
__global__ void __launch_bounds__(256) k_apply_t(KvGeom g, const double* __restrict__ coef,
                                                 const double* __restrict__ yh, size_t P, double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  AdjGrid A{g, P};
  const double* yu = yh;
  const double* yv = yh + P;
  const double* yw = yh + 2 * P;
  const double* yT = yh + 3 * P;
  const int e = A.at(i, j, k);
  const bool du = i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
  const bool dv = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz;
  const bool dw = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz - 1;
  double gu = 0.0, gv = 0.0, gw = 0.0;
  if (du) {
    // own u-face outputs: (i,j,k) c, (i+1) reads i as x-, (i-1) reads i as x+, ...
    gu = A.cy(coef, 0, yu, i, j, k) + A.cy(coef, 1, yu, i + 1, j, k) + A.cy(coef, 2, yu, i - 1, j, k) +
         A.cy(coef, 3, yu, i, j + 1, k) + A.cy(coef, 4, yu, i, j - 1, k) + A.cy(coef, 5, yu, i, j, k + 1) +
         A.cy(coef, 6, yu, i, j, k - 1);
    // v-faces (i', j') reading u at (i'-1, j'), (i', j'), (i'-1, j'+1), (i', j'+1)
    gu += A.cy(coef, 16, yv, i + 1, j, k) + A.cy(coef, 16, yv, i, j, k) + A.cy(coef, 16, yv, i + 1, j - 1, k) +
          A.cy(coef, 16, yv, i, j - 1, k);
    // w-faces (i', k') reading u at (i'-1, k'), (i', k'), (i'-1, k'+1), (i', k'+1)
    gu += A.cy(coef, 25, yw, i + 1, j, k) + A.cy(coef, 25, yw, i, j, k) + A.cy(coef, 25, yw, i + 1, j, k - 1) +
          A.cy(coef, 25, yw, i, j, k - 1);
    // cells i' reading u at i'-1 and i'
    gu += A.cy(coef, 34, yT, i + 1, j, k) + A.cy(coef, 34, yT, i, j, k);
  }
  if (dv) {
    gv = A.cy(coef, 9, yv, i, j, k) + A.cy(coef, 10, yv, i + 1, j, k) + A.cy(coef, 11, yv, i - 1, j, k) +
         A.cy(coef, 12, yv, i, j + 1, k) + A.cy(coef, 13, yv, i, j - 1, k) + A.cy(coef, 14, yv, i, j, k + 1) +
         A.cy(coef, 15, yv, i, j, k - 1);
    // u-faces (i', j') reading v at (i', j'-1), (i', j'), (i'+1, j'-1), (i'+1, j')
    gv += A.cy(coef, 7, yu, i, j + 1, k) + A.cy(coef, 7, yu, i, j, k) + A.cy(coef, 7, yu, i - 1, j + 1, k) +
          A.cy(coef, 7, yu, i - 1, j, k);
    // w-faces (j', k') reading v at (j'-1, k'), (j', k'), (j'-1, k'+1), (j', k'+1)
    gv += A.cy(coef, 26, yw, i, j + 1, k) + A.cy(coef, 26, yw, i, j, k) + A.cy(coef, 26, yw, i, j + 1, k - 1) +
          A.cy(coef, 26, yw, i, j, k - 1);
    gv += A.cy(coef, 35, yT, i, j + 1, k) + A.cy(coef, 35, yT, i, j, k);
  }
  if (dw) {
    gw = A.cy(coef, 18, yw, i, j, k) + A.cy(coef, 19, yw, i + 1, j, k) + A.cy(coef, 20, yw, i - 1, j, k) +
         A.cy(coef, 21, yw, i, j + 1, k) + A.cy(coef, 22, yw, i, j - 1, k) + A.cy(coef, 23, yw, i, j, k + 1) +
         A.cy(coef, 24, yw, i, j, k - 1);
    // u-faces (i', k') reading w at (i', k'-1), (i', k'), (i'+1, k'-1), (i'+1, k')
    gw += A.cy(coef, 8, yu, i, j, k + 1) + A.cy(coef, 8, yu, i, j, k) + A.cy(coef, 8, yu, i - 1, j, k + 1) +
          A.cy(coef, 8, yu, i - 1, j, k);
    // v-faces (j', k') reading w at (j', k'-1), (j', k'), (j'+1, k'-1), (j'+1, k')
    gw += A.cy(coef, 17, yv, i, j, k + 1) + A.cy(coef, 17, yv, i, j, k) + A.cy(coef, 17, yv, i, j - 1, k + 1) +
          A.cy(coef, 17, yv, i, j - 1, k);
    gw += A.cy(coef, 36, yT, i, j, k + 1) + A.cy(coef, 36, yT, i, j, k);
  }
  z[e] = gu;
  z[P + e] = gv;
  z[2 * P + e] = gw;
  // temperature: raw transpose, then P_T (symmetric in the orthogonal reading)
  double t = 0.0;
  const bool xz_in = i >= 1 && i <= g.nx && k >= 1 && k <= g.nz;
  if (xz_in) {
    if (g.bc == KV_BC_CC) {
      if (j >= 1 && j <= g.ny) t = gather_T(A, coef, yw, yT, i, j, k);
    } else if (j <= 1 || j >= g.ny) {
      const int jw = j <= 1 ? 0 : g.ny + 1, jn = j <= 1 ? 1 : g.ny;
      t = 0.5 * (gather_T(A, coef, yw, yT, i, jw, k) + gather_T(A, coef, yw, yT, i, jn, k));
    } else {
      t = gather_T(A, coef, yw, yT, i, j, k);
    }
  }
  z[3 * P + e] = t;
}

// yh = mask(y_vel) into vel (the velocity part's input to Pi_v) and P_T y_T into tout.
__global__ void __launch_bounds__(256) k_adj_prep(KvGeom g, const double* __restrict__ y, size_t P,
                                                  double* __restrict__ vel, double* __restrict__ tout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  const int e = i + g.X * (j + g.Y * k);
  const bool du = i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
  const bool dv = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz;
  const bool dw = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz - 1;
  vel[e] = du ? y[e] : 0.0;
  vel[P + e] = dv ? y[P + e] : 0.0;
  vel[2 * P + e] = dw ? y[2 * P + e] : 0.0;
  const double* T = y + 3 * P;
  double t = 0.0;
  if (i >= 1 && i <= g.nx && k >= 1 && k <= g.nz) {
    if (g.bc == KV_BC_CC) {
      if (j >= 1 && j <= g.ny) t = T[e];
    } else if (j <= 1 || j >= g.ny) {
      const int jw = j <= 1 ? 0 : g.ny + 1, jn = j <= 1 ? 1 : g.ny;
      t = 0.5 * (T[i + g.X * (jw + g.Y * k)] + T[i + g.X * (jn + g.Y * k)]);
    } else {
      t = T[e];
    }
  }
  tout[e] = t;
}

__device__ __forceinline__ double xmask(const KvGeom& g, const double* __restrict__ f, int F, int i, int j, int k) {
  bool d;
  if (F == 0) d = i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
  else if (F == 1) d = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz;
  else d = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz - 1;
  return d ? __ldg(f + i + g.X * (j + g.Y * k)) : 0.0;
}

// first-derivative weights at a cell-like index (as in kv_stencil.cu)
__device__ __forceinline__ void d1w(int t, int n, double ih, double& m, double& c, double& p) {
  if (t == 1) { m = -4.0 / 3.0 * ih; c = ih; p = 1.0 / 3.0 * ih; }
  else if (t == n) { m = -1.0 / 3.0 * ih; c = -ih; p = 4.0 / 3.0 * ih; }
  else { m = -0.5 * ih; c = 0.0; p = 0.5 * ih; }
}

// g(q) = d <yT, J_T x> / d Theta(q) = - sum over cells o next to q (and q itself) along each
// axis of a(o) yT(o) w(o; q - o): a = x's velocity averaged to the cell, w the first-derivative
// weight that Theta(q) carries at o.
__global__ void __launch_bounds__(256) k_grad_theta(KvGeom g, const double* __restrict__ x,
                                                    const double* __restrict__ yT, size_t P, double* __restrict__ gt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  const int q[3] = {i, j, k};
  const int n[3] = {g.nx, g.ny, g.nz};
  const double ih[3] = {g.ihx, g.ihy, g.ihz};
  double s = 0.0;
  for (int ax = 0; ax < 3; ++ax)
    for (int off = -1; off <= 1; ++off) {  // output cell o = q + off along ax
      int o[3] = {q[0], q[1], q[2]};
      o[ax] += off;
      if (!(o[0] >= 1 && o[0] <= g.nx && o[1] >= 1 && o[1] <= g.ny && o[2] >= 1 && o[2] <= g.nz)) continue;
      double m, c, p;
      d1w(o[ax], n[ax], ih[ax], m, c, p);
      const double w = off == 1 ? m : (off == 0 ? c : p);  // Theta(q) = Theta(o - off)
      if (w == 0.0) continue;
      int lo[3] = {o[0], o[1], o[2]};
      lo[ax] -= 1;
      const double a = 0.5 * (xmask(g, x + (size_t)ax * P, ax, lo[0], lo[1], lo[2]) +
                              xmask(g, x + (size_t)ax * P, ax, o[0], o[1], o[2]));
      s += a * __ldg(yT + o[0] + g.X * (o[1] + g.Y * o[2])) * w;
    }
  gt[i + g.X * (j + g.Y * k)] = -s;
}

// P_BC x's temperature read on the fly (as in the forward stencil)
__device__ __forceinline__ double xT_proj(const KvGeom& g, const double* __restrict__ T, int i, int j, int k) {
  if (i < 1 || i > g.nx || k < 1 || k > g.nz) return 0.0;
  if (g.bc == KV_BC_CC) return (j < 1 || j > g.ny) ? 0.0 : __ldg(T + i + g.X * (j + g.Y * k));
  if (j <= 1 || j >= g.ny) {
    const int jw = j <= 1 ? 0 : g.ny + 1, jn = j <= 1 ? 1 : g.ny;
    return 0.5 * (__ldg(T + i + g.X * (jw + g.Y * k)) + __ldg(T + i + g.X * (jn + g.Y * k)));
  }
  return __ldg(T + i + g.X * (j + g.Y * k));
}

__device__ __forceinline__ bool dof(const KvGeom& g, int F, const int o[3]) {
  const int n[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) {
    const int hi = (F == a) ? n[a] - 1 : n[a];
    if (o[a] < 1 || o[a] > hi) return false;
  }
  return true;
}

// value of P_BC x for field F at o (velocity masked, temperature projected)
__device__ __forceinline__ double xval(const KvGeom& g, const double* __restrict__ x, size_t P, int F, const int o[3]) {
  if (F == 3) return xT_proj(g, x + 3 * P, o[0], o[1], o[2]);
  return xmask(g, x + (size_t)F * P, F, o[0], o[1], o[2]);
}

// first-derivative weights along axis a at index t for a field that is face-like along a or not
__device__ __forceinline__ void d1w_any(bool face, int t, int n, double ih, double& m, double& c, double& p) {
  if (face) { m = -0.5 * ih; c = 0.0; p = 0.5 * ih; }
  else d1w(t, n, ih, m, c, p);
}

// D1 along axis a of (P_BC x)_F at the node o of field F
__device__ __forceinline__ double d1x(const KvGeom& g, const double* __restrict__ x, size_t P, int F, int a,
                                      const int o[3]) {
  const int n[3] = {g.nx, g.ny, g.nz};
  const double ih[3] = {g.ihx, g.ihy, g.ihz};
  double m, c, p;
  d1w_any(F == a, o[a], n[a], ih[a], m, c, p);
  int lo[3] = {o[0], o[1], o[2]}, hi[3] = {o[0], o[1], o[2]};
  lo[a] -= 1;
  hi[a] += 1;
  return m * xval(g, x, P, F, lo) + c * xval(g, x, P, F, o) + p * xval(g, x, P, F, hi);
}

// (P_BC x)_{cp} averaged to the node o of the velocity field c (cp != c): 4 points
__device__ __forceinline__ double interp4(const KvGeom& g, const double* __restrict__ x, size_t P, int cp, int c,
                                          const int o[3]) {
  double s = 0.0;
  for (int dc = -1; dc <= 0; ++dc)
    for (int dF = 0; dF <= 1; ++dF) {
      int t[3] = {o[0], o[1], o[2]};
      t[cp] += dc;
      t[c] += dF;
      s += xval(g, x, P, cp, t);
    }
  return 0.25 * s;
}

// d <yh, J x> / d U_c(q) for the three base velocity components c at the padded entry q:
// (A) J's advecting-velocity factors I_{c->F}(U_c) in every equation F, (B) the gradients
// D1(U_c) of the c-momentum equation's term -(v . grad) U_c.
__global__ void __launch_bounds__(256) k_grad_vel(KvGeom g, const double* __restrict__ x,
                                                  const double* __restrict__ yh, size_t P, double* __restrict__ gv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y || k >= g.Z) return;
  const int q[3] = {i, j, k};
  const int n[3] = {g.nx, g.ny, g.nz};
  const double ih[3] = {g.ihx, g.ihy, g.ihz};
  const int e = i + g.X * (j + g.Y * k);
  auto yv = [&](int F, const int o[3]) { return __ldg(yh + (size_t)F * P + o[0] + g.X * (o[1] + g.Y * o[2])); };
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    // (A) U_c(q) as advecting velocity
    for (int F = 0; F < 4; ++F) {
      if (F == c) {
        if (dof(g, c, q)) s -= d1x(g, x, P, c, c, q) * yv(c, q);
      } else if (F < 3) {
        // F-face o reads U_c at (o_c - 1, o_c) x (o_F, o_F + 1)
        for (int dc = 0; dc <= 1; ++dc)
          for (int dF = -1; dF <= 0; ++dF) {
            int o[3] = {q[0], q[1], q[2]};
            o[c] += dc;
            o[F] += dF;
            if (dof(g, F, o)) s -= 0.25 * d1x(g, x, P, F, c, o) * yv(F, o);
          }
      } else {
        // cell o reads U_c at o_c - 1 and o_c
        for (int dc = 0; dc <= 1; ++dc) {
          int o[3] = {q[0], q[1], q[2]};
          o[c] += dc;
          if (dof(g, 3, o)) s -= 0.5 * d1x(g, x, P, 3, c, o) * yv(3, o);
        }
      }
    }
    // (B) U_c(q) inside D1_{cp}(U_c) at the c-faces o = q + off e_cp
    for (int cp = 0; cp < 3; ++cp)
      for (int off = -1; off <= 1; ++off) {
        int o[3] = {q[0], q[1], q[2]};
        o[cp] += off;
        if (!dof(g, c, o)) continue;
        double m, cc, p;
        d1w_any(cp == c, o[cp], n[cp], ih[cp], m, cc, p);
        const double w = off == 1 ? m : (off == 0 ? cc : p);
        if (w == 0.0) continue;
        const double a = (cp == c) ? xval(g, x, P, c, o) : interp4(g, x, P, cp, c, o);
        s -= a * yv(c, o) * w;
      }
    gv[(size_t)c * P + e] = s;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// second-derivative weights (flux form, wall nodes at h/2)
__device__ __forceinline__ void d2w(bool face, int t, int n, double ih2, double& m, double& c, double& p) {
  if (face || (t != 1 && t != n)) { m = ih2; c = -2.0 * ih2; p = ih2; }
  else if (t == 1) { m = 2.0 * ih2; c = -3.0 * ih2; p = ih2; }
  else { m = ih2; c = -3.0 * ih2; p = 2.0 * ih2; }
}

// sums[0] += <yh_vel, Lap x_vel>, sums[1] += <yh_T, Lap P_T x_T> (block partials, atomics)
__global__ void __launch_bounds__(256) k_lap_dot(KvGeom g, const double* __restrict__ x, const double* __restrict__ yh,
                                                 size_t P, double* __restrict__ sums) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double sv = 0.0, st = 0.0;
  if (i < g.X && j < g.Y && k < g.Z) {
    const int t[3] = {i, j, k};
    const int n[3] = {g.nx, g.ny, g.nz};
    const double ih2[3] = {g.ihx * g.ihx, g.ihy * g.ihy, g.ihz * g.ihz};
    const int e = i + g.X * (j + g.Y * k);
    for (int F = 0; F < 3; ++F) {
      const double yo = yh[(size_t)F * P + e];
      if (yo == 0.0) continue;
      const double* f = x + (size_t)F * P;
      double lap = 0.0;
      for (int ax = 0; ax < 3; ++ax) {
        double m, c, p;
        d2w(ax == F, t[ax], n[ax], ih2[ax], m, c, p);
        int a[3] = {i, j, k}, b[3] = {i, j, k};
        a[ax] -= 1;
        b[ax] += 1;
        lap += m * xmask(g, f, F, a[0], a[1], a[2]) + c * xmask(g, f, F, i, j, k) +
               p * xmask(g, f, F, b[0], b[1], b[2]);
      }
      sv += yo * lap;
    }
    const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
    if (cell) {
      // P_T x_T read on the fly (as in the forward stencil)
      auto lT = [&](int ii, int jj, int kk) -> double {
        const double* T = x + 3 * P;
        if (ii < 1 || ii > g.nx || kk < 1 || kk > g.nz) return 0.0;
        if (g.bc == KV_BC_CC) return (jj < 1 || jj > g.ny) ? 0.0 : T[ii + g.X * (jj + g.Y * kk)];
        if (jj <= 1 || jj >= g.ny) {
          const int jw = jj <= 1 ? 0 : g.ny + 1, jn = jj <= 1 ? 1 : g.ny;
          return 0.5 * (T[ii + g.X * (jw + g.Y * kk)] + T[ii + g.X * (jn + g.Y * kk)]);
        }
        return T[ii + g.X * (jj + g.Y * kk)];
      };
      double lap = 0.0;
      for (int ax = 0; ax < 3; ++ax) {
        double m, c, p;
        d2w(false, t[ax], n[ax], ih2[ax], m, c, p);
        int a[3] = {i, j, k}, b[3] = {i, j, k};
        a[ax] -= 1;
        b[ax] += 1;
        lap += m * lT(a[0], a[1], a[2]) + c * lT(i, j, k) + p * lT(b[0], b[1], b[2]);
      }
      st = yh[3 * P + e] * lap;
    }
  }
  sv = warp_sum(sv);
  st = warp_sum(st);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums, sv);
    atomicAdd(sums + 1, st);
  }
}

}  // namespace

void kv_launch_adj_prep(const kv_grid* h, const double* y, double* vel, double* tout, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  k_adj_prep<<<grid, block, 0, s>>>(g, y, h->P, vel, tout);
}

void kv_launch_apply_t(const kv_grid* h, const double* coef, const double* yh, double* z, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  k_apply_t<<<grid, block, 0, s>>>(g, coef, yh, h->P, z);
}

void kv_launch_grad_theta(const kv_grid* h, const double* x, const double* yT, double* gt, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  k_grad_theta<<<grid, block, 0, s>>>(g, x, yT, h->P, gt);
}

void kv_launch_grad_vel(const kv_grid* h, const double* x, const double* yh, double* gv, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  k_grad_vel<<<grid, block, 0, s>>>(g, x, yh, h->P, gv);
}

void kv_launch_lap_dot(const kv_grid* h, const double* x, const double* yh, double* sums, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  k_lap_dot<<<grid, block, 0, s>>>(g, x, yh, h->P, sums);
}
