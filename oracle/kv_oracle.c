/*
 * kv_oracle.c -- plain, slow FP64 CPU oracle for the Krylov-vector evaluation of
 * Gelfgat, "Instability of natural convection in a laterally heated cube with perfectly
 * conducting horizontal boundaries" (arXiv 1905.11601), Section 3.1.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code with the CUDA path.
 *
 * What it computes, for a state (U, Theta) and a vector x = (u, v, w, T):
 *   y = Pi_v (+) P_T  applied to  J(U, Theta) P_BC x
 * where
 *   P_BC   puts x into the space of Eq (13): velocity entries outside the interior faces are
 *          zeroed and the temperature is projected onto the homogeneous boundary conditions;
 *   J      is the linearised operator of Eqs (8)-(9), written as the right-hand sides of
 *          Eqs (11)-(12) without the pressure gradient;
 *   Pi_v   is the SIMPLE / Chorin loop of Section 3.1 (solve Laplace(phi) = div v with Neumann
 *          conditions, v -= grad phi, p += phi, restore boundary values), the Poisson
 *          equation solved by the tensor-product factorisation of Eqs (14)-(18);
 *   P_T    is the temperature projection of Eqs (19)-(21) (Gram-matrix form).
 *
 * Discretisation (the paper reuses the finite-volume schemes of its reference [11], which is
 * not given; the readings below are stated once here and used throughout):
 *   - MAC grid of the unit cube; every field stored padded as (nz+2)(ny+2)(nx+2), x fastest;
 *     p and T at cell centres, u/v/w on x/y/z faces;
 *   - faces of axis a at x_t = xi_t - s sin(2 pi xi_t), xi_t = t/n_a, t = 0..n_a (Eq 22, the
 *     stretching parameter s = or_grid.stretch; s = 0 is the uniform grid, h_a = 1/n_a); cell
 *     centres at the midpoints of their two faces; cell widths dx_t = x_t - x_{t-1};
 *   - along an axis a cell-like index t = 1..n sits at its cell centre, indices 0 and n+1 are
 *     wall nodes on the walls; a face-like index t = 0..n sits on face t (index n+1 is padding);
 *   - diffusion in flux form: ((f+ - f)/(x+ - x) - (f - f-)/(x - x-)) / w, w the width of the
 *     node's control volume: the cell width at a cell-like node, the distance between the two
 *     adjacent cell centres at a face-like node (both h on the uniform grid);
 *   - advection (a.grad) b in the advective form of Eqs (8)-(9): a 3-point (non-uniform next
 *     to walls) central first derivative of b at b's node, times the advecting velocity
 *     averaged (2 or 4 nearest stored values) to that node;
 *   - optional first-order upwind advection (adv = 1): the derivative of b along each axis is
 *     the one-sided difference towards the upstream neighbour (the backward difference where
 *     the selecting velocity, averaged to b's node as above, is >= 0, else the forward one),
 *     over the actual node gap (h/2 to a wall node). In the linearised operator the base
 *     velocity selects in both advection terms, (U.grad) v and (v.grad) U, so J is the exact
 *     derivative of the upwind residual wherever no averaged base velocity changes sign;
 *   - buoyancy T e_z on a w-face: mean of the two adjacent cell temperatures;
 *   - divergence / gradient: the MAC differences (divided by the cell width / the distance
 *     between the two cell centres); the Poisson operator is D G with the wall faces excluded
 *     (homogeneous Neumann), its zero mode removed (pseudo-inverse); on a stretched axis the
 *     1D factor of D G is not symmetric, and its eigenpairs (Eq 15) come from the symmetric
 *     matrix dx^1/2 (D G) dx^-1/2 and E^-1 from a plain inversion of E;
 *   - the SIMPLE test's h_min is the smallest cell width;
 *   - temperature projection reading "orthogonal" (tproj = 0): Eq (21) read as
 *     T^ = (P_x (x) P_y (x) P_z) T*, P_a = E_a G_a^-1 E_a^T with E_a the 1D eigenvectors of the
 *     homogeneous-BC temperature operator extended to the wall nodes, G_a = E_a^T E_a;
 *     reading "oblique" (tproj = 1): keep the interior, set the wall nodes from the BCs.
 *     The two differ only at insulated (Neumann) walls.
 *
 * Parity unpinned: none of the functions below; the pins live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int nx, ny, nz;
  int bc;    /* 0: conducting spanwise walls (Eq 6); 1: insulated spanwise walls (Eq 7) */
  int tproj; /* 0: orthogonal (Gram) reading of Eq (21); 1: oblique reading */
  double gr, pr;
  double stretch; /* Eq (22) stretching parameter s, 0 <= s < 1/(2 pi); 0: uniform grid */
  int adv;        /* advection scheme: 0 central (the default reading), 1 first-order upwind */
} or_grid;

typedef struct {
  int passes;      /* SIMPLE passes done */
  double max_div;  /* max |D v| after the last pass (absolute) */
  double rel_div;  /* max |D v| h / max |v| */
  double phi_norm; /* ||phi||_2 of the last pass */
} or_stats;

/* Per-grid data that Eqs (15)-(20) say is computed once. */
typedef struct {
  or_grid g;
  int n[3];
  double h[3];
  int stretched;  /* stretch != 0: the coordinates below replace t h */
  double *xf[3];  /* face coordinates, n+1 per axis (Eq 22) */
  double *xc[3];  /* cell-like coordinates, n+2 per axis: walls at 0 and 1, centres between */
  /* Neumann pressure Laplacian (Eq 14 for phi): eigenvectors E (n x n, row = node, col = mode),
     E^-1, eigenvalues. */
  double *Ep[3], *Epinv[3], *lamp[3];
  /* Temperature projection P_a ((n+2) x (n+2)), Eq (21) per axis. */
  double *Pt[3];
} or_ctx;

#define FU 0
#define FV 1
#define FW 2
#define FT 3

static size_t pidx(const or_ctx* c, int i, int j, int k) {
  return (size_t)i + (size_t)(c->n[0] + 2) * ((size_t)j + (size_t)(c->n[1] + 2) * (size_t)k);
}
static size_t plen(const or_ctx* c) {
  return (size_t)(c->n[0] + 2) * (c->n[1] + 2) * (c->n[2] + 2);
}
/* compact n^3 index (cells 1..n stored at 0..n-1) */
static size_t cidx(const or_ctx* c, int i, int j, int k) {
  return (size_t)i + (size_t)c->n[0] * ((size_t)j + (size_t)c->n[1] * (size_t)k);
}

/* Is field F face-like along axis a? */
static int face_like(int F, int a) { return F == a; }

/* Coordinate of index t along axis a for field F. */
static double coord(const or_ctx* c, int F, int a, int t) {
  int n = c->n[a];
  if (c->stretched) {
    if (face_like(F, a)) return c->xf[a][t < n ? t : n];
    return c->xc[a][t <= 0 ? 0 : (t >= n + 1 ? n + 1 : t)];
  }
  if (face_like(F, a)) return (double)t / n;
  if (t <= 0) return 0.0;
  if (t >= n + 1) return 1.0;
  return ((double)t - 0.5) / n;
}

/* Width of cell t (1..n) along axis a. */
static double cell_width(const or_ctx* c, int a, int t) {
  return c->stretched ? c->xf[a][t] - c->xf[a][t - 1] : c->h[a];
}

/* Distance between the centres of cells t and t+1 along axis a (face t, 1..n-1). */
static double centre_gap(const or_ctx* c, int a, int t) {
  return c->stretched ? c->xc[a][t + 1] - c->xc[a][t] : c->h[a];
}

/* Width of the control volume of entry t of field F along axis a. */
static double cv_width(const or_ctx* c, int F, int a, int t) {
  return face_like(F, a) ? centre_gap(c, a, t) : cell_width(c, a, t);
}

/* Is (i,j,k) an unknown (interior) entry of field F? */
static int is_dof(const or_ctx* c, int F, int i, int j, int k) {
  int t[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    int hi = face_like(F, a) ? c->n[a] - 1 : c->n[a];
    if (t[a] < 1 || t[a] > hi) return 0;
  }
  return 1;
}

static double at(const or_ctx* c, const double* f, int i, int j, int k) { return f[pidx(c, i, j, k)]; }

/* Value of f at (i,j,k) shifted by s along axis a. */
static double nb(const or_ctx* c, const double* f, int i, int j, int k, int a, int s) {
  int t[3] = {i, j, k};
  t[a] += s;
  return at(c, f, t[0], t[1], t[2]);
}

/* Second derivative along axis a, flux form, at entry (i,j,k) of field F. */
static double d2(const or_ctx* c, const double* f, int F, int a, int i, int j, int k) {
  int t[3] = {i, j, k};
  double xm = coord(c, F, a, t[a] - 1), x0 = coord(c, F, a, t[a]), xp = coord(c, F, a, t[a] + 1);
  double fm = nb(c, f, i, j, k, a, -1), f0 = at(c, f, i, j, k), fp = nb(c, f, i, j, k, a, +1);
  return ((fp - f0) / (xp - x0) - (f0 - fm) / (x0 - xm)) / cv_width(c, F, a, t[a]);
}

/* First derivative along axis a, 3-point central (non-uniform next to walls). */
static double d1(const or_ctx* c, const double* f, int F, int a, int i, int j, int k) {
  int t[3] = {i, j, k};
  double xm = coord(c, F, a, t[a] - 1), x0 = coord(c, F, a, t[a]), xp = coord(c, F, a, t[a] + 1);
  double fm = nb(c, f, i, j, k, a, -1), f0 = at(c, f, i, j, k), fp = nb(c, f, i, j, k, a, +1);
  double dm = x0 - xm, dp = xp - x0;
  return (dm * dm * (fp - f0) + dp * dp * (f0 - fm)) / (dm * dp * (dm + dp));
}

/* Velocity component ac (stored on faces normal to axis comp) averaged to the node (i,j,k) of
   field F: itself if F == comp; else the mean over the bracketing faces along comp (t-1, t)
   and, for a face field F, the bracketing cells along F (t, t+1). */
static double interp(const or_ctx* c, const double* ac, int comp, int F, int i, int j, int k) {
  if (F == comp) return at(c, ac, i, j, k);
  double s = 0.0;
  int cnt = 0;
  for (int dc = -1; dc <= 0; ++dc) {
    int dFmax = (F < 3) ? 1 : 0;
    for (int dF = 0; dF <= dFmax; ++dF) {
      int t[3] = {i, j, k};
      t[comp] += dc;
      if (F < 3) t[F] += dF;
      s += at(c, ac, t[0], t[1], t[2]);
      ++cnt;
    }
  }
  return s / cnt;
}

/* One-sided first derivative along axis a: backward (towards index t-1) if up, else forward. */
static double d1_side(const or_ctx* c, const double* f, int F, int a, int i, int j, int k, int up) {
  int t[3] = {i, j, k};
  double x0 = coord(c, F, a, t[a]), f0 = at(c, f, i, j, k);
  if (up) return (f0 - nb(c, f, i, j, k, a, -1)) / (x0 - coord(c, F, a, t[a] - 1));
  return (nb(c, f, i, j, k, a, +1) - f0) / (coord(c, F, a, t[a] + 1) - x0);
}

/* (a . grad) b at entry (i,j,k) of field F; a = (a0, a1, a2) on their faces. Central, or
   with adv = 1 upwind along each axis by the sign of sel's component averaged to the node. */
static double advect_sel(const or_ctx* c, const double* const a[3], const double* const sel[3],
                         const double* b, int F, int i, int j, int k) {
  double s = 0.0;
  for (int comp = 0; comp < 3; ++comp) {
    double db;
    if (c->g.adv) db = d1_side(c, b, F, comp, i, j, k, interp(c, sel[comp], comp, F, i, j, k) >= 0.0);
    else db = d1(c, b, F, comp, i, j, k);
    s += interp(c, a[comp], comp, F, i, j, k) * db;
  }
  return s;
}

static double laplace(const or_ctx* c, const double* f, int F, int i, int j, int k) {
  return d2(c, f, F, 0, i, j, k) + d2(c, f, F, 1, i, j, k) + d2(c, f, F, 2, i, j, k);
}

/* ---------------------------------------------------------------------------------------- */
/* small dense linear algebra (row-major)                                                    */

/* Inverse of an m x m matrix by Gauss-Jordan elimination with partial pivoting. */
static int gj_inverse(int m, const double* A, double* Ainv) {
  double* W = (double*)malloc(sizeof(double) * (size_t)m * 2 * m);
  if (!W) return -1;
  for (int r = 0; r < m; ++r)
    for (int q = 0; q < 2 * m; ++q) W[(size_t)r * 2 * m + q] = q < m ? A[(size_t)r * m + q] : (q - m == r);
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (fabs(W[(size_t)r * 2 * m + col]) > fabs(W[(size_t)piv * 2 * m + col])) piv = r;
    if (W[(size_t)piv * 2 * m + col] == 0.0) { free(W); return -2; }
    if (piv != col)
      for (int q = 0; q < 2 * m; ++q) {
        double t = W[(size_t)col * 2 * m + q];
        W[(size_t)col * 2 * m + q] = W[(size_t)piv * 2 * m + q];
        W[(size_t)piv * 2 * m + q] = t;
      }
    double d = W[(size_t)col * 2 * m + col];
    for (int q = 0; q < 2 * m; ++q) W[(size_t)col * 2 * m + q] /= d;
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      double f = W[(size_t)r * 2 * m + col];
      if (f == 0.0) continue;
      for (int q = 0; q < 2 * m; ++q) W[(size_t)r * 2 * m + q] -= f * W[(size_t)col * 2 * m + q];
    }
  }
  for (int r = 0; r < m; ++r)
    for (int q = 0; q < m; ++q) Ainv[(size_t)r * m + q] = W[(size_t)r * 2 * m + m + q];
  free(W);
  return 0;
}

/* Eigen-decomposition of a symmetric m x m matrix by cyclic Jacobi rotations.
   On return V holds the eigenvectors as columns, lam the eigenvalues. */
static void jacobi_eig(int m, const double* S, double* V, double* lam) {
  double* A = (double*)malloc(sizeof(double) * (size_t)m * m);
  memcpy(A, S, sizeof(double) * (size_t)m * m);
  for (int r = 0; r < m; ++r)
    for (int q = 0; q < m; ++q) V[(size_t)r * m + q] = (r == q);
  double fro = 0.0;
  for (size_t e = 0; e < (size_t)m * m; ++e) fro += A[e] * A[e];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off += A[(size_t)p * m + q] * A[(size_t)p * m + q];
    if (off <= 1e-32 * fro) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        double apq = A[(size_t)p * m + q];
        if (apq == 0.0) continue;
        double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int r = 0; r < m; ++r) { /* columns p, q */
          double arp = A[(size_t)r * m + p], arq = A[(size_t)r * m + q];
          A[(size_t)r * m + p] = cs * arp - sn * arq;
          A[(size_t)r * m + q] = sn * arp + cs * arq;
        }
        for (int r = 0; r < m; ++r) { /* rows p, q */
          double apr = A[(size_t)p * m + r], aqr = A[(size_t)q * m + r];
          A[(size_t)p * m + r] = cs * apr - sn * aqr;
          A[(size_t)q * m + r] = sn * apr + cs * aqr;
        }
        for (int r = 0; r < m; ++r) {
          double vrp = V[(size_t)r * m + p], vrq = V[(size_t)r * m + q];
          V[(size_t)r * m + p] = cs * vrp - sn * vrq;
          V[(size_t)r * m + q] = sn * vrp + cs * vrq;
        }
      }
  }
  for (int r = 0; r < m; ++r) lam[r] = A[(size_t)r * m + r];
  free(A);
}

/* ---------------------------------------------------------------------------------------- */
/* set-up: Eqs (14)-(15) for phi; Eqs (15), (19)-(21) for the temperature                    */

/* Is the temperature condition on the walls of axis a Dirichlet (homogeneous after
   linearisation)? x walls: Eq (4); z walls: Eq (5); y walls: Eq (6) (CC) or Eq (7) (AA). */
static int t_dirichlet(const or_ctx* c, int a) { return !(a == 1 && c->g.bc == 1); }

/* Eq (15) for the Neumann Laplacian D G of phi on a stretched axis a: the 1D matrix
   A = dx^-1 K (K symmetric: the flux differences with the wall faces excluded, weights 1 / the
   centre gaps) is similar to the symmetric S = dx^1/2 A dx^-1/2, so A = E Lambda E^-1 with
   E = dx^-1/2 Q, S = Q Lambda Q^T. Modes sorted by decreasing eigenvalue; mode 0 is the
   constant vector, whose eigenvalue is exactly 0 (every row of K sums to zero). */
static void stretched_neumann_axis(or_ctx* c, int a) {
  int n = c->n[a];
  double* S = (double*)calloc((size_t)n * n, sizeof(double));
  double* Q = (double*)malloc(sizeof(double) * n * n);
  double* lam = (double*)malloc(sizeof(double) * n);
  for (int t = 1; t <= n; ++t) {
    double dx = cell_width(c, a, t);
    if (t < n) {
      double g = centre_gap(c, a, t);
      S[(size_t)(t - 1) * n + (t - 1)] -= 1.0 / (g * dx);
      S[(size_t)(t - 1) * n + t] = 1.0 / (g * sqrt(dx * cell_width(c, a, t + 1)));
    }
    if (t > 1) {
      double g = centre_gap(c, a, t - 1);
      S[(size_t)(t - 1) * n + (t - 1)] -= 1.0 / (g * dx);
      S[(size_t)(t - 1) * n + (t - 2)] = 1.0 / (g * sqrt(dx * cell_width(c, a, t - 1)));
    }
  }
  jacobi_eig(n, S, Q, lam);
  int* order = (int*)malloc(sizeof(int) * n);
  for (int m = 0; m < n; ++m) order[m] = m;
  for (int m = 0; m < n; ++m) /* selection sort, largest first */
    for (int q = m + 1; q < n; ++q)
      if (lam[order[q]] > lam[order[m]]) { int tmp = order[m]; order[m] = order[q]; order[q] = tmp; }
  for (int m = 0; m < n; ++m) {
    c->lamp[a][m] = m == 0 ? 0.0 : lam[order[m]];
    for (int t = 0; t < n; ++t)
      c->Ep[a][(size_t)t * n + m] = Q[(size_t)t * n + order[m]] / sqrt(cell_width(c, a, t + 1));
  }
  gj_inverse(n, c->Ep[a], c->Epinv[a]);
  free(S); free(Q); free(lam); free(order);
}

or_ctx* or_create(const or_grid* g) {
  if (!g || g->nx < 2 || g->ny < 2 || g->nz < 2) return NULL;
  if (!(g->stretch >= 0.0 && g->stretch < 0.5 / M_PI)) return NULL; /* Eq (22) must stay monotone */
  if (g->adv != 0 && g->adv != 1) return NULL;
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->g = *g;
  c->n[0] = g->nx;
  c->n[1] = g->ny;
  c->n[2] = g->nz;
  c->stretched = g->stretch != 0.0;
  for (int a = 0; a < 3; ++a) {
    int n = c->n[a];
    double h = 1.0 / n;
    c->h[a] = h;
    c->xf[a] = (double*)malloc(sizeof(double) * (n + 1));
    c->xc[a] = (double*)malloc(sizeof(double) * (n + 2));
    for (int t = 0; t <= n; ++t) {
      double xi = (double)t / n;
      c->xf[a][t] = xi - g->stretch * sin(2.0 * M_PI * xi); /* Eq (22) */
    }
    c->xf[a][0] = 0.0;
    c->xf[a][n] = 1.0;
    c->xc[a][0] = 0.0;
    c->xc[a][n + 1] = 1.0;
    for (int t = 1; t <= n; ++t) c->xc[a][t] = 0.5 * (c->xf[a][t - 1] + c->xf[a][t]);
    c->Ep[a] = (double*)malloc(sizeof(double) * n * n);
    c->Epinv[a] = (double*)malloc(sizeof(double) * n * n);
    c->lamp[a] = (double*)malloc(sizeof(double) * n);
    if (c->stretched) {
      stretched_neumann_axis(c, a);
    } else {
      /* Eq (15) for the Neumann Laplacian of phi: closed-form eigenpairs of the 1D matrix
         (phi_{t+1} - 2 phi_t + phi_{t-1}) / h^2 with the wall terms dropped (cosine basis). */
      for (int m = 0; m < n; ++m) {
        double alpha = sqrt((m == 0 ? 1.0 : 2.0) / n);
        double s = sin(M_PI * m / (2.0 * n));
        c->lamp[a][m] = -4.0 / (h * h) * s * s;
        for (int t = 0; t < n; ++t) c->Ep[a][(size_t)t * n + m] = alpha * cos(M_PI * m * (t + 0.5) / n);
      }
      gj_inverse(n, c->Ep[a], c->Epinv[a]);
    }

    /* Eqs (15), (19)-(21) for the temperature: D_aa with the homogeneous BCs folded in,
       its eigenvectors E_a, extended to the two wall nodes by the same BCs. P_a depends only
       on the span of the extended E_a (every interior vector, wall nodes set by the BCs), so
       the uniform-grid D_aa serves a stretched axis as well. */
    double* D = (double*)calloc((size_t)n * n, sizeof(double));
    int dir = t_dirichlet(c, a);
    for (int t = 0; t < n; ++t) {
      /* flux to the right / left neighbour, distance h inside, h/2 to a wall node */
      double wr = (t == n - 1) ? 2.0 : 1.0, wl = (t == 0) ? 2.0 : 1.0;
      if (t < n - 1) { D[(size_t)t * n + t + 1] += 1.0 / (h * h); D[(size_t)t * n + t] -= 1.0 / (h * h); }
      else if (dir) D[(size_t)t * n + t] -= wr / (h * h); /* wall value 0 */
      if (t > 0) { D[(size_t)t * n + t - 1] += 1.0 / (h * h); D[(size_t)t * n + t] -= 1.0 / (h * h); }
      else if (dir) D[(size_t)t * n + t] -= wl / (h * h);
    }
    double* E = (double*)malloc(sizeof(double) * n * n);
    double* lam = (double*)malloc(sizeof(double) * n);
    jacobi_eig(n, D, E, lam);
    int m2 = n + 2;
    double* Ex = (double*)calloc((size_t)m2 * n, sizeof(double)); /* (n+2) x n */
    for (int t = 0; t < n; ++t)
      for (int m = 0; m < n; ++m) Ex[(size_t)(t + 1) * n + m] = E[(size_t)t * n + m];
    if (!dir)
      for (int m = 0; m < n; ++m) {
        Ex[(size_t)0 * n + m] = E[(size_t)0 * n + m];             /* T_0 = T_1 */
        Ex[(size_t)(n + 1) * n + m] = E[(size_t)(n - 1) * n + m]; /* T_{n+1} = T_n */
      }
    double* G = (double*)calloc((size_t)n * n, sizeof(double));
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        double s = 0.0;
        for (int t = 0; t < m2; ++t) s += Ex[(size_t)t * n + p] * Ex[(size_t)t * n + q];
        G[(size_t)p * n + q] = s;
      }
    double* Gi = (double*)malloc(sizeof(double) * n * n);
    gj_inverse(n, G, Gi);
    /* P_a = E_a G_a^-1 E_a^T, formed as E_a (G_a^-1 E_a^T) */
    double* GE = (double*)calloc((size_t)n * m2, sizeof(double)); /* n x (n+2) */
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < m2; ++q) {
        double s = 0.0;
        for (int p2 = 0; p2 < n; ++p2) s += Gi[(size_t)p * n + p2] * Ex[(size_t)q * n + p2];
        GE[(size_t)p * m2 + q] = s;
      }
    c->Pt[a] = (double*)calloc((size_t)m2 * m2, sizeof(double));
    for (int r = 0; r < m2; ++r)
      for (int q = 0; q < m2; ++q) {
        double s = 0.0;
        for (int p = 0; p < n; ++p) s += Ex[(size_t)r * n + p] * GE[(size_t)p * m2 + q];
        c->Pt[a][(size_t)r * m2 + q] = s;
      }
    free(GE);
    free(D); free(E); free(lam); free(Ex); free(G); free(Gi);
  }
  return c;
}

void or_destroy(or_ctx* c) {
  if (!c) return;
  for (int a = 0; a < 3; ++a) {
    free(c->Ep[a]); free(c->Epinv[a]); free(c->lamp[a]); free(c->Pt[a]);
    free(c->xf[a]); free(c->xc[a]);
  }
  free(c);
}

/* Exposes the 1D matrices for the tests: which = 0 -> E (pressure), 1 -> E^-1, 2 -> lambda,
   3 -> P_a (temperature projection, (n+2)^2), 4 -> face coordinates (n+1), 5 -> cell-like
   coordinates (n+2, walls included). */
int or_axis_data(const or_ctx* c, int a, int which, double* out) {
  int n = c->n[a];
  switch (which) {
    case 0: memcpy(out, c->Ep[a], sizeof(double) * n * n); return 0;
    case 1: memcpy(out, c->Epinv[a], sizeof(double) * n * n); return 0;
    case 2: memcpy(out, c->lamp[a], sizeof(double) * n); return 0;
    case 3: memcpy(out, c->Pt[a], sizeof(double) * (n + 2) * (n + 2)); return 0;
    case 4: memcpy(out, c->xf[a], sizeof(double) * (n + 1)); return 0;
    case 5: memcpy(out, c->xc[a], sizeof(double) * (n + 2)); return 0;
  }
  return -1;
}

/* ---------------------------------------------------------------------------------------- */
/* temperature projection                                                                    */

/* Eq (21), orthogonal reading: T^ = (P_x (x) P_y (x) P_z) T, one 1D dense product per axis. */
void or_tproj_gram(const or_ctx* c, const double* T, double* out) {
  size_t P = plen(c);
  double* a = (double*)malloc(sizeof(double) * P);
  double* b = (double*)malloc(sizeof(double) * P);
  memcpy(a, T, sizeof(double) * P);
  int X = c->n[0] + 2, Y = c->n[1] + 2, Z = c->n[2] + 2;
  for (int ax = 0; ax < 3; ++ax) {
    int m2 = c->n[ax] + 2;
    const double* Pa = c->Pt[ax];
#pragma omp parallel for
    for (int k = 0; k < Z; ++k)
      for (int j = 0; j < Y; ++j)
        for (int i = 0; i < X; ++i) {
          int t[3] = {i, j, k};
          double s = 0.0;
          for (int q = 0; q < m2; ++q) {
            int u[3] = {i, j, k};
            u[ax] = q;
            s += Pa[(size_t)t[ax] * m2 + q] * at(c, a, u[0], u[1], u[2]);
          }
          b[pidx(c, i, j, k)] = s;
        }
    double* tmp = a; a = b; b = tmp;
  }
  memcpy(out, a, sizeof(double) * P);
  free(a);
  free(b);
}

/* The same projection written out in closed form: Dirichlet axes zero both wall nodes; an
   insulated axis replaces each wall pair (T_0, T_1), (T_n, T_{n+1}) by its mean (orthogonal
   reading) or copies the interior value to the wall (oblique reading). In place. */
void or_tproj_closed(const or_ctx* c, double* T) {
  int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
  int tp = c->g.tproj;
  if (!t_dirichlet(c, 1)) {
    for (int k = 0; k < n2 + 2; ++k)
      for (int i = 0; i < n0 + 2; ++i) {
        double* lo0 = &T[pidx(c, i, 0, k)];
        double* lo1 = &T[pidx(c, i, 1, k)];
        double* hi0 = &T[pidx(c, i, n1 + 1, k)];
        double* hi1 = &T[pidx(c, i, n1, k)];
        if (tp == 0) {
          double ml = 0.5 * (*lo0 + *lo1), mh = 0.5 * (*hi0 + *hi1);
          *lo0 = *lo1 = ml;
          *hi0 = *hi1 = mh;
        } else {
          *lo0 = *lo1;
          *hi0 = *hi1;
        }
      }
  }
  for (int k = 0; k < n2 + 2; ++k)
    for (int j = 0; j < n1 + 2; ++j)
      for (int i = 0; i < n0 + 2; ++i) {
        int wall = (i == 0 || i == n0 + 1 || k == 0 || k == n2 + 1);
        if (t_dirichlet(c, 1)) wall = wall || j == 0 || j == n1 + 1;
        if (wall) T[pidx(c, i, j, k)] = 0.0;
      }
}

/* The temperature projection used by the Krylov map: Eq (21) (orthogonal reading) or the
   oblique reading. */
static void tproj(const or_ctx* c, const double* T, double* out) {
  if (c->g.tproj == 0) {
    or_tproj_gram(c, T, out);
  } else {
    memcpy(out, T, sizeof(double) * plen(c));
    or_tproj_closed(c, out);
  }
}

/* ---------------------------------------------------------------------------------------- */
/* P_BC (Eq 13's space) and the linearised operator                                         */

/* x (u|v|w|T, 4 padded fields) -> P_BC x. */
void or_project_input(const or_ctx* c, const double* x, double* out) {
  size_t P = plen(c);
  for (int F = 0; F < 3; ++F)
    for (int k = 0; k < c->n[2] + 2; ++k)
      for (int j = 0; j < c->n[1] + 2; ++j)
        for (int i = 0; i < c->n[0] + 2; ++i) {
          size_t e = pidx(c, i, j, k);
          out[F * P + e] = is_dof(c, F, i, j, k) ? x[F * P + e] : 0.0;
        }
  tproj(c, x + 3 * P, out + 3 * P);
}

/* Right-hand sides of Eqs (11)-(12) without grad p, for x already in Eq (13)'s space:
     T* = (Pr Gr^1/2)^-1 Lap T - (U.grad) T - (v.grad) Theta          (cells)
     v* = Gr^-1/2 Lap v - (U.grad) v - (v.grad) U + T e_z              (interior faces)
   Entries outside the interior are written as 0 (SIMPLE step 3 done before step 1). */
static double jx_point(const or_ctx* c, const double* base, const double* xp, int F, int i, int j, int k) {
  size_t P = plen(c);
  double nu = 1.0 / sqrt(c->g.gr), kappa = 1.0 / (c->g.pr * sqrt(c->g.gr));
  const double* Ub[3] = {base, base + P, base + 2 * P};
  const double* Th = base + 3 * P;
  const double* xv[3] = {xp, xp + P, xp + 2 * P};
  const double* xT = xp + 3 * P;
  double r;
  if (F == FT) {
    r = kappa * laplace(c, xT, FT, i, j, k) - advect_sel(c, Ub, Ub, xT, FT, i, j, k) -
        advect_sel(c, xv, Ub, Th, FT, i, j, k);
  } else {
    r = nu * laplace(c, xv[F], F, i, j, k) - advect_sel(c, Ub, Ub, xv[F], F, i, j, k) -
        advect_sel(c, xv, Ub, Ub[F], F, i, j, k);
    if (F == FW) r += 0.5 * (at(c, xT, i, j, k) + at(c, xT, i, j, k + 1));
  }
  return r;
}

void or_jx_raw(const or_ctx* c, const double* base, const double* xp, double* ystar) {
  size_t P = plen(c);
  memset(ystar, 0, sizeof(double) * 4 * P);
  for (int F = 0; F < 4; ++F) {
#pragma omp parallel for
    for (int k = 1; k <= c->n[2]; ++k)
      for (int j = 1; j <= c->n[1]; ++j)
        for (int i = 1; i <= c->n[0]; ++i) {
          if (!is_dof(c, F, i, j, k)) continue;
          ystar[F * P + pidx(c, i, j, k)] = jx_point(c, base, xp, F, i, j, k);
        }
  }
}

/* Steady residual of Eqs (1)-(2) at a state S = (U, V, W, Theta) carrying its own
   (inhomogeneous) wall values, without grad P; entries outside the interior are 0. */
void or_residual_raw(const or_ctx* c, const double* S, double* F_out) {
  size_t P = plen(c);
  double nu = 1.0 / sqrt(c->g.gr), kappa = 1.0 / (c->g.pr * sqrt(c->g.gr));
  const double* Us[3] = {S, S + P, S + 2 * P};
  const double* Th = S + 3 * P;
  memset(F_out, 0, sizeof(double) * 4 * P);
  for (int F = 0; F < 4; ++F) {
#pragma omp parallel for
    for (int k = 1; k <= c->n[2]; ++k)
      for (int j = 1; j <= c->n[1]; ++j)
        for (int i = 1; i <= c->n[0]; ++i) {
          if (!is_dof(c, F, i, j, k)) continue;
          double r;
          if (F == FT) {
            r = kappa * laplace(c, Th, FT, i, j, k) - advect_sel(c, Us, Us, Th, FT, i, j, k);
          } else {
            r = nu * laplace(c, Us[F], F, i, j, k) - advect_sel(c, Us, Us, Us[F], F, i, j, k);
            if (F == FW) r += 0.5 * (at(c, Th, i, j, k) + at(c, Th, i, j, k + 1));
          }
          F_out[F * P + pidx(c, i, j, k)] = r;
        }
  }
}

/* ---------------------------------------------------------------------------------------- */
/* SIMPLE / Chorin pieces                                                                    */

/* b = D v on cells (compact n^3 array). */
void or_divergence(const or_ctx* c, const double* vel, double* b) {
  size_t P = plen(c);
  const double *u = vel, *v = vel + P, *w = vel + 2 * P;
#pragma omp parallel for
  for (int k = 1; k <= c->n[2]; ++k)
    for (int j = 1; j <= c->n[1]; ++j)
      for (int i = 1; i <= c->n[0]; ++i)
        b[cidx(c, i - 1, j - 1, k - 1)] = (at(c, u, i, j, k) - at(c, u, i - 1, j, k)) / cell_width(c, 0, i) +
                                          (at(c, v, i, j, k) - at(c, v, i, j - 1, k)) / cell_width(c, 1, j) +
                                          (at(c, w, i, j, k) - at(c, w, i, j, k - 1)) / cell_width(c, 2, k);
}

/* out[..] = sum_q M[t][q] in[.. q ..] along axis a of a compact n^3 array (M is n x n,
   row index = output index). */
static void apply_axis(const or_ctx* c, const double* M, int a, const double* in, double* out) {
  int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2], na = c->n[a];
#pragma omp parallel for
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        int t[3] = {i, j, k};
        double s = 0.0;
        for (int q = 0; q < na; ++q) {
          int u[3] = {i, j, k};
          u[a] = q;
          s += M[(size_t)t[a] * na + q] * in[cidx(c, u[0], u[1], u[2])];
        }
        out[cidx(c, i, j, k)] = s;
      }
}

/* Eq (18): phi = (E_x (x) E_y (x) E_z) Lambda^-1 (E_x^-1 (x) E_y^-1 (x) E_z^-1) b, with the
   Neumann zero mode (Lambda = 0) dropped (pseudo-inverse). Compact n^3 arrays. */
void or_poisson_tpd(const or_ctx* c, const double* b, double* phi) {
  int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
  size_t N = (size_t)n0 * n1 * n2;
  double* t1 = (double*)malloc(sizeof(double) * N);
  double* t2 = (double*)malloc(sizeof(double) * N);
  apply_axis(c, c->Epinv[0], 0, b, t1);
  apply_axis(c, c->Epinv[1], 1, t1, t2);
  apply_axis(c, c->Epinv[2], 2, t2, t1);
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        double L = c->lamp[0][i] + c->lamp[1][j] + c->lamp[2][k]; /* Eq (17) */
        size_t e = cidx(c, i, j, k);
        t1[e] = (i == 0 && j == 0 && k == 0) ? 0.0 : t1[e] / L;
      }
  /* E_a applied along axis a: row index of E is the node, column the mode */
  apply_axis(c, c->Ep[0], 0, t1, t2);
  apply_axis(c, c->Ep[1], 1, t2, t1);
  apply_axis(c, c->Ep[2], 2, t1, phi);
  free(t1);
  free(t2);
}

/* Step 2: v -= grad phi on interior faces; p += phi on cells (p padded, may be NULL). */
void or_correct(const or_ctx* c, const double* phi, double* vel, double* p) {
  size_t P = plen(c);
  int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
  for (int F = 0; F < 3; ++F)
    for (int k = 1; k <= n2; ++k)
      for (int j = 1; j <= n1; ++j)
        for (int i = 1; i <= n0; ++i) {
          if (!is_dof(c, F, i, j, k)) continue;
          int t[3] = {i - 1, j - 1, k - 1}, u[3] = {i - 1, j - 1, k - 1};
          u[F] += 1;
          int tf[3] = {i, j, k};
          double g = (phi[cidx(c, u[0], u[1], u[2])] - phi[cidx(c, t[0], t[1], t[2])]) / centre_gap(c, F, tf[F]);
          vel[F * P + pidx(c, i, j, k)] -= g;
        }
  if (p)
    for (int k = 1; k <= n2; ++k)
      for (int j = 1; j <= n1; ++j)
        for (int i = 1; i <= n0; ++i) p[pidx(c, i, j, k)] += phi[cidx(c, i - 1, j - 1, k - 1)];
}

/* Step 3: restore the homogeneous velocity BCs (zero all non-interior entries). */
static void restore_velocity_bc(const or_ctx* c, double* vel) {
  size_t P = plen(c);
  for (int F = 0; F < 3; ++F)
    for (int k = 0; k < c->n[2] + 2; ++k)
      for (int j = 0; j < c->n[1] + 2; ++j)
        for (int i = 0; i < c->n[0] + 2; ++i)
          if (!is_dof(c, F, i, j, k)) vel[F * P + pidx(c, i, j, k)] = 0.0;
}

/* The SIMPLE loop of Section 3.1 on the velocity part of y (in place), p accumulated. */
static void simple_loop(const or_ctx* c, double* vel, double* p, double tol, int max_passes,
                        or_stats* st) {
  int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
  size_t N = (size_t)n0 * n1 * n2, P = plen(c);
  double* b = (double*)malloc(sizeof(double) * N);
  double* phi = (double*)malloc(sizeof(double) * N);
  double hmin = c->h[0];
  if (c->h[1] < hmin) hmin = c->h[1];
  if (c->h[2] < hmin) hmin = c->h[2];
  if (c->stretched) {
    hmin = 1.0;
    for (int a = 0; a < 3; ++a)
      for (int t = 1; t <= c->n[a]; ++t)
        if (cell_width(c, a, t) < hmin) hmin = cell_width(c, a, t);
  }
  int pass = 0;
  double maxdiv = 0.0, rel = 0.0, phin = 0.0;
  for (pass = 1; pass <= max_passes; ++pass) {
    restore_velocity_bc(c, vel);
    or_divergence(c, vel, b);
    or_poisson_tpd(c, b, phi);
    or_correct(c, phi, vel, p);
    phin = 0.0;
    for (size_t e = 0; e < N; ++e) phin += phi[e] * phi[e];
    phin = sqrt(phin);
    or_divergence(c, vel, b);
    maxdiv = 0.0;
    for (size_t e = 0; e < N; ++e) if (fabs(b[e]) > maxdiv) maxdiv = fabs(b[e]);
    double vmax = 0.0;
    for (size_t e = 0; e < 3 * P; ++e) if (fabs(vel[e]) > vmax) vmax = fabs(vel[e]);
    rel = vmax > 0 ? maxdiv * hmin / vmax : 0.0;
    if (rel < tol) break;
  }
  if (pass > max_passes) pass = max_passes;
  if (st) { st->passes = pass; st->max_div = maxdiv; st->rel_div = rel; st->phi_norm = phin; }
  free(b);
  free(phi);
}

/* ---------------------------------------------------------------------------------------- */
/* the Krylov map, the Newton residual and one Arnoldi step                                  */

/* y = (Pi_v (+) P_T) J P_BC x; p (padded cell field, may be NULL) receives the accumulated
   pressure sum(phi). */
void or_krylov_vector(const or_ctx* c, const double* base, const double* x, double* y, double* p,
                      double tol, int max_passes, or_stats* st) {
  size_t P = plen(c);
  double* xp = (double*)malloc(sizeof(double) * 4 * P);
  double* ys = (double*)malloc(sizeof(double) * 4 * P);
  or_project_input(c, x, xp);
  or_jx_raw(c, base, xp, ys);
  if (p) memset(p, 0, sizeof(double) * P);
  memcpy(y, ys, sizeof(double) * 3 * P);
  simple_loop(c, y, p, tol, max_passes, st);
  tproj(c, ys + 3 * P, y + 3 * P);
  free(xp);
  free(ys);
}

/* Newton step 2 (Section 3.1): the residual of Eqs (1)-(2) at the state S, projected like a
   Krylov vector (the pressure gradient drops out under Pi_v). Returns ||F||_2. */
double or_newton_residual(const or_ctx* c, const double* S, double* F, double tol, int max_passes) {
  size_t P = plen(c);
  double* r = (double*)malloc(sizeof(double) * 4 * P);
  double* out = F ? F : (double*)malloc(sizeof(double) * 4 * P);
  or_residual_raw(c, S, r);
  memcpy(out, r, sizeof(double) * 3 * P);
  simple_loop(c, out, NULL, tol, max_passes, NULL);
  tproj(c, r + 3 * P, out + 3 * P);
  double s = 0.0;
  for (size_t e = 0; e < 4 * P; ++e) s += out[e] * out[e];
  free(r);
  if (!F) free(out);
  return sqrt(s);
}

static double dot(size_t m, const double* a, const double* b) {
  double s = 0.0;
  for (size_t e = 0; e < m; ++e) s += a[e] * b[e];
  return s;
}

/* One Arnoldi step with classical Gram-Schmidt applied twice: V holds j+2 packed vectors
   (4 padded fields each); w = A V_j is orthogonalised against V_0..V_j, normalised and
   stored in V_{j+1}; h[0..j+1] receives the Hessenberg column. */
void or_arnoldi_step(const or_ctx* c, const double* base, double* V, int j, double* h, double tol,
                     int max_passes) {
  size_t L = 4 * plen(c);
  double* w = V + (size_t)(j + 1) * L;
  or_krylov_vector(c, base, V + (size_t)j * L, w, NULL, tol, max_passes, NULL);
  for (int q = 0; q <= j + 1; ++q) h[q] = 0.0;
  double* hh = (double*)malloc(sizeof(double) * (j + 1));
  for (int pass = 0; pass < 2; ++pass) {
    for (int q = 0; q <= j; ++q) hh[q] = dot(L, V + (size_t)q * L, w);
    for (int q = 0; q <= j; ++q) {
      const double* vq = V + (size_t)q * L;
      for (size_t e = 0; e < L; ++e) w[e] -= hh[q] * vq[e];
      h[q] += hh[q];
    }
  }
  double beta = sqrt(dot(L, w, w));
  h[j + 1] = beta;
  if (beta > 0)
    for (size_t e = 0; e < L; ++e) w[e] /= beta;
  free(hh);
}

/* ---------------------------------------------------------------------------------------- */
/* adjoint (transpose) of the Krylov map and the gradient of <y, A x> with respect to the   */
/* base state; entries are formed one by one from the definition of J (no transposed        */
/* stencil is written by hand)                                                               */

/* z = J_raw^T ys, where J_raw is the map xp -> or_jx_raw(base, xp) on all 4 padded fields:
   z[F', p] = sum over interior outputs (F, o) within one cell of p of ys[F, o] J[(F,o),(F',p)],
   each entry J[(F,o),(F',p)] = (J e_{F',p})[F, o] evaluated pointwise. */
void or_jt_raw(const or_ctx* c, const double* base, const double* ys, double* z) {
  size_t P = plen(c);
  int X = c->n[0] + 2, Y = c->n[1] + 2, Z = c->n[2] + 2;
  memset(z, 0, sizeof(double) * 4 * P);
#pragma omp parallel
  {
    double* unit = (double*)calloc(4 * P, sizeof(double));
#pragma omp for
    for (int k = 0; k < Z; ++k)
      for (int j = 0; j < Y; ++j)
        for (int i = 0; i < X; ++i)
          for (int Fp = 0; Fp < 4; ++Fp) {
            size_t q = Fp * P + pidx(c, i, j, k);
            unit[q] = 1.0;
            double acc = 0.0;
            for (int F = 0; F < 4; ++F)
              for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                  for (int di = -1; di <= 1; ++di) {
                    int oi = i + di, oj = j + dj, ok = k + dk;
                    if (!is_dof(c, F, oi, oj, ok)) continue;
                    double yo = ys[F * P + pidx(c, oi, oj, ok)];
                    if (yo == 0.0) continue;
                    acc += yo * jx_point(c, base, unit, F, oi, oj, ok);
                  }
            unit[q] = 0.0;
            z[q] = acc;
          }
    free(unit);
  }
}

/* Transpose of the Krylov map (orthogonal reading of the temperature projection, in which
   P_BC, Pi_v and P_T are all symmetric): z = P_BC J_raw^T (Pi_v (+) P_T) y. */
void or_krylov_adjoint(const or_ctx* c, const double* base, const double* y, double* z, double tol, int max_passes) {
  size_t P = plen(c);
  double* yh = (double*)malloc(sizeof(double) * 4 * P);
  double* g = (double*)malloc(sizeof(double) * 4 * P);
  memcpy(yh, y, sizeof(double) * 3 * P);
  simple_loop(c, yh, NULL, tol, max_passes, NULL); /* masks (step 3) and projects */
  tproj(c, y + 3 * P, yh + 3 * P);
  or_jt_raw(c, base, yh, g);
  or_project_input(c, g, z);
  free(yh);
  free(g);
}

/* gb[q] = d <ys, J(base) xp> / d base[q] for every entry q of the packed base state. J is
   affine in the base state, so the derivative is the exact difference J(e_q) - J(0) applied
   to xp, evaluated at the interior outputs within one cell of q. Central advection only (with
   upwinding J is not affine in the base state): NaN everywhere for adv = 1. */
void or_grad_base(const or_ctx* c, const double* xp, const double* ys, double* gb) {
  size_t P = plen(c);
  int X = c->n[0] + 2, Y = c->n[1] + 2, Z = c->n[2] + 2;
  if (c->g.adv) {
    for (size_t q = 0; q < 4 * P; ++q) gb[q] = NAN;
    return;
  }
  memset(gb, 0, sizeof(double) * 4 * P);
#pragma omp parallel
  {
    double* unit = (double*)calloc(4 * P, sizeof(double));
    double* zero = (double*)calloc(4 * P, sizeof(double));
#pragma omp for
    for (int k = 0; k < Z; ++k)
      for (int j = 0; j < Y; ++j)
        for (int i = 0; i < X; ++i)
          for (int Fb = 0; Fb < 4; ++Fb) {
            size_t q = Fb * P + pidx(c, i, j, k);
            unit[q] = 1.0;
            double acc = 0.0;
            for (int F = 0; F < 4; ++F)
              for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                  for (int di = -1; di <= 1; ++di) {
                    int oi = i + di, oj = j + dj, ok = k + dk;
                    if (!is_dof(c, F, oi, oj, ok)) continue;
                    double yo = ys[F * P + pidx(c, oi, oj, ok)];
                    if (yo == 0.0) continue;
                    acc += yo * (jx_point(c, unit, xp, F, oi, oj, ok) - jx_point(c, zero, xp, F, oi, oj, ok));
                  }
            unit[q] = 0.0;
            gb[q] = acc;
          }
    free(unit);
    free(zero);
  }
}

/* d <ys, J xp> / d Gr: J depends on Gr through nu = Gr^-1/2 and kappa = (Pr Gr^1/2)^-1. */
double or_grad_gr(const or_ctx* c, const double* xp, const double* ys) {
  size_t P = plen(c);
  double sv = 0.0, st = 0.0;
  const double* xv[3] = {xp, xp + P, xp + 2 * P};
  for (int F = 0; F < 4; ++F)
    for (int k = 1; k <= c->n[2]; ++k)
      for (int j = 1; j <= c->n[1]; ++j)
        for (int i = 1; i <= c->n[0]; ++i) {
          if (!is_dof(c, F, i, j, k)) continue;
          double yo = ys[F * P + pidx(c, i, j, k)];
          if (F == FT) st += yo * laplace(c, xp + 3 * P, FT, i, j, k);
          else sv += yo * laplace(c, xv[F], F, i, j, k);
        }
  double d = -0.5 * pow(c->g.gr, -1.5);
  return d * sv + d / c->g.pr * st;
}
