// C ABI of libkv: grid handles, the Krylov-vector map, one Arnoldi step and the Newton
// residual (arXiv 1905.11601, Section 3.1). See include/kv.h for the contract.
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kv_internal.cuh"

namespace {

thread_local std::string g_create_error;

const char* const kPhaseName[KV_NPHASE] = {"kv:operator", "kv:divergence", "kv:tpf-contraction", "kv:correct",
                                           "kv:arnoldi-normalise", "kv:refine-residual", "kv:gs-dots",
                                           "kv:gs-update"};

#define KV_CHECK_CUDA(h, call)                                                              \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                        \
      return e_ == cudaErrorMemoryAllocation ? KV_ERR_NOMEM : KV_ERR_CUDA;                  \
    }                                                                                       \
  } while (0)

kv_status fail(kv_grid* h, kv_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

// Launch-error check after queuing kernels (does not synchronise).
kv_status check_launch(kv_grid* h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, KV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return KV_OK;
}

// Eq (15) for the pressure-correction Laplacian D G with homogeneous Neumann conditions on a
// uniform axis: eigenvectors alpha_m cos(pi m (t + 1/2) / n), eigenvalues -(4/h^2) sin^2(pi m / 2n).
// E is orthogonal, so E^-1 = E^T. Computed in long double, rounded once.
void neumann_axis(int n, std::vector<double>& fwd, std::vector<double>& inv, std::vector<double>& lam) {
  fwd.assign((size_t)n * n, 0.0);
  inv.assign((size_t)n * n, 0.0);
  lam.assign(n, 0.0);
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double h = 1.0L / n;
  for (int m = 0; m < n; ++m) {
    const long double alpha = sqrtl((m == 0 ? 1.0L : 2.0L) / n);
    const long double s = sinl(pi * m / (2.0L * n));
    lam[m] = (double)(-4.0L / (h * h) * s * s);
    for (int t = 0; t < n; ++t) {
      const double e = (double)(alpha * cosl(pi * m * (t + 0.5L) / n));
      fwd[(size_t)m * n + t] = e;  // forward: row = mode, column = node (E^-1 = E^T)
      inv[(size_t)t * n + m] = e;  // inverse: row = node, column = mode (E)
    }
  }
}

// Eigen-decomposition of a symmetric tridiagonal matrix (diagonal d, off-diagonal e[i]
// coupling rows i and i+1, e[n-1] unused) by the implicit QL iteration with Wilkinson shifts
// (Bowdler, Martin, Reinsch and Wilkinson, Numer. Math. 11, 1968). On return d holds the
// eigenvalues and column c of Z (row-major n x n, set to the identity here) the eigenvector of
// d[c]. Returns false if an eigenvalue did not converge within 60 QL sweeps.
bool tridiag_ql(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Z) {
  Z.assign((size_t)n * n, 0.0);
  for (int r = 0; r < n; ++r) Z[(size_t)r * n + r] = 1.0;
  e.resize(n);
  e[n - 1] = 0.0;
  for (int l = 0; l < n; ++l) {
    for (int sweep = 0;; ++sweep) {
      // the first negligible off-diagonal at or below row l splits the matrix there
      int m = l;
      while (m < n - 1 && fabs(e[m]) > 0x1p-53 * (fabs(d[m]) + fabs(d[m + 1]))) ++m;
      if (m == l) break;
      if (sweep == 60) return false;
      // shift: the eigenvalue of the leading 2x2 block nearer to d[l]
      const double theta = (d[l + 1] - d[l]) / (2.0 * e[l]);
      const double rho = hypot(theta, 1.0);
      double x = d[m] - d[l] + e[l] / (theta + copysign(rho, theta));
      // chase the bulge from row m up to row l with plane rotations
      double sn = 1.0, cs = 1.0, carry = 0.0;
      bool split = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = sn * e[i], b = cs * e[i];
        const double r = hypot(f, x);
        e[i + 1] = r;
        if (r == 0.0) {  // underflow: the matrix splits at i+1
          d[i + 1] -= carry;
          e[m] = 0.0;
          split = true;
          break;
        }
        sn = f / r;
        cs = x / r;
        const double y = d[i + 1] - carry;
        const double t = (d[i] - y) * sn + 2.0 * cs * b;
        carry = sn * t;
        d[i + 1] = y + carry;
        x = cs * t - b;
        for (int k = 0; k < n; ++k) {
          double* zr = &Z[(size_t)k * n];
          const double z1 = zr[i + 1], z0 = zr[i];
          zr[i + 1] = sn * z0 + cs * z1;
          zr[i] = cs * z0 - sn * z1;
        }
      }
      if (split) continue;
      d[l] -= carry;
      e[l] = x;
      e[m] = 0.0;
    }
  }
  return true;
}

// A stretched axis (Eq 22) with n cells and parameter sp: faces x_t = xi_t - sp sin(2 pi xi_t),
// cell centres at face midpoints, wall nodes at 0 and 1. Fills the KV_SW_N table rows (n+2
// each) of the operator weights, divergence and gradient, and the eigen-decomposition of
// Eq (15) for the pressure-correction Laplacian D G: its 1D factor A = dx^-1 K is similar to
// the symmetric tridiagonal S = dx^-1/2 K dx^-1/2 = Q Lambda Q^T, so E = dx^-1/2 Q and
// E^-1 = Q^T dx^1/2. Modes sorted by decreasing eigenvalue; mode 0 (the constants) has
// eigenvalue exactly 0. Layout of fwd / inv as in neumann_axis.
bool stretched_axis(int n, double sp, std::vector<double>& tab, std::vector<double>& fwd, std::vector<double>& inv,
                    std::vector<double>& lam, double& hmin, bool want_eigen = true) {
  const int L = n + 2;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> xf(n + 1), xc(n + 2), dx(n + 2, 0.0), gap(n + 2, 0.0);
  for (int t = 0; t <= n; ++t) {
    const double xi = (double)t / n;
    xf[t] = xi - sp * sin(two_pi * xi);
  }
  xf[0] = 0.0;
  xf[n] = 1.0;
  xc[0] = 0.0;
  xc[n + 1] = 1.0;
  for (int t = 1; t <= n; ++t) xc[t] = 0.5 * (xf[t - 1] + xf[t]);
  for (int t = 1; t <= n; ++t) dx[t] = xf[t] - xf[t - 1];
  for (int t = 1; t < n; ++t) gap[t] = xc[t + 1] - xc[t];
  hmin = 1.0;
  for (int t = 1; t <= n; ++t) hmin = fmin(hmin, dx[t]);

  tab.assign((size_t)KV_SW_N * L, 0.0);
  auto row = [&](int r, int t) -> double& { return tab[(size_t)r * L + t]; };
  // 3-point weights at x0 between xm and xp: first derivative (exact for quadratics) and the
  // flux-form second derivative over a control volume of width w
  auto put = [&](int r1, int r2, int t, double xm, double x0, double xp, double w) {
    const double dm = x0 - xm, dp = xp - x0;
    row(r1, t) = -dp / (dm * (dm + dp));
    row(r1 + 1, t) = (dp - dm) / (dm * dp);
    row(r1 + 2, t) = dm / (dp * (dm + dp));
    const double wm = 1.0 / (dm * w), wp = 1.0 / (dp * w);
    row(r2, t) = wm;
    row(r2 + 1, t) = -(wm + wp);
    row(r2 + 2, t) = wp;
  };
  for (int t = 1; t <= n; ++t) {
    row(KV_SW_IDC, t) = 1.0 / dx[t];
    put(KV_SW_C1, KV_SW_C2, t, xc[t - 1], xc[t], xc[t + 1], dx[t]);
  }
  for (int t = 1; t < n; ++t) {
    row(KV_SW_IDF, t) = 1.0 / gap[t];
    put(KV_SW_F1, KV_SW_F2, t, xf[t - 1], xf[t], xf[t + 1], gap[t]);
  }

  if (!want_eigen) return true;
  // S on cells c = 0..n-1 (cell t = c + 1)
  std::vector<double> d(n, 0.0), e(n, 0.0), Q;
  for (int c = 0; c < n; ++c) {
    const int t = c + 1;
    if (t < n) d[c] -= 1.0 / (gap[t] * dx[t]);
    if (t > 1) d[c] -= 1.0 / (gap[t - 1] * dx[t]);
    if (t < n) e[c] = 1.0 / (gap[t] * sqrt(dx[t] * dx[t + 1]));
  }
  if (!tridiag_ql(n, d, e, Q)) return false;
  std::vector<int> order(n);
  for (int m = 0; m < n; ++m) order[m] = m;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return d[a] > d[b]; });
  fwd.assign((size_t)n * n, 0.0);
  inv.assign((size_t)n * n, 0.0);
  lam.assign(n, 0.0);
  for (int m = 0; m < n; ++m) {
    const int q = order[m];
    lam[m] = m == 0 ? 0.0 : d[q];
    for (int c = 0; c < n; ++c) {
      const double z = Q[(size_t)c * n + q], w = sqrt(dx[c + 1]);
      fwd[(size_t)m * n + c] = z * w;  // E^-1: row = mode, column = node
      inv[(size_t)c * n + m] = z / w;  // E: row = node, column = mode
    }
  }
  return true;
}

kv_status validate(const kv_grid_desc* d, std::string& msg) {
  if (!d) {
    msg = "desc is NULL";
    return KV_ERR_ARG;
  }
  if (d->nx < 2 || d->ny < 2 || d->nz < 2 || d->nx > 1024 || d->ny > 1024 || d->nz > 1024) {
    msg = "nx, ny, nz must be in [2, 1024]";
    return KV_ERR_ARG;
  }
  if (d->spanwise_bc != KV_BC_CC && d->spanwise_bc != KV_BC_AA) {
    msg = "spanwise_bc must be KV_BC_CC or KV_BC_AA";
    return KV_ERR_ARG;
  }
  if (d->tproj != KV_TPROJ_ORTHOGONAL && d->tproj != KV_TPROJ_OBLIQUE) {
    msg = "tproj must be KV_TPROJ_ORTHOGONAL or KV_TPROJ_OBLIQUE";
    return KV_ERR_ARG;
  }
  if (d->precision != KV_PREC_FP64 && d->precision != KV_PREC_MIXED) {
    msg = "precision must be KV_PREC_FP64 or KV_PREC_MIXED";
    return KV_ERR_ARG;
  }
  if (d->refine_sweeps < 0 || d->refine_sweeps > 20) {
    msg = "refine_sweeps must be in [0, 20]";
    return KV_ERR_ARG;
  }
  if (d->cgs_passes != 0 && d->cgs_passes != 2) {
    msg = "cgs_passes must be 0 or 2";
    return KV_ERR_ARG;
  }
  if (!(d->gr > 0) || !(d->pr > 0) || !isfinite(d->gr) || !isfinite(d->pr)) {
    msg = "gr and pr must be finite and > 0";
    return KV_ERR_ARG;
  }
  if (d->tol < 0 || d->max_passes < 0 || d->max_passes > 100) {
    msg = "tol must be >= 0 and max_passes in [0, 100]";
    return KV_ERR_ARG;
  }
  if (!(d->stretch >= 0.0 && d->stretch < 0.15915494309189533)) {
    msg = "stretch must be in [0, 1/(2 pi))";
    return KV_ERR_ARG;
  }
  if (d->advection != KV_ADV_CENTRAL && d->advection != KV_ADV_UPWIND) {
    msg = "advection must be KV_ADV_CENTRAL or KV_ADV_UPWIND";
    return KV_ERR_ARG;
  }
  if (d->advection == KV_ADV_UPWIND && d->stretch != 0.0) {
    msg = "upwind advection takes the uniform grid only (stretch must be 0)";
    return KV_ERR_ARG;
  }
  return KV_OK;
}

void free_all(kv_grid* h) {
  cudaFree(h->base);
  cudaFree(h->coef);
  cudaFree(h->coef_df);
  cudaFree(h->xsplit);
  cudaFree(h->vstar);
  cudaFree(h->tpd_a);
  cudaFree(h->tpd_b);
  for (int a = 0; a < 6; ++a) cudaFree(h->Wm[a]);
  for (int a = 0; a < 3; ++a) cudaFree(h->lam[a]);
  cudaFree(h->sw);
  cudaFree(h->swd);
  cudaFree(h->coef_dfp);
  kv_fx_free(h);
  cudaFree(h->guard);
  h->red = nullptr;
  cudaFree(h->partials);
  cudaFree(h->hdev);
  cudaFree(h->solve_buf);
  cudaFree(h->stage);
  cudaFree(h->pipe);
  for (auto& e : h->pev)
    if (e) cudaEventDestroy(e);
  if (h->cs_in) cudaStreamDestroy(h->cs_in);
  if (h->cs_out) cudaStreamDestroy(h->cs_out);
  cudaFree(h->tmp4);
  cudaFree(h->adj);
  cudaFree(h->adjsum);
  for (auto& ge : h->graphs) cudaGraphExecDestroy(ge.exec);
  h->graphs.clear();
  if (h->cap) cudaStreamDestroy(h->cap);
  kv_mixed_free(h);
}

template <typename T>
kv_status dalloc(kv_grid* h, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(h, KV_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return KV_OK;
}

double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
}

// The projection part of the Krylov map for a momentum right-hand side in h->vstar:
// b = D v*; phi = L^+ b (Eq 18); v = v* - G phi; p = phi; repeated while the SIMPLE test
// fails and passes remain. Writes the velocity part of y.
//
// Every pass evaluates the stopping test of Section 3.1 on the device: the correction kernel
// reduces max |D v| and max |v|, and a one-thread kernel forms max |D v| h_min / max |v| and
// records it in the grid's guard (kv_guard_read). One-pass evaluations (max_passes <= 1) stay
// asynchronous: the guard is read later. The host reads the pass's figures only when it needs
// them: for st, and in the literal loop (max_passes > 1), which decides on the host whether
// another pass runs.
kv_status simple_project(kv_grid* h, double* yvel, double* p, kv_stats* st) {
  cudaStream_t s = h->s;
  const int max_passes = h->d.max_passes > 0 ? h->d.max_passes : 1;
  const bool literal = max_passes > 1;
  const bool want = st != nullptr || literal;
  const bool mixed = h->d.precision == KV_PREC_MIXED;
  const double tol = kv_simple_tol(h);
  int pass = 0;
  double maxdiv = 0, rel = 0;
  bool finite = true;
  const double* src = h->vstar;
  double* phi = mixed ? h->tpd_b : h->tpd_a;
  for (pass = 1; pass <= max_passes; ++pass) {
    { KvPhase ph(h, KV_PH_DIV, 1); kv_launch_divergence(h, src, h->tpd_a, s); }
    if (mixed)
      kv_launch_poisson_mixed(h, h->tpd_a, phi, st != nullptr, 1, s);  // slices written by the divergence
    else
      kv_launch_poisson(h, h->tpd_a, h->tpd_a, s);
    {
      KvPhase ph(h, KV_PH_CORRECT, 2);
      kv_launch_correct(h, src, phi, yvel, p, pass > 1, s, 1);
      kv_launch_guard_close(h, tol, literal ? 0 : 1, s);
    }
    kv_status ks = check_launch(h, "SIMPLE pass");
    if (ks != KV_OK) return ks;
    if (!want) break;
    double last[3];
    KV_CHECK_CUDA(h, cudaMemcpyAsync(last, &h->guard->last_maxdiv, sizeof last, cudaMemcpyDeviceToHost, s));
    KV_CHECK_CUDA(h, cudaStreamSynchronize(s));
    maxdiv = last[0];
    rel = last[2];
    finite = std::isfinite(last[0]) && std::isfinite(last[1]) && std::isfinite(last[2]);
    if (!finite || rel < tol || pass == max_passes) break;
    // next pass: project the corrected field again (copy it back as the new v*)
    KV_CHECK_CUDA(h, cudaMemcpyAsync(h->vstar, yvel, 3 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
    src = h->vstar;
  }
  if (pass > max_passes) pass = max_passes;
  if (st) {
    st->passes = pass;
    st->max_div = maxdiv;
    st->rel_div = rel;
    st->refine_residual = 0;
    st->device_error = 0;
    if (mixed) {
      unsigned long long rm = 0;
      unsigned int de = 0;
      KV_CHECK_CUDA(h, cudaMemcpyAsync(&rm, h->rmax, sizeof rm, cudaMemcpyDeviceToHost, s));
      KV_CHECK_CUDA(h, cudaMemcpyAsync(&de, h->derr, sizeof de, cudaMemcpyDeviceToHost, s));
      KV_CHECK_CUDA(h, cudaStreamSynchronize(s));
      st->refine_residual = bits_to_double(rm);
      st->device_error = (int)de;
      if (de) return fail(h, KV_ERR_CUDA, "a bounded wait in a tensor-core kernel expired");
    }
  }
  if (want && !finite)
    return fail(h, KV_ERR_ARG,
                "non-finite velocity or divergence after the projection (NaN or Inf in x or in the base flow)");
  if (literal && !(rel < tol))
    return fail(h, KV_ERR_NOT_CONVERGED, "SIMPLE did not reach the tolerance in max_passes passes");
  return KV_OK;
}

// Autotuner for the linearised-operator kernels: times each candidate block shape (and, for the
// double-float kernel of the mixed path, each register budget) on this grid's coefficients (the
// base state stands in for x; v* and a scratch vector take the output) and keeps the fastest.
// Runs once per handle, at the first kv_set_base_flow.
kv_status autotune_apply(kv_grid* h) {
  static const int cand[][2] = {{32, 8}, {64, 4}, {128, 2}, {32, 4}, {16, 16}, {256, 1}};  // <= 256 threads
  if (!h->tmp4) {  // one padded field of scratch for the temperature output
    kv_status s = dalloc(h, &h->tmp4, 4 * h->P);
    if (s != KV_OK) return s;
  }
  cudaEvent_t e0, e1;
  KV_CHECK_CUDA(h, cudaEventCreate(&e0));
  KV_CHECK_CUDA(h, cudaEventCreate(&e1));
  // times one configuration: warm-up, then three launches; false if it cannot launch here
  auto time_it = [&](bool df, float& ms) -> bool {
    auto launch = [&]() {
      if (df)
        kv_launch_apply_df(h, h->coef_df, h->base, h->vstar, h->tmp4, h->s);
      else
        kv_launch_apply(h, h->coef, h->base, h->vstar, h->tmp4, h->s);
    };
    launch();
    if (cudaGetLastError() != cudaSuccess) return false;
    cudaEventRecord(e0, h->s);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(e1, h->s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return false;
    return cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  };
  float best = 1e30f, ms = 0;
  int bx = 32, by = 8;
  for (auto& c : cand) {
    h->apply_bx = c[0];
    h->apply_by = c[1];
    if (time_it(false, ms) && ms < best) {
      best = ms;
      bx = c[0];
      by = c[1];
    }
  }
  h->apply_bx = bx;
  h->apply_by = by;
  if (h->d.precision == KV_PREC_MIXED) {
    // the double-float operator: variant 0 (split pass, then cells per row x rows per block, four
    // equation rows each, <= 512 threads) or variant 1 (the 2.5D march, planes per block)
    static const int dcand[][3] = {{0, 32, 1}, {0, 32, 2}, {0, 64, 1}, {0, 32, 4}, {0, 64, 2}, {0, 128, 1},
                                   {1, 0, 16}, {1, 0, 32}, {1, 0, 64}, {2, 0, 8},  {2, 0, 16}, {2, 0, 32},
                                   {2, 0, 64}};
    best = 1e30f;
    int dv = 0, dbx = 32, dby = 2;
    for (auto& c : dcand) {
      if (c[0] == 1 && 4 * h->P >= (size_t(1) << 31)) continue;  // the march indexes x with 32 bits
      if (c[0] == 2 && !h->fx_ok) continue;                        // fixed point: uniform cubic grids
      h->df_variant = c[0];
      h->df_bx = c[1];
      h->df_by = c[2];
      if (time_it(true, ms) && ms < best) {
        best = ms;
        dv = c[0];
        dbx = c[1];
        dby = c[2];
      }
    }
    h->df_variant = dv;
    h->df_bx = dbx;
    h->df_by = dby;
    // the tensor-core contractions' tile width: one mixed Poisson solve (b = tpd_a, phi = tpd_b,
    // their contents are immaterial for the timing) with each; 128 columns only if at least 3 %
    // faster (where the two tie, as at 256^3, the wide tile does better in block evaluations)
    if (!h->tile_pinned) {
      best = 1e30f;
      int tile = 256;
      for (int t : {256, 128}) {
        if (t == 128) best *= 0.97f;
        h->umma_tile = t;
        auto solve = [&]() { kv_launch_poisson_mixed(h, h->tpd_a, h->tpd_b, 0, 0, h->s); };
        solve();
        if (cudaGetLastError() != cudaSuccess) continue;
        cudaEventRecord(e0, h->s);
        for (int r = 0; r < 3; ++r) solve();
        cudaEventRecord(e1, h->s);
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < best) {
          best = ms;
          tile = t;
        }
      }
      h->umma_tile = tile;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tuned = true;
  return check_launch(h, "autotune");
}

}  // namespace

void kv_set_thread_error(const std::string& msg) { g_create_error = msg; }

KvPhase::KvPhase(kv_grid* h_, int phase_, int launches) : h(h_), phase(phase_), n(launches) {
  nvtxRangePushA(kPhaseName[phase]);  // a no-op unless a profiler is attached
  if (!h->prof_on) return;
  if (h->ev_pool.empty()) {
    if (cudaEventCreate(&a) != cudaSuccess) a = nullptr;
  } else {
    a = h->ev_pool.back();
    h->ev_pool.pop_back();
  }
  if (a) cudaEventRecord(a, h->s);
}

KvPhase::~KvPhase() {
  nvtxRangePop();
  h->launches[phase] += n;
  if (!a) return;
  cudaEvent_t b = nullptr;
  if (h->ev_pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) b = nullptr;
  } else {
    b = h->ev_pool.back();
    h->ev_pool.pop_back();
  }
  if (!b) {
    h->ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, h->s);
  h->pending.push_back({phase, a, b});
}

extern "C" {

kv_status kv_create_grid(const kv_grid_desc* desc, void* stream, kv_handle* out) {
  if (!out) {
    g_create_error = "out is NULL";
    return KV_ERR_ARG;
  }
  *out = nullptr;
  std::string msg;
  kv_status st = validate(desc, msg);
  if (st != KV_OK) {
    g_create_error = msg;
    return st;
  }
  kv_grid* h = new (std::nothrow) kv_grid();
  if (!h) {
    g_create_error = "host allocation failed";
    return KV_ERR_NOMEM;
  }
  h->d = *desc;
  h->s = (cudaStream_t)stream;
  cudaGetDevice(&h->dev);
  KvGeom& g = h->g;
  g.nx = desc->nx;
  g.ny = desc->ny;
  g.nz = desc->nz;
  g.X = g.nx + 2;
  g.Y = g.ny + 2;
  g.Z = g.nz + 2;
  g.hx = 1.0 / g.nx;
  g.hy = 1.0 / g.ny;
  g.hz = 1.0 / g.nz;
  g.ihx = (double)g.nx;
  g.ihy = (double)g.ny;
  g.ihz = (double)g.nz;
  g.ihx2 = g.ihx * g.ihx;
  g.ihy2 = g.ihy * g.ihy;
  g.ihz2 = g.ihz * g.ihz;
  g.nu = 1.0 / sqrt(desc->gr);
  g.kappa = 1.0 / (desc->pr * sqrt(desc->gr));
  g.bc = desc->spanwise_bc;
  g.tproj = desc->tproj;
  g.adv = desc->advection;
  h->P = (size_t)g.X * g.Y * g.Z;
  h->Nc = (size_t)g.nx * g.ny * g.nz;

  const int n[3] = {g.nx, g.ny, g.nz};
  if ((st = dalloc(h, &h->base, 4 * h->P)) || (st = dalloc(h, &h->coef, (size_t)KV_NCOEF * h->P)) ||
      (st = dalloc(h, &h->vstar, 3 * h->P)) ||
      (st = dalloc(h, &h->tpd_a, h->Nc)) || (st = dalloc(h, &h->tpd_b, h->Nc)) || (st = dalloc(h, &h->guard, 1))) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return st;
  }
  cudaMemset(h->guard, 0, sizeof(KvGuardDev));
  h->red = reinterpret_cast<unsigned long long*>(h->guard);  // guard->red, its first member
  h->hmin = fmin(g.hx, fmin(g.hy, g.hz));
  const bool stretched = desc->stretch != 0.0;
  std::vector<double> fwdm[3], invm[3], tabs;
  if (stretched) h->hmin = 1.0;
  for (int a = 0; a < 3; ++a) {
    std::vector<double>& fwd = fwdm[a];
    std::vector<double>& inv = invm[a];
    std::vector<double> lam;
    if (stretched) {
      std::vector<double> tab;
      double hm = 1.0;
      if (!stretched_axis(n[a], desc->stretch, tab, fwd, inv, lam, hm)) {
        g_create_error = "kv_create_grid: the tridiagonal eigensolver did not converge";
        free_all(h);
        delete h;
        return KV_ERR_NOT_CONVERGED;
      }
      h->hmin = fmin(h->hmin, hm);
      h->str.swo[a] = (int)tabs.size();
      tabs.insert(tabs.end(), tab.begin(), tab.end());
    } else {
      neumann_axis(n[a], fwd, inv, lam);
    }
    if ((st = dalloc(h, &h->Wm[a], fwd.size())) || (st = dalloc(h, &h->Wm[3 + a], inv.size())) ||
        (st = dalloc(h, &h->lam[a], lam.size()))) {
      g_create_error = h->err;
      free_all(h);
      delete h;
      return st;
    }
    cudaMemcpy(h->Wm[a], fwd.data(), fwd.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(h->Wm[3 + a], inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(h->lam[a], lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (stretched) {
    if ((st = dalloc(h, &h->sw, tabs.size()))) {
      g_create_error = h->err;
      free_all(h);
      delete h;
      return st;
    }
    cudaMemcpy(h->sw, tabs.data(), tabs.size() * sizeof(double), cudaMemcpyHostToDevice);
    h->str.sw = h->sw;
    if (desc->precision == KV_PREC_MIXED) {
      // the double-float kernels' copy: inverse widths and the Neumann Laplacian's weights as
      // FP32 pairs (rounded once from FP64)
      auto pair = [](double x) {
        const float hi = (float)x;
        return make_float2(hi, (float)(x - (double)hi));
      };
      std::vector<float2> td;
      for (int a = 0; a < 3; ++a) {
        const int L = n[a] + 2;
        const double* tab = tabs.data() + h->str.swo[a];
        const double* idc = tab + (size_t)KV_SW_IDC * L;
        const double* idf = tab + (size_t)KV_SW_IDF * L;
        h->str.swdo[a] = (int)td.size();
        std::vector<float2> rows((size_t)KV_SWD_N * L, make_float2(0.0f, 0.0f));
        for (int t = 0; t < L; ++t) {
          rows[(size_t)KV_SWD_IDC * L + t] = pair(idc[t]);
          rows[(size_t)KV_SWD_IDF * L + t] = pair(idf[t]);
          if (t >= 2 && t <= n[a]) rows[(size_t)KV_SWD_LWM * L + t] = pair(idc[t] * idf[t - 1]);
          if (t >= 1 && t <= n[a] - 1) rows[(size_t)KV_SWD_LWP * L + t] = pair(idc[t] * idf[t]);
        }
        td.insert(td.end(), rows.begin(), rows.end());
      }
      if ((st = dalloc(h, &h->swd, td.size()))) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return st;
      }
      cudaMemcpy(h->swd, td.data(), td.size() * sizeof(float2), cudaMemcpyHostToDevice);
      h->str.swd = h->swd;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_create_error = std::string("kv_create_grid: ") + cudaGetErrorString(e);
    free_all(h);
    delete h;
    return KV_ERR_CUDA;
  }
  if (desc->precision == KV_PREC_MIXED) {
    const double* f3[3] = {fwdm[0].data(), fwdm[1].data(), fwdm[2].data()};
    const double* i3[3] = {invm[0].data(), invm[1].data(), invm[2].data()};
    st = kv_mixed_setup(h, f3, i3);
    if (st != KV_OK) {
      g_create_error = h->err;
      free_all(h);
      delete h;
      return st;
    }
  }
  *out = h;
  return KV_OK;
}

kv_status kv_destroy_grid(kv_handle h) {
  if (!h) return KV_OK;
  cudaStreamSynchronize(h->s);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  free_all(h);
  delete h;
  return KV_OK;
}

kv_status kv_set_stream(kv_handle h, void* stream) {
  if (!h) return KV_ERR_ARG;
  h->s = (cudaStream_t)stream;
  return KV_OK;
}

kv_status kv_field_len(kv_handle h, size_t* field_len) {
  if (!h || !field_len) return fail(h, KV_ERR_ARG, "kv_field_len: NULL argument");
  *field_len = h->P;
  return KV_OK;
}

kv_status kv_field_sizes(kv_handle h, size_t* u, size_t* v, size_t* w, size_t* cell) {
  if (!h) return KV_ERR_ARG;
  if (!u && !v && !w && !cell) return fail(h, KV_ERR_ARG, "kv_field_sizes: every output is NULL");
  // one padded layout serves all four fields (the face fields keep their unused index n+1)
  if (u) *u = h->P;
  if (v) *v = h->P;
  if (w) *w = h->P;
  if (cell) *cell = h->P;
  return KV_OK;
}

// The base state is in h->base: assemble the coefficients of J for it (and their FP32 pairs).
static kv_status base_flow_ready(kv_grid* h) {
  kv_launch_assemble(h, h->base, h->coef, h->s);
  if (h->d.precision == KV_PREC_MIXED) {
    if (!h->coef_df) {
      kv_status s = dalloc(h, &h->coef_df, (size_t)KV_NCOEF_DF * h->P);
      if (s != KV_OK) return s;
    }
    if (!h->xsplit) {
      kv_status s = dalloc(h, &h->xsplit, 4 * h->P);
      if (s != KV_OK) return s;
    }
    if ((h->str.sw || h->g.adv) && !h->coef_dfp) {
      kv_status s = dalloc(h, &h->coef_dfp, (size_t)KV_NCOEF_DFP * h->P);
      if (s != KV_OK) return s;
    }
    kv_launch_coef_df(h, h->coef, h->coef_df, h->s);
    kv_status fs = kv_fx_setup(h);
    if (fs != KV_OK) return fail(h, fs, "kv_set_base_flow: the fixed-point operator's set-up failed");
  }
  kv_status ks = check_launch(h, "assemble");
  if (ks != KV_OK) return ks;
  h->has_base = true;
  if (!h->tuned) return autotune_apply(h);
  return KV_OK;
}

kv_status kv_set_base_flow(kv_handle h, const double* U, const double* V, const double* W, const double* Theta) {
  if (!h) return KV_ERR_ARG;
  if (!U || !V || !W || !Theta) return fail(h, KV_ERR_ARG, "kv_set_base_flow: NULL field");
  const double* f[4] = {U, V, W, Theta};
  for (int q = 0; q < 4; ++q)
    KV_CHECK_CUDA(h, cudaMemcpyAsync(h->base + (size_t)q * h->P, f[q], h->P * sizeof(double),
                                     cudaMemcpyDeviceToDevice, h->s));
  return base_flow_ready(h);
}

kv_status kv_set_base_flow_packed(kv_handle h, const double* base) {
  if (!h) return KV_ERR_ARG;
  if (!base) return fail(h, KV_ERR_ARG, "kv_set_base_flow_packed: base is NULL");
  KV_CHECK_CUDA(h, cudaMemcpyAsync(h->base, base, 4 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
  return base_flow_ready(h);
}

kv_status kv_set_tuning(kv_handle h, const int* cfg) {
  if (!h) return KV_ERR_ARG;
  if (!cfg) return fail(h, KV_ERR_ARG, "kv_set_tuning: cfg is NULL");
  const bool mixed = h->d.precision == KV_PREC_MIXED;
  const int bx = cfg[0], by = cfg[1];
  if (bx < 1 || by < 1 || bx * by > 256 || (bx * by) % 32 != 0)
    return fail(h, KV_ERR_ARG, "kv_set_tuning: the FP64 operator block needs bx, by >= 1, bx * by <= 256 and a "
                               "multiple of 32");
  int dv = -1, dbx = -1, dby = -1;
  if (mixed) {
    dv = cfg[2];
    dbx = cfg[3];
    dby = cfg[4];
    if (dv == 0) {
      if ((dbx != 32 && dbx != 64 && dbx != 128) || dby < 1 || dbx * 4 * dby > 512)
        return fail(h, KV_ERR_ARG, "kv_set_tuning: the split-pass operator needs cells per row 32, 64 or 128 and "
                                   "cells x 4 x rows <= 512");
    } else if (dv == 1) {
      if (dby < 1 || dby > 1024)
        return fail(h, KV_ERR_ARG, "kv_set_tuning: the march needs 1..1024 planes per block");
      if (4 * h->P >= (size_t(1) << 31))
        return fail(h, KV_ERR_ARG, "kv_set_tuning: the march indexes a packed vector with 32 bits; this grid is too "
                                   "large for it");
      dbx = 0;
    } else if (dv == 2) {
      if (dby < 1 || dby > 1024)
        return fail(h, KV_ERR_ARG, "kv_set_tuning: the fixed-point march needs 1..1024 planes per block");
      if (!kv_fx_eligible(h))
        return fail(h, KV_ERR_ARG, "kv_set_tuning: the fixed-point operator serves uniform cubic mixed-precision "
                                   "grids whose packed vectors fit 32-bit offsets");
      dbx = 0;
    } else {
      return fail(h, KV_ERR_ARG, "kv_set_tuning: cfg[2] (the mixed operator variant) must be 0, 1 or 2");
    }
  }
  h->apply_bx = bx;
  h->apply_by = by;
  if (mixed) {
    h->df_variant = dv;
    h->df_bx = dbx;
    h->df_by = dby;
  }
  h->tuned = true;
  h->pinned = true;
  for (auto& ge : h->graphs) cudaGraphExecDestroy(ge.exec);
  h->graphs.clear();
  return KV_OK;
}

// Captured graphs hold the kernels and launch shapes of the configuration they were captured
// with: a new configuration drops them (the next batch call captures again).
static void drop_graphs(kv_grid* h) {
  for (auto& ge : h->graphs) cudaGraphExecDestroy(ge.exec);
  h->graphs.clear();
}

kv_status kv_set_contraction_tile(kv_handle h, int columns) {
  if (!h) return KV_ERR_ARG;
  if (h->d.precision != KV_PREC_MIXED)
    return fail(h, KV_ERR_ARG, "kv_set_contraction_tile: only the mixed path contracts on the tensor cores");
  if (columns != 128 && columns != 256)
    return fail(h, KV_ERR_ARG, "kv_set_contraction_tile: the tile width must be 128 or 256 columns");
  h->umma_tile = columns;
  h->tile_pinned = true;
  drop_graphs(h);
  return KV_OK;
}

kv_status kv_contraction_tile(kv_handle h, int* columns) {
  if (!h) return KV_ERR_ARG;
  if (!columns) return fail(h, KV_ERR_ARG, "kv_contraction_tile: columns is NULL");
  *columns = h->d.precision == KV_PREC_MIXED ? h->umma_tile : -1;
  return KV_OK;
}

kv_status kv_guard_read(kv_handle h, kv_guard* out, int reset) {
  if (!h) return KV_ERR_ARG;
  if (!out) return fail(h, KV_ERR_ARG, "kv_guard_read: out is NULL");
  KvGuardDev gd;
  KV_CHECK_CUDA(h, cudaMemcpyAsync(&gd, h->guard, sizeof gd, cudaMemcpyDeviceToHost, h->s));
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
  out->checks = (long long)gd.checks;
  out->failed = (long long)gd.failed;
  out->nonfinite = (long long)gd.nonfinite;
  out->worst_rel_div = gd.worst_rel;
  if (reset) {
    // the counters and figures; red belongs to a pass in progress and is cleared by its close
    KV_CHECK_CUDA(h, cudaMemsetAsync(&h->guard->checks, 0, sizeof(KvGuardDev) - offsetof(KvGuardDev, checks), h->s));
    KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
  }
  return KV_OK;
}

kv_status kv_krylov_vector(kv_handle h, const double* x, double* y, double* p, kv_stats* st) {
  if (!h) return KV_ERR_ARG;
  if (!x || !y) return fail(h, KV_ERR_ARG, "kv_krylov_vector: x and y must be non-NULL");
  if (!h->has_base) return fail(h, KV_ERR_STATE, "kv_krylov_vector: no base flow set");
  const size_t L = 4 * h->P;
  if ((x < y + L && y < x + L)) return fail(h, KV_ERR_ARG, "kv_krylov_vector: x and y overlap");
  // J P_BC x: momentum right-hand side to vstar, projected temperature straight into y
  {
    KvPhase ph(h, KV_PH_STENCIL, h->d.precision == KV_PREC_MIXED ? 2 : 1);  // split + operator
    if (h->d.precision == KV_PREC_MIXED)
      kv_launch_apply_df(h, h->coef_df, x, h->vstar, y + 3 * h->P, h->s);
    else
      kv_launch_apply(h, h->coef, x, h->vstar, y + 3 * h->P, h->s);
  }
  kv_status ks = check_launch(h, "stencil");
  if (ks != KV_OK) return ks;
  return simple_project(h, y, p, st);
}

kv_status kv_krylov_vector_host(kv_handle h, const double* x_host, double* y_host, kv_stats* st) {
  if (!h) return KV_ERR_ARG;
  if (!x_host || !y_host) return fail(h, KV_ERR_ARG, "kv_krylov_vector_host: NULL argument");
  const size_t L = 4 * h->P;
  if (!h->stage) {
    kv_status s = dalloc(h, &h->stage, 2 * L);
    if (s != KV_OK) return s;
  }
  KV_CHECK_CUDA(h, cudaMemcpyAsync(h->stage, x_host, L * sizeof(double), cudaMemcpyHostToDevice, h->s));
  kv_status s = kv_krylov_vector(h, h->stage, h->stage + L, nullptr, st);
  if (s != KV_OK) return s;
  KV_CHECK_CUDA(h, cudaMemcpyAsync(y_host, h->stage + L, L * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
  return KV_OK;
}

kv_status kv_krylov_vector_host_stream(kv_handle h, const double* X_host, double* Y_host, int nb) {
  if (!h) return KV_ERR_ARG;
  if (nb == 0) return KV_OK;
  if (!X_host || !Y_host || nb < 0) return fail(h, KV_ERR_ARG, "kv_krylov_vector_host_stream: bad argument");
  if (!h->has_base) return fail(h, KV_ERR_STATE, "kv_krylov_vector_host_stream: no base flow set");
  const size_t L = 4 * h->P;
  if (!h->pipe) {
    kv_status s = dalloc(h, &h->pipe, 4 * L);
    if (s != KV_OK) return s;
  }
  if (!h->cs_in) {
    KV_CHECK_CUDA(h, cudaStreamCreateWithFlags(&h->cs_in, cudaStreamNonBlocking));
    KV_CHECK_CUDA(h, cudaStreamCreateWithFlags(&h->cs_out, cudaStreamNonBlocking));
    for (auto& e : h->pev) KV_CHECK_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaEvent_t* loaded = h->pev;
  cudaEvent_t* computed = h->pev + 2;
  cudaEvent_t* drained = h->pev + 4;
  // vector i: copied in on cs_in into x slot i % 2 (free once vector i - 2 is computed), computed
  // on the handle's stream into y slot i % 2 (free once vector i - 2 is copied out), copied out on
  // cs_out. The copy-in of i + 1 is queued before the evaluation of i, so it and the copy-out of
  // i - 1 overlap that evaluation.
  auto load = [&](int i) -> kv_status {
    const int b = i & 1;
    if (i >= 2) KV_CHECK_CUDA(h, cudaStreamWaitEvent(h->cs_in, computed[b], 0));
    KV_CHECK_CUDA(h, cudaMemcpyAsync(h->pipe + (size_t)b * L, X_host + (size_t)i * L, L * sizeof(double),
                                     cudaMemcpyHostToDevice, h->cs_in));
    KV_CHECK_CUDA(h, cudaEventRecord(loaded[b], h->cs_in));
    return KV_OK;
  };
  kv_status s = load(0);
  for (int i = 0; i < nb && s == KV_OK; ++i) {
    const int b = i & 1;
    double* xb = h->pipe + (size_t)b * L;
    double* yb = h->pipe + (size_t)(2 + b) * L;
    if (i + 1 < nb && (s = load(i + 1)) != KV_OK) break;
    KV_CHECK_CUDA(h, cudaStreamWaitEvent(h->s, loaded[b], 0));
    if (i >= 2) KV_CHECK_CUDA(h, cudaStreamWaitEvent(h->s, drained[b], 0));
    if ((s = kv_krylov_vector(h, xb, yb, nullptr, nullptr)) != KV_OK) break;
    KV_CHECK_CUDA(h, cudaEventRecord(computed[b], h->s));
    KV_CHECK_CUDA(h, cudaStreamWaitEvent(h->cs_out, computed[b], 0));
    KV_CHECK_CUDA(h, cudaMemcpyAsync(Y_host + (size_t)i * L, yb, L * sizeof(double), cudaMemcpyDeviceToHost,
                                     h->cs_out));
    KV_CHECK_CUDA(h, cudaEventRecord(drained[b], h->cs_out));
  }
  if (s != KV_OK) {
    cudaStreamSynchronize(h->cs_in);
    cudaStreamSynchronize(h->cs_out);
    return s;
  }
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->cs_out));
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->cs_in));
  return KV_OK;
}

kv_status kv_arnoldi_step(kv_handle h, double* V, int j, double* h_col) {
  if (!h) return KV_ERR_ARG;
  if (!V || !h_col || j < 0 || j > 4095) return fail(h, KV_ERR_ARG, "kv_arnoldi_step: bad argument");
  const size_t L = 4 * h->P;
  const int nq = j + 1;
  const size_t need_p = (size_t)(nq + 1) * kv_reduce_blocks();
  if (h->partials_cap < need_p) {
    cudaFree(h->partials);
    h->partials = nullptr;
    h->partials_cap = 0;
    kv_status s = dalloc(h, &h->partials, need_p);
    if (s != KV_OK) return s;
    h->partials_cap = need_p;
  }
  const size_t need_h = 3 * (size_t)nq + 6;
  if (h->hdev_cap < need_h) {
    cudaFree(h->hdev);
    h->hdev = nullptr;
    h->hdev_cap = 0;
    kv_status s = dalloc(h, &h->hdev, need_h);
    if (s != KV_OK) return s;
    h->hdev_cap = need_h;
  }
  double* w = V + (size_t)(j + 1) * L;
  kv_status s = kv_krylov_vector(h, V + (size_t)j * L, w, nullptr, nullptr);
  if (s != KV_OK) return s;
  double* h1 = h->hdev;               // [0, nq): first pass; [nq]: ||w||^2 before
  double* h2 = h->hdev + nq + 1;      // [nq+1, 2nq+1): second pass; [2nq+1]: ||w||^2 after pass 1
  double* hcol = h->hdev + 2 * nq + 3;  // [2nq+3, 3nq+4): the Hessenberg column (fused path)
  int* flag = reinterpret_cast<int*>(h->hdev + 3 * nq + 4);  // second update applied (fused path)
  std::vector<double> hh(need_h, 0.0);
  if (nq <= kv_fused_cgs_max()) {
    // mixed precision: sweeps 1 and 2 in double-float on the FP32 pipe
    const int df = h->d.precision == KV_PREC_MIXED;
    // Classical Gram-Schmidt. Sweep 1: h1 = V^T w and ||w||^2. Sweep 2: w -= V h1 fused with the
    // second pass's h2 = V^T w and ||w||^2, i.e. the components along V that remain after the
    // first update, measured. Sweep 3 (w -= V h2) is applied when they exceed the rounding level
    // of the sweep arithmetic relative to ||w|| (2^-46 for the double-float sweeps, 2^-50 in
    // FP64); below it the second update cannot improve the orthogonality. (ARPACK's DGKS test
    // decides from ||w|| alone because it has not computed h2; here sweep 2 has.) The decision
    // and the Hessenberg column are formed on the device, so the step synchronises once, at its
    // end, to return the column.
    {
      KvPhase ph(h, KV_PH_GS_DOTS, 2);
      kv_launch_dots_norm(V, L, nq, w, L, h->partials, h1, h1 + nq, df, h->s);
    }
    {
      KvPhase ph(h, KV_PH_GS_UPDATE, 2);
      kv_launch_update_dot(V, L, nq, h1, w, L, h->partials, h2, df, h->s);
    }
    {
      KvPhase ph(h, KV_PH_ARNOLDI, 2);
      kv_launch_gs_decide(h1, h2, nq, df ? 0x1p-46 : 0x1p-50, h->d.cgs_passes == 2, hcol, flag, h->s);
      kv_launch_update_small_scale(V, L, nq, h2, w, L, h->s, flag);
    }
    s = check_launch(h, "arnoldi");
    if (s != KV_OK) return s;
    KV_CHECK_CUDA(h, cudaMemcpyAsync(hh.data(), h->hdev, need_h * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
    if (df && std::isnan(hh[nq]))
      return fail(h, KV_ERR_ARG,
                  "kv_arnoldi_step: the new vector has entries outside the mixed-precision Gram-Schmidt range "
                  "(NaN, Inf or |x| >= 2^48); V[j+1] is undefined");
    int upd = 0;
    memcpy(&upd, &hh[3 * (size_t)nq + 4], sizeof upd);
    h->gs_steps += 1;
    h->gs_second += upd != 0;
    for (int q = 0; q <= nq; ++q) h_col[q] = hh[2 * (size_t)nq + 3 + q];
    return KV_OK;
  }
  // Beyond QF basis vectors: the same classical Gram-Schmidt with its measured second pass, as
  // separate sweeps: h1 = V^T w and ||w||^2 (chunks of QF vectors), w -= V h1 (one sweep over all
  // vectors; in mixed precision on both pipes), h2 = V^T w and ||w||^2 (chunks), then the device-side
  // decision and the third sweep fused with the normalisation.
  const int df = h->d.precision == KV_PREC_MIXED;
  {
    const int chunks = (nq + kv_fused_cgs_max() - 1) / kv_fused_cgs_max();
    KvPhase ph(h, KV_PH_GS_DOTS, 2 * chunks);
    kv_launch_dots_chunked(V, L, nq, w, L, h->partials, h1, 1, df, h->s);
  }
  {
    KvPhase ph(h, KV_PH_GS_UPDATE, 1);
    kv_launch_update_n(V, L, nq, h1, w, L, df, h->s);
  }
  {
    const int chunks = (nq + kv_fused_cgs_max() - 1) / kv_fused_cgs_max();
    KvPhase ph(h, KV_PH_GS_DOTS, 2 * chunks);
    kv_launch_dots_chunked(V, L, nq, w, L, h->partials, h2, 1, df, h->s);
  }
  {
    KvPhase ph(h, KV_PH_ARNOLDI, 2);
    kv_launch_gs_decide(h1, h2, nq, df ? 0x1p-46 : 0x1p-50, h->d.cgs_passes == 2, hcol, flag, h->s);
    kv_launch_update_small_scale_n(V, L, nq, h2, w, L, h->s, flag);
  }
  s = check_launch(h, "arnoldi");
  if (s != KV_OK) return s;
  KV_CHECK_CUDA(h, cudaMemcpyAsync(hh.data(), h->hdev, need_h * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
  if (df && (std::isnan(hh[nq]) || std::isnan(hh[2 * (size_t)nq + 1])))
    return fail(h, KV_ERR_ARG,
                "kv_arnoldi_step: the new vector has entries outside the mixed-precision Gram-Schmidt range "
                "(NaN, Inf or |x| >= 2^48); V[j+1] is undefined");
  int upd = 0;
  memcpy(&upd, &hh[3 * (size_t)nq + 4], sizeof upd);
  h->gs_steps += 1;
  h->gs_second += upd != 0;
  for (int q = 0; q <= nq; ++q) h_col[q] = hh[2 * (size_t)nq + 3 + q];
  return KV_OK;
}

kv_status kv_arnoldi_run(kv_handle h, double* V, int j0, int m, double* H, int ldh) {
  if (!h) return KV_ERR_ARG;
  if (!V || !H || j0 < 0 || m < 1 || j0 + m > 4096 || ldh < j0 + m + 1)
    return fail(h, KV_ERR_ARG, "kv_arnoldi_run: bad argument (j0 >= 0, m >= 1, j0 + m <= 4096, ldh >= j0 + m + 1)");
  const size_t L = 4 * h->P;
  const int J = j0 + m, ldd = J + 1;
  const int QC = kv_dcgs_chunk(), DSs = kv_dcgs_dots_stride();
  const int nch = (J + QC - 1) / QC;
  const size_t need_p = (size_t)(2 * QC + 3) * kv_reduce_blocks();
  if (h->partials_cap < need_p) {
    cudaFree(h->partials);
    h->partials = nullptr;
    h->partials_cap = 0;
    kv_status s = dalloc(h, &h->partials, need_p);
    if (s != KV_OK) return s;
    h->partials_cap = need_p;
  }
  // device scratch: the inner products (a block per chunk), the Hessenberg matrix (ldd x J,
  // column-major), the update's scalars (3) and the constant (1, 1, 0) of later chunks, its two
  // coefficient vectors (J each), the coefficient kernel's scratch (2 (J + 1)), an error flag
  const size_t n_dots = (size_t)DSs * (nch > 0 ? nch : 1), n_h = (size_t)ldd * J;
  const size_t need_h = n_dots + n_h + 6 + 2 * (size_t)J + 2 * (size_t)(J + 1) + 1;
  if (h->hdev_cap < need_h) {
    cudaFree(h->hdev);
    h->hdev = nullptr;
    h->hdev_cap = 0;
    kv_status s = dalloc(h, &h->hdev, need_h);
    if (s != KV_OK) return s;
    h->hdev_cap = need_h;
  }
  double* dots = h->hdev;
  double* Hd = dots + n_dots;
  double* s3 = Hd + n_h;
  double* one3 = s3 + 3;
  double* cuv = one3 + 3;
  double* cwv = cuv + J;
  double* scr = cwv + J;
  int* err = reinterpret_cast<int*>(scr + 2 * (size_t)(J + 1));
  // the columns of H before the run (those of the existing basis) go to the device; the
  // corrections of the deferred projections use them
  std::vector<double> hd(n_h + 6, 0.0);
  for (int c = 0; c < j0; ++c)
    for (int r = 0; r <= c + 1; ++r) hd[r + (size_t)ldd * c] = H[r + (size_t)ldh * c];
  hd[n_h + 3] = 1.0;
  hd[n_h + 4] = 1.0;
  KV_CHECK_CUDA(h, cudaMemcpyAsync(Hd, hd.data(), (n_h + 6) * sizeof(double), cudaMemcpyHostToDevice, h->s));
  KV_CHECK_CUDA(h, cudaMemsetAsync(err, 0, sizeof(int), h->s));
  const int df = h->d.precision == KV_PREC_MIXED;
  for (int j = j0; j < J; ++j) {
    double* u = V + (size_t)j * L;
    double* w = V + (size_t)(j + 1) * L;
    kv_status s = kv_krylov_vector(h, u, w, nullptr, nullptr);  // w = A u_j (u_j provisional)
    if (s != KV_OK) return s;
    const int nc = j > 0 ? (j + QC - 1) / QC : 1;
    {
      KvPhase ph(h, KV_PH_GS_DOTS, 2 * nc);
      kv_launch_dots2(V, L, j, u, w, L, h->partials, dots, df, h->s);
    }
    {
      KvPhase ph(h, KV_PH_ARNOLDI, 1);
      kv_launch_dcgs_coef(dots, Hd, ldd, j, j == j0, 0, s3, cuv, cwv, scr, err, h->s);
    }
    {
      KvPhase ph(h, KV_PH_GS_UPDATE, nc);
      kv_launch_update2(V, L, j, s3, one3, cuv, cwv, u, w, L, j != j0, 1, df, h->s);
    }
  }
  {
    // the last vector's deferred second projection and its normalisation
    const int nc = (J + QC - 1) / QC;
    KvPhase ph(h, KV_PH_ARNOLDI, 3 * nc + 1);
    double* u = V + (size_t)J * L;
    kv_launch_dots2(V, L, J, u, u, L, h->partials, dots, df, h->s);
    kv_launch_dcgs_coef(dots, Hd, ldd, J, 0, 1, s3, cuv, cwv, scr, err, h->s);
    kv_launch_update2(V, L, J, s3, one3, cuv, cwv, u, nullptr, L, 1, 0, df, h->s);
  }
  kv_status s = check_launch(h, "arnoldi run");
  if (s != KV_OK) return s;
  int herr = 0;
  KV_CHECK_CUDA(h, cudaMemcpyAsync(hd.data(), Hd, n_h * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  KV_CHECK_CUDA(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
  if (herr)
    return fail(h, KV_ERR_ARG,
                "kv_arnoldi_run: a vector of the run has entries outside the Gram-Schmidt sweeps' range or "
                "lies in the span of the basis; V and H are undefined");
  for (int c = j0; c < J; ++c)
    for (int r = 0; r <= c + 1; ++r) H[r + (size_t)ldh * c] = hd[r + (size_t)ldd * c];
  h->gs_steps += m;
  h->gs_second += m;
  return KV_OK;
}

kv_status kv_newton_residual(kv_handle h, const double* S, double* F, double* norm_out) {
  if (!h) return KV_ERR_ARG;
  if (!S) return fail(h, KV_ERR_ARG, "kv_newton_residual: S is NULL");
  const size_t L = 4 * h->P;
  double* out = F;
  if (!out) {
    if (!h->tmp4) {
      kv_status s = dalloc(h, &h->tmp4, L);
      if (s != KV_OK) return s;
    }
    out = h->tmp4;
  }
  if (S < out + L && out < S + L) return fail(h, KV_ERR_ARG, "kv_newton_residual: S and F overlap");
  { KvPhase ph(h, KV_PH_STENCIL, 1); kv_launch_stencil(h, 1, S, S, h->vstar, out + 3 * h->P, h->s); }
  kv_status s = check_launch(h, "residual stencil");
  if (s != KV_OK) return s;
  s = simple_project(h, out, nullptr, nullptr);
  if (s != KV_OK) return s;
  if (norm_out) {
    const size_t need_p = 2 * (size_t)kv_reduce_blocks();
    if (h->partials_cap < need_p) {
      cudaFree(h->partials);
      h->partials = nullptr;
      h->partials_cap = 0;
      s = dalloc(h, &h->partials, need_p);
      if (s != KV_OK) return s;
      h->partials_cap = need_p;
    }
    if (h->hdev_cap < 1) {
      s = dalloc(h, &h->hdev, 3);
      if (s != KV_OK) return s;
      h->hdev_cap = 3;
    }
    { KvPhase ph(h, KV_PH_ARNOLDI, 2); kv_launch_norm2(out, L, h->partials, h->hdev, h->s); }
    s = check_launch(h, "residual norm");
    if (s != KV_OK) return s;
    double n2 = 0;
    KV_CHECK_CUDA(h, cudaMemcpyAsync(&n2, h->hdev, sizeof n2, cudaMemcpyDeviceToHost, h->s));
    KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
    *norm_out = sqrt(n2);
  }
  return KV_OK;
}

// (Pi_v (+) P_T) y into h->adj: the output-side projections of the Krylov map, which are
// symmetric (orthogonal reading), applied to y.
static kv_status project_output_side(kv_grid* h, const double* y) {
  if (!h->adj) {
    kv_status s = dalloc(h, &h->adj, 4 * h->P);
    if (s != KV_OK) return s;
  }
  kv_launch_adj_prep(h, y, h->vstar, h->adj + 3 * h->P, h->s);
  kv_status s = check_launch(h, "adjoint prep");
  if (s != KV_OK) return s;
  return simple_project(h, h->adj, nullptr, nullptr);
}

kv_status kv_krylov_vector_adjoint(kv_handle h, const double* y, double* z) {
  if (!h) return KV_ERR_ARG;
  if (!y || !z) return fail(h, KV_ERR_ARG, "kv_krylov_vector_adjoint: y and z must be non-NULL");
  if (!h->has_base) return fail(h, KV_ERR_STATE, "kv_krylov_vector_adjoint: no base flow set");
  if (h->d.tproj != KV_TPROJ_ORTHOGONAL)
    return fail(h, KV_ERR_ARG, "kv_krylov_vector_adjoint: defined for the orthogonal temperature projection");
  if (h->str.sw)
    return fail(h, KV_ERR_ARG,
                "kv_krylov_vector_adjoint: defined on the uniform grid (the velocity projection of a stretched "
                "grid is not symmetric)");
  const size_t L = 4 * h->P;
  if (y < z + L && z < y + L) return fail(h, KV_ERR_ARG, "kv_krylov_vector_adjoint: y and z overlap");
  kv_status s = project_output_side(h, y);
  if (s != KV_OK) return s;
  { KvPhase ph(h, KV_PH_STENCIL, 1); kv_launch_apply_t(h, h->coef, h->adj, z, h->s); }
  return check_launch(h, "transpose stencil");
}

kv_status kv_base_flow_gradient(kv_handle h, const double* x, const double* y, double* g_base, double* dgr) {
  if (!h) return KV_ERR_ARG;
  if (!x || !y) return fail(h, KV_ERR_ARG, "kv_base_flow_gradient: x and y must be non-NULL");
  if (!h->has_base) return fail(h, KV_ERR_STATE, "kv_base_flow_gradient: no base flow set");
  if (h->d.tproj != KV_TPROJ_ORTHOGONAL)
    return fail(h, KV_ERR_ARG, "kv_base_flow_gradient: defined for the orthogonal temperature projection");
  if (h->str.sw)
    return fail(h, KV_ERR_ARG,
                "kv_base_flow_gradient: defined on the uniform grid (the velocity projection of a stretched "
                "grid is not symmetric)");
  if (h->g.adv)
    return fail(h, KV_ERR_ARG,
                "kv_base_flow_gradient: defined for central advection (with upwinding the operator is not "
                "affine in the base flow)");
  kv_status s = project_output_side(h, y);
  if (s != KV_OK) return s;
  if (g_base) {
    kv_launch_grad_vel(h, x, h->adj, g_base, h->s);
    kv_launch_grad_theta(h, x, h->adj + 3 * h->P, g_base + 3 * h->P, h->s);
  }
  if (dgr) {
    if (!h->adjsum) {
      s = dalloc(h, &h->adjsum, 2);
      if (s != KV_OK) return s;
    }
    KV_CHECK_CUDA(h, cudaMemsetAsync(h->adjsum, 0, 2 * sizeof(double), h->s));
    kv_launch_lap_dot(h, x, h->adj, h->adjsum, h->s);
    s = check_launch(h, "Grashof derivative");
    if (s != KV_OK) return s;
    double sums[2];
    KV_CHECK_CUDA(h, cudaMemcpyAsync(sums, h->adjsum, sizeof sums, cudaMemcpyDeviceToHost, h->s));
    KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
    const double d = -0.5 * pow(h->d.gr, -1.5);
    *dgr = d * sums[0] + d / h->d.pr * sums[1];
  }
  return check_launch(h, "base-flow gradient");
}

kv_status kv_profile_enable(kv_handle h, int on) {
  if (!h) return KV_ERR_ARG;
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
  for (auto& p : h->pending) {
    h->ev_pool.push_back(p.a);
    h->ev_pool.push_back(p.b);
  }
  h->pending.clear();
  for (int q = 0; q < KV_NPHASE; ++q) {
    h->prof_ms[q] = 0;
    h->prof_n[q] = 0;
    h->launches[q] = 0;
  }
  h->gs_steps = 0;
  h->gs_second = 0;
  h->prof_on = on != 0;
  return KV_OK;
}

kv_status kv_arnoldi_counts(kv_handle h, long long* steps, long long* second_updates) {
  if (!h) return KV_ERR_ARG;
  if (steps) *steps = h->gs_steps;
  if (second_updates) *second_updates = h->gs_second;
  return KV_OK;
}

kv_status kv_tuning(kv_handle h, int* cfg) {
  if (!h) return KV_ERR_ARG;
  if (!cfg) return fail(h, KV_ERR_ARG, "kv_tuning: cfg is NULL");
  if (!h->tuned) return fail(h, KV_ERR_STATE, "kv_tuning: no base flow set yet");
  const bool mixed = h->d.precision == KV_PREC_MIXED;
  cfg[0] = h->apply_bx;
  cfg[1] = h->apply_by;
  cfg[2] = mixed ? h->df_variant : -1;
  cfg[3] = mixed ? h->df_bx : -1;
  cfg[4] = mixed ? h->df_by : -1;
  return KV_OK;
}

kv_status kv_profile_get(kv_handle h, int phase, double* total_ms, long long* timed_launches, long long* launches) {
  if (!h) return KV_ERR_ARG;
  if (phase < 0 || phase >= KV_NPHASE) return fail(h, KV_ERR_ARG, "kv_profile_get: bad phase");
  KV_CHECK_CUDA(h, cudaStreamSynchronize(h->s));
  for (auto& p : h->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->prof_ms[p.phase] += ms;
      h->prof_n[p.phase] += 1;
    }
    h->ev_pool.push_back(p.a);
    h->ev_pool.push_back(p.b);
  }
  h->pending.clear();
  if (total_ms) *total_ms = h->prof_ms[phase];
  if (timed_launches) *timed_launches = h->prof_n[phase];
  if (launches) *launches = h->launches[phase];
  return KV_OK;
}

kv_status kv_selftest_wait_timeout(kv_handle h, int* device_error) {
  if (!h || !device_error) return KV_ERR_ARG;
  if (h->d.precision != KV_PREC_MIXED) return fail(h, KV_ERR_ARG, "kv_selftest_wait_timeout: needs a mixed grid");
  return kv_mixed_selftest_timeout(h, device_error);
}

kv_status kv_axis_data(int n, double stretch, double* E, double* E_inv, double* lambda, double* weights) {
  if (n < 2 || n > 1024 || !(stretch >= 0.0 && stretch < 0.15915494309189533)) {
    g_create_error = "kv_axis_data: n must be in [2, 1024] and stretch in [0, 1/(2 pi))";
    return KV_ERR_ARG;
  }
  std::vector<double> fwd, inv, lam, tab;
  double hm = 0.0;
  // the tables by the stretched formulas (at stretch = 0 they are the uniform grid's weights)
  if (!stretched_axis(n, stretch, tab, fwd, inv, lam, hm, stretch != 0.0)) {
    g_create_error = "kv_axis_data: the tridiagonal eigensolver did not converge";
    return KV_ERR_NOT_CONVERGED;
  }
  if (stretch == 0.0) neumann_axis(n, fwd, inv, lam);  // the closed form kv_create_grid uses
  const size_t nn = (size_t)n * n;
  // fwd: row = mode, column = cell (E^-1); inv: row = cell, column = mode (E)
  if (E) memcpy(E, inv.data(), nn * sizeof(double));
  if (E_inv) memcpy(E_inv, fwd.data(), nn * sizeof(double));
  if (lambda) memcpy(lambda, lam.data(), (size_t)n * sizeof(double));
  if (weights) memcpy(weights, tab.data(), tab.size() * sizeof(double));
  return KV_OK;
}

const char* kv_last_error(kv_handle h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

}  // extern "C"
