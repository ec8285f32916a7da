// Krylov solvers and the Newton iteration around the Krylov-vector map: the method's steps on
// either side of the hot path. Section 2 states the Newton method (residual F of the steady
// equations, solve J [u, p, theta] = F, U -> U - u); Section 3.1 solves the Jacobian systems with
// GMRES restarted after every 100 Krylov vectors until it saturates, then BiCGstab(2) from
// GMRES's last approximation. The paper defers both solvers to its reference [17]; they follow
// their published definitions: GMRES(m) by Saad and Schultz (1986), BiCGstab(l) by Sleijpen and
// Fokkema (1993) with l = 2.
//
// The host drives the iterations (a few scalars per step); every product with the Jacobian is
// kv_krylov_vector, every GMRES basis vector comes from kv_arnoldi_step, and the vector updates
// and inner products run in this file's kernel and the library's FP64 reduction kernels, on
// the handle's stream.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "kv_internal.cuh"

namespace {

#define KV_SOLVE_CUDA(h, call)                                                      \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return e_ == cudaErrorMemoryAllocation ? KV_ERR_NOMEM : KV_ERR_CUDA;          \
    }                                                                               \
  } while (0)

#define KV_SOLVE_TRY(call)         \
  do {                             \
    const kv_status s_ = (call);   \
    if (s_ != KV_OK) return s_;    \
  } while (0)

kv_status sfail(kv_grid* h, kv_status st, const char* msg) {
  h->err = msg;
  return st;
}

kv_status launched(kv_grid* h, const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string(what) + ": " + cudaGetErrorString(e);
    return KV_ERR_CUDA;
  }
  return KV_OK;
}

// y = a x + b y over n entries; b == 0 writes a x without reading y. x may be y.
__global__ void __launch_bounds__(256) k_axpby(size_t n, double a, const double* x, double b, double* y) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0.0) {
    for (; i < n; i += stride) y[i] = a * x[i];
  } else {
    for (; i < n; i += stride) y[i] = fma(a, x[i], b * y[i]);
  }
}

int axpby_blocks() {
  static const int nb = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? 4 * sms : 608;
  }();
  return nb;
}

kv_status axpby(kv_grid* h, double a, const double* x, double b, double* y) {
  k_axpby<<<axpby_blocks(), 256, 0, h->s>>>(4 * h->P, a, x, b, y);
  return launched(h, "axpby");
}

// The solvers' device scratch: block partial sums of up to 8 inner products, then `small`
// doubles (inner-product results, GMRES's combination coefficients).
kv_status scratch(kv_grid* h, size_t small) {
  const size_t need = (size_t)8 * kv_reduce_blocks() + small;
  if (h->solve_cap >= need) return KV_OK;
  cudaFree(h->solve_buf);
  h->solve_buf = nullptr;
  h->solve_cap = 0;
  KV_SOLVE_CUDA(h, cudaMalloc((void**)&h->solve_buf, need * sizeof(double)));
  h->solve_cap = need;
  return KV_OK;
}
double* small_buf(kv_grid* h) { return h->solve_buf + (size_t)8 * kv_reduce_blocks(); }

// out[q] = <V + q ld, w> for q < nq (nq <= 8), returned on the host (synchronises)
kv_status dots(kv_grid* h, const double* V, size_t ld, int nq, const double* w, double* out) {
  kv_launch_multidot(V, ld, nq, w, 4 * h->P, h->solve_buf, small_buf(h), 0, h->s);
  KV_SOLVE_TRY(launched(h, "inner products"));
  KV_SOLVE_CUDA(h, cudaMemcpyAsync(out, small_buf(h), nq * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  KV_SOLVE_CUDA(h, cudaStreamSynchronize(h->s));
  return KV_OK;
}

kv_status norm(kv_grid* h, const double* x, double* nrm) {
  double d = 0.0;
  KV_SOLVE_TRY(dots(h, x, 0, 1, x, &d));
  *nrm = d > 0.0 ? sqrt(d) : 0.0;
  return KV_OK;
}

bool overlaps(const double* a, size_t na, const double* b, size_t nb) { return a < b + nb && b < a + na; }

bool bad(double d) { return d == 0.0 || !isfinite(d); }

}  // namespace

extern "C" kv_status kv_gmres(kv_handle h, const double* b, double* x, double* V, int m, int max_restarts,
                              double tol, double sat, kv_solve_stats* st) {
  if (!h) return KV_ERR_ARG;
  if (!b || !x || !V || m < 1 || m > 4095 || max_restarts < 1 || !(tol >= 0.0) || !(sat > 0.0))
    return sfail(h, KV_ERR_ARG, "kv_gmres: bad argument");
  if (!h->has_base) return sfail(h, KV_ERR_STATE, "kv_gmres: no base flow set");
  const size_t L = 4 * h->P;
  const size_t LV = (size_t)(m + 1) * L;
  if (overlaps(x, L, V, LV) || overlaps(b, L, V, LV) || overlaps(x, L, b, L))
    return sfail(h, KV_ERR_ARG, "kv_gmres: b, x and V overlap");
  KV_SOLVE_TRY(scratch(h, (size_t)m + 8));
  kv_solve_stats S{};
  double bnorm = 0.0;
  KV_SOLVE_TRY(norm(h, b, &bnorm));
  if (bnorm == 0.0) {  // A x = 0: x = 0
    KV_SOLVE_CUDA(h, cudaMemsetAsync(x, 0, L * sizeof(double), h->s));
    KV_SOLVE_CUDA(h, cudaStreamSynchronize(h->s));
    S.converged = 1;
    if (st) *st = S;
    return KV_OK;
  }
  // H column-major: H[j * (m + 1) + i] = h_ij after the rotations (upper triangular R)
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hc(m + 2), c(m);
  double prev = -1.0;
  for (int cyc = 0; cyc < max_restarts; ++cyc) {
    // r = b - A x, the first basis vector
    KV_SOLVE_TRY(kv_krylov_vector(h, x, V, nullptr, nullptr));
    ++S.matvecs;
    KV_SOLVE_TRY(axpby(h, 1.0, b, -1.0, V));
    double beta = 0.0;
    KV_SOLVE_TRY(norm(h, V, &beta));
    if (beta <= tol * bnorm) {
      S.converged = 1;
      break;
    }
    if (prev >= 0.0 && beta > sat * prev) {  // no progress over the last cycle
      S.saturated = 1;
      break;
    }
    prev = beta;
    ++S.restarts;
    KV_SOLVE_TRY(axpby(h, 1.0 / beta, V, 0.0, V));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      KV_SOLVE_TRY(kv_arnoldi_step(h, V, j, hc.data()));
      ++S.matvecs;
      ++S.iterations;
      double* col = &H[(size_t)j * (m + 1)];
      for (int i = 0; i <= j + 1; ++i) col[i] = hc[i];
      // the earlier rotations on the new column, then the one that zeroes its last entry
      for (int i = 0; i < j; ++i) {
        const double a0 = col[i], a1 = col[i + 1];
        col[i] = cs[i] * a0 + sn[i] * a1;
        col[i + 1] = -sn[i] * a0 + cs[i] * a1;
      }
      const double d = hypot(col[j], col[j + 1]);
      cs[j] = d == 0.0 ? 1.0 : col[j] / d;
      sn[j] = d == 0.0 ? 0.0 : col[j + 1] / d;
      col[j] = d;
      col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      if (fabs(g[j + 1]) <= tol * bnorm) break;
    }
    // R y = g[0:k], then x += V y (kv_launch_update forms w -= V c, so c = -y)
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
      const double rii = H[(size_t)i * (m + 1) + i];
      y[i] = rii != 0.0 ? s / rii : 0.0;
    }
    for (int i = 0; i < k; ++i) c[i] = -y[i];
    KV_SOLVE_CUDA(h, cudaMemcpyAsync(small_buf(h), c.data(), k * sizeof(double), cudaMemcpyHostToDevice, h->s));
    kv_launch_update(V, L, k, small_buf(h), x, L, h->s);
    KV_SOLVE_TRY(launched(h, "GMRES update"));
  }
  // the residual of the returned x, recomputed
  KV_SOLVE_TRY(kv_krylov_vector(h, x, V, nullptr, nullptr));
  ++S.matvecs;
  KV_SOLVE_TRY(axpby(h, 1.0, b, -1.0, V));
  double r = 0.0;
  KV_SOLVE_TRY(norm(h, V, &r));
  S.rel_residual = r / bnorm;
  if (S.rel_residual <= tol) S.converged = 1;
  if (st) *st = S;
  return KV_OK;
}

extern "C" kv_status kv_bicgstab2(kv_handle h, const double* b, double* x, double* work, int max_iter, double tol,
                                  kv_solve_stats* st) {
  if (!h) return KV_ERR_ARG;
  if (!b || !x || !work || max_iter < 0 || !(tol >= 0.0)) return sfail(h, KV_ERR_ARG, "kv_bicgstab2: bad argument");
  if (!h->has_base) return sfail(h, KV_ERR_STATE, "kv_bicgstab2: no base flow set");
  const size_t L = 4 * h->P;
  if (overlaps(x, L, work, 8 * L) || overlaps(b, L, work, 8 * L) || overlaps(x, L, b, L))
    return sfail(h, KV_ERR_ARG, "kv_bicgstab2: b, x and work overlap");
  KV_SOLVE_TRY(scratch(h, 8));
  // work: shadow residual, r^_0..r^_2 (consecutive), u^_0..u^_2, a copy of x
  double* rt = work;
  double* rr[3] = {work + L, work + 2 * L, work + 3 * L};
  double* uu[3] = {work + 4 * L, work + 5 * L, work + 6 * L};
  double* xs = work + 7 * L;
  kv_solve_stats S{};
  double bnorm = 0.0;
  KV_SOLVE_TRY(norm(h, b, &bnorm));
  if (bnorm == 0.0) {
    KV_SOLVE_CUDA(h, cudaMemsetAsync(x, 0, L * sizeof(double), h->s));
    KV_SOLVE_CUDA(h, cudaStreamSynchronize(h->s));
    S.converged = 1;
    if (st) *st = S;
    return KV_OK;
  }
  KV_SOLVE_TRY(kv_krylov_vector(h, x, rr[0], nullptr, nullptr));
  S.matvecs = 1;
  KV_SOLVE_TRY(axpby(h, 1.0, b, -1.0, rr[0]));
  KV_SOLVE_CUDA(h, cudaMemcpyAsync(rt, rr[0], L * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
  KV_SOLVE_CUDA(h, cudaMemsetAsync(uu[0], 0, L * sizeof(double), h->s));
  double rho0 = 1.0, alpha = 0.0, omega = 1.0, rn = 0.0;
  KV_SOLVE_TRY(norm(h, rr[0], &rn));
  bool done = rn <= tol * bnorm;
  while (!done && S.iterations < max_iter) {
    rho0 = -omega * rho0;
    KV_SOLVE_CUDA(h, cudaMemcpyAsync(xs, x, L * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    bool brk = false;
    // BiCG part: two steps
    for (int j = 0; j < 2 && !brk; ++j) {
      double rho1 = 0.0;
      KV_SOLVE_TRY(dots(h, rr[j], 0, 1, rt, &rho1));
      if (bad(rho0)) {
        brk = true;
        break;
      }
      const double beta = alpha * rho1 / rho0;
      rho0 = rho1;
      for (int i = 0; i <= j; ++i) KV_SOLVE_TRY(axpby(h, 1.0, rr[i], -beta, uu[i]));
      KV_SOLVE_TRY(kv_krylov_vector(h, uu[j], uu[j + 1], nullptr, nullptr));
      double gamma = 0.0;
      KV_SOLVE_TRY(dots(h, uu[j + 1], 0, 1, rt, &gamma));
      if (bad(gamma)) {
        brk = true;
        break;
      }
      alpha = rho0 / gamma;
      for (int i = 0; i <= j; ++i) KV_SOLVE_TRY(axpby(h, -alpha, uu[i + 1], 1.0, rr[i]));
      KV_SOLVE_TRY(kv_krylov_vector(h, rr[j], rr[j + 1], nullptr, nullptr));
      KV_SOLVE_TRY(axpby(h, alpha, uu[0], 1.0, x));
      S.matvecs += 2;
    }
    // MR part: modified Gram-Schmidt on r^_1, r^_2 and the degree-2 residual polynomial
    double d3[3] = {0.0, 0.0, 0.0}, d2[2] = {0.0, 0.0};
    double sigma1 = 0.0, sigma2 = 0.0, g1p = 0.0, tau12 = 0.0;
    if (!brk) {
      KV_SOLVE_TRY(dots(h, rr[0], L, 3, rr[1], d3));  // <r0, r1>, <r1, r1>, <r2, r1>
      sigma1 = d3[1];
      brk = bad(sigma1);
    }
    if (!brk) {
      g1p = d3[0] / sigma1;
      tau12 = d3[2] / sigma1;
      KV_SOLVE_TRY(axpby(h, -tau12, rr[1], 1.0, rr[2]));
      KV_SOLVE_TRY(dots(h, rr[0], 2 * L, 2, rr[2], d2));  // <r0, r2>, <r2, r2>
      sigma2 = d2[1];
      brk = bad(sigma2);
    }
    if (brk) {  // the last complete iterate
      KV_SOLVE_CUDA(h, cudaMemcpyAsync(x, xs, L * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
      S.breakdown = 1;
      break;
    }
    const double g2p = d2[0] / sigma2;
    const double g2 = g2p, g1 = g1p - tau12 * g2, g1pp = g2;
    omega = g2;
    KV_SOLVE_TRY(axpby(h, g1, rr[0], 1.0, x));
    KV_SOLVE_TRY(axpby(h, -g2p, rr[2], 1.0, rr[0]));
    KV_SOLVE_TRY(axpby(h, -g2, uu[2], 1.0, uu[0]));
    KV_SOLVE_TRY(axpby(h, -g1, uu[1], 1.0, uu[0]));
    KV_SOLVE_TRY(axpby(h, g1pp, rr[1], 1.0, x));
    KV_SOLVE_TRY(axpby(h, -g1p, rr[1], 1.0, rr[0]));
    ++S.iterations;
    KV_SOLVE_TRY(norm(h, rr[0], &rn));
    done = rn <= tol * bnorm;
  }
  // the residual of the returned x, recomputed
  KV_SOLVE_TRY(kv_krylov_vector(h, x, uu[1], nullptr, nullptr));
  ++S.matvecs;
  KV_SOLVE_TRY(axpby(h, 1.0, b, -1.0, uu[1]));
  double r = 0.0;
  KV_SOLVE_TRY(norm(h, uu[1], &r));
  S.rel_residual = r / bnorm;
  S.converged = S.rel_residual <= tol;
  if (st) *st = S;
  return KV_OK;
}

extern "C" kv_status kv_newton(kv_handle h, double* S, double* V, double* work, const kv_newton_params* p,
                               kv_newton_stats* st) {
  if (!h) return KV_ERR_ARG;
  if (!S || !V || !work || !p || p->max_newton < 0 || p->max_newton > KV_NEWTON_HISTORY - 1 || !(p->tol >= 0.0) ||
      p->gmres_m < 1 || p->gmres_m > 4095 || p->gmres_max_restarts < 1 || !(p->lin_tol >= 0.0) ||
      !(p->gmres_sat > 0.0) || p->bicg_max_iter < 0)
    return sfail(h, KV_ERR_ARG, "kv_newton: bad argument");
  const size_t L = 4 * h->P;
  const size_t LV = (size_t)(p->gmres_m + 1) * L;
  if (overlaps(S, L, V, LV) || overlaps(S, L, work, 10 * L) || overlaps(V, LV, work, 10 * L))
    return sfail(h, KV_ERR_ARG, "kv_newton: S, V and work overlap");
  double* F = work;      // projected residual of S (the right-hand side)
  double* d = work + L;  // the Newton correction
  double* bw = work + 2 * L;
  kv_newton_stats N{};
  for (int it = 0;; ++it) {
    double nrm = 0.0;
    KV_SOLVE_TRY(kv_newton_residual(h, S, F, &nrm));
    N.res_norm[it] = nrm;
    N.n_res = it + 1;
    if (nrm < p->tol) {
      N.converged = 1;
      break;
    }
    if (it == p->max_newton) break;
    // the Jacobian at S, then J d = F: GMRES(m) until it converges or saturates, then BiCGstab(2)
    KV_SOLVE_TRY(kv_set_base_flow_packed(h, S));
    KV_SOLVE_CUDA(h, cudaMemsetAsync(d, 0, L * sizeof(double), h->s));
    kv_solve_stats gs{};
    KV_SOLVE_TRY(kv_gmres(h, F, d, V, p->gmres_m, p->gmres_max_restarts, p->lin_tol, p->gmres_sat, &gs));
    N.matvecs += gs.matvecs;
    N.gmres_restarts += gs.restarts;
    if (!gs.converged && p->bicg_max_iter > 0) {
      // BiCGstab(2) from GMRES's result; its correction replaces GMRES's only with a smaller
      // recomputed residual (started at the rounding level of the Krylov vectors it can stagnate
      // or diverge). GMRES's correction waits in V, free once GMRES has returned.
      KV_SOLVE_CUDA(h, cudaMemcpyAsync(V, d, L * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
      kv_solve_stats bs{};
      KV_SOLVE_TRY(kv_bicgstab2(h, F, d, bw, p->bicg_max_iter, p->lin_tol, &bs));
      N.matvecs += bs.matvecs;
      N.bicg_iterations += bs.iterations;
      // and, preferred that way, it is still dropped when the Newton step with it does not decrease
      // ||F|| (a correction can have the smaller linear residual and carry a large part the linear
      // residual does not see); bw, BiCGstab's workspace, is free again for the trial state
      bool take = bs.rel_residual < gs.rel_residual;
      if (take) {
        double* trial = bw;
        double ntry = 0.0;
        KV_SOLVE_CUDA(h, cudaMemcpyAsync(trial, S, L * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
        KV_SOLVE_TRY(axpby(h, -1.0, d, 1.0, trial));
        KV_SOLVE_TRY(kv_newton_residual(h, trial, bw + L, &ntry));
        take = ntry <= nrm;
      }
      if (!take) {
        KV_SOLVE_CUDA(h, cudaMemcpyAsync(d, V, L * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
        ++N.bicg_rejected;
      }
    }
    KV_SOLVE_TRY(axpby(h, -1.0, d, 1.0, S));
    ++N.iterations;
  }
  KV_SOLVE_CUDA(h, cudaStreamSynchronize(h->s));
  if (st) *st = N;
  return KV_OK;
}

extern "C" kv_status kv_axpby(kv_handle h, double a, const double* x, double b, double* y) {
  if (!h) return KV_ERR_ARG;
  if (!x || !y || !isfinite(a) || !isfinite(b)) return sfail(h, KV_ERR_ARG, "kv_axpby: bad argument");
  const size_t L = 4 * h->P;
  if (x != y && overlaps(x, L, y, L)) return sfail(h, KV_ERR_ARG, "kv_axpby: x and y overlap");
  return axpby(h, a, x, b, y);
}

extern "C" kv_status kv_combine(kv_handle h, const double* V, int k, const double* c, double* y) {
  if (!h) return KV_ERR_ARG;
  if (!V || !c || !y || k < 1 || k > 4096) return sfail(h, KV_ERR_ARG, "kv_combine: bad argument");
  const size_t L = 4 * h->P;
  if (overlaps(y, L, V, (size_t)k * L)) return sfail(h, KV_ERR_ARG, "kv_combine: y overlaps V");
  for (int i = 0; i < k; ++i)
    if (!isfinite(c[i])) return sfail(h, KV_ERR_ARG, "kv_combine: non-finite coefficient");
  KV_SOLVE_TRY(scratch(h, (size_t)k + 8));
  // y = 0, then y -= V (-c) (kv_launch_update forms w -= V c)
  std::vector<double> nc(k);
  for (int i = 0; i < k; ++i) nc[i] = -c[i];
  KV_SOLVE_CUDA(h, cudaMemsetAsync(y, 0, L * sizeof(double), h->s));
  KV_SOLVE_CUDA(h, cudaMemcpyAsync(small_buf(h), nc.data(), k * sizeof(double), cudaMemcpyHostToDevice, h->s));
  kv_launch_update(V, L, k, small_buf(h), y, L, h->s);
  KV_SOLVE_TRY(launched(h, "combine"));
  KV_SOLVE_CUDA(h, cudaStreamSynchronize(h->s));
  return KV_OK;
}

extern "C" kv_status kv_dot(kv_handle h, const double* x, const double* y, double* out) {
  if (!h) return KV_ERR_ARG;
  if (!x || !y || !out) return sfail(h, KV_ERR_ARG, "kv_dot: bad argument");
  KV_SOLVE_TRY(scratch(h, 8));
  return dots(h, x, 0, 1, y, out);
}
