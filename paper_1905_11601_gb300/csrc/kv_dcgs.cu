// The sweeps of the delayed classical Gram-Schmidt behind kv_arnoldi_run.
//
// Classical Gram-Schmidt applied twice (the Arnoldi orthogonalisation of Section 3.1 and
// kv_arnoldi_step) reads the basis in three sweeps per step: the inner products, the update with
// the next pass's inner products, and the second update. Here the second application of step j
// is deferred to step j + 1, where it shares that step's two sweeps (after Swirydowicz, Langou,
// Ananthan, Yang and Thomas, "Low synchronization Gram-Schmidt and generalized minimal residual
// algorithms", 2021): step j reads the final basis V_0..V_{j-1}, the provisional vector u_j (one
// projection, not normalised) and w = A u_j once for all inner products, then once more to write
// the final v_j = (u_j - V a) / beta and the next provisional vector, a combination of w, u_j and
// the basis whose coefficients follow from the inner products and the Hessenberg matrix
// (A v_j = (w - V H a) / beta by the Arnoldi relation of the final columns). In exact arithmetic
// the basis and the Hessenberg matrix are those of classical Gram-Schmidt applied twice.
//
// Arithmetic as the fused sweeps of kv_reduce.cu: in mixed precision the first basis vectors of
// each sweep in FP64 on the FP64 pipe and the rest in double-float on the FP32 pipe; with
// KV_PREC_FP64 every product in FP64.
#include "kv_df.cuh"
#include "kv_internal.cuh"

namespace {

constexpr int RT = 256;  // threads per block
constexpr int QD = 24;   // basis vectors per chunk of a sweep
#define KV_FOR_EACH_Q0(X)                                                                                       \
  X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) \
      X(20) X(21) X(22) X(23) X(24)

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// finite and |x| < 2^48: the range the double-float sweeps take (as in kv_reduce.cu)
__device__ __forceinline__ bool df_range(double x) {
  const unsigned int ex = ((unsigned int)__double2hiint(x) >> 20) & 0x7FFu;
  return ex < 1023u + 48u;
}

// FP64 share: the FP64 pipe keeps up with HBM for about 0.6 multiply-adds per 8-byte entry
// streamed. The inner-product sweep streams Q + 2 vectors and spends two multiply-adds per FP64
// basis vector; the update sweep streams Q + 4 and spends two per FP64 basis vector plus three.
template <int Q>
__host__ __device__ constexpr int dots2_k64() {
  return (3 * (Q + 2)) / 10 < Q ? (3 * (Q + 2)) / 10 : Q;
}
template <int Q>
__host__ __device__ constexpr int update2_k64() {
  return (3 * (Q + 4) - 15) / 10 < 0 ? 0 : ((3 * (Q + 4) - 15) / 10 < Q ? (3 * (Q + 4) - 15) / 10 : Q);
}

// U consecutive entries from e (zero past len), one 16-byte load when vec and U == 2
template <int U>
__device__ __forceinline__ void load_n(const double* __restrict__ p, size_t e, size_t len, bool vec,
                                       double (&out)[U]) {
  if constexpr (U == 2) {
    if (vec && e + 1 < len) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p + e));
      out[0] = t.x;
      out[1] = t.y;
    } else {
      out[0] = __ldg(p + e);
      out[1] = e + 1 < len ? __ldg(p + e + 1) : 0.0;
    }
  } else {
    out[0] = __ldg(p + e);
  }
}

// two adjacent entries per thread and iteration (twice the loads in flight) while the
// registers allow it
template <int Q>
__host__ __device__ constexpr int dots2_unroll() { return Q <= 10 ? 2 : 1; }

// Block partials (rows rb apart): [0, Q) <V_q, u>, [Q, 2Q) <V_q, w>, 2Q <u, w>, 2Q + 1 <u, u>
// (NaN if an entry of u or w is out of the double-float range), 2Q + 2 <w, w>.
template <int Q, bool DFM>
__global__ void __launch_bounds__(RT) k_dots2(const double* __restrict__ V, size_t ld, const double* __restrict__ u,
                                              const double* __restrict__ w, size_t len, size_t rb, int vec,
                                              double* __restrict__ partials) {
  constexpr int K64 = DFM ? dots2_k64<Q>() : Q;
  constexpr int QA = Q > 0 ? Q : 1;
  constexpr int R = 2 * Q + 3;
  constexpr int U = dots2_unroll<Q>();
  __shared__ double sm[R][RT / 32];
  double au[QA], aw[QA];
  DFAcc du[QA], dw[QA], uw, uu, ww;
  double uw64 = 0.0, uu64 = 0.0, ww64 = 0.0;
#pragma unroll
  for (int q = 0; q < QA; ++q) {
    au[q] = 0.0;
    aw[q] = 0.0;
  }
  bool bad = false;
  for (size_t e = ((size_t)blockIdx.x * RT + threadIdx.x) * U; e < len; e += (size_t)gridDim.x * RT * U) {
    double ud[U], wd[U], vd[QA][U];
    load_n<U>(u, e, len, vec, ud);
    load_n<U>(w, e, len, vec, wd);
#pragma unroll
    for (int q = 0; q < Q; ++q) load_n<U>(V + (size_t)q * ld, e, len, vec, vd[q]);
#pragma unroll
    for (int k = 0; k < U; ++k) {
#pragma unroll
      for (int q = 0; q < K64; ++q) {
        au[q] = fma(vd[q][k], ud[k], au[q]);
        aw[q] = fma(vd[q][k], wd[k], aw[q]);
      }
      if (DFM) {
        bad |= !df_range(ud[k]) || !df_range(wd[k]);
        const DF us = df_split(ud[k]), ws = df_split(wd[k]);
#pragma unroll
        for (int q = K64; q < Q; ++q) {
          const DF v = df_split(vd[q][k]);
          du[q].fma(v, us);
          dw[q].fma(v, ws);
        }
        uw.fma(us, ws);
        uu.fma(us, us);
        ww.fma(ws, ws);
      } else {
        uw64 = fma(ud[k], wd[k], uw64);
        uu64 = fma(ud[k], ud[k], uu64);
        ww64 = fma(wd[k], wd[k], ww64);
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double x;
    if (r < Q)
      x = r < K64 ? au[r] : du[r].value();
    else if (r < 2 * Q)
      x = r - Q < K64 ? aw[r - Q] : dw[r - Q].value();
    else if (r == 2 * Q)
      x = DFM ? uw.value() : uw64;
    else if (r == 2 * Q + 1)
      x = DFM ? (bad ? __longlong_as_double(0x7FF8000000000000LL) : uu.value()) : uu64;
    else
      x = DFM ? ww.value() : ww64;
    const double t = warp_sum_d(x);
    if (lane == 0) sm[r][warp] = t;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += RT) {
    double s = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) s += sm[r][wv];
    partials[(size_t)r * rb + blockIdx.x] = s;
  }
}

// u <- c0 u + sum_q cu_q V_q, w <- cw w + cwu u + sum_q cw_q V_q, both from the entering u;
// s3 = (c0, cw, cwu). Stored rounded to FP64.
template <int Q, bool DFM>
__global__ void __launch_bounds__(RT) k_update2(const double* __restrict__ V, size_t ld,
                                                const double* __restrict__ s3, const double* __restrict__ cuv,
                                                const double* __restrict__ cwv, double* __restrict__ u,
                                                double* __restrict__ w, size_t len, int write_u, int write_w) {
  constexpr int K64 = DFM ? update2_k64<Q>() : Q;
  constexpr int QA = Q > 0 ? Q : 1;
  __shared__ double cu64[QA], cw64[QA], c3[3];
  __shared__ DF cud[QA], cwd[QA];
  const int t = threadIdx.x;
  if (t < Q) {
    const double a = cuv[t], b = cwv[t];
    cu64[t] = a;
    cw64[t] = b;
    cud[t] = df_split(a);
    cwd[t] = df_split(b);
  }
  if (t < 3) c3[t] = s3[t];
  __syncthreads();
  const double c0 = c3[0], cw = c3[1], cwu = c3[2];
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    const double ud = u[e];
    const double wd = write_w ? w[e] : 0.0;
    double vd[QA];
#pragma unroll
    for (int q = 0; q < Q; ++q) vd[q] = __ldg(V + (size_t)q * ld + e);
    double un = c0 * ud, wn = fma(cw, wd, cwu * ud);
#pragma unroll
    for (int q = 0; q < K64; ++q) {
      un = fma(cu64[q], vd[q], un);
      wn = fma(cw64[q], vd[q], wn);
    }
    if (DFM && K64 < Q) {
      DFAcc a, b;
      a.start(df_split(un));
      b.start(df_split(wn));
#pragma unroll
      for (int q = K64; q < Q; ++q) {
        const DF v = df_split(vd[q]);
        a.fma(cud[q], v);
        b.fma(cwd[q], v);
      }
      const DF a1 = a.pair(), b1 = b.pair();
      un = df_f2d(a1.h) + df_f2d(a1.l);
      wn = df_f2d(b1.h) + df_f2d(b1.l);
    }
    if (write_u) u[e] = un;
    if (write_w) w[e] = wn;
  }
}

// Inner products of a step, chunk c (vectors 24c .. 24c + q_c - 1) at dots + DS c:
// [<V, u> (q_c), <V, w> (q_c), <u, w>, <u, u>, <w, w>] (the last three equal in every chunk).
constexpr int DS = 2 * QD + 3;
__host__ __device__ __forceinline__ int chunk_q(int j, int c) { return j - QD * c < QD ? j - QD * c : QD; }

// One step's coefficients (one warp). With a = <V, u>, b = <V, w>, bu = <u, w>, nu = <u, u>
// (u = u_j, w = A u_j, V = the final V_0..V_{j-1}):
//   beta = sqrt(nu - a.a): column j-1 += a, its subdiagonal = beta (the deferred second
//   projection of u_j), v_j = (u_j - V a) / beta;
//   d = H[0..j, 0..j-1] a, so that A v_j = (w - [V, v_j] d) / beta;
//   h = the first projection of A v_j on [V, v_j]: h_q = (b_q - d_q) / beta, q < j,
//   h_j = ((bu - a.b) / beta - d_j) / beta; column j = h (provisional);
//   u_{j+1} = A v_j - [V, v_j] h = w / beta - (kappa / beta) u_j - V e,
//   kappa = d_j / beta + h_j, e = d / beta + h - a kappa / beta.
// Outputs: s3 = (1 / beta, 1 / beta, -kappa / beta), cuv = -a / beta, cwv = -e (the update
// sweep's coefficients). first (the run's first step, v_j final on entry): a = 0, beta = 1,
// column j-1 untouched. final_only: column j-1 and v_j only (the run's last vector). scr: 2 (j + 1)
// doubles of scratch.
__global__ void k_dcgs_coef(const double* __restrict__ dots, double* __restrict__ Hd, int ldh, int j, int first,
                            int final_only, double* __restrict__ s3, double* __restrict__ cuv,
                            double* __restrict__ cwv, double* __restrict__ scr, int* __restrict__ err) {
  __shared__ double sh[4];  // beta, a.b, kappa
  const int lane = threadIdx.x;
  auto a_of = [&](int q) { return first ? 0.0 : dots[(size_t)DS * (q / QD) + q % QD]; };
  auto b_of = [&](int q) { return dots[(size_t)DS * (q / QD) + chunk_q(j, q / QD) + q % QD]; };
  const int q0 = j < QD ? j : QD;
  const double bu = dots[2 * q0], nu = dots[2 * q0 + 1];
  double aa = 0.0, ab = 0.0;
  for (int q = lane; q < j; q += 32) {
    const double a = a_of(q);
    aa = fma(a, a, aa);
    if (!final_only) ab = fma(a, b_of(q), ab);
  }
  for (int o = 16; o > 0; o >>= 1) {
    aa += __shfl_xor_sync(0xffffffffu, aa, o);
    ab += __shfl_xor_sync(0xffffffffu, ab, o);
  }
  if (lane == 0) {
    double beta = 1.0;
    if (!first) {
      const double b2 = nu - aa;
      if (!(b2 > 0.0) || !isfinite(b2)) *err = 1;
      beta = sqrt(b2);
    } else if (!isfinite(nu)) {
      *err = 1;
    }
    sh[0] = beta;
    sh[1] = ab;
  }
  __syncwarp();
  const double beta = sh[0];
  if (!first) {
    for (int q = lane; q < j; q += 32) Hd[q + (size_t)ldh * (j - 1)] += a_of(q);
    if (lane == 0) Hd[j + (size_t)ldh * (j - 1)] = beta;
  }
  for (int q = lane; q < j; q += 32) cuv[q] = -a_of(q) / beta;
  if (lane == 0) s3[0] = 1.0 / beta;
  if (final_only) return;
  __syncwarp();
  // d = H[0..j, 0..j-1] a (the final columns, j - 1 included), one row per lane
  double* d = scr;
  double* hq = scr + j + 1;
  for (int r = lane; r <= j; r += 32) {
    double t = 0.0;
    if (!first)
      for (int c = (r > 0 ? r - 1 : 0); c < j; ++c) t = fma(Hd[r + (size_t)ldh * c], a_of(c), t);
    d[r] = t;
  }
  __syncwarp();
  for (int q = lane; q < j; q += 32) hq[q] = (b_of(q) - d[q]) / beta;
  if (lane == 0) {
    hq[j] = ((bu - sh[1]) / beta - d[j]) / beta;
    sh[2] = d[j] / beta + hq[j];
  }
  __syncwarp();
  const double kappa = sh[2];
  for (int q = lane; q <= j; q += 32) Hd[q + (size_t)ldh * j] = hq[q];
  for (int q = lane; q < j; q += 32) cwv[q] = -(d[q] / beta + hq[q] - a_of(q) * kappa / beta);
  if (lane == 0) {
    s3[1] = 1.0 / beta;
    s3[2] = -kappa / beta;
  }
}

// Blocks of kernel K resident at once (at most cap): one wave.
template <auto K>
int wave(int cap) {
  static const int nb = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, RT, 0);
    return per * sms;
  }();
  return nb > 0 && nb < cap ? nb : cap;
}

}  // namespace

int kv_dcgs_chunk() { return QD; }
int kv_dcgs_dots_stride() { return DS; }

namespace {
void dots2_one(const double* V, size_t ld, int q, const double* u, const double* w, size_t len, double* partials,
               double* out, int df, cudaStream_t s) {
  const int rb = kv_reduce_blocks();
  int nb = rb;
  // V_q, u and w all start on 16-byte boundaries
  const int vec = (uintptr_t)V % 16 == 0 && ld % 2 == 0 && (uintptr_t)u % 16 == 0 && (uintptr_t)w % 16 == 0;
  if (df) {
    switch (q) {
#define KV_DOTS2_DF(Qn)                                                              \
  case Qn:                                                                           \
    nb = wave<k_dots2<Qn, true>>(rb);                                                \
    k_dots2<Qn, true><<<nb, RT, 0, s>>>(V, ld, u, w, len, (size_t)rb, vec, partials); \
    break;
      KV_FOR_EACH_Q0(KV_DOTS2_DF)
#undef KV_DOTS2_DF
    }
  } else {
    switch (q) {
#define KV_DOTS2_64(Qn)                                                               \
  case Qn:                                                                            \
    nb = wave<k_dots2<Qn, false>>(rb);                                                \
    k_dots2<Qn, false><<<nb, RT, 0, s>>>(V, ld, u, w, len, (size_t)rb, vec, partials); \
    break;
      KV_FOR_EACH_Q0(KV_DOTS2_64)
#undef KV_DOTS2_64
    }
  }
  kv_launch_finalize(partials, 2 * q + 3, nb, out, s);
}

void update2_one(const double* V, size_t ld, int q, const double* s3, const double* cuv, const double* cwv, double* u,
                 double* w, size_t len, int write_u, int write_w, int df, cudaStream_t s) {
  const int rb = kv_reduce_blocks();
  if (df) {
    switch (q) {
#define KV_UPD2_DF(Qn)                                                                                    \
  case Qn:                                                                                                \
    k_update2<Qn, true><<<wave<k_update2<Qn, true>>(rb), RT, 0, s>>>(V, ld, s3, cuv, cwv, u, w, len, write_u, \
                                                                      write_w);                           \
    break;
      KV_FOR_EACH_Q0(KV_UPD2_DF)
#undef KV_UPD2_DF
    }
  } else {
    switch (q) {
#define KV_UPD2_64(Qn)                                                                                      \
  case Qn:                                                                                                  \
    k_update2<Qn, false><<<wave<k_update2<Qn, false>>(rb), RT, 0, s>>>(V, ld, s3, cuv, cwv, u, w, len, write_u, \
                                                                        write_w);                           \
    break;
      KV_FOR_EACH_Q0(KV_UPD2_64)
#undef KV_UPD2_64
    }
  }
}
}  // namespace

void kv_launch_dots2(const double* V, size_t ld, int q, const double* u, const double* w, size_t len,
                     double* partials, double* dots, int df, cudaStream_t s) {
  if (q == 0) {
    dots2_one(V, ld, 0, u, w, len, partials, dots, df, s);
    return;
  }
  for (int c = 0; QD * c < q; ++c)
    dots2_one(V + (size_t)QD * c * ld, ld, chunk_q(q, c), u, w, len, partials, dots + (size_t)DS * c, df, s);
}

void kv_launch_dcgs_coef(const double* dots, double* Hd, int ldh, int j, int first, int final_only, double* s3,
                         double* cuv, double* cwv, double* scr, int* err, cudaStream_t s) {
  k_dcgs_coef<<<1, 32, 0, s>>>(dots, Hd, ldh, j, first, final_only, s3, cuv, cwv, scr, err);
}

void kv_launch_update2(const double* V, size_t ld, int q, const double* s3, const double* one3, const double* cuv,
                       const double* cwv, double* u, double* w, size_t len, int write_u, int write_w, int df,
                       cudaStream_t s) {
  if (q == 0) {
    update2_one(V, ld, 0, s3, cuv, cwv, u, w, len, write_u, write_w, df, s);
    return;
  }
  for (int c = 0; QD * c < q; ++c)
    update2_one(V + (size_t)QD * c * ld, ld, chunk_q(q, c), c == 0 ? s3 : one3, cuv + (size_t)QD * c,
                cwv + (size_t)QD * c, u, w, len, write_u, write_w, df, s);
}
