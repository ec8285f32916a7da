// FP64 reductions for the Arnoldi step: several inner products against one vector
// (classical Gram-Schmidt), the matching update, and the 2-norm. Partial sums per block are
// combined in a fixed order by a second kernel, so results are deterministic.
#include "kv_df.cuh"
#include "kv_internal.cuh"

namespace {

constexpr int RB = 1216;  // reduction blocks: 8 per SM on 152 SMs
constexpr int RT = 256;   // threads per block
constexpr int QB = 8;     // inner products accumulated per sweep over the vector
constexpr int QF = 24;    // largest basis handled by the fused Gram-Schmidt kernels
#define KV_FOR_EACH_NQ(X)                                                                                  \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) \
      X(20) X(21) X(22) X(23) X(24)

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partials[q * RB + block] = block's share of <V_q, w>, q = q0 .. q0 + nqb - 1
__global__ void __launch_bounds__(RT) k_multidot(const double* __restrict__ V, size_t ld, int q0, int nqb,
                                                 const double* __restrict__ w, size_t len,
                                                 double* __restrict__ partials) {
  double acc[QB];
#pragma unroll
  for (int q = 0; q < QB; ++q) acc[q] = 0.0;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    const double we = __ldg(w + e);
#pragma unroll
    for (int q = 0; q < QB; ++q)
      if (q < nqb) acc[q] = fma(__ldg(V + (size_t)(q0 + q) * ld + e), we, acc[q]);
  }
  __shared__ double sm[QB][RT / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // only the nqb accumulators in use: each warp-wide FP64 add occupies GB300's FP64 pipe (1/64 of
  // the FP32 rate) for about 16 cycles, so reducing all QB of them cost more than the sweep itself
  // on vectors of a few MB
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    if (q < nqb) {
      const double s = warp_sum(acc[q]);
      if (lane == 0) sm[q][warp] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < QB && (int)threadIdx.x < nqb) {
    double s = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) s += sm[threadIdx.x][wv];
    partials[(size_t)(q0 + threadIdx.x) * RB + blockIdx.x] = s;
  }
}

// out[q] (+)= sum_{b < nb} partials[q * RB + b]; one block per q
__global__ void __launch_bounds__(RT) k_finalize(const double* __restrict__ partials, int nb,
                                                 double* __restrict__ out, int accumulate) {
  const int q = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += RT) s += partials[(size_t)q * RB + b];
  s = warp_sum(s);
  __shared__ double sm[RT / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) t += sm[wv];
    out[q] = accumulate ? out[q] + t : t;
  }
}

// w[e] -= sum_q c[q] V_q[e]
__global__ void __launch_bounds__(RT) k_update(const double* __restrict__ V, size_t ld, int nq,
                                               const double* __restrict__ c, double* __restrict__ w, size_t len) {
  extern __shared__ double cs[];
  for (int q = threadIdx.x; q < nq; q += RT) cs[q] = c[q];
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s = fma(cs[q], __ldg(V + (size_t)q * ld + e), s);
    w[e] -= s;
  }
}

// FP32 value of a double from its high word (20 mantissa bits, truncated): integer operations
// only, so it stays off GB300's narrow FP64 pipe. Zero, denormals and tiny values map to 0.
// Only for quantities whose own rounding is negligible in the result.
__device__ __forceinline__ float hi_float(double d) {
  const unsigned int hi = (unsigned int)__double2hiint(d);
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  const unsigned int bits = (hi & 0x80000000u) | ((unsigned int)e << 23) | ((hi & 0xFFFFFu) << 3);
  return e > 0 ? __uint_as_float(bits) : 0.0f;
}

// Inner products <V_q, w> for q < nq (FP64), and with nrm also ||w||^2, in one sweep over w:
// partials[q * RB + block], the norm's share in partials[nq * RB + block].
template <int Q>
__global__ void __launch_bounds__(RT) k_dots(const double* __restrict__ V, size_t ld, int nq,
                                             const double* __restrict__ w, size_t len, int nrm,
                                             double* __restrict__ partials) {
  __shared__ double sm[Q + 1][RT / 32];
  double acc[Q + 1];
#pragma unroll
  for (int q = 0; q <= Q; ++q) acc[q] = 0.0;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    const double we = __ldg(w + e);
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = fma(__ldg(V + (size_t)q * ld + e), we, acc[q]);
    acc[Q] = fma(we, we, acc[Q]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q <= Q; ++q) {
    const double t = warp_sum(acc[q]);
    if (lane == 0) sm[q][warp] = t;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < nq || (nrm && t == Q)) {
    double s = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) s += sm[t][wv];
    partials[(size_t)(t < nq ? t : nq) * RB + blockIdx.x] = s;
  }
}

// First update fused with the second pass: w -= sum_q c[q] V_q (FP64), then the block's share of
// <V_q, w> (FP64: inner products of nearly orthogonal vectors need full precision) in
// partials[q * RB + block] and of the new ||w||^2 in partials[nq * RB + block].
template <int Q>
__global__ void __launch_bounds__(RT) k_update_dot(const double* __restrict__ V, size_t ld, int nq,
                                                   const double* __restrict__ c, double* __restrict__ w, size_t len,
                                                   double* __restrict__ partials) {
  __shared__ double cs[Q];
  __shared__ double sm[Q + 1][RT / 32];
  if (threadIdx.x < Q) cs[threadIdx.x] = (int)threadIdx.x < nq ? c[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[Q + 1];
#pragma unroll
  for (int q = 0; q <= Q; ++q) acc[q] = 0.0;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    double v[Q];
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      v[q] = __ldg(V + (size_t)q * ld + e);
      s = fma(cs[q], v[q], s);
    }
    const double w1 = w[e] - s;
    w[e] = w1;
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = fma(v[q], w1, acc[q]);
    acc[Q] = fma(w1, w1, acc[Q]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q <= Q; ++q) {
    const double t = warp_sum(acc[q]);
    if (lane == 0) sm[q][warp] = t;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < nq || t == Q) {
    double s = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) s += sm[t][wv];
    partials[(size_t)(t < nq ? t : nq) * RB + blockIdx.x] = s;
  }
}

// Second pass, second half, fused with the normalisation: w = (w - sum_q c[q] V_q) / beta. The
// second-pass coefficients are of rounding size relative to w, so their product with V is formed
// in FP32 from the high words (its error is ~1e-6 of a rounding-size correction) and subtracted
// in FP64. With V orthonormal and c = V^T w, beta^2 = ||w||^2 - ||c||^2 (c[nq] holds ||w||^2),
// which needs no further pass over w.
// With flag (the device-side decision of k_gs_decide) and *flag == 0 the second update is skipped:
// w = w / sqrt(c[Q]), without reading V.
template <int Q>
__global__ void __launch_bounds__(RT) k_update_small_scale(const double* __restrict__ V, size_t ld,
                                                           const double* __restrict__ c, double* __restrict__ w,
                                                           size_t len, const int* __restrict__ flag) {
  __shared__ float cs[Q];
  __shared__ double finv;
  const bool upd = flag == nullptr || *flag != 0;
  if (threadIdx.x < Q) cs[threadIdx.x] = (float)c[threadIdx.x];
  if (threadIdx.x == 0) {
    double s = 0.0;
    if (upd)
      for (int q = 0; q < Q; ++q) s = fma(c[q], c[q], s);
    const double b2 = c[Q] - s;
    finv = b2 > 0.0 || isnan(b2) ? 1.0 / sqrt(b2) : 0.0;
  }
  __syncthreads();
  const double f = finv;
  if (!upd) {
    for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) w[e] *= f;
    return;
  }
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) s = fmaf(cs[q], hi_float(__ldg(V + (size_t)q * ld + e)), s);
    w[e] = (w[e] - df_f2d(s)) * f;
  }
}

// The second-update decision and the Hessenberg column (one thread; nq <= QF): with
// h2n = ||h2||^2 (sequential FMA, the order k_update_small_scale uses), the update runs when
// forced or when h2n > theta^2 h2[nq]; the column is h1 + h2 and sqrt(h2[nq] - h2n) then, else
// h1 and sqrt(h2[nq]).
__global__ void k_gs_decide(const double* __restrict__ h1, const double* __restrict__ h2, int nq, double theta2,
                            int force, double* __restrict__ hcol, int* __restrict__ flag) {
  double h2n = 0.0;
  for (int q = 0; q < nq; ++q) h2n = fma(h2[q], h2[q], h2n);
  const double after = h2[nq];
  const int upd = force || !(h2n <= theta2 * after);
  *flag = upd;
  for (int q = 0; q < nq; ++q) hcol[q] = upd ? h1[q] + h2[q] : h1[q];
  const double b2 = upd ? after - h2n : after;
  hcol[nq] = b2 > 0.0 || isnan(b2) ? sqrt(b2) : 0.0;  // a NaN norm stays NaN
}

// ---- double-float Gram-Schmidt sweeps (mixed precision) -------------------------------------
//
// GB300's FP64 pipe cannot keep up with HBM in these sweeps (one FP64 multiply-add per 8 bytes
// read is already 1.4x the memory time), so the mixed-precision Arnoldi step forms the inner
// products and the first update in double-float arithmetic on the FP32 pipe (kv_df.cuh): the
// result of a sweep is within ~2^-46 of the sum of the magnitudes of its terms, against ~2^-53
// for FP64. Entries below 2^-103 in magnitude are flushed to zero (an absolute change of at
// most 2^-103 per entry); entries at or above 2^48 in the new vector (whose sums of squares
// could leave the FP32 range), NaN and Inf are reported by a NaN norm, which the host turns
// into an error.

// the new vector's entries must also satisfy |x| < 2^48: its squared norm, up to 2^31 entries,
// then stays below 2^127
__device__ __forceinline__ bool gs_in_range(double x) {
  const unsigned int ex = ((unsigned int)__double2hiint(x) >> 20) & 0x7FFu;
  return ex < 1023u + 48u;
}

// U consecutive entries p[e .. e+U-1] (zero past len), as one 16-byte load when vec (p and e
// 16-byte aligned)
template <int U>
__device__ __forceinline__ void load_u(const double* __restrict__ p, size_t e, size_t len, bool vec,
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

// Entries per thread and sweep iteration: two adjacent entries (16-byte loads, twice the loads
// in flight) while the registers allow it.
template <int Q>
__host__ __device__ constexpr int dots_unroll() { return Q <= 12 ? 2 : 1; }

// Both pipes at once: the FP64 pipe (2 multiply-adds per SM and clock) keeps up with HBM for
// about 0.6 multiply-adds per 8-byte entry streamed, so the first K64 basis vectors of a sweep
// run in plain FP64 and the rest in double-float on the FP32 pipe. The first sweep streams
// Q + 1 vectors and spends one FP64 multiply-add per FP64 vector; the fused sweep streams Q + 2
// and spends two.
template <int Q>
__host__ __device__ constexpr int dots_k64() { return (3 * (Q + 1)) / 5 < Q ? (3 * (Q + 1)) / 5 : Q; }
template <int Q>
__host__ __device__ constexpr int update_k64() { return (3 * (Q + 2)) / 10; }

// Block partials of <V_q, w> (q < Q) and ||w||^2, as k_dots: q < K64 in FP64, the others and
// the norm in double-float.
template <int Q>
__global__ void __launch_bounds__(RT) k_dots_df(const double* __restrict__ V, size_t ld,
                                                const double* __restrict__ w, size_t len, int nrm, int vec,
                                                double* __restrict__ partials) {
  constexpr int U = dots_unroll<Q>();
  constexpr int K64 = dots_k64<Q>();
  __shared__ double sm[Q + 1][RT / 32];
  double a64[K64 > 0 ? K64 : 1];
#pragma unroll
  for (int q = 0; q < K64; ++q) a64[q] = 0.0;
  DFAcc acc[Q + 1];
  bool bad = false;
  for (size_t e = ((size_t)blockIdx.x * RT + threadIdx.x) * U; e < len; e += (size_t)gridDim.x * RT * U) {
    double wd[U];
    double v[Q][U];
    load_u<U>(w, e, len, vec, wd);
#pragma unroll
    for (int q = 0; q < Q; ++q) load_u<U>(V + (size_t)q * ld, e, len, vec, v[q]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bad |= !gs_in_range(wd[u]);
#pragma unroll
      for (int q = 0; q < K64; ++q) a64[q] = fma(v[q][u], wd[u], a64[q]);
      const DF we = df_split(wd[u]);
#pragma unroll
      for (int q = K64; q < Q; ++q) acc[q].fma(df_split(v[q][u]), we);
      acc[Q].fma(we, we);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q <= Q; ++q) {
    double x = q < K64 ? a64[q < K64 ? q : 0] : acc[q].value();
    if (q == Q && bad) x = __longlong_as_double(0x7FF8000000000000LL);  // NaN: out of range
    const double t = warp_sum(x);
    if (lane == 0) sm[q][warp] = t;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < Q || (nrm && t == Q)) {
    double s = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) s += sm[t][wv];
    partials[(size_t)t * RB + blockIdx.x] = s;
  }
}

// w -= sum_q c[q] V_q, fused with the block partials of <V_q, w> and ||w||^2 of the updated w,
// as k_update_dot: the update and inner products of q < K64 in FP64 (the update first, on the
// FP64 value of w), the others and the norm in double-float. The updated w is stored rounded
// to FP64. One entry per thread and iteration; for Q <= 12 the next entry's loads are issued
// before the current entry's arithmetic (software prefetch), so the memory stream continues
// while a warp computes.
template <int Q>
__global__ void __launch_bounds__(RT, 2) k_update_dot_df(const double* __restrict__ V, size_t ld,
                                                         const double* __restrict__ c, double* __restrict__ w,
                                                         size_t len, double* __restrict__ partials) {
  constexpr int K64 = update_k64<Q>();
  constexpr bool PF = Q <= 12;
  __shared__ DF cs[Q];
  __shared__ double c64[K64 > 0 ? K64 : 1];
  __shared__ double sm[Q + 1][RT / 32];
  if (threadIdx.x < Q) {
    const DF x = df_split(c[threadIdx.x]);
    cs[threadIdx.x] = DF{-x.h, -x.l};
    if ((int)threadIdx.x < K64) c64[threadIdx.x] = c[threadIdx.x];
  }
  __syncthreads();
  double a64[K64 > 0 ? K64 : 1];
#pragma unroll
  for (int q = 0; q < K64; ++q) a64[q] = 0.0;
  DFAcc acc[Q + 1];
  const size_t stride = (size_t)gridDim.x * RT;
  size_t e = (size_t)blockIdx.x * RT + threadIdx.x;
  double vn[Q], wn = 0.0;
  if (PF && e < len) {
#pragma unroll
    for (int q = 0; q < Q; ++q) vn[q] = __ldg(V + (size_t)q * ld + e);
    wn = w[e];
  }
  for (; e < len; e += stride) {
    double vd[Q], wd;
    if (PF) {
#pragma unroll
      for (int q = 0; q < Q; ++q) vd[q] = vn[q];
      wd = wn;
      const size_t en = e + stride;
      if (en < len) {
#pragma unroll
        for (int q = 0; q < Q; ++q) vn[q] = __ldg(V + (size_t)q * ld + en);
        wn = w[en];
      }
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) vd[q] = __ldg(V + (size_t)q * ld + e);
      wd = w[e];
    }
    double w64 = wd;
#pragma unroll
    for (int q = 0; q < K64; ++q) w64 = fma(-c64[q], vd[q], w64);
    DFAcc a;
    a.start(df_split(w64));
    DF v[Q];
#pragma unroll
    for (int q = K64; q < Q; ++q) {
      v[q] = df_split(vd[q]);
      a.fma(cs[q], v[q]);
    }
    const DF w1 = a.pair();
    const double wo = df_f2d(w1.h) + df_f2d(w1.l);
    w[e] = wo;
#pragma unroll
    for (int q = 0; q < K64; ++q) a64[q] = fma(vd[q], wo, a64[q]);
#pragma unroll
    for (int q = K64; q < Q; ++q) acc[q].fma(v[q], w1);
    acc[Q].fma(w1, w1);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q <= Q; ++q) {
    const double t = warp_sum(q < K64 ? a64[q < K64 ? q : 0] : acc[q].value());
    if (lane == 0) sm[q][warp] = t;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t <= Q) {
    double s = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) s += sm[t][wv];
    partials[(size_t)t * RB + blockIdx.x] = s;
  }
}

// Any basis size (the sweeps beyond QF vectors): w -= sum_q c[q] V_q, the first k64 vectors in FP64
// on the FP64 pipe and the others in double-float on the FP32 pipe (the dual-pipe split of
// k_update_dot_df), without inner products; the updated w is stored rounded to FP64. Dynamic shared
// memory: k64 doubles, then nq - k64 FP32 pairs (the negated coefficients).
__global__ void __launch_bounds__(RT) k_update_n_df(const double* __restrict__ V, size_t ld, int nq, int k64,
                                                    const double* __restrict__ c, double* __restrict__ w, size_t len) {
  extern __shared__ double dyn[];
  double* c64 = dyn;
  DF* cs = reinterpret_cast<DF*>(dyn + k64);
  for (int q = threadIdx.x; q < nq; q += RT) {
    if (q < k64) {
      c64[q] = c[q];
    } else {
      const DF x = df_split(c[q]);
      cs[q - k64] = DF{-x.h, -x.l};
    }
  }
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    double w64 = w[e];
#pragma unroll 4
    for (int q = 0; q < k64; ++q) w64 = fma(-c64[q], __ldg(V + (size_t)q * ld + e), w64);
    DFAcc a;
    a.start(df_split(w64));
#pragma unroll 4
    for (int q = k64; q < nq; ++q) a.fma(cs[q - k64], df_split(__ldg(V + (size_t)q * ld + e)));
    const DF w1 = a.pair();
    w[e] = df_f2d(w1.h) + df_f2d(w1.l);
  }
}

// k_update_small_scale for any basis size (coefficients in dynamic shared memory, nq floats).
__global__ void __launch_bounds__(RT) k_update_small_scale_n(const double* __restrict__ V, size_t ld, int nq,
                                                             const double* __restrict__ c, double* __restrict__ w,
                                                             size_t len, const int* __restrict__ flag) {
  extern __shared__ float csn[];
  __shared__ double finv;
  const bool upd = flag == nullptr || *flag != 0;
  for (int q = threadIdx.x; q < nq; q += RT) csn[q] = (float)c[q];
  if (threadIdx.x == 0) {
    double s = 0.0;
    if (upd)
      for (int q = 0; q < nq; ++q) s = fma(c[q], c[q], s);
    const double b2 = c[nq] - s;
    finv = b2 > 0.0 || isnan(b2) ? 1.0 / sqrt(b2) : 0.0;
  }
  __syncthreads();
  const double f = finv;
  if (!upd) {
    for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) w[e] *= f;
    return;
  }
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) {
    float acc = 0.0f;
#pragma unroll 4
    for (int q = 0; q < nq; ++q) acc = fmaf(csn[q], hi_float(__ldg(V + (size_t)q * ld + e)), acc);
    w[e] = (w[e] - df_f2d(acc)) * f;
  }
}

// Blocks of kernel K that are resident at once on the device (at most RB): the sweeps below
// launch exactly one wave, so no partly filled second wave trails the memory stream.
template <auto K>
int wave_blocks() {
  static const int nb = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, RT, 0);
    const int n = per * sms;
    return n > 0 && n < RB ? n : RB;
  }();
  return nb;
}

// V_q and w start on 16-byte boundaries for every q
int aligned16(const double* V, size_t ld, const double* w) {
  return ((uintptr_t)V % 16 == 0) && (ld % 2 == 0) && ((uintptr_t)w % 16 == 0);
}

}  // namespace

int kv_reduce_blocks() { return RB; }

// out[r] = sum of partials[r * RB + b] over the nb blocks, r < rows (fixed order)
void kv_launch_finalize(const double* partials, int rows, int nb, double* out, cudaStream_t s) {
  k_finalize<<<rows, RT, 0, s>>>(partials, nb, out, 0);
}
int kv_fused_cgs_max() { return QF; }

void kv_launch_dots_norm(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                         double* h, double* nrm2, int df, cudaStream_t s) {
  const int nrm = nrm2 != nullptr;
  int nb = RB;
  const int vec = aligned16(V, ld, w);
  // one instantiation per basis size, so no predicated-off multiply-adds occupy the pipes
  if (df) {
    switch (nq) {
#define KV_DOTS_DF_CASE(Qn) \
  case Qn:                  \
    nb = wave_blocks<k_dots_df<Qn>>();                               \
    k_dots_df<Qn><<<nb, RT, 0, s>>>(V, ld, w, len, nrm, vec, partials); \
    break;
      KV_FOR_EACH_NQ(KV_DOTS_DF_CASE)
#undef KV_DOTS_DF_CASE
    }
  } else {
    switch (nq) {
#define KV_DOTS_CASE(Qn) \
  case Qn:               \
    nb = wave_blocks<k_dots<Qn>>();                                    \
    k_dots<Qn><<<nb, RT, 0, s>>>(V, ld, nq, w, len, nrm, partials); \
    break;
      KV_FOR_EACH_NQ(KV_DOTS_CASE)
#undef KV_DOTS_CASE
    }
  }
  k_finalize<<<nq + (nrm2 ? 1 : 0), RT, 0, s>>>(partials, nb, h, 0);  // h[nq] = ||w||^2 when asked
  if (nrm2 && nrm2 != h + nq) cudaMemcpyAsync(nrm2, h + nq, sizeof(double), cudaMemcpyDeviceToDevice, s);
}

void kv_launch_update_dot(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                          double* partials, double* h2, int df, cudaStream_t s) {
  int nb = RB;
  if (df) {
    switch (nq) {
#define KV_UPD_DF_CASE(Qn) \
  case Qn:                 \
    nb = wave_blocks<k_update_dot_df<Qn>>();                             \
    k_update_dot_df<Qn><<<nb, RT, 0, s>>>(V, ld, c, w, len, partials); \
    break;
      KV_FOR_EACH_NQ(KV_UPD_DF_CASE)
#undef KV_UPD_DF_CASE
    }
  } else {
    switch (nq) {
#define KV_UPD_CASE(Qn) \
  case Qn:              \
    nb = wave_blocks<k_update_dot<Qn>>();                                  \
    k_update_dot<Qn><<<nb, RT, 0, s>>>(V, ld, nq, c, w, len, partials); \
    break;
      KV_FOR_EACH_NQ(KV_UPD_CASE)
#undef KV_UPD_CASE
    }
  }
  k_finalize<<<nq + 1, RT, 0, s>>>(partials, nb, h2, 0);  // h2[nq] = ||w||^2 after the update
}

void kv_launch_gs_decide(const double* h1, const double* h2, int nq, double theta, int force, double* hcol,
                         int* flag, cudaStream_t s) {
  k_gs_decide<<<1, 1, 0, s>>>(h1, h2, nq, theta * theta, force, hcol, flag);
}

void kv_launch_update_small_scale(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                                  cudaStream_t s, const int* flag) {
  switch (nq) {
#define KV_SMALL_CASE(Qn) \
  case Qn:                \
    k_update_small_scale<Qn><<<wave_blocks<k_update_small_scale<Qn>>(), RT, 0, s>>>(V, ld, c, w, len, flag); \
    break;
    KV_FOR_EACH_NQ(KV_SMALL_CASE)
#undef KV_SMALL_CASE
  }
}

void kv_launch_dots_chunked(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                            double* h, int nrm, int df, cudaStream_t s) {
  // chunks of at most QF vectors, each one sweep over its vectors and w; ||w||^2 with the last
  for (int q0 = 0; q0 < nq; q0 += QF) {
    const int qc = nq - q0 < QF ? nq - q0 : QF;
    const bool last = q0 + qc == nq;
    kv_launch_dots_norm(V + (size_t)q0 * ld, ld, qc, w, len, partials, h + q0, (last && nrm) ? h + nq : nullptr, df,
                        s);
  }
}

void kv_launch_update_n(const double* V, size_t ld, int nq, const double* c, double* w, size_t len, int df,
                        cudaStream_t s) {
  if (!df) {
    kv_launch_update(V, ld, nq, c, w, len, s);
    return;
  }
  const int k64 = (3 * (nq + 2)) / 10;
  const size_t smem = (size_t)k64 * sizeof(double) + (size_t)(nq - k64) * sizeof(DF);
  k_update_n_df<<<wave_blocks<k_update_n_df>(), RT, smem, s>>>(V, ld, nq, k64, c, w, len);
}

void kv_launch_update_small_scale_n(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                                    cudaStream_t s, const int* flag) {
  k_update_small_scale_n<<<wave_blocks<k_update_small_scale_n>(), RT, (size_t)nq * sizeof(float), s>>>(V, ld, nq, c,
                                                                                                       w, len, flag);
}

void kv_launch_multidot(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                        double* out, int accumulate, cudaStream_t s) {
  const int nb = wave_blocks<k_multidot>();
  for (int q0 = 0; q0 < nq; q0 += QB) {
    const int nqb = nq - q0 < QB ? nq - q0 : QB;
    k_multidot<<<nb, RT, 0, s>>>(V, ld, q0, nqb, w, len, partials);
  }
  k_finalize<<<nq, RT, 0, s>>>(partials, nb, out, accumulate);
}

void kv_launch_update(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                      cudaStream_t s) {
  k_update<<<wave_blocks<k_update>(), RT, sizeof(double) * (size_t)nq, s>>>(V, ld, nq, c, w, len);
}

void kv_launch_norm2(const double* w, size_t len, double* partials, double* out, cudaStream_t s) {
  kv_launch_multidot(w, 0, 1, w, len, partials, out, 0, s);
}

