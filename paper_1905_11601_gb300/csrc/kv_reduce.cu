// FP64 reductions for the Arnoldi step: several inner products against one vector
// (classical Gram-Schmidt), the matching update, and the 2-norm. Partial sums per block are
// combined in a fixed order by a second kernel, so results are deterministic.
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
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)RB * RT) {
    const double we = __ldg(w + e);
#pragma unroll
    for (int q = 0; q < QB; ++q)
      if (q < nqb) acc[q] = fma(__ldg(V + (size_t)(q0 + q) * ld + e), we, acc[q]);
  }
  __shared__ double sm[QB][RT / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    const double s = warp_sum(acc[q]);
    if (lane == 0) sm[q][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < QB && (int)threadIdx.x < nqb) {
    double s = 0.0;
    for (int wv = 0; wv < RT / 32; ++wv) s += sm[threadIdx.x][wv];
    partials[(size_t)(q0 + threadIdx.x) * RB + blockIdx.x] = s;
  }
}

// out[q] (+)= sum_b partials[q * RB + b]; one block per q
__global__ void __launch_bounds__(RT) k_finalize(const double* __restrict__ partials, double* __restrict__ out,
                                                 int accumulate) {
  const int q = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < RB; b += RT) s += partials[(size_t)q * RB + b];
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

__global__ void __launch_bounds__(RT) k_scale_inv_sqrt(double* __restrict__ w, size_t len,
                                                       const double* __restrict__ nrm2) {
  const double n2 = *nrm2;
  const double f = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)gridDim.x * RT) w[e] *= f;
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
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)RB * RT) {
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
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)RB * RT) {
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
__global__ void __launch_bounds__(RT) k_update_small_scale(const double* __restrict__ V, size_t ld, int nq,
                                                           const double* __restrict__ c, double* __restrict__ w,
                                                           size_t len) {
  __shared__ float cs[QF];
  __shared__ double finv;
  if (threadIdx.x < QF) cs[threadIdx.x] = (int)threadIdx.x < nq ? (float)c[threadIdx.x] : 0.0f;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s = fma(c[q], c[q], s);
    const double b2 = c[nq] - s;
    finv = b2 > 0.0 ? 1.0 / sqrt(b2) : 0.0;
  }
  __syncthreads();
  const double f = finv;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < len; e += (size_t)RB * RT) {
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < QF; ++q)
      if (q < nq) s = fmaf(cs[q], hi_float(__ldg(V + (size_t)q * ld + e)), s);
    w[e] = (w[e] - (double)s) * f;
  }
}

}  // namespace

int kv_reduce_blocks() { return RB; }
int kv_fused_cgs_max() { return QF; }

void kv_launch_dots_norm(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                         double* h, double* nrm2, cudaStream_t s) {
  const int nrm = nrm2 != nullptr;
  // one instantiation per basis size, so no predicated-off multiply-adds occupy the FP64 pipe
  switch (nq) {
#define KV_DOTS_CASE(Qn) \
  case Qn:               \
    k_dots<Qn><<<RB, RT, 0, s>>>(V, ld, nq, w, len, nrm, partials); \
    break;
    KV_FOR_EACH_NQ(KV_DOTS_CASE)
#undef KV_DOTS_CASE
  }
  k_finalize<<<nq + (nrm2 ? 1 : 0), RT, 0, s>>>(partials, h, 0);  // h[nq] = ||w||^2 when asked
  if (nrm2 && nrm2 != h + nq) cudaMemcpyAsync(nrm2, h + nq, sizeof(double), cudaMemcpyDeviceToDevice, s);
}

void kv_launch_update_dot(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                          double* partials, double* h2, cudaStream_t s) {
  switch (nq) {
#define KV_UPD_CASE(Qn) \
  case Qn:              \
    k_update_dot<Qn><<<RB, RT, 0, s>>>(V, ld, nq, c, w, len, partials); \
    break;
    KV_FOR_EACH_NQ(KV_UPD_CASE)
#undef KV_UPD_CASE
  }
  k_finalize<<<nq + 1, RT, 0, s>>>(partials, h2, 0);  // h2[nq] = ||w||^2 after the update
}

void kv_launch_update_small_scale(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                                  cudaStream_t s) {
  k_update_small_scale<<<RB, RT, 0, s>>>(V, ld, nq, c, w, len);
}

void kv_launch_multidot(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                        double* out, int accumulate, cudaStream_t s) {
  for (int q0 = 0; q0 < nq; q0 += QB) {
    const int nqb = nq - q0 < QB ? nq - q0 : QB;
    k_multidot<<<RB, RT, 0, s>>>(V, ld, q0, nqb, w, len, partials);
  }
  k_finalize<<<nq, RT, 0, s>>>(partials, out, accumulate);
}

void kv_launch_update(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                      cudaStream_t s) {
  k_update<<<RB, RT, sizeof(double) * (size_t)nq, s>>>(V, ld, nq, c, w, len);
}

void kv_launch_norm2(const double* w, size_t len, double* partials, double* out, cudaStream_t s) {
  kv_launch_multidot(w, 0, 1, w, len, partials, out, 0, s);
}

void kv_launch_scale_inv_sqrt(double* w, size_t len, const double* nrm2, cudaStream_t s) {
  k_scale_inv_sqrt<<<RB, RT, 0, s>>>(w, len, nrm2);
}
