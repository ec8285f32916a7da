// FP64 reductions for the Arnoldi step: several inner products against one vector
// (classical Gram-Schmidt), the matching update, and the 2-norm. Partial sums per block are
// combined in a fixed order by a second kernel, so results are deterministic.
#include "kv_internal.cuh"

namespace {

constexpr int RB = 1216;  // reduction blocks: 8 per SM on 152 SMs
constexpr int RT = 256;   // threads per block
constexpr int QB = 8;     // inner products accumulated per sweep over the vector

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

}  // namespace

int kv_reduce_blocks() { return RB; }

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
