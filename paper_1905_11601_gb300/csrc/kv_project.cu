// Divergence and the fused velocity correction of the SIMPLE / Chorin step (Section 3.1):
// b = D v* on the cells; v = v* - G phi on the interior faces; p = phi; and the pointwise
// divergence residual max |D v| used as the SIMPLE stopping test.
#include "kv_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) k_divergence(KvGeom g, const double* __restrict__ vel, size_t P,
                                                    double* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  const int k = blockIdx.z + 1;
  if (i > g.nx || j > g.ny) return;
  const double* u = vel;
  const double* v = vel + P;
  const double* w = vel + 2 * P;
  const int e = i + g.X * (j + g.Y * k);
  const double d = (__ldg(u + e) - __ldg(u + e - 1)) * g.ihx + (__ldg(v + e) - __ldg(v + e - g.X)) * g.ihy +
                   (__ldg(w + e) - __ldg(w + e - g.X * g.Y)) * g.ihz;
  b[(i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1))] = d;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

struct Corr {
  KvGeom g;
  const double* __restrict__ vs;
  const double* __restrict__ phi;
  size_t P;
  __device__ __forceinline__ double ph(int i, int j, int k) const {  // padded cell index
    return __ldg(phi + (i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1)));
  }
  __device__ __forceinline__ int at(int i, int j, int k) const { return i + g.X * (j + g.Y * k); }
  __device__ __forceinline__ double u(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz)) return 0.0;
    return __ldg(vs + at(i, j, k)) - (ph(i + 1, j, k) - ph(i, j, k)) * g.ihx;
  }
  __device__ __forceinline__ double v(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz)) return 0.0;
    return __ldg(vs + P + at(i, j, k)) - (ph(i, j + 1, k) - ph(i, j, k)) * g.ihy;
  }
  __device__ __forceinline__ double w(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz - 1)) return 0.0;
    return __ldg(vs + 2 * P + at(i, j, k)) - (ph(i, j, k + 1) - ph(i, j, k)) * g.ihz;
  }
};

__global__ void __launch_bounds__(256) k_correct(KvGeom g, const double* __restrict__ vs,
                                                 const double* __restrict__ phi, size_t P,
                                                 double* __restrict__ out, double* __restrict__ p, int acc_p,
                                                 int check, unsigned long long* __restrict__ red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double dmax = 0.0, vmax = 0.0;
  if (i < g.X && j < g.Y) {
    Corr C{g, vs, phi, P};
    const int e = C.at(i, j, k);
    const double ur = C.u(i, j, k), vr = C.v(i, j, k), wr = C.w(i, j, k);
    out[e] = ur;
    out[P + e] = vr;
    out[2 * P + e] = wr;
    const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
    if (check) vmax = fmax(fabs(ur), fmax(fabs(vr), fabs(wr)));
    if (check && cell) {
      const double d = (ur - C.u(i - 1, j, k)) * g.ihx + (vr - C.v(i, j - 1, k)) * g.ihy + (wr - C.w(i, j, k - 1)) * g.ihz;
      dmax = fabs(d);
    }
    if (p) {
      if (cell)
        p[e] = (acc_p ? p[e] : 0.0) + C.ph(i, j, k);
      else if (!acc_p)
        p[e] = 0.0;
    }
  }
  if (!check) return;
  // block reduction of the two maxima, one atomic each per block
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  __shared__ double sd[8], sv[8];
  const int t = threadIdx.x + blockDim.x * threadIdx.y, warp = t >> 5, lane = t & 31;
  if (lane == 0) {
    sd[warp] = dmax;
    sv[warp] = vmax;
  }
  __syncthreads();
  if (t == 0) {
    double a = sd[0], b = sv[0];
    for (int q = 1; q < 8; ++q) {
      a = fmax(a, sd[q]);
      b = fmax(b, sv[q]);
    }
    atomic_max_nonneg(red, a);
    atomic_max_nonneg(red + 1, b);
  }
}

}  // namespace

void kv_launch_divergence(const kv_grid* h, const double* vel, double* b, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  k_divergence<<<grid, block, 0, s>>>(g, vel, h->P, b);
}

void kv_launch_correct(const kv_grid* h, const double* vstar, const double* phi, double* out_vel, double* p,
                       int accumulate_p, cudaStream_t s, int check) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  k_correct<<<grid, block, 0, s>>>(g, vstar, phi, h->P, out_vel, p, accumulate_p, check, h->red);
}
