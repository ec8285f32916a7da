// Tensor-product factorisation (TPF) Poisson solve of Eqs (14)-(18) for the SIMPLE pressure
// correction: phi = (E_x (x) E_y (x) E_z) Lambda^-1 (E_x^-1 (x) E_y^-1 (x) E_z^-1) b with the
// Neumann zero mode dropped. Each factor is one dense contraction along one axis of the
// n^3 array; every pass contracts the fastest axis and writes its output with the axes
// rotated (contracted axis slowest), so after three passes the array is back in (z, y, x)
// order and every pass reads and writes contiguously.
#include "kv_internal.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

struct ScaleInfo {
  const double* lx;  // eigenvalues per axis (Eq 15)
  const double* ly;
  const double* lz;
  int nx;            // r = my * nx + mx in the third forward pass
};

// D[m][r] = sum_a W[m][a] * X[r][a]   (W: M x K, X: R x K, D: M x R, all row-major)
// SCALE: D[m][r] /= lz[m] + ly[r / nx] + lx[r % nx] (Eq 17), zero mode set to 0.
template <bool SCALE>
__global__ void __launch_bounds__(256) k_gemm_axis(int M, int R, int K, const double* __restrict__ W,
                                                   const double* __restrict__ X, double* __restrict__ D,
                                                   ScaleInfo si) {
  __shared__ double Ws[BK][BM + 1];
  __shared__ double Xs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, r0 = blockIdx.x * BN;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = threadIdx.x + 256 * q;
      const int row = idx >> 4, kk = idx & 15;
      const int gk = k0 + kk;
      Ws[kk][row] = (m0 + row < M && gk < K) ? __ldg(W + (size_t)(m0 + row) * K + gk) : 0.0;
      Xs[kk][row] = (r0 + row < R && gk < K) ? __ldg(X + (size_t)(r0 + row) * K + gk) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = Ws[kk][ty + 16 * q];
        b[q] = Xs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int m = m0 + ty + 16 * p;
    if (m >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + tx + 16 * q;
      if (r >= R) continue;
      double v = acc[p][q];
      if (SCALE) {
        const int my = r / si.nx, mx = r - my * si.nx;
        const double lam = si.lz[m] + si.ly[my] + si.lx[mx];
        v = (m == 0 && r == 0) ? 0.0 : v / lam;
      }
      D[(size_t)m * R + r] = v;
    }
  }
}

void gemm_axis(int M, int R, int K, const double* W, const double* X, double* D, bool scale, ScaleInfo si,
               cudaStream_t s) {
  dim3 grid((R + BN - 1) / BN, (M + BM - 1) / BM);
  if (scale)
    k_gemm_axis<true><<<grid, 256, 0, s>>>(M, R, K, W, X, D, si);
  else
    k_gemm_axis<false><<<grid, 256, 0, s>>>(M, R, K, W, X, D, si);
}

}  // namespace

void kv_launch_poisson(kv_grid* h, double* b, double* phi, cudaStream_t s) {
  const int nx = h->g.nx, ny = h->g.ny, nz = h->g.nz;
  double* t = h->tpd_b;
  ScaleInfo none{nullptr, nullptr, nullptr, 1};
  ScaleInfo sc{h->lam[0], h->lam[1], h->lam[2], nx};
  // forward: b[k][j][i] -> [mx][k][j] -> [my][mx][k] -> [mz][my][mx] (scaled)
  { KvPhase ph(h, KV_PH_TPD, 1); gemm_axis(nx, nz * ny, nx, h->Wm[0], b, t, false, none, s); }
  { KvPhase ph(h, KV_PH_TPD, 1); gemm_axis(ny, nx * nz, ny, h->Wm[1], t, b, false, none, s); }
  { KvPhase ph(h, KV_PH_TPD, 1); gemm_axis(nz, ny * nx, nz, h->Wm[2], b, t, true, sc, s); }
  // inverse: [mz][my][mx] -> [i][mz][my] -> [j][i][mz] -> [k][j][i]
  { KvPhase ph(h, KV_PH_TPD, 1); gemm_axis(nx, nz * ny, nx, h->Wm[3], t, b, false, none, s); }
  { KvPhase ph(h, KV_PH_TPD, 1); gemm_axis(ny, nx * nz, ny, h->Wm[4], b, t, false, none, s); }
  { KvPhase ph(h, KV_PH_TPD, 1); gemm_axis(nz, ny * nx, nz, h->Wm[5], t, phi, false, none, s); }
}
