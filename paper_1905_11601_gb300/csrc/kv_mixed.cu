// Mixed-precision pressure-correction solve: phi = L^+ b (Eqs (14)-(18)) with the six per-axis
// contractions on the tensor cores (BF16 slices, FP32 accumulation; kv_umma.cu), won back to
// FP64-class accuracy by iterative refinement with a double-float residual:
//
//   phi = 0;  r = b   (the divergence writes r's slices; the first sweep stores phi, as FP32)
//   repeat S times:  phi += TPF(r)   (six tcgen05 contractions, the last one adds into phi)
//                    r = b - L phi   (7-point Neumann Laplacian in double-float, written as BF16 slices;
//                                     per-cell weights on a stretched grid, Eq (22))
//
// Each sweep reduces the error by roughly the FP32 accuracy of one tensor-core solve.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kv_df.cuh"
#include "kv_internal.cuh"

namespace {

int pad8(int n) { return (n + 7) & ~7; }

// r = b - L phi (L = D G with homogeneous Neumann walls) in double-float arithmetic on the FP32
// pipe (kv_df.cuh; about 2^-44 of |b| + |L phi|, far below what one tensor-core sweep resolves),
// then three BF16 slices of r into the first contraction's input layout [k][j][i_pad]. PhiT:
// float for phi after the first sweep (exact FP32 values, no split needed), double after
// later sweeps. With rmax, max |r| is reduced per block into *rmax.
__device__ __forceinline__ DF phi_pair(float x) { return DF{x, 0.0f}; }
__device__ __forceinline__ DF phi_pair(double x) { return df_split(x); }

// STR (stretched grid): along each axis L phi = LWP (phi+ - phi) + LWM (phi- - phi) with the
// KV_SWD_* weights of the cell (a wall neighbour contributes zero flux).
template <int A>
__device__ __forceinline__ DF lap_weight(const KvGeom& g, const KvStretch& S, int row, int t) {
  const int L = (A == 0 ? g.nx : (A == 1 ? g.ny : g.nz)) + 2;
  const float2 v = __ldg(S.swd + S.swdo[A] + row * L + t);
  return DF{v.x, v.y};
}

template <typename PhiT, bool STR>
__global__ void __launch_bounds__(256) k_residual_slices(KvGeom g, KvStretch S, const double* __restrict__ b,
                                                         const PhiT* __restrict__ phi, __nv_bfloat16* __restrict__ xs,
                                                         size_t slice, int pitch, unsigned long long* rmax,
                                                         float2 ihx2, float2 ihy2, float2 ihz2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  float rv = 0.0f;
  if (i < g.nx && j < g.ny) {
    const size_t sx = 1, sy = g.nx, sz = (size_t)g.nx * g.ny;
    const size_t e = i + sy * j + sz * k;
    // homogeneous Neumann walls: a missing neighbour contributes as the cell itself
    const PhiT cv = __ldg(phi + e);
    const DF c = phi_pair(cv);
    const DF c2 = DF{2.0f * c.h, 2.0f * c.l};  // exact
    const DF xm = phi_pair(i > 0 ? __ldg(phi + e - sx) : cv), xp = phi_pair(i < g.nx - 1 ? __ldg(phi + e + sx) : cv);
    const DF ym = phi_pair(j > 0 ? __ldg(phi + e - sy) : cv), yp = phi_pair(j < g.ny - 1 ? __ldg(phi + e + sy) : cv);
    const DF zm = phi_pair(k > 0 ? __ldg(phi + e - sz) : cv), zp = phi_pair(k < g.nz - 1 ? __ldg(phi + e + sz) : cv);
    DF lx, ly, lz;
    if (STR) {  // padded cell index t = compact index + 1
      lx = df_add(df_mul(df_sub(xp, c), lap_weight<0>(g, S, KV_SWD_LWP, i + 1)),
                  df_mul(df_sub(xm, c), lap_weight<0>(g, S, KV_SWD_LWM, i + 1)));
      ly = df_add(df_mul(df_sub(yp, c), lap_weight<1>(g, S, KV_SWD_LWP, j + 1)),
                  df_mul(df_sub(ym, c), lap_weight<1>(g, S, KV_SWD_LWM, j + 1)));
      lz = df_add(df_mul(df_sub(zp, c), lap_weight<2>(g, S, KV_SWD_LWP, k + 1)),
                  df_mul(df_sub(zm, c), lap_weight<2>(g, S, KV_SWD_LWM, k + 1)));
    } else {
      lx = df_mul(df_sub(df_add(xm, xp), c2), DF{ihx2.x, ihx2.y});
      ly = df_mul(df_sub(df_add(ym, yp), c2), DF{ihy2.x, ihy2.y});
      lz = df_mul(df_sub(df_add(zm, zp), c2), DF{ihz2.x, ihz2.y});
    }
    const DF r = df_sub(df_split(__ldg(b + e)), df_add(df_add(lx, ly), lz));
    const float rf = __fadd_rn(r.h, r.l);
    rv = fabsf(rf);
    kv_store_bf16x3(xs, slice, ((size_t)k * g.ny + j) * pitch + i, rf);
  }
  if (rmax) {
    for (int off = 16; off > 0; off >>= 1) rv = fmaxf(rv, __shfl_xor_sync(0xffffffffu, rv, off));
    __shared__ float sm[32];
    const int t = threadIdx.x + blockDim.x * threadIdx.y, nw = (blockDim.x * blockDim.y + 31) / 32;
    if ((t & 31) == 0) sm[t >> 5] = rv;
    __syncthreads();
    if (t == 0) {
      float m = sm[0];
      for (int q = 1; q < nw; ++q) m = fmaxf(m, sm[q]);
      atomicMax(rmax, (unsigned long long)__double_as_longlong(df_f2d(m)));
    }
  }
}

// b's three BF16 slices (the first sweep's right-hand side, r = b)
__global__ void __launch_bounds__(256) k_rhs_slices(KvGeom g, const double* __restrict__ b,
                                                    __nv_bfloat16* __restrict__ xs, size_t slice, int pitch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const DF r = df_split(__ldg(b + i + (size_t)g.nx * (j + (size_t)g.ny * k)));
  kv_store_bf16x3(xs, slice, ((size_t)k * g.ny + j) * pitch + i, __fadd_rn(r.h, r.l));
}

float2 host_pair(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// Three BF16 slices of an M x K FP64 matrix, rows padded to pitch (zero padding).
void split_matrix(const double* W, int M, int K, std::vector<__nv_bfloat16>& out) {
  const int pitch = pad8(K);
  const size_t slice = (size_t)M * pitch;
  out.assign(3 * slice, __float2bfloat16(0.0f));
  for (int m = 0; m < M; ++m)
    for (int k = 0; k < K; ++k) {
      double rem = W[(size_t)m * K + k];
      for (int s = 0; s < 3; ++s) {
        const __nv_bfloat16 v = __float2bfloat16_rn((float)rem);
        out[s * slice + (size_t)m * pitch + k] = v;
        rem -= (double)__bfloat162float(v);
      }
    }
}

struct PassSpec {
  int axis;  // contracted axis (0 = x, 1 = y, 2 = z)
  int a, b;  // axes of the output column index r = a * n_b + b
};
// forward x, y, z then inverse x, y, z; see kv_tpd.cu for the rotation of the axes
const PassSpec kPass[6] = {{0, 2, 1}, {1, 0, 2}, {2, 1, 0}, {0, 2, 1}, {1, 0, 2}, {2, 1, 0}};

}  // namespace

kv_status kv_mixed_setup(kv_grid* h, const double* const fwd[3], const double* const inv[3]) {
  const int n[3] = {h->g.nx, h->g.ny, h->g.nz};
  h->refine = h->d.refine_sweeps > 0 ? h->d.refine_sweeps : 2;
  // data slice buffers: the largest of the six layouts (rows x padded fastest extent)
  size_t cap = 0;
  for (int a = 0; a < 3; ++a) cap = std::max(cap, h->Nc / n[a] * (size_t)pad8(n[a]));
  h->xs_slice = cap;
  cudaError_t e;
  for (int q = 0; q < 2; ++q)
    if ((e = cudaMalloc(&h->xs[q], 3 * cap * sizeof(__nv_bfloat16))) != cudaSuccess) goto fail;
  for (int p = 0; p < 6; ++p) {
    const int a = kPass[p].axis;
    const double* W = p < 3 ? fwd[a] : inv[a];
    std::vector<__nv_bfloat16> sl;
    split_matrix(W, n[a], n[a], sl);
    if ((e = cudaMalloc(&h->wsl[p], sl.size() * sizeof(__nv_bfloat16))) != cudaSuccess) goto fail;
    if ((e = cudaMemcpy(h->wsl[p], sl.data(), sl.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      goto fail;
  }
  for (int a = 0; a < 3; ++a) {
    std::vector<double> lam(n[a]);
    if ((e = cudaMemcpy(lam.data(), h->lam[a], n[a] * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
      goto fail;
    std::vector<float> lf(lam.begin(), lam.end());
    if ((e = cudaMalloc(&h->lamf[a], n[a] * sizeof(float))) != cudaSuccess) goto fail;
    if ((e = cudaMemcpy(h->lamf[a], lf.data(), n[a] * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) goto fail;
  }
  if ((e = kv_umma_init()) != cudaSuccess) goto fail;
  if ((e = cudaMalloc(&h->derr, sizeof(unsigned int))) != cudaSuccess) goto fail;
  if ((e = cudaMemset(h->derr, 0, sizeof(unsigned int))) != cudaSuccess) goto fail;
  if ((e = cudaMalloc(&h->rmax, sizeof(unsigned long long))) != cudaSuccess) goto fail;
  if ((e = cudaMalloc(&h->phi32, h->Nc * sizeof(float))) != cudaSuccess) goto fail;
  for (int p = 0; p < 6; ++p) {
    const int a = kPass[p].axis;
    const int K = n[a], M = n[a];
    const int R = (int)(h->Nc / n[a]);
    const __nv_bfloat16* in = h->xs[p % 2];
    if (!kv_make_slice_map(&h->mapA[p], h->wsl[p], K, M, pad8(K), (size_t)M * pad8(K), kv_umma_box_rows_a()) ||
        !kv_make_data_map(&h->mapB[p], in, K, R, pad8(K), 1, h->xs_slice, h->xs_slice, kv_umma_box_rows_b()) ||
        !kv_make_data_map(&h->mapB128[p], in, K, R, pad8(K), 1, h->xs_slice, h->xs_slice, 128)) {
      h->err = "cuTensorMapEncodeTiled failed";
      return KV_ERR_CUDA;
    }
  }
  return KV_OK;
fail:
  h->err = std::string("mixed-precision set-up: ") + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? KV_ERR_NOMEM : KV_ERR_CUDA;
}

void kv_mixed_free(kv_grid* h) {
  for (int q = 0; q < 2; ++q) cudaFree(h->xs[q]);
  for (int p = 0; p < 6; ++p) cudaFree(h->wsl[p]);
  for (int a = 0; a < 3; ++a) cudaFree(h->lamf[a]);
  cudaFree(h->derr);
  cudaFree(h->rmax);
  cudaFree(h->phi32);
  kv_mixed_block_free(h);
}

void kv_mixed_block_free(kv_grid* h) {
  cudaFree(h->blk_vstar);
  cudaFree(h->blk_b);
  cudaFree(h->blk_phi);
  cudaFree(h->blk_phi32);
  for (int q = 0; q < 2; ++q) cudaFree(h->blk_xs[q]);
  h->blk_vstar = h->blk_b = h->blk_phi = nullptr;
  h->blk_phi32 = nullptr;
  h->blk_xs[0] = h->blk_xs[1] = nullptr;
  h->blk_cap = 0;
}

kv_status kv_mixed_block_setup(kv_grid* h, int cap) {
  if (h->blk_cap >= cap) return KV_OK;
  kv_mixed_block_free(h);
  const int n[3] = {h->g.nx, h->g.ny, h->g.nz};
  const size_t xsb = (size_t)3 * cap * h->xs_slice;
  cudaError_t e;
  if ((e = cudaMalloc(&h->blk_vstar, (size_t)cap * 3 * h->P * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->blk_b, (size_t)cap * h->Nc * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->blk_phi, (size_t)cap * h->Nc * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->blk_phi32, (size_t)cap * h->Nc * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&h->blk_xs[0], xsb * sizeof(__nv_bfloat16))) != cudaSuccess ||
      (e = cudaMalloc(&h->blk_xs[1], xsb * sizeof(__nv_bfloat16))) != cudaSuccess) {
    kv_mixed_block_free(h);
    h->err = std::string("block buffers: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? KV_ERR_NOMEM : KV_ERR_CUDA;
  }
  for (int p = 0; p < 6; ++p) {
    const int a = kPass[p].axis;
    const int K = n[a];
    const int R = (int)(h->Nc / n[a]);
    if (!kv_make_data_map(&h->blk_mapB[p], h->blk_xs[p % 2], K, R, pad8(K), cap, h->xs_slice,
                          (size_t)cap * h->xs_slice, kv_umma_box_rows_b()) ||
        !kv_make_data_map(&h->blk_mapB128[p], h->blk_xs[p % 2], K, R, pad8(K), cap, h->xs_slice,
                          (size_t)cap * h->xs_slice, 128)) {
      kv_mixed_block_free(h);
      h->err = "cuTensorMapEncodeTiled failed (block maps)";
      return KV_ERR_CUDA;
    }
  }
  h->blk_cap = cap;
  return KV_OK;
}

void kv_launch_poisson_mixed(kv_grid* h, const double* b, double* phi, int stats, int slices_ready, cudaStream_t s) {
  const KvGeom& g = h->g;
  const int n[3] = {g.nx, g.ny, g.nz};
  dim3 rb(32, 8, 1), rg((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  if (stats) cudaMemsetAsync(h->rmax, 0, sizeof(unsigned long long), s);
  if (!slices_ready) {
    KvPhase ph(h, KV_PH_REFINE, 1);
    k_rhs_slices<<<rg, rb, 0, s>>>(g, b, h->xs[0], h->xs_slice, pad8(g.nx));
  }
  const float2 cx = host_pair(g.ihx2), cy = host_pair(g.ihy2), cz = host_pair(g.ihz2);
  for (int sweep = 0; sweep < h->refine; ++sweep) {
    for (int p = 0; p < 6; ++p) {
      const PassSpec& ps = kPass[p];
      KvUmmaEpi ep{};
      ep.M = n[ps.axis];
      ep.R = (int)(h->Nc / n[ps.axis]);
      ep.na = n[ps.a];
      ep.nb = n[ps.b];
      ep.pitch = pad8(n[ps.b]);
      ep.slice = h->xs_slice;
      ep.out = h->xs[(p + 1) % 2];
      // the last contraction writes phi: the first of several sweeps as exact FP32 values (the
      // residual then reads 4-byte values it need not split), the second as phi32 + D in FP64,
      // later ones by adding; a single sweep stores FP64 directly
      const bool single = h->refine == 1;
      ep.mode = (p == 2) ? 1 : (p == 5 ? (sweep == 0 ? (single ? 3 : 4) : (sweep == 1 ? 5 : 2)) : 0);
      ep.phi = phi;
      ep.phi32 = h->phi32;
      ep.lz = h->lamf[ps.axis];
      ep.la = h->lamf[ps.a];
      ep.lb = h->lamf[ps.b];
      KvPhase ph(h, KV_PH_TPD, 1);
      const bool t128 = h->umma_tile == 128;
      kv_launch_umma_axis(&h->mapA[p], t128 ? &h->mapB128[p] : &h->mapB[p], n[ps.axis], ep, h->derr, s,
                          h->umma_tile);
    }
    if (sweep + 1 < h->refine) {
      KvPhase ph(h, KV_PH_REFINE, 1);
      unsigned long long* rm = stats ? h->rmax : nullptr;
      const bool str = h->str.sw != nullptr;
      if (sweep == 0) {
        auto kern = str ? k_residual_slices<float, true> : k_residual_slices<float, false>;
        kern<<<rg, rb, 0, s>>>(g, h->str, b, h->phi32, h->xs[0], h->xs_slice, pad8(g.nx), rm, cx, cy, cz);
      } else {
        auto kern = str ? k_residual_slices<double, true> : k_residual_slices<double, false>;
        kern<<<rg, rb, 0, s>>>(g, h->str, b, phi, h->xs[0], h->xs_slice, pad8(g.nx), rm, cx, cy, cz);
      }
    }
  }
}

void kv_launch_poisson_mixed_block(kv_grid* h, int nb, cudaStream_t s) {
  const KvGeom& g = h->g;
  const int n[3] = {g.nx, g.ny, g.nz};
  const size_t bslice = (size_t)h->blk_cap * h->xs_slice;  // elements between slices of the block buffers
  dim3 rb(32, 8, 1), rg((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  const float2 cx = host_pair(g.ihx2), cy = host_pair(g.ihy2), cz = host_pair(g.ihz2);
  const bool str = h->str.sw != nullptr;
  for (int sweep = 0; sweep < h->refine; ++sweep) {
    for (int p = 0; p < 6; ++p) {
      const PassSpec& ps = kPass[p];
      KvUmmaEpi ep{};
      ep.M = n[ps.axis];
      ep.R = (int)(h->Nc / n[ps.axis]);
      ep.na = n[ps.a];
      ep.nb = n[ps.b];
      ep.pitch = pad8(n[ps.b]);
      ep.slice = bslice;
      ep.out = h->blk_xs[(p + 1) % 2];
      const bool single = h->refine == 1;
      ep.mode = (p == 2) ? 1 : (p == 5 ? (sweep == 0 ? (single ? 3 : 4) : (sweep == 1 ? 5 : 2)) : 0);
      ep.phi = h->blk_phi;
      ep.phi32 = h->blk_phi32;
      ep.lz = h->lamf[ps.axis];
      ep.la = h->lamf[ps.a];
      ep.lb = h->lamf[ps.b];
      ep.nvec = nb;
      ep.vstride_out = h->xs_slice;
      ep.vstride_phi = h->Nc;
      KvPhase ph(h, KV_PH_TPD, 1);
      // the single-vector path's tile width, so that a block equals single calls bit for bit
      const bool t128 = h->umma_tile == 128;
      kv_launch_umma_axis(&h->mapA[p], t128 ? &h->blk_mapB128[p] : &h->blk_mapB[p], n[ps.axis], ep, h->derr, s,
                          h->umma_tile);
    }
    if (sweep + 1 < h->refine) {
      KvPhase ph(h, KV_PH_REFINE, nb);
      for (int v = 0; v < nb; ++v) {
        const double* b = h->blk_b + (size_t)v * h->Nc;
        __nv_bfloat16* xs = h->blk_xs[0] + (size_t)v * h->xs_slice;
        if (sweep == 0) {
          auto kern = str ? k_residual_slices<float, true> : k_residual_slices<float, false>;
          kern<<<rg, rb, 0, s>>>(g, h->str, b, h->blk_phi32 + (size_t)v * h->Nc, xs, bslice, pad8(g.nx), nullptr, cx,
                                 cy, cz);
        } else {
          auto kern = str ? k_residual_slices<double, true> : k_residual_slices<double, false>;
          kern<<<rg, rb, 0, s>>>(g, h->str, b, h->blk_phi + (size_t)v * h->Nc, xs, bslice, pad8(g.nx), nullptr, cx,
                                 cy, cz);
        }
      }
    }
  }
}

// Failure-detection self-test (no GPU fault): one contraction whose barriers expect 16 bytes
// more than the copies deliver, so the bounded waits expire after a few hundred tries; the
// kernel sets the device error flag and returns. Reads and clears the flag.
kv_status kv_mixed_selftest_timeout(kv_grid* h, int* device_error) {
  const int n[3] = {h->g.nx, h->g.ny, h->g.nz};
  const PassSpec& ps = kPass[0];
  KvUmmaEpi ep{};
  ep.M = n[ps.axis];
  ep.R = (int)(h->Nc / n[ps.axis]);
  ep.na = n[ps.a];
  ep.nb = n[ps.b];
  ep.pitch = pad8(n[ps.b]);
  ep.slice = h->xs_slice;
  ep.out = h->xs[1];
  ep.mode = 0;
  ep.wait_limit = 256;
  ep.extra_tx = 16;
  cudaError_t e = cudaMemsetAsync(h->derr, 0, sizeof(unsigned int), h->s);
  if (e == cudaSuccess) e = kv_launch_umma_axis(&h->mapA[0], &h->mapB[0], n[ps.axis], ep, h->derr, h->s);
  unsigned int de = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&de, h->derr, sizeof de, cudaMemcpyDeviceToHost, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->derr, 0, sizeof(unsigned int), h->s);
  if (e != cudaSuccess) {
    h->err = std::string("self-test: ") + cudaGetErrorString(e);
    return KV_ERR_CUDA;
  }
  *device_error = (int)de;
  return KV_OK;
}
