// Divergence and the fused velocity correction of the SIMPLE / Chorin step (Section 3.1):
// b = D v* on the cells; v = v* - G phi on the interior faces; p = phi; and the pointwise
// divergence residual max |D v| used as the SIMPLE stopping test. FP64 on the uniform or the
// stretched grid (Eq 22), and for the mixed precision path (uniform grid) the same arithmetic
// in double-float on the FP32 pipe.
#include "kv_df.cuh"
#include "kv_internal.cuh"

namespace {

// 1 / width along axis A at padded index t: 1/h on the uniform grid; on a stretched grid
// (Eq 22) the table row ROW: KV_SW_IDC (cell widths, cells t = 1..n) or KV_SW_IDF (distances
// between adjacent cell centres, faces t = 1..n-1).
template <bool STR, int A, int ROW>
__device__ __forceinline__ double inv_w(const KvGeom& g, const KvStretch& S, int t) {
  const double ih = A == 0 ? g.ihx : (A == 1 ? g.ihy : g.ihz);
  if (!STR) return ih;
  const int L = (A == 0 ? g.nx : (A == 1 ? g.ny : g.nz)) + 2;
  return __ldg(S.sw + S.swo[A] + ROW * L + t);
}

template <bool STR>
__global__ void __launch_bounds__(256) k_divergence(KvGeom g, KvStretch S, const double* __restrict__ vel, size_t P,
                                                    double* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  const int k = blockIdx.z + 1;
  if (i > g.nx || j > g.ny) return;
  const double* u = vel;
  const double* v = vel + P;
  const double* w = vel + 2 * P;
  const int e = i + g.X * (j + g.Y * k);
  const double d = (__ldg(u + e) - __ldg(u + e - 1)) * inv_w<STR, 0, KV_SW_IDC>(g, S, i) +
                   (__ldg(v + e) - __ldg(v + e - g.X)) * inv_w<STR, 1, KV_SW_IDC>(g, S, j) +
                   (__ldg(w + e) - __ldg(w + e - g.X * g.Y)) * inv_w<STR, 2, KV_SW_IDC>(g, S, k);
  b[(i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1))] = d;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <bool STR>
struct Corr {
  KvGeom g;
  KvStretch S;
  const double* __restrict__ vs;
  const double* __restrict__ phi;
  size_t P;
  __device__ __forceinline__ double ph(int i, int j, int k) const {  // padded cell index
    return __ldg(phi + (i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1)));
  }
  __device__ __forceinline__ int at(int i, int j, int k) const { return i + g.X * (j + g.Y * k); }
  __device__ __forceinline__ double u(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz)) return 0.0;
    return __ldg(vs + at(i, j, k)) - (ph(i + 1, j, k) - ph(i, j, k)) * inv_w<STR, 0, KV_SW_IDF>(g, S, i);
  }
  __device__ __forceinline__ double v(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz)) return 0.0;
    return __ldg(vs + P + at(i, j, k)) - (ph(i, j + 1, k) - ph(i, j, k)) * inv_w<STR, 1, KV_SW_IDF>(g, S, j);
  }
  __device__ __forceinline__ double w(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz - 1)) return 0.0;
    return __ldg(vs + 2 * P + at(i, j, k)) - (ph(i, j, k + 1) - ph(i, j, k)) * inv_w<STR, 2, KV_SW_IDF>(g, S, k);
  }
};

template <bool STR>
__global__ void __launch_bounds__(256) k_correct(KvGeom g, KvStretch S, const double* __restrict__ vs,
                                                 const double* __restrict__ phi, size_t P,
                                                 double* __restrict__ out, double* __restrict__ p, int acc_p,
                                                 int check, unsigned long long* __restrict__ red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double dmax = 0.0, vmax = 0.0;
  if (i < g.X && j < g.Y) {
    Corr<STR> C{g, S, vs, phi, P};
    const int e = C.at(i, j, k);
    const double ur = C.u(i, j, k), vr = C.v(i, j, k), wr = C.w(i, j, k);
    out[e] = ur;
    out[P + e] = vr;
    out[2 * P + e] = wr;
    const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
    if (check) vmax = fmax(fabs(ur), fmax(fabs(vr), fabs(wr)));
    if (check && cell) {
      const double d = (ur - C.u(i - 1, j, k)) * inv_w<STR, 0, KV_SW_IDC>(g, S, i) +
                       (vr - C.v(i, j - 1, k)) * inv_w<STR, 1, KV_SW_IDC>(g, S, j) +
                       (wr - C.w(i, j, k - 1)) * inv_w<STR, 2, KV_SW_IDC>(g, S, k);
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

// ---- the same two kernels in double-float arithmetic (mixed precision; kv_df.cuh) ----------

// Inverse width along axis A at padded index t as an FP32 pair: the uniform pair u, or on a
// stretched grid (STR) row ROW of the KV_SWD_* tables.
template <bool STR, int A, int ROW>
__device__ __forceinline__ DF inv_w_df(const KvGeom& g, const KvStretch& S, int t, float2 u) {
  if (!STR) return DF{u.x, u.y};
  const int L = (A == 0 ? g.nx : (A == 1 ? g.ny : g.nz)) + 2;
  const float2 v = __ldg(S.swd + S.swdo[A] + ROW * L + t);
  return DF{v.x, v.y};
}

// b = D v* in double-float; with xs also b's three BF16 slices in the tensor-core solve's input
// layout [k][j][i_pad] (the first sweep's right-hand side)
template <bool STR>
__global__ void __launch_bounds__(256) k_divergence_df(KvGeom g, KvStretch S, const double* __restrict__ vel, size_t P,
                                                       double* __restrict__ b, float2 ihx, float2 ihy, float2 ihz,
                                                       __nv_bfloat16* __restrict__ xs, size_t slice, int pitch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  const int k = blockIdx.z + 1;
  if (i > g.nx || j > g.ny) return;
  const double* u = vel;
  const double* v = vel + P;
  const double* w = vel + 2 * P;
  const int e = i + g.X * (j + g.Y * k);
  const DF dx = df_mul(df_sub(df_split(__ldg(u + e)), df_split(__ldg(u + e - 1))),
                       inv_w_df<STR, 0, KV_SWD_IDC>(g, S, i, ihx));
  const DF dy = df_mul(df_sub(df_split(__ldg(v + e)), df_split(__ldg(v + e - g.X))),
                       inv_w_df<STR, 1, KV_SWD_IDC>(g, S, j, ihy));
  const DF dz = df_mul(df_sub(df_split(__ldg(w + e)), df_split(__ldg(w + e - g.X * g.Y))),
                       inv_w_df<STR, 2, KV_SWD_IDC>(g, S, k, ihz));
  const DF d = df_add(df_add(dx, dy), dz);
  b[(i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1))] = df_value(d);
  if (xs) kv_store_bf16x3(xs, slice, ((size_t)(k - 1) * g.ny + (j - 1)) * pitch + (i - 1), __fadd_rn(d.h, d.l));
}

template <bool STR>
struct CorrDF {
  KvGeom g;
  KvStretch S;
  const double* __restrict__ vs;
  const double* __restrict__ phi;
  size_t P;
  float2 ihx, ihy, ihz;
  __device__ __forceinline__ DF ph(int i, int j, int k) const {  // padded cell index
    return df_split(__ldg(phi + (i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1))));
  }
  __device__ __forceinline__ int at(int i, int j, int k) const { return i + g.X * (j + g.Y * k); }
  __device__ __forceinline__ DF u(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz)) return DF{0.0f, 0.0f};
    return df_sub(df_split(__ldg(vs + at(i, j, k))),
                  df_mul(df_sub(ph(i + 1, j, k), ph(i, j, k)), inv_w_df<STR, 0, KV_SWD_IDF>(g, S, i, ihx)));
  }
  __device__ __forceinline__ DF v(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx && j >= 1 && j <= g.ny - 1 && k >= 1 && k <= g.nz)) return DF{0.0f, 0.0f};
    return df_sub(df_split(__ldg(vs + P + at(i, j, k))),
                  df_mul(df_sub(ph(i, j + 1, k), ph(i, j, k)), inv_w_df<STR, 1, KV_SWD_IDF>(g, S, j, ihy)));
  }
  __device__ __forceinline__ DF w(int i, int j, int k) const {
    if (!(i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz - 1)) return DF{0.0f, 0.0f};
    return df_sub(df_split(__ldg(vs + 2 * P + at(i, j, k))),
                  df_mul(df_sub(ph(i, j, k + 1), ph(i, j, k)), inv_w_df<STR, 2, KV_SWD_IDF>(g, S, k, ihz)));
  }
};

__device__ __forceinline__ float df_abs_hi(const DF a) { return fabsf(__fadd_rn(a.h, a.l)); }

// CHECK = 0: the corrected faces and p only, each input loaded and split once, inverse spacings
// passed as FP32 pairs (ih). CHECK = 1 adds max |D v| and max |v| for the SIMPLE test.
template <int CHECK, bool STR>
__global__ void __launch_bounds__(256) k_correct_df(KvGeom g, KvStretch S, const double* __restrict__ vs,
                                                    const double* __restrict__ phi, size_t P,
                                                    double* __restrict__ out, double* __restrict__ p, int acc_p,
                                                    unsigned long long* __restrict__ red, float2 ihx, float2 ihy,
                                                    float2 ihz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double dmax = 0.0, vmax = 0.0;
  if (i < g.X && j < g.Y) {
    const int e = i + g.X * (j + g.Y * k);
    const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
    // interior faces (the wall-normal faces i = nx etc. stay 0)
    const bool du = cell && i <= g.nx - 1, dv = cell && j <= g.ny - 1, dw = cell && k <= g.nz - 1;
    const size_t c = (size_t)(i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1));
    const size_t cy = g.nx, cz = (size_t)g.nx * g.ny;
    const double p0d = cell ? __ldg(phi + c) : 0.0;
    const DF p0 = df_split(p0d);
    DF ur{0.0f, 0.0f}, vr{0.0f, 0.0f}, wr{0.0f, 0.0f};
    if (du)
      ur = df_sub(df_split(__ldg(vs + e)),
                  df_mul(df_sub(df_split(__ldg(phi + c + 1)), p0), inv_w_df<STR, 0, KV_SWD_IDF>(g, S, i, ihx)));
    if (dv)
      vr = df_sub(df_split(__ldg(vs + P + e)),
                  df_mul(df_sub(df_split(__ldg(phi + c + cy)), p0), inv_w_df<STR, 1, KV_SWD_IDF>(g, S, j, ihy)));
    if (dw)
      wr = df_sub(df_split(__ldg(vs + 2 * P + e)),
                  df_mul(df_sub(df_split(__ldg(phi + c + cz)), p0), inv_w_df<STR, 2, KV_SWD_IDF>(g, S, k, ihz)));
    out[e] = df_value(ur);
    out[P + e] = df_value(vr);
    out[2 * P + e] = df_value(wr);
    if (CHECK) {
      vmax = (double)fmaxf(df_abs_hi(ur), fmaxf(df_abs_hi(vr), df_abs_hi(wr)));
      if (cell) {
        const CorrDF<STR> C{g, S, vs, phi, P, ihx, ihy, ihz};
        const DF d = df_add(df_add(df_mul(df_sub(ur, C.u(i - 1, j, k)), inv_w_df<STR, 0, KV_SWD_IDC>(g, S, i, ihx)),
                                   df_mul(df_sub(vr, C.v(i, j - 1, k)), inv_w_df<STR, 1, KV_SWD_IDC>(g, S, j, ihy))),
                            df_mul(df_sub(wr, C.w(i, j, k - 1)), inv_w_df<STR, 2, KV_SWD_IDC>(g, S, k, ihz)));
        dmax = fabs(df_value(d));
      }
    }
    if (p) {
      if (cell)
        p[e] = (acc_p ? p[e] : 0.0) + p0d;
      else if (!acc_p)
        p[e] = 0.0;
    }
  }
  if (!CHECK) return;
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

// x as an FP32 pair (host side)
float2 pair_of(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

}  // namespace

void kv_launch_divergence(const kv_grid* h, const double* vel, double* b, cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  const bool str = h->str.sw != nullptr;
  if (h->d.precision == KV_PREC_MIXED) {
    auto kern = str ? k_divergence_df<true> : k_divergence_df<false>;
    kern<<<grid, block, 0, s>>>(g, h->str, vel, h->P, b, pair_of(g.ihx), pair_of(g.ihy), pair_of(g.ihz), h->xs[0],
                                h->xs_slice, (g.nx + 7) & ~7);
  } else {
    auto kern = str ? k_divergence<true> : k_divergence<false>;
    kern<<<grid, block, 0, s>>>(g, h->str, vel, h->P, b);
  }
}

void kv_launch_correct(const kv_grid* h, const double* vstar, const double* phi, double* out_vel, double* p,
                       int accumulate_p, cudaStream_t s, int check) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.X + 31) / 32, (g.Y + 7) / 8, g.Z);
  const bool str = h->str.sw != nullptr;
  if (h->d.precision == KV_PREC_MIXED) {
    const float2 cx = pair_of(g.ihx), cy = pair_of(g.ihy), cz = pair_of(g.ihz);
    auto kern = str ? (check ? k_correct_df<1, true> : k_correct_df<0, true>)
                    : (check ? k_correct_df<1, false> : k_correct_df<0, false>);
    kern<<<grid, block, 0, s>>>(g, h->str, vstar, phi, h->P, out_vel, p, accumulate_p, h->red, cx, cy, cz);
  } else {
    auto kern = str ? k_correct<true> : k_correct<false>;
    kern<<<grid, block, 0, s>>>(g, h->str, vstar, phi, h->P, out_vel, p, accumulate_p, check, h->red);
  }
}
