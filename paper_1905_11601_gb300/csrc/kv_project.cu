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

// |v| as the bit pattern of a non-negative double: these order like the values, with +Inf above
// every finite value and NaN above +Inf, so a maximum over bit patterns propagates NaN (fmax
// would drop it)
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}

// max over the block of two bit patterns, then one atomicMax each into red[0], red[1]
__device__ __forceinline__ void block_max2(unsigned long long a, unsigned long long b,
                                           unsigned long long* __restrict__ red) {
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  __shared__ unsigned long long sa[32], sb[32];
  const int t = threadIdx.x + blockDim.x * threadIdx.y, warp = t >> 5, lane = t & 31;
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (t == 0) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    for (int q = 1; q < nw; ++q) {
      a = max(a, sa[q]);
      b = max(b, sb[q]);
    }
    atomicMax(red, a);
    atomicMax(red + 1, b);
  }
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
  unsigned long long dmax = 0, vmax = 0;
  if (i < g.X && j < g.Y) {
    Corr<STR> C{g, S, vs, phi, P};
    const int e = C.at(i, j, k);
    const double ur = C.u(i, j, k), vr = C.v(i, j, k), wr = C.w(i, j, k);
    out[e] = ur;
    out[P + e] = vr;
    out[2 * P + e] = wr;
    const bool cell = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny && k >= 1 && k <= g.nz;
    if (check) vmax = max(abs_bits(ur), max(abs_bits(vr), abs_bits(wr)));
    if (check && cell) {
      const double d = (ur - C.u(i - 1, j, k)) * inv_w<STR, 0, KV_SW_IDC>(g, S, i) +
                       (vr - C.v(i, j - 1, k)) * inv_w<STR, 1, KV_SW_IDC>(g, S, j) +
                       (wr - C.w(i, j, k - 1)) * inv_w<STR, 2, KV_SW_IDC>(g, S, k);
      dmax = abs_bits(d);
    }
    if (p) {
      if (cell)
        p[e] = (acc_p ? p[e] : 0.0) + C.ph(i, j, k);
      else if (!acc_p)
        p[e] = 0.0;
    }
  }
  if (!check) return;
  block_max2(dmax, vmax, red);  // one atomic each per block
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

// The same divergence as a march in z: a warp covers 31 cells of a row plus the face to their
// left (lane 0), so u(i-1) comes by shuffle and each u value is split once; w(k-1) is the
// previous plane's w, kept in a register; the next plane's loads are issued before this plane's
// arithmetic. kc planes per block.
constexpr int MD_Y = 8;
template <bool STR>
__global__ void __launch_bounds__(32 * MD_Y) k_divergence_df_march(KvGeom g, KvStretch S,
                                                                 const double* __restrict__ vel, size_t P,
                                                                 double* __restrict__ b, float2 ihx, float2 ihy,
                                                                 float2 ihz, __nv_bfloat16* __restrict__ xs,
                                                                 size_t slice, int pitch, int kc) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * 31 + tx;  // lane 0: the face left of this warp's first cell
  const int j = blockIdx.y * MD_Y + ty + 1;
  const int k0 = 1 + blockIdx.z * kc, k1 = min(k0 + kc, g.nz + 1);
  const bool row = i < g.X && j <= g.ny;       // loads stay inside the padded arrays
  const bool own = tx >= 1 && i <= g.nx && j <= g.ny;
  const double* u = vel;
  const double* v = vel + P;
  const double* w = vel + 2 * P;
  const size_t sz = (size_t)g.X * g.Y;
  const size_t e0 = (size_t)i + (size_t)g.X * j;  // padded index at k = 0
  struct In {
    double u, v, vm, w;
  };
  auto load = [&](int k, In& r) {
    r = In{0.0, 0.0, 0.0, 0.0};
    if (!row) return;
    const size_t e = e0 + sz * k;
    r.u = __ldg(u + e);
    if (tx >= 1) {
      r.v = __ldg(v + e);
      r.vm = __ldg(v + e - g.X);
      r.w = __ldg(w + e);
    }
  };
  DF wprev = (row && tx >= 1) ? df_split(__ldg(w + e0 + sz * (k0 - 1))) : DF{0.0f, 0.0f};
  In cur, nxt;
  load(k0, cur);
  const DF cx = inv_w_df<STR, 0, KV_SWD_IDC>(g, S, own ? i : 1, ihx);
  const DF cy = inv_w_df<STR, 1, KV_SWD_IDC>(g, S, own ? j : 1, ihy);
  for (int k = k0; k < k1; ++k) {
    if (k + 1 < k1) load(k + 1, nxt);
    const DF su = df_split(cur.u);
    const DF um{__shfl_up_sync(0xffffffffu, su.h, 1), __shfl_up_sync(0xffffffffu, su.l, 1)};
    const DF sw = df_split(cur.w);
    if (own) {
      const DF dx = df_mul(df_sub(su, um), cx);
      const DF dy = df_mul(df_sub(df_split(cur.v), df_split(cur.vm)), cy);
      const DF dz = df_mul(df_sub(sw, wprev), inv_w_df<STR, 2, KV_SWD_IDC>(g, S, k, ihz));
      const DF d = df_add(df_add(dx, dy), dz);
      b[(i - 1) + (size_t)g.nx * ((j - 1) + (size_t)g.ny * (k - 1))] = df_value(d);
      if (xs) kv_store_bf16x3(xs, slice, ((size_t)(k - 1) * g.ny + (j - 1)) * pitch + (i - 1), __fadd_rn(d.h, d.l));
    }
    wprev = sw;
    cur = nxt;
  }
}

__device__ __forceinline__ float df_abs_hi(const DF a) { return fabsf(__fadd_rn(a.h, a.l)); }

// The corrected faces and p only (no SIMPLE test), each input loaded and split once, inverse
// spacings passed as FP32 pairs (ih).
template <bool STR>
__global__ void __launch_bounds__(256) k_correct_df(KvGeom g, KvStretch S, const double* __restrict__ vs,
                                                    const double* __restrict__ phi, size_t P,
                                                    double* __restrict__ out, double* __restrict__ p, int acc_p,
                                                    float2 ihx, float2 ihy, float2 ihz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.X || j >= g.Y) return;
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
  if (p) {
    if (cell)
      p[e] = (acc_p ? p[e] : 0.0) + p0d;
    else if (!acc_p)
      p[e] = 0.0;
  }
}

// The double-float correction with the SIMPLE test, marching in z (the form the one-pass
// evaluations use). A warp owns 31 face columns of one row: lane 0 is a halo that forms the
// corrected face u(i-1) its neighbour's divergence needs (handed over by a warp shuffle) and
// writes nothing; v(j-1) is formed again by the thread itself (two more loads, no block-wide
// barrier); w(k-1) is the previous plane's value, kept in a register. So max |D v| costs about
// one extra corrected face and one double-float divergence per cell, with the same rounding of
// the faces as the stored velocity. The loads of plane k+1 are issued before plane k is computed.
// Outputs as k_correct_df.
constexpr int MC_Y = 8;
struct CorrIn {
  double u, v, w, c, cx, cy, cz;  // v* at (i, j, k); phi at the cell and its three plus neighbours
  double vm, cm;                  // v* at (i, j-1, k) and phi at the cell (i, j-1, k)
};
template <bool STR>
__global__ void __launch_bounds__(32 * MC_Y) k_correct_df_march(KvGeom g, KvStretch S, const double* __restrict__ vs,
                                                              const double* __restrict__ phi, size_t P,
                                                              double* __restrict__ out, double* __restrict__ p,
                                                              int acc_p, unsigned long long* __restrict__ red,
                                                              float2 ihx, float2 ihy, float2 ihz, int kc) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * 31 + tx - 1;  // -1 for the first block's halo lane
  const int j = blockIdx.y * MC_Y + ty;
  const int k0 = blockIdx.z * kc, k1 = min(k0 + kc, g.Z);
  const bool own = tx >= 1 && i < g.X && j < g.Y;
  const bool col = i >= 1 && i <= g.nx && j >= 1 && j <= g.ny;  // a column of cells
  const bool vface_m = col && j >= 2;                            // the face v(i, j-1) is interior
  const size_t cy = g.nx, cz = (size_t)g.nx * g.ny;
  const size_t e0 = (size_t)i + (size_t)g.X * (size_t)j;                  // padded index at k = 0
  const size_t c0 = col ? (size_t)(i - 1) + cy * (size_t)(j - 1) : 0;   // compact index at k = 1
  // the inputs of plane k (zero where the plane has no cell in this column); the loads stay
  // inside the arrays: phi is read at compact cells and their neighbours inside the grid
  auto load = [&](int k, CorrIn& r) {
    r = CorrIn{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (!col || k < 1 || k > g.nz) return;
    const size_t e = e0 + (size_t)g.X * g.Y * k, c = c0 + cz * (size_t)(k - 1);
    r.c = __ldg(phi + c);
    if (i <= g.nx - 1) {
      r.u = __ldg(vs + e);
      r.cx = __ldg(phi + c + 1);
    }
    if (j <= g.ny - 1) {
      r.v = __ldg(vs + P + e);
      r.cy = __ldg(phi + c + cy);
    }
    if (k <= g.nz - 1) {
      r.w = __ldg(vs + 2 * P + e);
      r.cz = __ldg(phi + c + cz);
    }
    if (vface_m) {
      r.vm = __ldg(vs + P + e - g.X);
      r.cm = __ldg(phi + c - cy);
    }
  };
  // corrected faces at (i, j, k) and v at (i, j-1, k): zero outside the interior faces
  auto faces = [&](int k, const CorrIn& r, DF& ur, DF& vr, DF& wr, DF& vmr) {
    ur = vr = wr = vmr = DF{0.0f, 0.0f};
    if (!col || k < 1 || k > g.nz) return;
    const DF p0 = df_split(r.c);
    if (i <= g.nx - 1)
      ur = df_sub(df_split(r.u), df_mul(df_sub(df_split(r.cx), p0), inv_w_df<STR, 0, KV_SWD_IDF>(g, S, i, ihx)));
    if (j <= g.ny - 1)
      vr = df_sub(df_split(r.v), df_mul(df_sub(df_split(r.cy), p0), inv_w_df<STR, 1, KV_SWD_IDF>(g, S, j, ihy)));
    if (k <= g.nz - 1)
      wr = df_sub(df_split(r.w), df_mul(df_sub(df_split(r.cz), p0), inv_w_df<STR, 2, KV_SWD_IDF>(g, S, k, ihz)));
    if (vface_m)
      vmr = df_sub(df_split(r.vm), df_mul(df_sub(p0, df_split(r.cm)), inv_w_df<STR, 1, KV_SWD_IDF>(g, S, j - 1, ihy)));
  };
  DF wprev{0.0f, 0.0f};
  CorrIn cur, nxt;
  if (k0 >= 1) {
    DF a, b, d;
    load(k0 - 1, cur);
    faces(k0 - 1, cur, a, b, wprev, d);
  }
  load(k0, cur);
  unsigned long long dmax = 0, vmax = 0;
  for (int k = k0; k < k1; ++k) {
    if (k + 1 < k1) load(k + 1, nxt);
    DF ur, vr, wr, vm;
    faces(k, cur, ur, vr, wr, vm);
    const DF um{__shfl_up_sync(0xffffffffu, ur.h, 1), __shfl_up_sync(0xffffffffu, ur.l, 1)};
    if (own) {
      const size_t e = e0 + (size_t)g.X * g.Y * k;
      out[e] = df_value(ur);
      out[P + e] = df_value(vr);
      out[2 * P + e] = df_value(wr);
      const unsigned int vb = max(__float_as_uint(df_abs_hi(ur)), max(__float_as_uint(df_abs_hi(vr)),
                                                                      __float_as_uint(df_abs_hi(wr))));
      vmax = max(vmax, abs_bits(df_f2d(__uint_as_float(vb))));
      const bool cell = col && k >= 1 && k <= g.nz;
      if (cell) {
        const DF d = df_add(df_add(df_mul(df_sub(ur, um), inv_w_df<STR, 0, KV_SWD_IDC>(g, S, i, ihx)),
                                   df_mul(df_sub(vr, vm), inv_w_df<STR, 1, KV_SWD_IDC>(g, S, j, ihy))),
                            df_mul(df_sub(wr, wprev), inv_w_df<STR, 2, KV_SWD_IDC>(g, S, k, ihz)));
        dmax = max(dmax, abs_bits(df_value(d)));
      }
      if (p) {
        if (cell)
          p[e] = (acc_p ? p[e] : 0.0) + cur.c;
        else if (!acc_p)
          p[e] = 0.0;
      }
    }
    wprev = wr;
    cur = nxt;
  }
  block_max2(dmax, vmax, red);
}

// One SIMPLE test closed on the device (one thread): see KvGuardDev.
__global__ void k_guard_close(KvGuardDev* __restrict__ gd, double hmin, double tol, int record) {
  const double md = __longlong_as_double((long long)gd->red[0]);
  const double vm = __longlong_as_double((long long)gd->red[1]);
  gd->red[0] = 0ull;
  gd->red[1] = 0ull;
  const double rel = vm > 0.0 ? md * hmin / vm : (md > 0.0 ? md : 0.0);
  const bool finite = isfinite(md) && isfinite(vm) && isfinite(rel);
  gd->last_maxdiv = md;
  gd->last_vmax = vm;
  gd->last_rel = finite ? rel : __longlong_as_double(0x7FF8000000000000LL);
  if (!record) return;
  gd->checks += 1ull;
  if (!finite) {
    gd->nonfinite += 1ull;
  } else {
    if (!(rel < tol)) gd->failed += 1ull;
    if (rel > gd->worst_rel) gd->worst_rel = rel;
  }
}

// x as an FP32 pair (host side)
float2 pair_of(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

}  // namespace

void kv_launch_divergence(const kv_grid* h, const double* vel, double* b, cudaStream_t s) {
  kv_launch_divergence_to(h, vel, b, h->xs[0], h->xs_slice, s);
}

void kv_launch_divergence_to(const kv_grid* h, const double* vel, double* b, __nv_bfloat16* xs, size_t slice,
                             cudaStream_t s) {
  const KvGeom& g = h->g;
  dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  const bool str = h->str.sw != nullptr;
  if (h->d.precision == KV_PREC_MIXED) {
    const int kc = 16;
    dim3 mblock(32, MD_Y, 1), mgrid((g.nx + 30) / 31, (g.ny + MD_Y - 1) / MD_Y, (g.nz + kc - 1) / kc);
    auto kern = str ? k_divergence_df_march<true> : k_divergence_df_march<false>;
    kern<<<mgrid, mblock, 0, s>>>(g, h->str, vel, h->P, b, pair_of(g.ihx), pair_of(g.ihy), pair_of(g.ihz), xs,
                                  slice, (g.nx + 7) & ~7, kc);
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
    if (check) {
      const int kc = 16;
      dim3 mb(32, MC_Y, 1), mg((g.X + 30) / 31, (g.Y + MC_Y - 1) / MC_Y, (g.Z + kc - 1) / kc);
      auto kern = str ? k_correct_df_march<true> : k_correct_df_march<false>;
      kern<<<mg, mb, 0, s>>>(g, h->str, vstar, phi, h->P, out_vel, p, accumulate_p, h->red, cx, cy, cz, kc);
      return;
    }
    auto kern = str ? k_correct_df<true> : k_correct_df<false>;
    kern<<<grid, block, 0, s>>>(g, h->str, vstar, phi, h->P, out_vel, p, accumulate_p, cx, cy, cz);
  } else {
    auto kern = str ? k_correct<true> : k_correct<false>;
    kern<<<grid, block, 0, s>>>(g, h->str, vstar, phi, h->P, out_vel, p, accumulate_p, check, h->red);
  }
}

void kv_launch_guard_close(const kv_grid* h, double tol, int record, cudaStream_t s) {
  k_guard_close<<<1, 1, 0, s>>>(h->guard, h->hmin, tol, record);
}
