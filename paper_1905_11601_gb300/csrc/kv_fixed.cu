// The mixed path's linearised operator J P_BC x (Eqs (8)-(9) as used by Eqs (11)-(12)) in
// fixed-point integer arithmetic, formed directly from the base state: uniform cubic grids.
//
// The double-float operator (kv_stencil.cu) reads 25 assembled coefficient pairs per cell, 2.7x
// the algorithmic bytes, and spends about eleven FP32 instructions on each product. Here the
// base state is converted once per base flow to fixed point (kv_fixed.cuh), and every Krylov
// vector is converted while it is staged; each term of the operator is then one product of two
// exact integer combinations, three 32 x 32 -> 64-bit multiply-adds. Per cell the kernel reads
// the four base fields and the four input fields and writes the four outputs: the algorithmic
// bytes. A pre-pass finds the input's largest magnitude (the grid of its fixed-point form) and
// writes the boundary zeros of the outputs.
#include <algorithm>
#include <cmath>

#include "kv_internal.cuh"

namespace {

// 8-byte asynchronous global -> shared copy; n = 0 fills the destination with zeros
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, unsigned int n) {
  const unsigned int d = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem), "r"(n) : "memory");
}

__device__ __forceinline__ unsigned int abs_hi(double v) {
  return (unsigned int)(__double2hiint(v)) & 0x7FFFFFFFu;  // monotonic in |v|; NaN above Inf
}

// The largest |x| over the entries P_BC keeps, as the high word of its bit pattern (one atomic
// max into xmax per block), and the padded-boundary entries of v* and T* (0, except the
// insulated walls' temperature nodes, which the operator writes from their neighbouring cells).
// Each warp takes whole x-rows of the padded array; along a row the kept entries of a field are
// one contiguous range, which each lane reads PF_U entries at a time (independent loads).
constexpr int PF_U = 9;  // 32 x 9 = 288 >= X for n <= 286; longer rows take further passes
__global__ void __launch_bounds__(256) k_fx_prepass(KvGeom g, const double* __restrict__ x, size_t P,
                                                    unsigned int* __restrict__ xmax, double* __restrict__ vstar,
                                                    double* __restrict__ tout) {
  __shared__ unsigned int wmax[8];
  const int lane = threadIdx.x & 31;
  const int nwarp = gridDim.x * (blockDim.x >> 5);
  const bool aa_t = g.bc == KV_BC_AA && g.tproj != KV_TPROJ_OBLIQUE;  // wall T nodes are read
  unsigned int m = 0;
  for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < g.Y * g.Z; row += nwarp) {
    const int j = row % g.Y, k = row / g.Y;
    const size_t e0 = (size_t)g.X * row;
    const bool jin = j >= 1 && j <= g.ny, kin = k >= 1 && k <= g.nz;
    // kept range [lo, hi] of each field on this row (empty: hi < lo)
    int hi_f[4];
    hi_f[0] = jin && kin ? g.nx - 1 : 0;
    hi_f[1] = j >= 1 && j <= g.ny - 1 && kin ? g.nx : 0;
    hi_f[2] = jin && k >= 1 && k <= g.nz - 1 ? g.nx : 0;
    hi_f[3] = kin && (jin || (aa_t && (j == 0 || j == g.ny + 1))) ? g.nx : 0;
    for (int i0 = 0; i0 < g.X; i0 += 32 * PF_U) {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        double vals[PF_U];
#pragma unroll
        for (int u = 0; u < PF_U; ++u) {
          const int i = i0 + lane + 32 * u;
          vals[u] = (i >= 1 && i <= hi_f[f]) ? __ldg(x + (size_t)f * P + e0 + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < PF_U; ++u) m = max(m, abs_hi(vals[u]));
      }
    }
    // boundary zeros: whole rows outside the interior, else the two ends of the row
    const bool row_in = jin && kin;
    const bool aa_row = g.bc == KV_BC_AA && (j == 0 || j == g.ny + 1) && kin;
    for (int i = lane; i < g.X; i += 32) {
      if (row_in && i >= 1 && i <= g.nx) continue;
      const size_t e = e0 + i;
      vstar[e] = 0.0;
      vstar[P + e] = 0.0;
      vstar[2 * P + e] = 0.0;
      if (!(aa_row && i >= 1 && i <= g.nx)) tout[e] = 0.0;
    }
  }
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  if (lane == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, wmax[w]);
    if (b) atomicMax(xmax, b);
  }
}

// the largest |value| of an array (high words of the bit patterns), for the base state's grid
__global__ void __launch_bounds__(256) k_fx_absmax(const double* __restrict__ a, size_t n,
                                                   unsigned int* __restrict__ out) {
  unsigned int m = 0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    m = max(m, abs_hi(__ldg(a + t)));
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// Upwind advection: the one-sided choice of each equation along each axis at every cell (bit set:
// backward, the selecting velocity >= 0), from the FP64 base state: bits 0-2 u (x, y, z), 3-5 v,
// 6-8 w, 9-11 T. The selecting velocity is the base component averaged to the equation's node,
// the 4-point sums taken in a fixed order (the two entries at t-1 along the component's axis,
// then the two at t), as in the coefficient assembly. 0 outside the cells.
__global__ void __launch_bounds__(256) k_fx_sel(KvGeom g, const double* __restrict__ base, size_t P,
                                                unsigned short* __restrict__ sel) {
  const int sy = g.X, sz = g.X * g.Y;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.X), j = (int)((e / g.X) % g.Y), k = (int)(e / sz);
    if (i < 1 || i > g.nx || j < 1 || j > g.ny || k < 1 || k > g.nz) {
      sel[e] = 0;
      continue;
    }
    const double* U = base;
    const double* V = base + P;
    const double* W = base + 2 * P;
    auto s4 = [](double a, double b, double c, double d) { return ((a + b) + c) + d; };
    unsigned int m = 0;
    // u on the x-face (i, j, k)
    m |= (__ldg(U + e) >= 0.0) << 0;
    m |= (s4(__ldg(V + e - sy), __ldg(V + e + 1 - sy), __ldg(V + e), __ldg(V + e + 1)) >= 0.0) << 1;
    m |= (s4(__ldg(W + e - sz), __ldg(W + e + 1 - sz), __ldg(W + e), __ldg(W + e + 1)) >= 0.0) << 2;
    // v on the y-face
    m |= (s4(__ldg(U + e - 1), __ldg(U + e - 1 + sy), __ldg(U + e), __ldg(U + e + sy)) >= 0.0) << 3;
    m |= (__ldg(V + e) >= 0.0) << 4;
    m |= (s4(__ldg(W + e - sz), __ldg(W + e + sy - sz), __ldg(W + e), __ldg(W + e + sy)) >= 0.0) << 5;
    // w on the z-face
    m |= (s4(__ldg(U + e - 1), __ldg(U + e - 1 + sz), __ldg(U + e), __ldg(U + e + sz)) >= 0.0) << 6;
    m |= (s4(__ldg(V + e - sy), __ldg(V + e - sy + sz), __ldg(V + e), __ldg(V + e + sz)) >= 0.0) << 7;
    m |= (__ldg(W + e) >= 0.0) << 8;
    // T at the cell (2-point sums)
    m |= (__ldg(U + e - 1) + __ldg(U + e) >= 0.0) << 9;
    m |= (__ldg(V + e - sy) + __ldg(V + e) >= 0.0) << 10;
    m |= (__ldg(W + e - sz) + __ldg(W + e) >= 0.0) << 11;
    sel[e] = (unsigned short)m;
  }
}

// the base state on its fixed-point grid (r0 = fx_r0(E))
__global__ void __launch_bounds__(256) k_fx_base(const double* __restrict__ a, size_t n, int r0,
                                                 int2* __restrict__ out) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const FX v = fx_of(__ldg(a + t), r0);
    out[t] = make_int2(v.h, v.l);
  }
}

// ---- the operator: a 2.5D march, two threads per cell ---------------------------------------
//
// A block owns FB_X x FB_Y cells and walks kc z-planes. Shared memory holds four planes of the
// eight staged fields (projected input and base state, fixed point, with a one-cell halo): at
// step k the threads issue the copies of plane k+2, form their cells' equations from planes
// k-1..k+1 (the first half of the block u and T, the second half v and w), convert and store
// plane k+2 into the slot plane k-2 used, and synchronise once. (A deeper ring, three compute
// slots and two planes in flight, measured slower: it needs a second barrier per plane.)
constexpr int FB_X = 32, FB_Y = 8;
constexpr int FT_X = FB_X + 2, FT_Y = FB_Y + 2, FPTS = FT_X * FT_Y;
constexpr int FCELLS = FB_X * FB_Y;
constexpr int FTHREADS = 2 * FCELLS;
constexpr int FVALS = 8 * FPTS;                         // values per plane: 4 input + 4 base fields
constexpr int FPER = (FVALS + FTHREADS - 1) / FTHREADS;  // values per thread per plane
constexpr int FIN = 4 * FPTS;                           // the input fields come first
constexpr int FRIN = FIN / FTHREADS;                    // values r < FRIN of a thread are input
constexpr size_t FSMEM = (size_t)4 * FVALS * sizeof(int2) + (size_t)FIN * sizeof(double);  // + xraw
static_assert(FIN / FTHREADS == 2 && (FIN + FTHREADS - 1) / FTHREADS == 3,
              "values r < 2 of a thread are input, r == 2 either, r > 2 base state");

// UPW: upwind advection, every cell with the one-sided weights its selector bits choose (sel).
template <bool UPW>
__global__ void __launch_bounds__(FTHREADS, 2)
    k_apply_fx_march(KvGeom g, const int2* __restrict__ bfx, const double* __restrict__ x, size_t P,
                     double* __restrict__ vstar, double* __restrict__ tout, FxConst K,
                     const unsigned int* __restrict__ xmax, const unsigned short* __restrict__ sel, int kc) {
  extern __shared__ int2 fst[];  // [slot][field][point]
  const int tid = threadIdx.x;
  const int half = tid / FCELLS;  // 0: u and T, 1: v and w (uniform per warp)
  const int tx = tid & 31, ty = (tid % FCELLS) >> 5;
  const int i = 1 + blockIdx.x * FB_X + tx, j = 1 + blockIdx.y * FB_Y + ty;
  const int k0 = 1 + blockIdx.z * kc;
  const int k1 = min(k0 + kc, g.nz + 1);  // planes k0 .. k1-1
  const bool active = i <= g.nx && j <= g.ny;
  const int sy = g.X, sz = g.X * g.Y;

  // the input's grid: |x| < 2^ex over the kept entries (from the pre-pass)
  const unsigned int mb = __ldg(xmax);
  const int eb = (int)((mb >> 20) & 0x7FFu);
  const bool nonfinite = eb == 0x7FF;
  const int ex = eb == 0 ? -1022 : eb - 1022;
  const int r0 = fx_r0(ex);
  const int ea = ex / 2, eb2 = ex - ex / 2;  // 2^ex in two in-range factors
  const double fout = K.f0 * fx_from_bits((unsigned long long)(ea + 1023) << 52) *
                      fx_from_bits((unsigned long long)(eb2 + 1023) << 52);

  // what this thread stages: value v = tid + r FTHREADS of a plane is field v / FPTS at tile point
  // v % FPTS. Input values (v < FIN): x_f at column col[r] for planes 1 <= k <= lim[r], 0 for the
  // others (lim 0: always 0), except the temperature rows next to insulated walls (lim < 0), which
  // are projected here. Base values: the column of the fixed-point base state (clamped into the
  // padded array for tile points past its edge, whose values no cell reads).
  unsigned int col[FPER];
  int lim[FPER];
#pragma unroll
  for (int r = 0; r < FPER; ++r) {
    const int v = tid + r * FTHREADS;
    col[r] = 0;
    lim[r] = 0;
    if (v < FVALS) {
      const int f = v / FPTS, pt = v - f * FPTS;
      const int ii = blockIdx.x * FB_X + pt % FT_X, jj = blockIdx.y * FB_Y + pt / FT_X;
      if (f >= 4) {
        col[r] = (unsigned int)((size_t)(f - 4) * P + min(ii, g.nx + 1) + (size_t)sy * min(jj, g.ny + 1));
      } else if (ii <= g.nx + 1 && jj <= g.ny + 1) {
        col[r] = (unsigned int)((size_t)f * P + ii + (size_t)sy * jj);
        const bool in_i = ii >= 1 && ii <= g.nx, in_j = jj >= 1 && jj <= g.ny;
        if (f == 0)
          lim[r] = (ii >= 1 && ii <= g.nx - 1 && in_j) ? g.nz : 0;
        else if (f == 1)
          lim[r] = (in_i && jj >= 1 && jj <= g.ny - 1) ? g.nz : 0;
        else if (f == 2)
          lim[r] = (in_i && in_j) ? g.nz - 1 : 0;
        else if (g.bc == KV_BC_CC)
          lim[r] = (in_i && in_j) ? g.nz : 0;
        else
          lim[r] = !in_i ? 0 : ((jj >= 2 && jj <= g.ny - 1) ? g.nz : -1);
      }
    }
  }
  const double* const xT = x + 3 * P;
  // the projected temperature at a row next to an insulated wall (Eq 13's P_BC for T)
  auto proj_t = [&](int ii, int jj, int kk) -> double {
    if (kk < 1 || kk > g.nz) return 0.0;
    const int jw = jj <= 1 ? 0 : g.ny + 1, jn = jj <= 1 ? 1 : g.ny;
    const double tn = __ldg(xT + ii + (size_t)sy * jn + (size_t)sz * kk);
    if (g.tproj == KV_TPROJ_OBLIQUE) return tn;
    return 0.5 * (tn + __ldg(xT + ii + (size_t)sy * jw + (size_t)sz * kk));
  };
  // Staging of plane kk into a slot, in two steps with the plane's compute between them. issue:
  // asynchronous copies (no registers held): the base state's pairs straight into the slot, the
  // input's FP64 values (zero-filled where P_BC gives 0) into this thread's entries of xraw.
  // finish: waits for them and converts the input to its fixed-point grid.
  double* const xraw = reinterpret_cast<double*>(fst + 4 * FVALS);
  auto issue = [&](int kk, int slot) {
#pragma unroll
    for (int r = 0; r < FPER; ++r) {
      const int v = tid + r * FTHREADS;
      if (r < FRIN || (r == FRIN && v < FIN)) {
        // lim < 0 compares as a large unsigned limit: the copy stays inside the column
        const unsigned int n = (unsigned)(kk - 1) < (unsigned)lim[r] ? 8u : 0u;
        cp_async8(xraw + v, x + (col[r] + (unsigned int)(sz * kk)), n);
      } else if (v < FVALS) {
        cp_async8(fst + slot * FVALS + v, bfx + (col[r] + (unsigned int)(sz * kk)), 8u);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto finish = [&](int kk, int slot) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
    for (int r = 0; r <= FRIN; ++r) {
      const int v = tid + r * FTHREADS;
      if (r < FRIN || v < FIN) {
        double xv = xraw[v];
        if (lim[r] < 0) {
          const int pt = v - 3 * FPTS;
          xv = proj_t(blockIdx.x * FB_X + pt % FT_X, blockIdx.y * FB_Y + pt / FT_X, kk);
        }
        const FX q = fx_of(xv, r0);
        fst[slot * FVALS + v] = make_int2(q.h, q.l);
      }
    }
  };
  for (int kk = k0 - 1; kk <= k0 + 1; ++kk) {
    issue(kk, kk & 3);
    finish(kk, kk & 3);
  }
  __syncthreads();
  const int cx = fx_class(i, g.nx), cy = fx_class(j, g.ny);
  // every cell of this warp's row segment is interior along x (cells 2 .. nx-1)
  const bool x_inner = blockIdx.x >= 1 && FB_X * (blockIdx.x + 1) <= g.nx - 1;
  const int pc = (ty + 1) * FT_X + (tx + 1);  // this cell's point in the tile
  const size_t Pz = P;
  for (int k = k0; k < k1; ++k) {
    const bool more = k + 1 < k1;
    if (more) issue(k + 2, (k + 2) & 3);
    if (active) {
      const int sm = ((k - 1) & 3) * FVALS + pc, s0 = (k & 3) * FVALS + pc, sp = ((k + 1) & 3) * FVALS + pc;
      auto X = [&](int f, int di, int dj, int dk) {
        const int2 t = fst[(dk < 0 ? sm : (dk > 0 ? sp : s0)) + f * FPTS + di + FT_X * dj];
        return FX{t.x, t.y};
      };
      auto B = [&](int f, int di, int dj, int dk) {
        const int2 t = fst[(dk < 0 ? sm : (dk > 0 ? sp : s0)) + (4 + f) * FPTS + di + FT_X * dj];
        return FX{t.x, t.y};
      };
      const int cz = fx_class(k, g.nz);
      const size_t e = (size_t)i + (size_t)sy * j + (size_t)sz * k;
      // a non-finite input: every result NaN (scaled by NaN)
      const double fo = nonfinite ? __longlong_as_double(0x7FF8000000000000ll) : fout;
      // the cell's equations with the derivative weights of its wall classes; fs scales the
      // result (3 where the interior first-derivative weights run without their factor 3)
      auto eqs = [&](W3i d1x, W3i d2x, W3i d1y, W3i d2y, W3i d1z, W3i d2z, const FxK& KK, int face,
                     double fs) {
        if (half == 0) {
          const long long tu = fx_eq_u(X, B, d1y, d2y, d1z, d2z, KK, face);
          vstar[e] = i <= g.nx - 1 ? fx_to_double(tu) * fs : 0.0;
          const double r = fx_to_double(fx_eq_t(X, B, d1x, d2x, d1y, d2y, d1z, d2z, KK, face)) * fs;
          // insulated wall pair: the cell and its wall node (Eq 21's projection for that pair)
          const bool pair = g.bc == KV_BC_AA && (j == 1 || j == g.ny);
          const double t = pair && g.tproj != KV_TPROJ_OBLIQUE ? 0.5 * r : r;
          tout[e] = t;
          if (pair) tout[(size_t)i + (size_t)sy * (j == 1 ? 0 : g.ny + 1) + (size_t)sz * k] = t;
        } else {
          const long long tv = fx_eq_v(X, B, d1x, d2x, d1z, d2z, KK, face);
          vstar[Pz + e] = j <= g.ny - 1 ? fx_to_double(tv) * fs : 0.0;
          const long long tw = fx_eq_w(X, B, d1x, d2x, d1y, d2y, KK, face);
          vstar[2 * Pz + e] = k <= g.nz - 1 ? fx_to_double(tw) * fs : 0.0;
        }
      };
      // interior weights as constants where the whole warp is interior (the weighted sums become
      // differences); the walls' weights per cell elsewhere
      const W3i I1{-3, 0, 3}, I2{1, -2, 1}, J1{-1, 0, 1};
      if (UPW) {
        const unsigned int b = __ldg(sel + e);
        const W3i dx2 = fx_d2(cx), dy2 = fx_d2(cy), dz2 = fx_d2(cz);
        if (half == 0) {
          const long long tu = fx_eq_u(X, B, fx_u1(cy, b & 2u), dy2, fx_u1(cz, b & 4u), dz2, K.k1, fx_u1_face(b & 1u));
          vstar[e] = i <= g.nx - 1 ? fx_to_double(tu) * fo : 0.0;
          const double r = fx_to_double(fx_eq_t(X, B, fx_u1(cx, b & 512u), dx2, fx_u1(cy, b & 1024u), dy2,
                                                fx_u1(cz, b & 2048u), dz2, K.k1, 12)) * fo;
          const bool pair = g.bc == KV_BC_AA && (j == 1 || j == g.ny);
          const double t = pair && g.tproj != KV_TPROJ_OBLIQUE ? 0.5 * r : r;
          tout[e] = t;
          if (pair) tout[(size_t)i + (size_t)sy * (j == 1 ? 0 : g.ny + 1) + (size_t)sz * k] = t;
        } else {
          const long long tv = fx_eq_v(X, B, fx_u1(cx, b & 8u), dx2, fx_u1(cz, b & 32u), dz2, K.k1, fx_u1_face(b & 16u));
          vstar[Pz + e] = j <= g.ny - 1 ? fx_to_double(tv) * fo : 0.0;
          const long long tw = fx_eq_w(X, B, fx_u1(cx, b & 64u), dx2, fx_u1(cy, b & 128u), dy2, K.k1,
                                       fx_u1_face(b & 256u));
          vstar[2 * Pz + e] = k <= g.nz - 1 ? fx_to_double(tw) * fo : 0.0;
        }
      } else if (cy == 0 && cz == 0 && x_inner)
        eqs(J1, I2, J1, I2, J1, I2, K.k3, 4, 3.0 * fo);
      else if (cy == 0 && cz == 0)
        eqs(fx_d1(cx), fx_d2(cx), I1, I2, I1, I2, K.k1, 12, fo);
      else
        eqs(fx_d1(cx), fx_d2(cx), fx_d1(cy), fx_d2(cy), fx_d1(cz), fx_d2(cz), K.k1, 12, fo);
    }
    if (more) finish(k + 2, (k + 2) & 3);
    __syncthreads();
  }
}

}  // namespace

// Grids the fixed-point operator serves: mixed precision, uniform and cubic (one h on all axes),
// offsets of a packed vector within 32 bits; kv_fx_setup adds a finite base state whose grid
// leaves the accumulators their headroom.
bool kv_fx_eligible(const kv_grid* h) {
  return h->d.precision == KV_PREC_MIXED && !h->str.sw && h->g.nx == h->g.ny && h->g.ny == h->g.nz &&
         4 * h->P < (size_t(1) << 31);
}

void kv_fx_free(kv_grid* h) {
  cudaFree(h->base_fx);
  cudaFree(h->fxmax);
  cudaFree(h->fx_sel);
  h->base_fx = nullptr;
  h->fxmax = nullptr;
  h->fx_sel = nullptr;
  h->fx_ok = false;
}

// Once per base flow: the base state's grid E (|U|, |V|, |W|, |Theta| and the constants below
// 2^E), the base state on it, and the constants of the operator. Synchronises the stream.
kv_status kv_fx_setup(kv_grid* h) {
  h->fx_ok = false;
  if (!kv_fx_eligible(h)) return KV_OK;
  if (!h->base_fx) {
    if (cudaMalloc(&h->base_fx, 4 * h->P * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&h->fxmax, 2 * sizeof(unsigned int)) != cudaSuccess ||
        (h->g.adv && cudaMalloc(&h->fx_sel, h->P * sizeof(unsigned short)) != cudaSuccess)) {
      kv_fx_free(h);
      cudaGetLastError();
      return KV_OK;  // the double-float operator stays in use
    }
  }
  cudaStream_t s = h->s;
  if (cudaMemsetAsync(h->fxmax + 1, 0, sizeof(unsigned int), s) != cudaSuccess) return KV_ERR_CUDA;
  k_fx_absmax<<<4 * 152, 256, 0, s>>>(h->base, 4 * h->P, h->fxmax + 1);
  unsigned int mb = 0;
  if (cudaMemcpyAsync(&mb, h->fxmax + 1, sizeof mb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return KV_ERR_CUDA;
  const int eb = (int)((mb >> 20) & 0x7FFu);
  if (eb == 0x7FF) return KV_OK;  // a non-finite base state: the double-float operator reports it
  // the march's shared memory (above the 48 KB default), set here, outside any stream capture
  if (cudaFuncSetAttribute(k_apply_fx_march<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FSMEM) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_apply_fx_march<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FSMEM) !=
          cudaSuccess) {
    cudaGetLastError();
    return KV_OK;  // the double-float operator stays in use
  }
  const double n = h->g.nx;
  const double kd_m = -24.0 * h->g.nu * n, kd_e = -24.0 * h->g.kappa * n, kb = -12.0 / n;
  int e = eb == 0 ? -1022 : eb - 1022;
  for (double c : {kd_m, kd_e, kb}) e = std::max(e, std::ilogb(c) + 1);
  const int r0 = fx_r0(e);
  FxConst K;
  K.k1 = FxK{fx_of(kd_m, r0), fx_of(kd_e, r0), fx_of(kb, r0)};
  K.k3 = FxK{fx_of(kd_m / 3.0, r0), fx_of(kd_e / 3.0, r0), fx_of(kb / 3.0, r0)};
  K.f0 = -n / 24.0 * std::ldexp(1.0, e - 50);
  K.e = e;
  k_fx_base<<<4 * 152, 256, 0, s>>>(h->base, 4 * h->P, r0, h->base_fx);
  if (h->g.adv) k_fx_sel<<<4 * 152, 256, 0, s>>>(h->g, h->base, h->P, h->fx_sel);
  if (cudaGetLastError() != cudaSuccess) return KV_ERR_CUDA;
  h->fxk = K;
  h->fx_ok = true;
  return KV_OK;
}

// J P_BC x by the fixed-point march (kc planes per block): pre-pass (input grid, boundary zeros),
// then the march. Launches: 2 (plus a 4-byte memset).
void kv_launch_apply_fx(const kv_grid* h, const double* x, double* vstar, double* tout, int kc, cudaStream_t s) {
  const KvGeom& g = h->g;
  cudaMemsetAsync(h->fxmax, 0, sizeof(unsigned int), s);
  k_fx_prepass<<<4 * 152, 256, 0, s>>>(g, x, h->P, h->fxmax, vstar, tout);
  dim3 grid((g.nx + FB_X - 1) / FB_X, (g.ny + FB_Y - 1) / FB_Y, (g.nz + kc - 1) / kc);
  if (g.adv)
    k_apply_fx_march<true><<<grid, FTHREADS, FSMEM, s>>>(g, h->base_fx, x, h->P, vstar, tout, h->fxk, h->fxmax,
                                                         h->fx_sel, kc);
  else
    k_apply_fx_march<false><<<grid, FTHREADS, FSMEM, s>>>(g, h->base_fx, x, h->P, vstar, tout, h->fxk, h->fxmax,
                                                          nullptr, kc);
}
