// Allocation-free variant of the FP64 Krylov-vector evaluation, for callers that must not
// allocate device memory: code running where cudaMalloc / cudaFree are unavailable or
// forbidden (an allocator owned by someone else, a memory budget fixed at start-up, a
// plugin that may not touch the device heap). It runs the same kernels as
// kv_krylov_vector; its scratch (momentum right-hand side, Poisson buffers, per-axis
// eigenvectors) lives in one file-scope __device__ array of fixed size instead of
// library-allocated buffers. Every GPU that loads the library holds that array until the
// process exits.
#include <math.h>
#include <string.h>

#include <atomic>
#include <string>

#include "kv_internal.cuh"

namespace {

constexpr int NMAX = KV_NOALLOC_MAX_N;
constexpr size_t PMAX = (size_t)(NMAX + 2) * (NMAX + 2) * (NMAX + 2);
constexpr size_t NCMAX = (size_t)NMAX * NMAX * NMAX;
// vstar (3 padded fields) | tpd_a | tpd_b | six n x n matrices | three eigenvalue vectors | 2 x u64
constexpr size_t OFF_VSTAR = 0;
constexpr size_t OFF_TPDA = OFF_VSTAR + 3 * PMAX;
constexpr size_t OFF_TPDB = OFF_TPDA + NCMAX;
constexpr size_t OFF_W = OFF_TPDB + NCMAX;
constexpr size_t OFF_LAM = OFF_W + 6 * (size_t)NMAX * NMAX;
constexpr size_t OFF_RED = OFF_LAM + 3 * (size_t)NMAX;
constexpr size_t SCRATCH_DOUBLES = OFF_RED + 2;

// The shared scratch. In host code this name is only a stand-in: the device address comes
// from cudaGetSymbolAddress, taken once per device below.
static __device__ __align__(256) double g_noalloc_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
// the array's device address per device, looked up once (host threads may race to store the
// same value; the atomic makes that well defined)
std::atomic<double*> g_scratch_addr[MAX_DEVICES];

kv_status noalloc_fail(kv_status st, const std::string& msg) {
  kv_set_thread_error(msg);  // read back with kv_last_error(NULL)
  return st;
}

// Eq (15) for the Neumann pressure Laplacian on the uniform axes, built on the device straight into
// the scratch (block a = axis a of n[a] cells): eigenvectors alpha_m cos(pi m (t + 1/2) / n) and
// eigenvalues -4 n^2 sin^2(pi m / 2n), the closed form kv_create_grid uses. The argument
// m (2t + 1) / (2n) is reduced exactly in integers (modulo 4n, a period of cos(pi x / 2n)) before
// cospi, so every entry carries cospi's own rounding only. fwd (E^-1 = E^T): row = mode,
// column = cell; inv (E): row = cell, column = mode.
__global__ void k_noalloc_tables(int n0, int n1, int n2, double* __restrict__ W, double* __restrict__ lam) {
  const int a = blockIdx.x;
  const int n = a == 0 ? n0 : (a == 1 ? n1 : n2);
  double* fwd = W + (size_t)a * NMAX * NMAX;
  double* inv = W + (size_t)(3 + a) * NMAX * NMAX;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int m = idx / n, t = idx - m * n;
    const int q = (m * (2 * t + 1)) % (4 * n);
    const double alpha = sqrt((m == 0 ? 1.0 : 2.0) / n);
    const double e = alpha * cospi((double)q / (2.0 * n));
    fwd[(size_t)m * n + t] = e;
    inv[(size_t)t * n + m] = e;
  }
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    const double sn = sinpi((double)m / (2.0 * n));
    lam[(size_t)a * NMAX + m] = -4.0 * (double)n * (double)n * sn * sn;
  }
}

}  // namespace

extern "C" kv_status kv_krylov_vector_noalloc(const kv_grid_desc* desc, const double* base, const double* x,
                                              double* y, void* stream) {
  if (!desc || !base || !x || !y) return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: NULL argument");
  if (desc->nx < 2 || desc->ny < 2 || desc->nz < 2 || desc->nx > NMAX || desc->ny > NMAX || desc->nz > NMAX)
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: nx, ny, nz must be in [2, " +
                                        std::to_string(NMAX) + "] (size of the static scratch)");
  if (desc->spanwise_bc != KV_BC_CC && desc->spanwise_bc != KV_BC_AA)
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: bad spanwise_bc");
  if (desc->tproj != KV_TPROJ_ORTHOGONAL && desc->tproj != KV_TPROJ_OBLIQUE)
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: bad tproj");
  if (desc->precision != KV_PREC_FP64)
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: only KV_PREC_FP64 is available");
  if (desc->stretch != 0.0)
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: the uniform grid only (stretch must be 0)");
  if (desc->advection != KV_ADV_CENTRAL)
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: central advection only");
  if (!(desc->gr > 0) || !(desc->pr > 0) || !isfinite(desc->gr) || !isfinite(desc->pr))
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: gr and pr must be finite and > 0");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(KV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: device ordinal >= 64");
  double* S = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!S) {  // set-up, once per device, with that device current
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(KV_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    S = (double*)p;
    g_scratch_addr[dev].store(S, std::memory_order_release);
  }
  cudaStream_t s = (cudaStream_t)stream;

  kv_grid h;  // a view over the static scratch; owns nothing
  h.d = *desc;
  h.s = s;
  h.dev = dev;
  KvGeom& g = h.g;
  g.nx = desc->nx;
  g.ny = desc->ny;
  g.nz = desc->nz;
  g.X = g.nx + 2;
  g.Y = g.ny + 2;
  g.Z = g.nz + 2;
  g.hx = 1.0 / g.nx;
  g.hy = 1.0 / g.ny;
  g.hz = 1.0 / g.nz;
  g.ihx = (double)g.nx;
  g.ihy = (double)g.ny;
  g.ihz = (double)g.nz;
  g.ihx2 = g.ihx * g.ihx;
  g.ihy2 = g.ihy * g.ihy;
  g.ihz2 = g.ihz * g.ihz;
  g.nu = 1.0 / sqrt(desc->gr);
  g.kappa = 1.0 / (desc->pr * sqrt(desc->gr));
  g.bc = desc->spanwise_bc;
  g.tproj = desc->tproj;
  g.adv = KV_ADV_CENTRAL;
  h.hmin = fmin(g.hx, fmin(g.hy, g.hz));
  h.P = (size_t)g.X * g.Y * g.Z;
  h.Nc = (size_t)g.nx * g.ny * g.nz;
  if (x < y + 4 * h.P && y < x + 4 * h.P) return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: x and y overlap");
  // the operator reads base directly (there is no library copy of it here) while y is written
  if (base < y + 4 * h.P && y < base + 4 * h.P)
    return noalloc_fail(KV_ERR_ARG, "kv_krylov_vector_noalloc: base and y overlap");
  h.base = const_cast<double*>(base);
  h.vstar = S + OFF_VSTAR;
  h.tpd_a = S + OFF_TPDA;
  h.tpd_b = S + OFF_TPDB;
  h.red = (unsigned long long*)(S + OFF_RED);

  // per-axis eigenvectors / eigenvalues for this size, written into the scratch by a kernel
  for (int a = 0; a < 3; ++a) {
    h.Wm[a] = S + OFF_W + (size_t)a * NMAX * NMAX;
    h.Wm[3 + a] = S + OFF_W + (size_t)(3 + a) * NMAX * NMAX;
    h.lam[a] = S + OFF_LAM + (size_t)a * NMAX;
  }
  k_noalloc_tables<<<3, 256, 0, s>>>(g.nx, g.ny, g.nz, S + OFF_W, S + OFF_LAM);
  // the divergence reduction must start at zero; everything else is fully overwritten
  if ((e = cudaMemsetAsync(h.red, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess)
    return noalloc_fail(KV_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  kv_launch_stencil(&h, 0, h.base, x, h.vstar, y + 3 * h.P, s);
  kv_launch_divergence(&h, h.vstar, h.tpd_a, s);
  kv_launch_poisson(&h, h.tpd_a, h.tpd_a, s);
  kv_launch_correct(&h, h.vstar, h.tpd_a, y, nullptr, 0, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(KV_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return KV_OK;
}
