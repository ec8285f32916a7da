// Internal declarations shared by the CUDA translation units of libkv.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "kv.h"
#include "kv_fixed.cuh"

// timed phases (kv_profile_get)
enum { KV_PH_STENCIL = 0, KV_PH_DIV = 1, KV_PH_TPD = 2, KV_PH_CORRECT = 3, KV_PH_ARNOLDI = 4, KV_PH_REFINE = 5,
       KV_PH_GS_DOTS = 6, KV_PH_GS_UPDATE = 7, KV_NPHASE = 8 };

// Assembled coefficients of the linearised operator per padded entry (kv_stencil.cu).
constexpr int KV_NCOEF = 37;
// coefficients the double-float operator reads (the plus coefficients of the own-field pairs
// are affine in the minus ones)
constexpr int KV_NCOEF_DF = 25;

// Per-axis tables of a stretched grid (Eq 22): KV_SW_N rows of n_a + 2 doubles per axis,
// indexed by the padded index t along the axis (rows for t outside their range are 0).
//   IDC      1 / cell width, cells t = 1..n (divergence)
//   IDF      1 / distance between the centres of cells t and t+1, faces t = 1..n-1 (gradient)
//   C1, C2   first / second derivative weights (minus, centre, plus) at a cell-like node t
//   F1, F2   the same at a face-like node t = 1..n-1
enum { KV_SW_IDC = 0, KV_SW_IDF = 1, KV_SW_C1 = 2, KV_SW_C2 = 5, KV_SW_F1 = 8, KV_SW_F2 = 11, KV_SW_N = 14 };
// The mixed path's copy as FP32 pairs (KV_SWD_N rows of n_a + 2 per axis): IDC and IDF as above,
// and the Neumann Laplacian's weights towards the lower / upper neighbour of cell t,
// LWM = IDC_t IDF_{t-1}, LWP = IDC_t IDF_t (0 where the face is a wall).
enum { KV_SWD_IDC = 0, KV_SWD_IDF = 1, KV_SWD_LWM = 2, KV_SWD_LWP = 3, KV_SWD_N = 4 };
// Assembled coefficients of the plus neighbours, which a stretched grid's double-float operator
// reads as well (the uniform one rebuilds them from the minus ones): per equation x+, y+, z+.
constexpr int KV_NCOEF_DFP = 12;

// Device-side description of the MAC grid.
struct KvGeom {
  int nx, ny, nz;   // cells per axis
  int X, Y, Z;      // padded extents n+2
  double hx, hy, hz;
  double ihx, ihy, ihz;  // 1/h per axis (no FP64 division in the kernels)
  double ihx2, ihy2, ihz2;  // 1/h^2 per axis
  double nu, kappa; // Gr^-1/2 and (Pr Gr^1/2)^-1 (Eqs (1)-(2) scaling)
  int bc;           // KV_BC_CC / KV_BC_AA
  int tproj;        // KV_TPROJ_*
  int adv;          // KV_ADV_* (upwind on uniform grids only)
};

// The device tables of a stretched grid (Eq 22); all null on a uniform grid. A separate kernel
// parameter, passed only to the kernels that read it, so that the uniform kernels' parameters
// (and their register allocation) are those of a uniform-only build.
struct KvStretch {
  const double* sw = nullptr;   // the KV_SW_* tables
  const float2* swd = nullptr;  // KV_PREC_MIXED: the KV_SWD_* tables
  int swo[3] = {0, 0, 0};       // offset of each axis' tables in sw
  int swdo[3] = {0, 0, 0};      // offset of each axis' tables in swd
};

// The SIMPLE stopping test of every one-pass Krylov vector, evaluated on the device (no host
// synchronisation) and accumulated until the host reads it (kv_guard_read): the correction
// kernel reduces max |D v| and max |v| into red (bit patterns of non-negative doubles, so NaN
// compares above every finite value and Inf), and k_guard_close turns them into the relative
// residual, counts the check, and clears red for the next one.
struct KvGuardDev {
  unsigned long long red[2];  // max |D v|, max |v| of the pass in progress (bits)
  unsigned long long checks, failed, nonfinite;
  double worst_rel;           // largest finite max |D v| h_min / max |v|
  double last_maxdiv, last_vmax, last_rel;  // the last pass closed
};

struct kv_grid {
  kv_grid_desc d;
  KvGeom g;
  cudaStream_t s = nullptr;
  int dev = 0;
  size_t P = 0;   // padded field length
  size_t Nc = 0;  // nx*ny*nz
  bool has_base = false;

  double* base = nullptr;   // 4P: U | V | W | Theta
  double* coef = nullptr;   // KV_NCOEF * P: assembled coefficients of J (per base flow)
  float2* coef_df = nullptr; // KV_PREC_MIXED, KV_NCOEF_DF * P: FP32 pairs of the coefficients it reads
  float2* xsplit = nullptr;  // KV_PREC_MIXED, 4P: P_BC x split into FP32 pairs (operator input)
  double* vstar = nullptr;  // 3P: momentum right-hand side before the projection
  double* tpd_a = nullptr;  // Nc: divergence / Poisson ping-pong buffers
  double* tpd_b = nullptr;  // Nc
  double* Wm[6] = {};       // per-axis GEMM operands: forward E_a^-1 (a = 0..2), inverse E_a
  double* lam[3] = {};      // eigenvalues of the 1D Neumann Laplacians (Eq 15)
  KvStretch str;            // stretched grid: views of sw / swd (all null on a uniform grid)
  double* sw = nullptr;     // stretched grid: the KV_SW_* weight tables
  float2* swd = nullptr;    // stretched KV_PREC_MIXED grid: the KV_SWD_* tables
  float2* coef_dfp = nullptr; // stretched or upwind KV_PREC_MIXED grid, KV_NCOEF_DFP * P: plus coefficients as pairs
  double hmin = 0.0;        // smallest cell width (the SIMPLE test)
  unsigned long long* red = nullptr;  // [0] max|D v| bits, [1] max|v| bits (guard->red, or the
                                      // allocation-free entry point's own pair)
  KvGuardDev* guard = nullptr;        // the device-side SIMPLE test (red points into it)
  double* partials = nullptr;         // Arnoldi block partial sums
  size_t partials_cap = 0;            // in doubles
  double* hdev = nullptr;             // Arnoldi coefficients on the device
  size_t hdev_cap = 0;
  double* solve_buf = nullptr;        // Krylov solvers: inner-product partials and small arrays
  size_t solve_cap = 0;
  double* stage = nullptr;            // 8P: staging for the host-buffer entry point
  double* pipe = nullptr;             // 16P: two x and two y staging vectors of the streamed host entry point
  cudaStream_t cs_in = nullptr, cs_out = nullptr;  // its copy streams (host to device, device to host)
  cudaEvent_t pev[6] = {};            // loaded[2], computed[2], drained[2]
  double* adj = nullptr;              // 4P: projected output-side vector of the transpose
  double* adjsum = nullptr;           // 2: reductions of the Grashof derivative
  double* tmp4 = nullptr;             // 4P: residual right-hand side scratch

  // mixed precision (KV_PREC_MIXED): BF16 slices of the six per-axis matrices, two ping-pong
  // slice buffers for the data, FP32 eigenvalues, the tensor maps of the six contractions
  int refine = 0;                        // Poisson refinement sweeps
  __nv_bfloat16* wsl[6] = {};
  __nv_bfloat16* xs[2] = {};
  float* phi32 = nullptr;                // Nc: phi after the first tensor-core sweep (exact FP32 values)
  size_t xs_slice = 0;                   // elements per data slice
  float* lamf[3] = {};
  CUtensorMap mapA[6], mapB[6];
  CUtensorMap mapB128[6];                // the data maps for the 128-column tile
  int umma_tile = 256;                   // the contractions' tile width (autotuner / kv_set_contraction_tile)

  // block evaluations (kv_krylov_vector_batch in mixed precision; kv_block.cu): per-vector
  // buffers for up to blk_cap vectors, allocated at the first block call
  int blk_cap = 0;
  double* blk_vstar = nullptr;           // blk_cap x 3P: each vector's momentum right-hand side
  double* blk_b = nullptr;               // blk_cap x Nc: divergences
  double* blk_phi = nullptr;             // blk_cap x Nc
  float* blk_phi32 = nullptr;            // blk_cap x Nc
  __nv_bfloat16* blk_xs[2] = {};         // 3 slices x blk_cap x xs_slice each: slice s of vector v at
                                         // s * blk_cap * xs_slice + v * xs_slice
  CUtensorMap blk_mapB[6], blk_mapB128[6];  // for the 256- and 128-column tiles
  // the fixed-point operator (kv_fixed.cu; uniform cubic mixed grids): the base state on its
  // fixed-point grid, the pre-pass maxima ([0] the input's, [1] the base state's), the constants
  int2* base_fx = nullptr;               // 4P
  unsigned int* fxmax = nullptr;         // 2
  unsigned short* fx_sel = nullptr;      // P, upwind advection: the one-sided choices per cell
  FxConst fxk{};
  bool fx_ok = false;                    // set per base flow by kv_fx_setup
  unsigned int* derr = nullptr;          // device error flag (bounded waits that expired)
  unsigned long long* rmax = nullptr;    // max |r| of the last refinement residual (bits)

  // launch counting (always) and per-phase CUDA-event timing (when profiling is on)
  long long launches[KV_NPHASE] = {};
  long long gs_steps = 0, gs_second = 0;  // Arnoldi steps, and of them those with the second update
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending { int phase; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  double prof_ms[KV_NPHASE] = {};
  long long prof_n[KV_NPHASE] = {};

  // CUDA graphs of kv_krylov_vector_batch, keyed by (X, Y, nb)
  struct GraphEntry {
    const double* X;
    double* Y;
    int nb;
    cudaGraphExec_t exec;
    long long launches[KV_NPHASE];
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap = nullptr;  // capture stream (the handle's stream may be the legacy one)

  // block shape of the linearised-operator kernel, chosen by timing (kv_autotune_apply)
  int apply_bx = 32, apply_by = 8;
  int df_variant = 0, df_bx = 32, df_by = 2;  // the mixed path's operator: 0, 1 double-float
                                              // (kv_stencil.cu), 2 fixed point (kv_fixed.cu)
  bool tuned = false;
  bool pinned = false;  // kv_set_tuning fixed the configuration: the autotuner does not run
  bool tile_pinned = false;  // kv_set_contraction_tile fixed the contractions' tile width

  std::string err;
};

// Phase timer: counts the launches of one phase and, with profiling on, brackets them with
// a pair of CUDA events on the handle's stream (resolved in kv_profile_get). Defined in kv_api.cu.
struct KvPhase {
  kv_grid* h;
  int phase, n;
  cudaEvent_t a = nullptr;
  KvPhase(kv_grid* h, int phase, int launches);
  ~KvPhase();
};

// kv_umma.cu
struct KvUmmaEpi {
  int mode;          // 0: BF16 slices of D; 1: slices of D / Lambda (Eq 17); 2: phi64 += D; 3: phi64 = D;
                     // 4: phi32 = D; 5: phi64 = phi32 + D
  int M, R;          // output rows / columns
  int nb, na;        // r = a * nb + b; output address (m * na + a) * pitch + b
  int pitch;         // padded fastest extent of the output layout
  size_t slice;      // elements between output slices
  __nv_bfloat16* out;
  double* phi;       // modes 2, 3, 5
  float* phi32;      // modes 4, 5
  const float* lz;   // mode 1: eigenvalues of the contracted (m) axis, then of a and b
  const float* la;
  const float* lb;
  unsigned int wait_limit;  // iterations of each bounded mbarrier wait (0: the default)
  unsigned int extra_tx;    // self-test only: bytes expected beyond what TMA delivers (0 normally)
  int nvec;                 // vectors contracted by the launch (block evaluations; 0 or 1: one)
  size_t vstride_out;       // elements between consecutive vectors' outputs within an output slice
  size_t vstride_phi;       // elements between consecutive vectors' phi (modes 2-5)
};
cudaError_t kv_umma_init();
bool kv_make_slice_map(CUtensorMap* map, const void* base, int cols, int rows, int pitch, size_t slice_elems,
                       int box_rows);
// The data operand's map: nvec vectors of `rows` x `cols` BF16 (row pitch `pitch`), vector v's rows
// `vec_elems` after vector v-1's, three slices `slice_elems` apart (a one-vector map for nvec = 1).
bool kv_make_data_map(CUtensorMap* map, const void* base, int cols, int rows, int pitch, int nvec, size_t vec_elems,
                      size_t slice_elems, int box_rows);
int kv_umma_box_rows_a();
int kv_umma_box_rows_b();  // rows of the data map's box for the default 256-column tile
// tile: output columns per tile, 256 (default) or 128; mapB's box must have that many rows
cudaError_t kv_launch_umma_axis(const CUtensorMap* mapA, const CUtensorMap* mapB, int K, const KvUmmaEpi& ep,
                                unsigned int* err, cudaStream_t s, int tile = 256);

// Three BF16 slices of r (r ~ s1 + s2 + s3 to about 2^-24 |r|) at offset o of slice buffers
// `slice` elements apart: the tensor-core solve's input format.
__device__ __forceinline__ void kv_store_bf16x3(__nv_bfloat16* xs, size_t slice, size_t o, float r) {
  const __nv_bfloat16 s1 = __float2bfloat16_rn(r);
  const float r1 = r - __bfloat162float(s1);
  const __nv_bfloat16 s2 = __float2bfloat16_rn(r1);
  const __nv_bfloat16 s3 = __float2bfloat16_rn(r1 - __bfloat162float(s2));
  xs[o] = s1;
  xs[slice + o] = s2;
  xs[2 * slice + o] = s3;
}

// kv_mixed.cu
kv_status kv_mixed_setup(kv_grid* h, const double* const fwd[3], const double* const inv[3]);
void kv_mixed_free(kv_grid* h);
// phi = L^+ b to FP64-class accuracy: BF16-split tensor-core TPF solve + double-float residual
// refinement (stats: also reduce max |r| into h->rmax)
// slices_ready: the BF16 slices of b are already in h->xs[0] (written by the divergence)
void kv_launch_poisson_mixed(kv_grid* h, const double* b, double* phi, int stats, int slices_ready, cudaStream_t s);
kv_status kv_mixed_selftest_timeout(kv_grid* h, int* device_error);
// The same solve for nb <= h->blk_cap vectors at once (h->blk_* buffers): the divergences have
// written each vector's b and BF16 slices; each of the 6 contractions per sweep is one launch for
// the whole block; the residuals run per vector.
kv_status kv_mixed_block_setup(kv_grid* h, int cap);
void kv_launch_poisson_mixed_block(kv_grid* h, int nb, cudaStream_t s);
void kv_mixed_block_free(kv_grid* h);

// kv_api.cu: sets the thread's message returned by kv_last_error(NULL)
void kv_set_thread_error(const std::string& msg);

// The SIMPLE tolerance of a grid: desc.tol, or the default of its precision. FP64 leaves
// max|D v| h_min / max|v| near 1e-14; the mixed path's two refinement sweeps leave about 1.4e-12
// at 256^3, where an unrefined tensor-core solve leaves about 1e-7.
inline double kv_simple_tol(const kv_grid* h) {
  return h->d.tol > 0 ? h->d.tol : (h->d.precision == KV_PREC_MIXED ? 1e-11 : 1e-12);
}

// kv_block.cu: Y_v = A X_v for v < nb <= h->blk_cap, mixed precision, with the block contractions
constexpr int KV_BLOCK_MAX = 16;
kv_status kv_krylov_block(kv_grid* h, const double* X, double* Y, int nb);

// kv_adjoint.cu
void kv_launch_adj_prep(const kv_grid* h, const double* y, double* vel, double* tout, cudaStream_t s);
void kv_launch_apply_t(const kv_grid* h, const double* coef, const double* yh, double* z, cudaStream_t s);
void kv_launch_grad_theta(const kv_grid* h, const double* x, const double* yT, double* gt, cudaStream_t s);
void kv_launch_lap_dot(const kv_grid* h, const double* x, const double* yh, double* sums, cudaStream_t s);
void kv_launch_grad_vel(const kv_grid* h, const double* x, const double* yh, double* gv, cudaStream_t s);

// kv_stencil.cu
// mode 0: y* = J P_BC x (Eqs (11)-(12)); mode 1: y* = F(S) (steady residual, x = base = S).
// Writes the three momentum fields (interior faces, zero elsewhere) to vstar and the
// projected temperature (all padded entries) to tout.
void kv_launch_stencil(const kv_grid* h, int mode, const double* base, const double* x, double* vstar,
                       double* tout, cudaStream_t s);

// Forms the assembled coefficients of J from the base state; then y* = J P_BC x from them.
void kv_launch_assemble(const kv_grid* h, const double* base, double* coef, cudaStream_t s);
void kv_launch_apply(const kv_grid* h, const double* coef, const double* x, double* vstar, double* tout,
                     cudaStream_t s);
// mixed precision: FP32-pair copy of the coefficients, and J P_BC x in double-float on the FP32 pipe
// (P_BC x is first split into h->xsplit)
void kv_launch_coef_df(const kv_grid* h, const double* coef, float2* cdf, cudaStream_t s);
// the padded-boundary entries of v* and T* (kv_stencil.cu)
void kv_launch_zero_boundary(const kv_grid* h, double* vstar, double* tout, cudaStream_t s);
// kv_fixed.cu
bool kv_fx_eligible(const kv_grid* h);
kv_status kv_fx_setup(kv_grid* h);
void kv_fx_free(kv_grid* h);
void kv_launch_apply_fx(const kv_grid* h, const double* x, double* vstar, double* tout, int kc, cudaStream_t s);
void kv_launch_apply_df(const kv_grid* h, const float2* cdf, const double* x, double* vstar, double* tout,
                        cudaStream_t s);

// kv_project.cu
void kv_launch_divergence(const kv_grid* h, const double* vel, double* b, cudaStream_t s);
// as kv_launch_divergence, with the mixed path's BF16 slices of b written to xs (slices `slice` apart)
void kv_launch_divergence_to(const kv_grid* h, const double* vel, double* b, __nv_bfloat16* xs, size_t slice,
                             cudaStream_t s);
// out_vel = vstar - G phi on interior faces (0 elsewhere); p (nullable) = phi (+ p if accumulate);
// with check != 0 also reduces max |D out_vel| and max |out_vel| into h->red (the SIMPLE test).
void kv_launch_correct(const kv_grid* h, const double* vstar, const double* phi, double* out_vel,
                       double* p, int accumulate_p, cudaStream_t s, int check = 1);
// Closes one SIMPLE test on the device: reads h->guard->red, stores the pass's figures in
// guard->last_*, counts the check when record != 0 (failed: rel >= tol; nonfinite: NaN or Inf),
// and clears red.
void kv_launch_guard_close(const kv_grid* h, double tol, int record, cudaStream_t s);

// kv_tpd.cu: phi = L^+ b by Eq (18), six per-axis contractions; b and phi compact n^3
// (x fastest). b is overwritten (used as scratch).
void kv_launch_poisson(kv_grid* h, double* b, double* phi, cudaStream_t s);

// kv_reduce.cu
// partial sums of <V_q, w> for q = 0..nq-1 (vectors of length len, stride between V_q = ld),
// then out[q] = sum of partials. If accumulate, out[q] += result.
int kv_reduce_blocks();
// out[r] = sum of the nb block partials of row r (rows laid out kv_reduce_blocks() apart)
void kv_launch_finalize(const double* partials, int rows, int nb, double* out, cudaStream_t s);
// kv_dcgs.cu: the sweeps of the delayed classical Gram-Schmidt (kv_arnoldi_run), in chunks of
// kv_dcgs_chunk() basis vectors. Inner products of the basis V_0..V_{q-1} with two vectors u and
// w: chunk c (from vector c kv_dcgs_chunk() on) at dots + c kv_dcgs_dots_stride() holds [<V, u>, <V, w>, <u, w>,
// ||u||^2 (NaN if a double-float sweep meets an entry of u or w outside its range), ||w||^2];
// partials: (2 kv_dcgs_chunk() + 3) kv_reduce_blocks() doubles (reused chunk by chunk).
int kv_dcgs_chunk();
int kv_dcgs_dots_stride();
void kv_launch_dots2(const double* V, size_t ld, int q, const double* u, const double* w, size_t len,
                     double* partials, double* dots, int df, cudaStream_t s);
// The coefficients of a step from those inner products and the Hessenberg matrix Hd (device,
// column-major, leading dimension ldh): column j-1 finalised (unless first), column j
// provisional; s3, cuv, cwv for kv_launch_update2. final_only: column j-1 and v_j only (the
// run's last vector; the inner products from kv_launch_dots2 with w = u). scr: 2 (j + 1)
// doubles. err: set on a failure.
void kv_launch_dcgs_coef(const double* dots, double* Hd, int ldh, int j, int first, int final_only, double* s3,
                         double* cuv, double* cwv, double* scr, int* err, cudaStream_t s);
// u <- s3[0] u + sum_q cuv_q V_q (if write_u), w <- s3[1] w + s3[2] u + sum_q cwv_q V_q (if
// write_w), both from the entering u; chunks after the first use one3 = (1, 1, 0).
void kv_launch_update2(const double* V, size_t ld, int q, const double* s3, const double* one3, const double* cuv,
                       const double* cwv, double* u, double* w, size_t len, int write_u, int write_w, int df,
                       cudaStream_t s);
void kv_launch_multidot(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                        double* out, int accumulate, cudaStream_t s);
// w -= sum_q c[q] V_q
void kv_launch_update(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                      cudaStream_t s);
// out[0] = ||w||^2 (via partials)
void kv_launch_norm2(const double* w, size_t len, double* partials, double* out, cudaStream_t s);
// Gram-Schmidt building blocks for nq <= kv_fused_cgs_max() vectors (one sweep each):
// h[q] = <V_q, w> (and h[nq] = ||w||^2 when nrm2 != nullptr, copied to nrm2);
// w -= V c fused with h2[q] = <V_q, w> and h2[nq] = ||w||^2 (FP64);
// w = (w - V c) / sqrt(c[nq] - ||c||^2) for rounding-size c = V^T w (product in FP32).
// df != 0 forms the first two sweeps in double-float arithmetic on the FP32 pipe (relative
// rounding ~2^-46; entries of w at or above 2^48 make h[nq] NaN).
int kv_fused_cgs_max();
void kv_launch_dots_norm(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                         double* h, double* nrm2, int df, cudaStream_t s);
void kv_launch_update_dot(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                          double* partials, double* h2, int df, cudaStream_t s);
void kv_launch_update_small_scale(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                                  cudaStream_t s, const int* flag = nullptr);
// The second-update decision of the fused Gram-Schmidt step on the device: from h1 (first pass,
// h1[nq] = ||w||^2 before it) and h2 (second pass, h2[nq] = ||w||^2 after the first update),
// *flag = force || ||h2||^2 > theta^2 ||w||^2, and hcol[0..nq] = the Hessenberg column that
// kv_launch_update_small_scale (given flag) then produces.
void kv_launch_gs_decide(const double* h1, const double* h2, int nq, double theta, int force, double* hcol,
                         int* flag, cudaStream_t s);
// The same sweeps for any basis size: inner products in chunks of at most kv_fused_cgs_max()
// vectors (h[q], and h[nq] = ||w||^2 when nrm); w -= V c over all vectors (df: FP64 for about
// 3 (nq + 2) / 10 of them, double-float for the others; else FP64); and the third sweep
// (flag-controlled, as kv_launch_update_small_scale).
void kv_launch_dots_chunked(const double* V, size_t ld, int nq, const double* w, size_t len, double* partials,
                            double* h, int nrm, int df, cudaStream_t s);
void kv_launch_update_n(const double* V, size_t ld, int nq, const double* c, double* w, size_t len, int df,
                        cudaStream_t s);
void kv_launch_update_small_scale_n(const double* V, size_t ld, int nq, const double* c, double* w, size_t len,
                                    cudaStream_t s, const int* flag);
