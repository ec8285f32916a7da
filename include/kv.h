/*
 * kv.h -- C ABI of the GB300 (sm_103a) Krylov-vector library.
 *
 * The library evaluates one Krylov vector of the Newton / Arnoldi stability method of
 * Gelfgat, arXiv 1905.11601, Section 3.1, for natural convection in a laterally heated
 * cube: for a steady state (U, Theta) and a vector x = (u, v, w, T) it computes
 *
 *     y = (Pi_v (+) P_T) J(U, Theta) P_BC x
 *
 *   P_BC  puts x into the constrained space of Eq (13) (velocity zero outside the interior
 *         faces, temperature projected onto the homogeneous boundary conditions);
 *   J     is the right-hand side of Eqs (11)-(12) without the pressure gradient, i.e. the
 *         linearised operator of Eqs (8)-(9);
 *   Pi_v  is the SIMPLE / Chorin velocity projection of Section 3.1 (Poisson equation for
 *         the pressure correction solved by the tensor-product factorisation, Eqs (14)-(18));
 *   P_T   is the temperature projection of Eqs (19)-(21).
 *
 * Grid and memory layout (shared by every array argument):
 *   - uniform staggered (MAC) grid of the unit cube with nx, ny, nz cells, h_a = 1 / n_a;
 *   - every field is a padded array of (nx+2)*(ny+2)*(nz+2) doubles, x fastest, element
 *     (i, j, k) at i + (nx+2) * (j + (ny+2) * k);
 *   - T and p sit at cell centres (cell index 1..n, wall nodes 0 and n+1 on the walls);
 *     u / v / w sit on x / y / z faces (face index 0..n along their own axis, index n+1
 *     unused) and are cell-like along the other two axes;
 *   - a "packed vector" is four consecutive fields u | v | w | T (4 * field_len doubles);
 *     a packed state U | V | W | Theta has the same layout.
 *
 * Ownership: every pointer argument is owned by the caller and never freed by the library.
 * Unless a function says otherwise, array pointers are DEVICE pointers (cudaMalloc'ed or
 * from torch) on the current device, and the work is queued on the handle's stream
 * (stream-ordered, asynchronous). Functions that return a host scalar synchronise that stream.
 *
 * Errors: functions return KV_OK or a negative kv_status; nothing is thrown across the ABI.
 * kv_last_error() returns a message for the last failed call on a handle (or, for a NULL
 * handle, for the last failed kv_create_grid on this thread).
 */
#ifndef KV_H
#define KV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kv_grid* kv_handle;

typedef enum {
  KV_OK = 0,
  KV_ERR_ARG = -1,           /* invalid argument (NULL pointer, size, enum value) */
  KV_ERR_CUDA = -2,          /* a CUDA call or kernel launch failed */
  KV_ERR_NOT_CONVERGED = -3, /* SIMPLE / refinement did not reach the tolerance */
  KV_ERR_STATE = -4,         /* call out of order (e.g. no base flow set) */
  KV_ERR_NOMEM = -5          /* device allocation failed */
} kv_status;

/* Spanwise thermal boundary conditions (Section 2). */
enum { KV_BC_CC = 0 /* conducting, Eq (6) */, KV_BC_AA = 1 /* insulated, Eq (7) */ };

/* Readings of the temperature projection Eq (21) at insulated walls (identical on the
   conducting walls): orthogonal = Gram-matrix projection onto the boundary-condition
   subspace (wall pair replaced by its mean); oblique = interior kept, wall node set from
   the condition. */
enum { KV_TPROJ_ORTHOGONAL = 0, KV_TPROJ_OBLIQUE = 1 };

/* Advection scheme of the linearised operator and the residual. Central: the derivative of
   the advected field is the 3-point central difference at its node (non-uniform next to a
   wall node), times the advecting velocity averaged to the node (Section 3's discretisation).
   Upwind (an option, not from the paper): along each axis the derivative is the one-sided
   difference towards the upstream neighbour, over the node gap (h/2 to a wall node), chosen
   by the sign of the base velocity's component averaged to the node (>= 0: backward; the
   4-point averages summed in the order (t-1 along the velocity's axis, then t; within each,
   t and t+1 along the node's face axis)). The linearisation keeps the base velocity's choice
   in both (U.grad)v and (v.grad)U, so it is the derivative of the upwind residual wherever no
   averaged base velocity is zero. */
enum { KV_ADV_CENTRAL = 0, KV_ADV_UPWIND = 1 };

/* Arithmetic of the Krylov-vector evaluation. FP64: every step in FP64. MIXED: the
   pressure-correction Poisson solve runs its per-axis contractions on the tensor cores
   (BF16 slices, FP32 accumulation) and is refined to FP64 accuracy with an FP64 residual;
   the other steps stay FP64. */
enum { KV_PREC_FP64 = 0, KV_PREC_MIXED = 1 };

typedef struct {
  int nx, ny, nz;    /* cells per axis, each >= 2 and <= 1024 */
  int spanwise_bc;   /* KV_BC_CC or KV_BC_AA */
  int tproj;         /* KV_TPROJ_ORTHOGONAL or KV_TPROJ_OBLIQUE */
  int precision;     /* KV_PREC_FP64 or KV_PREC_MIXED */
  double gr, pr;     /* Grashof and Prandtl numbers, > 0 */
  double tol;        /* SIMPLE stop: max|D v| * h_min / max|v| < tol (0 -> 1e-12 for KV_PREC_FP64,
                        1e-11 for KV_PREC_MIXED) */
  int max_passes;    /* SIMPLE passes at most (0 -> 1: one exact pass, residual reported) */
  int refine_sweeps; /* KV_PREC_MIXED: tensor-core solves per Poisson solve, each followed by an
                        FP64 residual (0 -> 2) */
  int cgs_passes;    /* kv_arnoldi_step: 0 = classical Gram-Schmidt whose second pass measures the
                        remaining components h2 = V^T w (fused with the first update) and applies
                        w -= V h2 only when ||h2|| exceeds the sweeps' rounding level (2^-46 ||w||
                        for KV_PREC_MIXED's double-float sweeps, 2^-50 ||w|| in FP64); 2 = always
                        apply it */
  double stretch;    /* grid stretching of Eq (22), Section 3.2: the faces of every axis sit at
                        x = xi - stretch sin(2 pi xi), xi = t/n; cell centres at the midpoints of
                        their faces. 0 = uniform grid; must be in [0, 1/(2 pi)) so the mapping stays
                        monotone (the paper uses up to 0.12). Both precisions; a stretched
                        KV_PREC_MIXED grid stores 12 more coefficient pairs per point (its operator
                        reads the plus-neighbour coefficients instead of rebuilding them). The
                        transpose, the base-flow gradient and kv_krylov_vector_noalloc take the
                        uniform grid only. */
  int advection;     /* KV_ADV_CENTRAL (0, the paper's discretisation) or KV_ADV_UPWIND: first-order
                        upwind derivatives in the advection terms of Eqs (8)-(9) and of the
                        residual of Eqs (1)-(2). Upwind takes the uniform grid only. A KV_PREC_MIXED
                        upwind grid keeps 2 B of one-sided choices per point for the fixed-point
                        operator (cubic grids) and stores 12 more coefficient pairs per point, as a
                        stretched one does, for the double-float operator. kv_base_flow_gradient
                        and kv_krylov_vector_noalloc take central advection only. */
} kv_grid_desc;

typedef struct {
  int passes;       /* SIMPLE passes performed */
  double max_div;   /* max |D v| after the last pass (absolute; the paper's pointwise test) */
  double rel_div;   /* max |D v| * h_min / max |v| */
  double refine_residual; /* KV_PREC_MIXED: max |b - L phi| before the last tensor-core sweep */
  int device_error; /* nonzero: a bounded wait inside a tensor-core kernel expired */
} kv_stats;

/* Creates a grid: validates desc, builds the per-axis eigen-decompositions of Eq (15)
   (computed once, Section 3.1; closed form on the uniform grid, a symmetric tridiagonal QL
   iteration on a stretched one, KV_ERR_NOT_CONVERGED if it fails) and allocates the library's
   device storage (base flow, Poisson scratch; a stretched grid adds 14 (n_a + 2) doubles of
   per-axis weights). stream: a cudaStream_t (NULL = legacy default stream). */
kv_status kv_create_grid(const kv_grid_desc* desc, void* stream, kv_handle* out);

/* Frees all device storage of the handle. NULL is accepted. */
kv_status kv_destroy_grid(kv_handle h);

/* Changes the stream later calls are queued on. */
kv_status kv_set_stream(kv_handle h, void* stream);

/* Number of doubles in one padded field, (nx+2)(ny+2)(nz+2). */
kv_status kv_field_len(kv_handle h, size_t* field_len);

/* Layout query: the number of doubles in each padded field of a vector, u (x-faces), v (y-faces),
   w (z-faces) and a cell field (T, p). All four use the one padded layout above, so all four are
   (nx+2)(ny+2)(nz+2); a packed vector is their concatenation. Any output may be NULL (not all). */
kv_status kv_field_sizes(kv_handle h, size_t* u, size_t* v, size_t* w, size_t* cell);

/* Copies the steady state that Eqs (8)-(9) are linearised about (Section 3.1: the Jacobian at the
   current Newton iterate or at the converged flow) into library storage: U, V, W (velocity on
   the x/y/z faces) and Theta (temperature at the cells, with its wall values, Eqs (4)-(7)); four
   device pointers to padded fields, read on the handle's stream and not kept. Also forms the
   coefficients of the linearised operator for this state (37 padded fields: 15 per velocity
   face, 13 per cell plus the fixed buoyancy weights), so that each Krylov vector is a
   fixed-coefficient 15/13-point product; a grid therefore holds about (4 + 37 + 3) padded
   fields plus two n^3 buffers of device memory. In KV_PREC_MIXED it adds 25 coefficient fields
   as FP32 pairs and, on uniform grids with nx = ny = nz, the base state on the fixed-point
   operator's grid (4 padded fields of 8 bytes; its scale is read back to the host, so the call
   synchronises the stream). The first call on a handle also runs the autotuner (unless
   kv_set_tuning fixed the configuration). Not for use inside a stream capture. */
kv_status kv_set_base_flow(kv_handle h, const double* U, const double* V, const double* W, const double* Theta);

/* As kv_set_base_flow, for a packed state U | V | W | Theta (one device pointer, 4 padded
   fields), the layout kv_newton and the state vectors of the solvers use. */
kv_status kv_set_base_flow_packed(kv_handle h, const double* base);

/* One Krylov vector (Eqs (11)-(13), Section 3.1): y = (Pi_v (+) P_T) J P_BC x.
   x, y: packed vectors (device, must not overlap). p: optional padded cell field that
   receives the pressure correction sum(phi) (zero mean, walls zero); may be NULL.
   Every pass evaluates the SIMPLE stopping test of Section 3.1 (max|D v| h_min / max|v| < tol)
   on the device. With desc.max_passes <= 1 and st == NULL the call does not synchronise: the
   test's outcome is accumulated in the grid's guard (kv_guard_read). With st, or with
   desc.max_passes > 1 (the literal loop: repeat while the test fails), the call synchronises
   the stream after each pass to read it and returns KV_ERR_NOT_CONVERGED when the literal loop
   ends above tol (y and p then hold the last pass), and KV_ERR_ARG when the velocity or its
   divergence is not finite (NaN or Inf in x or in the base flow; y is then undefined). */
kv_status kv_krylov_vector(kv_handle h, const double* x, double* y, double* p, kv_stats* st);

/* The device-side SIMPLE test of the one-pass evaluations (desc.max_passes <= 1) since the grid
   was created or last reset: every projection of the grid counts (Krylov vectors, also inside
   the batched, plan, host-buffer and solver calls; Newton residuals; the transpose's input
   projection). failed: tests at or above tol with finite values; nonfinite: NaN or Inf in the
   velocity or its divergence; worst_rel_div: the largest finite max|D v| h_min / max|v|. */
typedef struct {
  long long checks;
  long long failed;
  long long nonfinite;
  double worst_rel_div;
} kv_guard;

/* Synchronises the stream and copies the guard into *out (host); reset != 0 then clears it. */
kv_status kv_guard_read(kv_handle h, kv_guard* out, int reset);

/* As kv_krylov_vector, with x and y in HOST memory (pinned or pageable); the host-device
   copies are queued on the handle's stream and the call returns once y is in host memory. */
kv_status kv_krylov_vector_host(kv_handle h, const double* x_host, double* y_host, kv_stats* st);

/* A sequence of Krylov vectors between host buffers: Y_i = A X_i for i = 0..nb-1 (X_host,
   Y_host: nb consecutive packed vectors in host memory, page-locked for the copies to overlap).
   The same map as kv_krylov_vector, evaluated in order on the handle's stream from two device
   staging slots (4 packed vectors, allocated at the first call and kept by the handle), with the
   host-to-device copy of X_{i+1} and the device-to-host copy of Y_{i-1} on two copy streams of
   the handle, overlapping the evaluation of X_i (Section 3.1's many Krylov vectors per Newton or
   Arnoldi run come from the host in this form when they do not fit the device). Returns once
   every Y_i is in host memory; results equal nb calls of kv_krylov_vector_host. nb = 0 does
   nothing; KV_ERR_STATE without a base flow. */
kv_status kv_krylov_vector_host_stream(kv_handle h, const double* X_host, double* Y_host, int nb);

/* A block of Krylov vectors: Y_b = A X_b for b = 0..nb-1 (X, Y: nb consecutive packed vectors,
   device, not overlapping). The evaluation sequence is captured once into a CUDA graph, cached
   per (X, Y, nb) on the handle (up to 8 entries), and replayed with one graph launch on the
   handle's stream; results equal nb calls of kv_krylov_vector. Requires desc.max_passes <= 1
   (the graph contains no host-side SIMPLE test). The first call for a (X, Y, nb) captures, so
   make it outside any capture of your own. */
kv_status kv_krylov_vector_batch(kv_handle h, const double* X, double* Y, int nb);

/* Multi-grid plans: several grids (sizes, Grashof numbers, boundary types) evaluated by one
   graph launch. kv_plan_add queues y = A_h x for the grid h (its base flow must be set); the
   first kv_plan_launch captures every queued evaluation into one CUDA graph with one parallel
   branch per grid (evaluations of the same grid stay in order, since they share its scratch),
   later launches replay it on `stream` (cudaStream_t). Plans are immutable after the first
   launch. A plan does not own the grids; destroy the plan before its grids. */
typedef struct kv_plan* kv_plan_handle;
kv_status kv_plan_create(kv_plan_handle* out);
kv_status kv_plan_add(kv_plan_handle p, kv_handle h, const double* x, double* y);
kv_status kv_plan_launch(kv_plan_handle p, void* stream);
kv_status kv_plan_destroy(kv_plan_handle p);
const char* kv_plan_last_error(kv_plan_handle p);

/* One Arnoldi step (Section 3.1, the Krylov basis for the eigenvalue problem Eq (10)):
   V holds at least j+2 packed vectors (device), V_0..V_j orthonormal; computes
   w = A V_j, orthogonalises it against V_0..V_j by classical Gram-Schmidt (the second pass's
   correction when its measured coefficients exceed the rounding level, or always:
   desc.cgs_passes),
   stores w / ||w|| in V_{j+1} and writes the Hessenberg column H[0..j+1, j] to the HOST
   array h_col (j+2 doubles). Synchronises the stream. Inner products run over all stored
   entries of the four fields. With KV_PREC_MIXED and up to 24 basis vectors, the first two
   Gram-Schmidt sweeps run in double-float arithmetic on the FP32 pipe (relative rounding
   ~2^-46 instead of 2^-53); entries below 2^-103 in magnitude are then treated as 0, and a new
   vector with an entry of magnitude >= 2^48, NaN or Inf gives KV_ERR_ARG (V_{j+1} undefined).
   The decision on the second update is taken on the device and the step synchronises once, to
   return h_col. Up to 24 basis vectors the first update is fused with the second pass's inner
   products; beyond, the inner products run in chunks of 24 vectors and the update (in
   KV_PREC_MIXED on both the FP64 and FP32 pipes) is a sweep of its own. */
kv_status kv_arnoldi_step(kv_handle h, double* V, int j, double* h_col);

/* m Arnoldi steps in one call (Section 3.1; the same basis and Hessenberg matrix as m calls of
   kv_arnoldi_step with classical Gram-Schmidt applied twice, up to rounding), with the second
   projection of each new vector deferred to the next step, where it shares that step's sweeps
   over the basis (delayed classical Gram-Schmidt, after Swirydowicz et al., "Low
   synchronization Gram-Schmidt and generalized minimal residual algorithms", 2021): two sweeps
   over the basis per step instead of two to three. V holds at least j0 + m + 1 packed vectors
   (device), V_0..V_{j0} orthonormal on entry; on return V_0..V_{j0+m} are orthonormal. The
   Arnoldi operator is applied to each new vector before its second projection and
   normalisation (A is linear; the corrections use the Arnoldi relation of the final columns).
   H: HOST, column-major, leading dimension ldh >= j0 + m + 1. Columns 0..j0-1 (rows 0..c+1)
   are read: the Hessenberg matrix of the basis V_0..V_{j0} (needed by the deferred corrections);
   columns j0..j0+m-1 (rows 0..c+1) are written. Requires j0 >= 0, m >= 1 and j0 + m <= 4096
   (else KV_ERR_ARG); the sweeps take the basis in chunks of 24 vectors. Synchronises the stream
   once, at the end. KV_PREC_MIXED: the sweeps' arithmetic as kv_arnoldi_step's double-float sweeps (FP64
   for the first basis vectors of each sweep, double-float for the rest); a vector with an entry
   of magnitude >= 2^48, NaN or Inf, or one in the span of the basis, gives KV_ERR_ARG (V and H
   undefined). While the call runs, V_{j+1} holds intermediate vectors. */
kv_status kv_arnoldi_run(kv_handle h, double* V, int j0, int m, double* H, int ldh);

/* Transpose of the Krylov map: z = A^T y with A = (Pi_v (+) P_T) J P_BC (the adjoint eigenvalue
   problem of Eq (10) uses it). With the orthogonal reading of Eq (21) the three projections are
   symmetric, so A^T = P_BC J^T (Pi_v (+) P_T); J^T is applied from the same assembled
   coefficients as J (either advection scheme). y, z: packed vectors (device, must not overlap). Requires
   KV_TPROJ_ORTHOGONAL and the uniform grid (else KV_ERR_ARG: on a stretched grid Pi_v is
   symmetric only in the volume-weighted product) and a base flow (else KV_ERR_STATE). */
kv_status kv_krylov_vector_adjoint(kv_handle h, const double* y, double* z);

/* Sensitivity of <y, A x> to the base state and the Grashof number (with y the adjoint and x
   the direct eigenvector this gives the sensitivity of an eigenvalue of Eq (10)):
   g_base (device, packed U | V | W | Theta layout, nullable) = d<y, A x>/d(U, V, W, Theta):
   the velocity part from the advecting velocities and the velocity gradients of Eqs (8)-(9),
   the Theta part from the term -(v . grad) Theta of Eq (8); dgr (host, nullable) =
   d<y, A x>/d Gr, from the scalings Gr^-1/2 and (Pr Gr^1/2)^-1 of Eqs (1)-(2). x, y: packed
   vectors (device). Synchronises the stream when dgr is given. Same requirements as
   kv_krylov_vector_adjoint, and central advection (KV_ERR_ARG with KV_ADV_UPWIND, for which
   the operator is not affine in the base state). */
kv_status kv_base_flow_gradient(kv_handle h, const double* x, const double* y, double* g_base, double* dgr);

/* Newton step 2 of Section 3.1: the steady residual of Eqs (1)-(2) at the packed state S
   (device; carries its own inhomogeneous wall values, Eqs (4)-(7)), projected like a
   Krylov vector (the pressure gradient drops out). F: optional packed output (device);
   norm_out: optional HOST pointer receiving ||F||_2 (synchronises the stream). */
kv_status kv_newton_residual(kv_handle h, const double* S, double* F, double* norm_out);

/* ---- Newton-Krylov: the method's steps either side of the path ----------------------------
   Section 2 (Newton steps 1-4) and Section 3.1: the Jacobian systems are solved by GMRES
   restarted after every m Krylov vectors (m = 100 in the paper) until it saturates, then by
   BiCGstab(2) from GMRES's last approximation. The products with the Jacobian are
   kv_krylov_vector at the handle's base flow (A = projected J, Eqs (11)-(13)), so b, x and
   every vector below are packed vectors (device) in the space of Krylov vectors. Solvers:
   GMRES(m) of Saad and Schultz (1986); BiCGstab(l) of Sleijpen and Fokkema (1993), l = 2 (the
   paper defers both to its reference [17]). The host drives the iterations; every call
   synchronises the stream. */
typedef struct {
  int iterations;      /* GMRES: Arnoldi steps in all cycles; BiCGstab(2): iterations (two BiCG
                          steps = 4 Krylov vectors, then the minimal-residual update) */
  int restarts;        /* GMRES: cycles run */
  int matvecs;         /* Krylov-vector evaluations (products with A) */
  int converged;       /* rel_residual <= tol */
  int saturated;       /* GMRES: stopped because a cycle began with a residual above sat times
                          the previous cycle's */
  int breakdown;       /* BiCGstab(2): stopped on a zero or non-finite denominator; x is the last
                          complete iterate */
  double rel_residual; /* ||b - A x|| / ||b|| of the returned x, recomputed */
} kv_solve_stats;

/* Restarted GMRES(m) for A x = b, starting from x (in-out). V: caller-owned device workspace of
   m + 1 packed vectors (the Arnoldi basis; kv_arnoldi_step builds it). A cycle starts from
   r = b - A x, stops early once the Givens-rotated least-squares residual is at most tol ||b||,
   and adds the minimiser V y to x. Cycles repeat until converged, saturated (the cycle's starting
   residual above sat times the previous cycle's; the paper's hand-over to BiCGstab(2)) or
   max_restarts cycles. b = 0 gives x = 0. st (host, nullable) receives the statistics.
   KV_ERR_ARG for NULL or overlapping vectors, m outside 1..4095, max_restarts < 1, tol < 0,
   sat <= 0; KV_ERR_STATE without a base flow. */
kv_status kv_gmres(kv_handle h, const double* b, double* x, double* V, int m, int max_restarts, double tol,
                   double sat, kv_solve_stats* st);

/* BiCGstab(2) for A x = b, starting from x (in-out), shadow residual = the initial residual.
   work: caller-owned device workspace of 8 packed vectors. Stops when ||r|| <= tol ||b||, after
   max_iter iterations, or on a breakdown (see kv_solve_stats). b = 0 gives x = 0. Errors as
   kv_gmres. */
kv_status kv_bicgstab2(kv_handle h, const double* b, double* x, double* work, int max_iter, double tol,
                       kv_solve_stats* st);

/* Vector operations of the Krylov solvers and the eigenvalue driver, on packed vectors
   (device), stream-ordered: y = a x + b y (x may be y; b = 0 does not read y; a, b finite) and
   y = sum_{i<k} c[i] V_i (V: k consecutive packed vectors, c: HOST array of k finite values;
   y outside V; synchronises the stream). KV_ERR_ARG for NULL or overlapping vectors. */
kv_status kv_axpby(kv_handle h, double a, const double* x, double b, double* y);
kv_status kv_combine(kv_handle h, const double* V, int k, const double* c, double* y);
/* *out (HOST) = <x, y> over the packed entries (FP64; synchronises the stream). */
kv_status kv_dot(kv_handle h, const double* x, const double* y, double* out);

#define KV_NEWTON_HISTORY 64
typedef struct {
  int max_newton;         /* Newton corrections at most (0..KV_NEWTON_HISTORY - 1) */
  double tol;             /* stop once ||F(S)|| < tol (the projected residual, as kv_newton_residual) */
  int gmres_m;            /* Krylov vectors per GMRES cycle (the paper: 100) */
  int gmres_max_restarts; /* GMRES cycles per Newton step at most */
  double lin_tol;         /* relative residual of each linear solve */
  double gmres_sat;       /* GMRES saturation factor (e.g. 0.99) */
  int bicg_max_iter;      /* BiCGstab(2) iterations after an unconverged GMRES (0: none) */
} kv_newton_params;

typedef struct {
  int iterations;      /* Newton corrections applied */
  int matvecs;         /* Krylov-vector evaluations in the linear solves */
  int gmres_restarts;  /* GMRES cycles in all */
  int bicg_iterations; /* BiCGstab(2) iterations in all */
  int bicg_rejected;   /* BiCGstab(2) corrections not taken (recomputed residual not below GMRES's, or the
                          Newton step with it did not decrease ||F||) */
  int converged;       /* ||F(S)|| < tol at exit */
  int n_res;           /* entries of res_norm */
  double res_norm[KV_NEWTON_HISTORY]; /* ||F|| at the start of each Newton step */
} kv_newton_stats;

/* Newton's method (Section 2, steps 1-4) for the steady state S (device packed state, in-out,
   with its inhomogeneous wall values, which the corrections leave unchanged): F = the projected
   residual of S; stop once ||F|| < tol; set the base flow to S (the Jacobian at S) and solve
   A d = F with kv_gmres from d = 0, then kv_bicgstab2 from GMRES's result if GMRES did not
   converge, keeping the correction with the smaller recomputed residual (BiCGstab(2)'s only if
   the step with it also does not increase ||F||); S <- S - d. V: m + 1 packed vectors; work: 10 packed vectors (device, caller-owned).
   Leaves the handle's base flow at the last S that took a correction. st: host, nullable.
   KV_ERR_ARG for NULL or overlapping buffers or parameters outside their ranges. */
kv_status kv_newton(kv_handle h, double* S, double* V, double* work, const kv_newton_params* prm,
                    kv_newton_stats* st);

/* Instrumentation (not part of the method): launch counts per phase, always kept, and, when
   enabled, per-phase CUDA-event timings on the handle's stream. Phases: 0 = linearised
   operator stencil, 1 = divergence, 2 = TPF Poisson contractions (one timing per per-axis
   contraction launch), 3 = velocity correction, 4 = Arnoldi normalisation (and third
   Gram-Schmidt sweep), 5 = refinement residuals of the mixed-precision Poisson solve,
   6 = first Gram-Schmidt sweep (inner products), 7 = fused update + second-pass inner products.
   kv_profile_enable synchronises the stream and clears all counters. */
kv_status kv_profile_enable(kv_handle h, int on);
/* Synchronises the stream; total_ms / timed_launches: summed event time and number of timed
   brackets of the phase since the last kv_profile_enable; launches: kernels launched. Each
   output pointer (host) may be NULL. */
kv_status kv_profile_get(kv_handle h, int phase, double* total_ms, long long* timed_launches,
                         long long* launches);

/* The configuration the autotuner chose at the first kv_set_base_flow (cfg: host array of 5
   ints): cfg[0] x cfg[1], the FP64 operator's thread block; for KV_PREC_MIXED the operator:
   cfg[2] = 0 (double-float, split pass, then cfg[3] cells x cfg[4] rows of cells per block), 1
   (double-float 2.5D march, cfg[4] z-planes per block) or 2 (fixed-point 2.5D march from the base
   state, cfg[4] z-planes per block; uniform cubic grids); cfg[2..4] = -1 for KV_PREC_FP64.
   KV_ERR_STATE before the first base flow. */
kv_status kv_tuning(kv_handle h, int* cfg);

/* Fixes the operator configuration instead of timing the candidates (not part of the method: it
   lets every compiled variant be run and checked deterministically). cfg (host, 5 ints) as
   kv_tuning: cfg[0] x cfg[1] the FP64 operator's block (each >= 1, product <= 256 and a multiple
   of 32); for KV_PREC_MIXED, cfg[2] = 0 with cfg[3] in {32, 64, 128} cells and cfg[4] rows
   (cfg[3] x 4 x cfg[4] <= 512), or cfg[2] = 1 or 2 with cfg[4] in 1..1024 planes per block (only
   for grids whose packed vector has fewer than 2^31 doubles; 2 only on uniform grids with
   nx = ny = nz, and on a base flow with a non-finite value it runs as 1); cfg[2..4] are ignored
   for KV_PREC_FP64. Takes effect for the next evaluation; the autotuner does not run afterwards.
   KV_ERR_ARG for values outside these ranges. */
kv_status kv_set_tuning(kv_handle h, const int* cfg);

/* The tile width of the mixed path's tensor-core contractions (Eqs (14)-(18), kv_umma): output
   columns per tile, 256 or 128. The autotuner times both at the first kv_set_base_flow (one
   mixed Poisson solve each) unless this call or kv_set_tuning fixed the configuration;
   narrower tiles give more tiles per contraction, which fills 152 SMs better on small grids.
   KV_ERR_ARG for another width or a KV_PREC_FP64 grid. kv_contraction_tile reads it (host
   pointer; -1 for KV_PREC_FP64). */
kv_status kv_set_contraction_tile(kv_handle h, int columns);
kv_status kv_contraction_tile(kv_handle h, int* columns);

/* Instrumentation: Arnoldi steps since the last kv_profile_enable, and of them those that applied
   the second Gram-Schmidt update. Host pointers, each nullable. */
kv_status kv_arnoldi_counts(kv_handle h, long long* steps, long long* second_updates);

/* Allocation-free Krylov vector, for callers that cannot allocate device memory (code that
   runs under an allocator it does not own, inside a fixed memory budget, or in a plug-in that
   may not call cudaMalloc / cudaFree). The paper has no counterpart: it is a deployment
   variant of kv_krylov_vector in FP64 (one exact SIMPLE pass), computing the same y from a
   grid descriptor, a packed base state, x and y, all caller-owned device pointers; no handle
   is created. Its scratch is a fixed __device__ array of about 1.5 MB that every GPU loading
   the library keeps until the process exits, which limits the grid to
   KV_NOALLOC_MAX_N cells per axis; larger grids, a stretched grid, upwind advection and
   desc->precision != KV_PREC_FP64 return KV_ERR_ARG (message via kv_last_error(NULL)), as do
   x or base overlapping y. The per-axis tables of Eq (15) are written into the array by a
   kernel on `stream` at every call. The first call on a device looks up the array's device
   address (set-up); make that first call before any stream capture. All calls share the one
   array and it keeps the last call's contents, so calls that overlap on the GPU (other streams,
   other host threads) race: serialise them. stream: cudaStream_t. */
#define KV_NOALLOC_MAX_N 32
kv_status kv_krylov_vector_noalloc(const kv_grid_desc* desc, const double* base, const double* x, double* y,
                                   void* stream);

/* Failure-detection self-test (not part of the method): runs one tensor-core contraction of a
   KV_PREC_MIXED grid whose completion barriers expect more bytes than its copies deliver, so
   every bounded wait in the kernel expires (after a few hundred tries) and the kernel returns
   with its device error flag set instead of hanging; *device_error receives the flag (nonzero
   means the expiry was detected) and the flag is cleared. No fault, trap or unbounded wait is
   involved; the grid stays usable. Synchronises the stream. */
kv_status kv_selftest_wait_timeout(kv_handle h, int* device_error);

/* Host only (no device call): the per-axis data kv_create_grid builds for one axis of n cells
   (2 <= n <= 1024) with the Eq (22) stretching parameter `stretch` (as in kv_grid_desc).
   Eq (15) for the pressure-correction Laplacian D G with homogeneous Neumann walls:
     E      n x n, row-major, row = cell, column = mode (eigenvectors), nullable;
     E_inv  n x n, row-major, row = mode, column = cell, nullable;
     lambda n eigenvalues, mode 0 the constants (exactly 0), then decreasing, nullable.
   Closed form on the uniform grid (stretch = 0), the tridiagonal QL iteration otherwise.
   weights (nullable): 14 rows of n + 2 doubles, indexed by the padded index t along the axis,
   row-major, zero outside each row's range:
     0      1 / cell width (cells t = 1..n)
     1      1 / distance between the centres of cells t and t+1 (faces t = 1..n-1)
     2..4   first-derivative weights (t-1, t, t+1) at a cell-like node t = 1..n
     5..7   second-derivative (flux form) weights at a cell-like node
     8..10  first-derivative weights at a face-like node t = 1..n-1
     11..13 second-derivative weights at a face-like node
   All buffers are the caller's host memory. KV_ERR_ARG for a bad n or stretch,
   KV_ERR_NOT_CONVERGED if the eigensolver fails (message via kv_last_error(NULL)). */
kv_status kv_axis_data(int n, double stretch, double* E, double* E_inv, double* lambda, double* weights);

/* Message of the last failed call on h (NULL h: last failed kv_create_grid,
   kv_krylov_vector_noalloc or kv_axis_data on this thread). */
const char* kv_last_error(kv_handle h);

#ifdef __cplusplus
}
#endif

#endif /* KV_H */
