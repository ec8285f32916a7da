// A block of Krylov vectors evaluated together in mixed precision (Section 3.1's many Krylov
// vectors per Newton or Arnoldi run, here as independent right-hand sides): each vector's
// linearised operator, divergence and velocity correction are launched per vector, and each of
// the six tensor-core contractions of every refinement sweep is one launch for the whole block.
// One vector's contraction at 256^3 has 512 output tiles, 3.4 waves over the SMs; a block of 16
// has 8192, which fill the GPU evenly and amortise the persistent kernel's start and drain.
#include "kv_internal.cuh"

kv_status kv_krylov_block(kv_grid* h, const double* X, double* Y, int nb) {
  if (nb < 1 || nb > h->blk_cap) {
    h->err = "kv_krylov_block: block larger than the block buffers";
    return KV_ERR_ARG;
  }
  cudaStream_t s = h->s;
  const size_t L = 4 * h->P;
  const double tol = kv_simple_tol(h);
  for (int v = 0; v < nb; ++v) {
    double* vstar = h->blk_vstar + (size_t)v * 3 * h->P;
    {
      KvPhase ph(h, KV_PH_STENCIL, 2);
      kv_launch_apply_df(h, h->coef_df, X + (size_t)v * L, vstar, Y + (size_t)v * L + 3 * h->P, s);
    }
    {
      KvPhase ph(h, KV_PH_DIV, 1);
      kv_launch_divergence_to(h, vstar, h->blk_b + (size_t)v * h->Nc, h->blk_xs[0] + (size_t)v * h->xs_slice,
                              (size_t)h->blk_cap * h->xs_slice, s);
    }
  }
  kv_launch_poisson_mixed_block(h, nb, s);
  for (int v = 0; v < nb; ++v) {
    KvPhase ph(h, KV_PH_CORRECT, 2);
    kv_launch_correct(h, h->blk_vstar + (size_t)v * 3 * h->P, h->blk_phi + (size_t)v * h->Nc, Y + (size_t)v * L,
                      nullptr, 0, s, 1);
    kv_launch_guard_close(h, tol, 1, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string("kv_krylov_block: ") + cudaGetErrorString(e);
    return KV_ERR_CUDA;
  }
  return KV_OK;
}
