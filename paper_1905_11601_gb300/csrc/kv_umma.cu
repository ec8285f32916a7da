// Mixed-precision TPF Poisson solve (Eqs (14)-(18)) on the 5th-generation tensor cores.
//
// Each per-axis contraction D[m][r] = sum_k W[m][k] X[r][k] runs as a BF16 x BF16 -> FP32
// tcgen05 GEMM: W (the FP64 1D eigenvector matrix) and X (the data) are each split into
// three BF16 slices (x = x1 + x2 + x3, x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2),
// about 24 significant bits), and the six slice products with i + j <= 4 are accumulated in
// one FP32 TMEM accumulator, which gives about FP32 accuracy. The FP64 accuracy of the solve
// is won back by iterative refinement with an FP64 residual r = b - L phi (kv_mixed.cu).
//
// Kernel structure (persistent, one CTA per SM, 128 x 256 output tiles, cta_group::1):
//   warp 0      TMA producer, two phases per tile: per 64-wide k-chunk the three 128 x 64 tiles
//               of W_0..W_2 into a six-slot ring and the three 256 x 64 tiles of X_0..X_2 into a
//               three-slot ring (128-byte swizzle; each slot with a full[] mbarrier), so every
//               slice is loaded once per k-chunk and serves all the products with i + j >= 1;
//               then W_0 and X_0 again for the leading product (see the MMA warp);
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32 accumulators); lane 0 issues, per
//               k-chunk and X slice j, the tcgen05.mma (M=128, N=256, K=16) of the pairs (i, j)
//               with i + j <= 2, releases each slot with tcgen05.commit to its empty[] barrier
//               and, after a tile's last MMA, commits to that accumulator's full barrier;
//   warps 2-17  epilogue (four warps per TMEM lane quarter): tcgen05.ld of 16 accumulator
//               columns at a time, transposed through a swizzled 2 KB shared-memory buffer so that
//               stores run along r, then either the next pass's three BF16 slices (with the
//               1 / Lambda scaling of Eq (17) in the third forward pass) or phi (FP64, or FP32
//               after a first refinement sweep); then they release the accumulator, so the
//               epilogue of one tile overlaps the MMAs of the next.
// Every mbarrier wait has an iteration limit; on expiry the kernel sets an error flag and
// leaves without hanging.
#include <cuda.h>
#include <cuda_bf16.h>

#include "kv_df.cuh"
#include "kv_internal.cuh"

namespace {

constexpr int UM = 128, UK = 64;            // CTA tile rows; UK = one 128-byte swizzle row of BF16
constexpr int AR = 6;                       // W-slice ring (two k-chunks of three slices)
constexpr int A_BYTES = UM * UK * 2;        // 16 KB
constexpr int EPI_WARPS = 16;  // four per TMEM lane quarter, each taking a quarter of the columns
constexpr int EPI_CHUNK = 16;               // columns per TMEM load and transpose
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int EPI_BYTES = EPI_WARPS * 32 * EPI_CHUNK * 4;
// Tile width (output columns per tile, the MMA's N): 256 or 128. The X-slice ring holds 96 KB
// either way (three 32 KB slots, or six 16 KB slots: two k-chunks in flight). Two accumulator
// buffers: the epilogue of one tile overlaps the next tile's MMAs.
//
// The FP32 accumulation of the tensor core drops the low bits of products much smaller than the
// running sum, so the five small slice products (i + j >= 1) must not be accumulated onto the
// leading product W_0 X_0. With 256 columns (SPLIT false) the small products are summed over all
// of K first and W_0 X_0 is added after them, in a second pass over K that loads W_0 and X_0
// again. With 128 columns (SPLIT true) TMEM holds two accumulators per buffer, one for the small
// products and one for W_0 X_0, summed in the epilogue: one pass over K, a third fewer loads.
template <int UNT>
struct Tile {
  static constexpr int N = UNT;
  static constexpr bool SPLIT = UNT == 128;
  static constexpr int BR = 3 * 256 / UNT;
  static constexpr int B_BYTES = UNT * UK * 2;
  static constexpr int EPI_COLS = UNT / (EPI_WARPS / 4);
  static constexpr int NBARS = 2 * AR + 2 * BR + 4;
  static constexpr int SMEM = 256 /*barriers + TMEM slot*/ + 1024 /*alignment slack*/ + AR * A_BYTES +
                              BR * B_BYTES + EPI_BYTES;
  static constexpr int ACC_COLS = SPLIT ? 2 * UNT : UNT;  // TMEM columns of one buffer
  static constexpr int TMEM_COLS = 2 * ACC_COLS;
  static constexpr int NPH = SPLIT ? 1 : 2;               // passes over K per tile
  // instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 accumulator, M = 128, N = UNT
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UNT >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
  static_assert(NBARS * 8 + 4 <= 256, "barrier area");
  static_assert(SMEM <= 232448, "shared memory per block");
  static_assert(EPI_COLS % EPI_CHUNK == 0, "epilogue column blocks");
};
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity; false (and the error flag set) on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned int* err,
                                          uint32_t limit = WAIT_LIMIT) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  atomicOr(err, 1u);
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor (K-major operand, 128-byte swizzle, 8-row groups of 1024 B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// three-way BF16 split of an FP32 value
__device__ __forceinline__ void split3(float x, __nv_bfloat16& s1, __nv_bfloat16& s2, __nv_bfloat16& s3) {
  s1 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(s1);
  s2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(s2);
  s3 = __float2bfloat16_rn(r2);
}


}  // namespace


namespace {

// Persistent: CTA b handles tiles b, b + gridDim.x, ...; tile t covers vector t / (ntm ntr), and
// within it rows m0 = (t % ntm) * 128 and columns r0 = ((t / ntm) % ntr) * 256, so CTAs that run
// together share their X tiles in L2. A block of vectors is one launch: its tiles fill the GPU
// evenly where one vector's do not.
template <int UNT>
__global__ void __launch_bounds__(THREADS, 1)
    k_umma_axis(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int K,
                KvUmmaEpi ep, unsigned int* err) {
  using T = Tile<UNT>;
  constexpr int UN = T::N, BR = T::BR, B_BYTES = T::B_BYTES, EPI_COLS = T::EPI_COLS, NBARS = T::NBARS,
                TMEM_COLS = T::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  uint64_t* bars = (uint64_t*)smem_raw;  // fullA[AR] emptyA[AR] fullB[BR] emptyB[BR] accf[2] acce[2], TMEM slot
  uint32_t* tmem_slot = (uint32_t*)(bars + NBARS);
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 256 + 1023) & ~(uintptr_t)1023);
  uint8_t* aring = smem;
  uint8_t* bring = smem + AR * A_BYTES;
  float* epi = (float*)(bring + BR * B_BYTES);
  const uint32_t fullA0 = smem_u32(bars), emptyA0 = smem_u32(bars + AR);
  const uint32_t fullB0 = smem_u32(bars + 2 * AR), emptyB0 = smem_u32(bars + 2 * AR + BR);
  const uint32_t accf0 = smem_u32(bars + 2 * AR + 2 * BR), acce0 = smem_u32(bars + 2 * AR + 2 * BR + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntm = (ep.M + UM - 1) / UM, ntr = (ep.R + UN - 1) / UN, nvt = ntm * ntr;
  const int ntiles = nvt * (ep.nvec > 1 ? ep.nvec : 1);
  const uint32_t lim = ep.wait_limit ? ep.wait_limit : WAIT_LIMIT;
  const int kchunks = (K + UK - 1) / UK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < AR; ++s) {
      mbar_init(fullA0 + 8 * s, 1);
      mbar_init(emptyA0 + 8 * s, 1);
    }
    for (int s = 0; s < BR; ++s) {
      mbar_init(fullB0 + 8 * s, 1);
      mbar_init(emptyB0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);                  // tcgen05.commit after a tile's last MMA
      mbar_init(acce0 + 8 * b, EPI_WARPS * 32);     // every epilogue thread, after reading it
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
      uint32_t ga = 0, gb = 0;  // ring positions, continued across tiles
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int vec = t / nvt, tv = t - vec * nvt;
        const int m0 = (tv % ntm) * UM, r0 = (tv / ntm) * UN;
        // phase 0: the slices of the six products (of the five with i + j >= 1 without SPLIT);
        // phase 1 (without SPLIT): W_0 and X_0 only
        for (int ph = 0; ph < T::NPH && ok; ++ph) {
          const int ns = ph == 0 ? 3 : 1;
          for (int kc = 0; kc < kchunks && ok; ++kc) {
            for (int i = 0; i < ns && ok; ++i, ++ga) {
              const int s = ga % AR;
              if (!(ok = mbar_wait(emptyA0 + 8 * s, ((ga / AR) & 1u) ^ 1u, err, lim))) break;
              mbar_expect_tx(fullA0 + 8 * s, A_BYTES + ep.extra_tx);
              tma_load_3d(smem_u32(aring + s * A_BYTES), &mapA, kc * UK, m0, i, fullA0 + 8 * s);
            }
            for (int j = 0; j < ns && ok; ++j, ++gb) {
              const int s = gb % BR;
              if (!(ok = mbar_wait(emptyB0 + 8 * s, ((gb / BR) & 1u) ^ 1u, err, lim))) break;
              mbar_expect_tx(fullB0 + 8 * s, B_BYTES + ep.extra_tx);
              tma_load_4d(smem_u32(bring + s * B_BYTES), &mapB, kc * UK, r0, vec, j, fullB0 + 8 * s);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t ga = 0, gb = 0;
      int lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
        const int buf = lt & 1;
        const uint32_t use = (uint32_t)(lt >> 1);
        // the epilogue must have drained this accumulator (its previous tile)
        if (!(ok = mbar_wait(acce0 + 8 * buf, (use & 1u) ^ 1u, err, lim))) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(buf * T::ACC_COLS);
        const uint32_t acc_lead = T::SPLIT ? acc + (uint32_t)UN : acc;  // W_0 X_0 (see Tile)
        bool first = true, first_lead = true;
        for (int ph = 0; ph < T::NPH && ok; ++ph) {
          const int ns = ph == 0 ? 3 : 1;
          for (int kc = 0; kc < kchunks && ok; ++kc) {
            uint32_t aA[3];
            for (int i = 0; i < ns && ok; ++i) {
              const uint32_t p = ga + i;
              ok = mbar_wait(fullA0 + 8 * (p % AR), (p / AR) & 1u, err, lim);
              aA[i] = smem_u32(aring + (p % AR) * A_BYTES);
            }
            if (!ok) break;
            // X slice j meets the W slices i with i + j <= 2 (without SPLIT, phase 0: i + j >= 1)
            for (int j = 0; j < ns && ok; ++j, ++gb) {
              const int sb = gb % BR;
              if (!(ok = mbar_wait(fullB0 + 8 * sb, (gb / BR) & 1u, err, lim))) break;
              tc_fence_after();
              const uint32_t b = smem_u32(bring + sb * B_BYTES);
              // phase 0: i = 2 - j .. 0 (without SPLIT not (0, 0)); phase 1: (0, 0) only
              for (int i = ph == 0 ? 2 - j : 0; i >= 0; --i) {
                const bool lead = i + j == 0;
                if (!T::SPLIT && ph == 0 && lead) continue;
                const bool to_lead = T::SPLIT && lead;
#pragma unroll
                for (int kk = 0; kk < UK / 16; ++kk) {
                  const bool f = to_lead ? first_lead : first;
                  umma_bf16(to_lead ? acc_lead : acc, sdesc(aA[i] + kk * 32), sdesc(b + kk * 32), T::IDESC,
                            f ? 0u : 1u);
                  if (to_lead)
                    first_lead = false;
                  else
                    first = false;
                }
              }
              umma_commit(emptyB0 + 8 * sb);
            }
            for (int i = 0; i < ns; ++i) umma_commit(emptyA0 + 8 * ((ga + i) % AR));
            ga += ns;
          }
        }
        umma_commit(accf0 + 8 * buf);  // arrives once every MMA of this tile has completed
      }
    }
  } else {
    // epilogue warps 2..17 -> TMEM lane quarter (warp % 4), column block (warp - 2) / 4
    const int q = warp & 3;
    const int c0 = ((warp - 2) / 4) * EPI_COLS;
    float* tb = epi + (warp - 2) * 32 * EPI_CHUNK;
    // tb holds EPI_CHUNK = 16 columns x 32 rows, column-major, the row index XOR-swizzled by
    // 8 (col / 4): the column writes and the 4-column row reads below are bank-conflict free
    auto tix = [](int col, int row) { return col * 32 + (row ^ (8 * (col >> 2))); };
    // groups of 4 outputs are contiguous and 8-byte aligned (slices) or 32-byte aligned (phi)
    // when the inner extent and R are multiples of 4 (and the slice pitch and size are)
    const bool to_phi = ep.mode >= 2;
    // (and the per-vector offsets of a block keep that alignment)
    const bool vec4 = (ep.R % 4 == 0) && (to_phi || (ep.nb % 4 == 0 && ep.pitch % 4 == 0 && ep.slice % 4 == 0)) &&
                      (ep.nvec <= 1 || (ep.vstride_out % 4 == 0 && ep.vstride_phi % 4 == 0));
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int buf = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      if (!mbar_wait(accf0 + 8 * buf, use & 1u, err, lim)) break;
      tc_fence_after();
      const int vec = t / nvt, tv = t - vec * nvt;
      const int m0 = (tv % ntm) * UM, r0 = (tv / ntm) * UN;
      const int mrow0 = m0 + 32 * q;
      // this vector's outputs
      __nv_bfloat16* const vout = ep.out ? ep.out + (size_t)vec * ep.vstride_out : nullptr;
      double* const vphi = ep.phi ? ep.phi + (size_t)vec * ep.vstride_phi : nullptr;
      float* const vphi32 = ep.phi32 ? ep.phi32 + (size_t)vec * ep.vstride_phi : nullptr;
      for (int c = c0; c < c0 + EPI_COLS; c += EPI_CHUNK) {
        float v[EPI_CHUNK];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * T::ACC_COLS + c), v);
        if (T::SPLIT) {  // the small products' sum plus W_0 X_0
          float vl[EPI_CHUNK];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * T::ACC_COLS + UN + c), vl);
#pragma unroll
          for (int t2 = 0; t2 < EPI_CHUNK; ++t2) v[t2] = __fadd_rn(v[t2], vl[t2]);
        }
        // transpose: tb[col][row]
#pragma unroll
        for (int t2 = 0; t2 < EPI_CHUNK; ++t2) tb[tix(t2, lane)] = v[t2];
        __syncwarp();
        if (vec4) {
          // lane: 4 consecutive columns (4 (lane % 4) ..) of rows 8 it + lane / 4; 8-byte stores
          const int cc = 4 * (lane & 3);
          const int r = r0 + c + cc;
          if (r < ep.R) {  // R is a multiple of 4 here, so r < R covers all four columns
            int a = 0, bcol = r;
            if (!to_phi) {
              a = r / ep.nb;
              bcol = r - a * ep.nb;
            }
            for (int it = 0; it < 4; ++it) {
              const int row = 8 * it + (lane >> 2);
              const int m = mrow0 + row;
              if (m >= ep.M) break;
              float d[4];
#pragma unroll
              for (int t2 = 0; t2 < 4; ++t2) d[t2] = tb[tix(cc + t2, row)];
              if (to_phi) {
                const size_t o = (size_t)m * ep.R + r;
                if (ep.mode == 4) {
                  *reinterpret_cast<float4*>(vphi32 + o) = make_float4(d[0], d[1], d[2], d[3]);
                } else {
                  double2* p = reinterpret_cast<double2*>(vphi + o);
                  double2 p0 = make_double2(df_f2d(d[0]), df_f2d(d[1])), p1 = make_double2(df_f2d(d[2]), df_f2d(d[3]));
                  if (ep.mode == 2) {
                    const double2 q0 = p[0], q1 = p[1];
                    p0.x += q0.x;
                    p0.y += q0.y;
                    p1.x += q1.x;
                    p1.y += q1.y;
                  } else if (ep.mode == 5) {
                    const float4 q = *reinterpret_cast<const float4*>(vphi32 + o);
                    p0.x += df_f2d(q.x);
                    p0.y += df_f2d(q.y);
                    p1.x += df_f2d(q.z);
                    p1.y += df_f2d(q.w);
                  }
                  p[0] = p0;
                  p[1] = p1;
                }
              } else {
                if (ep.mode == 1) {
#pragma unroll
                  for (int t2 = 0; t2 < 4; ++t2) {
                    const float lam = ep.lz[m] + ep.la[a] + ep.lb[bcol + t2];
                    d[t2] = (m == 0 && r + t2 == 0) ? 0.0f : __fdividef(d[t2], lam);
                  }
                }
                __nv_bfloat16 s[3][4];
#pragma unroll
                for (int t2 = 0; t2 < 4; ++t2) split3(d[t2], s[0][t2], s[1][t2], s[2][t2]);
                const size_t o = ((size_t)m * ep.na + a) * ep.pitch + bcol;
#pragma unroll
                for (int sl = 0; sl < 3; ++sl)
                  *reinterpret_cast<uint2*>(vout + (size_t)sl * ep.slice + o) = *reinterpret_cast<const uint2*>(s[sl]);
              }
            }
          }
        } else {
          // lane: column lane % 16 of rows 16 (lane / 16) ..
          const int col = lane & (EPI_CHUNK - 1);
          const int r = r0 + c + col;
          if (r < ep.R) {
            int a = 0, bcol = r;
            if (!to_phi) {
              a = r / ep.nb;
              bcol = r - a * ep.nb;
            }
            for (int rr = 0; rr < 16; ++rr) {
              const int row = 16 * (lane >> 4) + rr;
              const int m = mrow0 + row;
              if (m >= ep.M) break;
              float d = tb[tix(col, row)];
              if (to_phi) {
                const size_t o = (size_t)m * ep.R + r;
                if (ep.mode == 4)
                  vphi32[o] = d;
                else if (ep.mode == 5)
                  vphi[o] = df_f2d(vphi32[o]) + df_f2d(d);
                else
                  vphi[o] = ep.mode == 2 ? vphi[o] + df_f2d(d) : df_f2d(d);
              } else {
                if (ep.mode == 1) {
                  const float lam = ep.lz[m] + ep.la[a] + ep.lb[bcol];
                  d = (m == 0 && r == 0) ? 0.0f : __fdividef(d, lam);
                }
                __nv_bfloat16 s1, s2, s3;
                split3(d, s1, s2, s3);
                const size_t o = ((size_t)m * ep.na + a) * ep.pitch + bcol;
                vout[o] = s1;
                vout[ep.slice + o] = s2;
                vout[2 * ep.slice + o] = s3;
              }
            }
          }
        }
        __syncwarp();
      }
      // the accumulator may be overwritten by the tile after next
      tc_fence_before();
      mbar_arrive(acce0 + 8 * buf);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

// 3D BF16 tensor map over `slices` arrays of rows x cols (row pitch `pitch` elements), box
// 64 x box_rows x 1, 128-byte swizzle, zero fill outside [0, cols) x [0, rows).
bool kv_make_slice_map(CUtensorMap* map, const void* base, int cols, int rows, int pitch, size_t slice_elems,
                       int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, 3};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)slice_elems * 2};
  cuuint32_t box[3] = {(cuuint32_t)UK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool kv_make_data_map(CUtensorMap* map, const void* base, int cols, int rows, int pitch, int nvec, size_t vec_elems,
                      size_t slice_elems, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)nvec, 3};
  cuuint64_t strides[3] = {(cuuint64_t)pitch * 2, (cuuint64_t)vec_elems * 2, (cuuint64_t)slice_elems * 2};
  cuuint32_t box[4] = {(cuuint32_t)UK, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int kv_umma_box_rows_a() { return UM; }
int kv_umma_box_rows_b() { return 256; }

// Raises the kernels' dynamic shared-memory limit (once per process, before any launch or capture).
cudaError_t kv_umma_init() {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_umma_axis<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tile<256>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_umma_axis<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tile<128>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaSuccess;
}

cudaError_t kv_launch_umma_axis(const CUtensorMap* mapA, const CUtensorMap* mapB, int K, const KvUmmaEpi& ep,
                                unsigned int* err, cudaStream_t s, int tile) {
  cudaError_t e0 = kv_umma_init();
  if (e0 != cudaSuccess) return e0;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int un = tile == 128 ? 128 : 256;  // the data map's box must have un rows
  const int tiles = ((ep.R + un - 1) / un) * ((ep.M + UM - 1) / UM) * (ep.nvec > 1 ? ep.nvec : 1);
  const int grid = tiles < sms ? tiles : sms;
  if (un == 128)
    k_umma_axis<128><<<grid, THREADS, Tile<128>::SMEM, s>>>(*mapA, *mapB, K, ep, err);
  else
    k_umma_axis<256><<<grid, THREADS, Tile<256>::SMEM, s>>>(*mapA, *mapB, K, ep, err);
  return cudaGetLastError();
}
