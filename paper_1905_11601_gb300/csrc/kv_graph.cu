// Batched evaluation and multi-grid plans, replayed from captured CUDA graphs.
//
// A Krylov-vector evaluation is a fixed sequence of about a dozen kernels (two dozen in mixed
// precision). For small grids the launch overhead dominates, and independent problems (a block
// of right-hand sides, several grids or Grashof numbers) leave the GPU idle between launches.
// The sequences are captured once into a CUDA graph and replayed: one graph launch per batch,
// with the evaluations of different grids on parallel branches of the graph. In mixed precision
// a batch is evaluated in blocks of up to KV_BLOCK_MAX vectors whose tensor-core contractions are
// one launch per axis for the whole block (kv_block.cu).
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "kv_internal.cuh"

namespace {

constexpr size_t GRAPH_CACHE = 8;

kv_status set_err(kv_grid* h, kv_status st, const std::string& m) {
  h->err = m;
  return st;
}

}  // namespace

extern "C" kv_status kv_krylov_vector_batch(kv_handle h, const double* X, double* Y, int nb) {
  if (!h) return KV_ERR_ARG;
  if (!X || !Y || nb < 1) return set_err(h, KV_ERR_ARG, "kv_krylov_vector_batch: bad argument");
  if (!h->has_base) return set_err(h, KV_ERR_STATE, "kv_krylov_vector_batch: no base flow set");
  if (h->d.max_passes > 1)
    return set_err(h, KV_ERR_ARG, "kv_krylov_vector_batch: needs max_passes <= 1 (no host-side SIMPLE test)");
  const size_t L = 4 * h->P;
  if (X < Y + (size_t)nb * L && Y < X + (size_t)nb * L)
    return set_err(h, KV_ERR_ARG, "kv_krylov_vector_batch: X and Y overlap");
  auto it = std::find_if(h->graphs.begin(), h->graphs.end(), [&](const kv_grid::GraphEntry& g) {
    return g.X == X && g.Y == Y && g.nb == nb;
  });
  // mixed precision: blocks of up to KV_BLOCK_MAX vectors share each contraction launch (their
  // buffers are allocated here, before any capture)
  const bool block = h->d.precision == KV_PREC_MIXED;
  if (it == h->graphs.end() && block) {
    const kv_status bs = kv_mixed_block_setup(h, nb < KV_BLOCK_MAX ? nb : KV_BLOCK_MAX);
    if (bs != KV_OK) return bs;
  }
  if (it == h->graphs.end()) {
    cudaError_t e;
    if (!h->cap && (e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking)) != cudaSuccess)
      return set_err(h, KV_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    // captured on a stream of its own (the handle's stream may be the legacy default stream);
    // the graph is launched on the handle's stream, which orders it after earlier work
    cudaStream_t s0 = h->s;
    const bool prof = h->prof_on;
    long long before[KV_NPHASE];
    std::copy(h->launches, h->launches + KV_NPHASE, before);
    h->prof_on = false;
    h->s = h->cap;
    kv_status st = KV_OK;
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      st = set_err(h, KV_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    } else {
      if (block) {
        for (int b0 = 0; b0 < nb && st == KV_OK; b0 += h->blk_cap) {
          const int cnt = nb - b0 < h->blk_cap ? nb - b0 : h->blk_cap;
          st = kv_krylov_block(h, X + (size_t)b0 * L, Y + (size_t)b0 * L, cnt);
        }
      } else {
        for (int b = 0; b < nb && st == KV_OK; ++b)
          st = kv_krylov_vector(h, X + (size_t)b * L, Y + (size_t)b * L, nullptr, nullptr);
      }
      e = cudaStreamEndCapture(h->cap, &graph);
      if (st == KV_OK && e != cudaSuccess)
        st = set_err(h, KV_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    h->s = s0;
    h->prof_on = prof;
    kv_grid::GraphEntry ge{X, Y, nb, nullptr, {}};
    for (int q = 0; q < KV_NPHASE; ++q) {
      ge.launches[q] = h->launches[q] - before[q];
      h->launches[q] = before[q];
    }
    if (st == KV_OK && (e = cudaGraphInstantiate(&ge.exec, graph, 0)) != cudaSuccess)
      st = set_err(h, KV_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    if (graph) cudaGraphDestroy(graph);
    if (st != KV_OK) return st;
    if (h->graphs.size() >= GRAPH_CACHE) {
      cudaGraphExecDestroy(h->graphs.front().exec);
      h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(ge);
    it = h->graphs.end() - 1;
  }
  cudaError_t e = cudaGraphLaunch(it->exec, h->s);
  if (e != cudaSuccess) return set_err(h, KV_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
  for (int q = 0; q < KV_NPHASE; ++q) h->launches[q] += it->launches[q];
  return KV_OK;
}

// ---- multi-grid plans ---------------------------------------------------------------------

struct kv_plan {
  struct Item {
    kv_handle h;
    const double* x;
    double* y;
  };
  std::vector<Item> items;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> branches;
  cudaStream_t origin = nullptr;
  std::string err;
};

extern "C" kv_status kv_plan_create(kv_plan** out) {
  if (!out) return KV_ERR_ARG;
  *out = new (std::nothrow) kv_plan();
  return *out ? KV_OK : KV_ERR_NOMEM;
}

extern "C" kv_status kv_plan_add(kv_plan* p, kv_handle h, const double* x, double* y) {
  if (!p || !h || !x || !y) return KV_ERR_ARG;
  if (p->exec) {
    p->err = "kv_plan_add: the plan has already been launched";
    return KV_ERR_STATE;
  }
  if (!h->has_base) {
    p->err = "kv_plan_add: the grid has no base flow";
    return KV_ERR_STATE;
  }
  if (h->d.max_passes > 1) {
    p->err = "kv_plan_add: needs max_passes <= 1";
    return KV_ERR_ARG;
  }
  p->items.push_back({h, x, y});
  return KV_OK;
}

static kv_status plan_capture(kv_plan* p) {
  cudaError_t e;
  // one branch per distinct grid (evaluations of one grid share its scratch and stay ordered)
  std::vector<kv_handle> grids;
  for (auto& it : p->items)
    if (std::find(grids.begin(), grids.end(), it.h) == grids.end()) grids.push_back(it.h);
  if ((e = cudaStreamCreateWithFlags(&p->origin, cudaStreamNonBlocking)) != cudaSuccess) {
    p->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
    return KV_ERR_CUDA;
  }
  p->branches.resize(grids.size(), nullptr);
  for (auto& b : p->branches)
    if ((e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking)) != cudaSuccess) {
      p->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      return KV_ERR_CUDA;
    }
  cudaEvent_t fork;
  std::vector<cudaEvent_t> joins(grids.size(), nullptr);
  cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (auto& j : joins) cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
  kv_status st = KV_OK;
  cudaGraph_t graph = nullptr;
  if ((e = cudaStreamBeginCapture(p->origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
    p->err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
    st = KV_ERR_CUDA;
  } else {
    cudaEventRecord(fork, p->origin);
    for (size_t gi = 0; gi < grids.size() && st == KV_OK; ++gi) {
      kv_handle h = grids[gi];
      cudaStreamWaitEvent(p->branches[gi], fork, 0);
      cudaStream_t s0 = h->s;
      const bool prof = h->prof_on;
      h->s = p->branches[gi];
      h->prof_on = false;
      for (auto& it : p->items)
        if (it.h == h && st == KV_OK) {
          st = kv_krylov_vector(h, it.x, it.y, nullptr, nullptr);
          if (st != KV_OK) p->err = h->err;
        }
      h->s = s0;
      h->prof_on = prof;
      cudaEventRecord(joins[gi], p->branches[gi]);
      cudaStreamWaitEvent(p->origin, joins[gi], 0);
    }
    e = cudaStreamEndCapture(p->origin, &graph);
    if (st == KV_OK && e != cudaSuccess) {
      p->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
      st = KV_ERR_CUDA;
    }
  }
  if (st == KV_OK && (e = cudaGraphInstantiate(&p->exec, graph, 0)) != cudaSuccess) {
    p->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
    st = KV_ERR_CUDA;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaEventDestroy(fork);
  for (auto& j : joins) cudaEventDestroy(j);
  return st;
}

extern "C" kv_status kv_plan_launch(kv_plan* p, void* stream) {
  if (!p) return KV_ERR_ARG;
  if (p->items.empty()) {
    p->err = "kv_plan_launch: empty plan";
    return KV_ERR_STATE;
  }
  if (!p->exec) {
    kv_status st = plan_capture(p);
    if (st != KV_OK) return st;
  }
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    p->err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
    return KV_ERR_CUDA;
  }
  return KV_OK;
}

extern "C" const char* kv_plan_last_error(kv_plan* p) { return p ? p->err.c_str() : ""; }

extern "C" kv_status kv_plan_destroy(kv_plan* p) {
  if (!p) return KV_OK;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  for (auto b : p->branches)
    if (b) cudaStreamDestroy(b);
  if (p->origin) cudaStreamDestroy(p->origin);
  delete p;
  return KV_OK;
}
