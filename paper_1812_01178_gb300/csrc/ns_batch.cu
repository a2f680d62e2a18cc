// Batched ensembles: many independent periodic-x instances of uneven sizes advanced together.
// Each instance is an ordinary context (its own fields, tables, partitioning) on a slice of one
// workspace.  Every stage of a sub-step is planned once for the whole ensemble: the stage's
// launches of all instances are grouped by kernel variant and each group becomes one persistent
// batched_kernel launch whose blocks walk the blocks of every instance in the group.  One time
// step (3 sub-steps x 10 stages) is captured as a single CUDA graph.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ns_internal.cuh"

namespace {

struct PlannedLaunch {
  cudaError_t (*enqueue)(const void*, const BatchMap&, unsigned, dim3, size_t, cudaStream_t);
  const void* dargs;
  BatchMap map;
  unsigned grid;
  dim3 block;
  size_t smem;
  int stage;
};

typedef cudaError_t (*StageFn)(LaunchSink&, int);
const StageFn BATCH_STAGES[] = {stage_rhs,       stage_adi_x,      stage_adi_y,     stage_adi_z,
                                stage_pois_divz, stage_pois_x_fwd, stage_pois_tdma, stage_pois_x_inv,
                                stage_pois_ifftz, stage_pois_refine, stage_project};
const char* BATCH_STAGE_NAMES[] = {"rhs",           "adi_x",         "adi_y",          "adi_z",
                                   "poisson_div_fftz", "poisson_x_fwd", "poisson_tdma_y", "poisson_x_inv",
                                   "poisson_ifftz", "poisson_refine", "project"};
constexpr int NBATCH_STAGES = 11;
constexpr size_t kArenaBase = 1 << 20;
constexpr size_t kArenaPerInstance = 64 << 10;


}  // namespace

struct ns_batch {
  std::vector<ns_ctx*> inst;
  std::vector<size_t> ws_off;
  cudaStream_t stream, cap_stream;
  void* ws;
  size_t ws_bytes;
  bool own_ws;
  char* arena;
  size_t arena_bytes, arena_used;
  std::vector<PlannedLaunch> plan[3];
  int num_sms;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  bool have_graph;
  std::string err;
};

namespace {

ns_status bfail(ns_batch* b, ns_status s, const std::string& m) {
  b->err = m;
  return s;
}

size_t instances_bytes(const ns_config* cfgs, int n, std::vector<size_t>* off) {
  size_t o = 0;
  for (int i = 0; i < n; ++i) {
    const size_t w = ns_workspace_bytes(&cfgs[i]);
    if (w == 0) return 0;
    if (off) off->push_back(o);
    o += al256(w);
  }
  return o;
}

void* arena_put(ns_batch* b, const void* host, size_t bytes, cudaError_t* e) {
  if (b->arena_used + al256(bytes) > b->arena_bytes) {
    *e = cudaErrorMemoryAllocation;
    return nullptr;
  }
  void* d = b->arena + b->arena_used;
  *e = cudaMemcpy(d, host, bytes, cudaMemcpyHostToDevice);
  b->arena_used += al256(bytes);
  return d;
}

// Plan every stage of every sub-step for the current instance settings.
ns_status make_plan(ns_batch* b) {
  b->arena_used = 0;
  for (int k = 0; k < 3; ++k) {
    b->plan[k].clear();
    for (int st = 0; st < NBATCH_STAGES; ++st) {
      BatchPlanner pl;
      for (ns_ctx* c : b->inst) {
        LaunchSink s{c, &pl};
        pl.next_instance();
        cudaError_t e = BATCH_STAGES[st](s, k);
        if (e != cudaSuccess) return bfail(b, NS_ERR_CUDA, std::string("plan ") + BATCH_STAGE_NAMES[st]);
      }
      pl.order();
      for (const BatchGroup& g : pl.groups) {
        const int n = (int)g.grid.size();
        cudaError_t e = cudaSuccess;
        PlannedLaunch L;
        L.enqueue = g.enqueue;
        L.dargs = arena_put(b, g.args.data(), g.args.size(), &e);
        if (e != cudaSuccess) return bfail(b, NS_ERR_CUDA, "plan arena (args)");
        const int* dfirst = (const int*)arena_put(b, g.first.data(), g.first.size() * sizeof(int), &e);
        if (e != cudaSuccess) return bfail(b, NS_ERR_CUDA, "plan arena (blocks)");
        const uint3* dgrid = (const uint3*)arena_put(b, g.grid.data(), g.grid.size() * sizeof(uint3), &e);
        if (e != cudaSuccess) return bfail(b, NS_ERR_CUDA, "plan arena (grids)");
        L.map.first = dfirst;
        L.map.grid = dgrid;
        L.map.n = n;
        L.map.total = g.first.back();
        L.block = g.block;
        L.smem = g.smem;
        const int threads = (int)(g.block.x * g.block.y * g.block.z);
        const long resident = (long)b->num_sms * g.blocks_per_sm(threads, g.smem);
        L.grid = (unsigned)(L.map.total < resident ? L.map.total : resident);
        if (L.grid == 0) L.grid = 1;
        L.stage = st;
        b->plan[k].push_back(L);
      }
    }
  }
  return NS_OK;
}

void drop_batch_graph(ns_batch* b) {
  if (b->have_graph) {
    cudaGraphExecDestroy(b->gexec);
    cudaGraphDestroy(b->graph);
    b->have_graph = false;
  }
}

ns_status run_plan(ns_batch* b, cudaStream_t s) {
  for (int k = 0; k < 3; ++k)
    for (const PlannedLaunch& L : b->plan[k]) {
      cudaError_t e = L.enqueue(L.dargs, L.map, L.grid, L.block, L.smem, s);
      if (e != cudaSuccess) return bfail(b, NS_ERR_CUDA, std::string("batched ") + BATCH_STAGE_NAMES[L.stage] +
                                                             ": " + cudaGetErrorString(e));
    }
  return NS_OK;
}

}  // namespace

extern "C" {

size_t ns_batch_workspace_bytes(const ns_config* cfgs, int n) {
  if (!cfgs || n <= 0) return 0;
  for (int i = 0; i < n; ++i)
    if (cfgs[i].bc_x != 0 || cfgs[i].precision != cfgs[0].precision) return 0;
  const size_t inst = instances_bytes(cfgs, n, nullptr);
  if (inst == 0) return 0;
  return inst + al256(kArenaBase + (size_t)n * kArenaPerInstance);
}

ns_status ns_batch_init(ns_batch** out, const ns_config* cfgs, const ns_fields* fields, int n, void* workspace,
                        size_t ws_bytes, void* cuda_stream) {
  if (!out || !cfgs || !fields || n <= 0) return NS_ERR_ARG;
  *out = nullptr;
  const size_t need = ns_batch_workspace_bytes(cfgs, n);
  if (need == 0) {
    ns_set_thread_error("batch: every instance must be valid, periodic in x (bc_x = 0) and of one precision");
    return NS_ERR_ARG;
  }
  ns_batch* b = new (std::nothrow) ns_batch();
  if (!b) return NS_ERR_ARG;
  b->stream = (cudaStream_t)cuda_stream;
  b->have_graph = false;
  cudaError_t e;
  if (workspace) {
    if (ws_bytes < need || (uintptr_t)workspace % 256) {
      delete b;
      ns_set_thread_error("batch: workspace too small or not 256-byte aligned");
      return NS_ERR_ARG;
    }
    b->ws = workspace;
    b->own_ws = false;
  } else {
    if ((e = cudaMalloc(&b->ws, need)) != cudaSuccess) {
      delete b;
      ns_set_thread_error((std::string("batch: cudaMalloc workspace failed: ") + cudaGetErrorString(e)).c_str());
      return NS_ERR_CUDA;
    }
    b->own_ws = true;
  }
  b->ws_bytes = need;
  const size_t inst_bytes = instances_bytes(cfgs, n, &b->ws_off);
  b->arena = (char*)b->ws + inst_bytes;
  b->arena_bytes = need - inst_bytes;
  b->arena_used = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  b->num_sms = 152;
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  ns_status st = NS_OK;
  for (int i = 0; i < n && st == NS_OK; ++i) {
    ns_ctx* c = nullptr;
    const size_t wi = ns_workspace_bytes(&cfgs[i]);
    st = ns_init(&c, &cfgs[i], &fields[i], (char*)b->ws + b->ws_off[i], wi, cuda_stream);
    if (st == NS_OK) b->inst.push_back(c);
    else b->err = std::string("instance ") + std::to_string(i) + ": " + ns_last_error(nullptr);
  }
  if (st == NS_OK && (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    st = NS_ERR_CUDA;
  if (st == NS_OK) st = make_plan(b);
  if (st != NS_OK) {
    ns_set_thread_error(b->err.c_str());
    for (ns_ctx* c : b->inst) ns_destroy(c);
    if (b->own_ws) cudaFree(b->ws);
    delete b;
    return st;
  }
  *out = b;
  return NS_OK;
}

ns_status ns_batch_step(ns_batch* b, int nsteps) {
  if (!b) return NS_ERR_ARG;
  if (nsteps < 0) return bfail(b, NS_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return NS_OK;
  cudaError_t e;
  if (!b->have_graph) {
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return bfail(b, NS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    ns_status s = run_plan(b, b->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (s != NS_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return bfail(b, NS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    if ((e = cudaGraphInstantiate(&b->gexec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      return bfail(b, NS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    b->graph = g;
    b->have_graph = true;
  }
  for (int s = 0; s < nsteps; ++s)
    if ((e = cudaGraphLaunch(b->gexec, b->stream)) != cudaSuccess)
      return bfail(b, NS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return NS_OK;
}

int ns_batch_launches_per_step(ns_batch* b) {
  if (!b) return 0;
  return (int)(b->plan[0].size() + b->plan[1].size() + b->plan[2].size());
}

ns_status ns_batch_autotune(ns_batch* b) {
  if (!b) return NS_ERR_ARG;
  for (ns_ctx* c : b->inst) {
    ns_status s = autotune_ctx(c, false);  // the x solver only: instances of one size keep one line shape
    if (s != NS_OK) return bfail(b, s, std::string("instance autotune: ") + ns_last_error(c));
  }
  drop_batch_graph(b);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, NS_ERR_CUDA, "sync");
  return make_plan(b);
}

ns_status ns_batch_set_partition(ns_batch* b, int i, int P, int mode) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return NS_ERR_ARG;
  ns_status s = ns_set_partition(b->inst[i], 0, P, mode);
  if (s != NS_OK) return bfail(b, s, ns_last_error(b->inst[i]));
  drop_batch_graph(b);
  return make_plan(b);
}

ns_ctx* ns_batch_instance(ns_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return nullptr;
  return b->inst[i];
}

ns_status ns_batch_sync(ns_batch* b) {
  if (!b) return NS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, NS_ERR_CUDA, cudaGetErrorString(e));
  return NS_OK;
}

const char* ns_batch_last_error(ns_batch* b) { return b ? b->err.c_str() : ns_last_error(nullptr); }

void ns_batch_destroy(ns_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_batch_graph(b);
  for (ns_ctx* c : b->inst) ns_destroy(c);
  cudaStreamDestroy(b->cap_stream);
  if (b->own_ws) cudaFree(b->ws);
  delete b;
}

}  // extern "C"
