// Batched integration of many independent CGL instances (uneven grids,
// boundary conditions and parameters) with one persistent grouped launch per
// mu-mode pass and the whole time step replayed as one CUDA graph.
//
// Each instance gets its own FP64-computed factors exp(c tau A_mu) (a factor-
// only plan).  All fields live in one packed buffer: instance i's N_i values
// start at offset_i = sum_{j<i} N_j.  For every pass (sweep, mode) the host
// builds a work list of (instance, first fiber, fibers per tile) items ordered
// by decreasing cost; a fixed grid of CTAs (SMs x resident CTAs) drains it
// through an atomic counter, so large and small instances share the machine
// without a launch per instance.  Passes are separated by kernel boundaries:
// no CTA ever waits for another.
//
// Fibers per tile come from an autotuner: for each (n, contiguous fibers or
// not, precision, right-hand sides, SM count) it times the mode-pass kernel on
// a synthetic 2048-fiber field for every admissible tile size and keeps the
// fastest, in memory and in the text file named by $CGL_AUTOTUNE_CACHE.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "plan.cuh"

using namespace cgl;

struct cgl_batch {
  int dev = 0;
  int count = 0;
  int scheme = 0, precision = 0;
  double tau = 0;
  size_t elem = 0;
  std::vector<cgl_plan*> plans;
  std::vector<int64_t> offsets;
  int64_t total = 0;
  void* work[3] = {nullptr, nullptr, nullptr};
  int* status = nullptr;
  int* counters = nullptr;
  struct Pass {
    int sweep = 0, mu = 0, nrhs = 1;
    size_t smem = 0;
    int grid = 0;
    int nitems = 0;
    ModePassArgs* table = nullptr;  // device, one entry per instance
    BatchItem* items = nullptr;     // device
  };
  std::vector<Pass> passes;
  std::vector<void*> allocations;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* graph_u = nullptr;
};

namespace {

// ------------------------------------------------------------------ autotuner

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, double>> g_tune;
bool g_tune_loaded = false;

std::string tune_key(int n, int contiguous, int precision, int nrhs, int sms) {
  char buf[96];
  std::snprintf(buf, sizeof(buf), "%d %d %d %d %d", n, contiguous, precision, nrhs, sms);
  return buf;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("CGL_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int n, c, p, r, s, tb;
  double ms;
  while (std::fscanf(f, "%d %d %d %d %d %d %lf", &n, &c, &p, &r, &s, &tb, &ms) == 7)
    g_tune[tune_key(n, c, p, r, s)] = {tb, ms};
  std::fclose(f);
}

void tune_store(const std::string& key, int tb, double ms) {
  const char* path = std::getenv("CGL_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %.6f\n", key.c_str(), tb, ms);
  std::fclose(f);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Time every admissible tile size for one mode pass shape.
int autotune(int n, int contiguous, int precision, int nrhs, int* tb_out, double* ms_out) {
  const int sms = sm_count();
  const std::string key = tune_key(n, contiguous, precision, nrhs, sms);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load();
  auto it = g_tune.find(key);
  if (it != g_tune.end()) {
    *tb_out = it->second.first;
    if (ms_out) *ms_out = it->second.second;
    return CGL_OK;
  }
  const size_t elem = precision == CGL_F64 ? sizeof(double2) : sizeof(float2);
  const int64_t fibers = 2048;
  const int64_t N = (int64_t)n * fibers;
  void *f0 = nullptr, *f1 = nullptr, *fac = nullptr;
  int* st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = CGL_OK;
  auto cleanup = [&]() {
    if (f0) cudaFree(f0);
    if (f1) cudaFree(f1);
    if (fac) cudaFree(fac);
    if (st) cudaFree(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&f0, N * elem) != cudaSuccess || cudaMalloc(&f1, N * elem) != cudaSuccess ||
      cudaMalloc(&fac, (size_t)n * n * elem) != cudaSuccess || cudaMalloc((void**)&st, sizeof(int)) != cudaSuccess) {
    cleanup();
    return fail(CGL_ENOMEM, "autotune: allocation failed");
  }
  cudaMemset(f0, 0, N * elem);
  cudaMemset(f1, 0, N * elem);
  cudaMemset(fac, 0, (size_t)n * n * elem);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ModePassArgs a{};
  a.g.d = contiguous ? 2 : 3;
  if (contiguous) {
    a.g.n[0] = n; a.g.n[1] = fibers; a.g.n[2] = 1;
    a.g.axis = 0; a.g.P = 1;
  } else {
    a.g.n[0] = 64; a.g.n[1] = n; a.g.n[2] = fibers / 64;
    a.g.axis = 1; a.g.P = 64;
  }
  a.g.n_ax = n;
  a.g.npencils = fibers;
  a.f.nin = nrhs; a.f.nrhs = nrhs; a.f.nextra = 0; a.f.nout = nrhs;
  a.f.in[0] = a.f.work[0] = a.f.out[0] = f0;
  a.f.in[1] = a.f.work[1] = a.f.out[1] = f1;
  a.f.extra[0] = a.f.extra[1] = a.f.extra[2] = f0;
  a.flags = 0;
  a.factor[0] = a.factor[1] = fac;
  a.status = st;
  const int tbmax = mode_tb_max(n, nrhs, elem);
  int best_tb = 1;
  double best = 1e30;
  for (int tb = 2; tb <= 64; tb *= 2) {
    if (tb > tbmax) break;
    float ms = 0;
    cudaError_t e = precision == CGL_F64 ? launch_mode_pass_tb<double>(a, tb, 0) : launch_mode_pass_tb<float>(a, tb, 0);
    cudaEventRecord(e0, 0);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r)
      e = precision == CGL_F64 ? launch_mode_pass_tb<double>(a, tb, 0) : launch_mode_pass_tb<float>(a, tb, 0);
    cudaEventRecord(e1, 0);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      status = fail(CGL_ECUDA, std::string("autotune: ") + cudaGetErrorString(cudaGetLastError()));
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / 3 < best) {
      best = ms / 3;
      best_tb = tb;
    }
  }
  cleanup();
  if (status) return status;
  g_tune[key] = {best_tb, best};
  tune_store(key, best_tb, best);
  *tb_out = best_tb;
  if (ms_out) *ms_out = best;
  return CGL_OK;
}

void free_batch(cgl_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cgl_plan* p : b->plans) free_plan(p);
  for (void* a : b->allocations) cudaFree(a);
  delete b;
}

int batch_alloc(cgl_batch* b, void** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail(CGL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  b->allocations.push_back(*ptr);
  return CGL_OK;
}

// Per-instance pass arguments for field buffer u (device tables).
int upload_tables(cgl_batch* b, void* u) {
  std::vector<ModePassArgs> host(b->count);
  for (auto& ps : b->passes) {
    for (int i = 0; i < b->count; ++i) {
      cgl_plan* p = b->plans[i];
      const size_t off = (size_t)b->offsets[i] * b->elem;
      void* bufs[NBUF] = {(char*)u + off, b->work[0] ? (char*)b->work[0] + off : nullptr,
                          b->work[1] ? (char*)b->work[1] + off : nullptr,
                          b->work[2] ? (char*)b->work[2] + off : nullptr};
      host[i] = make_mode_args(p, p->sweeps[ps.sweep], ps.mu, bufs);
      host[i].status = b->status;
    }
    CUDA_TRY(cudaMemcpy(ps.table, host.data(), host.size() * sizeof(ModePassArgs), cudaMemcpyHostToDevice));
  }
  return CGL_OK;
}

int enqueue_batch_step(cgl_batch* b, cudaStream_t s) {
  for (size_t k = 0; k < b->passes.size(); ++k) {
    const auto& ps = b->passes[k];
    CUDA_TRY(cudaMemsetAsync(b->counters + k, 0, sizeof(int), s));
    cudaError_t e =
        b->precision == CGL_F64
            ? launch_batched_mode_pass<double>(ps.table, ps.items, ps.nitems, b->counters + k, ps.nrhs, ps.smem, ps.grid, s)
            : launch_batched_mode_pass<float>(ps.table, ps.items, ps.nitems, b->counters + k, ps.nrhs, ps.smem, ps.grid, s);
    if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("batched mode pass: ") + cudaGetErrorString(e));
  }
  return CGL_OK;
}

int ensure_batch_graph(cgl_batch* b, void* u) {
  if (b->exec && b->graph_u == u) return CGL_OK;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  int st = upload_tables(b, u);
  if (st) return st;
  CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  st = enqueue_batch_step(b, b->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return fail(CGL_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  b->graph_u = u;
  return CGL_OK;
}

}  // namespace

extern "C" {

int cgl_autotune_mode_tile(int n, int contiguous, int precision, int nrhs, int* tb, double* ms) {
  if (!tb || n < 2 || n > 1024 || (nrhs != 1 && nrhs != 2) || (precision != CGL_F64 && precision != CGL_F32))
    return fail(CGL_EINVAL, "autotune: invalid arguments");
  cudaError_t e = prepare_kernels(0);
  if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  return autotune(n, contiguous ? 1 : 0, precision, nrhs, tb, ms);
}

int cgl_batch_create(cgl_batch** out, int count, const cgl_problem* probs, double tau, int scheme, int precision,
                     void* stream) {
  if (!out) return fail(CGL_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !probs) return fail(CGL_EINVAL, "count must be >= 1 and probs non-NULL");
  if (precision != CGL_F64 && precision != CGL_F32)
    return fail(CGL_EUNSUPPORTED, "batches run in CGL_F64 or CGL_F32");
  if (scheme != CGL_STRANG && scheme != CGL_SPLIT4 && scheme != CGL_LAWSON4 && scheme != CGL_LAWSON2 &&
      scheme != CGL_STRANG3T && scheme != CGL_SPLIT4_3T)
    return fail(scheme < CGL_STRANG || scheme > CGL_SPLIT4_3T ? CGL_EINVAL : CGL_EUNSUPPORTED,
                "batches support the exponential schemes strang, split4, lawson4, lawson2");
  for (int i = 0; i < count; ++i)
    for (int m = 0; m < probs[i].d && m < 3; ++m)
      if (probs[i].bc[m] == CGL_BC_PERIODIC)
        return fail(CGL_EUNSUPPORTED, "batches take finite-difference (Dirichlet/Neumann) problems");
  cgl_batch* b = new cgl_batch();
  cudaGetDevice(&b->dev);
  b->count = count;
  b->scheme = scheme;
  b->precision = precision;
  b->tau = tau;
  b->elem = precision == CGL_F64 ? sizeof(double2) : sizeof(float2);
  int st = CGL_OK;
  for (int i = 0; i < count && !st; ++i) {
    const cgl_problem& q = probs[i];
    cgl_plan* p = nullptr;
    st = plan_create_impl(&p, q.d, q.n, q.bc, q.lo, q.hi, q.a1, q.b1, q.a2, q.a3, q.b3, q.a4, q.b4, tau, scheme,
                          precision, stream, true);
    if (!st) {
      b->plans.push_back(p);
      b->offsets.push_back(b->total);
      b->total += p->N;
    } else {
      char msg[64];
      std::snprintf(msg, sizeof(msg), "instance %d: ", i);
      fail(st, msg + std::string(cgl_last_error()));
    }
  }
  const int nwork = st ? 0 : b->plans[0]->nwork;
  for (int w = 0; !st && w < nwork; ++w) st = batch_alloc(b, &b->work[w], b->total * b->elem);
  if (!st) st = batch_alloc(b, (void**)&b->status, sizeof(int));
  if (!st && cudaMemset(b->status, 0, sizeof(int)) != cudaSuccess) st = fail(CGL_ECUDA, "memset status");
  if (!st && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    st = fail(CGL_ECUDA, "stream create");
  // passes and their work lists
  const int sms = st ? 0 : sm_count();
  const int nsweeps = st ? 0 : (int)b->plans[0]->sweeps.size();
  const int d_max = 3;
  for (int sw = 0; !st && sw < nsweeps; ++sw) {
    for (int mu = 0; !st && mu < d_max; ++mu) {
      // instances with at least mu+1 directions take part in this pass
      bool any = false;
      for (cgl_plan* p : b->plans) any |= p->d > mu;
      if (!any) continue;
      cgl_batch::Pass ps;
      ps.sweep = sw;
      ps.mu = mu;
      ps.nrhs = b->plans[0]->sweeps[sw].nrhs;
      std::vector<BatchItem> items;
      std::vector<double> cost;
      for (int i = 0; i < count && !st; ++i) {
        cgl_plan* p = b->plans[i];
        if (p->d <= mu) continue;
        const int n = (int)p->n[mu];
        const bool contiguous = axis_P(p, mu) == 1;
        int tb = 1;
        st = autotune(n, contiguous, precision, ps.nrhs, &tb, nullptr);
        const int64_t np = p->N / n;
        tb = (int)std::min<int64_t>(tb, np);
        ps.smem = std::max(ps.smem, mode_smem_bytes(n, ps.nrhs, b->elem, tb));
        for (int64_t b0 = 0; b0 < np; b0 += tb) {
          items.push_back(BatchItem{i, tb, b0});
          cost.push_back((double)std::min<int64_t>(tb, np - b0) * n * n);
        }
      }
      if (st) break;
      std::vector<size_t> order(items.size());
      std::iota(order.begin(), order.end(), 0);
      std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
      std::vector<BatchItem> sorted(items.size());
      for (size_t k = 0; k < order.size(); ++k) sorted[k] = items[order[k]];
      ps.nitems = (int)sorted.size();
      st = batch_alloc(b, (void**)&ps.items, sorted.size() * sizeof(BatchItem));
      if (!st && cudaMemcpy(ps.items, sorted.data(), sorted.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) !=
                     cudaSuccess)
        st = fail(CGL_ECUDA, "upload work list");
      if (!st) st = batch_alloc(b, (void**)&ps.table, (size_t)count * sizeof(ModePassArgs));
      const int per_sm = precision == CGL_F64 ? batched_mode_blocks_per_sm<double>(ps.nrhs, ps.smem)
                                              : batched_mode_blocks_per_sm<float>(ps.nrhs, ps.smem);
      ps.grid = (int)std::min<int64_t>((int64_t)per_sm * sms, std::max(1, ps.nitems));
      b->passes.push_back(ps);
    }
  }
  if (!st) st = batch_alloc(b, (void**)&b->counters, std::max<size_t>(1, b->passes.size()) * sizeof(int));
  if (st) {
    free_batch(b);
    return st;
  }
  *out = b;
  return CGL_OK;
}

int cgl_batch_info(const cgl_batch* b, int64_t* total_points, int64_t* offsets, size_t* workspace_bytes,
                   int* launches_per_step) {
  if (!b) return fail(CGL_EINVAL, "batch is NULL");
  if (total_points) *total_points = b->total;
  if (offsets)
    for (int i = 0; i < b->count; ++i) offsets[i] = b->offsets[i];
  if (workspace_bytes) {
    int nw = 0;
    for (void* w : b->work) nw += w != nullptr;
    *workspace_bytes = (size_t)nw * b->total * b->elem;
  }
  if (launches_per_step) *launches_per_step = (int)b->passes.size();
  return CGL_OK;
}

int cgl_batch_step(cgl_batch* b, void* u, int64_t nsteps, void* stream) {
  if (!b || !u) return fail(CGL_EINVAL, "batch and u must be non-NULL");
  if (nsteps < 0) return fail(CGL_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return CGL_OK;
  CUDA_TRY(cudaSetDevice(b->dev));
  int st = ensure_batch_graph(b, u);
  if (st) return st;
  for (int64_t k = 0; k < nsteps; ++k) CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return CGL_OK;
}

int cgl_batch_last_device_status(cgl_batch* b, void* stream) {
  if (!b) return fail(CGL_EINVAL, "batch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, b->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemsetAsync(b->status, 0, sizeof(int), s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h & 2) return fail(CGL_ETIMEOUT, "a device-side wait timed out");
  return (h & 1) ? CGL_ENONFINITE : CGL_OK;
}

int cgl_batch_destroy(cgl_batch* b) {
  if (!b) return CGL_OK;
  cudaSetDevice(b->dev);
  free_batch(b);
  return CGL_OK;
}

}  // extern "C"
