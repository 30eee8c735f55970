// Batched integration of many independent CGL instances (uneven grids,
// boundary conditions and parameters): FP64 / FP32 take one persistent launch
// per time step (every mu-mode pass of every sweep in one work list, ordered
// per instance by dependency counters), BF16x3 one grouped launch per
// pointwise stage and mu-mode pass; the step is replayed as one CUDA graph.
//
// Each instance gets its own FP64-computed factors exp(c tau A_mu) (a factor-
// only plan).  All fields live in one packed buffer: instance i's N_i values
// start at offset_i = sum_{j<i} N_j.  For every pass (sweep, mode) the host
// builds a work list of (instance, first fiber, fibers per tile) items ordered
// by decreasing cost; the lists of a step's passes are concatenated, and a
// fixed grid of CTAs (SMs x resident CTAs) drains them through an atomic
// counter, so large and small instances share the machine without a launch
// per instance or per pass.  An item waits (bounded) until its instance's
// previous pass has finished; it never waits on a later item.
//
// Fibers per tile come from an autotuner: for each (n, contiguous fibers or
// not, precision, right-hand sides, SM count) it times the mode-pass kernel on
// a synthetic 2048-fiber field for every admissible tile size and keeps the
// fastest, in memory and in the text file named by $CGL_AUTOTUNE_CACHE.
//
// BF16x3 batches run every mode pass on the tensor cores: per sweep one
// grouped split prologue (a segment per instance), one persistent tcgen05
// pass per mode (a device table of per-instance pass arguments and tensor
// maps and a list of (instance, tile) records that the CTAs walk round-robin)
// and one grouped plane epilogue, over the BF16 / FP32 planes and factor
// splits that each instance's plan owns.
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
    int nitems = 0;
    ModePassArgs* table = nullptr;  // device, one entry per instance (inside `tables`)
  };
  std::vector<Pass> passes;
  // SIMT precisions: the whole step as one persistent launch over every
  // pass's items (StepArgs); tables of all passes in one array
  ModePassArgs* tables = nullptr;  // device [npass][count]
  StepItem* step_items = nullptr;
  int* need = nullptr;
  int* prev = nullptr;
  int step_nitems = 0;
  size_t step_smem = 0;
  int step_grid = 0;
  // BF16x3: per sweep, grouped pointwise stages and one grouped tcgen05 pass
  // per mode
  struct MmaMode {
    void* passes = nullptr;  // device MmaPassArgs[npass]
    void* maps = nullptr;    // device CUtensorMap[4 npass]
    void* tiles = nullptr;   // device int2 (pass, tile) of every tile per rhs
    int npass = 0;
    int64_t ctas = 0;        // tiles per rhs
  };
  struct MmaSweep {
    int sweep = 0, nrhs = 1;
    SplitSeg* pro = nullptr;  // device, one per instance
    EpiSeg* epi = nullptr;    // device, one per instance
    int64_t max_n = 0;
    std::vector<MmaMode> modes;
  };
  std::vector<MmaSweep> msweeps;
  int inject_wait_failure = 0;  // test hook: the step kernel's dependency waits cannot be met
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
  if (injected_alloc_failure()) {
    *ptr = nullptr;
    return fail(CGL_ENOMEM, "cudaMalloc: injected allocation failure");
  }
  cudaError_t e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail(CGL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  b->allocations.push_back(*ptr);
  return CGL_OK;
}

// Per-instance buffers of field buffer u: u, then the work fields.
void instance_bufs(const cgl_batch* b, void* u, int i, void** bufs) {
  const size_t off = (size_t)b->offsets[i] * b->elem;
  bufs[0] = (char*)u + off;
  for (int w = 0; w < 3; ++w) bufs[1 + w] = b->work[w] ? (char*)b->work[w] + off : nullptr;
}

// BF16x3: the pointwise segments of every sweep for field buffer u.
int upload_mma_segments(cgl_batch* b, void* u) {
  std::vector<SplitSeg> pro(b->count);
  std::vector<EpiSeg> epi(b->count);
  for (auto& ms : b->msweeps) {
    for (int i = 0; i < b->count; ++i) {
      cgl_plan* p = b->plans[i];
      const Sweep& sw = p->sweeps[ms.sweep];
      void* bufs[NBUF];
      instance_bufs(b, u, i, bufs);
      SplitSeg g{};
      for (int r = 0; r < 2; ++r) {
        g.in[r] = static_cast<const float2*>(bufs[sw.in[r]]);
        g.dst[r] = p->splits[r < sw.nrhs ? r : 0];
      }
      g.nin = sw.nin;
      g.op = sw.op;
      g.N = p->N;
      g.n1 = p->n[0];
      g.pitch = p->pitch;
      g.Npad = p->Npad;
      pro[i] = g;
      EpiSeg e{};
      for (int r = 0; r < 2; ++r) {
        e.y[r] = static_cast<const float*>(p->planes[r < sw.nrhs ? r : 0]);
        e.out[r] = static_cast<float2*>(bufs[sw.out[r]]);
      }
      for (int x = 0; x < kMaxExtra; ++x) e.ex[x] = static_cast<const float2*>(bufs[sw.extra[x]]);
      e.nextra = sw.nextra;
      e.nout = sw.nout;
      e.op = sw.op;
      e.N = p->N;
      e.n1 = p->n[0];
      e.pitch = p->pitch;
      e.Npad = p->Npad;
      epi[i] = e;
    }
    CUDA_TRY(cudaMemcpy(ms.pro, pro.data(), pro.size() * sizeof(SplitSeg), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(ms.epi, epi.data(), epi.size() * sizeof(EpiSeg), cudaMemcpyHostToDevice));
  }
  return CGL_OK;
}

// Per-instance pass arguments for field buffer u (device tables).
int upload_tables(cgl_batch* b, void* u) {
  if (b->precision == CGL_BF16X3) return upload_mma_segments(b, u);
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
  for (const auto& ms : b->msweeps) {
    SplitSeg none{};
    cudaError_t e = launch_split_prologue(none, ms.pro, b->count, ms.max_n, ms.nrhs, s);
    if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("batched split prologue: ") + cudaGetErrorString(e));
    for (const auto& md : ms.modes) {
      e = launch_mma_group(md.passes, md.maps, md.tiles, md.npass, md.ctas, ms.nrhs, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("batched tensor-core pass: ") + cudaGetErrorString(e));
    }
    EpiSeg enone{};
    e = launch_plane_epilogue(enone, ms.epi, b->count, ms.max_n, ms.nrhs, b->status, s);
    if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("batched plane epilogue: ") + cudaGetErrorString(e));
  }
  if (!b->passes.empty()) {
    const int npass = (int)b->passes.size();
    CUDA_TRY(cudaMemsetAsync(b->counters, 0, (2 + (size_t)npass * b->count) * sizeof(int), s));
    StepArgs a{};
    a.table = b->tables;
    a.items = b->step_items;
    a.nitems = b->step_nitems;
    a.need = b->need;
    a.prev = b->prev;
    a.npass = npass;
    a.count = b->count;
    a.counter = b->counters;
    a.status = b->status;
    a.spin_limit = b->inject_wait_failure ? kStepInjectedSpinLimit : kStepSpinLimit;
    a.want_bias = b->inject_wait_failure ? 1 : 0;
    cudaError_t e = b->precision == CGL_F64 ? launch_batched_step<double>(a, b->step_smem, b->step_grid, s)
                                            : launch_batched_step<float>(a, b->step_smem, b->step_grid, s);
    if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("batched step: ") + cudaGetErrorString(e));
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

// BF16x3: the grouped tensor-core passes of every sweep (pass arguments and
// tensor maps do not depend on the field buffer) and room for the pointwise
// segments.
int build_mma_sweeps(cgl_batch* b) {
  const int nsweeps = (int)b->plans[0]->sweeps.size();
  for (int sw = 0; sw < nsweeps; ++sw) {
    cgl_batch::MmaSweep ms;
    ms.sweep = sw;
    ms.nrhs = b->plans[0]->sweeps[sw].nrhs;
    for (cgl_plan* p : b->plans) ms.max_n = std::max(ms.max_n, p->N);
    int st = batch_alloc(b, (void**)&ms.pro, (size_t)b->count * sizeof(SplitSeg));
    if (!st) st = batch_alloc(b, (void**)&ms.epi, (size_t)b->count * sizeof(EpiSeg));
    if (st) return st;
    for (int mu = 0; mu < 3; ++mu) {
      std::vector<MmaPassArgs> args;
      std::vector<unsigned char> maps;
      std::vector<int64_t> ctas;
      std::vector<double> cost;
      for (int i = 0; i < b->count; ++i) {
        cgl_plan* p = b->plans[i];
        if (p->d <= mu) continue;
        const Sweep& w = p->sweeps[sw];
        MmaLaunch L{};
        L.n = (int)p->n[mu];
        L.P = mma_axis_P(p, mu);
        L.Q = mma_axis_Q(p, mu);
        L.N = p->Npad;
        L.pitch = p->pitch;
        L.nrhs = w.nrhs;
        for (int r = 0; r < 2; ++r) {
          const int rr = r < w.nrhs ? r : 0;
          L.tmA[r] = p->tmA[mu][rr];
          L.tmB[r] = p->tmB[w.fac[rr]][mu];
          // as in a single plan: mode passes alternate between the two plane
          // sets, the last one writes the FP32 planes
          L.out[r] = (mu == p->d - 1) ? p->planes[rr] : ((mu & 1) ? p->splits[rr] : p->splits_alt[rr]);
        }
        L.out_fp32 = mu == p->d - 1;
        L.status = b->status;
        L.grouped = 1;
        MmaPassArgs a;
        const int64_t c = mma_build_args(L, &a);
        if (c < 0) {
          char msg[96];
          std::snprintf(msg, sizeof(msg), "instance %d: mode %d not supported by the tensor-core pass", i, mu + 1);
          return fail(CGL_EUNSUPPORTED, msg);
        }
        args.push_back(a);
        // A maps as the plan's; B maps with the grouped pass's rows per tile
        alignas(64) unsigned char fm[2][kTensorMapBytes];
        for (int r = 0; r < 2; ++r) {
          const int rr = r < w.nrhs ? r : 0;
          CUDA_TRY(make_factor_tmap(fm[r], p->fsplit[w.fac[rr]][mu], L.n, 3, a.nc));
        }
        for (const void* m : {L.tmA[0], L.tmA[1], (const void*)fm[0], (const void*)fm[1]}) {
          const unsigned char* q = static_cast<const unsigned char*>(m);
          maps.insert(maps.end(), q, q + kTensorMapBytes);
        }
        ctas.push_back(c);
        cost.push_back((double)c * a.np);
      }
      if (args.empty()) continue;
      // largest passes first, so that the CTAs' round-robin shares of the
      // tiles come out even
      std::vector<size_t> order(args.size());
      std::iota(order.begin(), order.end(), 0);
      std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
      std::vector<MmaPassArgs> sargs(args.size());
      std::vector<unsigned char> smaps(maps.size());
      std::vector<int> tiles;  // (pass, tile) pairs
      cgl_batch::MmaMode md;
      for (size_t k = 0; k < order.size(); ++k) {
        const size_t o = order[k];
        sargs[k] = args[o];
        std::copy(maps.begin() + o * 4 * kTensorMapBytes, maps.begin() + (o + 1) * 4 * kTensorMapBytes,
                  smaps.begin() + k * 4 * kTensorMapBytes);
        for (int64_t t = 0; t < ctas[o]; ++t) {
          tiles.push_back((int)k);
          tiles.push_back((int)t);
        }
      }
      const int64_t total = (int64_t)tiles.size() / 2;
      if (total * ms.nrhs >= (int64_t)1 << 31) return fail(CGL_EUNSUPPORTED, "batch too large for one grouped pass");
      md.npass = (int)sargs.size();
      md.ctas = total;
      st = batch_alloc(b, &md.passes, sargs.size() * sizeof(MmaPassArgs));
      if (!st) st = batch_alloc(b, &md.maps, smaps.size());
      if (!st) st = batch_alloc(b, &md.tiles, tiles.size() * sizeof(int));
      if (st) return st;
      CUDA_TRY(cudaMemcpy(md.passes, sargs.data(), sargs.size() * sizeof(MmaPassArgs), cudaMemcpyHostToDevice));
      CUDA_TRY(cudaMemcpy(md.maps, smaps.data(), smaps.size(), cudaMemcpyHostToDevice));
      CUDA_TRY(cudaMemcpy(md.tiles, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice));
      ms.modes.push_back(md);
    }
    b->msweeps.push_back(ms);
  }
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
  if (precision != CGL_F64 && precision != CGL_F32 && precision != CGL_BF16X3)
    return fail(precision < CGL_F64 || precision > CGL_F64_TC ? CGL_EINVAL : CGL_EUNSUPPORTED,
                "batches run in CGL_F64, CGL_F32 or CGL_BF16X3");
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
  b->elem = precision == CGL_F64 ? sizeof(double2) : sizeof(float2);  // BF16x3: complex64 state
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
  if (!st && precision == CGL_BF16X3) st = build_mma_sweeps(b);
  // passes and their work lists (SIMT precisions)
  const int sms = st ? 0 : sm_count();
  const int nsweeps = (st || precision == CGL_BF16X3) ? 0 : (int)b->plans[0]->sweeps.size();
  const int d_max = 3;
  std::vector<StepItem> step_items;
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
      const int k = (int)b->passes.size();
      for (const BatchItem& it : sorted) step_items.push_back(StepItem{k, it.inst, it.tb, it.b0});
      b->passes.push_back(ps);
    }
  }
  // the step list, its dependency tables and the pass tables in one array
  if (!st && !b->passes.empty()) {
    const int npass = (int)b->passes.size();
    std::vector<int> need((size_t)npass * count, 0), prev((size_t)npass * count, -1), last(count, -1);
    for (const StepItem& it : step_items) need[(size_t)it.pass * count + it.inst] += 1;
    for (int k = 0; k < npass; ++k)
      for (int i = 0; i < count; ++i)
        if (need[(size_t)k * count + i] > 0) {
          prev[(size_t)k * count + i] = last[i];
          last[i] = k;
        }
    b->step_nitems = (int)step_items.size();
    for (const auto& ps : b->passes) b->step_smem = std::max(b->step_smem, ps.smem);
    st = batch_alloc(b, (void**)&b->step_items, step_items.size() * sizeof(StepItem));
    if (!st) st = batch_alloc(b, (void**)&b->need, need.size() * sizeof(int));
    if (!st) st = batch_alloc(b, (void**)&b->prev, prev.size() * sizeof(int));
    if (!st) st = batch_alloc(b, (void**)&b->tables, (size_t)npass * count * sizeof(ModePassArgs));
    if (!st && (cudaMemcpy(b->step_items, step_items.data(), step_items.size() * sizeof(StepItem),
                           cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(b->need, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(b->prev, prev.data(), prev.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
      st = fail(CGL_ECUDA, "upload work list");
    for (int k = 0; !st && k < npass; ++k) b->passes[k].table = b->tables + (size_t)k * count;
    if (!st) {
      const int per_sm = precision == CGL_F64 ? batched_step_blocks_per_sm<double>(b->step_smem)
                                              : batched_step_blocks_per_sm<float>(b->step_smem);
      b->step_grid = (int)std::min<int64_t>((int64_t)per_sm * sms, std::max(1, b->step_nitems));
    }
    if (!st) st = batch_alloc(b, (void**)&b->counters, (2 + (size_t)npass * count) * sizeof(int));
  }
  if (!st && !b->counters) st = batch_alloc(b, (void**)&b->counters, 2 * sizeof(int));
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
  if (launches_per_step) {
    int l = b->passes.empty() ? 0 : 1;  // SIMT precisions: one persistent launch per step
    for (const auto& ms : b->msweeps) l += 2 + (int)ms.modes.size();
    *launches_per_step = l;
  }
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

int cgl_batch_inject_wait_failure(cgl_batch* b, int on) {
  if (!b) return fail(CGL_EINVAL, "batch is NULL");
  if (b->passes.empty()) return fail(CGL_EUNSUPPORTED, "wait-failure injection: FP64 / FP32 batches only");
  CUDA_TRY(cudaSetDevice(b->dev));
  b->inject_wait_failure = on ? 1 : 0;
  if (b->exec) {  // the step's arguments are part of its graph: capture it again
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaGraphExecDestroy(b->exec));
    b->exec = nullptr;
    b->graph_u = nullptr;
  }
  return CGL_OK;
}

int cgl_batch_destroy(cgl_batch* b) {
  if (!b) return CGL_OK;
  cudaSetDevice(b->dev);
  free_batch(b);
  return CGL_OK;
}

}  // extern "C"
