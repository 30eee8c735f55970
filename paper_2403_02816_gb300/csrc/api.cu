// libcgl C ABI: plan creation (space discretisation and factor precompute),
// the per-scheme step programs, CUDA-graph replay, profiling hooks.
//
// A time step is a short program of "sweeps".  A sweep applies one linear
// flow exp(c tau K) (or K itself for the Runge-Kutta schemes) to one or two
// fields, with a pointwise prologue fused into its first pass and a pointwise
// epilogue fused into its last pass (see ProOp / EpiOp).  A sweep is d
// mu-mode passes (finite differences, eq. Tucker) or 2d-1 FFT pencil passes
// (periodic, Sec. 3.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "cgl_internal.cuh"
#include "plan.cuh"

using namespace cgl;

namespace cgl {

thread_local std::string g_last_error;

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

}  // namespace cgl


namespace cgl {

int64_t axis_P(const cgl_plan* p, int axis) {
  int64_t P = 1;
  for (int m = 0; m < axis; ++m) P *= p->n[m];
  return P;
}

// Periodic sizes the FFT passes take: 2 <= n <= 2048 with no prime factor
// above 7 (powers of two: radix-4/2 passes; else mixed radix 4, 2, 3, 5, 7).
bool fft_size_ok(int64_t n) {
  if (n < 2 || n > 2048) return false;
  for (int r : {2, 3, 5, 7})
    while (n % r == 0) n /= r;
  return n == 1;
}

// Tensor-core planes: the faster product with the first direction padded to
// the plane pitch, and the slower product.
int64_t mma_axis_P(const cgl_plan* p, int axis) {
  if (axis == 0) return 1;
  int64_t P = p->pitch;
  for (int m = 1; m < axis; ++m) P *= p->n[m];
  return P;
}
int64_t mma_axis_Q(const cgl_plan* p, int axis) {
  int64_t Q = 1;
  for (int m = axis + 1; m < p->d; ++m) Q *= p->n[m];
  return Q;
}

PassGeom geom(const cgl_plan* p, int axis) {
  PassGeom g{};
  g.d = p->d;
  for (int m = 0; m < 3; ++m) g.n[m] = p->n[m];
  g.axis = axis;
  g.n_ax = p->n[axis];
  g.P = axis_P(p, axis);
  g.npencils = p->N / p->n[axis];
  return g;
}

// Algorithmic flop count per grid point of the pointwise operators (real
// flops, transcendental calls not counted): g = 15, exact flow = 20,
// one RK4 step of u' = g(u) = 84, complex axpy = 4; the three-term
// operators compose two (prologue, end of step) or three (middle) exact flows.
double flow_flops(const cgl_plan* p) { return p->cubic ? 20.0 : 84.0; }
double pro_flops(const cgl_plan* p, const OpArgs& o) {
  switch (o.pro) {
    case PRO_FLOW: return flow_flops(p);
    case PRO_FLOW2: return 2 * flow_flops(p);
    case PRO_LAW4: return 15;
    case PRO_LAW2: return 23;
    case PRO_CQ: return 40;
    case PRO_CQ2: return 80;
    case PRO_CFLOW: return 160;  // one coupled RK4 step: 4 x (g_u, g_v) + combinations
    case PRO_CG: return 34;
    case PRO_CLAW2: return 42;
    default: return 0;
  }
}
double epi_flops(const cgl_plan* p, const OpArgs& o) {
  switch (o.epi) {
    case EPI_FLOW: return flow_flops(p);
    case EPI_FLOW2: return 2 * flow_flops(p);
    case EPI_SPLIT4: return flow_flops(p) + 4;
    case EPI_LAW4A: return 46;
    case EPI_LAW4B: return 19;
    case EPI_LAW2: return 19;
    case EPI_RK: return 25;
    case EPI_QC: return 40;
    case EPI_QC2: return 100;
    case EPI_SPLIT4_3T: return 44;
    case EPI_CFLOW: return 160;
    case EPI_CSPLIT4: return 168;
    case EPI_CLAW4P: return 84;
    case EPI_CLAW4W: return 96;
    case EPI_CLAW4B:
    case EPI_CLAW2: return 42;
    default: return 0;
  }
}

struct Timer {
  cgl_plan* p;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Timer(cgl_plan* p_, cudaStream_t s_) : p(p_), s(s_) {
    if (p->prof) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
    }
  }
  void done(const std::string& name, double flops, double bytes) {
    if (!p->prof) return;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    KernelStat& k = (*p->stats)[name];
    k.launches += 1;
    k.ms += ms;
    k.flops += flops;
    k.bytes += bytes;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
};

// Pointer of a sweep slot: buffer `id`, field `f` (coupled system: v is N
// values after u).
static void* slot_ptr(const cgl_plan* p, void* const* bufs, int id, int f) {
  void* b = bufs[id];
  return (b && f) ? static_cast<char*>(b) + (size_t)f * p->N * p->elem : b;
}

ModePassArgs make_mode_args(const cgl_plan* p, const Sweep& sw, int mu, void* const* bufs) {
  ModePassArgs a{};
  a.g = geom(p, mu);
  a.f.nin = sw.nin;
  a.f.nrhs = sw.nrhs;
  a.f.nextra = sw.nextra;
  a.f.nout = sw.nout;
  for (int r = 0; r < 2; ++r) {
    a.f.in[r] = slot_ptr(p, bufs, sw.in[r], sw.in_f[r]);
    a.f.work[r] = slot_ptr(p, bufs, sw.work[r], sw.work_f[r]);
    a.f.out[r] = slot_ptr(p, bufs, sw.out[r], sw.out_f[r]);
  }
  for (int x = 0; x < kMaxExtra; ++x) a.f.extra[x] = slot_ptr(p, bufs, sw.extra[x], sw.extra_f[x]);
  a.op = sw.op;
  a.flags = (mu == 0 ? PASS_PRO : 0) | (mu == p->d - 1 ? PASS_EPI : 0);
  for (int r = 0; r < 2; ++r) a.factor[r] = p->fac[sw.fac[r < sw.nrhs ? r : 0]][mu];
  a.status = p->status;
  return a;
}

int enqueue_sweep(cgl_plan* p, const Sweep& sw, void* u, cudaStream_t s) {
  void* bufs[NBUF] = {u, p->work[0], p->work[1], p->work[2]};
  PassFields f{};
  f.nin = sw.nin;
  f.nrhs = sw.nrhs;
  f.nextra = sw.nextra;
  f.nout = sw.nout;
  for (int r = 0; r < 2; ++r) {
    f.in[r] = slot_ptr(p, bufs, sw.in[r], sw.in_f[r]);
    f.work[r] = slot_ptr(p, bufs, sw.work[r], sw.work_f[r]);
    f.out[r] = slot_ptr(p, bufs, sw.out[r], sw.out_f[r]);
  }
  for (int x = 0; x < kMaxExtra; ++x) f.extra[x] = slot_ptr(p, bufs, sw.extra[x], sw.extra_f[x]);
  const double Nd = (double)p->N;
  const double es = (double)p->elem;
  const bool f64 = p->elem == sizeof(double2);

  if (sw.stencil) {
    StencilArgs a{};
    a.d = p->d;
    for (int mu = 0; mu < 3; ++mu) {
      a.n[mu] = p->n[mu];
      a.bc[mu] = p->bc[mu];
      if (mu < p->d) {
        const double L = p->hi[mu] - p->lo[mu];
        const double h = (p->bc[mu] == CGL_BC_DIRICHLET) ? L / (p->n[mu] + 1) : L / (p->n[mu] - 1);
        a.cr[mu] = p->a1 / (h * h);
        a.ci[mu] = p->b1 / (h * h);
        a.crf[mu] = (float)a.cr[mu];
        a.cif[mu] = (float)a.ci[mu];
      }
    }
    a.a2 = p->a2;
    a.a2f = (float)p->a2;
    a.x = f.in[0];
    for (int x = 0; x < kMaxExtra; ++x) a.extra[x] = f.extra[x];
    a.nextra = sw.nextra;
    a.out[0] = f.out[0];
    a.out[1] = f.out[1];
    a.nout = sw.nout;
    a.op = sw.op;
    a.status = p->status;
    Timer tm(p, s);
    cudaError_t e = f64 ? launch_kron_stencil<double>(a, s) : launch_kron_stencil<float>(a, s);
    if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("stencil: ") + cudaGetErrorString(e));
    tm.done(f64 ? "kron_stencil_f64" : "kron_stencil_f32", (8.0 * p->d + 4 + epi_flops(p, sw.op)) * Nd,
            (1.0 + sw.nextra + sw.nout) * Nd * es);
    return CGL_OK;
  }

  if (p->precision == CGL_F64_TC) {
    // FP64 prologue -> per mode: digit slicing + tensor-core pass -> FP64 epilogue
    OzSeg g{};
    g.in[0] = static_cast<const double2*>(f.in[0]);
    g.in[1] = static_cast<const double2*>(f.in[1]);
    g.nin = sw.nin;
    g.op = sw.op;
    for (int r = 0; r < 2; ++r) g.z[r] = static_cast<double*>(p->oz_z[r < sw.nrhs ? r : 0]);
    for (int x = 0; x < kMaxExtra; ++x) g.ex[x] = static_cast<const double2*>(f.extra[x]);
    g.nextra = sw.nextra;
    g.out[0] = static_cast<double2*>(f.out[0]);
    g.out[1] = static_cast<double2*>(f.out[1]);
    g.nout = sw.nout;
    g.N = p->N;
    g.n1 = p->n[0];
    g.pitch = p->pitch;
    g.Npad = p->Npad;
    {
      Timer tm(p, s);
      cudaError_t e = launch_oz_prologue(g, sw.nrhs, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("FP64 prologue: ") + cudaGetErrorString(e));
      tm.done("oz_prologue", pro_flops(p, sw.op) * Nd, (sw.nin * 16.0 + sw.nrhs * 16.0) * Nd);
    }
    for (int mu = 0; mu < p->d; ++mu) {
      for (int r = 0; r < sw.nrhs; ++r) {
        OzSliceArgs sl{};
        sl.z = static_cast<const double*>(p->oz_z[r]);
        sl.dst = static_cast<__nv_bfloat16*>(p->oz_dig[r]);
        sl.exps = p->oz_exp[r];
        sl.n = (int)p->n[mu];
        sl.P = mma_axis_P(p, mu);
        sl.Q = mma_axis_Q(p, mu);
        sl.N = p->Npad;
        sl.pitch = p->pitch;
        sl.status = p->status;
        Timer tm(p, s);
        cudaError_t e = launch_oz_slice(sl, s);
        if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("digit slicing: ") + cudaGetErrorString(e));
        tm.done("oz_slice", 0.0, (16.0 + 28.0) * Nd);
      }
      OzLaunch L{};
      L.n = (int)p->n[mu];
      L.P = mma_axis_P(p, mu);
      L.Q = mma_axis_Q(p, mu);
      L.N = p->Npad;
      L.pitch = p->pitch;
      L.nrhs = sw.nrhs;
      for (int r = 0; r < 2; ++r) {
        const int rr = r < sw.nrhs ? r : 0;
        L.tmA[r] = p->oz_tmA[mu][rr];
        L.tmB[r] = p->tmB[sw.fac[rr]][mu];
        L.aexp[r] = p->oz_exp[rr];
        L.bexp[r] = p->fexp[sw.fac[rr]][mu];
        L.out[r] = static_cast<double*>(p->oz_z[rr]);
      }
      L.status = p->status;
      Timer tm(p, s);
      cudaError_t e = launch_oz_pass(L, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("tensor-core FP64 pass: ") + cudaGetErrorString(e));
      // issued tensor flops: 28 digit products of a (2n x 2n) real GEMM per fiber
      tm.done("oz_mode_f64tc", 28.0 * 8.0 * (double)p->n[mu] * Nd * sw.nrhs, (28.0 + 16.0) * Nd * sw.nrhs);
    }
    {
      Timer tm(p, s);
      cudaError_t e = launch_oz_epilogue(g, sw.nrhs, p->status, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("FP64 epilogue: ") + cudaGetErrorString(e));
      tm.done("oz_epilogue", epi_flops(p, sw.op) * Nd, (sw.nrhs * 16.0 + (sw.nextra + sw.nout) * 16.0) * Nd);
    }
    return CGL_OK;
  }

  if (p->precision == CGL_BF16X3) {
    // split prologue -> d tensor-core mode passes -> plane epilogue
    {
      Timer tm(p, s);
      SplitSeg g{};
      g.in[0] = static_cast<const float2*>(f.in[0]);
      g.in[1] = static_cast<const float2*>(f.in[1]);
      g.nin = sw.nin;
      g.op = sw.op;
      g.dst[0] = p->splits[0];
      g.dst[1] = p->splits[1];
      g.N = p->N;
      g.n1 = p->n[0];
      g.pitch = p->pitch;
      g.Npad = p->Npad;
      cudaError_t e = launch_split_prologue(g, nullptr, 1, p->N, sw.nrhs, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("split prologue: ") + cudaGetErrorString(e));
      tm.done("split_prologue", pro_flops(p, sw.op) * Nd, (sw.nin * 8.0 + sw.nrhs * 12.0) * Nd);
    }
    for (int mu = 0; mu < p->d; ++mu) {
      MmaLaunch L{};
      L.n = (int)p->n[mu];
      L.P = mma_axis_P(p, mu);
      L.Q = mma_axis_Q(p, mu);
      L.N = p->Npad;
      L.pitch = p->pitch;
      L.nrhs = sw.nrhs;
      for (int r = 0; r < 2; ++r) {
        const int rr = r < sw.nrhs ? r : 0;
        L.tmA[r] = p->tmA[mu][rr];
        L.tmB[r] = p->tmB[sw.fac[rr]][mu];
        // mode mu reads splits (mu even) or splits_alt (mu odd) and writes the
        // other set: the row blocks of one fiber tile are separate work
        // items, so an in-place pass would overwrite input that the tile's
        // other items still read
        L.out[r] = (mu == p->d - 1) ? p->planes[rr] : ((mu & 1) ? p->splits[rr] : p->splits_alt[rr]);
      }
      L.out_fp32 = mu == p->d - 1;
      L.status = p->status;
      Timer tm(p, s);
      cudaError_t e = launch_mma_pass(L, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("tensor-core mode pass: ") + cudaGetErrorString(e));
      // issued tensor flops: 6 split products of a (2n x 2n) real GEMM per fiber
      tm.done("mma_mode_bf16x3", 6.0 * 8.0 * (double)p->n[mu] * Nd * sw.nrhs,
              (12.0 + (L.out_fp32 ? 8.0 : 12.0)) * Nd * sw.nrhs);
    }
    {
      Timer tm(p, s);
      EpiSeg g{};
      g.y[0] = static_cast<const float*>(p->planes[0]);
      g.y[1] = static_cast<const float*>(p->planes[1]);
      for (int x = 0; x < kMaxExtra; ++x) g.ex[x] = static_cast<const float2*>(f.extra[x]);
      g.nextra = sw.nextra;
      g.op = sw.op;
      g.out[0] = static_cast<float2*>(f.out[0]);
      g.out[1] = static_cast<float2*>(f.out[1]);
      g.nout = sw.nout;
      g.N = p->N;
      g.n1 = p->n[0];
      g.pitch = p->pitch;
      g.Npad = p->Npad;
      cudaError_t e = launch_plane_epilogue(g, nullptr, 1, p->N, sw.nrhs, p->status, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("plane epilogue: ") + cudaGetErrorString(e));
      tm.done("plane_epilogue", epi_flops(p, sw.op) * Nd, (sw.nrhs * 8.0 + (sw.nextra + sw.nout) * 8.0) * Nd);
    }
    return CGL_OK;
  }

  if (!p->periodic) {
    for (int mu = 0; mu < p->d; ++mu) {
      const ModePassArgs a = make_mode_args(p, sw, mu, bufs);
      double flops = 8.0 * (double)p->n[mu] * Nd * sw.nrhs;
      double rd = (mu == 0 ? sw.nin : sw.nrhs), wr = (mu == p->d - 1 ? sw.nout : sw.nrhs);
      if (mu == 0) flops += pro_flops(p, sw.op) * Nd;
      if (mu == p->d - 1) { flops += epi_flops(p, sw.op) * Nd; rd += sw.nextra; }
      Timer tm(p, s);
      cudaError_t e = f64 ? launch_mode_pass<double>(a, s) : launch_mode_pass<float>(a, s);
      if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("mode pass: ") + cudaGetErrorString(e));
      tm.done(f64 ? "mode_pass_f64" : "mode_pass_f32", flops, (rd + wr) * Nd * es);
    }
    return CGL_OK;
  }

  // periodic: forward passes along axes 0..d-2, the last axis does
  // forward + symbol + inverse, then inverse passes d-2..0.
  struct PassPlan { int axis, flags; };
  std::vector<PassPlan> passes;
  const int d = p->d;
  for (int mu = 0; mu < d - 1; ++mu) passes.push_back({mu, PASS_FWD});
  passes.push_back({d - 1, PASS_FWD | PASS_MUL | PASS_INV});
  for (int mu = d - 2; mu >= 0; --mu) passes.push_back({mu, PASS_INV});
  passes.front().flags |= PASS_PRO;
  passes.back().flags |= PASS_EPI;

  for (size_t k = 0; k < passes.size(); ++k) {
    const int mu = passes[k].axis;
    FftPassArgs a{};
    a.g = geom(p, mu);
    a.f = f;
    a.op = sw.op;
    a.flags = passes[k].flags;
    for (int r = 0; r < sw.nrhs; ++r) {
      const int fi = sw.fac[r];
      for (int m = 0; m < d; ++m)
        a.sym[r].vec[m] = (fi == FAC_K) ? p->ksym[m] : (fi == FAC_K2) ? p->ksym2[m] : p->fac[fi][m];
      a.sym[r].sum_form = (fi == FAC_K || fi == FAC_K2) ? 1 : 0;
    }
    a.twiddle = p->twiddle[mu];
    a.twform = p->twform[mu];
    a.twplain = p->twplain[mu];
    a.status = p->status;
    const double nn = (double)p->n[mu];
    const double fft = 5.0 * std::log2(nn) * Nd * sw.nrhs;  // 5 n log2 n per pencil
    double flops = 0;
    if (a.flags & PASS_FWD) flops += fft;
    if (a.flags & PASS_INV) flops += fft;
    if (a.flags & PASS_MUL) flops += 6.0 * Nd * sw.nrhs;
    if (a.flags & PASS_PRO) flops += pro_flops(p, sw.op) * Nd;
    if (a.flags & PASS_EPI) flops += epi_flops(p, sw.op) * Nd;
    double rd = (a.flags & PASS_PRO) ? sw.nin : sw.nrhs;
    double wr = (a.flags & PASS_EPI) ? sw.nout : sw.nrhs;
    if (a.flags & PASS_EPI) rd += sw.nextra;
    Timer tm(p, s);
    cudaError_t e = f64 ? launch_fft_pass<double>(a, s) : launch_fft_pass<float>(a, s);
    if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("fft pass: ") + cudaGetErrorString(e));
    tm.done(f64 ? "fft_pass_f64" : "fft_pass_f32", flops, (rd + wr) * Nd * es);
  }
  return CGL_OK;
}

int enqueue_step(cgl_plan* p, void* u, cudaStream_t s) {
  for (const Sweep& sw : p->sweeps) {
    int st = enqueue_sweep(p, sw, u, s);
    if (st != CGL_OK) return st;
  }
  return CGL_OK;
}

int launches_per_step(const cgl_plan* p) {
  if (!p->periodic && (p->scheme == CGL_RK4 || p->scheme == CGL_RK2)) return (int)p->sweeps.size();  // stencils
  int per = p->periodic ? 2 * p->d - 1 : p->d;
  if (p->precision == CGL_BF16X3) per = p->d + 2;  // split prologue + d mode passes + plane epilogue
  if (p->precision == CGL_F64_TC) {
    // prologue, per mode one slicing launch per rhs and the pass, epilogue
    int total = 0;
    for (const Sweep& sw : p->sweeps) total += 2 + p->d * (sw.nrhs + 1);
    return total;
  }
  return (int)p->sweeps.size() * per;
}

// ------------------------------------------------------------ space discretisation

// 2nd-order FD d^2/dx^2 (the workloads' discretisation; the paper prints the
// 4th-order matrices of Sec. 4.1.1/4.2): Dirichlet on n interior nodes,
// h = L/(n+1), tridiag(1,-2,1)/h^2; Neumann on n nodes including both ends,
// h = L/(n-1), ghost reflection giving rows (-2, 2) and (2, -2).
// A = (a1 + i b1) D2 + (a2/d) I, n x n complex, column-major.
std::vector<double2> fd_direction_matrix(const cgl_plan* p, int mu) {
  const int n = (int)p->n[mu];
  const double L = p->hi[mu] - p->lo[mu];
  const double h = (p->bc[mu] == CGL_BC_DIRICHLET) ? L / (n + 1) : L / (n - 1);
  const double ih2 = 1.0 / (h * h);
  std::vector<double2> A((size_t)n * n, make_double2(0.0, 0.0));
  auto put = [&](int i, int j, double v) {
    A[(size_t)i + (size_t)j * n].x += p->a1 * v * ih2;
    A[(size_t)i + (size_t)j * n].y += p->b1 * v * ih2;
  };
  for (int i = 0; i < n; ++i) {
    put(i, i, -2.0);
    if (i > 0) put(i, i - 1, (p->bc[mu] == CGL_BC_NEUMANN && i == n - 1) ? 2.0 : 1.0);
    if (i < n - 1) put(i, i + 1, (p->bc[mu] == CGL_BC_NEUMANN && i == 0) ? 2.0 : 1.0);
    A[(size_t)i + (size_t)i * n].x += p->a2 / p->d;
  }
  return A;
}

double norm1(const std::vector<double2>& A, int n) {
  double best = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += std::hypot(A[(size_t)i + (size_t)j * n].x, A[(size_t)i + (size_t)j * n].y);
    best = std::max(best, s);
  }
  return best;
}

// Allocations left before the injected failure (-1: none armed).
static std::atomic<long long> g_alloc_countdown{-1};

bool injected_alloc_failure() {
  long long c = g_alloc_countdown.load();
  while (c >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
  }
  return false;
}

int dev_alloc(cgl_plan* p, void** ptr, size_t bytes) {
  if (injected_alloc_failure()) {
    *ptr = nullptr;
    return fail(CGL_ENOMEM, "cudaMalloc: injected allocation failure");
  }
  cudaError_t e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail(CGL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  p->allocations.push_back(*ptr);
  return CGL_OK;
}

// Copy an FP64 vector to a working-precision buffer.
int make_working(cgl_plan* p, const double2* src64, int64_t count, void** dst, cudaStream_t s) {
  if (p->elem == sizeof(double2)) {
    *dst = (void*)src64;
    return CGL_OK;
  }
  int st = dev_alloc(p, dst, count * sizeof(float2));
  if (st) return st;
  CUDA_TRY(convert_f64_to_f32(src64, (float2*)*dst, count, s));
  return CGL_OK;
}

int build_factors(cgl_plan* p, cudaStream_t s) {
  // FD: exp(c tau A_mu) per distinct c and direction, shared between
  // directions with identical (n, bc, lo, hi).
  int st;
  if (!p->periodic) {
    int64_t nmax = 0;
    for (int m = 0; m < p->d; ++m) nmax = std::max(nmax, p->n[m]);
    double2 *dA = nullptr, *dW = nullptr;
    if ((st = dev_alloc(p, (void**)&dA, nmax * nmax * sizeof(double2)))) return st;
    if ((st = dev_alloc(p, (void**)&dW, 3 * nmax * nmax * sizeof(double2)))) return st;
    for (int c = 0; c < p->nfac; ++c) {
      for (int mu = 0; mu < p->d; ++mu) {
        int same = -1;
        for (int nu = 0; nu < mu; ++nu) {
          if (p->n[nu] != p->n[mu]) continue;
          if (p->user_mats) {
            const auto& x = p->userA[nu];
            const auto& y = p->userA[mu];
            bool eq = true;
            for (size_t k = 0; eq && k < x.size(); ++k) eq = x[k].x == y[k].x && x[k].y == y[k].y;
            if (eq) same = nu;
          } else if (p->bc[nu] == p->bc[mu] && p->lo[nu] == p->lo[mu] && p->hi[nu] == p->hi[mu]) {
            same = nu;
          }
        }
        if (same >= 0) {
          p->fac64[c][mu] = p->fac64[c][same];
          p->fac[c][mu] = p->fac[c][same];
          p->fsplit[c][mu] = p->fsplit[c][same];
          p->fexp[c][mu] = p->fexp[c][same];
          std::memcpy(p->tmB[c][mu], p->tmB[c][same], kTensorMapBytes);
          continue;
        }
        const int n = (int)p->n[mu];
        std::vector<double2> A = p->user_mats ? p->userA[mu] : fd_direction_matrix(p, mu);
        CUDA_TRY(cudaMemcpyAsync(dA, A.data(), A.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
        if ((st = dev_alloc(p, (void**)&p->fac64[c][mu], (size_t)n * n * sizeof(double2)))) return st;
        CUDA_TRY(expm_device(dA, p->cval[c] * p->tau, n, p->fac64[c][mu], dW, norm1(A, n), s));
        if ((st = make_working(p, p->fac64[c][mu], (int64_t)n * n, &p->fac[c][mu], s))) return st;
        if (p->precision == CGL_BF16X3) {
          if ((st = dev_alloc(p, &p->fsplit[c][mu], mma_factor_bytes(n)))) return st;
          CUDA_TRY(launch_factor_split(p->fac64[c][mu], n, p->fsplit[c][mu], s));
          CUDA_TRY(make_factor_tmap(p->tmB[c][mu], p->fsplit[c][mu], n));
        }
        if (p->precision == CGL_F64_TC) {
          if ((st = dev_alloc(p, &p->fsplit[c][mu], oz_factor_bytes(n)))) return st;
          if ((st = dev_alloc(p, (void**)&p->fexp[c][mu], (size_t)mma_pad16(n) * sizeof(int)))) return st;
          CUDA_TRY(launch_oz_factor_slice(p->fac64[c][mu], n, p->fsplit[c][mu], p->fexp[c][mu], s));
          CUDA_TRY(make_factor_tmap(p->tmB[c][mu], p->fsplit[c][mu], n, 7, oz_rows_per_cta(mma_pad16(n))));
        }
        // the host copy of A must stay alive until the upload has completed
        CUDA_TRY(cudaStreamSynchronize(s));
      }
    }
    return CGL_OK;
  }
  // periodic: per-direction symbol vectors; the inverse FFT's 1/n_mu is
  // folded into each factor of the product form, 1/N into each term of
  // the sum form.
  for (int mu = 0; mu < p->d; ++mu) {
    const int n = (int)p->n[mu];
    const double L = p->hi[mu] - p->lo[mu];
    for (int c = 0; c < p->nfac; ++c) {
      if ((st = dev_alloc(p, (void**)&p->fac64[c][mu], n * sizeof(double2)))) return st;
      CUDA_TRY(periodic_symbol_device(p->fac64[c][mu], n, L, p->cval[c] * p->tau, p->a1, p->b1, p->a2 / p->d,
                                      mu == 0 ? p->adv[c] : 0.0, 1.0 / n, 0, s));
      if ((st = make_working(p, p->fac64[c][mu], n, &p->fac[c][mu], s))) return st;
    }
    if (p->scheme == CGL_RK4 || p->scheme == CGL_RK2) {
      // K symbols (sum form); the coupled system's u and v differ in the
      // advection term on direction 1
      for (int f = 0; f < p->nfield; ++f) {
        const double adv = (mu == 0) ? (f == 0 ? p->a0 : -p->a0) : 0.0;
        double2* k64 = nullptr;
        if ((st = dev_alloc(p, (void**)&k64, n * sizeof(double2)))) return st;
        CUDA_TRY(periodic_symbol_device(k64, n, L, 0.0, p->a1, p->b1, p->a2 / p->d, adv, 1.0 / (double)p->N, 1, s));
        if ((st = make_working(p, k64, n, f == 0 ? &p->ksym[mu] : &p->ksym2[mu], s))) return st;
      }
    }
    const size_t treal = p->precision == CGL_F64 ? sizeof(double) : sizeof(float);
    if ((st = dev_alloc(p, &p->twiddle[mu], 2 * 3 * (size_t)n * treal))) return st;
    if ((st = dev_alloc(p, (void**)&p->twform[mu], 2 * (size_t)n * sizeof(int)))) return st;
    CUDA_TRY(fma_twiddles_device(p->twiddle[mu], p->twform[mu], n, p->precision == CGL_F64, s));
    if ((n & (n - 1)) != 0) {  // mixed-radix passes take plain twiddles
      if ((st = dev_alloc(p, &p->twplain[mu], 2 * (size_t)n * p->elem))) return st;
      CUDA_TRY(plain_twiddles_device(p->twplain[mu], n, p->precision == CGL_F64, s));
    }
  }
  return CGL_OK;
}

void build_program(cgl_plan* p) {
  const double tau = p->tau;
  NlParams nl{p->a3, p->b3, p->a4, p->b4, p->cubic, tau};
  nl.a5 = p->a5;
  auto base = [&]() {
    Sweep s;
    s.op.nl = nl;
    return s;
  };
  p->sweeps.clear();
  if (p->coupled) {
    // coupled system (eq. coupled): every sweep carries both fields, u as
    // rhs 0 and v as rhs 1 (the second field of each buffer), with factors
    // 2 k (u) and 2 k + 1 (v); phi is the coupled RK4 flow
    auto pair = [&](Sweep& s, int in, int work, int out, int k) {
      s.nin = 2; s.in[0] = s.in[1] = in; s.in_f[0] = 0; s.in_f[1] = 1;
      s.nrhs = 2; s.fac[0] = 2 * k; s.fac[1] = 2 * k + 1;
      s.work[0] = s.work[1] = work; s.work_f[0] = 0; s.work_f[1] = 1;
      s.nout = 2; s.out[0] = s.out[1] = out; s.out_f[0] = 0; s.out_f[1] = 1;
    };
    if (p->scheme == CGL_STRANG) {  // eq. Strang
      Sweep s = base();
      pair(s, BUF_U, BUF_U, BUF_U, 0);
      s.op.pro = PRO_CFLOW; s.op.t0 = tau / 2;
      s.op.epi = EPI_CFLOW; s.op.te = tau / 2;
      p->sweeps.push_back(s);
    } else if (p->scheme == CGL_LAWSON4) {
      // eq. lawson4 with E = exp(tau K / 2) (factor pair k = 0), each sweep
      // carrying u and v: a = E W; p and w from b = E g(W) and a; q = E p;
      // W_{n+1} = E w + tau/6 g(q)
      Sweep s1 = base();
      pair(s1, BUF_U, BUF_W0, BUF_W0, 0);  // a -> W0
      Sweep s2 = base();
      pair(s2, BUF_U, BUF_W1, BUF_W1, 0);  // p -> W1
      s2.op.pro = PRO_CG;
      s2.op.epi = EPI_CLAW4P;
      s2.nextra = 2; s2.extra[0] = s2.extra[1] = BUF_W0; s2.extra_f[0] = 0; s2.extra_f[1] = 1;
      Sweep s3 = s2;  // w -> W2
      pair(s3, BUF_U, BUF_W2, BUF_W2, 0);
      s3.op.epi = EPI_CLAW4W;
      Sweep s4 = base();
      pair(s4, BUF_W1, BUF_W0, BUF_W0, 0);  // q = E p -> W0 (a is no longer read)
      Sweep s5 = base();
      pair(s5, BUF_W2, BUF_U, BUF_U, 0);  // E w + tau/6 g(q) -> W
      s5.op.epi = EPI_CLAW4B;
      s5.nextra = 2; s5.extra[0] = s5.extra[1] = BUF_W0; s5.extra_f[0] = 0; s5.extra_f[1] = 1;
      for (Sweep* sw : {&s1, &s2, &s3, &s4, &s5}) p->sweeps.push_back(*sw);
    } else if (p->scheme == CGL_RK4 || p->scheme == CGL_RK2) {
      // eq. RK4 / RK2 on W' = K W + g(W): each stage is a sweep per field
      // (K x_f with that field's symbol, FAC_K / FAC_K2) whose epilogue forms
      // k_f = K x_f + g_f(x_f; x_other) and the stage update (extras: x_f,
      // u_n, acc, x_other).  Stage arguments alternate between W0 and W1
      // (x_1 = W), so the v sweep still reads the old x_u; acc lives in W2;
      // each field's passes work in the next stage-argument slot.
      const int stages = p->scheme == CGL_RK4 ? 4 : 2;
      int xcur = BUF_U;
      for (int st = 1; st <= stages; ++st) {
        const int xnext = (xcur == BUF_W0) ? BUF_W1 : BUF_W0;
        for (int f = 0; f < 2; ++f) {
          Sweep s = base();
          s.in[0] = xcur; s.in_f[0] = f;
          s.fac[0] = f == 0 ? FAC_K : FAC_K2;
          s.work[0] = xnext; s.work_f[0] = f;
          s.op.epi = EPI_RK; s.op.rk_scheme = stages; s.op.rk_stage = st; s.op.rk_coupled = 1;
          s.nextra = 4;
          s.extra[0] = xcur; s.extra_f[0] = f;
          s.extra[1] = BUF_U; s.extra_f[1] = f;
          s.extra[2] = BUF_W2; s.extra_f[2] = f;
          s.extra[3] = xcur; s.extra_f[3] = 1 - f;
          if (st < stages) {
            s.nout = 2; s.out[0] = xnext; s.out_f[0] = f; s.out[1] = BUF_W2; s.out_f[1] = f;
          } else {
            s.nout = 1; s.out[0] = BUF_U; s.out_f[0] = f;
          }
          p->sweeps.push_back(s);
        }
        xcur = xnext;
      }
    } else if (p->scheme == CGL_LAWSON2) {
      // eq. lawson2b with E = exp(tau K): v = E(W + tau g(W)) -> W0;
      // W_{n+1} = E(W + tau/2 g(W)) + tau/2 g(v)
      Sweep s1 = base();
      pair(s1, BUF_U, BUF_W0, BUF_W0, 0);
      s1.op.pro = PRO_CLAW2; s1.op.t0 = tau;
      Sweep s2 = base();
      pair(s2, BUF_U, BUF_U, BUF_U, 0);
      s2.op.pro = PRO_CLAW2; s2.op.t0 = tau / 2;
      s2.op.epi = EPI_CLAW2;
      s2.nextra = 2; s2.extra[0] = s2.extra[1] = BUF_W0; s2.extra_f[0] = 0; s2.extra_f[1] = 1;
      p->sweeps.push_back(s1);
      p->sweeps.push_back(s2);
    } else {  // eq. Richardson: c = 1 (k = 0), c = 1/2 (k = 1)
      Sweep s1 = base();  // u_{n2} = phi_{tau/2}(E_1 phi_{tau/2}(W)) -> W0
      pair(s1, BUF_U, BUF_W0, BUF_W0, 0);
      s1.op.pro = PRO_CFLOW; s1.op.t0 = tau / 2;
      s1.op.epi = EPI_CFLOW; s1.op.te = tau / 2;
      Sweep s2 = base();  // v = phi_{tau/2}(E_{1/2} phi_{tau/4}(W)) -> W1
      pair(s2, BUF_U, BUF_W1, BUF_W1, 1);
      s2.op.pro = PRO_CFLOW; s2.op.t0 = tau / 4;
      s2.op.epi = EPI_CFLOW; s2.op.te = tau / 2;
      Sweep s3 = base();  // W = 4/3 phi_{tau/4}(E_{1/2} v) - 1/3 u_{n2}
      pair(s3, BUF_W1, BUF_U, BUF_U, 1);
      s3.op.pro = PRO_NONE;
      s3.op.epi = EPI_CSPLIT4; s3.op.te = tau / 4;
      s3.nextra = 2; s3.extra[0] = s3.extra[1] = BUF_W0; s3.extra_f[0] = 0; s3.extra_f[1] = 1;
      p->sweeps.push_back(s1);
      p->sweeps.push_back(s2);
      p->sweeps.push_back(s3);
    }
    for (Sweep& s : p->sweeps) single_copies(s.op);
    return;
  }
  switch (p->scheme) {
    case CGL_STRANG: {  // eq. Strang
      Sweep s = base();
      s.op.pro = PRO_FLOW; s.op.t0 = tau / 2;
      s.op.epi = EPI_FLOW; s.op.te = tau / 2;
      s.fac[0] = 0;
      p->sweeps.push_back(s);
      break;
    }
    case CGL_STRANG3T: {  // strang_3t (Sec. 4.3): P*_{tau/2} e^{tau K} P_{tau/2}
      Sweep s = base();
      s.op.pro = PRO_CQ; s.op.t0 = tau / 2;
      s.op.epi = EPI_QC; s.op.te = tau / 2;
      s.fac[0] = 0;
      p->sweeps.push_back(s);
      break;
    }
    case CGL_SPLIT4_3T: {  // split4_3t (Sec. 4.3); factor 0: c = 1, factor 1: c = 1/2
      // sweep 1: [E_1 P_{tau/2} u, E_{1/2} P_{tau/4} u] -> (u_{n2} = P*_{tau/2}(.),
      //          v = P_{tau/4} P*_{tau/4}(.), quintic quarter flows merged);
      // sweep 2: E_{1/2} v -> 4/3 P*_{tau/4}(.) - 1/3 u_{n2}
      Sweep s1 = base();
      s1.op.pro = PRO_CQ2; s1.op.t0 = tau / 2; s1.op.t1 = tau / 4;
      s1.nrhs = 2; s1.fac[0] = 0; s1.fac[1] = 1; s1.work[0] = BUF_W0; s1.work[1] = BUF_W1;
      s1.op.epi = EPI_QC2; s1.op.te = tau / 2;
      s1.nout = 2; s1.out[0] = BUF_W0; s1.out[1] = BUF_W1;
      Sweep s2 = base();
      s2.in[0] = BUF_W1; s2.fac[0] = 1; s2.work[0] = BUF_W1;
      s2.op.epi = EPI_SPLIT4_3T; s2.op.te = tau / 4;
      s2.nextra = 1; s2.extra[0] = BUF_W0;
      s2.out[0] = BUF_U;
      p->sweeps.push_back(s1);
      p->sweeps.push_back(s2);
      break;
    }
    case CGL_SPLIT4: {  // eq. Richardson; factor 0: c = 1, factor 1: c = 1/2
      Sweep s1 = base();
      s1.op.pro = PRO_FLOW2; s1.op.t0 = tau / 2; s1.op.t1 = tau / 4;
      s1.nrhs = 2; s1.fac[0] = 0; s1.fac[1] = 1; s1.work[0] = BUF_W0; s1.work[1] = BUF_W1;
      s1.op.epi = EPI_FLOW2; s1.op.te = tau / 2;
      s1.nout = 2; s1.out[0] = BUF_W0; s1.out[1] = BUF_W1;  // u_{n2}, v
      Sweep s2 = base();
      s2.in[0] = BUF_W1; s2.fac[0] = 1; s2.work[0] = BUF_W1;
      s2.op.epi = EPI_SPLIT4; s2.op.te = tau / 4;
      s2.nextra = 1; s2.extra[0] = BUF_W0;
      s2.out[0] = BUF_U;
      p->sweeps.push_back(s1);
      p->sweeps.push_back(s2);
      break;
    }
    case CGL_LAWSON4: {  // eq. lawson4 with E = exp(tau K/2), factor 0: c = 1/2
      Sweep s1 = base();
      s1.op.pro = PRO_LAW4;
      s1.nrhs = 2; s1.work[0] = BUF_W0; s1.work[1] = BUF_W1;
      s1.op.epi = EPI_LAW4A;
      s1.nout = 2; s1.out[0] = BUF_W0; s1.out[1] = BUF_W1;  // p, w
      Sweep s2 = base();
      s2.nin = 2; s2.in[0] = BUF_W0; s2.in[1] = BUF_W1;
      s2.nrhs = 2; s2.work[0] = BUF_W0; s2.work[1] = BUF_W1;
      s2.op.epi = EPI_LAW4B;
      s2.out[0] = BUF_U;
      p->sweeps.push_back(s1);
      p->sweeps.push_back(s2);
      break;
    }
    case CGL_LAWSON2: {  // eq. lawson2b, factor 0: c = 1
      Sweep s = base();
      s.op.pro = PRO_LAW2;
      s.nrhs = 2; s.work[0] = BUF_W0; s.work[1] = BUF_W1;
      s.op.epi = EPI_LAW2;
      s.out[0] = BUF_U;
      p->sweeps.push_back(s);
      break;
    }
    case CGL_RK4:
    case CGL_RK2: {  // eq. RK4 / eq. RK2: stage s computes K x_s with x_1 = u
      const int stages = p->scheme == CGL_RK4 ? 4 : 2;
      if (!p->periodic) {
        // finite differences: one stencil launch per stage (eq. kronsumv);
        // the stage arguments alternate between W1 and W0 because a stencil
        // reads neighbours and cannot write over its input
        int xb = BUF_U;
        for (int st = 1; st <= stages; ++st) {
          Sweep s = base();
          s.stencil = true;
          s.in[0] = xb;
          s.op.epi = EPI_RK; s.op.rk_scheme = stages; s.op.rk_stage = st;
          s.nextra = 3; s.extra[0] = xb; s.extra[1] = BUF_U; s.extra[2] = BUF_W2;
          if (st < stages) {
            const int nb = (xb == BUF_W1) ? BUF_W0 : BUF_W1;
            s.nout = 2; s.out[0] = nb; s.out[1] = BUF_W2;
            xb = nb;
          } else {
            s.nout = 1; s.out[0] = BUF_U;
          }
          p->sweeps.push_back(s);
        }
        break;
      }
      for (int st = 1; st <= stages; ++st) {
        Sweep s = base();
        s.in[0] = (st == 1) ? BUF_U : BUF_W1;  // x_s
        s.fac[0] = FAC_K;
        s.work[0] = BUF_W0;
        s.op.epi = EPI_RK; s.op.rk_scheme = stages; s.op.rk_stage = st;
        s.nextra = 3; s.extra[0] = s.in[0]; s.extra[1] = BUF_U; s.extra[2] = BUF_W2;
        if (st < stages) { s.nout = 2; s.out[0] = BUF_W1; s.out[1] = BUF_W2; }
        else { s.nout = 1; s.out[0] = BUF_U; }
        p->sweeps.push_back(s);
      }
      break;
    }
  }
  for (Sweep& s : p->sweeps) single_copies(s.op);
}

bool finite_all(std::initializer_list<double> v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

// Kernel attributes are set once per process and device, before any capture.
cudaError_t prepare_kernels(int dev) {
  static bool done[64] = {false};
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  cudaError_t e;
  if ((e = prepare_fft_pass<double>()) != cudaSuccess) return e;
  if ((e = prepare_fft_pass<float>()) != cudaSuccess) return e;
  if ((e = prepare_mode_pass<double>()) != cudaSuccess) return e;
  if ((e = prepare_mode_pass<float>()) != cudaSuccess) return e;
  if ((e = prepare_mma_pass()) != cudaSuccess) return e;
  if ((e = prepare_oz_pass()) != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) done[dev] = true;
  return cudaSuccess;
}

int ensure_graph(cgl_plan* p, void* u) {
  if (p->exec && p->graph_u == u) return CGL_OK;
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
  int st = enqueue_step(p, u, p->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
  if (st != CGL_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&p->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    p->exec = nullptr;
    return fail(CGL_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  p->graph_u = u;
  return CGL_OK;
}

void free_plan(cgl_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  for (void* a : p->allocations) cudaFree(a);
  delete p;
}

}  // namespace cgl

extern "C" {

const char* cgl_strerror(int status) {
  switch (status) {
    case CGL_OK: return "ok";
    case CGL_EINVAL: return "invalid argument";
    case CGL_ENOMEM: return "device allocation failed";
    case CGL_ECUDA: return "CUDA runtime error";
    case CGL_EUNSUPPORTED: return "unsupported configuration";
    case CGL_ETIMEOUT: return "device-side wait timed out";
    case CGL_ENONFINITE: return "non-finite value produced";
    default: return "unknown status";
  }
}

const char* cgl_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace cgl {

int plan_create_impl(cgl_plan** out, int d, const int64_t* n, const int* bc, const double* lo, const double* hi,
                     double a1, double b1, double a2, double a3, double b3, double a4, double b4, double tau,
                     int scheme, int precision, void* stream, bool minimal, const double* const* A,
                     const double* coupled) {
  g_last_error.clear();
  if (!out) return fail(CGL_EINVAL, "out is NULL");
  *out = nullptr;
  if (d < 1 || d > 3) return fail(CGL_EINVAL, "d must be 1, 2 or 3");
  if (!n || !bc || !lo || !hi) return fail(CGL_EINVAL, "n, bc, lo, hi must be non-NULL");
  if (!finite_all({a1, b1, a2, a3, b3, a4, b4, tau})) return fail(CGL_EINVAL, "parameters must be finite");
  if (!(a1 > 0)) return fail(CGL_EINVAL, "alpha1 must be positive");
  if (!(tau > 0)) return fail(CGL_EINVAL, "tau must be positive");
  if (scheme < CGL_STRANG || scheme > CGL_SPLIT4_3T) return fail(CGL_EINVAL, "unknown scheme");
  if (precision != CGL_F64 && precision != CGL_F32 && precision != CGL_BF16X3 && precision != CGL_F64_TC)
    return fail(CGL_EINVAL, "unknown precision");
  int nper = 0;
  for (int m = 0; m < d; ++m) {
    if (bc[m] < CGL_BC_DIRICHLET || bc[m] > CGL_BC_PERIODIC) return fail(CGL_EINVAL, "unknown boundary condition");
    if (n[m] < 2) return fail(CGL_EINVAL, "n_mu must be >= 2");
    if (!std::isfinite(lo[m]) || !std::isfinite(hi[m]) || !(hi[m] > lo[m]))
      return fail(CGL_EINVAL, "domain must satisfy lo < hi (finite)");
    nper += bc[m] == CGL_BC_PERIODIC;
  }
  if (nper != 0 && nper != d)
    return fail(CGL_EUNSUPPORTED, "mixing periodic and finite-difference directions is not supported");
  if (coupled) {
    if (!finite_all({coupled[0], coupled[1]})) return fail(CGL_EINVAL, "parameters must be finite");
    if (nper != d) return fail(CGL_EUNSUPPORTED, "the coupled system is periodic (Fourier) only");
    if (scheme == CGL_STRANG3T || scheme == CGL_SPLIT4_3T)
      return fail(CGL_EUNSUPPORTED, "the coupled system has no three-term splittings");
    if (precision == CGL_BF16X3 || precision == CGL_F64_TC)
      return fail(CGL_EUNSUPPORTED, "the coupled system runs in CGL_F64 or CGL_F32");
  }
  const bool periodic = nper == d;
  for (int m = 0; m < d; ++m) {
    if (periodic && !fft_size_ok(n[m]))
      return fail(CGL_EUNSUPPORTED, "periodic sizes must be 2^a 3^b 5^c 7^d <= 2048");
    if (!periodic && n[m] > 1024) return fail(CGL_EUNSUPPORTED, "finite-difference sizes must be <= 1024");
  }
  if (A) {
    if (periodic) return fail(CGL_EINVAL, "caller-supplied direction matrices need non-periodic directions");
    if (scheme == CGL_RK4 || scheme == CGL_RK2)
      return fail(CGL_EUNSUPPORTED, "caller-supplied direction matrices support the exponential schemes only");
    for (int m = 0; m < d; ++m) {
      if (!A[m]) return fail(CGL_EINVAL, "every direction matrix must be non-NULL");
      for (int64_t k = 0; k < 2 * n[m] * n[m]; ++k)
        if (!std::isfinite(A[m][k])) return fail(CGL_EINVAL, "direction matrices must be finite");
    }
  }
  if (precision == CGL_BF16X3 || precision == CGL_F64_TC) {
    if (periodic)
      return fail(CGL_EUNSUPPORTED, "the tensor-core precisions apply to the finite-difference mode products only");
    for (int m = 0; m < d; ++m)
      if (n[m] > 256) return fail(CGL_EUNSUPPORTED, "the tensor-core precisions need every n_mu <= 256");
  }

  cgl_plan* p = new cgl_plan();
  cudaGetDevice(&p->dev);
  p->d = d;
  if (A) {
    p->user_mats = true;
    for (int m = 0; m < d; ++m) {
      p->userA[m].resize((size_t)n[m] * n[m]);
      for (size_t k = 0; k < p->userA[m].size(); ++k) p->userA[m][k] = make_double2(A[m][2 * k], A[m][2 * k + 1]);
    }
  }
  p->N = 1;
  for (int m = 0; m < d; ++m) {
    p->n[m] = n[m];
    p->bc[m] = bc[m];
    p->lo[m] = lo[m];
    p->hi[m] = hi[m];
    p->N *= n[m];
  }
  p->a1 = a1; p->b1 = b1; p->a2 = a2; p->a3 = a3; p->b3 = b3; p->a4 = a4; p->b4 = b4;
  p->tau = tau;
  p->scheme = scheme;
  p->precision = precision;
  p->periodic = periodic;
  p->cubic = (a4 == 0.0 && b4 == 0.0);
  // F64 and F64_TC: complex128; F32 and BF16x3: complex64
  p->elem = (precision == CGL_F64 || precision == CGL_F64_TC) ? sizeof(double2) : sizeof(float2);
  switch (scheme) {
    case CGL_STRANG:
    case CGL_STRANG3T:
    case CGL_LAWSON2: p->nfac = 1; p->cval[0] = 1.0; break;
    case CGL_SPLIT4:
    case CGL_SPLIT4_3T: p->nfac = 2; p->cval[0] = 1.0; p->cval[1] = 0.5; break;
    case CGL_LAWSON4: p->nfac = 1; p->cval[0] = 0.5; break;
    default: p->nfac = 0;
  }
  switch (scheme) {
    case CGL_STRANG:
    case CGL_STRANG3T: p->nwork = 0; break;
    case CGL_RK4:
    case CGL_RK2: p->nwork = 3; break;
    default: p->nwork = 2;
  }
  if (coupled) {
    // one factor per (c, field): slot 2 k + f has c = cval[k] of the single
    // field scheme and advection +a0 (u, f = 0) or -a0 (v, f = 1)
    p->coupled = true;
    p->nfield = 2;
    p->a0 = coupled[0];
    p->a5 = coupled[1];
    const int nc = p->nfac;
    const double cv[2] = {p->cval[0], p->cval[1]};
    for (int k = 0; k < nc; ++k)
      for (int f = 0; f < 2; ++f) {
        p->cval[2 * k + f] = cv[k];
        p->adv[2 * k + f] = f == 0 ? p->a0 : -p->a0;
      }
    p->nfac = 2 * nc;
    if (scheme == CGL_LAWSON4) p->nwork = 3;  // a (then q), p, w
  }
  cudaStream_t s = (cudaStream_t)stream;
  int st = CGL_OK;
  cudaError_t e = prepare_kernels(p->dev);
  if (e != cudaSuccess) {
    delete p;
    return fail(CGL_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  }
  if (!minimal) {
    e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = fail(CGL_ECUDA, std::string("stream create: ") + cudaGetErrorString(e));
  }
  if (!st) st = dev_alloc(p, (void**)&p->status, sizeof(int));
  if (!st && cudaMemsetAsync(p->status, 0, sizeof(int), s) != cudaSuccess) st = fail(CGL_ECUDA, "memset status");
  for (int w = 0; !st && !minimal && w < p->nwork; ++w) st = dev_alloc(p, &p->work[w], p->nfield * p->N * p->elem);
  if (!st && precision == CGL_BF16X3) {
    // planes with the first direction padded to a multiple of 64, zeroed once:
    // the padding is never written afterwards (mode passes store rows i < n)
    p->pitch = mma_pitch(p->n[0]);
    p->Npad = p->N / p->n[0] * p->pitch;
    const int nr = scheme == CGL_STRANG ? 1 : 2;
    for (int r = 0; !st && r < nr; ++r) {
      st = dev_alloc(p, &p->splits[r], 12 * (size_t)p->Npad);
      if (!st && d > 1) st = dev_alloc(p, &p->splits_alt[r], 12 * (size_t)p->Npad);
      if (!st) st = dev_alloc(p, &p->planes[r], 8 * (size_t)p->Npad);
      void* bufs[3] = {p->splits[r], p->splits_alt[r], p->planes[r]};
      const size_t sizes[3] = {12 * (size_t)p->Npad, 12 * (size_t)p->Npad, 8 * (size_t)p->Npad};
      for (int k = 0; !st && k < 3; ++k)
        if (bufs[k] && cudaMemsetAsync(bufs[k], 0, sizes[k], s) != cudaSuccess) st = fail(CGL_ECUDA, "memset planes");
      for (int mu = 0; !st && mu < d; ++mu) {
        e = make_state_tmap(p->tmA[mu][r], (mu & 1) ? p->splits_alt[r] : p->splits[r], (int)p->n[mu],
                            mma_axis_P(p, mu), mma_axis_Q(p, mu), p->Npad, p->pitch);
        if (e != cudaSuccess) st = fail(CGL_ECUDA, std::string("tensor map: ") + cudaGetErrorString(e));
      }
    }
  }
  if (!st && precision == CGL_F64_TC && !minimal) {
    // FP64 planes and digit planes with the first direction padded to a
    // multiple of 64, zeroed once (the padding stays zero: the prologue
    // writes grid points only, slicing turns zero planes into zero digits and
    // the passes store rows i < n); per-fiber exponents for the largest
    // fiber count over the modes
    p->pitch = mma_pitch(p->n[0]);
    p->Npad = p->N / p->n[0] * p->pitch;
    int64_t fibers = 0;
    for (int mu = 0; mu < d; ++mu) fibers = std::max<int64_t>(fibers, p->Npad / p->n[mu]);
    const int nr = (scheme == CGL_STRANG || scheme == CGL_STRANG3T) ? 1 : 2;
    for (int r = 0; !st && r < nr; ++r) {
      st = dev_alloc(p, &p->oz_z[r], 16 * (size_t)p->Npad);
      if (!st) st = dev_alloc(p, &p->oz_dig[r], 28 * (size_t)p->Npad);
      if (!st) st = dev_alloc(p, (void**)&p->oz_exp[r], (size_t)fibers * sizeof(int));
      if (!st && (cudaMemsetAsync(p->oz_z[r], 0, 16 * (size_t)p->Npad, s) != cudaSuccess ||
                  cudaMemsetAsync(p->oz_dig[r], 0, 28 * (size_t)p->Npad, s) != cudaSuccess))
        st = fail(CGL_ECUDA, "memset planes");
      for (int mu = 0; !st && mu < d; ++mu) {
        e = make_state_tmap(p->oz_tmA[mu][r], p->oz_dig[r], (int)p->n[mu], mma_axis_P(p, mu), mma_axis_Q(p, mu),
                            p->Npad, p->pitch, 7);
        if (e != cudaSuccess) st = fail(CGL_ECUDA, std::string("tensor map: ") + cudaGetErrorString(e));
      }
    }
  }
  if (!st) st = build_factors(p, s);
  if (!st) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(CGL_ECUDA, std::string("plan set-up: ") + cudaGetErrorString(e));
  }
  if (st) {
    free_plan(p);
    return st;
  }
  build_program(p);
  *out = p;
  return CGL_OK;
}

}  // namespace cgl

extern "C" {

int cgl_inject_alloc_failure(long long after) {
  if (after < -1) return fail(CGL_EINVAL, "after must be >= -1");
  g_alloc_countdown.store(after);
  return CGL_OK;
}

int cgl_plan_create(cgl_plan** out, int d, const int64_t* n, const int* bc, const double* lo, const double* hi,
                    double a1, double b1, double a2, double a3, double b3, double a4, double b4, double tau,
                    int scheme, int precision, void* stream) {
  return plan_create_impl(out, d, n, bc, lo, hi, a1, b1, a2, a3, b3, a4, b4, tau, scheme, precision, stream, false);
}

int cgl_plan_create_ex(cgl_plan** out, int d, const int64_t* n, const double* const* A, double a3, double b3,
                       double a4, double b4, double tau, int scheme, int precision, void* stream) {
  if (!out) return fail(CGL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!A) return fail(CGL_EINVAL, "A is NULL");
  if (d < 1 || d > 3) return fail(CGL_EINVAL, "d must be 1, 2 or 3");
  // the boundary labels, domain and a1, b1, a2 are not used with caller-supplied matrices
  const int bc[3] = {CGL_BC_DIRICHLET, CGL_BC_DIRICHLET, CGL_BC_DIRICHLET};
  const double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  return plan_create_impl(out, d, n, bc, lo, hi, 1.0, 0.0, 0.0, a3, b3, a4, b4, tau, scheme, precision, stream, false,
                          A);
}

int cgl_plan_create_coupled(cgl_plan** out, int d, const int64_t* n, const double* lo, const double* hi,
                            double a0, double a1, double b1, double a2, double a3, double b3, double a4, double b4,
                            double a5, double tau, int scheme, int precision, void* stream) {
  if (d < 1 || d > 3) {
    if (out) *out = nullptr;
    return fail(CGL_EINVAL, "d must be 1, 2 or 3");
  }
  const int bc[3] = {CGL_BC_PERIODIC, CGL_BC_PERIODIC, CGL_BC_PERIODIC};
  const double cpl[2] = {a0, a5};
  return plan_create_impl(out, d, n, bc, lo, hi, a1, b1, a2, a3, b3, a4, b4, tau, scheme, precision, stream, false,
                          nullptr, cpl);
}

int cgl_fd4_matrix(int n, double lo, double hi, int right_bc, double* out) {
  if (!out) return fail(CGL_EINVAL, "out is NULL");
  if (n < 6) return fail(CGL_EINVAL, "n must be >= 6");
  if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo)) return fail(CGL_EINVAL, "need lo < hi (finite)");
  if (right_bc != CGL_BC_DIRICHLET && right_bc != CGL_BC_NEUMANN)
    return fail(CGL_EINVAL, "right_bc must be CGL_BC_DIRICHLET or CGL_BC_NEUMANN");
  const double h = right_bc == CGL_BC_DIRICHLET ? (hi - lo) / (n + 1) : (hi - lo) / n;
  const double s = 1.0 / (12.0 * h * h);
  auto at = [&](int i, int j) -> double& { return out[(size_t)i + (size_t)j * n]; };
  for (size_t k = 0; k < (size_t)n * n; ++k) out[k] = 0.0;
  const double centred[5] = {-1, 16, -30, 16, -1};
  for (int i = 1; i < n - 1; ++i)
    for (int o = -2; o <= 2; ++o)
      if (i + o >= 0 && i + o < n) at(i, i + o) = centred[o + 2] * s;
  // first internal node: one-sided fourth-order row (the zero boundary value drops out)
  const double first[5] = {-15, -4, 14, -6, 1};
  for (int j = 0; j < 5; ++j) at(0, j) = first[j] * s;
  if (right_bc == CGL_BC_DIRICHLET) {
    for (int j = 0; j < n; ++j) at(n - 1, j) = 0.0;
    for (int j = 0; j < 5; ++j) at(n - 1, n - 1 - j) = first[j] * s;
  } else {
    // last two nodes: Neumann closure of the semi-internal grid
    const double penult[6] = {1, -6, 14, -4, -15, 10};
    const double last[5] = {1, -8.0 / 3.0, -6, 56, -145.0 / 3.0};
    for (int j = 0; j < n; ++j) at(n - 2, j) = at(n - 1, j) = 0.0;
    for (int j = 0; j < 6; ++j) at(n - 2, n - 6 + j) = penult[j] * s;
    for (int j = 0; j < 5; ++j) at(n - 1, n - 5 + j) = last[j] * s;
  }
  return CGL_OK;
}

int cgl_plan_destroy(cgl_plan* p) {
  if (!p) return CGL_OK;
  cudaSetDevice(p->dev);
  free_plan(p);
  return CGL_OK;
}

int cgl_step(cgl_plan* p, void* u, int64_t nsteps, void* stream) {
  if (!p || !u) return fail(CGL_EINVAL, "plan and u must be non-NULL");
  if (nsteps < 0) return fail(CGL_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return CGL_OK;
  CUDA_TRY(cudaSetDevice(p->dev));
  int st = ensure_graph(p, u);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t k = 0; k < nsteps; ++k) CUDA_TRY(cudaGraphLaunch(p->exec, s));
  return CGL_OK;
}

int cgl_step_host(cgl_plan* p, void* u_host, int64_t nsteps, void* stream) {
  if (!p || !u_host) return fail(CGL_EINVAL, "plan and u_host must be non-NULL");
  if (nsteps < 0) return fail(CGL_EINVAL, "nsteps must be >= 0");
  CUDA_TRY(cudaSetDevice(p->dev));
  if (!p->host_stage) {
    int st = dev_alloc(p, &p->host_stage, p->nfield * p->N * p->elem);
    if (st) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = p->nfield * p->N * p->elem;
  CUDA_TRY(cudaMemcpyAsync(p->host_stage, u_host, bytes, cudaMemcpyHostToDevice, s));
  int st = cgl_step(p, p->host_stage, nsteps, stream);
  if (st) return st;
  CUDA_TRY(cudaMemcpyAsync(u_host, p->host_stage, bytes, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return CGL_OK;
}

int cgl_linear_flow(cgl_plan* p, double c, void* u, void* stream) {
  if (!p || !u) return fail(CGL_EINVAL, "plan and u must be non-NULL");
  int idx = -1;
  for (int k = p->nfac - 1; k >= 0; --k)
    if (p->cval[k] == c) idx = k;  // the first factor with this c (coupled: u's, v's follows)
  if (idx < 0) return fail(CGL_EINVAL, "c is not one of the plan's factor values");
  CUDA_TRY(cudaSetDevice(p->dev));
  Sweep s;
  s.op.nl = NlParams{p->a3, p->b3, p->a4, p->b4, p->cubic, p->tau};
  single_copies(s.op);
  s.fac[0] = idx;
  if (p->coupled) {  // both fields, each with its own symbol
    s.nin = s.nrhs = s.nout = 2;
    s.fac[1] = idx + 1;
    s.in_f[1] = s.work_f[1] = s.out_f[1] = 1;
  }
  return enqueue_sweep(p, s, u, (cudaStream_t)stream);
}

int cgl_plan_factor(cgl_plan* p, double c, int mu, double* host_out) {
  if (!p || !host_out) return fail(CGL_EINVAL, "plan and host_out must be non-NULL");
  if (mu < 0 || mu >= p->d) return fail(CGL_EINVAL, "mu out of range");
  int idx = -1;
  for (int k = p->nfac - 1; k >= 0; --k)
    if (p->cval[k] == c) idx = k;
  if (idx < 0) return fail(CGL_EINVAL, "c is not one of the plan's factor values");
  CUDA_TRY(cudaSetDevice(p->dev));
  const size_t count = p->periodic ? (size_t)p->n[mu] : (size_t)p->n[mu] * p->n[mu];
  CUDA_TRY(cudaMemcpy(host_out, p->fac64[idx][mu], count * sizeof(double2), cudaMemcpyDeviceToHost));
  return CGL_OK;
}

int cgl_plan_info(const cgl_plan* p, size_t* field_bytes, size_t* workspace_bytes, int* launches) {
  if (!p) return fail(CGL_EINVAL, "plan is NULL");
  if (field_bytes) *field_bytes = p->nfield * p->N * p->elem;
  if (workspace_bytes) *workspace_bytes = (size_t)p->nwork * p->nfield * p->N * p->elem;
  if (launches) *launches = launches_per_step(p);
  return CGL_OK;
}

int cgl_last_device_status(cgl_plan* p, void* stream) {
  if (!p) return fail(CGL_EINVAL, "plan is NULL");
  CUDA_TRY(cudaSetDevice(p->dev));
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h & 2) return fail(CGL_ETIMEOUT, "a device-side wait timed out");
  return (h & 1) ? CGL_ENONFINITE : CGL_OK;
}

int cgl_profile_step(cgl_plan* p, void* u, int64_t nsteps, void* stream, cgl_kernel_time* out, int max_kernels,
                     int* count) {
  if (!p || !u || !count || (max_kernels > 0 && !out)) return fail(CGL_EINVAL, "NULL argument");
  CUDA_TRY(cudaSetDevice(p->dev));
  cudaStream_t s = (cudaStream_t)stream;
  std::map<std::string, KernelStat> stats;
  p->prof = true;
  p->stats = &stats;
  int st = CGL_OK;
  for (int64_t k = 0; k < nsteps && st == CGL_OK; ++k) st = enqueue_step(p, u, s);
  p->prof = false;
  p->stats = nullptr;
  if (st) return st;
  CUDA_TRY(cudaStreamSynchronize(s));
  int c = 0;
  for (auto& kv : stats) {
    if (c >= max_kernels) break;
    std::memset(out[c].name, 0, sizeof(out[c].name));
    std::strncpy(out[c].name, kv.first.c_str(), sizeof(out[c].name) - 1);
    out[c].launches = kv.second.launches;
    out[c].total_ms = kv.second.ms;
    out[c].flops = kv.second.flops;
    out[c].bytes = kv.second.bytes;
    ++c;
  }
  *count = c;
  return CGL_OK;
}

int cgl_rel_error(const void* x, const void* y, int64_t count, int precision, double* out, void* stream) {
  if (!x || !y || !out) return fail(CGL_EINVAL, "NULL argument");
  if (count <= 0) return fail(CGL_EINVAL, "count must be positive");
  if (precision == CGL_BF16X3) precision = CGL_F32;  // complex64 state
  if (precision == CGL_F64_TC) precision = CGL_F64;   // complex128 state
  if (precision != CGL_F64 && precision != CGL_F32) return fail(CGL_EINVAL, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = rel_error_blocks(count);
  double* scratch = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&scratch, (5 * (size_t)nb + 3) * sizeof(double), s));
  cudaError_t e = rel_error_device(x, y, count, precision, scratch, nb, out, s);
  cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("rel_error: ") + cudaGetErrorString(e));
  CUDA_TRY(cudaStreamSynchronize(s));
  return CGL_OK;
}

}  // extern "C"
