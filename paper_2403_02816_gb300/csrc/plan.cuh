// Internal plan layout shared by the libcgl host translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "cgl_internal.cuh"

namespace cgl {

// Records `msg` as the calling thread's last error and returns `status`.
int fail(int status, const std::string& msg);

// Fault injection (cgl_inject_alloc_failure): true when the library's
// device allocation about to be made is the one set to fail.
bool injected_alloc_failure();

enum { BUF_U = 0, BUF_W0 = 1, BUF_W1 = 2, BUF_W2 = 3, NBUF = 4 };
constexpr int FAC_K = -1;   // the Runge-Kutta sweeps apply K, not an exponential
constexpr int FAC_K2 = -2;  // ... the coupled system's v field (advection -a0)

struct Sweep {
  int nin = 1, in[2] = {BUF_U, BUF_U};
  int nrhs = 1, fac[2] = {0, 0}, work[2] = {BUF_U, BUF_U};
  int nextra = 0, extra[kMaxExtra] = {BUF_U, BUF_U, BUF_U, BUF_U};
  int nout = 1, out[2] = {BUF_U, BUF_U};
  OpArgs op{};
  bool stencil = false;  // FD Runge-Kutta stage: K x as a stencil + epilogue, one launch
  // field of each slot within its buffer (coupled system: 0 = u, 1 = v, N
  // values further)
  int in_f[2] = {0, 0}, work_f[2] = {0, 0}, extra_f[kMaxExtra] = {0, 0, 0, 0}, out_f[2] = {0, 0};
};

struct KernelStat {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};

}  // namespace cgl

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return cgl::fail(_e == cudaErrorMemoryAllocation ? CGL_ENOMEM : CGL_ECUDA,         \
                       std::string(#expr) + ": " + cudaGetErrorString(_e));              \
  } while (0)

struct cgl_plan {
  int dev = 0;
  int d = 0;
  int64_t n[3] = {1, 1, 1};
  int bc[3] = {0, 0, 0};
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  double a1 = 0, b1 = 0, a2 = 0, a3 = 0, b3 = 0, a4 = 0, b4 = 0, tau = 0;
  int scheme = 0, precision = 0, periodic = 0, cubic = 0;
  // coupled two-field system (eq. coupled): advection a0, cross-coupling a5;
  // the state is u followed by v (nfield = 2 fields of N values)
  bool coupled = false;
  int nfield = 1;
  double a0 = 0, a5 = 0;
  bool user_mats = false;            // direction matrices supplied by the caller
  std::vector<double2> userA[3];     // their host copies (n_mu x n_mu, column-major)
  int64_t N = 0;
  size_t elem = 0;

  int nfac = 0;
  double cval[4] = {0, 0, 0, 0};
  double adv[4] = {0, 0, 0, 0};         // advection speed of each factor's field (periodic direction 1)
  void* fac[4][3] = {{nullptr}};        // working-precision factors / symbol vectors
  double2* fac64[4][3] = {{nullptr}};   // FP64 masters
  void* ksym[3] = {nullptr};            // K symbol vectors (periodic Runge-Kutta)
  void* ksym2[3] = {nullptr};           // the coupled system's v field
  void* twiddle[3] = {nullptr};         // FFT twiddle tables per axis: [fwd, inv][n][tau, m_re, m_im]
  int* twform[3] = {nullptr};           // [fwd, inv][n] twiddle form (0: m = cos, 1: m = sin)
  void* twplain[3] = {nullptr};         // mixed-radix axes: [fwd, inv][n] plain twiddles (T2)
  std::vector<void*> allocations;

  int nwork = 0;
  void* work[3] = {nullptr, nullptr, nullptr};
  int* status = nullptr;
  void* host_stage = nullptr;  // device field for cgl_step_host

  std::vector<cgl::Sweep> sweeps;

  // BF16x3 tensor-core path: per-rhs BF16x3 state planes and FP32 output
  // planes, per-(factor, mode) BF16x3 factor splits, and their TMA maps.
  void* splits[2] = {nullptr, nullptr};
  void* splits_alt[2] = {nullptr, nullptr};  // second set: mode passes alternate, none writes over its input
  void* planes[2] = {nullptr, nullptr};
  int64_t pitch = 0, Npad = 0;  // planes: first direction padded to `pitch`, Npad values per plane
  void* fsplit[2][3] = {{nullptr}};
  alignas(64) unsigned char tmA[3][2][cgl::kTensorMapBytes];
  alignas(64) unsigned char tmB[2][3][cgl::kTensorMapBytes];
  // FP64-accurate tensor-core path (CGL_F64_TC): per-rhs FP64 planes, 14
  // BF16 digit planes and per-fiber exponents, their TMA maps per mode; the
  // factor digits use fsplit / tmB, their per-row exponents fexp
  void* oz_z[2] = {nullptr, nullptr};
  void* oz_dig[2] = {nullptr, nullptr};
  int* oz_exp[2] = {nullptr, nullptr};
  int* fexp[2][3] = {{nullptr}};
  alignas(64) unsigned char oz_tmA[3][2][cgl::kTensorMapBytes];

  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* graph_u = nullptr;

  // profiling (when `prof` is set, launches are bracketed by events)
  bool prof = false;
  std::map<std::string, cgl::KernelStat>* stats = nullptr;
};

namespace cgl {

int64_t axis_P(const cgl_plan* p, int axis);
int64_t mma_axis_P(const cgl_plan* p, int axis);
int64_t mma_axis_Q(const cgl_plan* p, int axis);
PassGeom geom(const cgl_plan* p, int axis);
int dev_alloc(cgl_plan* p, void** ptr, size_t bytes);
cudaError_t prepare_kernels(int dev);
void free_plan(cgl_plan* p);
// Arguments of mode pass `mu` of sweep `sw` over the buffers {u, W0, W1, W2}.
ModePassArgs make_mode_args(const cgl_plan* p, const Sweep& sw, int mu, void* const* bufs);
// Plan construction; `minimal` skips the workspace, the capture stream and
// the tensor-core buffers (factors only, for batches).
// A (optional): caller-supplied direction matrices A_mu, complex n_mu x n_mu
// column-major as (re, im) doubles, replacing (a1 + i b1) D2_mu + a2/d.
// coupled (optional): {a0, a5} of the coupled two-field system (eq. coupled).
int plan_create_impl(cgl_plan** out, int d, const int64_t* n, const int* bc, const double* lo, const double* hi,
                     double a1, double b1, double a2, double a3, double b3, double a4, double b4, double tau,
                     int scheme, int precision, void* stream, bool minimal, const double* const* A = nullptr,
                     const double* coupled = nullptr);

}  // namespace cgl
