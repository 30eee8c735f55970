// Relative error norms (Sec. 4 measures relative errors against a reference
// solution): ||x-y||_2/||y||_2 and ||x-y||_inf/||y||_inf, FP64 accumulation,
// plus a count of non-finite entries of x (the blow-ups the paper's tables
// mark with a cross).  Two launches: per-block partials, then one block
// folds them.
#include <algorithm>

#include "plan.cuh"  // cgl::fail (last-error message)

namespace cgl {

constexpr int kNormThreads = 256;
constexpr int kNormMaxBlocks = 1024;
constexpr int kNormFields = 5;  // sum|d|^2, sum|y|^2, max|d|, max|y|, nonfinite

template <class T2>
__global__ void __launch_bounds__(kNormThreads) rel_error_partial(const T2* __restrict__ x,
                                                                  const T2* __restrict__ y, int64_t count,
                                                                  double* partial) {
  double sd = 0, sy = 0, md = 0, my = 0, nf = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T2 a = x[i], b = y[i];
    const double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y;
    const double d2 = dx * dx + dy * dy;
    const double y2 = (double)b.x * (double)b.x + (double)b.y * (double)b.y;
    if (!(isfinite((double)a.x) && isfinite((double)a.y))) { nf += 1; continue; }
    sd += d2;
    sy += y2;
    md = fmax(md, d2);
    my = fmax(my, y2);
  }
  __shared__ double red[kNormFields][kNormThreads / 32];
  double v[kNormFields] = {sd, sy, md, my, nf};
#pragma unroll
  for (int f = 0; f < kNormFields; ++f) {
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v[f], o);
      v[f] = (f == 2 || f == 3) ? fmax(v[f], w) : v[f] + w;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int f = 0; f < kNormFields; ++f) red[f][warp] = v[f];
  __syncthreads();
  if (threadIdx.x == 0) {
    double r[kNormFields] = {0, 0, 0, 0, 0};
    for (int w = 0; w < kNormThreads / 32; ++w)
      for (int f = 0; f < kNormFields; ++f)
        r[f] = (f == 2 || f == 3) ? fmax(r[f], red[f][w]) : r[f] + red[f][w];
    for (int f = 0; f < kNormFields; ++f) partial[f * gridDim.x + blockIdx.x] = r[f];
  }
}

__global__ void rel_error_final(const double* partial, int nblocks, double* result) {
  __shared__ double red[kNormFields][kNormThreads];
  double v[kNormFields] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int f = 0; f < kNormFields; ++f) {
      const double w = partial[f * nblocks + b];
      v[f] = (f == 2 || f == 3) ? fmax(v[f], w) : v[f] + w;
    }
  for (int f = 0; f < kNormFields; ++f) red[f][threadIdx.x] = v[f];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int f = 0; f < kNormFields; ++f) {
        const double w = red[f][threadIdx.x + s];
        red[f][threadIdx.x] = (f == 2 || f == 3) ? fmax(red[f][threadIdx.x], w) : red[f][threadIdx.x] + w;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sd = red[0][0], sy = red[1][0], md = red[2][0], my = red[3][0];
    result[0] = sy > 0 ? sqrt(sd / sy) : (sd > 0 ? INFINITY : 0.0);
    result[1] = my > 0 ? sqrt(md / my) : (md > 0 ? INFINITY : 0.0);
    result[2] = red[4][0];
  }
}

int rel_error_blocks(int64_t count) {
  const int64_t b = (count + kNormThreads - 1) / kNormThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, kNormMaxBlocks));
}

// d_partial: kNormFields * nblocks + 3 doubles of device scratch.
cudaError_t rel_error_device(const void* x, const void* y, int64_t count, int precision, double* d_partial,
                             int nblocks, double* h_out, cudaStream_t s) {
  double* result = d_partial + kNormFields * nblocks;
  if (precision == CGL_F64)
    rel_error_partial<double2><<<nblocks, kNormThreads, 0, s>>>((const double2*)x, (const double2*)y, count,
                                                                 d_partial);
  else
    rel_error_partial<float2><<<nblocks, kNormThreads, 0, s>>>((const float2*)x, (const float2*)y, count,
                                                                d_partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rel_error_final<<<1, kNormThreads, 0, s>>>(d_partial, nblocks, result);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(h_out, result, 3 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(s);
}

}  // namespace cgl

// ---------------------------------------------------------------------------
// Allocation-free variant of the error norms (cgl_rel_error_noalloc).
//
// Same arithmetic as rel_error_device, but its per-block partial sums live in
// the file-scope device array below instead of a cudaMallocAsync buffer, so a
// call performs no device allocation of any kind.  Each block of the variant
// reduces one fixed chunk of kStaticChunk values, so the array's capacity
// (kStaticMaxBlocks partial records) bounds the accepted count at
// kStaticMaxBlocks * kStaticChunk values; larger counts are rejected.
// ---------------------------------------------------------------------------

#include <mutex>

namespace cgl {

constexpr int kStaticChunk = 65536;     // values reduced by one block
constexpr int kStaticMaxBlocks = 4096;  // partial records the array holds
static_assert((int64_t)kStaticChunk * kStaticMaxBlocks == CGL_REL_ERROR_NOALLOC_MAX_COUNT,
              "header limit must match the scratch capacity");

// Scratch shared by every call on a device: kNormFields partials per block,
// then 3 result slots.  164 KiB, resident on each GPU that loads the library
// until the process exits.
static __device__ __align__(256) double g_norm_scratch[kNormFields * kStaticMaxBlocks + 3];

template <class T2>
__global__ void __launch_bounds__(kNormThreads) rel_error_partial_chunked(const T2* __restrict__ x,
                                                                          const T2* __restrict__ y,
                                                                          int64_t count, double* partial) {
  double sd = 0, sy = 0, md = 0, my = 0, nf = 0;
  const int64_t beg = (int64_t)blockIdx.x * kStaticChunk;
  const int64_t end = min(count, beg + kStaticChunk);
  for (int64_t i = beg + threadIdx.x; i < end; i += kNormThreads) {
    const T2 a = x[i], b = y[i];
    const double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y;
    const double d2 = dx * dx + dy * dy;
    const double y2 = (double)b.x * (double)b.x + (double)b.y * (double)b.y;
    if (!(isfinite((double)a.x) && isfinite((double)a.y))) { nf += 1; continue; }
    sd += d2;
    sy += y2;
    md = fmax(md, d2);
    my = fmax(my, y2);
  }
  __shared__ double red[kNormFields][kNormThreads / 32];
  double v[kNormFields] = {sd, sy, md, my, nf};
#pragma unroll
  for (int f = 0; f < kNormFields; ++f) {
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v[f], o);
      v[f] = (f == 2 || f == 3) ? fmax(v[f], w) : v[f] + w;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int f = 0; f < kNormFields; ++f) red[f][warp] = v[f];
  __syncthreads();
  if (threadIdx.x == 0) {
    double r[kNormFields] = {0, 0, 0, 0, 0};
    for (int w = 0; w < kNormThreads / 32; ++w)
      for (int f = 0; f < kNormFields; ++f)
        r[f] = (f == 2 || f == 3) ? fmax(r[f], red[f][w]) : r[f] + red[f][w];
    for (int f = 0; f < kNormFields; ++f) partial[f * gridDim.x + blockIdx.x] = r[f];
  }
}

// Device address of g_norm_scratch, looked up once per device with that
// device current.  In host code the array's name is only a host-side shadow,
// never a device pointer, so kernels get the address found here.
static std::mutex g_scratch_mutex;
static double* g_scratch_ptr[64] = {nullptr};

static cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_norm_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace cgl

extern "C" int cgl_rel_error_noalloc(const void* x, const void* y, int64_t count, int precision, double* out,
                                     void* stream) {
  using namespace cgl;
  if (!x || !y || !out) return fail(CGL_EINVAL, "NULL argument");
  if (count <= 0) return fail(CGL_EINVAL, "count must be positive");
  if (count > CGL_REL_ERROR_NOALLOC_MAX_COUNT)
    return fail(CGL_EINVAL, "count exceeds CGL_REL_ERROR_NOALLOC_MAX_COUNT (the static scratch capacity)");
  if (precision == CGL_BF16X3) precision = CGL_F32;  // complex64 state, as cgl_rel_error
  if (precision == CGL_F64_TC) precision = CGL_F64;   // complex128 state
  if (precision != CGL_F64 && precision != CGL_F32) return fail(CGL_EINVAL, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  double* partial = nullptr;
  cudaError_t e = static_scratch(&partial);
  if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  const int nblocks = (int)((count + kStaticChunk - 1) / kStaticChunk);
  double* result = partial + kNormFields * nblocks;
  if (precision == CGL_F64)
    rel_error_partial_chunked<double2><<<nblocks, kNormThreads, 0, s>>>((const double2*)x, (const double2*)y,
                                                                        count, partial);
  else
    rel_error_partial_chunked<float2><<<nblocks, kNormThreads, 0, s>>>((const float2*)x, (const float2*)y,
                                                                       count, partial);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return fail(CGL_ECUDA, std::string("rel_error_noalloc: ") + cudaGetErrorString(e));
  rel_error_final<<<1, kNormThreads, 0, s>>>(partial, nblocks, result);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return fail(CGL_ECUDA, std::string("rel_error_noalloc: ") + cudaGetErrorString(e));
  if ((e = cudaMemcpyAsync(out, result, 3 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(CGL_ECUDA, std::string("rel_error_noalloc: ") + cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(CGL_ECUDA, std::string("rel_error_noalloc: ") + cudaGetErrorString(e));
  return CGL_OK;
}
