// Learned residual corrector for the coarse periodic step: training and
// inference kernels.
//
// The corrected step is u_{n+1} = C(u_n) + N(x): C a coarse Lawson4 step
// (eq. lawson4), x = 9 planes (Re, Im of C(u_n); Re, Im of u_n; the
// parameters a1, b1, a2, a3, b3 as constant planes), N a stack of 3x3
// convolutions with circular padding (the periodic boundary), ReLU between
// layers, 2 output planes.  Weights: FP32 masters, BF16 copies used by every
// convolution, FP32 accumulation; Adam (Kingma & Ba 2015) on the masters.
//
// Activations are NCHW FP32 (W fastest).  A 3x3 convolution is an implicit
// GEMM on the tensor cores (conv_mma.cu: per 128-pixel tile, nine
// accumulating 128 x Cout x Cin MMAs with BF16 operands, FP32 accumulation).
// The backward pass w.r.t. the input is the same convolution with the kernel
// flipped and the channel roles swapped; the weight gradient is an implicit
// GEMM on the tensor cores too (K = pixels, BF16 x and dy, FP32
// accumulation), per-CTA partial sums finished with atomics.  The layers here
// are 9..32 channels wide: about 144 flop per byte of activation traffic, so
// these convolutions are bounded by memory, not by arithmetic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "plan.cuh"

using namespace cgl;

namespace cgl {

constexpr int kTile = 16;
constexpr int kMaxCh = 32;

// ------------------------------------------------------------------ kernels

// x[b][c][i][j] from complex64 coarse results / states [P][H][W] selected by
// idx (or b itself) and parameters [P][5].
template <class T2>
__global__ void features_kernel(const T2* __restrict__ coarse, const T2* __restrict__ un,
                                const float* __restrict__ params, const int* __restrict__ idx, int B, int H, int W,
                                float* __restrict__ x) {
  const int64_t HW = (int64_t)H * W;
  const int64_t total = (int64_t)B * HW;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / HW);
    const int64_t p = e - (int64_t)b * HW;
    const int src = idx ? idx[b] : b;
    const T2 c = coarse[(int64_t)src * HW + p];
    const T2 u = un[(int64_t)src * HW + p];
    float* xb = x + (int64_t)b * 9 * HW + p;
    xb[0 * HW] = (float)c.x;
    xb[1 * HW] = (float)c.y;
    xb[2 * HW] = (float)u.x;
    xb[3 * HW] = (float)u.y;
    for (int k = 0; k < 5; ++k) xb[(4 + k) * HW] = params[(int64_t)src * 5 + k];
  }
}

// dy *= (a > 0)
__global__ void relu_backward_kernel(float* __restrict__ dy, const float* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(a[i] > 0.f)) dy[i] = 0.f;
}

// r = C(u_n) + out - target (complex64 [P] selected by idx), or r = out -
// target when the target is the correction itself (correction != 0);
// dout = 2 r / count; loss partial sums in FP64.
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ scales,
                            const float2* __restrict__ coarse,
                            const float2* __restrict__ target, const int* __restrict__ idx, int B, int64_t HW,
                            int correction, float* __restrict__ dout, double* __restrict__ loss_sum) {
  const double inv = 1.0 / (2.0 * (double)B * (double)HW);
  double s = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)B * HW;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / HW);
    const int64_t p = e - (int64_t)b * HW;
    const int src = idx ? idx[b] : b;
    const float scale = scales[b];
    const float2 c = correction ? make_float2(0.f, 0.f) : coarse[(int64_t)src * HW + p];
    const float2 t = target[(int64_t)src * HW + p];
    const float* ob = out + (int64_t)b * 2 * HW + p;
    // residual in units of the output scale: (C(u_n) + scale*out - target) / scale
    const float rr = (fmaf(scale, ob[0], c.x) - t.x) / scale, ri = (fmaf(scale, ob[HW], c.y) - t.y) / scale;
    s += (double)rr * rr + (double)ri * ri;
    float* db = dout + (int64_t)b * 2 * HW + p;
    db[0] = (float)(2.0 * inv) * rr;
    db[HW] = (float)(2.0 * inv) * ri;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, s * inv);
}

// Adam on FP32 masters, BF16 copies refreshed.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ pbf, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pbf[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = __float2bfloat16_rn(p[i]);
}

// wr[ci][co][8-k] = w[co][ci][k]: the kernel of the input-gradient convolution.
__global__ void flip_weights_kernel(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wr, int Cin,
                                    int Cout) {
  const int n = Cin * Cout * 9;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int k = e % 9, ci = (e / 9) % Cin, co = e / (9 * Cin);
    wr[((int64_t)ci * Cout + co) * 9 + (8 - k)] = w[e];
  }
}

// u = C(u_n) + scale * raw network output, in the state's precision
template <class T2>
__global__ void residual_add_kernel(const T2* __restrict__ coarse, const float* __restrict__ out,
                                    const float* __restrict__ scales, int B, int64_t HW, T2* __restrict__ u) {
  using T = decltype(T2{}.x);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)B * HW;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / HW);
    const int64_t p = e - (int64_t)b * HW;
    const T2 c = coarse[e];
    const float* ob = out + (int64_t)b * 2 * HW + p;
    const float scale = scales[b];
    T2 r;
    r.x = fma((T)scale, (T)ob[0], c.x);
    r.y = fma((T)scale, (T)ob[HW], c.y);
    u[e] = r;
  }
}

// b = scale_s * a for sample s of each [per_sample] block
__global__ void scale_copy_kernel(const float* __restrict__ a, const float* __restrict__ scale,
                                  float* __restrict__ b, int64_t n, int64_t per_sample) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = scale[i / per_sample] * a[i];
}

// Output scale of each sample: mode 0, the output scale itself; mode 1, the
// output scale times the RMS over the sample of |C(u_n) - u_n| (the coarse
// increment), which follows the size of the correction from sample to
// sample.  One block per sample; samples selected by idx (or b).
template <class T2>
__global__ void sample_scale_kernel(const T2* __restrict__ coarse, const T2* __restrict__ un,
                                    const int* __restrict__ idx, int64_t HW, float out_scale, int mode,
                                    float* __restrict__ scale) {
  const int b = blockIdx.x;
  if (mode == 0) {
    if (threadIdx.x == 0) scale[b] = out_scale;
    return;
  }
  const int src = idx ? idx[b] : b;
  double acc = 0;
  for (int64_t p = threadIdx.x; p < HW; p += blockDim.x) {
    const T2 c = coarse[(int64_t)src * HW + p], u = un[(int64_t)src * HW + p];
    const double dx = (double)c.x - (double)u.x, dy = (double)c.y - (double)u.y;
    acc += dx * dx + dy * dy;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const float r = (float)sqrt(t / (double)HW);
    scale[b] = out_scale * (r > 0.f ? r : 1.f);
  }
}

}  // namespace cgl

// ------------------------------------------------------------------ host side

struct cgl_corrector {
  int dev = 0;
  int H = 0, W = 0, hidden = 0, nlayers = 0, max_batch = 0;
  struct Layer {
    int cin, cout, relu;
    int64_t w_off, b_off;
  };
  std::vector<Layer> layers;
  int64_t nparams = 0;
  float* master = nullptr;
  __nv_bfloat16* wbf = nullptr;
  __nv_bfloat16* wflip = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int64_t t = 0;
  float out_scale = 1.f;  // N(x) = out_scale * (last convolution)
  int target_mode = 0;    // 0: target = fine state; 1: target = the correction (fine - coarse)
  int scale_mode = 0;     // 0: N = out_scale a; 1: N = out_scale rms(C(u_n) - u_n) a, per sample
  float* sample_scale = nullptr;  // device [max_batch]: the scale of each sample of the last call
  std::vector<float*> acts;  // acts[0] = features, acts[l+1] = output of layer l
  std::vector<float*> dys;   // dys[l] = loss gradient w.r.t. layer l's output (after its ReLU mask)
  double* loss = nullptr;
  int* status = nullptr;  // device word: bit 1 = a bounded tensor-core wait gave up
  std::vector<void*> allocations;
};

namespace {

int corr_alloc(cgl_corrector* c, void** p, size_t bytes) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return fail(CGL_ENOMEM, "cudaMalloc: injected allocation failure");
  }
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(CGL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocations.push_back(*p);
  return CGL_OK;
}

void free_corrector(cgl_corrector* c) {
  if (!c) return;
  for (void* a : c->allocations) cudaFree(a);
  delete c;
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 32); }

cudaError_t launch_conv(const float* x, const __nv_bfloat16* w, const float* bias, float* y, int B, int cin, int cout,
                        int H, int W, int relu, int* status, cudaStream_t s) {
  return launch_conv_mma(x, w, bias, y, B, cin, cout, H, W, relu, status, s);
}

cudaError_t prepare_corrector_kernels() {
  return prepare_conv_mma();
}

// splitmix64 (Steele, Lea & Flood 2014): a counter-based generator for the
// initial weights.
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

int forward_pass(cgl_corrector* c, int B, cudaStream_t s) {
  for (int l = 0; l < c->nlayers; ++l) {
    const auto& L = c->layers[l];
    cudaError_t e = launch_conv(c->acts[l], c->wbf + L.w_off, c->master + L.b_off, c->acts[l + 1], B, L.cin, L.cout,
                                c->H, c->W, L.relu, c->status, s);
    if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("conv forward: ") + cudaGetErrorString(e));
  }
  return CGL_OK;
}

int check_batch(cgl_corrector* c, int B) {
  if (!c) return fail(CGL_EINVAL, "corrector is NULL");
  if (B < 1 || B > c->max_batch) return fail(CGL_EINVAL, "batch must be in 1..max_batch");
  return CGL_OK;
}

// features -> forward -> loss -> backward (gradients in c->grad); loss to *loss_out.
int loss_backward(cgl_corrector* c, const void* coarse, const void* un, const void* target, const float* params,
                  const int* idx, int B, double* loss_out, cudaStream_t s) {
  const int64_t HW = (int64_t)c->H * c->W;
  features_kernel<float2><<<grid_for(B * HW), 256, 0, s>>>((const float2*)coarse, (const float2*)un, params, idx, B, c->H,
                                                   c->W, c->acts[0]);
  CUDA_TRY(cudaGetLastError());
  int st = forward_pass(c, B, s);
  if (st) return st;
  CUDA_TRY(cudaMemsetAsync(c->loss, 0, sizeof(double), s));
  CUDA_TRY(cudaMemsetAsync(c->grad, 0, c->nparams * sizeof(float), s));
  sample_scale_kernel<float2><<<B, 256, 0, s>>>((const float2*)coarse, (const float2*)un, idx, HW, c->out_scale,
                                                c->scale_mode, c->sample_scale);
  CUDA_TRY(cudaGetLastError());
  loss_kernel<<<grid_for(B * HW), 256, 0, s>>>(c->acts[c->nlayers], c->sample_scale, (const float2*)coarse,
                                               (const float2*)target, idx, B, HW, c->target_mode,
                                               c->dys[c->nlayers - 1], c->loss);
  CUDA_TRY(cudaGetLastError());
  for (int l = c->nlayers - 1; l >= 0; --l) {
    const auto& L = c->layers[l];
    float* dy = c->dys[l];
    if (l < c->nlayers - 1) {
      relu_backward_kernel<<<grid_for(B * L.cout * HW), 256, 0, s>>>(dy, c->acts[l + 1], (int64_t)B * L.cout * HW);
      CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(launch_wgrad_mma(c->acts[l], dy, c->grad + L.w_off, c->grad + L.b_off, B, L.cin, L.cout, c->H, c->W,
                              c->status, s));
    if (l > 0) {
      flip_weights_kernel<<<grid_for(L.cin * L.cout * 9), 256, 0, s>>>(c->wbf + L.w_off, c->wflip, L.cin, L.cout);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(launch_conv(dy, c->wflip, nullptr, c->dys[l - 1], B, L.cout, L.cin, c->H, c->W, 0, c->status, s));
    }
  }
  if (loss_out) {
    CUDA_TRY(cudaMemcpyAsync(loss_out, c->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return CGL_OK;
}

}  // namespace

extern "C" {

int cgl_corrector_create(cgl_corrector** out, int height, int width, int hidden, int layers, int max_batch,
                         uint64_t seed, void* stream) {
  if (!out) return fail(CGL_EINVAL, "out is NULL");
  *out = nullptr;
  if (height < kTile || width < kTile || height % kTile || width % kTile)
    return fail(CGL_EINVAL, "height and width must be positive multiples of 16");
  if (hidden < 1 || hidden > kMaxCh || layers < 2 || layers > 16 || max_batch < 1)
    return fail(CGL_EINVAL, "hidden in 1..32, layers in 2..16, max_batch >= 1");
  cudaError_t e = prepare_corrector_kernels();
  if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  cgl_corrector* c = new cgl_corrector();
  cudaGetDevice(&c->dev);
  c->H = height;
  c->W = width;
  c->hidden = hidden;
  c->nlayers = layers;
  c->max_batch = max_batch;
  int64_t off = 0;
  for (int l = 0; l < layers; ++l) {
    cgl_corrector::Layer L;
    L.cin = l == 0 ? 9 : hidden;
    L.cout = l == layers - 1 ? 2 : hidden;
    L.relu = l < layers - 1;
    L.w_off = off;
    off += (int64_t)L.cout * L.cin * 9;
    L.b_off = off;
    off += L.cout;
    c->layers.push_back(L);
  }
  c->nparams = off;
  int st = CGL_OK;
  const int64_t HW = (int64_t)height * width;
  st = corr_alloc(c, (void**)&c->master, off * sizeof(float));
  if (!st) st = corr_alloc(c, (void**)&c->wbf, off * sizeof(__nv_bfloat16));
  if (!st) st = corr_alloc(c, (void**)&c->wflip, (size_t)kMaxCh * kMaxCh * 9 * sizeof(__nv_bfloat16));
  if (!st) st = corr_alloc(c, (void**)&c->grad, off * sizeof(float));
  if (!st) st = corr_alloc(c, (void**)&c->m, off * sizeof(float));
  if (!st) st = corr_alloc(c, (void**)&c->v, off * sizeof(float));
  if (!st) st = corr_alloc(c, (void**)&c->loss, sizeof(double));
  if (!st) st = corr_alloc(c, (void**)&c->sample_scale, (size_t)max_batch * sizeof(float));
  if (!st) st = corr_alloc(c, (void**)&c->status, sizeof(int));
  if (!st && cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) st = fail(CGL_ECUDA, "memset status");
  for (int l = 0; !st && l <= layers; ++l) {
    const int ch = l == 0 ? 9 : c->layers[l - 1].cout;
    float* a = nullptr;
    st = corr_alloc(c, (void**)&a, (size_t)max_batch * ch * HW * sizeof(float));
    c->acts.push_back(a);
  }
  for (int l = 0; !st && l < layers; ++l) {
    float* g = nullptr;
    st = corr_alloc(c, (void**)&g, (size_t)max_batch * c->layers[l].cout * HW * sizeof(float));
    c->dys.push_back(g);
  }
  if (!st) {
    // He-uniform initial weights from splitmix64(seed, index); last layer
    // scaled by 0.1 so the untrained correction starts small; zero biases.
    std::vector<float> h(off, 0.f);
    for (int l = 0; l < layers; ++l) {
      const auto& L = c->layers[l];
      const double bound = std::sqrt(6.0 / (L.cin * 9.0)) * (l == layers - 1 ? 0.1 : 1.0);
      for (int64_t k = 0; k < (int64_t)L.cout * L.cin * 9; ++k) {
        const double u = (splitmix64(seed ^ (uint64_t)(L.w_off + k) * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
        h[L.w_off + k] = (float)((2.0 * u - 1.0) * bound);
      }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(c->master, h.data(), off * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(c->m, 0, off * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(c->v, 0, off * sizeof(float), s) != cudaSuccess)
      st = fail(CGL_ECUDA, "corrector initialisation");
    if (!st) {
      to_bf16_kernel<<<grid_for(off), 256, 0, s>>>(c->master, c->wbf, off);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        st = fail(CGL_ECUDA, "corrector initialisation");
    }
  }
  if (st) {
    free_corrector(c);
    return st;
  }
  *out = c;
  return CGL_OK;
}

int cgl_corrector_num_params(const cgl_corrector* c, int64_t* count) {
  if (!c || !count) return fail(CGL_EINVAL, "NULL argument");
  *count = c->nparams;
  return CGL_OK;
}

int cgl_corrector_set_weights(cgl_corrector* c, const float* host, int64_t count) {
  if (!c || !host || count != c->nparams) return fail(CGL_EINVAL, "weights: NULL or wrong count");
  CUDA_TRY(cudaMemcpy(c->master, host, count * sizeof(float), cudaMemcpyHostToDevice));
  to_bf16_kernel<<<grid_for(count), 256>>>(c->master, c->wbf, count);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemset(c->m, 0, count * sizeof(float)));
  CUDA_TRY(cudaMemset(c->v, 0, count * sizeof(float)));
  CUDA_TRY(cudaDeviceSynchronize());
  c->t = 0;
  return CGL_OK;
}

int cgl_corrector_get_weights(const cgl_corrector* c, float* host, int64_t count) {
  if (!c || !host || count != c->nparams) return fail(CGL_EINVAL, "weights: NULL or wrong count");
  CUDA_TRY(cudaMemcpy(host, c->master, count * sizeof(float), cudaMemcpyDeviceToHost));
  return CGL_OK;
}

int cgl_corrector_forward(cgl_corrector* c, const void* coarse, const void* un, const float* params, const int* idx,
                          int batch, float* out, void* stream) {
  int st = check_batch(c, batch);
  if (st) return st;
  if (!coarse || !un || !params || !out) return fail(CGL_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t HW = (int64_t)c->H * c->W;
  features_kernel<float2><<<grid_for(batch * HW), 256, 0, s>>>((const float2*)coarse, (const float2*)un, params, idx, batch,
                                                       c->H, c->W, c->acts[0]);
  CUDA_TRY(cudaGetLastError());
  if ((st = forward_pass(c, batch, s))) return st;
  sample_scale_kernel<float2><<<batch, 256, 0, s>>>((const float2*)coarse, (const float2*)un, idx, HW,
                                                    c->out_scale, c->scale_mode, c->sample_scale);
  CUDA_TRY(cudaGetLastError());
  scale_copy_kernel<<<grid_for(batch * 2 * HW), 256, 0, s>>>(c->acts[c->nlayers], c->sample_scale, out,
                                                             (int64_t)batch * 2 * HW, 2 * HW);
  CUDA_TRY(cudaGetLastError());
  return CGL_OK;
}

int cgl_corrector_gradients(cgl_corrector* c, const void* coarse, const void* un, const void* target,
                            const float* params, const int* idx, int batch, float* grads_host, double* loss,
                            void* stream) {
  int st = check_batch(c, batch);
  if (st) return st;
  if (!coarse || !un || !target || !params) return fail(CGL_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = loss_backward(c, coarse, un, target, params, idx, batch, loss, s))) return st;
  if (grads_host) {
    CUDA_TRY(cudaMemcpyAsync(grads_host, c->grad, c->nparams * sizeof(float), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return CGL_OK;
}

int cgl_corrector_train_step(cgl_corrector* c, const void* coarse, const void* un, const void* target,
                             const float* params, const int* idx, int batch, float lr, double* loss, void* stream) {
  int st = check_batch(c, batch);
  if (st) return st;
  if (!coarse || !un || !target || !params || !(lr > 0.f)) return fail(CGL_EINVAL, "NULL argument or lr <= 0");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = loss_backward(c, coarse, un, target, params, idx, batch, loss, s))) return st;
  c->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)c->t), c2 = 1.f - std::pow(b2, (float)c->t);
  adam_kernel<<<grid_for(c->nparams), 256, 0, s>>>(c->master, c->grad, c->m, c->v, c->wbf, c->nparams, lr, b1, b2,
                                                   1e-8f, c1, c2);
  CUDA_TRY(cudaGetLastError());
  return CGL_OK;
}

int cgl_corrector_apply(cgl_corrector* c, const void* coarse, const void* un, const float* params, int batch,
                        void* u_out, void* stream) {
  int st = check_batch(c, batch);
  if (st) return st;
  if (!coarse || !un || !params || !u_out) return fail(CGL_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t HW = (int64_t)c->H * c->W;
  features_kernel<float2><<<grid_for(batch * HW), 256, 0, s>>>((const float2*)coarse, (const float2*)un, params, nullptr,
                                                       batch, c->H, c->W, c->acts[0]);
  CUDA_TRY(cudaGetLastError());
  if ((st = forward_pass(c, batch, s))) return st;
  sample_scale_kernel<float2><<<batch, 256, 0, s>>>((const float2*)coarse, (const float2*)un, nullptr, HW,
                                                    c->out_scale, c->scale_mode, c->sample_scale);
  CUDA_TRY(cudaGetLastError());
  residual_add_kernel<float2><<<grid_for(batch * HW), 256, 0, s>>>((const float2*)coarse, c->acts[c->nlayers],
                                                                   c->sample_scale, batch, HW, (float2*)u_out);
  CUDA_TRY(cudaGetLastError());
  return CGL_OK;
}

int cgl_corrector_apply_c128(cgl_corrector* c, const void* coarse, const void* un, const float* params, int batch,
                             void* u_out, void* stream) {
  int st = check_batch(c, batch);
  if (st) return st;
  if (!coarse || !un || !params || !u_out) return fail(CGL_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t HW = (int64_t)c->H * c->W;
  features_kernel<double2><<<grid_for(batch * HW), 256, 0, s>>>((const double2*)coarse, (const double2*)un, params,
                                                                nullptr, batch, c->H, c->W, c->acts[0]);
  CUDA_TRY(cudaGetLastError());
  if ((st = forward_pass(c, batch, s))) return st;
  sample_scale_kernel<double2><<<batch, 256, 0, s>>>((const double2*)coarse, (const double2*)un, nullptr, HW,
                                                     c->out_scale, c->scale_mode, c->sample_scale);
  CUDA_TRY(cudaGetLastError());
  residual_add_kernel<double2><<<grid_for(batch * HW), 256, 0, s>>>((const double2*)coarse, c->acts[c->nlayers],
                                                                    c->sample_scale, batch, HW, (double2*)u_out);
  CUDA_TRY(cudaGetLastError());
  return CGL_OK;
}

int cgl_corrector_set_scale_mode(cgl_corrector* c, int mode) {
  if (!c || (mode != 0 && mode != 1)) return fail(CGL_EINVAL, "mode must be 0 (global) or 1 (per sample)");
  c->scale_mode = mode;
  return CGL_OK;
}

int cgl_corrector_set_target_mode(cgl_corrector* c, int mode) {
  if (!c || (mode != 0 && mode != 1)) return fail(CGL_EINVAL, "mode must be 0 (fine state) or 1 (correction)");
  c->target_mode = mode;
  return CGL_OK;
}

int cgl_corrector_set_output_scale(cgl_corrector* c, float scale) {
  if (!c || !(scale > 0.f) || !std::isfinite(scale)) return fail(CGL_EINVAL, "scale must be positive and finite");
  c->out_scale = scale;
  return CGL_OK;
}

int cgl_corrector_layer_state(const cgl_corrector* c, int kind, int layer, float* dst, int64_t count,
                              void* stream) {
  if (!c || !dst) return fail(CGL_EINVAL, "NULL argument");
  const int64_t HW = (int64_t)c->H * c->W;
  const float* src = nullptr;
  int ch = 0;
  if (kind == 0 && layer >= 0 && layer <= c->nlayers) {
    src = c->acts[layer];
    ch = layer == 0 ? 9 : c->layers[layer - 1].cout;
  } else if (kind == 1 && layer >= 0 && layer < c->nlayers) {
    src = c->dys[layer];
    ch = c->layers[layer].cout;
  } else {
    return fail(CGL_EINVAL, "kind must be 0 (activation, layer 0..layers) or 1 (gradient, layer 0..layers-1)");
  }
  if (count < 1 || count > (int64_t)c->max_batch * ch * HW) return fail(CGL_EINVAL, "count out of range");
  CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(float), cudaMemcpyDefault, (cudaStream_t)stream));
  return CGL_OK;
}

int cgl_corrector_last_device_status(cgl_corrector* c, void* stream) {
  if (!c) return fail(CGL_EINVAL, "corrector is NULL");
  CUDA_TRY(cudaSetDevice(c->dev));
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return (h & 2) ? CGL_ETIMEOUT : CGL_OK;
}

int cgl_corrector_destroy(cgl_corrector* c) {
  if (!c) return CGL_OK;
  cudaSetDevice(c->dev);
  free_corrector(c);
  return CGL_OK;
}

}  // extern "C"
