// 3x3 convolution with circular padding on the 5th-generation tensor cores
// (the corrector's forward and input-gradient convolutions).
//
// Implicit GEMM per tile of 128 consecutive output pixels of one sample
// (pixel index p = i W + j, one TMEM lane each):
//   Y[p, co] = sum_{tap t, ci} X[ci, p + shift_t] W[co, ci, t],
// i.e. nine accumulating GEMMs of 128 x Cout x Cin.  For every tap the CTA
// gathers its im2col tile X_t[p, ci] (circular neighbours, zero for padded
// channels and for pixels past H W) as BF16 (round to nearest even) into
// shared memory in the K-major layout without swizzle: 16-byte rows of eight
// channels, core matrices of 8 pixels x 16 bytes contiguous (SBO = 128 B
// between 8-pixel groups), the next eight channels one 2 KB block further
// (LBO).  The weights sit in shared memory for the whole kernel in the same
// layout (rows = output channels).  One thread issues
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = Cout rounded up to 16,
// K = 16) for all taps and channel blocks into one FP32 TMEM accumulator and
// commits to an mbarrier; after a bounded wait every warp reads its 32 lanes
// (tcgen05.ld), adds the bias, applies ReLU and stores FP32 NCHW, coalesced
// along the pixel index.  CTAs walk the tiles with stride gridDim.x.
//
// Operand rounding: activations (or incoming gradients) and weights enter
// the MMA as BF16, products accumulate in FP32.  A wait that times out sets
// bit 1 of *status and the CTA stops; TMEM is freed on every path.
#include <cuda_bf16.h>

#include <algorithm>
#include <string>

#include "plan.cuh"
#include "tc_ptx.cuh"

namespace cgl {

constexpr int kConvM = 128;
constexpr int kConvMmaThreads = 128;

struct ConvMmaArgs {
  const float* x;           // [B][Cin][H][W]
  const __nv_bfloat16* w;   // [Cout][Cin][3][3]
  const float* bias;        // [Cout] or null
  float* y;                 // [B][Cout][H][W]
  int B, Cin, Cout, H, W, relu;
  int kc;                   // Cin rounded up to a multiple of 16
  int nn;                   // Cout rounded up to a multiple of 16 (<= 32)
  int* status;
};

static size_t conv_mma_smem(int kc, int nn) {
  const size_t a = 9 * (size_t)(kc / 8) * kConvM * 16;
  const size_t b = 9 * (size_t)(kc / 8) * nn * 16;
  return a + b + 16;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(lo))) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(hi))) << 16);
}

__global__ void __launch_bounds__(kConvMmaThreads) conv3x3_mma_kernel(const ConvMmaArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int nq = a.kc / 8;  // 8-channel chunks
  uint8_t* As = smem;                                   // [9][nq][128 px][16 B]
  uint8_t* Bs = As + 9 * nq * kConvM * 16;              // [9][nq][nn][16 B]
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + 9 * nq * a.nn * 16);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t HW = (int64_t)a.H * a.W;

  // weights, once: row n = output channel, 16-byte rows of eight input channels
  for (int e = tid; e < 9 * nq * a.nn; e += kConvMmaThreads) {
    const int n = e % a.nn, q = (e / a.nn) % nq, t = e / (a.nn * nq);
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ci = q * 8 + k;
      v[k] = (n < a.Cout && ci < a.Cin) ? __bfloat162float(a.w[((int64_t)n * a.Cin + ci) * 9 + t]) : 0.f;
    }
    *reinterpret_cast<uint4*>(Bs + (size_t)e * 16) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  }
  if (tid == 0) {
    mbar_init(smem_u32(bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), 32);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t idesc = idesc_bf16(kConvM, a.nn, 0);
  const int64_t tpi = (HW + kConvM - 1) / kConvM;
  const int64_t ntiles = (int64_t)a.B * tpi;
  uint32_t parity = 0;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = (int)(tile / tpi);
    const int64_t p = (tile - (int64_t)b * tpi) * kConvM + tid;
    const bool valid = p < HW;
    const int pi = valid ? (int)(p / a.W) : 0, pj = valid ? (int)(p - (int64_t)pi * a.W) : 0;
    const float* xb = a.x + (int64_t)b * a.Cin * HW;
    // im2col of the nine taps: this thread's pixel, all channel chunks
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
      const int si = (pi + t / 3 - 1 + a.H) % a.H, sj = (pj + t % 3 - 1 + a.W) % a.W;
      const int64_t src = (int64_t)si * a.W + sj;
      for (int q = 0; q < nq; ++q) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int ci = q * 8 + k;
          v[k] = (valid && ci < a.Cin) ? xb[(int64_t)ci * HW + src] : 0.f;
        }
        *reinterpret_cast<uint4*>(As + ((size_t)(t * nq + q) * kConvM + tid) * 16) =
            make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      for (int t = 0; t < 9; ++t) {
        for (int kk = 0; kk < a.kc / 16; ++kk) {
          const int q = t * nq + 2 * kk;
          const uint64_t ad = smem_desc(a0 + (uint32_t)q * kConvM * 16, kConvM * 16, 128, 0);
          const uint64_t bd = smem_desc(b0 + (uint32_t)q * a.nn * 16, (uint32_t)a.nn * 16, 128, 0);
          mma_bf16(tmem, ad, bd, idesc, (t > 0 || kk > 0) ? 1u : 0u);
        }
      }
      mma_commit(smem_u32(bar));
    }
    const bool ok = __syncthreads_and(mbar_wait(smem_u32(bar), parity)) != 0;
    parity ^= 1u;
    if (!ok) {
      if (tid == 0 && a.status) atomicOr(a.status, 2);
      break;
    }
    tc_fence_after();
    // epilogue: warp w holds TMEM lanes 32 w .. 32 w + 31 = pixels p
    uint32_t r[32];
    const uint32_t lane_addr = static_cast<uint32_t>(warp * 32) << 16;
    tmem_ld16(tmem + lane_addr, r);
    if (a.nn > 16) tmem_ld16(tmem + lane_addr + 16, r + 16);
    if (valid) {
      float* yb = a.y + (int64_t)b * a.Cout * HW + p;
      for (int co = 0; co < a.Cout; ++co) {
        float v = __uint_as_float(r[co]) + (a.bias ? a.bias[co] : 0.f);
        if (a.relu) v = fmaxf(v, 0.f);
        yb[(int64_t)co * HW] = v;
      }
    }
    (void)lane;
    tc_fence_before();
    __syncthreads();  // TMEM read and the im2col tile consumed before the next tile
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 32);
  }
}

// ------------------------------------------------------------------ weight gradient

// Weight and bias gradients of the 3x3 circular convolution on the tensor
// cores:
//   dW[co, ci, t] = sum_{b, p} dy[b, co, p] x[b, ci, p + shift_t],
//   db[co] = sum_{b, p} dy[b, co, p],
// per 128-pixel tile an implicit GEMM D[m, co] += sum_p A[m, p] B[co, p] with
// K = the tile's pixels, rows m = t Cin + ci (the nine shifted copies of x)
// plus one row of ones (m = 9 Cin: the bias gradient), in M-tiles of 128
// rows; B = dy.  Both operands are BF16 (rounded to nearest even) in the
// K-major layout without swizzle: 16-byte rows of eight pixels, core
// matrices of 8 rows x 16 bytes contiguous (SBO = 128 B between 8-row
// groups), the next eight pixels one block of all rows further (LBO).  FP32
// accumulation in TMEM (one accumulator of nn columns per M-tile) over a run
// of tiles of one sample; the CTA then adds its partial sums to dw / db with
// atomics.  Bounded waits as in the forward kernel.
struct WgradMmaArgs {
  const float* x;    // [B][Cin][H][W]
  const float* dy;   // [B][Cout][H][W]
  float* dw;         // [Cout][Cin][3][3], accumulated into
  float* db;         // [Cout], accumulated into
  int B, Cin, Cout, H, W;
  int nn;            // Cout rounded up to a multiple of 16
  int mpad;          // 9 Cin + 1 rounded up to a multiple of 128
  int tiles_per_cta;
  int* status;
};

static size_t wgrad_mma_smem(int mpad, int nn) {
  return (size_t)mpad * kConvM * 2 + (size_t)nn * kConvM * 2 + 9 * kConvM * sizeof(int) + 16;
}

__global__ void __launch_bounds__(kConvMmaThreads) conv3x3_wgrad_mma_kernel(const WgradMmaArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* As = smem;                                  // [16 pixel chunks][mpad rows][16 B]
  uint8_t* Bs = As + (size_t)a.mpad * kConvM * 2;      // [16 pixel chunks][nn rows][16 B]
  int* soff = reinterpret_cast<int*>(Bs + (size_t)a.nn * kConvM * 2);   // [9 taps][128 pixels]
  uint64_t* bar = reinterpret_cast<uint64_t*>(soff + 9 * kConvM);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b = blockIdx.y;
  const int64_t HW = (int64_t)a.H * a.W;
  const int mtiles = a.mpad / kConvM;
  const int rows9 = 9 * a.Cin;
  int cols = 32;
  while (cols < mtiles * a.nn) cols *= 2;
  if (tid == 0) {
    mbar_init(smem_u32(bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t idesc = idesc_bf16(kConvM, a.nn, 0);
  const int64_t tpi = (HW + kConvM - 1) / kConvM;
  const float* xb = a.x + (int64_t)b * a.Cin * HW;
  const float* dyb = a.dy + (int64_t)b * a.Cout * HW;
  uint32_t parity = 0;
  bool ok = true;
  int done = 0;
  for (int k = 0; k < a.tiles_per_cta; ++k) {
    const int64_t tile = (int64_t)blockIdx.x * a.tiles_per_cta + k;
    if (tile >= tpi) break;
    const int64_t p0 = tile * kConvM;
    // source offset of each pixel of the tile under each tap (circular
    // neighbours), -1 past the image
    {
      const int64_t p = p0 + tid;
      const int pi = p < HW ? (int)(p / a.W) : 0, pj = p < HW ? (int)(p - (int64_t)pi * a.W) : 0;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int si = (pi + t / 3 - 1 + a.H) % a.H, sj = (pj + t % 3 - 1 + a.W) % a.W;
        soff[t * kConvM + tid] = p < HW ? si * a.W + sj : -1;
      }
    }
    __syncthreads();
    // A rows: eight pixels of one shifted channel (or ones) per 16-byte row
    for (int e = tid; e < a.mpad * 16; e += kConvMmaThreads) {
      const int m = e % a.mpad, kq = e / a.mpad;
      const int64_t pp = p0 + kq * 8;
      float v[8];
      if (m < rows9) {
        const int t = m / a.Cin, ci = m - t * a.Cin;
        const float* xc = xb + (int64_t)ci * HW;
        const int* so = soff + t * kConvM + kq * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int o = so[q];
          v[q] = o >= 0 ? xc[o] : 0.f;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (m == rows9 && pp + q < HW) ? 1.f : 0.f;
      }
      *reinterpret_cast<uint4*>(As + (size_t)e * 16) =
          make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
    for (int e = tid; e < a.nn * 16; e += kConvMmaThreads) {
      const int co = e % a.nn, kq = e / a.nn;
      const int64_t pp = p0 + kq * 8;
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (co < a.Cout && pp + q < HW) ? dyb[(int64_t)co * HW + pp + q] : 0.f;
      *reinterpret_cast<uint4*>(Bs + (size_t)e * 16) =
          make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      for (int mt = 0; mt < mtiles; ++mt)
        for (int kk = 0; kk < kConvM / 16; ++kk) {
          const uint64_t ad = smem_desc(a0 + (uint32_t)(2 * kk * a.mpad + mt * kConvM) * 16, (uint32_t)a.mpad * 16,
                                        128, 0);
          const uint64_t bd = smem_desc(b0 + (uint32_t)(2 * kk * a.nn) * 16, (uint32_t)a.nn * 16, 128, 0);
          mma_bf16(tmem + (uint32_t)(mt * a.nn), ad, bd, idesc, (done > 0 || kk > 0) ? 1u : 0u);
        }
      mma_commit(smem_u32(bar));
    }
    ok = __syncthreads_and(mbar_wait(smem_u32(bar), parity)) != 0;
    parity ^= 1u;
    if (!ok) {
      if (tid == 0 && a.status) atomicOr(a.status, 2);
      break;
    }
    ++done;
  }
  tc_fence_after();
  if (ok && done > 0) {
    const uint32_t lane_addr = static_cast<uint32_t>(warp * 32) << 16;
    for (int mt = 0; mt < mtiles; ++mt) {
      uint32_t r[32];
      tmem_ld16(tmem + lane_addr + (uint32_t)(mt * a.nn), r);
      if (a.nn > 16) tmem_ld16(tmem + lane_addr + (uint32_t)(mt * a.nn + 16), r + 16);
      const int m = mt * kConvM + tid;
      if (m < rows9) {
        const int t = m / a.Cin, ci = m - t * a.Cin;
        for (int co = 0; co < a.Cout; ++co)
          atomicAdd(&a.dw[((int64_t)co * a.Cin + ci) * 9 + t], __uint_as_float(r[co]));
      } else if (m == rows9) {
        for (int co = 0; co < a.Cout; ++co) atomicAdd(&a.db[co], __uint_as_float(r[co]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, cols);
  }
}

cudaError_t launch_wgrad_mma(const float* x, const float* dy, float* dw, float* db, int B, int cin, int cout, int H,
                             int W, int* status, cudaStream_t s) {
  if (cin < 1 || cin > 32 || cout < 1 || cout > 32 || W % 8 != 0) return cudaErrorInvalidValue;
  WgradMmaArgs a{};
  a.x = x;
  a.dy = dy;
  a.dw = dw;
  a.db = db;
  a.B = B;
  a.Cin = cin;
  a.Cout = cout;
  a.H = H;
  a.W = W;
  a.nn = (cout + 15) / 16 * 16;
  a.mpad = (9 * cin + 1 + kConvM - 1) / kConvM * kConvM;
  a.status = status;
  const int64_t tpi = ((int64_t)H * W + kConvM - 1) / kConvM;
  // about two CTAs per SM over the batch
  const int64_t per_sample = std::max<int64_t>(1, std::min<int64_t>(tpi, (2 * 152 + B - 1) / B));
  a.tiles_per_cta = (int)((tpi + per_sample - 1) / per_sample);
  const unsigned gx = (unsigned)((tpi + a.tiles_per_cta - 1) / a.tiles_per_cta);
  conv3x3_wgrad_mma_kernel<<<dim3(gx, (unsigned)B), kConvMmaThreads, wgrad_mma_smem(a.mpad, a.nn), s>>>(a);
  return cudaGetLastError();
}

cudaError_t prepare_conv_mma() {
  cudaError_t e = cudaFuncSetAttribute(conv3x3_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)conv_mma_smem(32, 32));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(conv3x3_wgrad_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)wgrad_mma_smem(384, 32));
}

cudaError_t launch_conv_mma(const float* x, const __nv_bfloat16* w, const float* bias, float* y, int B, int cin,
                            int cout, int H, int W, int relu, int* status, cudaStream_t s) {
  if (cin < 1 || cin > 32 || cout < 1 || cout > 32) return cudaErrorInvalidValue;
  ConvMmaArgs a{};
  a.x = x;
  a.w = w;
  a.bias = bias;
  a.y = y;
  a.B = B;
  a.Cin = cin;
  a.Cout = cout;
  a.H = H;
  a.W = W;
  a.relu = relu;
  a.kc = (cin + 15) / 16 * 16;
  a.nn = (cout + 15) / 16 * 16;
  a.status = status;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (int64_t)B * (((int64_t)H * W + kConvM - 1) / kConvM);
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, 2 * (int64_t)sms);
  conv3x3_mma_kernel<<<grid, kConvMmaThreads, conv_mma_smem(a.kc, a.nn), s>>>(a);
  return cudaGetLastError();
}

}  // namespace cgl

extern "C" int cgl_conv3x3(const float* x, const uint16_t* w, const float* bias, float* y, int B, int cin, int cout,
                           int H, int W, int relu, int* status, void* stream) {
  using namespace cgl;
  if (!x || !w || !y) return fail(CGL_EINVAL, "x, w and y must be non-NULL");
  if (B < 1 || H < 1 || W < 1 || cin < 1 || cin > 32 || cout < 1 || cout > 32)
    return fail(CGL_EINVAL, "need B, H, W >= 1 and 1 <= Cin, Cout <= 32");
  cudaError_t e = prepare_conv_mma();
  if (e == cudaSuccess)
    e = launch_conv_mma(x, reinterpret_cast<const __nv_bfloat16*>(w), bias, y, B, cin, cout, H, W, relu, status,
                        (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(CGL_ECUDA, std::string("conv3x3: ") + cudaGetErrorString(e));
  return CGL_OK;
}
