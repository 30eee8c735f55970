// mu-mode product pass (Sec. 3.1): V = U x_mu F, i.e. for every fiber along
// axis mu, v_i = sum_j F_{ij} u_j with the dense n x n complex factor
// F = exp(c tau A_mu).  A chain of d passes is the Tucker operator
// (eq. Tucker).  SIMT kernel for FP64 (parity path) and FP32.
//
// A CTA owns `tb` whole fibers of every right-hand side: it loads them into
// shared memory (applying the sweep's prologue on the first pass), then each
// thread accumulates a 4-wide register block of outputs for both right-hand
// sides and applies the sweep's epilogue before storing.  Two thread
// mappings keep global accesses coalesced:
//   mode 1 (P == 1, fibers contiguous): consecutive threads take consecutive
//     rows i (F read column-major, coalesced); block = 4 fibers.
//   other modes (P > 1, fibers strided): consecutive threads take consecutive
//     fibers t (outputs of one row i are adjacent in memory); block = 4 rows,
//     whose factor entries are a broadcast load.
#include <algorithm>

#include "cgl_internal.cuh"

namespace cgl {

constexpr int kModeThreads = 256;
constexpr int kModeMaxSmem = 96 * 1024;

// Field loads go to L2 (each value is read once per pass; in the batched
// step kernel, values another CTA wrote earlier in the same launch must not
// come from a stale L1 line).
template <class T2> __device__ __forceinline__ T2 ldm(const void* base, int64_t off) {
  return __ldcg(reinterpret_cast<const T2*>(base) + off);
}

// acc += f * z
template <class T2> __device__ __forceinline__ void cmac(T2& acc, T2 f, T2 z) {
  acc.x = fma(f.x, z.x, acc.x);
  acc.x = fma(-f.y, z.y, acc.x);
  acc.y = fma(f.x, z.y, acc.y);
  acc.y = fma(f.y, z.x, acc.y);
}

template <class T>
__device__ __forceinline__ void finish_point(const ModePassArgs& a, typename C2<T>::type* y, int64_t off,
                                             bool& bad) {
  using T2 = typename C2<T>::type;
  if (a.flags & PASS_EPI) {
    T2 ex[kMaxExtra], o[2];
    for (int x = 0; x < a.f.nextra; ++x) ex[x] = ldm<T2>(a.f.extra[x], off);
    const int no = apply_epilogue<T, T2>(a.op, y, ex, o);
    for (int x = 0; x < no && x < a.f.nout; ++x) {
      reinterpret_cast<T2*>(a.f.out[x])[off] = o[x];
      bad |= !finite2(o[x]);
    }
  } else {
    reinterpret_cast<T2*>(a.f.work[0])[off] = y[0];
    if (a.f.nrhs > 1) reinterpret_cast<T2*>(a.f.work[1])[off] = y[1];
  }
}

// One tile: fibers b0 .. b0+tbmax-1 (clipped) of the pass described by `a`,
// using `smem_raw` (tbmax * (n+1) * NRHS values + tbmax offsets).
template <class T, int NRHS>
__device__ __forceinline__ void mode_tile(const ModePassArgs& a, int tbmax, int64_t b0, unsigned char* smem_raw) {
  using T2 = typename C2<T>::type;
  const int n = (int)a.g.n_ax;
  const int pitch = n + 1;
  const int64_t P = a.g.P;
  const int tb = (int)min((int64_t)tbmax, a.g.npencils - b0);

  T2* Z0 = reinterpret_cast<T2*>(smem_raw);
  T2* Z1 = Z0 + tbmax * pitch;
  int64_t* pbase = reinterpret_cast<int64_t*>(Z0 + NRHS * tbmax * pitch);

  for (int t = threadIdx.x; t < tb; t += kModeThreads) {
    const int64_t b = b0 + t;
    pbase[t] = (b % P) + P * (int64_t)n * (b / P);
  }
  __syncthreads();

  // ---- load (+ prologue)
  const int cnt = tb * n;
  for (int e = threadIdx.x; e < cnt; e += kModeThreads) {
    int t, j;
    if (P == 1) { t = e / n; j = e - t * n; }
    else { j = e / tb; t = e - j * tb; }
    const int64_t off = pbase[t] + P * j;
    T2 z[2];
    if (a.flags & PASS_PRO) {
      T2 in[2];
      in[0] = ldm<T2>(a.f.in[0], off);
      in[1] = a.f.nin > 1 ? ldm<T2>(a.f.in[1], off) : in[0];
      apply_prologue<T, T2>(a.op, in, z);
    } else {
      z[0] = ldm<T2>(a.f.work[0], off);
      if (NRHS > 1) z[1] = ldm<T2>(a.f.work[1], off);
    }
    Z0[t * pitch + j] = z[0];
    if (NRHS > 1) Z1[t * pitch + j] = z[1];
  }
  __syncthreads();

  const T2* F0 = reinterpret_cast<const T2*>(a.factor[0]);
  const T2* F1 = reinterpret_cast<const T2*>(a.factor[NRHS > 1 ? 1 : 0]);
  bool bad = false;

  if constexpr (sizeof(T) == 4) {
    // FP32: 4 rows x 4 fibers per thread and right-hand side, so each factor
    // load (4 consecutive rows, two 16-byte loads) and each fiber value feed
    // 16 complex multiply-adds.  Consecutive threads take consecutive row
    // blocks for contiguous fibers (P == 1) and consecutive fiber blocks
    // otherwise, which keeps the epilogue's stores coalesced.
    const int ni = (n + 3) / 4, nt = (tb + 3) / 4;
    const int items = ni * nt;
    for (int w = threadIdx.x; w < items; w += kModeThreads) {
      int ig, tg;
      if (P == 1) { tg = w / ni; ig = w - tg * ni; }
      else { ig = w / nt; tg = w - ig * nt; }
      const int i0 = ig * 4, t0 = tg * 4;
      const int ilim = min(4, n - i0), tlim = min(4, tb - t0);
      T2 acc0[4][4], acc1[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) { acc0[u][v] = mk<T2>(0, 0); acc1[u][v] = mk<T2>(0, 0); }
      const bool full_i = (ilim == 4) && ((n & 1) == 0);
      for (int j = 0; j < n; ++j) {
        T2 f0[4], f1[4], z0[4], z1[4];
        const T2* c0 = F0 + i0 + (int64_t)j * n;
        const T2* c1 = F1 + i0 + (int64_t)j * n;
        if (full_i) {
          const float4 a01 = __ldg(reinterpret_cast<const float4*>(c0));
          const float4 a23 = __ldg(reinterpret_cast<const float4*>(c0) + 1);
          f0[0] = mk<T2>(a01.x, a01.y); f0[1] = mk<T2>(a01.z, a01.w);
          f0[2] = mk<T2>(a23.x, a23.y); f0[3] = mk<T2>(a23.z, a23.w);
          if (NRHS > 1) {
            const float4 b01 = __ldg(reinterpret_cast<const float4*>(c1));
            const float4 b23 = __ldg(reinterpret_cast<const float4*>(c1) + 1);
            f1[0] = mk<T2>(b01.x, b01.y); f1[1] = mk<T2>(b01.z, b01.w);
            f1[2] = mk<T2>(b23.x, b23.y); f1[3] = mk<T2>(b23.z, b23.w);
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            f0[u] = u < ilim ? c0[u] : mk<T2>(0, 0);
            if (NRHS > 1) f1[u] = u < ilim ? c1[u] : mk<T2>(0, 0);
          }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int t = min(t0 + v, tb - 1);
          z0[v] = Z0[t * pitch + j];
          if (NRHS > 1) z1[v] = Z1[t * pitch + j];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            cmac(acc0[u][v], f0[u], z0[v]);
            if (NRHS > 1) cmac(acc1[u][v], f1[u], z1[v]);
          }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (v >= tlim) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u >= ilim) continue;
          T2 y[2] = {acc0[u][v], acc1[u][v]};
          finish_point<T>(a, y, pbase[t0 + v] + P * (i0 + u), bad);
        }
      }
    }
  } else if (P == 1) {
    // rows i fast, 4 fibers per thread
    const int tgroups = (tb + 3) / 4;
    const int items = n * tgroups;
    for (int w = threadIdx.x; w < items; w += kModeThreads) {
      const int tg = w / n;
      const int i = w - tg * n;
      const int t0 = tg * 4;
      T2 acc0[4], acc1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { acc0[u] = mk<T2>(0, 0); acc1[u] = mk<T2>(0, 0); }
      const int tlim = min(4, tb - t0);
      for (int j = 0; j < n; ++j) {
        const T2 f0 = F0[i + (int64_t)j * n];
        const T2 f1 = NRHS > 1 ? F1[i + (int64_t)j * n] : f0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < tlim) {
            cmac(acc0[u], f0, Z0[(t0 + u) * pitch + j]);
            if (NRHS > 1) cmac(acc1[u], f1, Z1[(t0 + u) * pitch + j]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u < tlim) {
          T2 y[2] = {acc0[u], acc1[u]};
          finish_point<T>(a, y, pbase[t0 + u] + i, bad);
        }
      }
    }
  } else {
    // fibers t fast, 4 rows per thread
    const int igroups = (n + 3) / 4;
    const int items = tb * igroups;
    for (int w = threadIdx.x; w < items; w += kModeThreads) {
      const int ig = w / tb;
      const int t = w - ig * tb;
      const int i0 = ig * 4;
      const int ilim = min(4, n - i0);
      T2 acc0[4], acc1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { acc0[u] = mk<T2>(0, 0); acc1[u] = mk<T2>(0, 0); }
      for (int j = 0; j < n; ++j) {
        const T2 z0 = Z0[t * pitch + j];
        const T2 z1 = NRHS > 1 ? Z1[t * pitch + j] : z0;
        const T2* c0 = F0 + i0 + (int64_t)j * n;
        const T2* c1 = F1 + i0 + (int64_t)j * n;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < ilim) {
            cmac(acc0[u], c0[u], z0);
            if (NRHS > 1) cmac(acc1[u], c1[u], z1);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u < ilim) {
          T2 y[2] = {acc0[u], acc1[u]};
          finish_point<T>(a, y, pbase[t] + P * (i0 + u), bad);
        }
      }
    }
  }
  if (bad && a.status) atomicOr(a.status, 1);
}

template <class T, int NRHS>
__global__ void __launch_bounds__(kModeThreads) mode_pass_kernel(const ModePassArgs a, int tbmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mode_tile<T, NRHS>(a, tbmax, (int64_t)blockIdx.x * tbmax, smem_raw);
}

// Polls of a dependency wait (with a 128 ns sleep each) before the step
// kernel gives up: about half a second.

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One persistent launch per time step of a batch: CTAs claim items of the
// pass-major list through counter[0]; an item waits (thread 0, bounded) for
// done[prev pass][instance] to reach that pass's item count for the
// instance, runs the tile, and after a device-wide fence counts itself in
// done[pass][instance].  Items are claimed in list order and only wait on
// earlier items, which running CTAs hold, so the launch always progresses.
// A wait that gives up sets bit 1 of *status and counter[1]; every CTA then
// stops at its next claim.
template <class T>
__global__ void __launch_bounds__(kModeThreads) batched_step_kernel(const StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item, s_go;
  int* abort_flag = a.counter + 1;
  int* done = a.counter + 2;
  for (;;) {
    if (threadIdx.x == 0) {
      s_go = ld_acquire(abort_flag) == 0;
      s_item = s_go ? atomicAdd(a.counter, 1) : a.nitems;
      if (s_go && s_item < a.nitems) {
        const StepItem it = a.items[s_item];
        const int pk = a.prev[it.pass * a.count + it.inst];
        if (pk >= 0) {
          const int* d = done + pk * a.count + it.inst;
          const int want = a.need[pk * a.count + it.inst] + a.want_bias;
          long long spins = 0;
          while (ld_acquire(d) < want) {
            if (++spins > a.spin_limit || ld_acquire(abort_flag)) {
              s_go = 0;
              break;
            }
            __nanosleep(128);
          }
          if (!s_go) {
            atomicOr(a.status, 2);
            atomicExch(abort_flag, 1);
          }
        }
      }
      __threadfence();
    }
    __syncthreads();
    const int it = s_item, go = s_go;
    __syncthreads();
    if (!go || it >= a.nitems) break;
    const StepItem si = a.items[it];
    const ModePassArgs pa = a.table[si.pass * a.count + si.inst];
    if (pa.f.nrhs > 1) mode_tile<T, 2>(pa, si.tb, si.b0, smem_raw);
    else mode_tile<T, 1>(pa, si.tb, si.b0, smem_raw);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(done + si.pass * a.count + si.inst, 1);
  }
}

template <class T> cudaError_t launch_batched_step(const StepArgs& a, size_t smem, int grid, cudaStream_t s) {
  batched_step_kernel<T><<<grid, kModeThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class T> int batched_step_blocks_per_sm(size_t smem) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batched_step_kernel<T>, kModeThreads, smem);
  return std::max(b, 1);
}

static int mode_tb(int n, int nrhs, size_t elem, int64_t npencils) {
  const size_t per = (size_t)(n + 1) * elem * nrhs + sizeof(int64_t);
  int tb = (int)std::min<size_t>(16, kModeMaxSmem / per);
  tb = std::max(tb, 1);
  return (int)std::min<int64_t>(tb, npencils);
}

int mode_tb_max(int n, int nrhs, size_t elem) {
  const size_t per = (size_t)(n + 1) * elem * nrhs + sizeof(int64_t);
  return std::max<int>(1, (int)(kModeMaxSmem / per));
}

size_t mode_smem_bytes(int n, int nrhs, size_t elem, int tb) {
  return (size_t)tb * (n + 1) * elem * nrhs + (size_t)tb * sizeof(int64_t);
}

template <class T> cudaError_t launch_mode_pass_tb(const ModePassArgs& a, int tb, cudaStream_t s) {
  using T2 = typename C2<T>::type;
  const int n = (int)a.g.n_ax;
  const int nrhs = a.f.nrhs;
  tb = (int)std::min<int64_t>(std::max(tb, 1), a.g.npencils);
  const int64_t grid = (a.g.npencils + tb - 1) / tb;
  const size_t smem = mode_smem_bytes(n, nrhs, sizeof(T2), tb);
  if (nrhs > 1)
    mode_pass_kernel<T, 2><<<(unsigned)grid, kModeThreads, smem, s>>>(a, tb);
  else
    mode_pass_kernel<T, 1><<<(unsigned)grid, kModeThreads, smem, s>>>(a, tb);
  return cudaGetLastError();
}

template <class T> cudaError_t launch_mode_pass(const ModePassArgs& a, cudaStream_t s) {
  using T2 = typename C2<T>::type;
  const int n = (int)a.g.n_ax;
  const int nrhs = a.f.nrhs;
  const int tb = mode_tb(n, nrhs, sizeof(T2), a.g.npencils);
  const int64_t grid = (a.g.npencils + tb - 1) / tb;
  const size_t smem = (size_t)tb * (n + 1) * sizeof(T2) * nrhs + (size_t)tb * sizeof(int64_t);
  if (nrhs > 1)
    mode_pass_kernel<T, 2><<<(unsigned)grid, kModeThreads, smem, s>>>(a, tb);
  else
    mode_pass_kernel<T, 1><<<(unsigned)grid, kModeThreads, smem, s>>>(a, tb);
  return cudaGetLastError();
}

// Opt in to large dynamic shared memory; called at plan creation, outside any
// stream capture.
template <class T> cudaError_t prepare_mode_pass() {
  cudaError_t e = cudaFuncSetAttribute(mode_pass_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kModeMaxSmem + 4096);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mode_pass_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kModeMaxSmem + 4096);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(batched_step_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kModeMaxSmem + 4096);
}

template cudaError_t prepare_mode_pass<double>();
template cudaError_t prepare_mode_pass<float>();
template cudaError_t launch_mode_pass_tb<double>(const ModePassArgs&, int, cudaStream_t);
template cudaError_t launch_mode_pass_tb<float>(const ModePassArgs&, int, cudaStream_t);
template cudaError_t launch_batched_step<double>(const StepArgs&, size_t, int, cudaStream_t);
template cudaError_t launch_batched_step<float>(const StepArgs&, size_t, int, cudaStream_t);
template int batched_step_blocks_per_sm<double>(size_t);
template int batched_step_blocks_per_sm<float>(size_t);

template cudaError_t launch_mode_pass<double>(const ModePassArgs&, cudaStream_t);
template cudaError_t launch_mode_pass<float>(const ModePassArgs&, cudaStream_t);

}  // namespace cgl
