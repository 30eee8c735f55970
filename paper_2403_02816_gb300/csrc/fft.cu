// Periodic linear flow exp(c tau K) u = F^{-1}(E .* F u) (Sec. 3.2) as
// pencil passes: one kernel launch transforms every pencil along one axis.
//
// A CTA owns up to kTile/n whole pencils.  It loads them (coalesced, applying
// the sweep's nonlinear prologue on the first pass), runs a Stockham
// autosort FFT in shared memory (one radix-2 stage when log2 n is odd, then
// radix-4 stages; each thread keeps its butterflies in registers between the
// read and the write half of a stage), optionally multiplies by the
// separable Fourier symbol and runs the inverse FFT (last axis), and stores
// (applying the sweep's epilogue on the last pass).  The forward transform is
// unnormalised; the 1/N of the inverse is folded into the symbol vectors.
#include "cgl_internal.cuh"

namespace cgl {

constexpr int kFftThreads = 256;
constexpr int kFftTile = 2048;  // complex elements of one field per CTA (8 per thread)
constexpr int kFftMaxSmem = 200 * 1024;

template <class T2, int R> __device__ __forceinline__ void dft_small(T2* x, bool inv);

template <class T2> __device__ __forceinline__ void dft2(T2* x) {
  const T2 a = x[0], b = x[1];
  x[0] = cadd(a, b);
  x[1] = csub(a, b);
}

// y_k = sum_r x_r exp(-+ 2 pi i r k / 4)
template <class T2> __device__ __forceinline__ void dft4(T2* x, bool inv) {
  const T2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
  const T2 s13 = cadd(x[1], x[3]), d13 = csub(x[1], x[3]);
  // -i*d13 (forward) or +i*d13 (inverse)
  const T2 rot = inv ? mk<T2>(-d13.y, d13.x) : mk<T2>(d13.y, -d13.x);
  x[0] = cadd(s02, s13);
  x[2] = csub(s02, s13);
  x[1] = cadd(d02, rot);
  x[3] = csub(d02, rot);
}

// One Stockham stage of radix R on `tb` pencils of length n stored with
// pitch `pitch` in s.  p = product of the radices already applied.
// Butterfly i of a pencil (k = i mod p) reads x_r = s[i + r n/R],
// multiplies by exp(-+2 pi i r k/(pR)), does a length-R DFT and writes
// s[(i-k)R + k + r p].
template <class T2, int R>
__device__ __forceinline__ void fft_stage(T2* s, int pitch, int n, int lognb, int tb, int p,
                                          const T2* tw, bool inv) {
  constexpr int BPT = 8 / R;
  const int nb = n / R;
  const int total = tb * nb;
  const int twstride = n / (p * R);
  T2 v[BPT][R];
  int dst[BPT];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int q = threadIdx.x + b * kFftThreads;
    dst[b] = -1;
    if (q < total) {
      const int t = q >> lognb;
      const int i = q & (nb - 1);
      const int k = i & (p - 1);
      const T2* src = s + t * pitch + i;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = src[r * nb];
      if (p > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const T2 w = tw[r * k * twstride];
          v[b][r] = inv ? cmulc(v[b][r], w) : cmul(v[b][r], w);
        }
      }
      if (R == 2) dft2(v[b]);
      else dft4(v[b], inv);
      dst[b] = t * pitch + (i - k) * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    if (dst[b] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[dst[b] + r * p] = v[b][r];
    }
  }
  __syncthreads();
}

template <class T2>
__device__ void fft_tile(T2* s, int pitch, int n, int logn, int tb, const T2* tw, bool inv) {
  int p = 1;
  if (logn & 1) {
    fft_stage<T2, 2>(s, pitch, n, logn - 1, tb, p, tw, inv);
    p = 2;
  }
  while (p < n) {
    fft_stage<T2, 4>(s, pitch, n, logn - 2, tb, p, tw, inv);
    p *= 4;
  }
}

template <class T2> __device__ __forceinline__ T2 ldf(const void* base, int64_t off) {
  return reinterpret_cast<const T2*>(base)[off];
}
template <class T2> __device__ __forceinline__ void stf(void* base, int64_t off, T2 v) {
  reinterpret_cast<T2*>(base)[off] = v;
}

template <class T>
__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(const FftPassArgs a) {
  using T2 = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = (int)a.g.n_ax;
  const int logn = __ffs(n) - 1;
  const int tbmax = max(1, kFftTile / n);
  const int pitch = n + 1;
  const int64_t b0 = (int64_t)blockIdx.x * tbmax;
  const int tb = (int)min((int64_t)tbmax, a.g.npencils - b0);
  const int64_t P = a.g.P;
  const int nrhs = a.f.nrhs;

  T2* tile0 = reinterpret_cast<T2*>(smem_raw);
  T2* tile1 = tile0 + tbmax * pitch;
  T2* tw = tile1 + (nrhs > 1 ? tbmax * pitch : 0);
  T2* pfac = tw + n;                                       // [kMaxRhs][tbmax]
  int64_t* pbase = reinterpret_cast<int64_t*>(pfac + kMaxRhs * tbmax);
  T2* tiles[2] = {tile0, tile1};

  const T2* twg = reinterpret_cast<const T2*>(a.twiddle);
  for (int m = threadIdx.x; m < n; m += kFftThreads) tw[m] = twg[m];
  for (int t = threadIdx.x; t < tb; t += kFftThreads) {
    const int64_t b = b0 + t;
    const int64_t p = b % P, q = b / P;
    pbase[t] = p + P * (int64_t)n * q;
    if (a.flags & PASS_MUL) {
      // indices of the other axes of this pencil
      int64_t kk[3];
      int64_t rem = p;
      for (int mu = 0; mu < a.g.axis; ++mu) { kk[mu] = rem % a.g.n[mu]; rem /= a.g.n[mu]; }
      rem = q;
      for (int mu = a.g.axis + 1; mu < a.g.d; ++mu) { kk[mu] = rem % a.g.n[mu]; rem /= a.g.n[mu]; }
      for (int r = 0; r < nrhs; ++r) {
        const Symbol& S = a.sym[r];
        T2 acc = S.sum_form ? mk<T2>(0, 0) : mk<T2>(1, 0);
        for (int mu = 0; mu < a.g.d; ++mu) {
          if (mu == a.g.axis) continue;
          const T2 v = reinterpret_cast<const T2*>(S.vec[mu])[kk[mu]];
          acc = S.sum_form ? cadd(acc, v) : cmul(acc, v);
        }
        pfac[r * tbmax + t] = acc;
      }
    }
  }
  __syncthreads();

  // ---- load (+ prologue)
  const int cnt = tb * n;
  for (int e = threadIdx.x; e < cnt; e += kFftThreads) {
    int t, j;
    if (P == 1) { t = e >> logn; j = e & (n - 1); }
    else { j = e / tb; t = e - j * tb; }
    const int64_t off = pbase[t] + P * j;
    T2 z[2];
    if (a.flags & PASS_PRO) {
      T2 in[2];
      in[0] = ldf<T2>(a.f.in[0], off);
      in[1] = a.f.nin > 1 ? ldf<T2>(a.f.in[1], off) : in[0];
      apply_prologue<T, T2>(a.op, in, z);
    } else {
      z[0] = ldf<T2>(a.f.work[0], off);
      z[1] = nrhs > 1 ? ldf<T2>(a.f.work[1], off) : z[0];
    }
    tile0[t * pitch + j] = z[0];
    if (nrhs > 1) tile1[t * pitch + j] = z[1];
  }
  __syncthreads();

  // ---- transforms
  for (int r = 0; r < nrhs; ++r) {
    T2* s = tiles[r];
    if (a.flags & PASS_FWD) fft_tile<T2>(s, pitch, n, logn, tb, tw, false);
    if (a.flags & PASS_MUL) {
      const Symbol& S = a.sym[r];
      const T2* va = reinterpret_cast<const T2*>(S.vec[a.g.axis]);
      for (int e = threadIdx.x; e < cnt; e += kFftThreads) {
        const int t = e >> logn, j = e & (n - 1);
        const T2 c = pfac[r * tbmax + t];
        const T2 f = S.sum_form ? cadd(c, va[j]) : cmul(c, va[j]);
        s[t * pitch + j] = cmul(s[t * pitch + j], f);
      }
      __syncthreads();
    }
    if (a.flags & PASS_INV) fft_tile<T2>(s, pitch, n, logn, tb, tw, true);
  }

  // ---- store (+ epilogue)
  bool bad = false;
  for (int e = threadIdx.x; e < cnt; e += kFftThreads) {
    int t, j;
    if (P == 1) { t = e >> logn; j = e & (n - 1); }
    else { j = e / tb; t = e - j * tb; }
    const int64_t off = pbase[t] + P * j;
    T2 y[2];
    y[0] = tile0[t * pitch + j];
    y[1] = nrhs > 1 ? tile1[t * pitch + j] : y[0];
    if (a.flags & PASS_EPI) {
      T2 ex[kMaxExtra], o[2];
      for (int x = 0; x < a.f.nextra; ++x) ex[x] = ldf<T2>(a.f.extra[x], off);
      const int no = apply_epilogue<T, T2>(a.op, y, ex, o);
      for (int x = 0; x < no && x < a.f.nout; ++x) {
        stf<T2>(a.f.out[x], off, o[x]);
        bad |= !finite2(o[x]);
      }
    } else {
      stf<T2>(a.f.work[0], off, y[0]);
      if (nrhs > 1) stf<T2>(a.f.work[1], off, y[1]);
    }
  }
  if (bad && a.status) atomicOr(a.status, 1);
}

static size_t fft_smem_bytes(int n, int nrhs, size_t elem) {
  const int tbmax = std::max(1, kFftTile / n);
  const int pitch = n + 1;
  return (size_t)tbmax * pitch * elem * (nrhs > 1 ? 2 : 1) + (size_t)n * elem +
         (size_t)kMaxRhs * tbmax * elem + (size_t)tbmax * sizeof(int64_t);
}

template <class T> cudaError_t launch_fft_pass(const FftPassArgs& a, cudaStream_t s) {
  using T2 = typename C2<T>::type;
  const int n = (int)a.g.n_ax;
  const int tbmax = std::max(1, kFftTile / n);
  const int64_t grid = (a.g.npencils + tbmax - 1) / tbmax;
  const size_t smem = fft_smem_bytes(n, a.f.nrhs, sizeof(T2));
  fft_pass_kernel<T><<<(unsigned)grid, kFftThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Opt in to large dynamic shared memory; called at plan creation, outside any
// stream capture.
template <class T> cudaError_t prepare_fft_pass() {
  return cudaFuncSetAttribute(fft_pass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem);
}

template cudaError_t prepare_fft_pass<double>();
template cudaError_t prepare_fft_pass<float>();
template cudaError_t launch_fft_pass<double>(const FftPassArgs&, cudaStream_t);
template cudaError_t launch_fft_pass<float>(const FftPassArgs&, cudaStream_t);

}  // namespace cgl
