// One-time FP64 precompute on the GPU (Sec. 3.1: the small exponentials are
// computed once for a constant step; Sec. 3.2: the tensor E).
//
// expm_device: exp(X) for an n x n complex matrix X = scale * A by truncated
// Taylor series with scaling and squaring (Moler & Van Loan, "Nineteen
// dubious ways to compute the exponential of a matrix", 2003, method 3; the
// paper lists Taylor approximations beside Pade for this step):
//   s = max(0, ceil(log2(||X||_1 / theta))),  Y = X / 2^s,
//   T_m(Y) = I + Y (I + Y/2 (I + Y/3 ( ... (I + Y/m)))),  exp(X) = T_m(Y)^(2^s).
// With theta = 1/2 and m = 18 the truncation term ||Y||^19/19! < 2e-23
// relative, far below FP64 rounding.
#include <cmath>

#include "cgl_internal.cuh"

namespace cgl {

constexpr int kExpmTaylorDegree = 18;
constexpr double kExpmTheta = 0.5;
constexpr int kGemmTile = 16;

// C = alpha * (A @ B) + (add_identity ? I : 0), all n x n column-major complex.
__global__ void zgemm_kernel(const double2* __restrict__ A, const double2* __restrict__ B,
                             double2* __restrict__ C, int n, double alpha, int add_identity) {
  __shared__ double2 As[kGemmTile][kGemmTile + 1];
  __shared__ double2 Bs[kGemmTile][kGemmTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * kGemmTile + ty;
  const int col = blockIdx.x * kGemmTile + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < n; k0 += kGemmTile) {
    // As[ty][tx] = A[row, k0 + tx]; Bs[ty][tx] = B[k0 + ty, col]
    const int ka = k0 + tx, kb = k0 + ty;
    As[ty][tx] = (row < n && ka < n) ? A[row + (int64_t)ka * n] : make_double2(0.0, 0.0);
    Bs[ty][tx] = (kb < n && col < n) ? B[kb + (int64_t)col * n] : make_double2(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGemmTile; ++k) {
      const double2 a = As[ty][k], b = Bs[k][tx];
      acc.x = fma(a.x, b.x, acc.x);
      acc.x = fma(-a.y, b.y, acc.x);
      acc.y = fma(a.x, b.y, acc.y);
      acc.y = fma(a.y, b.x, acc.y);
    }
    __syncthreads();
  }
  if (row < n && col < n) {
    double2 v = make_double2(alpha * acc.x, alpha * acc.y);
    if (add_identity && row == col) v.x += 1.0;
    C[row + (int64_t)col * n] = v;
  }
}

// Y = scale * A ; T = I + Y / m
__global__ void expm_init_kernel(const double2* A, double scale, int n, int m, double2* Y, double2* T) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int row = (int)(idx % n), col = (int)(idx / n);
  const double2 a = A[idx];
  const double2 y = make_double2(scale * a.x, scale * a.y);
  Y[idx] = y;
  double2 t = make_double2(y.x / m, y.y / m);
  if (row == col) t.x += 1.0;
  T[idx] = t;
}

static cudaError_t zgemm(const double2* A, const double2* B, double2* C, int n, double alpha, int add_id,
                         cudaStream_t s) {
  dim3 blk(kGemmTile, kGemmTile);
  dim3 grd((n + kGemmTile - 1) / kGemmTile, (n + kGemmTile - 1) / kGemmTile);
  zgemm_kernel<<<grd, blk, 0, s>>>(A, B, C, n, alpha, add_id);
  return cudaGetLastError();
}

cudaError_t expm_device(const double2* dA, double scale, int n, double2* dOut, double2* work,
                        double norm1, cudaStream_t s) {
  // work: Y | T0 | T1
  double2* Y = work;
  double2* T0 = work + (int64_t)n * n;
  double2* T1 = work + 2 * (int64_t)n * n;
  const double xnorm = std::fabs(scale) * norm1;
  int sq = 0;
  if (xnorm > kExpmTheta) sq = (int)std::ceil(std::log2(xnorm / kExpmTheta));
  const double ys = scale / std::ldexp(1.0, sq);
  const int m = kExpmTaylorDegree;
  const int64_t nn = (int64_t)n * n;
  expm_init_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(dA, ys, n, m, Y, T0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Horner: T <- I + (Y T) / k, k = m-1 .. 1
  double2* cur = T0;
  double2* nxt = T1;
  for (int k = m - 1; k >= 1; --k) {
    if ((e = zgemm(Y, cur, nxt, n, 1.0 / k, 1, s)) != cudaSuccess) return e;
    std::swap(cur, nxt);
  }
  // squaring
  for (int i = 0; i < sq; ++i) {
    if ((e = zgemm(cur, cur, nxt, n, 1.0, 0, s)) != cudaSuccess) return e;
    std::swap(cur, nxt);
  }
  return cudaMemcpyAsync(dOut, cur, nn * sizeof(double2), cudaMemcpyDeviceToDevice, s);
}

// Fourier symbol of one periodic direction (Sec. 3.2), FFT order
// m = 0..ceil(n/2)-1, then the negative frequencies, kappa = 2 pi m / L:
//   sum_form = 0: exp(ctau * ((ar + i ai)(-kappa^2) + beta + i adv kappa')) * post
//   sum_form = 1: ((ar + i ai)(-kappa^2) + beta + i adv kappa') * post
// kappa' = kappa except at the Nyquist mode of an even n, where the first
// derivative's symbol is 0 (adv: the advection speed of eq. (coupled) on its
// direction, 0 elsewhere).
__global__ void periodic_symbol_kernel(double2* out, int n, double L, double ctau, double ar, double ai,
                                       double beta, double adv, double post, int sum_form) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int m = (k <= (n - 1) / 2) ? k : k - n;
  const double kap = 2.0 * M_PI * (double)m / L;
  const double k2 = kap * kap;
  const double k1 = (2 * k == n) ? 0.0 : kap;
  const double re = -ar * k2 + beta;
  const double im = -ai * k2 + adv * k1;
  if (sum_form) {
    out[k] = make_double2(re * post, im * post);
  } else {
    const double mag = exp(ctau * re) * post;
    double sn, cs;
    sincos(ctau * im, &sn, &cs);
    out[k] = make_double2(mag * cs, mag * sn);
  }
}

cudaError_t periodic_symbol_device(double2* dOut, int n, double L, double ctau, double ar, double ai,
                                   double beta, double adv, double post, int sum_form, cudaStream_t s) {
  periodic_symbol_kernel<<<(n + 127) / 128, 128, 0, s>>>(dOut, n, L, ctau, ar, ai, beta, adv, post, sum_form);
  return cudaGetLastError();
}

// Plain twiddles exp(-+2 pi i m / n) (forward table, then inverse), for the
// mixed-radix passes: T2 tab[2][n].
template <class T2> __global__ void plain_twiddle_kernel(T2* tab, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double sn, cs;
  sincospi(2.0 * (double)m / (double)n, &sn, &cs);
  tab[m].x = cs;
  tab[m].y = -sn;
  tab[n + m].x = cs;
  tab[n + m].y = sn;
}

cudaError_t plain_twiddles_device(void* tab, int n, int f64, cudaStream_t s) {
  if (f64) plain_twiddle_kernel<double2><<<(n + 127) / 128, 128, 0, s>>>((double2*)tab, n);
  else plain_twiddle_kernel<float2><<<(n + 127) / 128, 128, 0, s>>>((float2*)tab, n);
  return cudaGetLastError();
}

// Twiddles w = exp(-+2 pi i m / n) = c + i s (forward: s = -sinpi(2m/n);
// inverse: s = +sinpi(2m/n)), stored for the FMA butterfly a +- w b:
//   form 0 (|c| >= |s|): w b = c ((b.x - tau b.y) + i (b.y + tau b.x)), tau = s/c
//   form 1 (|c| <  |s|): w b = s (-(b.y + tau b.x) + i (b.x - tau b.y)), tau = -c/s
// so both forms share u = b.x - tau b.y, v = b.y + tau b.x with |tau| <= 1.
template <class T> __global__ void fma_twiddle_kernel(T* tab, int* form, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double sn, cs;
  sincospi(2.0 * (double)m / (double)n, &sn, &cs);
  for (int dir = 0; dir < 2; ++dir) {
    const double c = cs, s = dir ? sn : -sn;
    double tau, mre, mim;
    int f;
    if (fabs(c) >= fabs(s)) { tau = s / c; mre = c; mim = c; f = 0; }
    else { tau = -c / s; mre = -s; mim = s; f = 1; }
    T* e = tab + ((int64_t)dir * n + m) * 3;
    e[0] = (T)tau;
    e[1] = (T)mre;
    e[2] = (T)mim;
    form[dir * n + m] = f;
  }
}

cudaError_t fma_twiddles_device(void* tab, int* form, int n, int f64, cudaStream_t s) {
  if (f64) fma_twiddle_kernel<double><<<(n + 127) / 128, 128, 0, s>>>((double*)tab, form, n);
  else fma_twiddle_kernel<float><<<(n + 127) / 128, 128, 0, s>>>((float*)tab, form, n);
  return cudaGetLastError();
}

__global__ void f64_to_f32_kernel(const double2* src, float2* dst, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

cudaError_t convert_f64_to_f32(const double2* src, float2* dst, int64_t count, cudaStream_t s) {
  f64_to_f32_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

}  // namespace cgl
