// K x for finite-difference directions as a stencil (Sec. 3.1, eq. kronsumv:
// K u = vec(sum_mu U x_mu A_mu)), fused with a Runge-Kutta stage epilogue,
// for eq. RK4 / eq. RK2 on Dirichlet/Neumann grids.
//
// A_mu = (a1 + i b1) D2_mu + (a2/d) I with the 2nd-order matrices of the plan
// (Dirichlet: interior nodes, h = L/(n+1), tridiag(1, -2, 1)/h^2; Neumann:
// both boundary nodes, h = L/(n-1), first row (-2, 2)/h^2, last (2, -2)/h^2),
// so at grid point j
//   (K x)_j = sum_mu c_mu (w_l x_{j - e_mu} - 2 x_j + w_r x_{j + e_mu}) + a2 x_j,
// c_mu = (a1 + i b1)/h_mu^2, neighbours outside the grid taken as zero and the
// Neumann ghost reflection giving w = 2 on the inward neighbour of a
// boundary node.  One thread per grid point along the contiguous direction,
// grid y / z over directions 2 / 3; every read is a coalesced load of the
// stage argument (neighbours come from L1/L2), so the kernel is bound by
// HBM traffic: the stage argument, the extra inputs of the epilogue and its
// outputs.  The output buffers must differ from x (neighbours are read).
#include "cgl_internal.cuh"

namespace cgl {

constexpr int kStencilThreads = 256;

template <class T>
__global__ void __launch_bounds__(kStencilThreads) kron_stencil_kernel(const StencilArgs a) {
  using T2 = typename C2<T>::type;
  const int n0 = (int)a.n[0];
  const int j0 = blockIdx.x * kStencilThreads + threadIdx.x;
  if (j0 >= n0) return;
  const int j1 = blockIdx.y, j2 = blockIdx.z;
  const int64_t i = j0 + a.n[0] * (j1 + a.n[1] * (int64_t)j2);
  const T2* x = reinterpret_cast<const T2*>(a.x);
  const T2 xc = x[i];
  const int jj[3] = {j0, j1, j2};
  T lr = 0, li = 0;  // sum_mu c_mu * second difference
  int64_t stride = 1;
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    if (mu < a.d) {
      const int nm = (int)a.n[mu], jm = jj[mu];
      const T2 l = jm > 0 ? x[i - stride] : mk<T2>(0, 0);
      const T2 r = jm < nm - 1 ? x[i + stride] : mk<T2>(0, 0);
      T wl = 1, wr = 1;
      if (a.bc[mu] == CGL_BC_NEUMANN) {
        if (jm == 0) wr = 2;
        if (jm == nm - 1) wl = 2;
      }
      const T dr = fma(wl, l.x, fma(wr, r.x, T(-2) * xc.x));
      const T di = fma(wl, l.y, fma(wr, r.y, T(-2) * xc.y));
      const T cr = pv<T>(a.cr[mu], a.crf[mu]), ci = pv<T>(a.ci[mu], a.cif[mu]);
      lr = fma(cr, dr, fma(-ci, di, lr));
      li = fma(cr, di, fma(ci, dr, li));
      stride *= a.n[mu];
    }
  }
  const T a2 = pv<T>(a.a2, a.a2f);
  T2 y[2];
  y[0] = mk<T2>(fma(a2, xc.x, lr), fma(a2, xc.y, li));
  y[1] = y[0];
  T2 ex[kMaxExtra], o[2];
#pragma unroll
  for (int e = 0; e < kMaxExtra; ++e)
    if (e < a.nextra) ex[e] = reinterpret_cast<const T2*>(a.extra[e])[i];
  const int no = apply_epilogue<T, T2>(a.op, y, ex, o);
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (k < no && k < a.nout) {
      reinterpret_cast<T2*>(a.out[k])[i] = o[k];
      bad |= !finite2(o[k]);
    }
  }
  if (bad && a.status) atomicOr(a.status, 1);
}

template <class T> cudaError_t launch_kron_stencil(const StencilArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)((a.n[0] + kStencilThreads - 1) / kStencilThreads), (unsigned)a.n[1], (unsigned)a.n[2]);
  kron_stencil_kernel<T><<<grid, kStencilThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_kron_stencil<double>(const StencilArgs&, cudaStream_t);
template cudaError_t launch_kron_stencil<float>(const StencilArgs&, cudaStream_t);

}  // namespace cgl
