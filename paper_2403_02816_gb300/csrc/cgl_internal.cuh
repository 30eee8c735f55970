// Internal declarations shared by the libcgl translation units.
//
// Layout: a field is N complex values (T2 = double2 or float2), index 1
// fastest (the paper's vec(U), Sec. 3.1).  A "pass" works on pencils/fibers
// along one axis mu: pencil b in [0, N/n_mu) has its element j at
//   (b % P) + P*j + P*n_mu*(b / P),   P = n_1*...*n_{mu-1}.
// Each CTA owns whole pencils, so every pass may run in place.
#pragma once

#include <cuda_bf16.h>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cgl.h"

namespace cgl {

constexpr int kMaxRhs = 2;
constexpr int kMaxExtra = 4;

// ---------------------------------------------------------------- complex

template <class T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };

template <class T2> __host__ __device__ __forceinline__ T2 mk(decltype(T2{}.x) re, decltype(T2{}.x) im) {
  T2 r; r.x = re; r.y = im; return r;
}
template <class T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <class T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <class T2, class T> __device__ __forceinline__ T2 cscale(T2 a, T s) { return mk<T2>(a.x * s, a.y * s); }
template <class T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return mk<T2>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <class T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
  return mk<T2>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// a + s*b  (s real)
template <class T2, class T> __device__ __forceinline__ T2 caxpy(T2 a, T s, T2 b) {
  return mk<T2>(fma(s, b.x, a.x), fma(s, b.y, a.y));
}

// ---------------------------------------------------------------- operators

// Prologue: maps the pass inputs (1 or 2 fields) to the fields transformed by
// the linear flow.  Epilogue: maps the transformed fields and extra inputs to
// the outputs.  Both are pointwise and evaluated once per grid point.
enum ProOp : int {
  PRO_NONE = 0,    // z_r = in_r
  PRO_FLOW = 1,    // z0 = phi_{t0}(in0)                              (Strang)
  PRO_FLOW2 = 2,   // z0 = phi_{t0}(in0), z1 = phi_{t1}(in0)           (split4, first sweep)
  PRO_LAW4 = 3,    // z0 = in0, z1 = g(in0)                            (Lawson4, first sweep)
  PRO_LAW2 = 4,    // z0 = in0 + tau g(in0), z1 = in0 + tau/2 g(in0)   (Lawson2)
  PRO_CQ = 5,      // z0 = phi^c_{t0}(phi^q_{t0}(in0))                 (strang_3t)
  PRO_CQ2 = 6,     // z0 = phi^c_{t0}(phi^q_{t0}(in0)), z1 likewise t1 (split4_3t, first sweep)
  PRO_CFLOW = 7,   // (z0, z1) = phi_{t0}(in0, in1): coupled system, u and v (eq. coupled)
  PRO_CG = 8,      // (z0, z1) = g(in0, in1)                           (coupled Lawson4)
  PRO_CLAW2 = 9    // (z0, z1) = (in0, in1) + t0 g(in0, in1)           (coupled Lawson2)
};
enum EpiOp : int {
  EPI_NONE = 0,    // out_r = y_r
  EPI_FLOW = 1,    // out0 = phi_t(y0)                                 (Strang)
  EPI_FLOW2 = 2,   // out0 = phi_t(y0), out1 = phi_t(y1)               (split4, first sweep)
  EPI_SPLIT4 = 3,  // out0 = 4/3 phi_t(y0) - 1/3 e0                    (split4, second sweep)
  EPI_LAW4A = 4,   // (a, b) -> (p, w)                                 (Lawson4, first sweep)
  EPI_LAW4B = 5,   // (q, r) -> r + tau/6 g(q)                         (Lawson4, second sweep)
  EPI_LAW2 = 6,    // (v, w) -> w + tau/2 g(v)                         (Lawson2)
  EPI_RK = 7,      // Runge-Kutta stage, see rk_stage()
  EPI_QC = 8,      // out0 = phi^q_t(phi^c_t(y0))                      (strang_3t)
  EPI_QC2 = 9,     // out0 = phi^q_t(phi^c_t(y0)),                     (split4_3t, first sweep)
                   // out1 = phi^c_{t/2}(phi^q_t(phi^c_{t/2}(y1)))
  EPI_SPLIT4_3T = 10, // out0 = 4/3 phi^q_t(phi^c_t(y0)) - 1/3 e0      (split4_3t, second sweep)
  EPI_CFLOW = 11,     // (out0, out1) = phi_t(y0, y1)                  (coupled system)
  EPI_CSPLIT4 = 12,   // (out0, out1) = 4/3 phi_t(y0, y1) - 1/3 (e0, e1) (coupled split4)
  EPI_CLAW4P = 13,    // b = y, a = e -> p = a + tau g(u3)            (coupled Lawson4)
  EPI_CLAW4W = 14,    // b = y, a = e -> w = a + tau/6 b + tau/3 (g(u2) + g(u3))
  EPI_CLAW4B = 15,    // r = y, q = e -> r + tau/6 g(q)
  EPI_CLAW2 = 16      // w = y, v = e -> w + tau/2 g(v)               (coupled Lawson2)
};

// Nonlinear model parameters (eq. 1) and the per-pass operator constants.
struct NlParams {
  double a3, b3, a4, b4;
  int cubic;       // a4 = b4 = 0: exact flow (eq. exsolcub); else one RK4 step
  double tau;
  // FP32 copies (set by single_copies): FP32 kernels read these, so no
  // FP64-to-FP32 conversion runs per grid point
  float a3f, b3f, a4f, b4f, tauf;
  // coupled system (eq. coupled): cross-coupling a5 |other|^2
  double a5;
  float a5f;
};

struct OpArgs {
  int pro, epi;
  double t0, t1;   // prologue flow times
  double te;       // epilogue flow time
  int rk_scheme;   // 4 or 2 (EPI_RK)
  int rk_stage;    // 1-based stage (EPI_RK)
  int rk_coupled;  // EPI_RK of one field of the coupled system: e3 = the other field's stage argument
  NlParams nl;
  float t0f, t1f, tef;  // FP32 copies of t0, t1, te
};

// Fill the FP32 copies of an operator's parameters.
inline void single_copies(OpArgs& o) {
  o.t0f = (float)o.t0;
  o.t1f = (float)o.t1;
  o.tef = (float)o.te;
  o.nl.a3f = (float)o.nl.a3;
  o.nl.b3f = (float)o.nl.b3;
  o.nl.a4f = (float)o.nl.a4;
  o.nl.b4f = (float)o.nl.b4;
  o.nl.tauf = (float)o.nl.tau;
  o.nl.a5f = (float)o.nl.a5;
}

// The parameter in the working precision: the FP64 value or its FP32 copy.
template <class T> __device__ __forceinline__ T pv(double d, float f) {
  if constexpr (sizeof(T) == sizeof(double)) return d;
  else return f;
}

// g(u) = (a3 + i b3)|u|^2 u + (a4 + i b4)|u|^4 u  (eq. 1)
template <class T, class T2> __device__ __forceinline__ T2 nl_g(const NlParams& p, T2 u) {
  const T rho = fma(u.x, u.x, u.y * u.y);
  const T cr = rho * fma(pv<T>(p.a4, p.a4f), rho, pv<T>(p.a3, p.a3f));
  const T ci = rho * fma(pv<T>(p.b4, p.b4f), rho, pv<T>(p.b3, p.b3f));
  return mk<T2>(fma(cr, u.x, -ci * u.y), fma(cr, u.y, ci * u.x));
}

// Lambda(x) = -log|1-x|/x, Lambda(0) = 1; with it the exact flows read
// u0 exp((a + i b) r t Lambda(k a r t)) (eq. exsolcub and its quintic
// counterpart in Sec. 4.3), defined also for a = 0.
template <class T> __device__ __forceinline__ T lambda_fn(T x) {
  if (fabs(x) < T(1e-8)) return T(1) + x * (T(0.5) + x * (T(1) / T(3)));
  const T lg = (x < T(1)) ? log1p(-x) : log(x - T(1));
  return -lg / x;
}

// Exact flow of u' = (a + i b) rho^k u over time t, rho = |u|^2, k = 1 (cubic)
// or 2 (quintic): |u|^{2k} obeys r' = 2k a r^{k+1}, giving
// u(t) = u0 exp((a + i b) rho^k t Lambda(2k a rho^k t)).
template <class T, class T2> __device__ __forceinline__ T2 exact_power_flow(T2 u, T a, T b, int k, T t) {
  const T rho = fma(u.x, u.x, u.y * u.y);
  const T rk = (k == 1) ? rho : rho * rho;
  const T s = rk * t * lambda_fn<T>(T(2 * k) * a * rk * t);
  const T m = exp(a * s);
  T sn, cs;
  sincos(b * s, &sn, &cs);
  return mk<T2>(m * fma(u.x, cs, -u.y * sn), m * fma(u.x, sn, u.y * cs));
}

// phi_t: nonlinear flow of the splitting schemes (Sec. 2.1): exact for the
// cubic model (eq. exsolcub); one RK4 step of u' = g(u) otherwise (Sec. 4.3).
template <class T, class T2> __device__ __forceinline__ T2 nl_flow(const NlParams& p, T2 u, T t) {
  if (p.cubic) return exact_power_flow<T, T2>(u, pv<T>(p.a3, p.a3f), pv<T>(p.b3, p.b3f), 1, t);
  const T h = t * T(0.5);
  const T2 k1 = nl_g<T, T2>(p, u);
  const T2 k2 = nl_g<T, T2>(p, caxpy(u, h, k1));
  const T2 k3 = nl_g<T, T2>(p, caxpy(u, h, k2));
  const T2 k4 = nl_g<T, T2>(p, caxpy(u, t, k3));
  const T2 s = caxpy(cadd(k1, k4), T(2), cadd(k2, k3));  // k1 + 2 k2 + 2 k3 + k4
  return caxpy(u, t * (T(1) / T(6)), s);
}

// Coupled system (Sec. 4.5, eq. coupled): the nonlinear parts of the u and v
// equations, g_u = ((a3 + i b3)|u|^2 + (a4 + i b4)|u|^4 + a5 |v|^2) u and g_v
// with u and v exchanged.
template <class T, class T2> __device__ __forceinline__ void nl_g2(const NlParams& p, T2 u, T2 v, T2& gu, T2& gv) {
  const T a3 = pv<T>(p.a3, p.a3f), b3 = pv<T>(p.b3, p.b3f), a4 = pv<T>(p.a4, p.a4f), b4 = pv<T>(p.b4, p.b4f);
  const T a5 = pv<T>(p.a5, p.a5f);
  const T ru = fma(u.x, u.x, u.y * u.y), rv = fma(v.x, v.x, v.y * v.y);
  const T cur = fma(ru, fma(a4, ru, a3), a5 * rv), cui = ru * fma(b4, ru, b3);
  const T cvr = fma(rv, fma(a4, rv, a3), a5 * ru), cvi = rv * fma(b4, rv, b3);
  gu = mk<T2>(fma(cur, u.x, -cui * u.y), fma(cur, u.y, cui * u.x));
  gv = mk<T2>(fma(cvr, v.x, -cvi * v.y), fma(cvr, v.y, cvi * v.x));
}

// Nonlinear sub-flow of the coupled system: one RK4 step of (u, v)' = g(u, v)
// over time t (the coupled flow has no closed form; Sec. 4.3 uses one RK4
// step for the cubic-quintic model).
template <class T, class T2> __device__ __forceinline__ void nl_flow2(const NlParams& p, T2& u, T2& v, T t) {
  const T h = t * T(0.5);
  T2 k1u, k1v, k2u, k2v, k3u, k3v, k4u, k4v;
  nl_g2<T, T2>(p, u, v, k1u, k1v);
  nl_g2<T, T2>(p, caxpy(u, h, k1u), caxpy(v, h, k1v), k2u, k2v);
  nl_g2<T, T2>(p, caxpy(u, h, k2u), caxpy(v, h, k2v), k3u, k3v);
  nl_g2<T, T2>(p, caxpy(u, t, k3u), caxpy(v, t, k3v), k4u, k4v);
  const T s = t * (T(1) / T(6));
  u = caxpy(u, s, caxpy(cadd(k1u, k4u), T(2), cadd(k2u, k3u)));
  v = caxpy(v, s, caxpy(cadd(k1v, k4v), T(2), cadd(k2v, k3v)));
}

// Three-term splitting (Sec. 4.3): the cubic and quintic parts of g with
// their exact flows, phi^c (eq. exsolcub) and phi^q, composed as
// P_t = phi^c_t o phi^q_t before the linear flow and P*_t = phi^q_t o phi^c_t
// after it.
template <class T, class T2> __device__ __forceinline__ T2 flow_c(const NlParams& p, T2 u, T t) {
  return exact_power_flow<T, T2>(u, pv<T>(p.a3, p.a3f), pv<T>(p.b3, p.b3f), 1, t);
}
template <class T, class T2> __device__ __forceinline__ T2 flow_q(const NlParams& p, T2 u, T t) {
  return exact_power_flow<T, T2>(u, pv<T>(p.a4, p.a4f), pv<T>(p.b4, p.b4f), 2, t);
}

template <class T, class T2>
__device__ __forceinline__ void apply_prologue(const OpArgs& o, const T2* in, T2* z) {
  switch (o.pro) {
    case PRO_FLOW:
      z[0] = nl_flow<T, T2>(o.nl, in[0], pv<T>(o.t0, o.t0f));
      break;
    case PRO_FLOW2:
      z[0] = nl_flow<T, T2>(o.nl, in[0], pv<T>(o.t0, o.t0f));
      z[1] = nl_flow<T, T2>(o.nl, in[0], pv<T>(o.t1, o.t1f));
      break;
    case PRO_LAW4:
      z[0] = in[0];
      z[1] = nl_g<T, T2>(o.nl, in[0]);
      break;
    case PRO_CQ:
      z[0] = flow_c<T, T2>(o.nl, flow_q<T, T2>(o.nl, in[0], pv<T>(o.t0, o.t0f)), pv<T>(o.t0, o.t0f));
      break;
    case PRO_CQ2:
      z[0] = flow_c<T, T2>(o.nl, flow_q<T, T2>(o.nl, in[0], pv<T>(o.t0, o.t0f)), pv<T>(o.t0, o.t0f));
      z[1] = flow_c<T, T2>(o.nl, flow_q<T, T2>(o.nl, in[0], pv<T>(o.t1, o.t1f)), pv<T>(o.t1, o.t1f));
      break;
    case PRO_CFLOW:
      z[0] = in[0];
      z[1] = in[1];
      nl_flow2<T, T2>(o.nl, z[0], z[1], pv<T>(o.t0, o.t0f));
      break;
    case PRO_CG:
      nl_g2<T, T2>(o.nl, in[0], in[1], z[0], z[1]);
      break;
    case PRO_CLAW2: {
      T2 g0, g1;
      nl_g2<T, T2>(o.nl, in[0], in[1], g0, g1);
      const T t0 = pv<T>(o.t0, o.t0f);
      z[0] = caxpy(in[0], t0, g0);
      z[1] = caxpy(in[1], t0, g1);
      break;
    }
    case PRO_LAW2: {
      const T2 gn = nl_g<T, T2>(o.nl, in[0]);
      const T tau = pv<T>(o.nl.tau, o.nl.tauf);
      z[0] = caxpy(in[0], tau, gn);
      z[1] = caxpy(in[0], tau * T(0.5), gn);
      break;
    }
    default:
      z[0] = in[0];
      z[1] = in[1];
  }
}

// g of one field of the coupled system given the other field: g_u(u; v) =
// ((a3 + i b3)|u|^2 + (a4 + i b4)|u|^4 + a5 |v|^2) u (eq. coupled).
template <class T, class T2> __device__ __forceinline__ T2 nl_g_cross(const NlParams& p, T2 u, T2 v) {
  const T rho = fma(u.x, u.x, u.y * u.y), rv = fma(v.x, v.x, v.y * v.y);
  const T cr = fma(rho, fma(pv<T>(p.a4, p.a4f), rho, pv<T>(p.a3, p.a3f)), pv<T>(p.a5, p.a5f) * rv);
  const T ci = rho * fma(pv<T>(p.b4, p.b4f), rho, pv<T>(p.b3, p.b3f));
  return mk<T2>(fma(cr, u.x, -ci * u.y), fma(cr, u.y, ci * u.x));
}

// Runge-Kutta stage epilogue on y = K x (eq. RK4 / eq. RK2):
// extras e0 = x (stage argument), e1 = u_n, e2 = acc (coupled system: e3 =
// the other field's stage argument, for g); outputs o0, o1.
//   RK4 s=1..3: k = y + g(x); acc (+)= w_s k; x_next = u_n + c_{s+1} k  -> (x_next, acc)
//   RK4 s=4   : u_{n+1} = u_n + tau/6 (acc + k)                        -> (u_{n+1})
//   RK2 s=1   : acc = k; x_next = u_n + tau k ; s=2: u_n + tau/2 (acc + k)
template <class T, class T2>
__device__ __forceinline__ int rk_stage(const OpArgs& o, T2 y, const T2* e, T2* out) {
  const T tau = pv<T>(o.nl.tau, o.nl.tauf);
  const T2 k = cadd(y, o.rk_coupled ? nl_g_cross<T, T2>(o.nl, e[0], e[3]) : nl_g<T, T2>(o.nl, e[0]));
  if (o.rk_scheme == 4) {
    switch (o.rk_stage) {
      case 1: out[1] = k; out[0] = caxpy(e[1], tau * T(0.5), k); return 2;
      case 2: out[1] = caxpy(e[2], T(2), k); out[0] = caxpy(e[1], tau * T(0.5), k); return 2;
      case 3: out[1] = caxpy(e[2], T(2), k); out[0] = caxpy(e[1], tau, k); return 2;
      default: out[0] = caxpy(e[1], tau * (T(1) / T(6)), cadd(e[2], k)); return 1;
    }
  }
  if (o.rk_stage == 1) { out[1] = k; out[0] = caxpy(e[1], tau, k); return 2; }
  out[0] = caxpy(e[1], tau * T(0.5), cadd(e[2], k));
  return 1;
}

// Returns the number of outputs written.
template <class T, class T2>
__device__ __forceinline__ int apply_epilogue(const OpArgs& o, const T2* y, const T2* e, T2* out) {
  const T tau = pv<T>(o.nl.tau, o.nl.tauf);
  switch (o.epi) {
    case EPI_FLOW:
      out[0] = nl_flow<T, T2>(o.nl, y[0], pv<T>(o.te, o.tef));
      return 1;
    case EPI_FLOW2:
      out[0] = nl_flow<T, T2>(o.nl, y[0], pv<T>(o.te, o.tef));
      out[1] = nl_flow<T, T2>(o.nl, y[1], pv<T>(o.te, o.tef));
      return 2;
    case EPI_QC:
      out[0] = flow_q<T, T2>(o.nl, flow_c<T, T2>(o.nl, y[0], pv<T>(o.te, o.tef)), pv<T>(o.te, o.tef));
      return 1;
    case EPI_QC2: {
      // end of S^3_tau, and the middle P*_{tau/4} P_{tau/4} of the two half
      // steps with its two quintic quarter flows merged into one of tau/2
      // (exact flows: semigroup)
      const T te = pv<T>(o.te, o.tef);
      out[0] = flow_q<T, T2>(o.nl, flow_c<T, T2>(o.nl, y[0], te), te);
      out[1] = flow_c<T, T2>(o.nl, flow_q<T, T2>(o.nl, flow_c<T, T2>(o.nl, y[1], te * T(0.5)), te), te * T(0.5));
      return 2;
    }
    case EPI_SPLIT4_3T: {
      const T te = pv<T>(o.te, o.tef);
      const T2 f = flow_q<T, T2>(o.nl, flow_c<T, T2>(o.nl, y[0], te), te);
      out[0] = mk<T2>(fma(T(4) / T(3), f.x, -(T(1) / T(3)) * e[0].x),
                      fma(T(4) / T(3), f.y, -(T(1) / T(3)) * e[0].y));
      return 1;
    }
    case EPI_SPLIT4: {
      const T2 f = nl_flow<T, T2>(o.nl, y[0], pv<T>(o.te, o.tef));
      out[0] = mk<T2>(fma(T(4) / T(3), f.x, -(T(1) / T(3)) * e[0].x),
                      fma(T(4) / T(3), f.y, -(T(1) / T(3)) * e[0].y));
      return 1;
    }
    case EPI_LAW4A: {
      // a = E u, b = E g(u) with E = exp(tau K / 2); Lawson4 (eq. lawson4)
      // rewritten with E^2 = exp(tau K):  u2 = a + tau/2 b, u3 = a + tau/2 g(u2),
      // p = a + tau g(u3) (so u4 = E p), w = a + tau/6 b + tau/3 (g(u2)+g(u3))
      // (so u_{n+1} = E w + tau/6 g(E p)).
      const T2 a = y[0], b = y[1];
      const T2 g2 = nl_g<T, T2>(o.nl, caxpy(a, tau * T(0.5), b));
      const T2 g3 = nl_g<T, T2>(o.nl, caxpy(a, tau * T(0.5), g2));
      out[0] = caxpy(a, tau, g3);
      out[1] = caxpy(caxpy(a, tau * (T(1) / T(6)), b), tau * (T(1) / T(3)), cadd(g2, g3));
      return 2;
    }
    case EPI_LAW4B:
      out[0] = caxpy(y[1], tau * (T(1) / T(6)), nl_g<T, T2>(o.nl, y[0]));
      return 1;
    case EPI_LAW2:
      out[0] = caxpy(y[1], tau * T(0.5), nl_g<T, T2>(o.nl, y[0]));
      return 1;
    case EPI_RK:
      return rk_stage<T, T2>(o, y[0], e, out);
    case EPI_CFLOW:
      out[0] = y[0];
      out[1] = y[1];
      nl_flow2<T, T2>(o.nl, out[0], out[1], pv<T>(o.te, o.tef));
      return 2;
    case EPI_CSPLIT4: {
      T2 f0 = y[0], f1 = y[1];
      nl_flow2<T, T2>(o.nl, f0, f1, pv<T>(o.te, o.tef));
      out[0] = mk<T2>(fma(T(4) / T(3), f0.x, -(T(1) / T(3)) * e[0].x),
                      fma(T(4) / T(3), f0.y, -(T(1) / T(3)) * e[0].y));
      out[1] = mk<T2>(fma(T(4) / T(3), f1.x, -(T(1) / T(3)) * e[1].x),
                      fma(T(4) / T(3), f1.y, -(T(1) / T(3)) * e[1].y));
      return 2;
    }
    case EPI_CLAW4P:
    case EPI_CLAW4W: {
      // Lawson4 on the pair with E = exp(tau K / 2): a = E W (extras), b =
      // E g(W) (this sweep); u2 = a + tau/2 b, u3 = a + tau/2 g(u2)
      T2 g2[2], g3[2];
      nl_g2<T, T2>(o.nl, caxpy(e[0], tau * T(0.5), y[0]), caxpy(e[1], tau * T(0.5), y[1]), g2[0], g2[1]);
      nl_g2<T, T2>(o.nl, caxpy(e[0], tau * T(0.5), g2[0]), caxpy(e[1], tau * T(0.5), g2[1]), g3[0], g3[1]);
      for (int f = 0; f < 2; ++f)
        out[f] = o.epi == EPI_CLAW4P
                     ? caxpy(e[f], tau, g3[f])
                     : caxpy(caxpy(e[f], tau * (T(1) / T(6)), y[f]), tau * (T(1) / T(3)), cadd(g2[f], g3[f]));
      return 2;
    }
    case EPI_CLAW4B:
    case EPI_CLAW2: {
      T2 g0, g1;
      nl_g2<T, T2>(o.nl, e[0], e[1], g0, g1);
      const T c = o.epi == EPI_CLAW4B ? tau * (T(1) / T(6)) : tau * T(0.5);
      out[0] = caxpy(y[0], c, g0);
      out[1] = caxpy(y[1], c, g1);
      return 2;
    }
    default:
      out[0] = y[0];
      out[1] = y[1];
      return 2;
  }
}

__device__ __forceinline__ bool finite2(double2 v) { return isfinite(v.x) && isfinite(v.y); }
__device__ __forceinline__ bool finite2(float2 v) { return isfinite(v.x) && isfinite(v.y); }

// ---------------------------------------------------------------- passes

// Field pointers of one pass (any may alias, see the layout note above).
struct PassFields {
  void* in[kMaxRhs];       // prologue inputs (first pass of a sweep)
  void* work[kMaxRhs];     // fields transformed by the linear flow
  void* extra[kMaxExtra];  // epilogue extra inputs (last pass)
  void* out[kMaxRhs];      // epilogue outputs (last pass)
  int nin, nrhs, nextra, nout;
};

// One pass over the pencils of axis `axis`.
struct PassGeom {
  int d;
  int64_t n[3];
  int axis;
  int64_t n_ax;      // pencil length
  int64_t P;         // element stride along the axis
  int64_t npencils;  // N / n_ax
};

enum PassFlags : int {
  PASS_PRO = 1,   // read `in`, apply prologue
  PASS_FWD = 2,   // forward FFT along the axis (periodic)
  PASS_MUL = 4,   // multiply by the separable Fourier symbol (last axis)
  PASS_INV = 8,   // inverse FFT along the axis (periodic)
  PASS_EPI = 16   // apply epilogue, write `out`
};

// Fourier symbol of one right-hand side: product form (exp(c tau K), the
// tensor E of Sec. 3.2 with the inverse-FFT 1/N folded in) or sum form (K).
struct Symbol {
  const void* vec[3];  // per-axis vectors in FFT order (T2)
  int sum_form;        // 0: prod_mu vec_mu[k_mu]   1: sum_mu vec_mu[k_mu]
};

struct FftPassArgs {
  PassGeom g;
  PassFields f;
  OpArgs op;
  int flags;
  Symbol sym[kMaxRhs];
  const void* twiddle;  // T[2][n_ax][3]: FMA-butterfly form of exp(-+2 pi i m / n_ax), see fft.cu
  const int* twform;    // int[2][n_ax]
  const void* twplain;  // T2[2][n_ax]: exp(-+2 pi i m / n_ax) (mixed-radix n_ax)
  int* status;          // device status word (bit 0: non-finite output)
};

struct ModePassArgs {
  PassGeom g;
  PassFields f;
  OpArgs op;
  int flags;                     // PASS_PRO / PASS_EPI
  const void* factor[kMaxRhs];   // n x n column-major T2 per rhs
  int* status;
};

// Launchers (return cudaError_t of the launch).
template <class T> cudaError_t launch_fft_pass(const FftPassArgs& a, cudaStream_t s);
template <class T> cudaError_t launch_mode_pass(const ModePassArgs& a, cudaStream_t s);
template <class T> cudaError_t prepare_fft_pass();
template <class T> cudaError_t prepare_mode_pass();

// Mode pass with an explicit number of fibers per CTA (tb), and the
// persistent step kernel over many instances (batch.cu).
struct BatchItem {
  int inst;     // index into the per-instance ModePassArgs table
  int tb;       // fibers per tile
  int64_t b0;   // first fiber
};
int mode_tb_max(int n, int nrhs, size_t elem);
size_t mode_smem_bytes(int n, int nrhs, size_t elem, int tb);
// One launch per time step over many instances (batch.cu): the work items of
// every pass of the step in one list; an item of pass k for instance i runs
// once every item of instance i's previous pass has finished.
struct StepItem {
  int pass;     // pass (sweep, mode) of the step
  int inst;     // instance
  int tb;       // fibers per tile
  int64_t b0;   // first fiber
};
struct StepArgs {
  const ModePassArgs* table;  // [npass][count] pass arguments
  const StepItem* items;      // pass-major
  int nitems;
  const int* need;            // [npass][count]: items of (pass, instance)
  const int* prev;            // [npass][count]: the instance's previous pass, or -1
  int npass, count;
  int* counter;               // [2 + npass count], zeroed before the launch: next item, abort, done counts
  int* status;
  long long spin_limit;       // polls of a dependency wait before it gives up (kStepSpinLimit)
  int want_bias;              // added to every dependency target: 1 makes each wait unreachable (fault injection)
};
// Polls of the batch step's dependency waits (128 ns apart: about 0.5 s).
constexpr long long kStepSpinLimit = 1ll << 22;
// Polls before an injected, unreachable wait gives up (about 0.15 ms).
constexpr long long kStepInjectedSpinLimit = 1024;
template <class T> cudaError_t launch_batched_step(const StepArgs& a, size_t smem, int grid, cudaStream_t s);
template <class T> int batched_step_blocks_per_sm(size_t smem);
template <class T> cudaError_t launch_mode_pass_tb(const ModePassArgs& a, int tb, cudaStream_t s);
// stencil.cu: K x on finite-difference directions (eq. kronsumv as a
// stencil) fused with a Runge-Kutta stage epilogue; out must not alias x.
struct StencilArgs {
  int d;
  int64_t n[3];
  int bc[3];
  double cr[3], ci[3];  // (a1 + i b1) / h_mu^2
  double a2;
  float crf[3], cif[3], a2f;  // FP32 copies
  const void* x;              // stage argument
  const void* extra[kMaxExtra];
  int nextra;
  void* out[2];
  int nout;
  OpArgs op;
  int* status;
};
template <class T> cudaError_t launch_kron_stencil(const StencilArgs& a, cudaStream_t s);

// conv_mma.cu: 3x3 circular convolution on the tensor cores (BF16 operands,
// FP32 accumulation), y = conv(x, w) + bias (optional ReLU); Cin, Cout <= 32.
cudaError_t prepare_conv_mma();
cudaError_t launch_conv_mma(const float* x, const __nv_bfloat16* w, const float* bias, float* y, int B, int cin,
                            int cout, int H, int W, int relu, int* status, cudaStream_t s);
// Weight and bias gradients of that convolution on the tensor cores (BF16 x
// and dy, FP32 accumulation), added into dw [Cout][Cin][3][3] and db [Cout].
cudaError_t launch_wgrad_mma(const float* x, const float* dy, float* dw, float* db, int B, int cin, int cout, int H,
                             int W, int* status, cudaStream_t s);

// expm.cu: FP64 complex n x n exponential of (scale * A) on the device.
// dA: n x n column-major double2 (device); dOut: same layout.  work: 3*n*n double2.
cudaError_t expm_device(const double2* dA, double scale, int n, double2* dOut, double2* work,
                        double norm1, cudaStream_t s);
// Periodic symbols: vec[k] = exp(c*tau*(alpha*(-kappa_k^2) + beta + i adv kappa'_k)) * post  (sum_form = 0)
//                   vec[k] = (alpha*(-kappa_k^2) + beta + i adv kappa'_k) * post              (sum_form = 1)
// kappa' = kappa but 0 at the Nyquist mode of an even n.
cudaError_t periodic_symbol_device(double2* dOut, int n, double L, double ctau, double ar,
                                   double ai, double beta, double adv, double post, int sum_form,
                                   cudaStream_t s);
// Plain twiddles exp(-+2 pi i m/n), T2[2][n] (forward, inverse), for the
// mixed-radix FFT passes.
cudaError_t plain_twiddles_device(void* tab, int n, int f64, cudaStream_t s);
// FFT twiddles for the FMA butterflies: for w = exp(-+2 pi i m/n) = c + i s,
// form 0 (|c| >= |s|): tau = s/c, m_re = m_im = c; form 1: tau = -c/s,
// m_re = -s, m_im = s.  Tables in T (double when f64, else float).
cudaError_t fma_twiddles_device(void* tab, int* form, int n, int f64, cudaStream_t s);
cudaError_t convert_f64_to_f32(const double2* src, float2* dst, int64_t count, cudaStream_t s);

// mma_mode.cu: BF16x3 mu-mode product on tcgen05 (complex64 state).
struct MmaLaunch {
  int n;              // mode length n_mu (<= 256)
  int64_t P, Q, N;    // faster (first direction padded) / slower products, plane length
  int64_t pitch;      // mode 1: distance between fibers in the planes
  int nrhs;
  const void* tmA[kMaxRhs];  // CUtensorMap (128 bytes) of each rhs's BF16x3 planes
  const void* tmB[kMaxRhs];  // CUtensorMap of each rhs's factor splits
  int out_fp32;       // 1: FP32 planes, 0: BF16x3 planes
  void* out[kMaxRhs];
  int* status;
  int grouped = 0;    // 1: row blocking of the persistent grouped pass (launch_mma_group)
};
struct MmaPassArgs {
  int n;             // mode length n_mu (<= 256)
  int np;            // n rounded up to a multiple of 16: size of the padded factor
  int64_t P, Q;      // products of the faster (first one padded) / slower sizes
  int64_t pitch;     // mode 1: distance between fibers in the planes (>= np)
  int64_t per_q;     // MN-major: fiber tiles per slab, ceil(P / 128)
  int a_mn;          // 1: A is MN-major (P > 1, P % 64 == 0); 0: K-major (mode 1)
  int out_fp32;      // 1: FP32 planes (re, im); 0: BF16x3 planes (6)
  void* out[kMaxRhs];
  int64_t N;         // plane length (padded field size)
  int nc;            // output rows per tile (multiple of 16, <= 128 when np > 128)
  int nsub;          // row blocks per component: ceil(np / nc)
  int both;          // 1: a tile's nc = 2 np rows are both components (grouped pass, np <= 64)
  int tmem_cols;     // power of two >= 2 nc
  int stages;        // pipeline depth
  int* status;
};
constexpr size_t kTensorMapBytes = 128;
// Padded sizes of the tensor-core path: factors to a multiple of 16, the
// planes' first direction to a multiple of 64.
inline int mma_pad16(int n) { return (n + 15) / 16 * 16; }
inline int64_t mma_pitch(int64_t n1) { return (n1 + 63) / 64 * 64; }
// Output rows of one component per CTA: half of np when np >= 64 is a
// multiple of 32, else np up to 128, else np / 2 rounded up to 16 (two
// CTAs per SM in every case but np <= 128 odd multiples of 16).
inline int mma_rows_per_cta(int np) {
  if (np >= 64 && np % 32 == 0) return np / 2;
  if (np <= 128) return np;
  return (np / 2 + 15) / 16 * 16;
}
// nsplit: BF16 planes per component in the box (3 for BF16x3, 7 for the
// Ozaki digits); rows: output rows per box (0: those of the BF16x3 pass).
cudaError_t make_state_tmap(void* map_out, const void* splits, int n, int64_t P, int64_t Q, int64_t N,
                            int64_t pitch, int nsplit = 3);
cudaError_t make_factor_tmap(void* map_out, const void* fsplit, int n, int nsplit = 3, int rows = 0);
size_t mma_factor_bytes(int n);
size_t mma_smem_bytes(int nc);
cudaError_t prepare_mma_pass();
// Fills the pass arguments; returns the CTAs per rhs, or -1 for an
// unsupported geometry.
int64_t mma_build_args(const MmaLaunch& L, MmaPassArgs* out);
cudaError_t launch_mma_pass(const MmaLaunch& L, cudaStream_t s);
// One persistent launch over a group of passes (one CTA per SM): device
// arrays of MmaPassArgs, of four CUtensorMaps per pass (A rhs 0 / 1, B rhs
// 0 / 1) and of the ntiles (pass, tile within the pass) pairs (int2) of the
// group, in the order the CTAs take them.
cudaError_t launch_mma_group(const void* passes, const void* maps, const void* tiles, int npass, int64_t ntiles,
                             int nrhs, cudaStream_t s);
// Pointwise stages around the tensor-core passes, one field per segment
// (planes: first direction padded to `pitch`, Npad values per plane).
struct SplitSeg {
  const float2* in[2];
  int nin;
  OpArgs op;
  void* dst[2];        // six BF16 planes per rhs
  int64_t N, n1, pitch, Npad;
};
struct EpiSeg {
  const float* y[2];   // FP32 planes (re, im) per rhs
  const float2* ex[kMaxExtra];
  int nextra;
  OpArgs op;
  float2* out[2];
  int nout;
  int64_t N, n1, pitch, Npad;
};
// segs == nullptr: the single segment `one`; else nseg device segments.
cudaError_t launch_split_prologue(const SplitSeg& one, const SplitSeg* segs, int nseg, int64_t max_n, int nrhs,
                                  cudaStream_t s);
cudaError_t launch_plane_epilogue(const EpiSeg& one, const EpiSeg* segs, int nseg, int64_t max_n, int nrhs,
                                  int* status, cudaStream_t s);
cudaError_t launch_factor_split(const double2* F, int n, void* out, cudaStream_t s);

// oz_mode.cu: FP64-accurate mu-mode product on tcgen05 by the Ozaki
// splitting (seven exact 7-bit BF16 digits per operand, 28 products in seven
// exact FP32 level accumulators; complex128 state).
struct OzLaunch {
  int n;              // mode length n_mu (<= 256)
  int64_t P, Q, N;    // faster (first direction padded) / slower products, plane length
  int64_t pitch;      // mode 1: distance between fibers in the planes
  int nrhs;
  const void* tmA[kMaxRhs];  // CUtensorMap of each rhs's 14 digit planes ([digit][re, im])
  const void* tmB[kMaxRhs];  // CUtensorMap of each rhs's factor digits
  const int* aexp[kMaxRhs];  // per-fiber exponents of each rhs's state digits
  const int* bexp[kMaxRhs];  // per-output-row exponents of each rhs's factor digits
  double* out[kMaxRhs];      // FP64 planes (re, im) per rhs
  int* status;
};
struct OzPassArgs {
  int n, np;
  int64_t P, Q, pitch, per_q;
  int a_mn;
  int64_t N;
  int nc, nsub, tmem_cols;
  const int* aexp[kMaxRhs];
  const int* bexp[kMaxRhs];
  double* out[kMaxRhs];
  int* status;
};
struct OzSliceArgs {
  const double* z;       // FP64 planes [2][N]
  __nv_bfloat16* dst;    // 14 BF16 planes [digit][re, im][N]
  int* exps;             // per-fiber exponents (fiber q (mode 1) or q P + p)
  int n;
  int64_t P, Q, N, pitch;
  int* status;
};
struct OzSeg {
  const double2* in[2];
  int nin;
  OpArgs op;
  double* z[2];          // FP64 planes (re, im) per rhs, Npad values each
  const double2* ex[kMaxExtra];
  int nextra;
  double2* out[2];
  int nout;
  int64_t N, n1, pitch, Npad;
};
int oz_rows_per_cta(int np);
size_t oz_factor_bytes(int n);
cudaError_t prepare_oz_pass();
int64_t oz_build_args(const OzLaunch& L, OzPassArgs* out);
cudaError_t launch_oz_pass(const OzLaunch& L, cudaStream_t s);
cudaError_t launch_oz_slice(const OzSliceArgs& a, cudaStream_t s);
cudaError_t launch_oz_factor_slice(const double2* F, int n, void* out, int* fexp, cudaStream_t s);
cudaError_t launch_oz_prologue(const OzSeg& g, int nrhs, cudaStream_t s);
cudaError_t launch_oz_epilogue(const OzSeg& g, int nrhs, int* status, cudaStream_t s);

// norms.cu
cudaError_t rel_error_device(const void* x, const void* y, int64_t count, int precision,
                             double* d_partial, int nblocks, double* h_out, cudaStream_t s);
int rel_error_blocks(int64_t count);

}  // namespace cgl
