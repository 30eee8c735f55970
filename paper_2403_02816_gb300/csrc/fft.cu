// Periodic linear flow exp(c tau K) u = F^{-1}(E .* F u) (Sec. 3.2) as
// pencil passes: one kernel launch transforms every pencil along one axis.
//
// A CTA owns up to kTile/n whole pencils of each right-hand side.  It loads
// them (coalesced, applying the sweep's nonlinear prologue on the first
// pass), runs a Stockham autosort FFT in shared memory (radix-4 stages first,
// so the twiddle-free stage is a radix-4 one, and one radix-2 stage last when
// log2 n is odd; each thread keeps its butterflies of both right-hand sides
// in registers between the read and the write half of a stage), optionally
// multiplies by the separable Fourier symbol and runs the inverse FFT (last
// axis), and stores (applying the sweep's epilogue on the last pass).  The
// forward transform is unnormalised; the 1/N of the inverse is folded into
// the symbol vectors.  In FP64 the pass is bound by the FP64 pipe: the layout
// keeps the DP instruction count near 3.5 per point and radix-2 level.
#include "cgl_internal.cuh"

namespace cgl {

constexpr int kFftThreads = 256;
constexpr int kFftTile = 2048;  // complex elements of one field per CTA (8 per thread)
constexpr int kFftTileMR = 1024;  // mixed radix: smaller tiles, more CTAs on small grids
constexpr int kFftMaxSmem = 200 * 1024;

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

// Twiddle w = c + i s in FMA-butterfly form (built by fma_twiddles_device):
// form 0 (|c| >= |s|): w = c (1 + i tau), m_re = m_im = c;
// form 1 (|c| <  |s|): w = s (i - tau),   m_re = -s, m_im = s;  |tau| <= 1.
// With u = b.x - tau b.y and v = b.y + tau b.x:
//   form 0: w b = m_re u + i m_im v;   form 1: w b = m_re v + i m_im u.
template <class T> struct Tw {
  T tau, mre, mim;
  int form;
};

template <class T> __device__ __forceinline__ Tw<T> load_tw(const T* tt, const int* tf, int m) {
  Tw<T> w;
  w.tau = tt[3 * m];
  w.mre = tt[3 * m + 1];
  w.mim = tt[3 * m + 2];
  w.form = tf[m];
  return w;
}

// (a, b) <- (a + w b, a - w b): two FMAs for u, v and four for the outputs,
// against eight operations with a plain complex multiply.
template <class T, class T2> __device__ __forceinline__ void fma_bfly(T2& a, T2& b, const Tw<T>& w) {
  const T u = fma(-w.tau, b.y, b.x);
  const T v = fma(w.tau, b.x, b.y);
  const T P = w.form ? v : u;
  const T Q = w.form ? u : v;
  const T2 a0 = a;
  a = mk<T2>(fma(w.mre, P, a0.x), fma(w.mim, Q, a0.y));
  b = mk<T2>(fma(-w.mre, P, a0.x), fma(-w.mim, Q, a0.y));
}

// One Stockham stage of radix R on `tb` pencils of length n, for NR tiles
// (right-hand sides) at once; tile r starts at s0 + r * tile_stride.
// p = product of the radices already applied.  Butterfly i of a pencil
// (k = i mod p) reads x_r = s[i + r n/R], multiplies by w_r = exp(-+2 pi i r k/(pR)),
// does a length-R DFT and writes s[(i-k)R + k + r p].  With twiddles
// (p > 1) the radix-4 DFT of (x0, w1 x1, w2 x2, w3 x3), w3 = w1 w2, is done as
// four FMA butterflies: (x0, x2) and (x1, x3) with w2, then (x0, x1) with w1
// and (x2, x3) with -+i w1 (table entry m1 + n/4); outputs y0 y1 y2 y3 =
// x0 x2 x1 x3.  tt/tf: this direction's twiddle table.
template <class T, class T2, int R, int NR>
__device__ __forceinline__ void fft_stage(T2* s0, int tile_stride, int pitch, int n, int lognb, int tb, int p,
                                          const T* tt, const int* tf, bool inv) {
  constexpr int BPT = 8 / R;
  const int nb = n / R;
  const int total = tb * nb;
  const int twstride = n / (p * R);
  T2 v[NR][BPT][R];
  int dst[BPT];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int q = threadIdx.x + b * kFftThreads;
    dst[b] = -1;
    if (q < total) {
      const int t = q >> lognb;
      const int i = q & (nb - 1);
      const int k = i & (p - 1);
      const int src = t * pitch + i;
#pragma unroll
      for (int rr = 0; rr < NR; ++rr)
#pragma unroll
        for (int r = 0; r < R; ++r) v[rr][b][r] = s0[rr * tile_stride + src + r * nb];
      if (p == 1) {
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          if (R == 2) dft2(v[rr][b]);
          else dft4(v[rr][b], inv);
        }
      } else if (R == 2) {
        const Tw<T> w = load_tw(tt, tf, k * twstride);
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) fma_bfly<T, T2>(v[rr][b][0], v[rr][b][1], w);
      } else {
        const int m1 = k * twstride;
        const Tw<T> w1 = load_tw(tt, tf, m1), w2 = load_tw(tt, tf, 2 * m1), w3 = load_tw(tt, tf, m1 + n / 4);
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          T2* x = v[rr][b];
          fma_bfly<T, T2>(x[0], x[2], w2);
          fma_bfly<T, T2>(x[1], x[3], w2);
          fma_bfly<T, T2>(x[0], x[1], w1);
          fma_bfly<T, T2>(x[2], x[3], w3);
          const T2 y1 = x[2];
          x[2] = x[1];
          x[1] = y1;
        }
      }
      dst[b] = t * pitch + (i - k) * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    if (dst[b] >= 0) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr)
#pragma unroll
        for (int r = 0; r < R; ++r) s0[rr * tile_stride + dst[b] + r * p] = v[rr][b][r];
    }
  }
  __syncthreads();
}

template <class T, class T2, int NR>
__device__ void fft_tile(T2* s0, int tile_stride, int pitch, int n, int logn, int tb, const T* tt, const int* tf,
                         bool inv) {
  int p = 1;
  for (int st = 0; st < logn / 2; ++st) {
    fft_stage<T, T2, 4, NR>(s0, tile_stride, pitch, n, logn - 2, tb, p, tt, tf, inv);
    p *= 4;
  }
  if (logn & 1) fft_stage<T, T2, 2, NR>(s0, tile_stride, pitch, n, logn - 1, tb, p, tt, tf, inv);
}

// ---------------------------------------------------------------------------
// Mixed-radix passes (n = 2^a 3^b 5^c 7^d, not a power of two): the same
// Stockham recursion with radices 4, 2, 3, 5, 7 in that order, out of place
// between two tiles, plain complex twiddles w_(pR)^(r k) and R-point DFTs
// whose roots of unity come from the same n-point table (w_R^j = w_n^(j n/R)).
// ---------------------------------------------------------------------------

template <class T2, int R>
__device__ __forceinline__ void mr_stage(const T2* src, T2* dst, int nrhs_tiles, int tile_stride, int pitch, int n,
                                         int tb, int p, const T2* tw, bool inv) {
  const int nb = n / R;
  const int total = tb * nb;
  const int twstep = n / (p * R);
  const int rstep = n / R;
  for (int q = threadIdx.x; q < total; q += kFftThreads) {
    const int t = q / nb, i = q - t * nb;
    const int k = i % p;
    const int so = t * pitch + i;
    const int dso = t * pitch + (i - k) * R + k;
    for (int rr = 0; rr < nrhs_tiles; ++rr) {
      T2 x[R];
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = src[rr * tile_stride + so + r * nb];
      if (k > 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], tw[r * k * twstep]);
      }
      if constexpr (R == 2) {
        dft2(x);
      } else if constexpr (R == 4) {
        dft4(x, inv);
      } else {
        // odd R: with a_r = x_r + x_(R-r), b_r = x_r - x_(R-r) and
        // w^(r m) = c + i s (the table's sign for this direction),
        // y_m = x_0 + sum_r (c a_r + i s b_r) and y_(R-m) = x_0 + sum_r (c a_r - i s b_r)
        constexpr int H = (R - 1) / 2;
        T2 a[H], b[H];
#pragma unroll
        for (int r = 1; r <= H; ++r) {
          a[r - 1] = cadd(x[r], x[R - r]);
          b[r - 1] = csub(x[r], x[R - r]);
        }
        T2 y0 = x[0];
#pragma unroll
        for (int r = 0; r < H; ++r) y0 = cadd(y0, a[r]);
#pragma unroll
        for (int m = 1; m <= H; ++m) {
          T2 A = x[0], B = mk<T2>(0, 0);
#pragma unroll
          for (int r = 1; r <= H; ++r) {
            const T2 w = tw[((r * m) % R) * rstep];
            A = mk<T2>(fma(w.x, a[r - 1].x, A.x), fma(w.x, a[r - 1].y, A.y));
            B = mk<T2>(fma(w.y, b[r - 1].x, B.x), fma(w.y, b[r - 1].y, B.y));
          }
          // i B = (-B.y, B.x)
          x[m] = mk<T2>(A.x - B.y, A.y + B.x);
          x[R - m] = mk<T2>(A.x + B.y, A.y - B.x);
        }
        x[0] = y0;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) dst[rr * tile_stride + dso + r * p] = x[r];
    }
  }
  __syncthreads();
}

// Transform the NR tiles starting in `a`; returns the tile holding the result
// (a or b).  tw: this direction's plain table (forward or inverse).
template <class T2, int NR>
__device__ T2* mr_tile(T2* a, T2* b, int tile_stride, int pitch, int n, int tb, const T2* tw, bool inv) {
  int m = n, p = 1;
  T2 *src = a, *dst = b;
  while (m > 1) {
    if (m % 4 == 0) { mr_stage<T2, 4>(src, dst, NR, tile_stride, pitch, n, tb, p, tw, inv); p *= 4; m /= 4; }
    else if (m % 2 == 0) { mr_stage<T2, 2>(src, dst, NR, tile_stride, pitch, n, tb, p, tw, inv); p *= 2; m /= 2; }
    else if (m % 3 == 0) { mr_stage<T2, 3>(src, dst, NR, tile_stride, pitch, n, tb, p, tw, inv); p *= 3; m /= 3; }
    else if (m % 5 == 0) { mr_stage<T2, 5>(src, dst, NR, tile_stride, pitch, n, tb, p, tw, inv); p *= 5; m /= 5; }
    else { mr_stage<T2, 7>(src, dst, NR, tile_stride, pitch, n, tb, p, tw, inv); p *= 7; m /= 7; }
    T2* x = src;
    src = dst;
    dst = x;
  }
  return src;
}

template <class T2> __device__ __forceinline__ T2 ldf(const void* base, int64_t off) {
  return reinterpret_cast<const T2*>(base)[off];
}
template <class T2> __device__ __forceinline__ void stf(void* base, int64_t off, T2 v) {
  reinterpret_cast<T2*>(base)[off] = v;
}

template <class T, int NR, bool MR>
__device__ __forceinline__ void fft_pass_body(const FftPassArgs& a, unsigned char* smem_raw) {
  using T2 = typename C2<T>::type;
  const int n = (int)a.g.n_ax;
  const int logn = __ffs(n) - 1;  // power-of-two passes only
  const int tbmax = max(1, (MR ? kFftTileMR : kFftTile) / n);
  const int pitch = n + 1;
  const int tile_stride = tbmax * pitch;
  const int64_t b0 = (int64_t)blockIdx.x * tbmax;
  const int tb = (int)min((int64_t)tbmax, a.g.npencils - b0);
  const int64_t P = a.g.P;

  T2* tile0 = reinterpret_cast<T2*>(smem_raw);
  T2* tile1 = tile0 + NR * tile_stride;               // mixed radix: second (ping-pong) tile
  T2* pfac = tile0 + (MR ? 2 : 1) * NR * tile_stride;  // [kMaxRhs][tbmax]
  int64_t* pbase = reinterpret_cast<int64_t*>(pfac + kMaxRhs * tbmax);
  T* tt = reinterpret_cast<T*>(pbase + tbmax);  // [2][n][3] twiddles (forward, inverse)
  int* tf = reinterpret_cast<int*>(tt + 6 * n);  // [2][n] twiddle forms
  // mixed radix: [2][n] plain twiddles, 16-byte aligned (tbmax may be odd)
  T2* twp = reinterpret_cast<T2*>((reinterpret_cast<uintptr_t>(pbase + tbmax) + 15) & ~uintptr_t(15));

  if constexpr (MR) {
    const T2* twg = reinterpret_cast<const T2*>(a.twplain);
    for (int m = threadIdx.x; m < 2 * n; m += kFftThreads) twp[m] = twg[m];
  } else {
    const T* ttg = reinterpret_cast<const T*>(a.twiddle);
    for (int m = threadIdx.x; m < 6 * n; m += kFftThreads) tt[m] = ttg[m];
    for (int m = threadIdx.x; m < 2 * n; m += kFftThreads) tf[m] = a.twform[m];
  }
  // (pencil t, position j) of element e: pencil-major for contiguous
  // pencils, position-major otherwise
  auto split = [&](int e, int& t, int& j) {
    if (P == 1) {
      if (MR) { t = e / n; j = e - t * n; }
      else { t = e >> logn; j = e & (n - 1); }
    } else {
      j = e / tb;
      t = e - j * tb;
    }
  };
  for (int t = threadIdx.x; t < tb; t += kFftThreads) {
    const int64_t b = b0 + t;
    const int64_t p = b % P, q = b / P;
    pbase[t] = p + P * (int64_t)n * q;
    if (a.flags & PASS_MUL) {
      // indices of the other axes of this pencil
      int64_t kk[3] = {0, 0, 0};
      int64_t rem = p;
      for (int mu = 0; mu < a.g.axis; ++mu) { kk[mu] = rem % a.g.n[mu]; rem /= a.g.n[mu]; }
      rem = q;
      for (int mu = a.g.axis + 1; mu < a.g.d; ++mu) { kk[mu] = rem % a.g.n[mu]; rem /= a.g.n[mu]; }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
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
    split(e, t, j);
    const int64_t off = pbase[t] + P * j;
    T2 z[2];
    if (a.flags & PASS_PRO) {
      T2 in[2];
      in[0] = ldf<T2>(a.f.in[0], off);
      in[1] = a.f.nin > 1 ? ldf<T2>(a.f.in[1], off) : in[0];
      apply_prologue<T, T2>(a.op, in, z);
    } else {
      z[0] = ldf<T2>(a.f.work[0], off);
      if (NR > 1) z[1] = ldf<T2>(a.f.work[1], off);
    }
    tile0[t * pitch + j] = z[0];
    if (NR > 1) tile0[tile_stride + t * pitch + j] = z[1];
  }
  __syncthreads();

  // ---- transforms (all right-hand sides together)
  T2* cur = tile0;  // tile holding the data (mixed radix ping-pongs)
  if (a.flags & PASS_FWD) {
    if constexpr (MR) cur = mr_tile<T2, NR>(cur, cur == tile0 ? tile1 : tile0, tile_stride, pitch, n, tb, twp, false);
    else fft_tile<T, T2, NR>(tile0, tile_stride, pitch, n, logn, tb, tt, tf, false);
  }
  if (a.flags & PASS_MUL) {
    for (int e = threadIdx.x; e < cnt; e += kFftThreads) {
      int t, j;
      if (MR) { t = e / n; j = e - t * n; }
      else { t = e >> logn; j = e & (n - 1); }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const Symbol& S = a.sym[r];
        const T2 va = reinterpret_cast<const T2*>(S.vec[a.g.axis])[j];
        const T2 c = pfac[r * tbmax + t];
        const T2 f = S.sum_form ? cadd(c, va) : cmul(c, va);
        T2* sp = cur + r * tile_stride + t * pitch + j;
        *sp = cmul(*sp, f);
      }
    }
    __syncthreads();
  }
  if (a.flags & PASS_INV) {
    if constexpr (MR) cur = mr_tile<T2, NR>(cur, cur == tile0 ? tile1 : tile0, tile_stride, pitch, n, tb, twp + n, true);
    else fft_tile<T, T2, NR>(tile0, tile_stride, pitch, n, logn, tb, tt + 3 * n, tf + n, true);
  }

  // ---- store (+ epilogue)
  bool bad = false;
  for (int e = threadIdx.x; e < cnt; e += kFftThreads) {
    int t, j;
    split(e, t, j);
    const int64_t off = pbase[t] + P * j;
    T2 y[2];
    y[0] = cur[t * pitch + j];
    y[1] = NR > 1 ? cur[tile_stride + t * pitch + j] : y[0];
    if (a.flags & PASS_EPI) {
      T2 ex[kMaxExtra], o[2];
#pragma unroll
      for (int x = 0; x < kMaxExtra; ++x)
        if (x < a.f.nextra) ex[x] = ldf<T2>(a.f.extra[x], off);
      const int no = apply_epilogue<T, T2>(a.op, y, ex, o);
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        if (x < no && x < a.f.nout) {
          stf<T2>(a.f.out[x], off, o[x]);
          bad |= !finite2(o[x]);
        }
      }
    } else {
      stf<T2>(a.f.work[0], off, y[0]);
      if (NR > 1) stf<T2>(a.f.work[1], off, y[1]);
    }
  }
  if (bad && a.status) atomicOr(a.status, 1);
}

template <class T, int NR, bool MR = false>
__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(const FftPassArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fft_pass_body<T, NR, MR>(a, smem_raw);
}

// ---------------------------------------------------------------------------
// Four-step pass with the pencils in registers (FP32, 16 <= n <= 1024).  n = A * B with B = 2^ceil(log2(n)/2) >= A.  A pencil
// is held by A threads, thread t holding the B elements j = t + A r.  The
// DFT splits as X[s + B q] = sum_t w_A^(t q) w_n^(t s) sum_r x[t + A r] w_B^(r s):
// the inner B-point DFT runs in each thread's registers, then the twiddle
// w_n^(t s), then one transpose through shared memory (row s of a pencil's
// B x A block, padded rows and pencils so no two lanes of a half-warp share
// a bank), then A-point DFTs over t, again in registers.  Thread u ends up
// holding X[u + A r'], r' = 0..B-1: the same layout it loaded, so the symbol
// multiply and the inverse transform follow without another exchange, and
// a forward-symbol-inverse pass touches shared memory for two transposes
// where the Stockham pass above reads and writes its tile once per stage.
// Threads map to (pencil, t) with t fastest when pencils are contiguous
// (P = 1) and the pencil fastest otherwise, so every load and store of a
// warp covers whole contiguous runs.  All loads of a thread are issued before
// their first use.
// ---------------------------------------------------------------------------

constexpr size_t kFourStepExMax = 80 * 1024;  // above this, the fields share one exchange buffer

template <int LOGN> struct FourStep {
  static constexpr int n = 1 << LOGN;
  static constexpr int B = 1 << ((LOGN + 1) / 2);  // elements per thread
  static constexpr int A = n / B;                  // threads per pencil
  static constexpr int PP = kFftThreads / A;       // pencils per CTA
  static constexpr int RS = A + 1;                 // row stride of the exchange block
  static constexpr int PS = (B * RS) | 1;          // pencil stride (odd)
};

// One in-register Stockham stage of radix R on M values (all indices are
// compile-time): butterfly i (k = i mod P) takes v[i + r M/R], applies
// w_(PR)^(r k) (table entries of an n-point table, n = NTAB) and writes
// o[(i - k) R + k + r P].
template <class T, class T2, int M, int R, int P, int NTAB>
__device__ __forceinline__ void reg_stage(T2* v, const T* tt, const int* tf, bool inv) {
  constexpr int nb = M / R;
  constexpr int ts = NTAB / (P * R);
  T2 o[M];
#pragma unroll
  for (int i = 0; i < nb; ++i) {
    const int k = i % P;
    T2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[i + r * nb];
    if (k == 0) {
      if (R == 2) dft2(x);
      else dft4(x, inv);
    } else if (R == 2) {
      const Tw<T> w = load_tw(tt, tf, k * ts);
      fma_bfly<T, T2>(x[0], x[1], w);
    } else {
      const int m1 = k * ts;
      const Tw<T> w1 = load_tw(tt, tf, m1), w2 = load_tw(tt, tf, 2 * m1), w3 = load_tw(tt, tf, m1 + NTAB / 4);
      fma_bfly<T, T2>(x[0], x[2], w2);
      fma_bfly<T, T2>(x[1], x[3], w2);
      fma_bfly<T, T2>(x[0], x[1], w1);
      fma_bfly<T, T2>(x[2], x[3], w3);
      const T2 y1 = x[2];
      x[2] = x[1];
      x[1] = y1;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) o[(i - k) * R + k + r * P] = x[r];
  }
#pragma unroll
  for (int j = 0; j < M; ++j) v[j] = o[j];
}

// M-point DFT of v in registers, natural order in and out: radix-4 stages
// while they fit, then one radix-2 stage.
template <class T, class T2, int M, int P, int NTAB>
__device__ __forceinline__ void dft_reg(T2* v, const T* tt, const int* tf, bool inv) {
  if constexpr (P * 4 <= M) {
    reg_stage<T, T2, M, 4, P, NTAB>(v, tt, tf, inv);
    dft_reg<T, T2, M, P * 4, NTAB>(v, tt, tf, inv);
  } else if constexpr (P * 2 <= M) {
    reg_stage<T, T2, M, 2, P, NTAB>(v, tt, tf, inv);
  }
}

// One transform (forward or inverse) of the NR fields held by this thread.
// tt/tf/tw: this direction's tables; ex: exchange buffers.
template <class T, class T2, int NR, int LOGN>
__device__ __forceinline__ void four_step(T2 (&v)[NR][FourStep<LOGN>::B], T2* ex, int pp, int t, const T* tt,
                                          const int* tf, const T2* tw, bool inv) {
  using G = FourStep<LOGN>;
  constexpr int A = G::A, B = G::B, PS = G::PS, RS = G::RS, PP = G::PP;
  constexpr bool kSeq = (size_t)NR * PP * PS * sizeof(T2) > kFourStepExMax;
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) {
    dft_reg<T, T2, B, 1, G::n>(v[rr], tt, tf, inv);
#pragma unroll
    for (int s = 1; s < B; ++s) v[rr][s] = cmul(v[rr][s], tw[t * s]);
  }
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) {
    T2* e = ex + (kSeq ? 0 : rr * PP * PS) + pp * PS;
    if (kSeq || rr == 0) __syncthreads();  // earlier readers of the buffer are done
#pragma unroll
    for (int s = 0; s < B; ++s) e[s * RS + t] = v[rr][s];
    if (kSeq || rr == NR - 1) __syncthreads();
    if (kSeq || rr == NR - 1) {
#pragma unroll
      for (int r2 = kSeq ? rr : 0; r2 <= rr; ++r2) {
        const T2* e2 = ex + (kSeq ? 0 : r2 * PP * PS) + pp * PS;
#pragma unroll
        for (int m = 0; m < B / A; ++m) {
          T2 y[A];
#pragma unroll
          for (int tq = 0; tq < A; ++tq) y[tq] = e2[(t + A * m) * RS + tq];
          dft_reg<T, T2, A, 1, G::n>(y, tt, tf, inv);
#pragma unroll
          for (int q = 0; q < A; ++q) v[r2][m + (B / A) * q] = y[q];
        }
      }
    }
  }
}

template <class T, int NR, int LOGN>
__global__ void __launch_bounds__(kFftThreads) fft4_pass_kernel(const FftPassArgs a) {
  using T2 = typename C2<T>::type;
  using G = FourStep<LOGN>;
  constexpr int n = G::n, A = G::A, B = G::B, PP = G::PP, PS = G::PS;
  constexpr bool kSeq = (size_t)NR * PP * PS * sizeof(T2) > kFourStepExMax;
  constexpr int NX = kSeq ? 1 : NR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* ex = reinterpret_cast<T2*>(smem_raw);  // [NX][PP][PS]
  T2* tw = ex + NX * PP * PS;                // [2][n] plain twiddles (forward, inverse)
  T2* pfac = tw + 2 * n;                     // [kMaxRhs][PP]
  int64_t* pbase = reinterpret_cast<int64_t*>(pfac + kMaxRhs * PP);
  T* tt = reinterpret_cast<T*>(pbase + PP);  // [2][n][3]
  int* tf = reinterpret_cast<int*>(tt + 6 * n);

  const int64_t P = a.g.P;
  const int64_t b0 = (int64_t)blockIdx.x * PP;
  const int tb = (int)min((int64_t)PP, a.g.npencils - b0);
  const T* ttg = reinterpret_cast<const T*>(a.twiddle);
  for (int m = threadIdx.x; m < 6 * n; m += kFftThreads) tt[m] = ttg[m];
  for (int m = threadIdx.x; m < 2 * n; m += kFftThreads) {
    const int form = a.twform[m];
    const T tau = ttg[3 * m], mre = ttg[3 * m + 1], mim = ttg[3 * m + 2];
    tf[m] = form;
    tw[m] = form ? mk<T2>(tau * mre, mim) : mk<T2>(mre, tau * mre);
  }
  for (int t = threadIdx.x; t < tb; t += kFftThreads) {
    const int64_t b = b0 + t;
    const int64_t p = b % P, q = b / P;
    pbase[t] = p + P * (int64_t)n * q;
    if (a.flags & PASS_MUL) {
      int64_t kk[3] = {0, 0, 0};
      int64_t rem = p;
      for (int mu = 0; mu < a.g.axis; ++mu) { kk[mu] = rem % a.g.n[mu]; rem /= a.g.n[mu]; }
      rem = q;
      for (int mu = a.g.axis + 1; mu < a.g.d; ++mu) { kk[mu] = rem % a.g.n[mu]; rem /= a.g.n[mu]; }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const Symbol& S = a.sym[r];
        T2 acc = S.sum_form ? mk<T2>(0, 0) : mk<T2>(1, 0);
        for (int mu = 0; mu < a.g.d; ++mu) {
          if (mu == a.g.axis) continue;
          const T2 v = reinterpret_cast<const T2*>(S.vec[mu])[kk[mu]];
          acc = S.sum_form ? cadd(acc, v) : cmul(acc, v);
        }
        pfac[r * PP + t] = acc;
      }
    }
  }
  __syncthreads();

  int pp, t;
  if (P == 1) { t = threadIdx.x % A; pp = threadIdx.x / A; }
  else { pp = threadIdx.x % PP; t = threadIdx.x / PP; }
  const bool live = pp < tb;
  const int64_t base = live ? pbase[pp] : 0;

  // ---- load (+ prologue): element j = t + A r of pencil pp
  T2 v[NR][B];
#pragma unroll
  for (int rr = 0; rr < NR; ++rr)
#pragma unroll
    for (int r = 0; r < B; ++r) v[rr][r] = mk<T2>(0, 0);
  if (live) {
    if ((a.flags & PASS_PRO) && a.op.pro != PRO_NONE) {
      // an operator prologue: the first input field's loads first, parked in
      // this thread's own slots of the exchange buffer (free until the first
      // transpose, whose opening barrier orders these reads before its
      // writes); then the operator as a rolled loop over chunks of four
      // elements, each chunk appended at the top of v while v shifts down
      // by four, for the reason given at the store.  A second input field
      // (the coupled system's v) is read inside the loop.
      constexpr int CH = B < 4 ? B : 4;
      T2* park = ex + pp * PS;
      {
        T2 in0[B];
#pragma unroll
        for (int r = 0; r < B; ++r) in0[r] = ldf<T2>(a.f.in[0], base + P * (t + A * r));
#pragma unroll
        for (int r = 0; r < B; ++r) park[t + A * r] = in0[r];
      }
#pragma unroll 1
      for (int r0 = 0; r0 < B; r0 += CH) {
        T2 z0[CH], z1[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const T2 x = park[t + A * (r0 + c)];
          T2 in[2] = {x, x}, z[2];
          if (a.f.nin > 1) in[1] = ldf<T2>(a.f.in[1], base + P * (t + A * (r0 + c)));
          apply_prologue<T, T2>(a.op, in, z);
          z0[c] = z[0];
          z1[c] = z[1];
        }
#pragma unroll
        for (int r = 0; r + CH < B; ++r) {
          v[0][r] = v[0][r + CH];
          if (NR > 1) v[NR - 1][r] = v[NR - 1][r + CH];
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          v[0][B - CH + c] = z0[c];
          if (NR > 1) v[NR - 1][B - CH + c] = z1[c];
        }
      }
    } else if (a.flags & PASS_PRO) {
      // copy prologue: z_r = in_r
#pragma unroll
      for (int r = 0; r < B; ++r) {
        v[0][r] = ldf<T2>(a.f.in[0], base + P * (t + A * r));
        if (NR > 1) v[NR - 1][r] = ldf<T2>(a.f.in[a.f.nin > 1 ? 1 : 0], base + P * (t + A * r));
      }
    } else {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr)
#pragma unroll
        for (int r = 0; r < B; ++r) v[rr][r] = ldf<T2>(a.f.work[rr], base + P * (t + A * r));
    }
  }

  // ---- transforms
  if (a.flags & PASS_FWD) four_step<T, T2, NR, LOGN>(v, ex, pp, t, tt, tf, tw, false);
  if (a.flags & PASS_MUL) {
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
      const Symbol& S = a.sym[rr];
      const T2* va = reinterpret_cast<const T2*>(S.vec[a.g.axis]);
      const T2 c = pfac[rr * PP + (live ? pp : 0)];
#pragma unroll
      for (int r = 0; r < B; ++r) {
        const T2 e = va[t + A * r];
        v[rr][r] = cmul(v[rr][r], S.sum_form ? cadd(c, e) : cmul(c, e));
      }
    }
  }
  if (a.flags & PASS_INV) four_step<T, T2, NR, LOGN>(v, ex, pp, t, tt + 3 * n, tf + n, tw + n, true);

  // ---- store (+ epilogue).  The epilogue runs as a rolled loop over chunks
  // of four elements (extra inputs of a chunk loaded first); after each chunk
  // the register arrays shift down by four, so the loop body addresses fixed
  // registers and holds one short copy of the operator code: unrolled over
  // all B elements that code outgrew the instruction cache.
  if (!live) return;
  bool bad = false;
  if (a.flags & PASS_EPI) {
    constexpr int CH = B < 4 ? B : 4;
#pragma unroll 1
    for (int r0 = 0; r0 < B; r0 += CH) {
      T2 ex4[CH][kMaxExtra];
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int x = 0; x < kMaxExtra; ++x)
          if (x < a.f.nextra) ex4[c][x] = ldf<T2>(a.f.extra[x], base + P * (t + A * (r0 + c)));
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int64_t off = base + P * (t + A * (r0 + c));
        T2 y[2] = {v[0][c], v[NR - 1][c]}, o[2];
        const int no = apply_epilogue<T, T2>(a.op, y, ex4[c], o);
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          if (x < no && x < a.f.nout) {
            stf<T2>(a.f.out[x], off, o[x]);
            bad |= !finite2(o[x]);
          }
        }
      }
#pragma unroll
      for (int rr = 0; rr < NR; ++rr)
#pragma unroll
        for (int r = 0; r + CH < B; ++r) v[rr][r] = v[rr][r + CH];
    }
  } else {
#pragma unroll
    for (int rr = 0; rr < NR; ++rr)
#pragma unroll
      for (int r = 0; r < B; ++r) stf<T2>(a.f.work[rr], base + P * (t + A * r), v[rr][r]);
  }
  if (bad && a.status) atomicOr(a.status, 1);
}

template <class T, int LOGN> static size_t fft4_smem_bytes(int nrhs) {
  using G = FourStep<LOGN>;
  using T2 = typename C2<T>::type;
  const bool seq = (size_t)nrhs * G::PP * G::PS * sizeof(T2) > kFourStepExMax;
  const size_t nx = seq ? 1 : (size_t)nrhs;
  // exchange | plain twiddles | pencil factors | pencil bases | FMA twiddles | forms
  return nx * G::PP * G::PS * sizeof(T2) + 2 * (size_t)G::n * sizeof(T2) + (size_t)kMaxRhs * G::PP * sizeof(T2) +
         (size_t)G::PP * sizeof(int64_t) + 6 * (size_t)G::n * sizeof(T) + 2 * (size_t)G::n * sizeof(int);
}

// Largest log2 n the four-step pass handles for element type T.  FP64 keeps
// the Stockham pass: its FP64-bound passes run faster with the Stockham
// kernel's ~100 registers (two CTAs per SM) than with the four-step
// kernel's ~230 (one CTA per SM): 7.9e8 against 6.5e8 grid-pt.steps/s on
// the 128^3 split4 workload.
template <class T> constexpr int fft4_max_logn() { return sizeof(T) == 4 ? 10 : 0; }
constexpr int kFft4MinLogn = 4;

template <class T, int LOGN>
static cudaError_t launch_fft4(const FftPassArgs& a, cudaStream_t s) {
  using G = FourStep<LOGN>;
  const int64_t grid = (a.g.npencils + G::PP - 1) / G::PP;
  const size_t smem = fft4_smem_bytes<T, LOGN>(a.f.nrhs);
  if (a.f.nrhs > 1) fft4_pass_kernel<T, 2, LOGN><<<(unsigned)grid, kFftThreads, smem, s>>>(a);
  else fft4_pass_kernel<T, 1, LOGN><<<(unsigned)grid, kFftThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class T, int LOGN> static cudaError_t prepare_fft4() {
  cudaError_t e = cudaFuncSetAttribute(fft4_pass_kernel<T, 1, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fft4_smem_bytes<T, LOGN>(1));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fft4_pass_kernel<T, 2, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fft4_smem_bytes<T, LOGN>(2));
}

// Dispatch on log2 n (compile-time sizes).  Returns cudaErrorNotSupported
// for sizes outside [kFft4MinLogn, fft4_max_logn<T>()].
template <class T, int LOGN = kFft4MinLogn>
static cudaError_t fft4_dispatch(int logn, bool prepare, const FftPassArgs* a, cudaStream_t s) {
  if constexpr (LOGN > fft4_max_logn<T>()) {
    return cudaErrorNotSupported;
  } else {
    if (logn == LOGN) return prepare ? prepare_fft4<T, LOGN>() : launch_fft4<T, LOGN>(*a, s);
    return fft4_dispatch<T, LOGN + 1>(logn, prepare, a, s);
  }
}

static size_t fft_smem_bytes(int n, int nrhs, size_t elem, bool mr = false) {
  const int tbmax = std::max(1, (mr ? kFftTileMR : kFftTile) / n);
  const int pitch = n + 1;
  // tiles (two when mixed radix) | pencil factors | pencil bases | twiddles:
  // [2][n][3] of T + forms [2][n], or plain [2][n] of T2 (mixed radix)
  const size_t tw = mr ? (size_t)2 * n * elem + 16 : (size_t)6 * n * (elem / 2) + (size_t)2 * n * sizeof(int);
  return (size_t)tbmax * pitch * elem * nrhs * (mr ? 2 : 1) + (size_t)kMaxRhs * tbmax * elem +
         (size_t)tbmax * sizeof(int64_t) + tw;
}

bool fft_is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

template <class T> cudaError_t launch_fft_pass(const FftPassArgs& a, cudaStream_t s) {
  using T2 = typename C2<T>::type;
  const int n = (int)a.g.n_ax;
  const bool mr = !fft_is_pow2(n);
  const int tbmax = std::max(1, (mr ? kFftTileMR : kFftTile) / n);
  const int64_t grid = (a.g.npencils + tbmax - 1) / tbmax;
  if (mr) {
    const size_t smem = fft_smem_bytes(n, a.f.nrhs, sizeof(T2), true);
    if (smem > kFftMaxSmem || !a.twplain) return cudaErrorInvalidValue;
    if (a.f.nrhs > 1)
      fft_pass_kernel<T, 2, true><<<(unsigned)grid, kFftThreads, smem, s>>>(a);
    else
      fft_pass_kernel<T, 1, true><<<(unsigned)grid, kFftThreads, smem, s>>>(a);
    return cudaGetLastError();
  }
  const int logn = __builtin_ctz((unsigned)n);
  if (logn >= kFft4MinLogn && logn <= fft4_max_logn<T>()) return fft4_dispatch<T>(logn, false, &a, s);
  const size_t smem = fft_smem_bytes(n, a.f.nrhs, sizeof(T2));
  if (a.f.nrhs > 1)
    fft_pass_kernel<T, 2><<<(unsigned)grid, kFftThreads, smem, s>>>(a);
  else
    fft_pass_kernel<T, 1><<<(unsigned)grid, kFftThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Opt in to large dynamic shared memory; called at plan creation, outside any
// stream capture.
template <class T> cudaError_t prepare_fft_pass() {
  cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fft_pass_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fft_pass_kernel<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fft_pass_kernel<T, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem);
  if (e != cudaSuccess) return e;
  for (int logn = kFft4MinLogn; logn <= fft4_max_logn<T>(); ++logn)
    if ((e = fft4_dispatch<T>(logn, true, nullptr, nullptr)) != cudaSuccess) return e;
  return cudaSuccess;
}

template cudaError_t prepare_fft_pass<double>();
template cudaError_t prepare_fft_pass<float>();
template cudaError_t launch_fft_pass<double>(const FftPassArgs&, cudaStream_t);
template cudaError_t launch_fft_pass<float>(const FftPassArgs&, cudaStream_t);

}  // namespace cgl
