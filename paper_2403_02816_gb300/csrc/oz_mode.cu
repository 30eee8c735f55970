// FP64-accurate mu-mode product (Sec. 3.1, eq. Tucker) on the 5th-generation
// tensor cores by the Ozaki splitting (Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012; with
// integer slices as in Ootomo, Ozaki & Yokota, IJHPCA 2024).
//
// Each row of A (a fiber of the state: the 2n real values of one mode-mu
// line, components re and im) and each row of the real form of the factor
// (an output (c', i): the 2n values over (c, j)) is scaled by a power of two
// 2^e above its largest magnitude and cut into seven signed 7-bit digits:
//   x = 2^e sum_{a=0..6} d_a 2^{-7(a+1)} + r,   |d_0| <= 128, |d_a| <= 64,
//   |r| <= 2^{e-50}.
// Digit a is stored as the BF16 value d_a 2^{-7a} (exact: 8 significant
// bits, and the exponent range holds the scale), so the product of digits a
// and b carries its weight 2^{-7(a+b)} itself.  Products of one level
// L = a + b then share one power-of-two scale, and a level is one FP32
// tensor-memory accumulator whose partial sums are that scale times an
// integer below 2^24 for L <= 3 (K = 2n <= 512 terms: K (2 * 128 * 64 +
// (L - 1) 64 * 64) <= 2^24), i.e. exact whatever the accumulation order and
// rounding.  Levels 4..6 (relative weights 2^-28..2^-42) are FP32
// accumulators too, summed into one tail in the epilogue, whose rounding
// stays below 2^-46 of level 0.  The 28 products with a + b <= 6 are BF16
// GEMMs; the dropped products (a + b >= 7) and the digit remainders r are
// below 2^-46 of the row scales' product.  The epilogue turns the four exact
// levels into their integers (exact 32-bit conversions), rounds the tail at
// 2^-31 of level 0, combines them in 64-bit integer arithmetic, converts once
// to FP64 and applies the two power-of-two scales.
//
// The seven level accumulators are consecutive blocks of nc TMEM columns
// (level L at columns [L nc, (L + 1) nc)), and the factor's digit planes
// are consecutive blocks of nc rows in shared memory, so one MMA of A digit a
// against B digits b0..b1 (N = (b1 - b0 + 1) nc <= 256) writes product
// (a, b) straight into block a + b, its level: about ten MMAs per K step
// instead of 28, each reading its A digit from shared memory once.
//
// A pass is: slice the FP64 state planes of the mode's fibers (per-fiber
// exponent), then the tensor-core GEMM writing FP64 planes.  One CTA =
// 128 fibers (TMEM lanes) x nc <= 64 output rows of one component; the seven
// level accumulators take 7 nc <= 448 TMEM columns.  Pipeline, copy / MMA
// thread roles, bounded waits and the abort path follow the BF16x3 pass.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "cgl_internal.cuh"
#include "tc_ptx.cuh"

namespace cgl {

constexpr int kOzThreads = 128;
constexpr int kOzM = 128;
constexpr int kOzK = 16;       // K of one tcgen05.mma
constexpr int kOzStageK = 32;  // K per pipeline stage
constexpr int kOzStages = 2;
constexpr uint32_t kOzKRowBytes = kOzStageK * 2;  // K-major rows: 64 bytes, 64-byte swizzle
constexpr uint32_t kOzKSwizzleDesc = 4;

// ------------------------------------------------------------------ slicing

// |x| as an ordered integer (positive doubles order like their bit patterns).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

// Exponent e with |x| < 2^e for every x of a row whose largest |x| has the
// bit pattern `mx` (e = biased exponent - 1022; any e for an all-zero row).
__device__ __forceinline__ int row_exponent(unsigned long long mx) {
  return static_cast<int>((mx >> 52) & 0x7FF) - 1022;
}

// round(x 2^{49 - e}) for |x| < 2^e, from the bits of x (integer arithmetic
// only): |result| <= 2^49.
__device__ __forceinline__ long long fixed49(double x, int e) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (E) m |= 1ull << 52;
  // x = m 2^{max(E, 1) - 1075}; |x| < 2^e makes the shift <= -3
  const int r = e - 49 + 1075 - (E ? E : 1);
  long long v = 0;
  if (r >= 1 && r < 63) v = static_cast<long long>((m + (1ull << (r - 1))) >> r);
  return (b >> 63) ? -v : v;
}

// Seven signed digits of v (|v| <= 2^49), most significant first:
// v = sum_a d_a 2^{7(6 - a)}, |d_0| <= 128, -64 <= d_a <= 63 for a >= 1.
// Balanced base-128 recoding: with t = v + 64 sum_a 2^{7a}, every 7-bit field
// of t below the top one is d_a + 64, and t >> 42 is d_0 + 64 (one 64-bit
// add and seven field extractions instead of a rounding division per digit).
__device__ __forceinline__ void digits7(long long v, int* d) {
  constexpr long long kOff = 64ll * ((1ll << 42) + (1ll << 35) + (1ll << 28) + (1ll << 21) + (1ll << 14) +
                                     (1ll << 7) + 1ll);
  const long long t = v + kOff;
  d[0] = static_cast<int>(t >> 42) - 64;
#pragma unroll
  for (int k = 1; k < 7; ++k) d[k] = static_cast<int>((t >> (7 * (6 - k))) & 127) - 64;
}

// Digit d (|d| <= 128) of position s as the BF16 value d 2^{-7s} (exact).
__device__ __forceinline__ __nv_bfloat16 digit_bf16(int d, int s) {
  return __float2bfloat16_rn(static_cast<float>(d) * __int_as_float((127 - 7 * s) << 23));
}

__device__ __forceinline__ int64_t oz_plane_index(int64_t i, int64_t n1, int64_t pitch) {
  return pitch == n1 ? i : i + (pitch - n1) * (i / n1);
}

// Mode 1 (contiguous fibers): one warp per fiber q, values z[c][pitch q + j].
__global__ void oz_slice_rows_kernel(const OzSliceArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < a.Q; q += nwarps) {
    const double* zr = a.z + a.pitch * q;
    const double* zi = zr + a.N;
    unsigned long long mx = 0;
    for (int j = lane; j < a.n; j += 32) mx = max(mx, max(abs_bits(zr[j]), abs_bits(zi[j])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (mx >= 0x7FF0000000000000ull) {
      if (lane == 0) atomicOr(a.status, 1);  // non-finite state
      mx = 0;
    }
    const int e = row_exponent(mx);
    if (lane == 0) a.exps[q] = e;
    for (int j = lane; j < a.n; j += 32) {
      int dr[7], di[7];
      digits7(fixed49(zr[j], e), dr);
      digits7(fixed49(zi[j], e), di);
      const int64_t o = a.pitch * q + j;
#pragma unroll
      for (int s = 0; s < 7; ++s) {
        a.dst[(2 * s) * a.N + o] = digit_bf16(dr[s], s);
        a.dst[(2 * s + 1) * a.N + o] = digit_bf16(di[s], s);
      }
    }
  }
}

// Modes > 1 (strided fibers): one thread per fiber (p, q), values
// z[c][p + P j + P n q]; consecutive threads take consecutive p.
__global__ void oz_slice_cols_kernel(const OzSliceArgs a) {
  const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  for (int64_t q = blockIdx.y; q < a.Q; q += gridDim.y) {
    const int64_t base = p + a.P * a.n * q;
    unsigned long long mx = 0;
    for (int j = 0; j < a.n; ++j)
      mx = max(mx, max(abs_bits(a.z[base + a.P * j]), abs_bits(a.z[a.N + base + a.P * j])));
    if (mx >= 0x7FF0000000000000ull) {
      atomicOr(a.status, 1);
      mx = 0;
    }
    const int e = row_exponent(mx);
    a.exps[q * a.P + p] = e;
    for (int j = 0; j < a.n; ++j) {
      const int64_t o = base + a.P * j;
      int dr[7], di[7];
      digits7(fixed49(a.z[o], e), dr);
      digits7(fixed49(a.z[a.N + o], e), di);
#pragma unroll
      for (int s = 0; s < 7; ++s) {
        a.dst[(2 * s) * a.N + o] = digit_bf16(dr[s], s);
        a.dst[(2 * s + 1) * a.N + o] = digit_bf16(di[s], s);
      }
    }
  }
}

// Real form of an FP64 factor F (n x n, column-major), rows (c', i) over K =
// (c, j) (row (0, i): [Fr_i., -Fi_i.], row (1, i): [Fi_i., Fr_i.]), each row
// i scaled by 2^{fexp[i]} above its largest entry and cut into seven digits:
// out[s][row][col], zero-padded to 2np x 2np.  One block per i < np.
__global__ void oz_factor_slice_kernel(const double2* F, int n, int np, __nv_bfloat16* out, int* fexp) {
  const int i = blockIdx.x;
  __shared__ unsigned long long red[32];
  unsigned long long mx = 0;
  if (i < n)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double2 f = F[i + static_cast<int64_t>(j) * n];
      mx = max(mx, max(abs_bits(f.x), abs_bits(f.y)));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
    red[0] = mx;
  }
  __syncthreads();
  const int e = row_exponent(red[0]);
  if (threadIdx.x == 0) fexp[i] = e;
  const int64_t K = 2ll * np, total = 4ll * np * np;
  for (int col = threadIdx.x; col < 2 * np; col += blockDim.x) {
    const int c = col / np, j = col % np;
    double2 f = make_double2(0.0, 0.0);
    if (i < n && j < n) f = F[i + static_cast<int64_t>(j) * n];
    const double v0 = (c == 0) ? f.x : -f.y;  // row (re, i)
    const double v1 = (c == 0) ? f.y : f.x;   // row (im, i)
    int d0[7], d1[7];
    digits7(fixed49(v0, e), d0);
    digits7(fixed49(v1, e), d1);
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      out[s * total + static_cast<int64_t>(i) * K + col] = digit_bf16(d0[s], s);
      out[s * total + static_cast<int64_t>(np + i) * K + col] = digit_bf16(d1[s], s);
    }
  }
}

// ------------------------------------------------------------------ pointwise stages

// Start of a sweep: prologue in FP64 on complex128 inputs -> FP64 planes
// (re, im) of each rhs, first direction padded to `pitch`.
__global__ void oz_prologue_kernel(const OzSeg g, int nrhs) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < g.N;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double2 in[2], z[2];
    in[0] = g.in[0][i];
    in[1] = g.nin > 1 ? g.in[1][i] : in[0];
    apply_prologue<double, double2>(g.op, in, z);
    const int64_t ip = oz_plane_index(i, g.n1, g.pitch);
    for (int r = 0; r < nrhs; ++r) {
      g.z[r][ip] = z[r].x;
      g.z[r][g.Npad + ip] = z[r].y;
    }
  }
}

// End of a sweep: FP64 planes of each rhs + extras -> epilogue -> complex128.
__global__ void oz_epilogue_kernel(const OzSeg g, int nrhs, int* status) {
  bool bad = false;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < g.N;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t ip = oz_plane_index(i, g.n1, g.pitch);
    double2 y[2], ex[kMaxExtra], o[2];
    y[0] = make_double2(g.z[0][ip], g.z[0][g.Npad + ip]);
    y[1] = nrhs > 1 ? make_double2(g.z[1][ip], g.z[1][g.Npad + ip]) : y[0];
    for (int x = 0; x < g.nextra; ++x) ex[x] = g.ex[x][i];
    const int no = apply_epilogue<double, double2>(g.op, y, ex, o);
    if (no > 0 && g.nout > 0) { g.out[0][i] = o[0]; bad |= !finite2(o[0]); }
    if (no > 1 && g.nout > 1) { g.out[1][i] = o[1]; bad |= !finite2(o[1]); }
  }
  if (bad && status) atomicOr(status, 1);
}

// ------------------------------------------------------------------ the GEMM pass

static __host__ __device__ constexpr uint32_t oz_stage_bytes(int nc) {
  return 7u * (kOzM * kOzStageK * 2u) + 7u * (static_cast<uint32_t>(nc) * kOzStageK * 2u);
}

// 32 lanes x 32 bit, 16 consecutive columns; the caller waits (tcgen05.wait::ld).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// 2^k as a double (0 below the normal range).
__device__ __forceinline__ double pow2(int k) {
  return k < -1022 ? 0.0 : __longlong_as_double(static_cast<long long>(k + 1023) << 52);
}

// CTA (tile, half, sub): 128 fibers x output rows [sub nc, (sub + 1) nc) of
// component c' = half; TMEM columns [L nc, (L + 1) nc) hold level L.
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_mode_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                   const OzPassArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int rhs = blockIdx.y;
  const int64_t bx = blockIdx.x;
  const CUtensorMap* tmA = rhs ? &tmA1 : &tmA0;
  const CUtensorMap* tmB = rhs ? &tmB1 : &tmB0;
  const int n = a.n, np = a.np, nc = a.nc;
  const int nkc = (np + kOzStageK - 1) / kOzStageK;
  const int nk = 2 * nkc;  // K = 2 np over (component c, position j)
  const uint32_t a_bytes = kOzM * kOzStageK * 2;
  const uint32_t b_bytes = static_cast<uint32_t>(nc) * kOzStageK * 2;
  const uint32_t stage_bytes = oz_stage_bytes(nc);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kOzStages * stage_bytes);
  uint64_t* empty = full + kOzStages;
  uint64_t* accum = empty + kOzStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* counters = abort_flag + 1;  // stages loaded / consumed / committed
  const int warp = threadIdx.x >> 5;

  const int64_t tile = bx / (2 * a.nsub);
  const int part = static_cast<int>(bx % (2 * a.nsub));
  const int half = part / a.nsub;
  const int sub = part % a.nsub;
  int64_t q0 = 0, p0 = 0;
  if (a.a_mn) {
    q0 = tile / a.per_q;
    p0 = (tile - q0 * a.per_q) * kOzM;
  } else {
    q0 = tile * kOzM;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accum), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 32) {
    int slot = 0, c = 0, j0 = 0, loaded = 0;
    uint32_t phase = 0;
    bool ok = true;
    const int rowB = half * np + sub * nc, pq = static_cast<int>(p0 / 64);
    for (int kb = 0; kb < nk; ++kb) {
      if (kb >= kOzStages && !mbar_wait(smem_u32(&empty[slot]), phase ^ 1u)) { ok = false; break; }
      const uint32_t st = smem_u32(base + slot * stage_bytes), bar = smem_u32(&full[slot]);
      mbar_expect_tx(bar, stage_bytes);
      if (a.a_mn)
        tma_load_5d(st, tmA, bar, 0, j0, pq, static_cast<int>(q0 + a.Q * c), 0);
      else
        tma_load_4d(st, tmA, bar, j0, static_cast<int>(q0), c, 0);
      tma_load_4d(st + 7 * a_bytes, tmB, bar, j0, rowB, c, 0);
      loaded = kb + 1;
      if (++slot == kOzStages) { slot = 0; phase ^= 1u; }
      j0 += kOzStageK;
      if (j0 >= np) { j0 = 0; ++c; }
    }
    counters[0] = loaded;
    if (!ok) *abort_flag = 1;
  }
  if (threadIdx.x == 0) {
    // digits of B per MMA: N = span nc <= 256
    const int span = min(7, 256 / nc);
    const uint64_t a0 = a.a_mn ? smem_desc(smem_u32(base), kOzStageK * 128u, 1024, 2)
                               : smem_desc(smem_u32(base), 16, 8 * kOzKRowBytes, kOzKSwizzleDesc);
    const uint64_t b0 = smem_desc(smem_u32(base + 7 * a_bytes), 16, 8 * kOzKRowBytes, kOzKSwizzleDesc);
    const uint32_t a_ks = a.a_mn ? 2048u / 16 : 32u / 16, b_ks = 32u / 16;
    const uint32_t a_sp = a_bytes / 16, b_sp = b_bytes / 16;
    int slot = 0, j0 = 0, consumed = 0, committed = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      if (!mbar_wait(smem_u32(&full[slot]), phase)) { ok = false; break; }
      consumed = kb + 1;
      tc_fence_after();
      const uint32_t so = slot * (stage_bytes / 16);
      const int ksteps = min(kOzStageK, np - j0) / kOzK;
      for (int ks = 0; ks < ksteps; ++ks) {
        const bool first = kb == 0 && ks == 0;
        // A digit x against B digits y0 .. y0 + cnt - 1 into level blocks
        // x + y0 ..; the MMAs of digit 0 cover all seven blocks and come
        // first, so at the first K step they overwrite and the rest add
#pragma unroll
        for (int x = 0; x < 7; ++x) {
          const uint64_t ad = a0 + (so + x * a_sp + ks * a_ks);
          for (int y0 = 0; y0 <= 6 - x; y0 += span) {
            const int cnt = min(span, 7 - x - y0);
            const uint64_t bd = b0 + (so + y0 * b_sp + ks * b_ks);
            mma_bf16(tmem + static_cast<uint32_t>((x + y0) * nc), ad, bd, idesc_bf16(kOzM, cnt * nc, a.a_mn),
                     (first && x == 0) ? 0u : 1u);
          }
        }
      }
      mma_commit(smem_u32(&empty[slot]));
      committed = kb + 1;
      if (++slot == kOzStages) { slot = 0; phase ^= 1u; }
      j0 += kOzStageK;
      if (j0 >= np) j0 = 0;
    }
    counters[1] = consumed;
    counters[2] = committed;
    if (ok) mma_commit(smem_u32(accum));
    else *abort_flag = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    atomicOr(a.status, 2);
    const int loaded = counters[0], consumed = counters[1], committed = counters[2];
    for (int kb = consumed; kb < loaded; ++kb) mbar_wait(smem_u32(&full[kb % kOzStages]), (kb / kOzStages) & 1);
    if (committed > 0)
      mbar_wait(smem_u32(&empty[(committed - 1) % kOzStages]), ((committed - 1) / kOzStages) & 1);
  }
  __syncthreads();

  bool good = (*abort_flag == 0);
  if (good && !mbar_wait(smem_u32(accum), 0)) {
    good = false;
    atomicOr(a.status, 2);
  }
  good = __syncthreads_and(good) != 0;
  tc_fence_after();
  if (good) {
    const int m = threadIdx.x;  // TMEM lane = fiber of the tile
    const uint32_t lane_addr = static_cast<uint32_t>(warp * 32) << 16;
    // this fiber's exponent (fibers past the slab end read as exponent 0;
    // their outputs are not stored)
    int ea = 0;
    if (a.a_mn) {
      if (p0 + m < a.P) ea = a.aexp[rhs][q0 * a.P + p0 + m];
    } else {
      if (q0 + m < a.Q) ea = a.aexp[rhs][q0 + m];
    }
    const int* fe = a.bexp[rhs];
    double* out = a.out[rhs] + static_cast<int64_t>(half) * a.N;
    const int64_t tile0 = p0 + a.P * static_cast<int64_t>(n) * q0;
    const bool store_mn = a.a_mn && (p0 + m < a.P);
    const int pitch_s = nc + 1;  // mode 1: FP64 staging tile [128][nc + 1]
    double* stage = reinterpret_cast<double*>(base);
    for (int c0 = 0; c0 < nc; c0 += 16) {
      uint32_t r[7][16];
#pragma unroll
      for (int L = 0; L < 7; ++L) tmem_ld16_nowait(tmem + lane_addr + static_cast<uint32_t>(L * nc + c0), r[L]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int i = sub * nc + c0 + t;  // output row of component `half`
        // accumulator k < 4 holds 2^{-7k} x an integer below 2^24: scaled by
        // 2^{7k} it converts to int32 exactly; the tail, levels 4..6 (below
        // 0.06 in level-0 units), is rounded at 2^-31 of them.  (Conversions to 32-bit
        // integers: a float-to-int64 conversion per accumulator made the pass
        // 20% slower.)
        long long I = static_cast<long long>(__float2int_rn(__uint_as_float(r[0][t]))) * (1ll << 31);
        I += static_cast<long long>(__float2int_rn(__uint_as_float(r[1][t]) * 128.0f)) * (1ll << 24);
        I += static_cast<long long>(__float2int_rn(__uint_as_float(r[2][t]) * 16384.0f)) * (1ll << 17);
        I += static_cast<long long>(__float2int_rn(__uint_as_float(r[3][t]) * 2097152.0f)) * (1ll << 10);
        const float tail = __uint_as_float(r[4][t]) + (__uint_as_float(r[5][t]) + __uint_as_float(r[6][t]));
        I += static_cast<long long>(__float2int_rn(tail * 2147483648.0f));
        // sum_{a,b} d_a d'_b 2^{-7(a+b+2)} = I 2^{-45}, times 2^{ea + fe[i]}
        const double v = static_cast<double>(I) * pow2(ea + (i < np ? fe[i] : 0) - 45);
        if (a.a_mn) {
          if (store_mn && i < n) out[tile0 + a.P * i + m] = v;
        } else {
          stage[m * pitch_s + c0 + t] = v;
        }
      }
    }
    if (!a.a_mn) {
      __syncthreads();
      // each fiber's nc outputs are one contiguous run of the plane
      for (int e = threadIdx.x; e < kOzM * nc; e += kOzThreads) {
        const int f = e / nc, t = e - f * nc;
        const int64_t q = q0 + f;
        const int i = sub * nc + t;
        if (q < a.Q && i < n) out[a.pitch * q + i] = stage[f * pitch_s + t];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// ------------------------------------------------------------------ host side

static size_t oz_smem_bytes(int nc) { return kOzStages * static_cast<size_t>(oz_stage_bytes(nc)) + 1024 + 256; }

// Output rows per CTA: the whole np up to 64 rows, else blocks of 48 or 64
// rows with the fewest rows past np (64 on ties): seven level accumulators of
// nc columns fit the 512 of TMEM up to nc = 73.  (With five accumulators,
// levels 4..6 sharing one, blocks of 64 and 96 rows ran at the same fraction
// of the tensor peak on the 256^3 Lawson4 step, so the rows computed past np
// decide.)
int oz_rows_per_cta(int np) {
  if (np <= 64) return np;
  const int w64 = (np + 63) / 64 * 64 - np, w48 = (np + 47) / 48 * 48 - np;
  return w48 < w64 ? 48 : 64;
}

size_t oz_factor_bytes(int n) {
  const size_t np = mma_pad16(n);
  return 7 * 4 * np * np * 2;
}

cudaError_t prepare_oz_pass() {
  return cudaFuncSetAttribute(oz_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(oz_smem_bytes(64)));
}

int64_t oz_build_args(const OzLaunch& L, OzPassArgs* out) {
  OzPassArgs a{};
  a.n = L.n;
  a.np = mma_pad16(L.n);
  a.P = L.P;
  a.Q = L.Q;
  a.pitch = L.pitch;
  a.per_q = (L.P + kOzM - 1) / kOzM;
  a.a_mn = L.P > 1 ? 1 : 0;
  a.N = L.N;
  a.nc = oz_rows_per_cta(a.np);
  a.nsub = (a.np + a.nc - 1) / a.nc;
  int cols = 32;
  while (cols < 7 * a.nc) cols *= 2;
  a.tmem_cols = cols;
  for (int r = 0; r < kMaxRhs; ++r) {
    a.aexp[r] = L.aexp[r];
    a.bexp[r] = L.bexp[r];
    a.out[r] = L.out[r];
  }
  a.status = L.status;
  *out = a;
  if (L.n < 1 || L.n > 256 || (a.a_mn && L.P % 64 != 0) || (!a.a_mn && L.pitch < a.np)) return -1;
  // mode 1 stages its FP64 tile [128][nc + 1] in the pipeline buffers
  if (!a.a_mn && static_cast<size_t>(kOzM) * (a.nc + 1) * 8 > kOzStages * static_cast<size_t>(oz_stage_bytes(a.nc)))
    return -1;
  const int64_t mtiles = a.a_mn ? a.per_q * L.Q : (L.Q + kOzM - 1) / kOzM;
  return 2 * a.nsub * mtiles;
}

cudaError_t launch_oz_pass(const OzLaunch& L, cudaStream_t s) {
  OzPassArgs a;
  const int64_t ctas = oz_build_args(L, &a);
  if (ctas < 0) return cudaErrorInvalidValue;
  const CUtensorMap* A0 = reinterpret_cast<const CUtensorMap*>(L.tmA[0]);
  const CUtensorMap* A1 = reinterpret_cast<const CUtensorMap*>(L.tmA[L.nrhs > 1 ? 1 : 0]);
  const CUtensorMap* B0 = reinterpret_cast<const CUtensorMap*>(L.tmB[0]);
  const CUtensorMap* B1 = reinterpret_cast<const CUtensorMap*>(L.tmB[L.nrhs > 1 ? 1 : 0]);
  dim3 grid(static_cast<unsigned>(ctas), static_cast<unsigned>(L.nrhs));
  oz_mode_kernel<<<grid, kOzThreads, oz_smem_bytes(a.nc), s>>>(*A0, *A1, *B0, *B1, a);
  return cudaGetLastError();
}

cudaError_t launch_oz_slice(const OzSliceArgs& a, cudaStream_t s) {
  if (a.P == 1) {
    const int64_t blocks = std::min<int64_t>((a.Q + 7) / 8, 152 * 16);
    oz_slice_rows_kernel<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, s>>>(a);
  } else {
    const unsigned bx = static_cast<unsigned>((a.P + 127) / 128);
    const unsigned by = static_cast<unsigned>(std::min<int64_t>(a.Q, 65535));
    oz_slice_cols_kernel<<<dim3(bx, by), 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_oz_factor_slice(const double2* F, int n, void* out, int* fexp, cudaStream_t s) {
  const int np = mma_pad16(n);
  oz_factor_slice_kernel<<<np, 256, 0, s>>>(F, n, np, static_cast<__nv_bfloat16*>(out), fexp);
  return cudaGetLastError();
}

cudaError_t launch_oz_prologue(const OzSeg& g, int nrhs, cudaStream_t s) {
  const unsigned bx = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((g.N + 255) / 256, 152 * 16)));
  oz_prologue_kernel<<<bx, 256, 0, s>>>(g, nrhs);
  return cudaGetLastError();
}

cudaError_t launch_oz_epilogue(const OzSeg& g, int nrhs, int* status, cudaStream_t s) {
  const unsigned bx = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((g.N + 255) / 256, 152 * 16)));
  oz_epilogue_kernel<<<bx, 256, 0, s>>>(g, nrhs, status);
  return cudaGetLastError();
}

}  // namespace cgl
