// mu-mode product (Sec. 3.1, eq. Tucker) on the 5th-generation tensor cores:
// BF16x3 split operands, FP32 accumulation in tensor memory.
//
// Complex contraction as a real GEMM.  For mode mu with fibers m (the other
// coordinates) the product v = F u over each fiber is
//   C[m, (c', i)] = sum_{(c, j)} A[m, (c, j)] B[(c, j), (c', i)],
// c, c' in {re, im}, A[m, (c, j)] = component c of u at position j of fiber m,
// B the real form of F: [[Fr, -Fi], [Fi, Fr]] laid out as N rows (c', i) of K
// = 2n contiguous values.  The state is held as three BF16 planes per
// component (x = h + m + l, h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)),
// the factor likewise (split once from FP64), and six products
// (lh, hl, mm, mh, hm, hh) accumulate in FP32 tensor memory: about 24
// significant bits, i.e. FP32 accuracy.
//
// Kernel shape: one CTA per tile of 128 fibers (TMEM lanes) x one block of
// output rows of one component (re or im; nc = n or n/2 <= 128 rows, so that
// two CTAs share an SM and one's epilogue overlaps the other's MMAs), with the
// (h,h) product and the five correction products in separate TMEM
// accumulators that the epilogue adds in FP32.  K advances kStageK per
// pipeline stage, two stages within half an SM's shared memory; one thread
// fills a stage with one TMA copy for the three A splits and one for the
// three B splits (A: K-major for mode 1 whose fibers are contiguous, MN-major
// for the other modes; B: K-major), another issues its tcgen05.mma and frees
// it with tcgen05.commit.  The copy engine's cost goes with the number of
// copies and the issuing threads' with their instruction count, so both are
// kept minimal: a few large boxes, incremental slot / phase / descriptor
// arithmetic.  Every mbarrier wait is bounded: on
// timeout the kernel sets bit 1 of the status word, skips its stores, waits
// (bounded) for its own copies, frees its TMEM and returns.
//
// A pass must not write over its input: the CTAs of one fiber tile (its
// components and row blocks) all read the tile's whole input.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "cgl_internal.cuh"
#include "tc_ptx.cuh"

namespace cgl {

constexpr int kMmaThreads = 128;
constexpr int kMmaM = 128;
constexpr int kMmaK = 16;  // K of one tcgen05.mma
// K per pipeline stage (one copy per operand) and stages per CTA.  Measured on
// the 256^3 mode passes (ms per pass, two CTAs per SM unless noted): K 16 x 4
// stages 0.390, K 32 x 2 stages 0.332, K 32 x 3 stages (one CTA per SM)
// 0.469, K 32 x 4 / K 64 x 2 (one CTA per SM, issue on one thread) 0.56.
constexpr int kStageK = 32;
constexpr int kMaxStages = 2;
constexpr int kSmemPerCta = 113 * 1024;  // two CTAs per SM
// K-major rows of kStageK BF16 values: swizzle span = row bytes
constexpr uint32_t kKRowBytes = kStageK * 2;
constexpr uint32_t kKSwizzleDesc = kKRowBytes == 32 ? 6 : kKRowBytes == 64 ? 4 : 2;


__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

// ------------------------------------------------------------------ the GEMM pass

// One pipeline stage: three A splits (128 fibers x kStageK) and three B
// splits (nc output rows x kStageK).
static __host__ __device__ constexpr uint32_t mma_stage_bytes(int nc) {
  return 3u * (kMmaM * kStageK * 2u) + 3u * (static_cast<uint32_t>(nc) * kStageK * 2u);
}

// CTA (tile, half, sub): 128 fibers x output rows [sub nc, (sub + 1) nc) of
// component c' = half.  TMEM columns [0, nc): the (h, h) product; [nc, 2nc):
// the five correction products.  Keeping the large term in its own
// accumulator keeps the accumulator rounding of the many small MMAs relative
// to the small terms.  Rows i >= n (padding, or the other component's rows
// when nsub nc > np) are computed and discarded.
__global__ void __launch_bounds__(kMmaThreads, 1)
    mma_mode_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                    const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                    const MmaPassArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int rhs = blockIdx.y;
  const int64_t bx = blockIdx.x;
  const CUtensorMap* tmA = rhs ? &tmA1 : &tmA0;
  const CUtensorMap* tmB = rhs ? &tmB1 : &tmB0;
  const int n = a.n, np = a.np;
  // K = 2 np runs over (component c, position j); a stage holds kStageK
  // values of j of one component (the copies fill j >= n with zeros)
  const int nkc = (np + kStageK - 1) / kStageK;
  const int nk = 2 * nkc;
  const int S = a.stages;
  const uint32_t a_bytes = kMmaM * kStageK * 2;
  const int nc = a.nc;
  const uint32_t b_bytes = static_cast<uint32_t>(nc) * kStageK * 2;
  const uint32_t stage_bytes = mma_stage_bytes(nc);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* accum = empty + S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5;

  // the two halves of a fiber tile are adjacent blocks, so the second read
  // of the tile's A data is served from L2
  // CTA (tile, component, row block); the CTAs of one fiber tile are adjacent
  // blocks, so the repeated reads of the tile's A data are served from L2
  const int64_t tile = bx / (2 * a.nsub);
  const int part = (int)(bx % (2 * a.nsub));
  const int half = part / a.nsub;
  const int sub = part % a.nsub;
  int64_t q0 = 0, p0 = 0;
  if (a.a_mn) {
    q0 = tile / a.per_q;
    p0 = (tile - q0 * a.per_q) * kMmaM;  // a last tile of 64 fibers reads zeros for its second half
  } else {
    q0 = tile * kMmaM;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
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
  const uint32_t d_main = tmem, d_corr = tmem + nc;

  // thread 32 copies stages in as slots free up; thread 0 issues the MMAs
  // of each stage as it lands and frees the slot with tcgen05.commit.  Slot
  // and phase advance incrementally (no divisions on the issuing threads).
  int* counters = abort_flag + 1;  // stages loaded / consumed / committed
  if (threadIdx.x == 32) {
    int slot = 0, c = 0, j0 = 0, loaded = 0;
    uint32_t phase = 0;
    bool ok = true;
    const int rowB = half * np + sub * nc, pq = (int)(p0 / 64);
    for (int kb = 0; kb < nk; ++kb) {
      // the slot's previous stage (kb - S) must have been consumed
      if (kb >= S && !mbar_wait(smem_u32(&empty[slot]), phase ^ 1u)) { ok = false; break; }
      const uint32_t st = smem_u32(base + slot * stage_bytes), bar = smem_u32(&full[slot]);
      mbar_expect_tx(bar, stage_bytes);
      // one box each for the three A splits and the three B splits
      if (a.a_mn)
        tma_load_5d(st, tmA, bar, 0, j0, pq, (int)(q0 + a.Q * c), 0);
      else
        tma_load_4d(st, tmA, bar, j0, (int)q0, c, 0);
      tma_load_4d(st + 3 * a_bytes, tmB, bar, j0, rowB, c, 0);
      loaded = kb + 1;
      if (++slot == S) { slot = 0; phase ^= 1u; }
      j0 += kStageK;
      if (j0 >= np) { j0 = 0; ++c; }
    }
    counters[0] = loaded;
    if (!ok) *abort_flag = 1;
  }
  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_bf16(kMmaM, nc, a.a_mn);
    // descriptors of slot 0 / split 0 / K step 0; the other operands differ
    // only in the start address (16-byte units in the low bits).  MN-major A:
    // two 64-fiber halves of kStageK rows of 128 B, 8-row groups 1024 B
    // apart, one K step = 16 rows = 2048 B.  K-major A / B: rows of
    // kKRowBytes, 8-row groups 8 rows apart, one K step = 32 B along the
    // (swizzled) row.
    const uint64_t a0 = a.a_mn ? smem_desc(smem_u32(base), kStageK * 128u, 1024, 2)
                               : smem_desc(smem_u32(base), 16, 8 * kKRowBytes, kKSwizzleDesc);
    const uint64_t b0 = smem_desc(smem_u32(base + 3 * a_bytes), 16, 8 * kKRowBytes, kKSwizzleDesc);
    const uint32_t a_ks = a.a_mn ? 2048u / 16 : 32u / 16, b_ks = 32u / 16;
    const uint32_t a_sp = a_bytes / 16, b_sp = b_bytes / 16;
    // split products: five corrections (l,h) (h,l) (m,m) (m,h) (h,m), then (h,h)
    constexpr uint32_t pa[6] = {2, 0, 1, 1, 0, 0};
    constexpr uint32_t pb[6] = {0, 2, 1, 0, 1, 0};
    int slot = 0, j0 = 0, consumed = 0, committed = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      if (!mbar_wait(smem_u32(&full[slot]), phase)) { ok = false; break; }
      consumed = kb + 1;
      tc_fence_after();
      const uint32_t so = slot * (stage_bytes / 16);
      const int ksteps = min(kStageK, np - j0) / kMmaK;
      for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
          const uint64_t ad = a0 + (so + pa[pr] * a_sp + ks * a_ks);
          const uint64_t bd = b0 + (so + pb[pr] * b_sp + ks * b_ks);
          const bool first = kb == 0 && ks == 0;
          if (pr < 5) mma_bf16(d_corr, ad, bd, idesc, (!first || pr > 0) ? 1u : 0u);
          else mma_bf16(d_main, ad, bd, idesc, first ? 0u : 1u);
        }
      }
      mma_commit(smem_u32(&empty[slot]));
      committed = kb + 1;
      if (++slot == S) { slot = 0; phase ^= 1u; }
      j0 += kStageK;
      if (j0 >= np) j0 = 0;
    }
    counters[1] = consumed;
    counters[2] = committed;
    if (ok) mma_commit(smem_u32(accum));
    else *abort_flag = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // give up: wait (bounded) for this CTA's own copies and MMAs in flight
    atomicOr(a.status, 2);
    const int loaded = counters[0], consumed = counters[1], committed = counters[2];
    for (int kb = consumed; kb < loaded; ++kb) mbar_wait(smem_u32(&full[kb % S]), (kb / S) & 1);
    if (committed > 0) mbar_wait(smem_u32(&empty[(committed - 1) % S]), ((committed - 1) / S) & 1);
  }
  __syncthreads();

  bool good = (*abort_flag == 0);
  if (good && !mbar_wait(smem_u32(accum), 0)) {
    good = false;
    atomicOr(a.status, 2);
  }
  // the TMEM loads below are warp-collective: take one CTA-wide decision
  good = __syncthreads_and(good) != 0;
  tc_fence_after();
  if (good) {
    const int m = threadIdx.x;  // TMEM lane = fiber of the tile
    const uint32_t lane_addr = static_cast<uint32_t>(warp * 32) << 16;
    // strided fibers (modes > 1): stage 16 output rows x 128 fibers in the
    // (now idle) pipeline buffers and store them as 16-byte chunks along the
    // contiguous fiber index.  Contiguous fibers (mode 1): stage the whole
    // FP32 tile [128 fibers][nc] (pitch nc + 4 floats: conflict-free 16-byte
    // stores) and write each fiber's nc outputs as one contiguous run.
    const int64_t tile0 = p0 + a.P * (int64_t)n * q0;
    const int64_t pvalid = a.P - p0;  // fibers of this tile inside the slab: 128 or 64
    const int pitch = nc + 4;
    for (int c0 = 0; c0 < nc; c0 += 16) {
      const int i0 = sub * nc + c0;  // first output row of this chunk
      uint32_t rm[16], rc[16];
      tmem_ld16(d_main + lane_addr + c0, rm);
      tmem_ld16(d_corr + lane_addr + c0, rc);
      float v[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(rm[t]) + __uint_as_float(rc[t]);
      if (!a.a_mn) {
        float4* so = reinterpret_cast<float4*>(reinterpret_cast<float*>(base) + m * pitch + c0);
#pragma unroll
        for (int t = 0; t < 4; ++t) so[t] = make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
        continue;
      }
      if (a.out_fp32) {
        float* so = reinterpret_cast<float*>(base);  // [16 rows][128 fibers]
#pragma unroll
        for (int t = 0; t < 16; ++t) so[t * kMmaM + m] = v[t];
        __syncthreads();
        float* o = reinterpret_cast<float*>(a.out[rhs]) + (int64_t)half * a.N + tile0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = threadIdx.x + k * kMmaThreads;  // float4 chunk: row c / 32, column (c % 32) * 4
          const int row = c >> 5, col = (c & 31) * 4;
          if (i0 + row < n && col < pvalid)
            *reinterpret_cast<float4*>(o + a.P * (i0 + row) + col) =
                *reinterpret_cast<const float4*>(so + row * kMmaM + col);
        }
        __syncthreads();
      } else {
        __nv_bfloat16* so = reinterpret_cast<__nv_bfloat16*>(base);  // [3 splits][16 rows][128 fibers]
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          __nv_bfloat16 sh, sm, sl;
          split3(v[t], sh, sm, sl);
          so[(0 * 16 + t) * kMmaM + m] = sh;
          so[(1 * 16 + t) * kMmaM + m] = sm;
          so[(2 * 16 + t) * kMmaM + m] = sl;
        }
        __syncthreads();
        __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(a.out[rhs]);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int c = threadIdx.x + k * kMmaThreads;  // 16-byte chunk of 8 fibers
          const int s = c >> 8, row = (c >> 4) & 15, col = (c & 15) * 8;
          if (i0 + row < n && col < pvalid)
            *reinterpret_cast<uint4*>(o + (int64_t)(s * 2 + half) * a.N + tile0 + a.P * (i0 + row) + col) =
                *reinterpret_cast<const uint4*>(so + (s * 16 + row) * kMmaM + col);
        }
        __syncthreads();
      }
    }
    if (!a.a_mn) {
      __syncthreads();
      // 8 outputs per thread and pass; a warp covers two fibers' runs
      const int cpf = nc / 8;
      const float* so = reinterpret_cast<const float*>(base);
      for (int e = threadIdx.x; e < kMmaM * cpf; e += kMmaThreads) {
        const int f = e / cpf, ch = e - f * cpf;
        const int64_t q = q0 + f;
        // rows i >= n are not stored (a chunk that starts below n ends below
        // np <= the fiber pitch, its rows past n being zero rows of the padded
        // factor)
        if (q >= a.Q || sub * nc + ch * 8 >= n) continue;
        const float4 x0 = *reinterpret_cast<const float4*>(so + f * pitch + ch * 8);
        const float4 x1 = *reinterpret_cast<const float4*>(so + f * pitch + ch * 8 + 4);
        const int64_t off = a.pitch * q + sub * nc + ch * 8;
        if (a.out_fp32) {
          float4* d4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.out[rhs]) + (int64_t)half * a.N + off);
          d4[0] = x0;
          d4[1] = x1;
        } else {
          const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
          uint32_t w[3][4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(x[2 * k], h0, m0, l0);
            split3(x[2 * k + 1], h1, m1, l1);
            w[0][k] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) |
                      (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
            w[1][k] = static_cast<uint32_t>(__bfloat16_as_ushort(m0)) |
                      (static_cast<uint32_t>(__bfloat16_as_ushort(m1)) << 16);
            w[2][k] = static_cast<uint32_t>(__bfloat16_as_ushort(l0)) |
                      (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
          }
          __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(a.out[rhs]);
#pragma unroll
          for (int sp = 0; sp < 3; ++sp)
            *reinterpret_cast<uint4*>(o + (int64_t)(sp * 2 + half) * a.N + off) =
                make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
        }
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

// ------------------------------------------------------------------ grouped persistent pass (batches)

// The mode passes of a batch's instances in one persistent launch.  Work
// item g = (tile g / nrhs of the group, rhs = g mod nrhs); CTA x takes items
// x, x + G, x + 2G, ... (G = grid size, one CTA per SM).
struct MmaTable {
  const MmaPassArgs* passes;  // device, one per pass
  const CUtensorMap* maps;    // device, four per pass: A of rhs 0 / 1, B of rhs 0 / 1
  const int2* tiles;          // device, (pass, tile within the pass) of each tile of the group
  int npass;
  int nrhs;
  int64_t items;              // tiles * nrhs
};

// Warps 0-15: epilogue, in four groups of four (warp w reads TMEM lanes
// 32 (w mod 4) ...; group w / 4 takes every fourth 16-column chunk); warp 16:
// copies; warp 17: MMAs and the TMEM allocation.  A ring of kGrpStages stage
// slots sized for the largest stage (nc = 128) runs across items, and two
// accumulator pairs in TMEM let the epilogue of one item run under the MMAs
// of the next.  The epilogue is latency-bound (dependent TMEM loads, splits
// and stores per chunk): with four warps it held the pass back, with eight
// or sixteen it does not.
constexpr int kGrpEpiWarps = 16;
constexpr int kGrpEpiGroups = kGrpEpiWarps / 4;
constexpr int kGrpCopyWarp = kGrpEpiWarps, kGrpMmaWarp = kGrpEpiWarps + 1;
constexpr int kGrpThreads = 32 * (kGrpEpiWarps + 2);
constexpr int kGrpStages = 4;
constexpr uint32_t kGrpSlotBytes = mma_stage_bytes(128);
constexpr uint32_t kGrpAccCols = 256;  // columns of one accumulator pair: main [0, nc), corrections [nc, 2nc)
constexpr size_t kGrpSmem = (size_t)kGrpStages * kGrpSlotBytes + 1024 + 256;

// One work item with its pass's arguments, read once into registers (the
// inline-asm memory clobbers would otherwise make every use re-read them).
struct GrpWork {
  int pass, rhs;
  int64_t bx;  // tile within the pass
  int n, np, nc, nsub, both, a_mn, out_fp32;
  int64_t per_q, P, Q, N, pitch;
  void* out;
};

__device__ __forceinline__ GrpWork grp_work(const MmaTable& t, int64_t g) {
  const int2 e = __ldg(&t.tiles[g / t.nrhs]);
  GrpWork w;
  w.pass = e.x;
  w.bx = e.y;
  w.rhs = (int)(g % t.nrhs);
  const MmaPassArgs* a = &t.passes[w.pass];
  w.n = __ldg(&a->n);
  w.np = __ldg(&a->np);
  w.nc = __ldg(&a->nc);
  w.nsub = __ldg(&a->nsub);
  w.both = __ldg(&a->both);
  w.a_mn = __ldg(&a->a_mn);
  w.out_fp32 = __ldg(&a->out_fp32);
  w.per_q = __ldg(&a->per_q);
  w.P = __ldg(&a->P);
  w.Q = __ldg(&a->Q);
  w.N = __ldg(&a->N);
  w.pitch = __ldg(&a->pitch);
  w.out = a->out[w.rhs];
  return w;
}

// Tile bx of a pass: fiber tile, output component (half) and row block
// (sub); with `both` a tile has every row of both components (half = sub = 0).
struct GrpTile {
  int64_t q0, p0;
  int half, sub;
};

__device__ __forceinline__ GrpTile grp_tile(const GrpWork& a) {
  GrpTile g;
  const int parts = a.both ? 1 : 2 * a.nsub;
  const int64_t tile = a.bx / parts;
  const int part = (int)(a.bx % parts);
  g.half = part / a.nsub;
  g.sub = part % a.nsub;
  if (a.a_mn) {
    g.q0 = tile / a.per_q;
    g.p0 = (tile - g.q0 * a.per_q) * kMmaM;
  } else {
    g.q0 = tile * kMmaM;
    g.p0 = 0;
  }
  return g;
}

// Bounded wait that also gives up once another role of the CTA has.
__device__ __forceinline__ bool grp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  return false;
}

__global__ void __launch_bounds__(kGrpThreads, 1) mma_group_kernel(const MmaTable t) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kGrpStages * kGrpSlotBytes);
  uint64_t* empty = full + kGrpStages;
  uint64_t* tfull = empty + kGrpStages;  // [2] accumulator pair b written
  uint64_t* tempty = tfull + 2;          // [2] accumulator pair b read out
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* counters = reinterpret_cast<int*>(tmem_slot + 2);  // stages loaded / consumed / committed
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  constexpr uint32_t a_bytes = kMmaM * kStageK * 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGrpStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), kGrpEpiWarps);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    counters[0] = counters[1] = counters[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kGrpMmaWarp) tmem_alloc(smem_u32(tmem_slot), 2 * kGrpAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kGrpCopyWarp && lane == 0) {
    // copies: every stage of every item of this CTA, as ring slots free up;
    // the next item's record and arguments are read one item ahead
    int slot = 0, kc = 0;
    uint32_t phase = 0;
    bool ok = true;
    GrpWork nxt;
    if (blockIdx.x < t.items) nxt = grp_work(t, blockIdx.x);
    for (int64_t g = blockIdx.x; g < t.items && ok; g += G) {
      const GrpWork a = nxt;
      if (g + G < t.items) nxt = grp_work(t, g + G);
      const CUtensorMap* tmA = &t.maps[4 * a.pass + a.rhs];
      const CUtensorMap* tmB = &t.maps[4 * a.pass + 2 + a.rhs];
      tensormap_acquire(tmA);
      tensormap_acquire(tmB);
      const GrpTile tl = grp_tile(a);
      const int np = a.np, nc = a.nc, a_mn = a.a_mn;
      const int64_t Q = a.Q;
      const int nk = 2 * ((np + kStageK - 1) / kStageK);
      const uint32_t stage_bytes = mma_stage_bytes(nc);
      const int rowB = tl.half * np + tl.sub * nc, pq = (int)(tl.p0 / 64);
      int c = 0, j0 = 0;
      for (int kb = 0; kb < nk; ++kb) {
        // the slot's previous stage (kc - kGrpStages) must have been consumed
        if (kc >= kGrpStages && !grp_wait(smem_u32(&empty[slot]), phase ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        const uint32_t st = smem_u32(base + slot * kGrpSlotBytes), bar = smem_u32(&full[slot]);
        mbar_expect_tx(bar, stage_bytes);
        if (a_mn)
          tma_load_5d(st, tmA, bar, 0, j0, pq, (int)(tl.q0 + Q * c), 0);
        else
          tma_load_4d(st, tmA, bar, j0, (int)tl.q0, c, 0);
        tma_load_4d(st + 3 * a_bytes, tmB, bar, j0, rowB, c, 0);
        ++kc;
        if (++slot == kGrpStages) { slot = 0; phase ^= 1u; }
        j0 += kStageK;
        if (j0 >= np) { j0 = 0; ++c; }
      }
    }
    counters[0] = kc;
    if (!ok) *abort_flag = 1;
  } else if (warp == kGrpMmaWarp && lane == 0) {
    // MMAs: item i into accumulator pair i mod 2, once the epilogue has read
    // that pair's previous item out
    int slot = 0, consumed = 0, committed = 0, itn = 0;
    uint32_t phase = 0;
    bool ok = true;
    constexpr uint32_t pa[6] = {2, 0, 1, 1, 0, 0};  // (l,h) (h,l) (m,m) (m,h) (h,m), then (h,h)
    constexpr uint32_t pb[6] = {0, 2, 1, 0, 1, 0};
    GrpWork nxt;
    if (blockIdx.x < t.items) nxt = grp_work(t, blockIdx.x);
    for (int64_t g = blockIdx.x; g < t.items && ok; g += G, ++itn) {
      const GrpWork a = nxt;
      if (g + G < t.items) nxt = grp_work(t, g + G);
      const int np = a.np, nc = a.nc, a_mn = a.a_mn;
      const int nk = 2 * ((np + kStageK - 1) / kStageK);
      const int b = itn & 1, u = itn >> 1;
      if (u >= 1 && !grp_wait(smem_u32(&tempty[b]), (uint32_t)(u - 1) & 1u, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_main = tmem + b * kGrpAccCols, d_corr = d_main + nc;
      const uint32_t idesc = idesc_bf16(kMmaM, nc, a_mn);
      const uint32_t b_bytes = static_cast<uint32_t>(nc) * kStageK * 2;
      const uint64_t a0 = a_mn ? smem_desc(smem_u32(base), kStageK * 128u, 1024, 2)
                               : smem_desc(smem_u32(base), 16, 8 * kKRowBytes, kKSwizzleDesc);
      const uint64_t b0 = smem_desc(smem_u32(base + 3 * a_bytes), 16, 8 * kKRowBytes, kKSwizzleDesc);
      const uint32_t a_ks = a_mn ? 2048u / 16 : 32u / 16, b_ks = 32u / 16;
      const uint32_t a_sp = a_bytes / 16, b_sp = b_bytes / 16;
      int j0 = 0;
      for (int kb = 0; kb < nk; ++kb) {
        if (!grp_wait(smem_u32(&full[slot]), phase, abort_flag)) { ok = false; break; }
        ++consumed;
        tc_fence_after();
        const uint32_t so = slot * (kGrpSlotBytes / 16);
        const int ksteps = min(kStageK, np - j0) / kMmaK;
        for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
          for (int pr = 0; pr < 6; ++pr) {
            const uint64_t ad = a0 + (so + pa[pr] * a_sp + ks * a_ks);
            const uint64_t bd = b0 + (so + pb[pr] * b_sp + ks * b_ks);
            const bool first = kb == 0 && ks == 0;
            if (pr < 5) mma_bf16(d_corr, ad, bd, idesc, (!first || pr > 0) ? 1u : 0u);
            else mma_bf16(d_main, ad, bd, idesc, first ? 0u : 1u);
          }
        }
        mma_commit(smem_u32(&empty[slot]));
        ++committed;
        if (++slot == kGrpStages) { slot = 0; phase ^= 1u; }
        j0 += kStageK;
        if (j0 >= np) j0 = 0;
      }
      if (ok) mma_commit(smem_u32(&tfull[b]));
    }
    counters[1] = consumed;
    counters[2] = committed;
    if (!ok) *abort_flag = 1;
  } else if (warp < kGrpEpiWarps) {
    // epilogue: thread m = TMEM lane m = fiber m of the tile; results go
    // straight from registers to global memory (strided fibers: a warp's
    // stores cover 32 consecutive fibers; contiguous fibers: each thread
    // writes 16 consecutive outputs of its fiber)
    const int quarter = warp & 3, group = warp >> 2;
    const int m = quarter * 32 + lane;
    const uint32_t lane_addr = static_cast<uint32_t>(quarter * 32) << 16;
    int itn = 0;
    for (int64_t g = blockIdx.x; g < t.items; g += G, ++itn) {
      const GrpWork a = grp_work(t, g);
      const int n = a.n, nc = a.nc;
      const int b = itn & 1, u = itn >> 1;
      const bool okw = grp_wait(smem_u32(&tfull[b]), (uint32_t)u & 1u, abort_flag);
      // the TMEM loads are warp-collective: one decision per warp
      if (!__all_sync(0xffffffffu, okw)) break;
      tc_fence_after();
      const GrpTile tl = grp_tile(a);
      const uint32_t d_main = tmem + b * kGrpAccCols + lane_addr, d_corr = d_main + nc;
      const int64_t tile0 = tl.p0 + a.P * (int64_t)n * tl.q0;
      const int64_t pvalid = a.P - tl.p0;
      const bool fiber_ok = a.a_mn ? (m < pvalid) : (tl.q0 + m < a.Q);
      for (int c0 = 16 * group; c0 < nc; c0 += 16 * kGrpEpiGroups) {
        // component and first output row of this 16-column chunk (np is a
        // multiple of 16, so a chunk never straddles the two components)
        const int half = a.both ? c0 / a.np : tl.half;
        const int i0 = a.both ? c0 - half * a.np : tl.sub * nc + c0;
        uint32_t rm[16], rc[16];
        tmem_ld16_issue(d_main + c0, rm);
        tmem_ld16_issue(d_corr + c0, rc);
        tmem_ld_wait();
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(rm[q]) + __uint_as_float(rc[q]);
        if (!fiber_ok || i0 >= n) continue;
        if (a.a_mn) {
          if (a.out_fp32) {
            float* o = reinterpret_cast<float*>(a.out) + (int64_t)half * a.N + tile0 + m;
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (i0 + q < n) o[a.P * (i0 + q)] = v[q];
          } else {
            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(a.out) + tile0 + m;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              if (i0 + q < n) {
                __nv_bfloat16 sh, sm, sl;
                split3(v[q], sh, sm, sl);
                const int64_t off = a.P * (i0 + q);
                o[(int64_t)(0 + half) * a.N + off] = sh;
                o[(int64_t)(2 + half) * a.N + off] = sm;
                o[(int64_t)(4 + half) * a.N + off] = sl;
              }
            }
          }
        } else {
          // rows i0 .. i0 + 15 of fiber q: a chunk that starts below n ends
          // at or below np <= the fiber pitch; its rows past n are zero rows
          // of the padded factor
          const int64_t off = a.pitch * (tl.q0 + m) + i0;
          if (a.out_fp32) {
            float4* d4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.out) + (int64_t)half * a.N + off);
#pragma unroll
            for (int k = 0; k < 4; ++k) d4[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
          } else {
            uint32_t w[3][8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              __nv_bfloat16 h0, m0, l0, h1, m1, l1;
              split3(v[2 * k], h0, m0, l0);
              split3(v[2 * k + 1], h1, m1, l1);
              w[0][k] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) |
                        (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
              w[1][k] = static_cast<uint32_t>(__bfloat16_as_ushort(m0)) |
                        (static_cast<uint32_t>(__bfloat16_as_ushort(m1)) << 16);
              w[2][k] = static_cast<uint32_t>(__bfloat16_as_ushort(l0)) |
                        (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
            }
            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(a.out);
#pragma unroll
            for (int sp = 0; sp < 3; ++sp) {
              uint4* d = reinterpret_cast<uint4*>(o + (int64_t)(sp * 2 + half) * a.N + off);
              d[0] = make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
              d[1] = make_uint4(w[sp][4], w[sp][5], w[sp][6], w[sp][7]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // give up: wait (bounded) for this CTA's own copies and MMAs in flight
    if (t.npass > 0) atomicOr(t.passes[0].status, 2);
    const int loaded = counters[0], consumed = counters[1], committed = counters[2];
    for (int k = consumed; k < loaded; ++k) mbar_wait(smem_u32(&full[k % kGrpStages]), (k / kGrpStages) & 1);
    if (committed > 0)
      mbar_wait(smem_u32(&empty[(committed - 1) % kGrpStages]), ((committed - 1) / kGrpStages) & 1);
  }
  __syncthreads();
  if (warp == kGrpMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * kGrpAccCols);
  }
}

// ------------------------------------------------------------------ pointwise stages

// Planes are laid out with the first direction padded to a pitch (a multiple
// of 64): point i of the field (n_1 fastest) sits at
//   plane_index(i) = i + (pitch - n_1) floor(i / n_1).
__device__ __forceinline__ int64_t plane_index(int64_t i, int64_t n1, int64_t pitch) {
  return pitch == n1 ? i : i + (pitch - n1) * (i / n1);
}

// A block's segment copied to shared memory: every thread reads its field
// pointers and operator coefficients there instead of from global memory
// (dependent loads ahead of every point's data loads).
template <class Seg> __device__ __forceinline__ const Seg& stage_segment(const Seg* segs, Seg* smem_seg) {
  static_assert(sizeof(Seg) % 8 == 0, "segment copied in 8-byte words");
  const uint64_t* src = reinterpret_cast<const uint64_t*>(segs + blockIdx.y);
  uint64_t* dst = reinterpret_cast<uint64_t*>(smem_seg);
  for (int k = threadIdx.x; k < (int)(sizeof(Seg) / 8); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  return *smem_seg;
}

// Start of a sweep: prologue on complex64 inputs, BF16x3 planes of each rhs
// (one field per segment; blockIdx.y selects the segment in table mode).
template <bool kTable>
__global__ void split_prologue_kernel(const SplitSeg one, const SplitSeg* __restrict__ segs, int nrhs) {
  __shared__ __align__(16) SplitSeg sseg;
  const SplitSeg& g = kTable ? stage_segment(segs, &sseg) : one;
  const int64_t P = g.Npad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    float2 in[2], z[2];
    in[0] = g.in[0][i];
    in[1] = g.nin > 1 ? g.in[1][i] : in[0];
    apply_prologue<float, float2>(g.op, in, z);
    const int64_t ip = plane_index(i, g.n1, g.pitch);
    for (int r = 0; r < nrhs; ++r) {
      __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(g.dst[r]);
      __nv_bfloat16 h, m, l;
      split3(z[r].x, h, m, l);
      d[0 * P + ip] = h;
      d[2 * P + ip] = m;
      d[4 * P + ip] = l;
      split3(z[r].y, h, m, l);
      d[1 * P + ip] = h;
      d[3 * P + ip] = m;
      d[5 * P + ip] = l;
    }
  }
}

// End of a sweep: FP32 planes of each rhs + extras -> epilogue -> complex64.
template <bool kTable>
__global__ void plane_epilogue_kernel(const EpiSeg one, const EpiSeg* __restrict__ segs, int nrhs, int* status) {
  __shared__ __align__(16) EpiSeg sseg;
  const EpiSeg& g = kTable ? stage_segment(segs, &sseg) : one;
  const int64_t P = g.Npad;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ip = plane_index(i, g.n1, g.pitch);
    float2 y[2], ex[kMaxExtra], o[2];
    y[0] = make_float2(g.y[0][ip], g.y[0][P + ip]);
    y[1] = nrhs > 1 ? make_float2(g.y[1][ip], g.y[1][P + ip]) : y[0];
    for (int x = 0; x < g.nextra; ++x) ex[x] = g.ex[x][i];
    const int no = apply_epilogue<float, float2>(g.op, y, ex, o);
    if (no > 0 && g.nout > 0) { g.out[0][i] = o[0]; bad |= !finite2(o[0]); }
    if (no > 1 && g.nout > 1) { g.out[1][i] = o[1]; bad |= !finite2(o[1]); }
  }
  if (bad && status) atomicOr(status, 1);
}

// Real form of an FP64 factor F (n x n, column-major), split in three BF16
// matrices and zero-padded to np = n rounded up to 16:
// out[s][row (c', i)][col (c, j)], rows and columns c * np + (i or j), K =
// col contiguous; entries with i >= n or j >= n are zero.
__global__ void factor_split_kernel(const double2* F, int n, int np, __nv_bfloat16* out) {
  const int64_t total = 4ll * np * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / (2 * np)), col = (int)(e % (2 * np));
    const int cp = row / np, i = row % np, c = col / np, j = col % np;
    double v = 0;
    if (i < n && j < n) {
      const double2 f = F[i + (int64_t)j * n];
      if (cp == 0) v = (c == 0) ? f.x : -f.y;
      else v = (c == 0) ? f.y : f.x;
    }
    const __nv_bfloat16 h = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(h);
    const __nv_bfloat16 m = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(m);
    const __nv_bfloat16 l = __double2bfloat16(r2);
    out[e] = h;
    out[total + e] = m;
    out[2 * total + e] = l;
  }
}

// ------------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static CUtensorMapSwizzle k_major_swizzle() {
  return kKRowBytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                          : (kKRowBytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
}

// A operand map of one rhs for mode geometry (n, P, Q) over a buffer of six
// BF16 planes of N values each, plane 2 s + c = split s of component c.  One
// box holds a whole pipeline stage of A, the three splits one after another,
// so a stage takes one copy instruction:
//   P == 1 (mode 1, K-major): dims (j, q, c, s), fibers `pitch` apart, box
//     (K, 128, 1, 3), swizzle span = K values: [s][128 fibers][K j];
//   P > 1 (MN-major, P % 64 == 0): dims (p mod 64, j, p / 64, q + Q c, s),
//     box (64, K, 2, 1, 3), 128-byte swizzle: [s][two 64-fiber halves][K j][64],
// K = kStageK; positions j >= n and fiber groups p >= P read as zero.
cudaError_t make_state_tmap(void* map_out, const void* splits, int n, int64_t P, int64_t Q, int64_t N,
                            int64_t pitch, int nsplit) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if ((P > 1 && P % 64 != 0) || (P == 1 && (pitch < n || pitch % 8 != 0))) return cudaErrorInvalidValue;
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(map_out);
  std::memset(m, 0, sizeof(CUtensorMap));
  CUresult r;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (P == 1) {
    const cuuint64_t dims[4] = {(cuuint64_t)n, (cuuint64_t)Q, 2, (cuuint64_t)nsplit};
    const cuuint64_t strides[3] = {(cuuint64_t)pitch * 2, (cuuint64_t)N * 2, (cuuint64_t)N * 4};
    const cuuint32_t box[4] = {(cuuint32_t)kStageK, (cuuint32_t)kMmaM, 1, (cuuint32_t)nsplit};
    r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(splits), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, k_major_swizzle(), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[5] = {64, (cuuint64_t)n, (cuuint64_t)(P / 64), (cuuint64_t)(2 * Q), (cuuint64_t)nsplit};
    const cuuint64_t strides[4] = {(cuuint64_t)P * 2, 128, (cuuint64_t)P * n * 2, (cuuint64_t)N * 4};
    const cuuint32_t box[5] = {64, (cuuint32_t)kStageK, 2, 1, (cuuint32_t)nsplit};
    r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(splits), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// B operand map over three padded (2np x 2np) BF16 factor splits, the K index
// of a row split as (j, c): dims (j, row, c, s) (the copy engine walks a box
// in planes of its first two dimensions, so these are the large ones); one
// box = nc output rows x kStageK positions j of one component, all three
// splits ([s][nc rows][K]); rows past 2np read as zero.
cudaError_t make_factor_tmap(void* map_out, const void* fsplit, int n, int nsplit, int rows) {
  const int np = mma_pad16(n), nc = rows > 0 ? rows : mma_rows_per_cta(np);
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(map_out);
  std::memset(m, 0, sizeof(CUtensorMap));
  const cuuint64_t dims[4] = {(cuuint64_t)np, (cuuint64_t)2 * np, 2, (cuuint64_t)nsplit};
  const cuuint64_t strides[3] = {(cuuint64_t)4 * np, (cuuint64_t)2 * np, (cuuint64_t)8 * np * np};
  const cuuint32_t box[4] = {(cuuint32_t)kStageK, (cuuint32_t)nc, 1, (cuuint32_t)nsplit};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(fsplit), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, k_major_swizzle(), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t mma_factor_bytes(int n) {
  const size_t np = mma_pad16(n);
  return 3 * 4 * np * np * 2;
}

// Pipeline depth: up to kMaxStages stages within kSmemPerCta (two CTAs per
// SM, so that one's epilogue runs under the other's MMAs), at least two.
static int mma_stages(int nc) {
  const int fit = (int)((kSmemPerCta - 1024 - 256) / mma_stage_bytes(nc));
  return fit < 2 ? 2 : (fit > kMaxStages ? kMaxStages : fit);
}
size_t mma_smem_bytes(int nc) { return (size_t)mma_stages(nc) * mma_stage_bytes(nc) + 1024 + 256; }

constexpr size_t kMaxDynSmem = 227 * 1024;

// Largest shared-memory need over the supported mode lengths (up to 256),
// within the per-CTA limit.
static size_t mma_smem_limit() {
  size_t m = 0;
  for (int np = 16; np <= 256; np += 16) {
    const size_t b = mma_smem_bytes(mma_rows_per_cta(np));
    if (b <= kMaxDynSmem && b > m) m = b;
  }
  return m;
}

cudaError_t prepare_mma_pass() {
  const int lim = (int)mma_smem_limit();
  cudaError_t e = cudaFuncSetAttribute(mma_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mma_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGrpSmem);
  return e;
}

int64_t mma_build_args(const MmaLaunch& L, MmaPassArgs* out) {
  MmaPassArgs a{};
  a.n = L.n;
  a.np = mma_pad16(L.n);
  a.P = L.P;
  a.Q = L.Q;
  a.pitch = L.pitch;
  a.per_q = (L.P + kMmaM - 1) / kMmaM;
  a.a_mn = L.P > 1 ? 1 : 0;
  a.out_fp32 = L.out_fp32;
  a.out[0] = L.out[0];
  a.out[1] = L.out[1];
  a.N = L.N;
  const int64_t mtiles = a.a_mn ? a.per_q * L.Q : (L.Q + kMmaM - 1) / kMmaM;
  a.both = 0;
  if (L.grouped) {
    // persistent grouped pass (one CTA per SM, two accumulator pairs of at
    // most 128 rows in TMEM): rows of both components in one tile when
    // 2 np <= 128, else one component per tile, in two row blocks past 128
    a.both = a.np <= 64 ? 1 : 0;
    a.nc = a.both ? 2 * a.np : (a.np <= 128 ? a.np : mma_pad16((a.np + 1) / 2));
    a.nsub = a.both ? 1 : (a.np + a.nc - 1) / a.nc;
  } else {
    a.nc = mma_rows_per_cta(a.np);
    a.nsub = (a.np + a.nc - 1) / a.nc;
  }
  int cols = 32;
  while (cols < 2 * a.nc) cols *= 2;
  a.tmem_cols = cols;
  a.stages = mma_stages(a.nc);
  a.status = L.status;
  *out = a;
  if (L.n < 1 || L.n > 256 || (a.a_mn && L.P % 64 != 0) || (!a.a_mn && L.pitch < a.np)) return -1;
  if (L.grouped) return (a.both ? 1 : 2 * a.nsub) * mtiles;  // tiles per rhs
  if (mma_smem_bytes(a.nc) > mma_smem_limit()) return -1;
  // mode 1 stages its FP32 tile [128][nc + 4] in the pipeline buffers
  if (!a.a_mn && (size_t)kMmaM * (a.nc + 4) * 4 > (size_t)a.stages * mma_stage_bytes(a.nc)) return -1;
  return 2 * a.nsub * mtiles;  // CTAs per rhs: (fiber tile, component, row block)
}

cudaError_t launch_mma_pass(const MmaLaunch& L, cudaStream_t s) {
  MmaPassArgs a;
  const int64_t ctas = mma_build_args(L, &a);
  if (ctas < 0) return cudaErrorInvalidValue;
  const CUtensorMap* A0 = reinterpret_cast<const CUtensorMap*>(L.tmA[0]);
  const CUtensorMap* A1 = reinterpret_cast<const CUtensorMap*>(L.tmA[L.nrhs > 1 ? 1 : 0]);
  const CUtensorMap* B0 = reinterpret_cast<const CUtensorMap*>(L.tmB[0]);
  const CUtensorMap* B1 = reinterpret_cast<const CUtensorMap*>(L.tmB[L.nrhs > 1 ? 1 : 0]);
  dim3 grid((unsigned)ctas, (unsigned)L.nrhs);
  mma_mode_kernel<<<grid, kMmaThreads, mma_smem_bytes(a.nc), s>>>(*A0, *A1, *B0, *B1, a);
  return cudaGetLastError();
}

cudaError_t launch_mma_group(const void* passes, const void* maps, const void* tiles, int npass, int64_t ntiles,
                             int nrhs, cudaStream_t s) {
  if (npass < 1 || ntiles < 1 || (nrhs != 1 && nrhs != 2)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const MmaTable t{static_cast<const MmaPassArgs*>(passes), static_cast<const CUtensorMap*>(maps),
                   static_cast<const int2*>(tiles), npass, nrhs, ntiles * nrhs};
  const int64_t grid = std::min<int64_t>(t.items, std::max(1, sms));
  mma_group_kernel<<<(unsigned)grid, kGrpThreads, kGrpSmem, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_split_prologue(const SplitSeg& one, const SplitSeg* segs, int nseg, int64_t max_n, int nrhs,
                                  cudaStream_t s) {
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((max_n + 255) / 256, segs ? 64 : 152 * 16));
  if (segs) split_prologue_kernel<true><<<dim3(bx, (unsigned)nseg), 256, 0, s>>>(one, segs, nrhs);
  else split_prologue_kernel<false><<<bx, 256, 0, s>>>(one, nullptr, nrhs);
  return cudaGetLastError();
}

cudaError_t launch_plane_epilogue(const EpiSeg& one, const EpiSeg* segs, int nseg, int64_t max_n, int nrhs,
                                  int* status, cudaStream_t s) {
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((max_n + 255) / 256, segs ? 64 : 152 * 16));
  if (segs) plane_epilogue_kernel<true><<<dim3(bx, (unsigned)nseg), 256, 0, s>>>(one, segs, nrhs, status);
  else plane_epilogue_kernel<false><<<bx, 256, 0, s>>>(one, nullptr, nrhs, status);
  return cudaGetLastError();
}

cudaError_t launch_factor_split(const double2* F, int n, void* out, cudaStream_t s) {
  const int np = mma_pad16(n);
  const int64_t total = 4ll * np * np;
  factor_split_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(
      F, n, np, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

}  // namespace cgl
