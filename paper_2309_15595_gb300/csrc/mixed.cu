// Reduced-precision Chebyshev filter on the 5th-generation tensor cores.
//
// Complex product as one real GEMM (planar, no wasted flops):
//   [Wr | Wi] = [Ar | Ai] * [[Yr, Yi], [-Yi, Yr]]        (M = N, K = 2N, cols = 2n)
// Every real operand x is split into two BF16 planes, hi = bf16(x),
// lo = bf16(x - hi), and the product uses three MMAs per K block,
// hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory (split-BF16 x3).
// The recurrence state is kept in FP32 (its 2^-24 rounding is far below the
// 2^-15 of the split products, and FP32 math avoids the slow FP64 pipe): the
// epilogue reads the FP32 tile from TMEM, forms Y_new = alpha (W - c Y_cur) +
// beta Y_prev (Eq. 1), stores it over Y_prev and also writes the BF16 hi/lo
// planes of Y_new in the K-major layout the next step's MMA reads, so no
// separate conversion pass runs per degree. The FP64 input V is converted once
// before the first step and the result converted back once after the last.
//
// Accumulation: the tensor cores' FP32 accumulation over the whole K = 2N
// range lost precision in proportion to K (measured: the filter's error grew
// linearly with N, to 1e-3 per degree at N = 20000). So the K range is cut into
// chunks of 256: each chunk's products go into one of two TMEM accumulators
// (double-buffered, so the MMAs of the next chunk run while the epilogue warps
// drain this one), and the epilogue warps add the chunk sums into FP32
// registers with round-to-nearest adds.
//
// Kernel structure (one 128 x 256 output tile per CTA, 10 warps):
//   warp 0   TMA producer: A_hi, A_lo (128 x 32) and B_hi, B_lo (256 x 32) per
//            K block into a 4-stage shared-memory ring of 48 KB stages (64B
//            swizzle: one K block of 32 BF16 is a 64-byte row)
//   warp 1   TMEM allocator and single-thread MMA issuer (tcgen05.mma, M=128,
//            N=256, K=16, kind::f16 with BF16 inputs)
//   warps 2-9 epilogue: warp w reads TMEM lane quarter w % 4 and half of the
//            complex columns; per-chunk drain into FP32 register sums, then the
//            fused Eq. 1 update
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the kernel
// records an error code and winds down instead of spinning.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mixed.cuh"

namespace chase {
#define RC_M(call)                     \
  do {                                 \
    const int _rc = (call);            \
    if (_rc != CHASE_OK) return _rc;   \
  } while (0)
namespace {

// K block of 32 BF16 (64-byte rows, 64B swizzle) and a 4-stage ring: three
// stages stay in flight while one is consumed, enough bytes in flight to
// cover the TMA latency at the MMA rate.
constexpr int TM = 128, TN = 256, TK = 32, STAGES = 4;
constexpr int A_TILE = TM * TK * 2;                 // 8 KB
constexpr int B_TILE = TN * TK * 2;                 // 16 KB
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;  // 48 KB
constexpr int KPAD = 64;                            // K-half padding of the planes
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int NTHREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr int CHUNK_KB = 8;              // K blocks (of 32) per accumulation chunk: 256 values
constexpr uint32_t TMEM_COLS = 512;      // two 128 x 256 FP32 accumulators
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

struct Params {
  int64_t N, Np, j0, ncols;     // rows, padded K half, first active column, end column
  const float2* Ycur;           // FP32 recurrence state, ld N
  float2* Yprev;
  float alpha, beta, gamma;
  __nv_bfloat16* Bn_hi;         // next-step operand planes (rows = B^T rows, ld = 2 Np)
  __nv_bfloat16* Bn_lo;
  int write_next;
  int group;                    // row blocks per sweep of the grouped raster order
  int* err;
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: returns false (and records `code`) after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (globaltimer() - t0 > kWaitLimitNs) {
      atomicExch(err, code);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// UMMA shared-memory descriptor, K-major operand with the 64-byte swizzle:
// 8-row x 64-byte atoms, SBO = 512 B between atoms, version 1 (sm_100+).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)4 << 61;             // SWIZZLE_64B
  return d;
}
// Instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, M x N.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void split2(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __double2bfloat16(x);
  lo = __double2bfloat16(x - (double)__bfloat162float(hi));
}
__device__ __forceinline__ void split2f(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// B^T row of complex column j: tile j/128 holds 256 rows, real parts first.
__device__ __forceinline__ int64_t brow_re(int64_t j) { return (j >> 7) * 256 + (j & 127); }

// ---------------------------------------------------------------- kernel
// One 128 x 256 output tile (row block rb, column tile ct of the active
// columns) of one filter step; the per-problem kernel and the grouped kernel
// (many problems in one launch) both run it.
__device__ __forceinline__ void mixed_tile(const CUtensorMap* tmAh, const CUtensorMap* tmAl,
                                           const CUtensorMap* tmBh, const CUtensorMap* tmBl,
                                           const Params& P, unsigned rb, unsigned ct,
                                           bool maps_in_global) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment of the shared-window address (swizzle atoms)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars[0..S) full, bars[S..2S) empty, bars[2S + b] accumulator b full,
  // bars[2S + 2 + b] accumulator b drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)rb * TM;
  const int64_t tile = (P.j0 >> 7) + ct;          // absolute 128-column tile
  const int nkb = (int)((2 * P.Np) / TK);
  const int nchunks = (nkb + CHUNK_KB - 1) / CHUNK_KB;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[STAGES + s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars[2 * STAGES + b]), 1);
      mbar_init(smem_u32(&bars[2 * STAGES + 2 + b]), EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------- TMA producer
    if (maps_in_global) {  // tensor maps read from global memory by the TMA unit
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmAh) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmAl) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmBh) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmBl) : "memory");
    }
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(smem_u32(&bars[STAGES + s]), ph ^ 1u, P.err, 1)) {
        s_abort = 1;
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const uint32_t full = smem_u32(&bars[s]);
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(full, STAGE_BYTES);
      const int kx = kb * TK;
      tma_load_2d(smem_u32(st), tmAh, kx, (int)m0, full);
      tma_load_2d(smem_u32(st + A_TILE), tmAl, kx, (int)m0, full);
      tma_load_2d(smem_u32(st + 2 * A_TILE), tmBh, kx, (int)(tile * TN), full);
      tma_load_2d(smem_u32(st + 2 * A_TILE + B_TILE), tmBl, kx, (int)(tile * TN), full);
      ++issued;
    }
    // drain: every issued stage must land before the CTA may exit
    for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
      mbar_wait(smem_u32(&bars[kb % STAGES]), (uint32_t)(kb / STAGES) & 1u, P.err, 2);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------- MMA issuer
    int kb = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int b = c & 1;
      const uint32_t acc_tm = tmem + (uint32_t)(b * TN);
      if (c >= 2 &&
          !mbar_wait(smem_u32(&bars[2 * STAGES + 2 + b]), (uint32_t)((c >> 1) - 1) & 1u, P.err, 5)) {
        ok = false;
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int kend = min(nkb, (c + 1) * CHUNK_KB);
      for (; kb < kend; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&bars[s]), ph, P.err, 3) || *(volatile int*)&s_abort) {
          ok = false;
          s_abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t ah = st, al = st + A_TILE, bh = st + 2 * A_TILE, bl = bh + B_TILE;
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 BF16 along K
          // each chunk restarts its accumulator
          const uint32_t acc0 = (kb > c * CHUNK_KB || kk > 0) ? 1u : 0u;
          umma_bf16(acc_tm, sdesc_sw64(ah + off), sdesc_sw64(bh + off), acc0);
          umma_bf16(acc_tm, sdesc_sw64(ah + off), sdesc_sw64(bl + off), 1u);
          umma_bf16(acc_tm, sdesc_sw64(al + off), sdesc_sw64(bh + off), 1u);
        }
        umma_commit(smem_u32(&bars[STAGES + s]));  // stage free once these MMAs finish
      }
      umma_commit(smem_u32(&bars[2 * STAGES + b]));  // chunk c ready (or aborted)
    }
    if (!ok) {
      s_abort = 1;
      umma_commit(smem_u32(&bars[2 * STAGES]));
      umma_commit(smem_u32(&bars[2 * STAGES + 1]));
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------- epilogue
    const int q = warp & 3;                  // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;           // complex columns [h*64, h*64 + 64) of the tile
    const int64_t row = m0 + q * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    float sre[64], sim[64];                  // chunk sums, round-to-nearest FP32 adds
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      sre[j] = 0.f;
      sim[j] = 0.f;
    }
    bool go = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      const bool ok = mbar_wait(smem_u32(&bars[2 * STAGES + b]), (uint32_t)(c >> 1) & 1u, P.err, 4);
      // warp-uniform decision: tcgen05.ld is a whole-warp instruction
      go = __all_sync(0xffffffffu, ok && !*(volatile int*)&s_abort);
      if (!go) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tl + (uint32_t)(b * TN + h * 64);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float v[32];
        tmem_ld32(ta + half * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) sre[half * 32 + j] += v[j];
        tmem_ld32(ta + 128 + half * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) sim[half * 32 + j] += v[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars[2 * STAGES + 2 + b]));
    }
    if (go && row < P.N) {
#pragma unroll
      for (int jj = 0; jj < 64; ++jj) {  // fully unrolled: the sums stay in registers
        const int64_t col = tile * 128 + h * 64 + jj;
        if (col < P.j0 || col >= P.ncols) continue;
        const float2 yc = P.Ycur[row + col * P.N];
        float2* yp = P.Yprev + row + col * P.N;
        float vr = P.alpha * fmaf(-P.gamma, yc.x, sre[jj]);
        float vi = P.alpha * fmaf(-P.gamma, yc.y, sim[jj]);
        if (P.beta != 0.0f) {
          const float2 y0 = *yp;
          vr = fmaf(P.beta, y0.x, vr);
          vi = fmaf(P.beta, y0.y, vi);
        }
        *yp = make_float2(vr, vi);
        if (P.write_next) {
          __nv_bfloat16 rh, rl, ih, il, nh, nl;
          split2f(vr, rh, rl);
          split2f(vi, ih, il);
          split2f(-vi, nh, nl);
          const int64_t br = brow_re(col), bi = br + 128, ld = 2 * P.Np;
          P.Bn_hi[br * ld + row] = rh;
          P.Bn_lo[br * ld + row] = rl;
          P.Bn_hi[br * ld + P.Np + row] = nh;
          P.Bn_lo[br * ld + P.Np + row] = nl;
          P.Bn_hi[bi * ld + row] = ih;
          P.Bn_lo[bi * ld + row] = il;
          P.Bn_hi[bi * ld + P.Np + row] = rh;
          P.Bn_lo[bi * ld + P.Np + row] = rl;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    mixed_filter_kernel(const __grid_constant__ CUtensorMap tmAh,
                        const __grid_constant__ CUtensorMap tmAl,
                        const __grid_constant__ CUtensorMap tmBh,
                        const __grid_constant__ CUtensorMap tmBl, Params P) {
  unsigned rb, ct;  // row block and column tile of this CTA (grouped raster order)
  grouped_tile(blockIdx.x + blockIdx.y * gridDim.x, gridDim.x, gridDim.y, P.group, rb, ct);
  mixed_tile(&tmAh, &tmAl, &tmBh, &tmBl, P, rb, ct, false);
}

// Many problems' filter steps in one launch: entry p of the table holds problem
// p's tensor maps, step parameters and first CTA index; CTA id looks up its
// problem (binary search on the first indices) and runs that problem's tile
// id - first in the same raster order as the per-problem launch, so every
// problem's results are those of its own launch.
struct alignas(64) GroupEntry {
  CUtensorMap ah, al, bh, bl;
  Params P;
  int first, nrow, ncol, pad;
};

__global__ void __launch_bounds__(NTHREADS, 1)
    mixed_filter_grouped_kernel(const GroupEntry* __restrict__ tab, int count) {
  const int id = (int)blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {  // last entry with first <= id
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].first <= id) lo = mid;
    else hi = mid - 1;
  }
  const GroupEntry* e = tab + lo;
  const Params P = e->P;
  unsigned rb, ct;
  grouped_tile((unsigned)(id - e->first), (unsigned)e->nrow, (unsigned)e->ncol, P.group, rb, ct);
  mixed_tile(&e->ah, &e->al, &e->bh, &e->bl, P, rb, ct, true);
}

// ----------------------------------------------------------- conversions
// A (column-major complex) -> row-major planes [Ar | Ai], K half padded to Np.
__global__ void split_a_kernel(int64_t N, int64_t Np, const double2* __restrict__ A, int64_t lda,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  __shared__ double2 tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + tx, k = k0 + r;
    tile[r][tx] = (i < N && k < N) ? A[i + k * lda] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int64_t ld = 2 * Np;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, k = k0 + tx;
    if (i < N && k < N) {
      const double2 a = tile[tx][r];
      __nv_bfloat16 h, l;
      split2(a.x, h, l);
      hi[i * ld + k] = h;
      lo[i * ld + k] = l;
      split2(a.y, h, l);
      hi[i * ld + Np + k] = h;
      lo[i * ld + Np + k] = l;
    }
  }
}

// Columns j0..ncols of Y (column-major complex) -> B^T planes (K-major rows)
// and the FP32 recurrence state S (ld N).
__global__ void split_y_kernel(int64_t N, int64_t Np, int64_t j0, const double2* __restrict__ Y,
                               int64_t ldy, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, float2* __restrict__ S) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = j0 + blockIdx.y;
  if (k >= N) return;
  const double2 y = Y[k + j * ldy];
  S[k + j * N] = make_float2((float)y.x, (float)y.y);
  __nv_bfloat16 rh, rl, ih, il, nh, nl;
  split2(y.x, rh, rl);
  split2(y.y, ih, il);
  split2(-y.y, nh, nl);
  const int64_t br = brow_re(j), bi = br + 128, ld = 2 * Np;
  hi[br * ld + k] = rh;
  lo[br * ld + k] = rl;
  hi[br * ld + Np + k] = nh;
  lo[br * ld + Np + k] = nl;
  hi[bi * ld + k] = ih;
  lo[bi * ld + k] = il;
  hi[bi * ld + Np + k] = rh;
  lo[bi * ld + Np + k] = rl;
}

// FP32 state -> FP64 columns of V.
__global__ void state_to_f64_kernel(int64_t N, const float2* __restrict__ S, double2* __restrict__ V,
                                    int64_t ldv) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (k >= N) return;
  const float2 v = S[k + j * N];
  V[k + j * ldv] = make_double2((double)v.x, (double)v.y);
}

PFN_cuTensorMapEncodeTiled_v12000 lookup_encoder() {
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}
// The driver's tensor-map encoder, looked up once (thread-safe static
// initialisation; contexts may be created from several host threads).
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = lookup_encoder();
  return fn;
}
bool get_encoder() { return encoder() != nullptr; }

// rows x (2 Np) BF16, row-major; box = 64 (K) x box_rows.
bool make_map(CUtensorMap* m, void* base, int64_t rows, int64_t Np, int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * Np), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * Np * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

struct Maps {
  CUtensorMap ah, al, bh[2], bl[2];
};

}  // namespace

// Layout of MixedWork: Ahi/Alo = N x 2Np planes; Yhi/Ylo = two B^T plane pairs
// (ping-pong), each brows x 2Np with brows = 256 * ceil(ne / 128); maps after.
cudaError_t mixed_alloc(MixedWork& w, int64_t N, int64_t ne) {
  w.N = N;
  w.ne = ne;
  const int64_t Np = cdiv(N, KPAD) * KPAD;
  const int64_t brows = cdiv(ne, 128) * 256;
  const size_t a_bytes = (size_t)N * 2 * Np * sizeof(__nv_bfloat16);
  const size_t b_bytes = (size_t)brows * 2 * Np * sizeof(__nv_bfloat16);
  if (!get_encoder()) return cudaErrorNotSupported;
  cudaError_t e;
  if ((e = cudaMalloc(&w.Ahi, a_bytes)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.Alo, a_bytes)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.Yhi, 2 * b_bytes)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.Ylo, 2 * b_bytes)) != cudaSuccess) return e;
  // zero padding (K columns >= N of each half are never written afterwards)
  if ((e = cudaMemset(w.Ahi, 0, a_bytes)) != cudaSuccess) return e;
  if ((e = cudaMemset(w.Alo, 0, a_bytes)) != cudaSuccess) return e;
  if ((e = cudaMemset(w.Yhi, 0, 2 * b_bytes)) != cudaSuccess) return e;
  if ((e = cudaMemset(w.Ylo, 0, 2 * b_bytes)) != cudaSuccess) return e;
  Maps* maps = nullptr;
  if ((e = cudaMallocHost(&maps, sizeof(Maps))) != cudaSuccess) return e;
  w.maps = maps;
  bool ok = make_map(&maps->ah, w.Ahi, N, Np, TM) && make_map(&maps->al, w.Alo, N, Np, TM);
  for (int b = 0; b < 2; ++b) {
    char* yh = static_cast<char*>(w.Yhi) + b * b_bytes;
    char* yl = static_cast<char*>(w.Ylo) + b * b_bytes;
    ok = ok && make_map(&maps->bh[b], yh, brows, Np, TN) && make_map(&maps->bl[b], yl, brows, Np, TN);
  }
  if (!ok) return cudaErrorInvalidValue;
  if ((e = cudaMalloc(&w.S32, (size_t)2 * N * ne * sizeof(float2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.err, sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemset(w.err, 0, sizeof(int))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(mixed_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              SMEM_BYTES);
}

void mixed_free(MixedWork& w) {
  if (w.Ahi) cudaFree(w.Ahi);
  if (w.Alo) cudaFree(w.Alo);
  if (w.Yhi) cudaFree(w.Yhi);
  if (w.Ylo) cudaFree(w.Ylo);
  if (w.err) cudaFree(w.err);
  if (w.S32) cudaFree(w.S32);
  if (w.maps) cudaFreeHost(w.maps);
  w = MixedWork{};
}

namespace {
// Operand planes of A and of Y_0 = V (into operand buffer 0 and FP32 state 0).
void mixed_prologue(cudaStream_t s, int64_t N, const double2* A, int64_t lda, const double2* V,
                    int64_t ldv, int64_t ncols, MixedWork& w) {
  const int64_t Np = cdiv(N, KPAD) * KPAD;
  split_a_kernel<<<dim3((unsigned)cdiv(N, 32), (unsigned)cdiv(N, 32), 1), dim3(32, 8, 1), 0, s>>>(
      N, Np, A, lda, static_cast<__nv_bfloat16*>(w.Ahi), static_cast<__nv_bfloat16*>(w.Alo));
  count_launch();
  split_y_kernel<<<dim3((unsigned)cdiv(N, 256), (unsigned)ncols, 1), 256, 0, s>>>(
      N, Np, 0, V, ldv, static_cast<__nv_bfloat16*>(w.Yhi), static_cast<__nv_bfloat16*>(w.Ylo),
      static_cast<float2*>(w.S32));
  count_launch();
}

// Parameters of filter step i (1-based) and the operand-plane buffer it reads.
Params step_params(int64_t N, int64_t ncols, const int32_t* degs, double c, const double* al,
                   const double* be, int i, int group, MixedWork& w, int* bin_out) {
  const int64_t Np = cdiv(N, KPAD) * KPAD;
  const int64_t brows = cdiv(w.ne, 128) * 256;
  const size_t b_elems = (size_t)brows * 2 * Np;
  float2* st[2] = {static_cast<float2*>(w.S32), static_cast<float2*>(w.S32) + (size_t)N * w.ne};
  const int dmax = degs[ncols - 1];
  const int src = (i - 1) & 1, dst = i & 1;   // FP32 state buffers
  const int bout = i & 1;                      // operand plane buffer written
  Params P;
  P.N = N;
  P.Np = Np;
  P.j0 = std::lower_bound(degs, degs + ncols, i) - degs;
  P.ncols = ncols;
  P.Ycur = st[src];
  P.Yprev = st[dst];
  P.alpha = (float)al[i];
  P.beta = (i == 1) ? 0.0f : (float)be[i];
  P.gamma = (float)c;
  P.Bn_hi = static_cast<__nv_bfloat16*>(w.Yhi) + bout * b_elems;
  P.Bn_lo = static_cast<__nv_bfloat16*>(w.Ylo) + bout * b_elems;
  P.write_next = i < dmax;
  P.group = group;
  P.err = w.err;
  *bin_out = (i - 1) & 1;
  return P;
}

unsigned step_col_tiles(const Params& P) {
  return (unsigned)((P.ncols - 1) / 128 - P.j0 / 128 + 1);
}

// ----------------------------------------------- raster-order autotuner
// The grouped raster order (`group` row blocks per sweep of the column tiles)
// decides how many CTAs resident at one time share A's planes and the operand
// planes in L2; the best group depends on N, on the number of column tiles and
// on the device. The first filter call for a shape (per device, N, column
// tiles) times filter step 1 twice with each candidate (step 1 reads only the
// start block and ignores the state it overwrites, so repeating it changes
// nothing) and keeps the fastest; later calls reuse it. The arithmetic of a
// tile does not depend on the order, so the choice never changes a result.
// Measured at C3 (N = 40000, 3000 vectors, one group for every run): 1 / 2 /
// 4 / 8 / 16 / 32 / 64 / all row blocks: 0.67 / 0.74 / 0.77 / 0.80 / 0.81 /
// 0.82 / 0.88 / 0.76 of the sustained bf16 peak: sharing a column tile of the
// operand planes (82 MB) across many row blocks matters more than sharing a row
// block of A's planes (41 MB).
// The candidates are timed in turn, three times each (the fastest time of each
// counts), and one replaces the default only when it is faster by more than 3 %:
// single timings of step 1 picked 16 or 32 in some runs (C3 filter 0.80 of the
// peak instead of 0.90).
constexpr int kGroupCandidates[] = {64, 32, 128, 16};
constexpr int kDefaultGroup = 64;
constexpr int kTuneRepeats = 3;
constexpr float kTuneMargin = 0.97f;
static_assert(kGroupCandidates[0] == kDefaultGroup, "the default is timed first");
std::mutex g_tune_mutex;
std::map<std::tuple<int, int64_t, unsigned>, int> g_tuned_group;

int tuned_group(int64_t N, unsigned coltiles) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tuned_group.find(std::make_tuple(dev, N, coltiles));
  return it == g_tuned_group.end() ? 0 : it->second;
}

int tune_group(cudaStream_t s, const Maps* maps, Params P, dim3 grid) {
  const int cached = tuned_group(P.N, grid.y);
  if (cached) return cached;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return kDefaultGroup;
  constexpr int nc = (int)(sizeof(kGroupCandidates) / sizeof(int));
  float t[nc];
  for (int i = 0; i < nc; ++i) t[i] = 1e30f;
  for (int rep = 0; rep < kTuneRepeats; ++rep) {
    for (int i = 0; i < nc; ++i) {
      P.group = kGroupCandidates[i];
      cudaEventRecord(e0, s);
      mixed_filter_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(maps->ah, maps->al, maps->bh[0],
                                                             maps->bl[0], P);
      count_launch();
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t[i] = std::min(t[i], ms);
    }
  }
  int best = kDefaultGroup;
  float best_ms = t[0];  // kGroupCandidates[0] is the default
  for (int i = 1; i < nc; ++i)
    if (t[i] < kTuneMargin * best_ms) {
      best_ms = t[i];
      best = kGroupCandidates[i];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned_group[std::make_tuple(dev, P.N, grid.y)] = best;
  return best;
}

int check_err(cudaStream_t s, int* err) {
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  if (herr != 0) {
    fprintf(stderr, "[chase] tensor-core filter: pipeline wait expired (code %d)\n", herr);
    return CHASE_CUDA_FAIL();
  }
  return CHASE_OK;
}
}  // namespace

int mixed_filter(cudaStream_t s, int64_t N, const double2* A, int64_t lda, double2* V,
                 int64_t ldv, int64_t ncols, const int32_t* degs, double c, const double* al,
                 const double* be, double2* W, int64_t ldw, MixedWork& w, bool autotune) {
  if (ncols == 0) return CHASE_OK;
  if (!w.maps || N != w.N || ncols > w.ne) return CHASE_ERR_INVALID_ARG;
  (void)W;
  (void)ldw;
  const Maps* maps = static_cast<const Maps*>(w.maps);
  mixed_prologue(s, N, A, lda, V, ldv, ncols, w);
  if (cudaMemsetAsync(w.err, 0, sizeof(int), s) != cudaSuccess) return CHASE_CUDA_FAIL();
  const int dmax = degs[ncols - 1];
  int group = kDefaultGroup;
  for (int i = 1; i <= dmax; ++i) {
    int bin = 0;
    Params P = step_params(N, ncols, degs, c, al, be, i, group, w, &bin);
    const dim3 grid((unsigned)cdiv(N, TM), step_col_tiles(P), 1);
    if (i == 1 && autotune) P.group = group = tune_group(s, maps, P, grid);
    mixed_filter_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(maps->ah, maps->al, maps->bh[bin],
                                                           maps->bl[bin], P);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return CHASE_CUDA_FAIL();
  }
  // even degrees: every column's final value is in state buffer 0
  state_to_f64_kernel<<<dim3((unsigned)cdiv(N, 256), (unsigned)ncols, 1), 256, 0, s>>>(
      N, static_cast<const float2*>(w.S32), V, ldv);
  count_launch();
  return check_err(s, w.err);
}

cudaError_t mixed_group_reserve(MixedGroupTable& t, size_t entries) {
  if (entries <= t.capacity) return cudaSuccess;
  mixed_group_free(t);
  cudaError_t e;
  if ((e = cudaMalloc(&t.dev, entries * sizeof(GroupEntry))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&t.host, entries * sizeof(GroupEntry))) != cudaSuccess) return e;
  t.capacity = entries;
  return cudaSuccess;
}

void mixed_group_free(MixedGroupTable& t) {
  if (t.dev) cudaFree(t.dev);
  if (t.host) cudaFreeHost(t.host);
  t = MixedGroupTable{};
}

size_t mixed_group_entries(int count, const MixedGroupItem* items) {
  size_t n = 0;
  for (int k = 0; k < count; ++k)
    if (items[k].ncols > 0) n += (size_t)items[k].degs[items[k].ncols - 1];
  return n;
}

int mixed_filter_grouped(cudaStream_t s, int count, const MixedGroupItem* items,
                         MixedGroupTable& t, int* launches) {
  static std::once_flag attr_once[kMaxDevices];
  once_per_device(attr_once, []() {
    cudaFuncSetAttribute(mixed_filter_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM_BYTES);
  });
  int dmax_all = 0;
  for (int k = 0; k < count; ++k) {
    const MixedGroupItem& it = items[k];
    if (it.ncols == 0) continue;
    if (!it.w || !it.w->maps || it.N != it.w->N || it.ncols > it.w->ne)
      return CHASE_ERR_INVALID_ARG;
    dmax_all = std::max(dmax_all, (int)it.degs[it.ncols - 1]);
  }
  if (dmax_all == 0) return CHASE_OK;
  if (mixed_group_entries(count, items) > t.capacity) return CHASE_ERR_INVALID_ARG;
  // operand planes of every problem, then the step table: for step i the
  // entries of the problems still filtering, with their first CTA indices
  for (int k = 0; k < count; ++k) {
    const MixedGroupItem& it = items[k];
    if (it.ncols == 0) continue;
    mixed_prologue(s, it.N, it.A, it.lda, it.V, it.ldv, it.ncols, *it.w);
    if (cudaMemsetAsync(it.w->err, 0, sizeof(int), s) != cudaSuccess) return CHASE_CUDA_FAIL();
  }
  GroupEntry* host = static_cast<GroupEntry*>(t.host);
  std::vector<size_t> off(dmax_all + 2, 0);
  std::vector<int> ctas(dmax_all + 1, 0);
  size_t n = 0;
  for (int i = 1; i <= dmax_all; ++i) {
    off[i] = n;
    int first = 0;
    for (int k = 0; k < count; ++k) {
      const MixedGroupItem& it = items[k];
      if (it.ncols == 0 || it.degs[it.ncols - 1] < i) continue;
      const Maps* maps = static_cast<const Maps*>(it.w->maps);
      const int g = tuned_group(it.N, (unsigned)((it.ncols - 1) / 128 + 1));
      int bin = 0;
      GroupEntry& e = host[n++];
      e.P = step_params(it.N, it.ncols, it.degs, it.c, it.al, it.be, i,
                        g ? g : kDefaultGroup, *it.w, &bin);
      e.ah = maps->ah;
      e.al = maps->al;
      e.bh = maps->bh[bin];
      e.bl = maps->bl[bin];
      e.nrow = (int)cdiv(it.N, TM);
      e.ncol = (int)step_col_tiles(e.P);
      e.first = first;
      e.pad = 0;
      first += e.nrow * e.ncol;
    }
    ctas[i] = first;
  }
  off[dmax_all + 1] = n;
  if (cudaMemcpyAsync(t.dev, host, n * sizeof(GroupEntry), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return CHASE_CUDA_FAIL();
  // the degree steps of all problems as one CUDA graph: one grouped launch per step
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  const GroupEntry* dev = static_cast<const GroupEntry*>(t.dev);
  for (int i = 1; i <= dmax_all; ++i) {
    mixed_filter_grouped_kernel<<<(unsigned)ctas[i], NTHREADS, SMEM_BYTES, s>>>(
        dev + off[i], (int)(off[i + 1] - off[i]));
    count_launch();
  }
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (ce != cudaSuccess || !graph) return CHASE_CUDA_FAIL();
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return CHASE_CUDA_FAIL();
  const cudaError_t le = cudaGraphLaunch(exec, s);
  if (le != cudaSuccess) {
    cudaGraphExecDestroy(exec);
    return CHASE_CUDA_FAIL();
  }
  if (launches) *launches = dmax_all;
  for (int k = 0; k < count; ++k) {
    const MixedGroupItem& it = items[k];
    if (it.ncols == 0) continue;
    state_to_f64_kernel<<<dim3((unsigned)cdiv(it.N, 256), (unsigned)it.ncols, 1), 256, 0, s>>>(
        it.N, static_cast<const float2*>(it.w->S32), it.V, it.ldv);
    count_launch();
  }
  const cudaError_t se = cudaStreamSynchronize(s);
  cudaGraphExecDestroy(exec);
  if (se != cudaSuccess) return CHASE_CUDA_FAIL();
  for (int k = 0; k < count; ++k)
    if (items[k].ncols > 0) RC_M(check_err(s, items[k].w->err));
  return CHASE_OK;
}

}  // namespace chase
