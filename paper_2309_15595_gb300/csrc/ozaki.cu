// FP64-accurate complex GEMM on the BF16 tensor cores (error-free splitting in
// the manner of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012), used for the FP64 filter (also
// grouped over many problems for the batched sequence), the Lanczos block
// product, the Rayleigh-Ritz products, the residual product A V and the
// CholeskyQR products.
//
// Same planar real form as the mixed filter: W = [Ar | Ai] [[Yr, Yi], [-Yi, Yr]].
// The diagonal of A is taken out of the digit planes and applied exactly in
// FP64 in the epilogue (A_ii B_ij): the row scales then follow the off-diagonal
// entries, which keeps their relative precision when A is diagonally dominant.
// Row i of the left operand is scaled by 2^-e_i and column j of the right one
// by 2^-f_j so every entry x has |x| < 1/2, then cut into S = 6 signed 8-bit
// digits, x = sum_s d_s 2^-8s + r with |r| <= 2^-49 and |d_s| <= 128 (the
// balanced base-256 digits of rint(x 2^48), in integer arithmetic); every digit
// is exact in BF16. The product keeps the 21 digit pairs
// (s, t) with s + t <= 7; pair (s, t) contributes at weight 2^-8(s+t).
// Digit products are < 2^14 and exact; the FP32 tensor-memory accumulator of
// one level L = s + t stays an exact integer over a chunk of 256 K values
// (at most (L-1) 2^22 <= 2^24 for L <= 5), so after every chunk the epilogue
// warps move levels 2-5 into exact int64 accumulators (shifted into one common
// scale, at most 2^54 in total) and levels 6-7, whose weights are at most
// 2^-32 of the leading level, into an FP32 accumulator (its rounding is then
// below 2^-56 of the leading level).
// The result is W = 2^(e_i + f_j) (acc 2^-40 + acc67 2^-48), accurate to a few
// units of 2^-48 relative to |A_i.| |Y_.j| per term: FP64-class.
// Extended variant (LMAX = 8): the five pairs of level 8 are kept too (26 MMAs
// per K step instead of 21, level 8 drained into the FP32 accumulator at weight
// 2^-64). The dropped pairs then weigh at most 2^-58 instead of 2^-50 of
// 2^(e_i + f_j) per term, so a product over K terms whose result cancels
// almost completely (a Gram of nearly orthonormal columns with entries near 1,
// the residual X - T U of a triangular solve) keeps an error near the digit
// rounding of its operands instead of sqrt(K) 2^-50 of the scales.
//
// Kernel structure (128 x 64 real output tile = 32 complex columns, 10 warps):
//   warp 0    TMA producer: 6 A digit tiles (128 x 32) and 6 B digit tiles
//             (64 x 32) per K block into a 3-stage ring (64B swizzle)
//   warp 1    TMEM allocator and MMA issuer: 21 (26) tcgen05.mma (M=128,
//             N=64, K=16) per 16-wide K step, one accumulator per level (6 (7)
//             x 64 TMEM columns); after each 256-wide chunk it hands the
//             accumulators to the epilogue and waits until they are drained
//   warps 2-9 epilogue: warp w owns TMEM lane quarter w % 4 and half of the
//             complex columns; int64/FP32 accumulators in registers; at the
//             end forms the FP64 result and applies the fused update.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "ozaki.cuh"

namespace chase {
namespace {

constexpr int OS = 6;                    // digits per operand
static_assert(OS == 6, "the epilogue keeps levels 2-5 exact and levels 6-7 in FP32");
constexpr int TM = 128, TN = 64, TK = 32, STAGES = 3;
constexpr int CHUNK_KB = 8;              // K blocks per exact chunk (256 values)
constexpr int A_TILE = TM * TK * 2;      // 8 KB per digit
constexpr int B_TILE = TN * TK * 2;      // 4 KB per digit
constexpr int STAGE_BYTES = OS * (A_TILE + B_TILE);  // 72 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int NTHREADS = 320;
constexpr uint32_t TMEM_COLS = 512;
constexpr int KPAD = 128;                // K-half padding: 2 Np is a multiple of 256
constexpr int HC = TN / 4;               // complex columns per epilogue warp half (16)
constexpr int CT = TN / 2;               // complex columns per tile (32)
constexpr unsigned long long kWaitLimitNs = 4000000000ull;
constexpr unsigned kGroup = 8;           // row blocks per sweep of the column tiles

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
// K-major operand, 64-byte swizzle: 8-row x 64-byte atoms, SBO = 512 B.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
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
// 16 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// B^T row of complex column j: tiles of CT complex columns, TN rows each,
// real parts first.
__device__ __forceinline__ int64_t brow_re(int64_t j) { return (j / CT) * TN + (j % CT); }

struct Params {
  int64_t N, Np, j0, ncols;   // rows, padded K half, first active column, end column
  int64_t brows;              // rows of one B digit plane
  int64_t arows;              // rows of one A digit plane (= N)
  const int* escale_a;        // per row: exponent e_i
  const double2* diag;        // diagonal of A, applied exactly in FP64
  const double2* Bsrc;        // right operand in FP64 (absolute columns, ld ldbs)
  int64_t ldbs;
  const int* escale_b;        // per complex column: exponent f_j
  int mode;                   // EPI_STORE / EPI_FILTER / EPI_RESID
  double alpha, beta, gamma;  // filter
  const double2* X;           // filter/resid: B operand in FP64 (ld ldx)
  int64_t ldx;
  double2* Y;                 // store/filter destination (ld ldy)
  int64_t ldy;
  const double* theta;        // resid
  double* partial;            // resid: [32-row tile + col * ceil(N / 32)]
  int* err;
};

// ---------------------------------------------------------------- kernel
// One 128 x 64 output tile (row block rb, column tile ct of the active
// columns); the per-problem kernel and the grouped kernel (the filter steps
// of many problems in one launch) both run it.
template <int LMAX>
__device__ __forceinline__ void ozaki_tile(const CUtensorMap* tmA, const CUtensorMap* tmB,
                                           const Params& P, unsigned rb, unsigned ct,
                                           bool maps_in_global) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // [0,S) full, [S,2S) empty, [2S] accumulators full, [2S+1] accumulators empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)rb * TM;
  const int64_t tile = P.j0 / CT + ct;            // absolute CT-column tile
  const int nkb = (int)((2 * P.Np) / TK);
  const int nchunks = nkb / CHUNK_KB;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[STAGES + s]), 1);
    }
    mbar_init(smem_u32(&bars[2 * STAGES]), 1);
    mbar_init(smem_u32(&bars[2 * STAGES + 1]), 8);
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

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------ TMA producer
      if (maps_in_global) {  // tensor maps read from global memory by the TMA unit
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmA)
                     : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmB)
                     : "memory");
      }
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&bars[STAGES + s]), ph ^ 1u, P.err, 11)) {
          s_abort = 1;
          break;
        }
        if (*(volatile int*)&s_abort) break;
        const uint32_t full = smem_u32(&bars[s]);
        uint8_t* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(full, STAGE_BYTES);
        const int kx = kb * TK;
#pragma unroll
        for (int d = 0; d < OS; ++d) {
          // digit planes are stacked along rows: digit d of row r is row d * rows + r
          tma_load_2d(smem_u32(st + d * A_TILE), tmA, kx, (int)(d * P.arows + m0), full);
        }
#pragma unroll
        for (int d = 0; d < OS; ++d) {
          tma_load_2d(smem_u32(st + OS * A_TILE + d * B_TILE), tmB, kx,
                      (int)(d * P.brows + tile * TN), full);
        }
        ++issued;
      }
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
        mbar_wait(smem_u32(&bars[kb % STAGES]), (uint32_t)(kb / STAGES) & 1u, P.err, 12);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------ MMA issuer
      int kb = 0;
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        if (c > 0 && !mbar_wait(smem_u32(&bars[2 * STAGES + 1]), (uint32_t)(c - 1) & 1u, P.err, 13)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int kc = 0; kc < CHUNK_KB; ++kc, ++kb) {
          const int s = kb % STAGES;
          const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
          if (!mbar_wait(smem_u32(&bars[s]), ph, P.err, 14) || *(volatile int*)&s_abort) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk) {
            const uint32_t off = kk * 32;
#pragma unroll
            for (int L = 2; L <= LMAX; ++L) {
              const int sa0 = L - OS > 1 ? L - OS : 1;  // first pair of level L
#pragma unroll
              for (int sa = sa0; sa < L && sa <= OS; ++sa) {
                const int tb = L - sa;
                // every level restarts each 256-long chunk (levels 2-5 then stay
                // exact integers below 2^24)
                const uint32_t acc = (kc == 0 && kk == 0 && sa == sa0) ? 0u : 1u;
                umma_bf16(tmem + (uint32_t)((L - 2) * TN),
                          sdesc_sw64(st + (sa - 1) * A_TILE + off),
                          sdesc_sw64(st + OS * A_TILE + (tb - 1) * B_TILE + off), acc);
              }
            }
          }
          umma_commit(smem_u32(&bars[STAGES + s]));
        }
        umma_commit(smem_u32(&bars[2 * STAGES]));  // chunk c ready
      }
      if (!ok) {
        s_abort = 1;
        umma_commit(smem_u32(&bars[2 * STAGES]));
      }
    }
  } else {
    // ------------------------------------------------------- epilogue warps
    const int q = warp & 3;                   // TMEM lane quarter
    const int h = (warp - 2) >> 2;            // complex column half: [h*24, h*24+24)
    const int64_t row = m0 + q * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    long long acc[2 * HC];                    // re[0..16), im[16..32): levels 2-5, weight 2^-40
    // levels 6-LMAX, weight 2^-48. In the extended variant they are summed over
    // the chunks in FP64: its products are Grams whose diagonal adds squared
    // digits coherently (sum_k d_3(x_k)^2 grows like K), where FP32 sums over
    // K = 80000 lost about 2^-44 of the scale (orthogonality 2e-11 at
    // N = 40000 after CholeskyQR2); per chunk the values stay below 2^25.
    using Acc67 = typename std::conditional<LMAX == 8, double, float>::type;
    Acc67 acc67[2 * HC];
#pragma unroll
    for (int j = 0; j < 2 * HC; ++j) {
      acc[j] = 0;
      acc67[j] = Acc67(0);
    }
    bool go = true;
    for (int c = 0; c < nchunks; ++c) {
      const bool ok = mbar_wait(smem_u32(&bars[2 * STAGES]), (uint32_t)c & 1u, P.err, 15);
      go = __all_sync(0xffffffffu, ok && !*(volatile int*)&s_abort);
      if (!go) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // levels 2..5 are exact integers below 2^24 per chunk: int64 at weight
      // 2^-40 (level L shifted by 8 (5 - L) bits). Levels 6 and 7 (weights
      // 2^-48, 2^-56, at most 2^-24 of the leading level) go to FP32 registers
      // per chunk. (Accumulating them in TMEM over the whole K range instead
      // lost accuracy at K = 80000: a Ritz-value floor near 1e-10 ||A||.)
      // loads issued two levels at a time, one wait per pair (the TMEM load
      // latency is paid 6 times per chunk instead of 12)
#pragma unroll
      for (int part = 0; part < 2; ++part) {  // real columns, then imaginary
#pragma unroll
        for (int g = 0; g < LMAX / 2; ++g) {  // levels 2-3, 4-5, 6-7 (, 8)
          float v[2][HC];
#pragma unroll
          for (int l = 0; l < 2; ++l)
            if (2 + 2 * g + l <= LMAX)
              tmem_ld16(tl + (uint32_t)((2 * g + l) * TN + part * CT + h * HC), v[l]);
          tmem_wait_ld();
#pragma unroll
          for (int l = 0; l < 2; ++l) {
            const int L = 2 + 2 * g + l;
            if (L > LMAX) continue;
            if (L <= 5) {
              const int sh = 8 * (5 - L);
#pragma unroll
              for (int j = 0; j < HC; ++j)
                acc[part * HC + j] += (long long)__float2int_rn(v[l][j]) << sh;
            } else {
              const Acc67 w = L == 6 ? Acc67(1) : (L == 7 ? Acc67(0x1p-8) : Acc67(0x1p-16));
#pragma unroll
              for (int j = 0; j < HC; ++j)
                acc67[part * HC + j] = fma(w, (Acc67)v[l][j], acc67[part * HC + j]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars[2 * STAGES + 1]));
    }
    // ------------------------------------------------ FP64 result + update
    double rsq[HC];
    if (go && row < P.N) {
      const double sa = ldexp(1.0, P.escale_a[row]);
      const double2 dg = P.diag ? P.diag[row] : make_double2(0.0, 0.0);
#pragma unroll
      for (int jj = 0; jj < HC; ++jj) {
        const int64_t col = tile * CT + h * HC + jj;
        rsq[jj] = 0.0;
        if (col < P.j0 || col >= P.ncols) continue;
        const double sc = sa * ldexp(1.0, P.escale_b[col]);
        const double2 b = P.diag ? P.Bsrc[row + col * P.ldbs] : make_double2(0.0, 0.0);
        const double lr = fma((double)acc[jj], 0x1p-40, (double)acc67[jj] * 0x1p-48);
        const double li = fma((double)acc[HC + jj], 0x1p-40, (double)acc67[HC + jj] * 0x1p-48);
        const double wr = fma(dg.x, b.x, fma(-dg.y, b.y, sc * lr));
        const double wi = fma(dg.x, b.y, fma(dg.y, b.x, sc * li));
        if (P.mode == EPI_STORE) {
          P.Y[row + col * P.ldy] = make_double2(wr, wi);
        } else if (P.mode == EPI_FILTER) {
          const double2 x = P.X[row + col * P.ldx];
          double2* yp = P.Y + row + col * P.ldy;
          double vr = P.alpha * fma(-P.gamma, x.x, wr);
          double vi = P.alpha * fma(-P.gamma, x.y, wi);
          if (P.beta != 0.0) {
            const double2 y0 = *yp;
            vr = fma(P.beta, y0.x, vr);
            vi = fma(P.beta, y0.y, vi);
          }
          *yp = make_double2(vr, vi);
        } else {
          const double2 x = P.X[row + col * P.ldx];
          const double th = P.theta[col];
          const double dx = fma(-th, x.x, wr), dy = fma(-th, x.y, wi);
          rsq[jj] = fma(dx, dx, dy * dy);
        }
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < HC; ++jj) rsq[jj] = 0.0;
    }
    if (P.mode == EPI_RESID && go) {
      // per column: sum over this warp's 32 rows, one partial per 32-row tile
      const int64_t nt32 = (P.N + 31) / 32;
      const int64_t t32 = (int64_t)rb * 4 + q;
#pragma unroll
      for (int jj = 0; jj < HC; ++jj) {
        double v = rsq[jj];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        const int64_t col = tile * CT + h * HC + jj;
        if (lane == 0 && t32 < nt32 && col >= P.j0 && col < P.ncols) P.partial[t32 + col * nt32] = v;
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

template <int LMAX>
__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      Params P) {
  unsigned rb, ct;  // row block and column tile of this CTA (grouped raster order)
  grouped_tile(blockIdx.x + blockIdx.y * gridDim.x, gridDim.x, gridDim.y, kGroup, rb, ct);
  ozaki_tile<LMAX>(&tmA, &tmB, P, rb, ct, false);
}

// Many problems' filter steps in one launch: entry p of the table holds problem
// p's tensor maps, step parameters and first CTA index; CTA id finds its
// problem (binary search on the first indices) and runs that problem's tile
// id - first in the raster order of the per-problem launch, so each problem's
// result is that of its own launch.
struct OzGroupEntry {  // aligned as its tensor maps
  CUtensorMap a, b;
  Params P;
  int first, nrow, ncol, pad;
};

__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_filter_grouped_kernel(const OzGroupEntry* __restrict__ tab, int count) {
  const int id = (int)blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {  // last entry with first <= id
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].first <= id) lo = mid;
    else hi = mid - 1;
  }
  const OzGroupEntry* e = tab + lo;
  const Params P = e->P;
  unsigned rb, ct;
  grouped_tile((unsigned)(id - e->first), (unsigned)e->nrow, (unsigned)e->ncol, kGroup, rb, ct);
  ozaki_tile<7>(&e->a, &e->b, P, rb, ct, true);
}

// ------------------------------------------------------------ digit prep
// |x| < 1/2: x = sum_s d_s 2^-8s + r with |r| <= 2^-49 and integer digits
// |d_s| <= 128 (exact in BF16). X = rint(x 2^48) (|X| <= 2^47) is written in
// balanced base 256, the low digits in [-128, 127] and the leading one in
// [-128, 128]; so sum_s d_s 2^-8s = X 2^-48 exactly. Integer arithmetic: the
// FP64 pipe (1/64 of the FP32 rate on this part) does one multiply and one
// conversion per value instead of a multiply, a rounding and a subtraction
// per digit.
__device__ __forceinline__ void digits_of(double x, __nv_bfloat16* d) {
  long long X = __double2ll_rn(x * 0x1p48);
#pragma unroll
  for (int s = OS - 1; s > 0; --s) {
    const int low = (int)(((unsigned)X + 128u) & 255u) - 128;  // X mod 256, balanced
    d[s] = __float2bfloat16_rn((float)low);
    X = (X - low) >> 8;  // exact: X - low is a multiple of 256
  }
  d[0] = __float2bfloat16_rn((float)X);
}

__device__ __forceinline__ int scale_exp(double mx) {
  if (!(mx > 0.0)) return 0;
  int E;
  frexp(mx, &E);  // mx = f 2^E, f in [0.5, 1)
  return E + 1;   // mx 2^-(E+1) in [0.25, 0.5)
}

// Row maxima of A (column-major): amax[i] = max_k max(|Re A_ik|, |Im A_ik|),
// as the bit pattern of a non-negative double (monotone in unsigned order).
__global__ void rowmax_kernel(int64_t M, int64_t K, bool skip_diag, const double2* __restrict__ A,
                              int64_t lda, unsigned long long* __restrict__ amax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t k0 = (int64_t)blockIdx.y * 256, k1 = min(K, k0 + 256);
  double m = 0.0;
  for (int64_t k = k0; k < k1; ++k) {
    if (skip_diag && k == i) continue;  // the diagonal is applied separately, exactly
    const double2 a = A[i + k * lda];
    m = fmax(m, fmax(fabs(a.x), fabs(a.y)));
  }
  atomicMax(&amax[i], (unsigned long long)__double_as_longlong(m));
}

__global__ void diag_kernel(int64_t N, const double2* __restrict__ A, int64_t lda,
                            double2* __restrict__ d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) d[i] = A[i + i * lda];
}

__global__ void exps_kernel(int64_t n, const unsigned long long* __restrict__ mx, int* __restrict__ e) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) e[i] = scale_exp(__longlong_as_double((long long)mx[i]));
}

// A (M x K, column-major) -> OS digit planes, each M rows x 2 Np (row-major
// [Ar | Ai]), stacked; skip_diag leaves the diagonal out (square A).
__global__ void slice_a_kernel(int64_t M, int64_t K, int64_t Np, bool skip_diag,
                               const double2* __restrict__ A, int64_t lda,
                               const int* __restrict__ ea, __nv_bfloat16* __restrict__ out) {
  __shared__ double2 tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + tx, k = k0 + r;
    tile[r][tx] = (i < M && k < K) ? A[i + k * lda] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int64_t ld = 2 * Np;
  const size_t plane = (size_t)M * ld;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, k = k0 + tx;
    if (i < M && k < K) {
      const double2 a = (skip_diag && i == k) ? make_double2(0.0, 0.0) : tile[tx][r];
      const double s = ldexp(1.0, -ea[i]);
      __nv_bfloat16 dr[OS], di[OS];
      digits_of(a.x * s, dr);
      digits_of(a.y * s, di);
#pragma unroll
      for (int d = 0; d < OS; ++d) {
        out[d * plane + i * ld + k] = dr[d];
        out[d * plane + i * ld + Np + k] = di[d];
      }
    }
  }
}

// X (M x K, column-major) <- the value its six digits represent when X is the
// left operand (row i scaled by 2^-e_i): sum_s d_s 2^(e_i - 8s).
__global__ void round_left_kernel(int64_t M, int64_t K, double2* __restrict__ X, int64_t ldx,
                                  const int* __restrict__ ea) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y;
  if (i >= M || k >= K) return;
  const double2 x = X[i + k * ldx];
  const double s = ldexp(1.0, -ea[i]);
  __nv_bfloat16 dr[OS], di[OS];
  digits_of(x.x * s, dr);
  digits_of(x.y * s, di);
  double vr = 0.0, vi = 0.0;
#pragma unroll
  for (int d = OS - 1; d >= 0; --d) {  // exact: 48 bits below the scale
    vr = (vr + __bfloat162float(dr[d])) * (1.0 / 256.0);
    vi = (vi + __bfloat162float(di[d])) * (1.0 / 256.0);
  }
  X[i + k * ldx] = make_double2(ldexp(vr, ea[i]), ldexp(vi, ea[i]));
}

// Left operand X^H for X (K x M, column-major): row i of X^H is conj(X[:, i]),
// contiguous, so no transpose is needed. Exponents per row come from colexp.
__global__ void slice_ct_kernel(int64_t M, int64_t K, int64_t Np, const double2* __restrict__ X,
                                int64_t ldx, const int* __restrict__ ea,
                                __nv_bfloat16* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (k >= K) return;
  const double2 x = X[k + i * ldx];
  const double s = ldexp(1.0, -ea[i]);
  __nv_bfloat16 dr[OS], di[OS];
  digits_of(x.x * s, dr);
  digits_of(-x.y * s, di);
  const int64_t ld = 2 * Np;
  const size_t plane = (size_t)M * ld;
#pragma unroll
  for (int d = 0; d < OS; ++d) {
    out[d * plane + i * ld + k] = dr[d];
    out[d * plane + i * ld + Np + k] = di[d];
  }
}

// Column maxima of Y (complex columns j0 .. j0 + gridDim.x): one CTA per column.
__global__ void colexp_kernel(int64_t N, int64_t j0, const double2* __restrict__ Y, int64_t ldy,
                              int* __restrict__ eb) {
  __shared__ double red[256];
  const int64_t j = j0 + blockIdx.x;
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < N; k += 256) {
    const double2 y = Y[k + j * ldy];
    m = fmax(m, fmax(fabs(y.x), fabs(y.y)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s >= 1; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) eb[j] = scale_exp(red[0]);
}

// Y columns -> OS digit planes of B^T (rows: 32-column tiles of 64 rows), stacked
// with `brows` rows per plane. Real row: [Yr | -Yi]; imaginary row: [Yi | Yr].
__global__ void slice_b_kernel(int64_t N, int64_t Np, int64_t brows, int64_t j0,
                               const double2* __restrict__ Y, int64_t ldy, const int* __restrict__ eb,
                               __nv_bfloat16* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = j0 + blockIdx.y;
  if (k >= N) return;
  const double2 y = Y[k + j * ldy];
  const double s = ldexp(1.0, -eb[j]);
  __nv_bfloat16 dr[OS], di[OS];
  digits_of(y.x * s, dr);
  digits_of(y.y * s, di);
  const int64_t ld = 2 * Np;
  const size_t plane = (size_t)brows * ld;
  const int64_t br = brow_re(j), bi = br + CT;
#pragma unroll
  for (int d = 0; d < OS; ++d) {
    __nv_bfloat16* o = out + d * plane;
    const __nv_bfloat16 ndi = __hneg(di[d]);
    o[br * ld + k] = dr[d];
    o[br * ld + Np + k] = ndi;
    o[bi * ld + k] = di[d];
    o[bi * ld + Np + k] = dr[d];
  }
}

// The right-operand digits of many problems' filter steps in one launch: one
// CTA (256 threads) per active column of every problem. It forms the column's
// maximum with the reduction of colexp_kernel, then the column's digits as
// slice_b_kernel does, so each problem's planes are those of its own launches.
struct OzSliceEntry {
  const double2* B;          // right operand (absolute columns, ld ldb)
  int64_t ldb, N, Np, brows, j0;
  int* eb;                   // column exponents
  __nv_bfloat16* out;        // digit planes
  int first, pad;            // first CTA of this problem
};

__global__ void __launch_bounds__(256)
    slice_b_grouped_kernel(const OzSliceEntry* __restrict__ tab, int count) {
  __shared__ double red[256];
  __shared__ int s_e;
  const int id = (int)blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {  // last entry with first <= id
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].first <= id) lo = mid;
    else hi = mid - 1;
  }
  const OzSliceEntry& e = tab[lo];
  const int64_t N = e.N, j = e.j0 + (id - e.first);
  const double2* __restrict__ Y = e.B + j * e.ldb;
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < N; k += 256) {
    const double2 y = Y[k];
    m = fmax(m, fmax(fabs(y.x), fabs(y.y)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    s_e = scale_exp(red[0]);
    e.eb[j] = s_e;
  }
  __syncthreads();
  const double sc = ldexp(1.0, -s_e);
  const int64_t ld = 2 * e.Np;
  const size_t plane = (size_t)e.brows * ld;
  const int64_t br = brow_re(j), bi = br + CT;
  for (int64_t k = threadIdx.x; k < N; k += 256) {
    const double2 y = Y[k];
    __nv_bfloat16 dr[OS], di[OS];
    digits_of(y.x * sc, dr);
    digits_of(y.y * sc, di);
#pragma unroll
    for (int d = 0; d < OS; ++d) {
      __nv_bfloat16* o = e.out + d * plane;
      const __nv_bfloat16 ndi = __hneg(di[d]);
      o[br * ld + k] = dr[d];
      o[br * ld + e.Np + k] = ndi;
      o[bi * ld + k] = di[d];
      o[bi * ld + e.Np + k] = dr[d];
    }
  }
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
  CUtensorMap a, b;
};

// Launch parameters of A * B[:, j0:ncols_end] with epilogue ep (A's digits in w).
Params product_params(const OzakiWork& w, int64_t ncols_end, int64_t j0, const double2* B,
                      int64_t ldb, const Epilogue& ep) {
  Params P;
  P.N = w.N;
  P.Np = w.Np;
  P.brows = w.brows;
  P.arows = w.N;
  P.j0 = j0;
  P.ncols = ncols_end;
  P.escale_a = w.ea;
  P.escale_b = w.eb;
  P.diag = w.diag;
  P.Bsrc = B;
  P.ldbs = ldb;
  P.mode = ep.mode;
  P.alpha = ep.alpha;
  P.beta = ep.beta;
  P.gamma = ep.gamma;
  P.X = ep.X;
  P.ldx = ep.ldx;
  P.Y = ep.Y;
  P.ldy = ep.ldy;
  P.theta = ep.theta;
  P.partial = ep.partial;
  P.err = w.err;
  return P;
}

}  // namespace

int64_t ozaki_np(int64_t N) { return cdiv(N, KPAD) * KPAD; }

cudaError_t ozaki_alloc(OzakiWork& w, int64_t N, int64_t ne) {
  w.N = N;
  w.ne = ne;
  w.Np = ozaki_np(N);
  w.brows = cdiv(ne, CT) * TN;
  const size_t a_elems = (size_t)OS * N * 2 * w.Np;
  const size_t b_elems = (size_t)OS * w.brows * 2 * w.Np;
  if (!get_encoder()) return cudaErrorNotSupported;
  cudaError_t e;
  if ((e = cudaMalloc(&w.Ad, a_elems * 2)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.Bd, b_elems * 2)) != cudaSuccess) return e;
  if ((e = cudaMemset(w.Ad, 0, a_elems * 2)) != cudaSuccess) return e;
  if ((e = cudaMemset(w.Bd, 0, b_elems * 2)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.ea, N * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.eb, ne * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.amax, N * sizeof(unsigned long long))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.diag, N * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.err, sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemset(w.err, 0, sizeof(int))) != cudaSuccess) return e;
  // general left operands of the N x n^2 products: X^H (ne x N) or Q (N x ne)
  const int64_t npe = ozaki_np(ne);
  w.l_elems = (size_t)OS * std::max((size_t)ne * 2 * w.Np, (size_t)N * 2 * npe);
  if ((e = cudaMalloc(&w.Ld, w.l_elems * 2)) != cudaSuccess) return e;
  if ((e = cudaMemset(w.Ld, 0, w.l_elems * 2)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.el, std::max(N, ne) * sizeof(int))) != cudaSuccess) return e;
  Maps* maps = nullptr;
  if ((e = cudaMallocHost(&maps, sizeof(Maps))) != cudaSuccess) return e;
  w.maps = maps;
  // digit planes stacked along rows: OS * N rows (A), OS * brows rows (B)
  if (!make_map(&maps->a, w.Ad, (int64_t)OS * N, w.Np, TM) ||
      !make_map(&maps->b, w.Bd, (int64_t)OS * w.brows, w.Np, TN))
    return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(ozaki_gemm_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_BYTES)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(ozaki_gemm_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              SMEM_BYTES);
}

void ozaki_free(OzakiWork& w) {
  void* bufs[] = {w.Ad, w.Bd, w.ea, w.eb, w.amax, w.err, w.diag, w.Ld, w.el};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (w.maps) cudaFreeHost(w.maps);
  w = OzakiWork{};
}

cudaError_t ozaki_prepare_a(cudaStream_t s, const double2* A, int64_t lda, OzakiWork& w) {
  const int64_t N = w.N;
  cudaError_t e = cudaMemsetAsync(w.amax, 0, N * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  rowmax_kernel<<<dim3((unsigned)cdiv(N, 256), (unsigned)cdiv(N, 256), 1), 256, 0, s>>>(
      N, N, true, A, lda, w.amax);
  count_launch();
  exps_kernel<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(N, w.amax, w.ea);
  count_launch();
  diag_kernel<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(N, A, lda, w.diag);
  count_launch();
  slice_a_kernel<<<dim3((unsigned)cdiv(N, 32), (unsigned)cdiv(N, 32), 1), dim3(32, 8, 1), 0, s>>>(
      N, N, w.Np, true, A, lda, w.ea, static_cast<__nv_bfloat16*>(w.Ad));
  count_launch();
  w.A_ready = A;
  return cudaGetLastError();
}

cudaError_t ozaki_gemm(cudaStream_t s, int64_t ncols_end, int64_t j0, const double2* B,
                       int64_t ldb, const Epilogue& ep, OzakiWork& w) {
  const int64_t N = w.N;
  const int64_t n = ncols_end - j0;
  if (n <= 0) return cudaSuccess;
  // digits of the active columns of B
  colexp_kernel<<<(unsigned)n, 256, 0, s>>>(N, j0, B, ldb, w.eb);
  count_launch();
  slice_b_kernel<<<dim3((unsigned)cdiv(N, 256), (unsigned)n, 1), 256, 0, s>>>(
      N, w.Np, w.brows, j0, B, ldb, w.eb, static_cast<__nv_bfloat16*>(w.Bd));
  count_launch();
  const Maps* maps = static_cast<const Maps*>(w.maps);
  const Params P = product_params(w, ncols_end, j0, B, ldb, ep);
  const dim3 grid((unsigned)cdiv(N, TM), (unsigned)((ncols_end - 1) / CT - j0 / CT + 1), 1);
  ozaki_gemm_kernel<7><<<grid, NTHREADS, SMEM_BYTES, s>>>(maps->a, maps->b, P);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_gemm_general(cudaStream_t s, int64_t M, int64_t K, const double2* X,
                               int64_t ldx, bool conj_trans, int64_t ncols, const double2* B,
                               int64_t ldb, const Epilogue& ep, OzakiWork& w, bool extended) {
  if (M <= 0 || ncols <= 0 || K <= 0) return cudaSuccess;
  const int64_t Kp = ozaki_np(K);
  if (Kp > w.Np || ncols > w.ne || (size_t)OS * M * 2 * Kp > w.l_elems)
    return cudaErrorInvalidValue;
  __nv_bfloat16* L = static_cast<__nv_bfloat16*>(w.Ld);
  // The K padding of the left planes must be zero (the right operand's padding
  // then only has to be finite, which digits always are). The slicing writes
  // k < K only, so the planes are cleared whenever their layout changes.
  cudaError_t e;
  if (M != w.l_M || K != w.l_K) {
    if ((e = cudaMemsetAsync(L, 0, (size_t)OS * M * 2 * Kp * 2, s)) != cudaSuccess) return e;
    w.l_M = M;
    w.l_K = K;
  }
  if (conj_trans) {  // left = X^H, X is K x M
    colexp_kernel<<<(unsigned)M, 256, 0, s>>>(K, 0, X, ldx, w.el);
    count_launch();
    slice_ct_kernel<<<dim3((unsigned)cdiv(K, 256), (unsigned)M, 1), 256, 0, s>>>(M, K, Kp, X, ldx,
                                                                                 w.el, L);
    count_launch();
  } else {           // left = X, M x K
    if ((e = cudaMemsetAsync(w.amax, 0, M * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    rowmax_kernel<<<dim3((unsigned)cdiv(M, 256), (unsigned)cdiv(K, 256), 1), 256, 0, s>>>(
        M, K, false, X, ldx, w.amax);
    count_launch();
    exps_kernel<<<(unsigned)cdiv(M, 256), 256, 0, s>>>(M, w.amax, w.el);
    count_launch();
    slice_a_kernel<<<dim3((unsigned)cdiv(M, 32), (unsigned)cdiv(K, 32), 1), dim3(32, 8, 1), 0, s>>>(
        M, K, Kp, false, X, ldx, w.el, L);
    count_launch();
  }
  // right operand digits, K rows
  colexp_kernel<<<(unsigned)ncols, 256, 0, s>>>(K, 0, B, ldb, w.eb);
  count_launch();
  slice_b_kernel<<<dim3((unsigned)cdiv(K, 256), (unsigned)ncols, 1), 256, 0, s>>>(
      K, Kp, w.brows, 0, B, ldb, w.eb, static_cast<__nv_bfloat16*>(w.Bd));
  count_launch();
  CUtensorMap ma, mb;
  if (!make_map(&ma, L, (int64_t)OS * M, Kp, TM) ||
      !make_map(&mb, w.Bd, (int64_t)OS * w.brows, Kp, TN))
    return cudaErrorInvalidValue;
  Params P;
  P.N = M;
  P.Np = Kp;
  P.brows = w.brows;
  P.arows = M;
  P.j0 = 0;
  P.ncols = ncols;
  P.escale_a = w.el;
  P.escale_b = w.eb;
  P.diag = nullptr;
  P.Bsrc = B;
  P.ldbs = ldb;
  P.mode = ep.mode;
  P.alpha = ep.alpha;
  P.beta = ep.beta;
  P.gamma = ep.gamma;
  P.X = ep.X;
  P.ldx = ep.ldx;
  P.Y = ep.Y;
  P.ldy = ep.ldy;
  P.theta = ep.theta;
  P.partial = ep.partial;
  P.err = w.err;
  const dim3 grid((unsigned)cdiv(M, TM), (unsigned)((ncols - 1) / CT + 1), 1);
  if (extended)
    ozaki_gemm_kernel<8><<<grid, NTHREADS, SMEM_BYTES, s>>>(ma, mb, P);
  else
    ozaki_gemm_kernel<7><<<grid, NTHREADS, SMEM_BYTES, s>>>(ma, mb, P);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_round_left(cudaStream_t s, int64_t M, int64_t K, double2* X, int64_t ldx,
                             OzakiWork& w) {
  if (M <= 0 || K <= 0) return cudaSuccess;
  if (M > w.N) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(w.amax, 0, M * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  rowmax_kernel<<<dim3((unsigned)cdiv(M, 256), (unsigned)cdiv(K, 256), 1), 256, 0, s>>>(
      M, K, false, X, ldx, w.amax);
  count_launch();
  exps_kernel<<<(unsigned)cdiv(M, 256), 256, 0, s>>>(M, w.amax, w.el);
  count_launch();
  round_left_kernel<<<dim3((unsigned)cdiv(M, 256), (unsigned)K, 1), 256, 0, s>>>(M, K, X, ldx,
                                                                                 w.el);
  count_launch();
  return cudaGetLastError();
}

namespace {
__global__ void exp_max_kernel(int64_t n, const int* __restrict__ e, int* __restrict__ out) {
  __shared__ int red[256];
  int m = -100000;
  for (int64_t i = threadIdx.x; i < n; i += 256) m = max(m, e[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}
}  // namespace

cudaError_t ozaki_left_exp_max(cudaStream_t s, int64_t M, OzakiWork& w, int* out) {
  if (M <= 0) return cudaSuccess;
  exp_max_kernel<<<1, 256, 0, s>>>(M, w.el, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_group_reserve(OzakiGroupTable& t, size_t entries) {
  if (entries <= t.capacity) return cudaSuccess;
  ozaki_group_free(t);
  cudaError_t e;
  if ((e = cudaMalloc(&t.dev, entries * sizeof(OzGroupEntry))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&t.host, entries * sizeof(OzGroupEntry))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&t.sdev, entries * sizeof(OzSliceEntry))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&t.shost, entries * sizeof(OzSliceEntry))) != cudaSuccess) return e;
  t.capacity = entries;
  return cudaSuccess;
}

void ozaki_group_free(OzakiGroupTable& t) {
  if (t.dev) cudaFree(t.dev);
  if (t.host) cudaFreeHost(t.host);
  if (t.sdev) cudaFree(t.sdev);
  if (t.shost) cudaFreeHost(t.shost);
  t = OzakiGroupTable{};
}

size_t ozaki_group_entries(int count, const OzakiGroupItem* items) {
  size_t n = 0;
  for (int k = 0; k < count; ++k)
    if (items[k].ncols > 0) n += (size_t)items[k].degs[items[k].ncols - 1];
  return n;
}

int ozaki_filter_grouped(cudaStream_t s, int count, const OzakiGroupItem* items,
                         OzakiGroupTable& t, int* launches) {
  static std::once_flag attr_once[kMaxDevices];
  once_per_device(attr_once, []() {
    cudaFuncSetAttribute(ozaki_filter_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM_BYTES);
  });
  int dmax_all = 0;
  for (int k = 0; k < count; ++k) {
    const OzakiGroupItem& it = items[k];
    if (it.ncols == 0) continue;
    if (!it.w || !it.w->maps || !it.w->A_ready || it.N != it.w->N || it.ncols > it.w->ne ||
        !it.V || !it.W || it.ldv < it.N || it.ldw < it.N)
      return CHASE_ERR_INVALID_ARG;
    dmax_all = std::max(dmax_all, (int)it.degs[it.ncols - 1]);
  }
  if (dmax_all == 0) return CHASE_OK;
  if (ozaki_group_entries(count, items) > t.capacity) return CHASE_ERR_INVALID_ARG;
  // step table: for step i the entries of the problems still filtering, with
  // their first CTA indices (gemm) and first column indices (digits)
  OzGroupEntry* host = static_cast<OzGroupEntry*>(t.host);
  OzSliceEntry* shost = static_cast<OzSliceEntry*>(t.shost);
  std::vector<size_t> off(dmax_all + 2, 0);
  std::vector<int> ctas(dmax_all + 1, 0), cols(dmax_all + 1, 0);
  size_t n = 0;
  for (int i = 1; i <= dmax_all; ++i) {
    off[i] = n;
    int first = 0, sfirst = 0;
    for (int k = 0; k < count; ++k) {
      const OzakiGroupItem& it = items[k];
      if (it.ncols == 0 || it.degs[it.ncols - 1] < i) continue;
      OzakiWork& w = *it.w;
      // the per-problem filter's step i (Eq. 1): Y_d = al[i] (A - c I) Y_s + be[i] Y_d
      const int64_t j0 = std::lower_bound(it.degs, it.degs + it.ncols, i) - it.degs;
      double2* buf[2] = {it.V, it.W};
      const int64_t ld[2] = {it.ldv, it.ldw};
      const int sp = (i - 1) & 1, d = i & 1;
      Epilogue ep{};
      ep.mode = EPI_FILTER;
      ep.alpha = it.al[i];
      ep.beta = (i == 1) ? 0.0 : it.be[i];
      ep.gamma = it.c;
      ep.X = buf[sp];
      ep.ldx = ld[sp];
      ep.Y = buf[d];
      ep.ldy = ld[d];
      OzSliceEntry& se = shost[n];
      se.B = buf[sp];
      se.ldb = ld[sp];
      se.N = it.N;
      se.Np = w.Np;
      se.brows = w.brows;
      se.j0 = j0;
      se.eb = w.eb;
      se.out = static_cast<__nv_bfloat16*>(w.Bd);
      se.first = sfirst;
      se.pad = 0;
      sfirst += (int)(it.ncols - j0);
      OzGroupEntry& e = host[n];
      const Maps* maps = static_cast<const Maps*>(w.maps);
      e.a = maps->a;
      e.b = maps->b;
      e.P = product_params(w, it.ncols, j0, buf[sp], ld[sp], ep);
      e.nrow = (int)cdiv(it.N, TM);
      e.ncol = (int)((it.ncols - 1) / CT - j0 / CT + 1);
      e.first = first;
      e.pad = 0;
      first += e.nrow * e.ncol;
      ++n;
    }
    ctas[i] = first;
    cols[i] = sfirst;
  }
  off[dmax_all + 1] = n;
  if (cudaMemcpyAsync(t.dev, host, n * sizeof(OzGroupEntry), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(t.sdev, shost, n * sizeof(OzSliceEntry), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    return CHASE_CUDA_FAIL();
  // the degree steps of all problems as one CUDA graph: per step one grouped
  // digit launch and one grouped product launch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  const OzGroupEntry* dev = static_cast<const OzGroupEntry*>(t.dev);
  const OzSliceEntry* sdev = static_cast<const OzSliceEntry*>(t.sdev);
  for (int i = 1; i <= dmax_all; ++i) {
    const int cnt = (int)(off[i + 1] - off[i]);
    slice_b_grouped_kernel<<<(unsigned)cols[i], 256, 0, s>>>(sdev + off[i], cnt);
    count_launch();
    ozaki_filter_grouped_kernel<<<(unsigned)ctas[i], NTHREADS, SMEM_BYTES, s>>>(dev + off[i],
                                                                               cnt);
    count_launch();
  }
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (ce != cudaSuccess || !graph) return CHASE_CUDA_FAIL();
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return CHASE_CUDA_FAIL();
  const cudaError_t le = cudaGraphLaunch(exec, s);
  const cudaError_t se = le == cudaSuccess ? cudaStreamSynchronize(s) : le;
  cudaGraphExecDestroy(exec);
  if (se != cudaSuccess) return CHASE_CUDA_FAIL();
  if (launches) *launches = 2 * dmax_all;
  int rc = CHASE_OK;
  for (int k = 0; k < count; ++k)
    if (items[k].ncols > 0) {
      const int r = ozaki_check(s, *items[k].w);
      if (rc == CHASE_OK) rc = r;
    }
  return rc;
}

int ozaki_check(cudaStream_t s, OzakiWork& w) {
  int herr = 0;
  if (cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  if (herr != 0) {
    fprintf(stderr, "[chase] emulated-FP64 GEMM: pipeline wait expired (code %d)\n", herr);
    cudaMemsetAsync(w.err, 0, sizeof(int), s);
    return CHASE_CUDA_FAIL();
  }
  return CHASE_OK;
}

}  // namespace chase
