// Complex FP64 GEMM kernels on the DFMA pipe.
//
// On sm_103 the FP64 rate is two DFMA per clock per SM (about 1.2 TFLOP/s for
// the GPU), so every product here is bound by the FP64 pipe as soon as a tile
// reuses each loaded element a few times. The kernels use 64 x 64 output tiles,
// 256 threads with 4 x 4 complex accumulators each, and double-buffered shared
// memory; the epilogues fuse the Chebyshev three-term update (Eq. 1), plain
// stores, and the per-column residual sums of squares (Alg. 2 residual lines).
#include <algorithm>

#include "common.cuh"

namespace chase {
namespace {

constexpr int BM = 64, BN = 64, BK = 8, NT = 256;
constexpr int kMaxSplits = 8;

// A operand: normal (M x K column-major) or conjugate-transpose of a K x M
// column-major X (Gram products X^H Y).
template <bool ACONJT>
__device__ __forceinline__ void load_a(const double2* __restrict__ A, int64_t lda, int64_t M,
                                       int64_t m0, int64_t k0, int64_t kend, int t,
                                       double2 (&ra)[2]) {
  if (!ACONJT) {
    const int r = t & 63, kk = t >> 6;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t row = m0 + r, k = k0 + kk + 4 * h;
      ra[h] = (row < M && k < kend) ? A[row + k * lda] : make_double2(0.0, 0.0);
    }
  } else {
    const int kk = t & 7, r = t >> 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t row = m0 + r + 32 * h, k = k0 + kk;
      ra[h] = (row < M && k < kend) ? conjz(A[k + row * lda]) : make_double2(0.0, 0.0);
    }
  }
}

template <bool ACONJT>
__device__ __forceinline__ void store_a(double2 (*As)[BM], int t, const double2 (&ra)[2]) {
  if (!ACONJT) {
    const int r = t & 63, kk = t >> 6;
    As[kk][r] = ra[0];
    As[kk + 4][r] = ra[1];
  } else {
    const int kk = t & 7, r = t >> 3;
    As[kk][r] = ra[0];
    As[kk][r + 32] = ra[1];
  }
}

__device__ __forceinline__ void load_b(const double2* __restrict__ B, int64_t ldb, int64_t n,
                                       int64_t n0, int64_t k0, int64_t kend, int t,
                                       double2 (&rb)[2]) {
  const int kk = t & 7, c = t >> 3;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t col = n0 + c + 32 * h, k = k0 + kk;
    rb[h] = (col < n && k < kend) ? B[k + col * ldb] : make_double2(0.0, 0.0);
  }
}

__device__ __forceinline__ void store_b(double2 (*Bs)[BN], int t, const double2 (&rb)[2]) {
  const int kk = t & 7, c = t >> 3;
  Bs[kk][c] = rb[0];
  Bs[kk][c + 32] = rb[1];
}

// One 64 x 64 tile of P = op(A) * B over k in [kbeg, kend).
template <bool ACONJT, int EPI>
__global__ void __launch_bounds__(NT)
    zgemm_kernel(int64_t M, int64_t n, int64_t K, const double2* __restrict__ A, int64_t lda,
                 const double2* __restrict__ B, int64_t ldb, Epilogue ep, int64_t kchunk,
                 int64_t split_stride, bool upper_only) {
  if (upper_only && blockIdx.x > blockIdx.y) return;
  __shared__ double2 As[2][BK][BM];
  __shared__ double2 Bs[2][BK][BN];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);

  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  const int64_t nkt = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  double2 ra[2], rb[2];
  if (nkt > 0) {
    load_a<ACONJT>(A, lda, M, m0, kbeg, kend, t, ra);
    load_b(B, ldb, n, n0, kbeg, kend, t, rb);
    store_a<ACONJT>(As[0], t, ra);
    store_b(Bs[0], t, rb);
  }
  __syncthreads();
  for (int64_t kt = 0; kt < nkt; ++kt) {
    const int cur = kt & 1;
    const bool more = kt + 1 < nkt;
    if (more) {
      const int64_t k0 = kbeg + (kt + 1) * BK;
      load_a<ACONJT>(A, lda, M, m0, k0, kend, t, ra);
      load_b(B, ldb, n, n0, k0, kend, t, rb);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[cur][kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[cur][kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    if (more) {
      store_a<ACONJT>(As[cur ^ 1], t, ra);
      store_b(Bs[cur ^ 1], t, rb);
    }
    __syncthreads();
  }

  // ------------------------------------------------------------- epilogue
  if (EPI == EPI_STORE) {
    double2* Y = ep.Y + (int64_t)blockIdx.z * split_stride;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t col = n0 + ty + 16 * j;
      if (col >= n) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t row = m0 + tx + 16 * i;
        if (row < M) Y[row + col * ep.ldy] = acc[i][j];
      }
    }
  } else if (EPI == EPI_FILTER) {
    // Eq. 1: Y_new = alpha (A Y_cur - gamma Y_cur) + beta Y_prev, in place over Y_prev.
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t col = n0 + ty + 16 * j;
      if (col >= n) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t row = m0 + tx + 16 * i;
        if (row >= M) continue;
        const double2 x = ep.X[row + col * ep.ldx];
        double2 v = make_double2(ep.alpha * fma(-ep.gamma, x.x, acc[i][j].x),
                                 ep.alpha * fma(-ep.gamma, x.y, acc[i][j].y));
        double2* yp = ep.Y + row + col * ep.ldy;
        if (ep.beta != 0.0) {
          const double2 y = *yp;
          v.x = fma(ep.beta, y.x, v.x);
          v.y = fma(ep.beta, y.y, v.y);
        }
        *yp = v;
      }
    }
  } else {  // EPI_RESID: sum_rows |P - theta_col X|^2 for this row tile
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t col = n0 + ty + 16 * j;
      double s = 0.0;
      if (col < n) {
        const double th = ep.theta[col];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t row = m0 + tx + 16 * i;
          if (row < M) {
            const double2 x = ep.X[row + col * ep.ldx];
            const double dx = fma(-th, x.x, acc[i][j].x), dy = fma(-th, x.y, acc[i][j].y);
            s = fma(dx, dx, fma(dy, dy, s));
          }
        }
      }
#pragma unroll
      for (int off = 8; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (tx == 0 && col < n) ep.partial[blockIdx.x + col * gridDim.x] = s;
    }
  }
}

__global__ void resid_reduce_kernel(const double* __restrict__ partial, int64_t ntiles, int64_t n,
                                    double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int64_t t = 0; t < ntiles; ++t) s += partial[t + j * ntiles];
  out[j] = sqrt(s);
}

// G[i, j] = sum_z ws[z][i + j m] (fixed order); hermitian: lower from upper.
__global__ void gram_reduce_kernel(int64_t m, int64_t n, int splits, const double2* __restrict__ ws,
                                   double2* __restrict__ G, int64_t ldg, bool hermitian) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= m) return;
  const size_t mn = (size_t)m * n;
  double2 v = make_double2(0.0, 0.0);
  if (!hermitian || i <= j) {
    for (int z = 0; z < splits; ++z) v = cadd(v, ws[z * mn + i + j * m]);
    if (hermitian && i == j) v.y = 0.0;
  } else {
    for (int z = 0; z < splits; ++z) v = cadd(v, ws[z * mn + j + i * m]);
    v = conjz(v);
  }
  G[i + j * ldg] = v;
}

__global__ void hermitian_part_kernel(int64_t n, double2* G, int64_t ldg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n || i > j) return;
  if (i == j) {
    G[i + i * ldg].y = 0.0;
    return;
  }
  const double2 a = G[i + j * ldg], b = G[j + i * ldg];
  const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  G[i + j * ldg] = h;
  G[j + i * ldg] = conjz(h);
}

// ------------------------------------------------------------- skinny GEMM
constexpr int SK_ROWS = 128, SK_K = 128, kMaxSkinnySplits = 64;

template <int NV>
__global__ void __launch_bounds__(SK_ROWS)
    skinny_kernel(int64_t M, int n, const double2* __restrict__ A, int64_t lda,
                  const double2* __restrict__ B, int64_t ldb, double2* __restrict__ ws,
                  int64_t kchunk) {
  __shared__ double2 Bs[SK_K][NV];
  const int t = threadIdx.x;
  const int64_t row = (int64_t)blockIdx.x * SK_ROWS + t;
  const int64_t k0 = (int64_t)blockIdx.y * kchunk;
  const int64_t k1 = min(M, k0 + kchunk);
  double2 acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = make_double2(0.0, 0.0);
  for (int64_t kb = k0; kb < k1; kb += SK_K) {
    for (int e = t; e < SK_K * NV; e += SK_ROWS) {
      const int kk = e % SK_K, c = e / SK_K;
      const int64_t k = kb + kk;
      Bs[kk][c] = (k < k1 && c < n) ? B[k + c * ldb] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int kn = (int)min((int64_t)SK_K, k1 - kb);
    if (row < M) {
      for (int kk = 0; kk < kn; ++kk) {
        const double2 a = A[row + (kb + kk) * lda];
#pragma unroll
        for (int c = 0; c < NV; ++c) cfma(acc[c], a, Bs[kk][c]);
      }
    }
    __syncthreads();
  }
  if (row < M) {
    double2* w = ws + (size_t)blockIdx.y * M * NV;
#pragma unroll
    for (int c = 0; c < NV; ++c) w[row + c * M] = acc[c];
  }
}

template <int NV>
__global__ void skinny_reduce_kernel(int64_t M, int n, int splits, const double2* __restrict__ ws,
                                     double2* __restrict__ P, int64_t ldp) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= M) return;
  for (int c = 0; c < n; ++c) {
    double2 v = make_double2(0.0, 0.0);
    for (int z = 0; z < splits; ++z) v = cadd(v, ws[(size_t)z * M * NV + row + c * M]);
    P[row + c * ldp] = v;
  }
}

std::once_flag g_sms_once[kMaxDevices];
int g_num_sms[kMaxDevices] = {};

}  // namespace

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 152;
  once_per_device(g_sms_once, [dev]() {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
    g_num_sms[dev] = n;
  });
  return g_num_sms[dev];
}

int64_t zgemm_row_tiles(int64_t M) { return cdiv(M, BM); }

cudaError_t zgemm_nn(cudaStream_t s, int64_t M, int64_t n, int64_t K, const double2* A,
                     int64_t lda, const double2* B, int64_t ldb, const Epilogue& ep) {
  if (M <= 0 || n <= 0) return cudaSuccess;
  dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(n, BN), 1);
  switch (ep.mode) {
    case EPI_STORE:
      zgemm_kernel<false, EPI_STORE><<<grid, NT, 0, s>>>(M, n, K, A, lda, B, ldb, ep, K, 0, false); count_launch();
      break;
    case EPI_FILTER:
      zgemm_kernel<false, EPI_FILTER><<<grid, NT, 0, s>>>(M, n, K, A, lda, B, ldb, ep, K, 0, false); count_launch();
      break;
    default:
      zgemm_kernel<false, EPI_RESID><<<grid, NT, 0, s>>>(M, n, K, A, lda, B, ldb, ep, K, 0, false); count_launch();
      break;
  }
  return cudaGetLastError();
}

cudaError_t resid_reduce(cudaStream_t s, const double* partial, int64_t ntiles, int64_t n,
                         double* out) {
  if (n <= 0) return cudaSuccess;
  resid_reduce_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(partial, ntiles, n, out); count_launch();
  return cudaGetLastError();
}

size_t gram_workspace_elems(int64_t m, int64_t n) { return (size_t)kMaxSplits * m * n; }

cudaError_t zgram(cudaStream_t s, int64_t K, int64_t m, int64_t n, const double2* X, int64_t ldx,
                  const double2* Y, int64_t ldy, double2* G, int64_t ldg, bool hermitian,
                  double2* ws, size_t ws_elems) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (ws_elems < (size_t)m * n) return cudaErrorInvalidValue;  // no room for one partial
  const int64_t tm = cdiv(m, BM), tn = cdiv(n, BN);
  const int64_t tiles = hermitian ? tm * (tm + 1) / 2 : tm * tn;
  // split-K factor: the one (up to the workspace, 8, and K / 512) whose CTA
  // count fills the last wave best (3 resident CTAs per SM); ties to fewer splits
  const int64_t slots = 3 * (int64_t)num_sms();
  const int64_t smax = std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)kMaxSplits, std::max<int64_t>(1, K / 512),
                            (int64_t)(ws_elems / ((size_t)m * n))}));
  int64_t splits = 1;
  double best = -1.0;
  for (int64_t sp = 1; sp <= smax; ++sp) {
    const int64_t ctas = tiles * sp;
    const double eff = (double)ctas / (double)(cdiv(ctas, slots) * slots);
    if (eff > best + 1e-9) {
      best = eff;
      splits = sp;
    }
  }
  const int64_t kchunk = cdiv(cdiv(K, splits), BK) * BK;
  Epilogue ep{};
  ep.mode = EPI_STORE;
  ep.Y = ws;
  ep.ldy = m;
  dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)splits);
  zgemm_kernel<true, EPI_STORE><<<grid, NT, 0, s>>>(m, n, K, X, ldx, Y, ldy, ep, kchunk,
                                                    m * n, hermitian); count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g2((unsigned)cdiv(m, 128), (unsigned)n, 1);
  gram_reduce_kernel<<<g2, 128, 0, s>>>(m, n, (int)splits, ws, G, ldg, hermitian); count_launch();
  return cudaGetLastError();
}

cudaError_t hermitian_part(cudaStream_t s, int64_t n, double2* G, int64_t ldg) {
  if (n <= 0) return cudaSuccess;
  dim3 g((unsigned)cdiv(n, 128), (unsigned)n, 1);
  hermitian_part_kernel<<<g, 128, 0, s>>>(n, G, ldg); count_launch();
  return cudaGetLastError();
}

size_t skinny_workspace_elems(int64_t M, int64_t n) {
  (void)n;
  return (size_t)kMaxSkinnySplits * M * 8;
}

cudaError_t zgemm_skinny(cudaStream_t s, int64_t M, int64_t n, const double2* A, int64_t lda,
                         const double2* B, int64_t ldb, double2* P, int64_t ldp, double2* ws) {
  if (M <= 0 || n <= 0) return cudaSuccess;
  if (n > 8) return cudaErrorInvalidValue;
  const int64_t rt = cdiv(M, SK_ROWS);
  int64_t splits = std::max<int64_t>(1, std::min<int64_t>(kMaxSkinnySplits, cdiv(4 * num_sms(), rt)));
  const int64_t kchunk = cdiv(cdiv(M, splits), SK_K) * SK_K;
  splits = cdiv(M, kchunk);
  dim3 grid((unsigned)rt, (unsigned)splits, 1);
  const unsigned rb = (unsigned)cdiv(M, 128);
  if (n <= 1) {
    skinny_kernel<1><<<grid, SK_ROWS, 0, s>>>(M, (int)n, A, lda, B, ldb, ws, kchunk); count_launch();
    skinny_reduce_kernel<1><<<rb, 128, 0, s>>>(M, (int)n, (int)splits, ws, P, ldp); count_launch();
  } else if (n <= 2) {
    skinny_kernel<2><<<grid, SK_ROWS, 0, s>>>(M, (int)n, A, lda, B, ldb, ws, kchunk); count_launch();
    skinny_reduce_kernel<2><<<rb, 128, 0, s>>>(M, (int)n, (int)splits, ws, P, ldp); count_launch();
  } else if (n <= 4) {
    skinny_kernel<4><<<grid, SK_ROWS, 0, s>>>(M, (int)n, A, lda, B, ldb, ws, kchunk); count_launch();
    skinny_reduce_kernel<4><<<rb, 128, 0, s>>>(M, (int)n, (int)splits, ws, P, ldp); count_launch();
  } else {
    skinny_kernel<8><<<grid, SK_ROWS, 0, s>>>(M, (int)n, A, lda, B, ldb, ws, kchunk); count_launch();
    skinny_reduce_kernel<8><<<rb, 128, 0, s>>>(M, (int)n, (int)splits, ws, P, ldp); count_launch();
  }
  return cudaGetLastError();
}

}  // namespace chase
