// CholeskyQR building blocks (Alg. 3 / Alg. 4): blocked right-looking upper
// Cholesky G = U^H U with the first failing pivot reported like LAPACK POTRF's
// info, and the triangular solve X <- X U^{-1} done per row panel (rows of
// X U^{-1} are independent, so each CTA solves its own rows left to right and
// needs no grid-wide ordering).
#include <algorithm>

#include "common.cuh"

namespace chase {
namespace {

constexpr int NB = kNB;  // 64
constexpr int FT = 256;  // threads

// Unblocked Cholesky of the kb x kb diagonal block at (k0, k0), in shared
// memory, plus the inverse of the resulting upper-triangular block.
__global__ void __launch_bounds__(FT)
    potf2_kernel(double2* G, int64_t ldg, int64_t k0, int kb, double2* dinv_blk, int* info) {
  extern __shared__ double2 sm[];
  double2* S = sm;             // kb x kb, column-major, ld NB
  double2* W = sm + NB * NB;   // inverse
  __shared__ int failed;
  const int t = threadIdx.x;
  if (*info != 0) return;
  if (t == 0) failed = 0;
  for (int e = t; e < NB * NB; e += FT) {
    const int r = e % NB, c = e / NB;
    S[e] = (r < kb && c < kb && r <= c) ? G[(k0 + r) + (k0 + c) * ldg] : make_double2(0.0, 0.0);
    W[e] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (t == 0) {
      const double p = S[j + j * NB].x;
      if (!(p > 0.0)) {  // also catches NaN
        failed = 1;
        *info = (int)(k0 + j + 1);
      } else {
        S[j + j * NB] = make_double2(sqrt(p), 0.0);
      }
    }
    __syncthreads();
    if (failed) return;
    const double rd = 1.0 / S[j + j * NB].x;
    for (int c = j + 1 + t; c < kb; c += FT) S[j + c * NB] = cscale(rd, S[j + c * NB]);
    __syncthreads();
    // G(r, c) -= conj(U(j, r)) U(j, c) for j < r <= c
    const int rem = kb - j - 1;
    for (int e = t; e < rem * rem; e += FT) {
      const int r = j + 1 + e % rem, c = j + 1 + e / rem;
      if (r <= c) S[r + c * NB] = csub(S[r + c * NB], cmulc(S[j + r * NB], S[j + c * NB]));
    }
    __syncthreads();
  }
  // inverse of the upper-triangular block, one column per thread
  if (t < kb) {
    const int c = t;
    W[c + c * NB] = make_double2(1.0 / S[c + c * NB].x, 0.0);
    for (int r = c - 1; r >= 0; --r) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = r + 1; l <= c; ++l) acc = cadd(acc, cmul(S[r + l * NB], W[l + c * NB]));
      W[r + c * NB] = cscale(-1.0 / S[r + r * NB].x, acc);
    }
  }
  __syncthreads();
  for (int e = t; e < NB * NB; e += FT) {
    const int r = e % NB, c = e / NB;
    if (r < kb && c < kb) G[(k0 + r) + (k0 + c) * ldg] = (r <= c) ? S[e] : make_double2(0.0, 0.0);
    dinv_blk[e] = W[e];
  }
}

// Panel: U(k-block, j) = W^H G(k-block, j) for one 64-column block j.
__global__ void __launch_bounds__(FT)
    panel_kernel(int64_t n, double2* G, int64_t ldg, int64_t k0, int kb, const double2* dinv_blk,
                 const int* info) {
  extern __shared__ double2 sm[];
  double2* Wt = sm;            // W, ld NB
  double2* P = sm + NB * NB;   // G block, ld NB
  if (*info != 0) return;
  const int t = threadIdx.x;
  const int64_t c0 = k0 + kb + (int64_t)blockIdx.x * NB;
  const int cb = (int)min((int64_t)NB, n - c0);
  for (int e = t; e < NB * NB; e += FT) {
    const int r = e % NB, c = e / NB;
    Wt[e] = dinv_blk[e];
    P[e] = (r < kb && c < cb) ? G[(k0 + r) + (c0 + c) * ldg] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int e = t; e < kb * cb; e += FT) {
    const int r = e % kb, c = e / kb;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l <= r; ++l) acc = cadd(acc, cmulc(Wt[l + r * NB], P[l + c * NB]));
    G[(k0 + r) + (c0 + c) * ldg] = acc;
  }
}

// Trailing update of upper tiles: G(i, j) -= sum_l conj(U(l, i)) U(l, j),
// l over the k-block rows, k0 + kb <= i <= j (tile-wise upper).
__global__ void __launch_bounds__(FT)
    trailing_kernel(int64_t n, double2* G, int64_t ldg, int64_t k0, int kb, const int* info) {
  if (*info != 0) return;
  if (blockIdx.x > blockIdx.y) return;
  __shared__ double2 Ui[NB][NB / 4 + 1];  // staged in 4 chunks of 16 rows
  __shared__ double2 Uj[NB][NB / 4 + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t s0 = k0 + kb;
  const int64_t i0 = s0 + (int64_t)blockIdx.x * NB, j0 = s0 + (int64_t)blockIdx.y * NB;
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0.0, 0.0);
  for (int l0 = 0; l0 < kb; l0 += NB / 4) {
    for (int e = t; e < NB * (NB / 4); e += FT) {
      const int ll = e % (NB / 4), c = e / (NB / 4);
      const int64_t l = k0 + l0 + ll;
      const bool okl = (l0 + ll) < kb;
      Ui[c][ll] = (okl && i0 + c < n) ? G[l + (i0 + c) * ldg] : make_double2(0.0, 0.0);
      Uj[c][ll] = (okl && j0 + c < n) ? G[l + (j0 + c) * ldg] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int ll = 0; ll < NB / 4; ++ll) {
      double2 a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = conjz(Ui[tx + 16 * q][ll]);
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Uj[ty + 16 * q][ll];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc[p][q], a[p], b[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t j = j0 + ty + 16 * q;
    if (j >= n) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t i = i0 + tx + 16 * p;
      if (i < n && i <= j) G[i + j * ldg] = csub(G[i + j * ldg], acc[p][q]);
    }
  }
}

// Row-panel triangular solve X <- X U^{-1}. Each CTA owns 64 rows of X and
// walks the 64-column blocks left to right:
//   T = X(rows, jb) - X(rows, 0:jb) U(0:jb, jb);  X(rows, jb) = T W_jb
constexpr int RP = 64, TK = 8;
__global__ void __launch_bounds__(FT)
    trsm_kernel(int64_t m, int64_t n, double2* X, int64_t ldx, const double2* U, int64_t ldu,
                const double2* dinv, const int* info) {
  if (*info != 0) return;
  extern __shared__ double2 sm[];
  double2* Ts = sm;                 // [c'][r]  NB x RP
  double2* Ws = sm + NB * RP;       // [c'][c]  NB x NB
  double2* Xs = Ws + NB * NB;       // [k][r]   TK x RP
  double2* Us = Xs + TK * RP;       // [k][c]   TK x NB
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * RP;
  const int64_t nblk = cdiv(n, NB);
  for (int64_t jb = 0; jb < nblk; ++jb) {
    const int64_t c0 = jb * NB;
    const int cb = (int)min((int64_t)NB, n - c0);
    double2 acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t r = r0 + tx + 16 * p, c = ty + 16 * q;
        acc[p][q] = (r < m && c < cb) ? X[r + (c0 + c) * ldx] : make_double2(0.0, 0.0);
      }
    for (int64_t l0 = 0; l0 < c0; l0 += TK) {
      __syncthreads();
      for (int e = t; e < TK * RP; e += FT) {
        const int r = e % RP, k = e / RP;
        const int64_t row = r0 + r;
        Xs[k * RP + r] = (row < m) ? X[row + (l0 + k) * ldx] : make_double2(0.0, 0.0);
      }
      for (int e = t; e < TK * NB; e += FT) {
        const int k = e % TK, c = e / TK;
        Us[k * NB + c] = (c < cb) ? U[(l0 + k) + (c0 + c) * ldu] : make_double2(0.0, 0.0);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        double2 a[4], b[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) a[p] = Xs[k * RP + tx + 16 * p];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Us[k * NB + ty + 16 * q];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            double2& o = acc[p][q];
            o.x = fma(-a[p].x, b[q].x, o.x);
            o.x = fma(a[p].y, b[q].y, o.x);
            o.y = fma(-a[p].x, b[q].y, o.y);
            o.y = fma(-a[p].y, b[q].x, o.y);
          }
      }
    }
    __syncthreads();
    // T -> shared, W_jb -> shared
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) Ts[(ty + 16 * q) * RP + tx + 16 * p] = acc[p][q];
    const double2* Wb = dinv + jb * NB * NB;
    for (int e = t; e < NB * NB; e += FT) {
      const int cp = e % NB, c = e / NB;
      Ws[cp * NB + c] = Wb[cp + c * NB];
    }
    __syncthreads();
    double2 out[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) out[p][q] = make_double2(0.0, 0.0);
    for (int cp = 0; cp < cb; ++cp) {
      double2 a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = Ts[cp * RP + tx + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Ws[cp * NB + ty + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(out[p][q], a[p], b[q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t r = r0 + tx + 16 * p;
        const int c = ty + 16 * q;
        if (r < m && c < cb) X[r + (c0 + c) * ldx] = out[p][q];
      }
  }
}

__global__ void trace_shift_kernel(int64_t n, double2* G, int64_t ldg, double factor,
                                   double* scratch) {
  __shared__ double red[256];
  const int t = threadIdx.x;
  double s = 0.0;
  for (int64_t i = t; i < n; i += 256) s += G[i + i * ldg].x;
  red[t] = s;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  const double shift = factor * red[0];
  if (t == 0) scratch[0] = shift;
  for (int64_t i = t; i < n; i += 256) G[i + i * ldg].x += shift;
}

// Largest of non-negative doubles (NaN counted as +inf) into *out, which holds
// the bit pattern of a non-negative double (monotone in unsigned order): the
// result does not depend on the order of the atomics.
__device__ __forceinline__ void atomic_max_nonneg(double* out, double v) {
  if (!(v <= 1.7976931348623157e308)) v = __longlong_as_double(0x7ff0000000000000ll);
  atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_max256(double m, double* red) {
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  return red[0];
}

// max over the upper triangle of |U_ij - delta_ij|: one CTA per column
__global__ void __launch_bounds__(256)
    dev_identity_kernel(int64_t n, const double2* __restrict__ U, int64_t ldu,
                        double* __restrict__ out) {
  __shared__ double red[256];
  const int64_t j = blockIdx.x;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i <= j; i += 256) {
    double2 u = U[i + j * ldu];
    if (i == j) u.x -= 1.0;
    m = fmax(m, sqrt(u.x * u.x + u.y * u.y));
  }
  m = block_max256(m, red);
  if (threadIdx.x == 0) atomic_max_nonneg(out, m);
}

// max_j (max_i |R_ij|) / (max_i |X_ij|), |z| = max(|Re z|, |Im z|): one CTA per column
__global__ void __launch_bounds__(256)
    col_ratio_kernel(int64_t m, const double2* __restrict__ R, int64_t ldr,
                     const double2* __restrict__ X, int64_t ldx, double* __restrict__ out) {
  __shared__ double red[256];
  const int64_t j = blockIdx.x;
  double mr = 0.0, mx = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += 256) {
    const double2 r = R[i + j * ldr], x = X[i + j * ldx];
    mr = fmax(mr, fmax(fabs(r.x), fabs(r.y)));
    mx = fmax(mx, fmax(fabs(x.x), fabs(x.y)));
  }
  mr = block_max256(mr, red);
  __syncthreads();
  mx = block_max256(mx, red);
  if (threadIdx.x == 0) atomic_max_nonneg(out, mx > 0.0 ? mr / mx : (mr > 0.0 ? __longlong_as_double(0x7ff0000000000000ll) : 0.0));
}

// strict lower triangle of the n x n M set to zero
__global__ void zero_lower_kernel(int64_t n, double2* __restrict__ M, int64_t ldm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < n && i > j) M[i + j * ldm] = make_double2(0.0, 0.0);
}

// M = I (set) or M -= I (subtract), n x n, ld ldm
__global__ void identity_kernel(int64_t n, double2* __restrict__ M, int64_t ldm, bool subtract) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n) return;
  if (subtract) {
    if (i == j) M[i + j * ldm].x -= 1.0;
  } else {
    M[i + j * ldm] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// kb x kb diagonal-block inverse (ld NB) into the diagonal block of Y (ld ldy)
__global__ void copy_dinv_kernel(int kb, const double2* __restrict__ W, double2* __restrict__ Y,
                                 int64_t ldy) {
  const int r = threadIdx.x, c = blockIdx.x;
  if (r < kb && c < kb) Y[r + (int64_t)c * ldy] = r <= c ? W[r + c * NB] : make_double2(0.0, 0.0);
}

// Y = U^{-1} for the leading n x n block of U (upper triangular, diagonal-block
// inverses in dinv, block b at dinv + b NB^2), recursively:
// inv([[U11, U12], [0, U22]]) = [[Y11, -Y11 U12 Y22], [0, Y22]], split at a
// multiple of NB so the leaves are the stored diagonal-block inverses.
cudaError_t trinv_rec(cudaStream_t s, int64_t n, const double2* U, int64_t ldu,
                      const double2* dinv, double2* Y, int64_t ldy, double2* T) {
  if (n <= NB) {
    copy_dinv_kernel<<<(unsigned)n, NB, 0, s>>>((int)n, dinv, Y, ldy); count_launch();
    return cudaGetLastError();
  }
  const int64_t n1 = cdiv(cdiv(n, 2), NB) * NB, n2 = n - n1;
  cudaError_t e = trinv_rec(s, n1, U, ldu, dinv, Y, ldy, T);
  if (e != cudaSuccess) return e;
  e = trinv_rec(s, n2, U + n1 + n1 * ldu, ldu, dinv + (n1 / NB) * NB * NB, Y + n1 + n1 * ldy,
                ldy, T);
  if (e != cudaSuccess) return e;
  Epilogue ep{};
  ep.mode = EPI_STORE;  // T = U12 Y22 (n1 x n2, ld n1)
  ep.Y = T;
  ep.ldy = n1;
  e = zgemm_nn(s, n1, n2, n2, U + n1 * ldu, ldu, Y + n1 + n1 * ldy, ldy, ep);
  if (e != cudaSuccess) return e;
  Epilogue e2{};
  e2.mode = EPI_FILTER;  // Y12 = -(Y11 T) (beta = 0: the old Y12 is not read)
  e2.alpha = -1.0;
  e2.beta = 0.0;
  e2.gamma = 0.0;
  e2.X = Y + n1 * ldy;
  e2.ldx = ldy;
  e2.Y = Y + n1 * ldy;
  e2.ldy = ldy;
  return zgemm_nn(s, n1, n2, n1, Y, ldy, T, n1, e2);
}

std::once_flag g_attr_once[kMaxDevices];
void set_attrs() {
  once_per_device(g_attr_once, []() {
    cudaFuncSetAttribute(potf2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * NB * NB * (int)sizeof(double2));
    cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * NB * NB * (int)sizeof(double2));
    cudaFuncSetAttribute(trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (NB * RP + NB * NB + TK * RP + TK * NB) * (int)sizeof(double2));
  });
}

}  // namespace

cudaError_t potrf_upper(cudaStream_t s, int64_t n, double2* G, int64_t ldg, double2* dinv,
                        int* info) {
  set_attrs();
  cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t sm2 = 2 * NB * NB * sizeof(double2);
  for (int64_t k0 = 0, b = 0; k0 < n; k0 += NB, ++b) {
    const int kb = (int)std::min<int64_t>(NB, n - k0);
    potf2_kernel<<<1, FT, sm2, s>>>(G, ldg, k0, kb, dinv + b * NB * NB, info); count_launch();
    const int64_t rest = n - k0 - kb;
    if (rest > 0) {
      panel_kernel<<<(unsigned)cdiv(rest, NB), FT, sm2, s>>>(n, G, ldg, k0, kb, dinv + b * NB * NB,
                                                             info); count_launch();
      const unsigned tt = (unsigned)cdiv(rest, NB);
      trailing_kernel<<<dim3(tt, tt, 1), FT, 0, s>>>(n, G, ldg, k0, kb, info); count_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t trsm_right_upper(cudaStream_t s, int64_t m, int64_t n, double2* X, int64_t ldx,
                             const double2* U, int64_t ldu, const double2* dinv, const int* info) {
  set_attrs();
  if (m <= 0 || n <= 0) return cudaSuccess;
  const size_t smem = (NB * RP + NB * NB + TK * RP + TK * NB) * sizeof(double2);
  trsm_kernel<<<(unsigned)cdiv(m, RP), FT, smem, s>>>(m, n, X, ldx, U, ldu, dinv, info); count_launch();
  return cudaGetLastError();
}

cudaError_t triangular_inverse(cudaStream_t s, int64_t n, const double2* U, int64_t ldu,
                               const double2* dinv, double2* Y, int64_t ldy, double2* T) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemset2DAsync(Y, ldy * sizeof(double2), 0, n * sizeof(double2), n, s);
  if (e != cudaSuccess) return e;
  return trinv_rec(s, n, U, ldu, dinv, Y, ldy, T);
}

cudaError_t max_dev_identity(cudaStream_t s, int64_t n, const double2* U, int64_t ldu,
                             double* out) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  dev_identity_kernel<<<(unsigned)n, 256, 0, s>>>(n, U, ldu, out); count_launch();
  return cudaGetLastError();
}

cudaError_t max_col_ratio(cudaStream_t s, int64_t m, int64_t n, const double2* R, int64_t ldr,
                          const double2* X, int64_t ldx, double* out) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess || m <= 0 || n <= 0) return e;
  col_ratio_kernel<<<(unsigned)n, 256, 0, s>>>(m, R, ldr, X, ldx, out); count_launch();
  return cudaGetLastError();
}

cudaError_t zero_lower(cudaStream_t s, int64_t n, double2* M, int64_t ldm) {
  if (n <= 1) return cudaSuccess;
  zero_lower_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(n, M, ldm);
  count_launch();
  return cudaGetLastError();
}

cudaError_t set_identity(cudaStream_t s, int64_t n, double2* M, int64_t ldm, bool subtract) {
  identity_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(n, M, ldm, subtract);
  count_launch();
  return cudaGetLastError();
}

cudaError_t add_trace_shift(cudaStream_t s, int64_t n, double2* G, int64_t ldg, double factor,
                            double* scratch) {
  trace_shift_kernel<<<1, 256, 0, s>>>(n, G, ldg, factor, scratch); count_launch();
  return cudaGetLastError();
}

}  // namespace chase
