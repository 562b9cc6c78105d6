// Householder QR of a tall block on the device: the fallback of Alg. 4 when
// the shifted CholeskyQR cannot finish (its POTRF, or a POTRF of the
// CholeskyQR2 that follows it, reports a non-positive pivot).
//
// Blocked right-looking factorisation with panels of NBH = 64 columns. Within a
// panel, column c gets the reflector H_c = I - tau_c v_c v_c^H (v_c(c) = 1) with
// H_c^H x = beta_c e_c, beta_c = -sign(Re x_c) ||x||, tau_c = (beta_c - x_c) /
// beta_c, v_c = x / (x_c - beta_c) below the diagonal (the standard complex
// Householder vector), and H_c^H is applied to the rest of the panel. The
// panel's reflectors are then gathered into one block reflector
// H = H_1 ... H_k = I - V T V^H (T upper triangular: T_jj = tau_j,
// T(0:j, j) = -tau_j T(0:j, 0:j) V(:, 0:j)^H v_j), and H^H is applied to the
// trailing columns with two FP64 GEMMs (W = V^H C, C -= V (T^H W)). Q is formed
// afterwards by applying the block reflectors to [I; 0] in reverse panel order
// (Q = H_1 H_2 ... [I; 0]); finally column j of Q is multiplied by sign(beta_j)
// so that R = Q^H X has a positive real diagonal, which makes Q the unique QR
// factor the CholeskyQR variants produce.
//
// Every reduction has a fixed order (per-block partial sums, then a fixed-order
// sum of the partials), so results are reproducible run to run.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "householder.cuh"

namespace chase {
namespace {

constexpr int NBH = kHouseholderNB;  // 64 columns per panel
constexpr int HT = 256;              // threads of the row kernels
constexpr int kMaxRowBlocks = 256;   // partial sums per reduction

__host__ __device__ inline int row_blocks(int64_t rows) {
  const int64_t b = (rows + 2 * HT - 1) / (2 * HT);
  return (int)(b < 1 ? 1 : (b > kMaxRowBlocks ? kMaxRowBlocks : b));
}

// Sum of |x_i|^2 over rows c+1 .. m-1 of column c: one partial per block.
__global__ void __launch_bounds__(HT)
    hh_norm_kernel(int64_t m, const double2* __restrict__ X, int64_t ldx, int64_t c,
                   double* __restrict__ part) {
  __shared__ double red[HT];
  const double2* x = X + c * ldx;
  double s = 0.0;
  for (int64_t i = c + 1 + (int64_t)blockIdx.x * HT + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * HT)
    s += cabs2(x[i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = HT / 2; w >= 1; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Reflector of column c from alpha = X(c, c) and the partial sums: writes
// beta (real, the R diagonal), tau and the scale 1 / (alpha - beta) of the
// vector; X(c, c) becomes beta. A column that is already e_c-shaped (x below
// the diagonal zero, alpha real) gets tau = 0 (H = I).
__global__ void hh_reflector_kernel(double2* __restrict__ X, int64_t ldx, int64_t c, int nb,
                                    const double* __restrict__ part, double* __restrict__ beta,
                                    double2* __restrict__ tau, double2* __restrict__ scale,
                                    int* __restrict__ bad) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  const double2 a = X[c + c * ldx];
  if (s == 0.0 && a.y == 0.0) {
    beta[c] = a.x;
    tau[c] = make_double2(0.0, 0.0);
    scale[0] = make_double2(0.0, 0.0);
    return;
  }
  const double nrm = sqrt(a.x * a.x + a.y * a.y + s);
  const double b = a.x >= 0.0 ? -nrm : nrm;
  if (!isfinite(b)) *bad = 1;
  beta[c] = b;
  tau[c] = make_double2((b - a.x) / b, -a.y / b);
  const double2 d = make_double2(a.x - b, a.y);  // |d| >= |b| > 0
  const double dd = d.x * d.x + d.y * d.y;
  scale[0] = make_double2(d.x / dd, -d.y / dd);
  X[c + c * ldx] = make_double2(b, 0.0);
}

// w_l = v^H X(:, l) for the panel columns l = c+1 .. cend-1 (at most NBH - 1),
// v(c) = 1, v(i) = scale X(i, c) below: one partial per block and column.
// Threads walk rows (coalesced column reads); columns go in chunks of 16
// register accumulators.
constexpr int DCH = 16;
__global__ void __launch_bounds__(HT)
    hh_dots_kernel(int64_t m, const double2* __restrict__ X, int64_t ldx, int64_t c, int ncols,
                   const double2* __restrict__ scale, double2* __restrict__ part) {
  __shared__ double2 red[HT / 32][NBH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2 sc = scale[0];
  for (int l0 = 0; l0 < ncols; l0 += DCH) {
    double2 acc[DCH];
#pragma unroll
    for (int l = 0; l < DCH; ++l) acc[l] = make_double2(0.0, 0.0);
    const int nl = min(DCH, ncols - l0);
    for (int64_t i = c + (int64_t)blockIdx.x * HT + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * HT) {
      const double2 v = i == c ? make_double2(1.0, 0.0) : cmul(sc, X[i + c * ldx]);
      const double2 vc = conjz(v);
      const double2* xr = X + i + (c + 1 + l0) * ldx;
#pragma unroll
      for (int l = 0; l < DCH; ++l)
        if (l < nl) acc[l] = cadd(acc[l], cmul(vc, xr[l * ldx]));
    }
#pragma unroll
    for (int l = 0; l < DCH; ++l) {
      double2 v = acc[l];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
      }
      if (lane == 0 && l < nl) red[warp][l0 + l] = v;
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < ncols; l += HT) {
    double2 v = make_double2(0.0, 0.0);
    for (int w = 0; w < HT / 32; ++w) v = cadd(v, red[w][l]);
    part[(int64_t)blockIdx.x * NBH + l] = v;
  }
}

// X(:, l) -= conj(tau) v w_l for the panel columns right of c, and the
// reflector stored below the diagonal of column c (v, without its unit head).
__global__ void __launch_bounds__(HT)
    hh_update_kernel(int64_t m, double2* __restrict__ X, int64_t ldx, int64_t c, int ncols,
                     const double2* __restrict__ tau, const double2* __restrict__ scale,
                     const double2* __restrict__ part, int nb) {
  __shared__ double2 w[NBH];
  const double2 tc = conjz(tau[c]);
  for (int l = threadIdx.x; l < ncols; l += HT) {
    double2 v = make_double2(0.0, 0.0);
    for (int b = 0; b < nb; ++b) v = cadd(v, part[(int64_t)b * NBH + l]);
    w[l] = cmul(tc, v);
  }
  __syncthreads();
  const double2 sc = scale[0];
  for (int64_t i = c + (int64_t)blockIdx.x * HT + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * HT) {
    double2 v = make_double2(1.0, 0.0);
    if (i > c) {
      v = cmul(sc, X[i + c * ldx]);
      X[i + c * ldx] = v;
    }
    for (int l = 0; l < ncols; ++l) {
      double2& x = X[i + (c + 1 + l) * ldx];
      x = csub(x, cmul(v, w[l]));
    }
  }
}

// Explicit panel reflectors: Vp(r, j) = 0 above the diagonal, 1 on it, the
// stored vector below (r = i - k0), for rows k0 .. m-1.
__global__ void hh_build_vp_kernel(int64_t m, const double2* __restrict__ X, int64_t ldx,
                                   int64_t k0, int kb, double2* __restrict__ Vp, int64_t ldv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k0 + r >= m) return;
  double2 v;
  if (j >= kb || r < j) v = make_double2(0.0, 0.0);
  else if (r == j) v = make_double2(1.0, 0.0);
  else v = X[(k0 + r) + (k0 + j) * ldx];
  Vp[r + (int64_t)j * ldv] = v;
}

// T of the block reflector from S = V^H V (kb x kb, ld NBH) and tau, one CTA of
// NBH threads, T (NBH x NBH, ld NBH) built in place in global memory:
// T_jj = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) S(0:j, j).
__global__ void hh_larft_kernel(int kb, const double2* __restrict__ S,
                                const double2* __restrict__ tau, double2* T) {
  __shared__ double2 z[NBH];
  const int t = threadIdx.x;
  for (int j = 0; j < NBH; ++j) T[t + j * NBH] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (t < j) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = t; k < j; ++k) acc = cadd(acc, cmul(T[t + k * NBH], S[k + j * NBH]));
      z[t] = acc;
    }
    __syncthreads();
    const double2 tj = tau[j];
    if (t < j) T[t + j * NBH] = cscale(-1.0, cmul(tj, z[t]));
    if (t == j) T[j + j * NBH] = tj;
    __syncthreads();
  }
}

// W2 = op(T) W for W of kb x n (ld NBH): op = T^H (adjoint) or T.
__global__ void hh_tmul_kernel(int kb, int64_t n, const double2* __restrict__ T, bool adjoint,
                               const double2* __restrict__ W, double2* __restrict__ W2) {
  const int r = threadIdx.x;  // NBH
  const int64_t col = blockIdx.x;
  if (col >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  if (r < kb) {
    if (adjoint) {  // (T^H)(r, k) = conj(T(k, r)), nonzero for k <= r
      for (int k = 0; k <= r; ++k) acc = cadd(acc, cmulc(T[k + r * NBH], W[k + col * NBH]));
    } else {        // T(r, k), nonzero for k >= r
      for (int k = r; k < kb; ++k) acc = cadd(acc, cmul(T[r + k * NBH], W[k + col * NBH]));
    }
  }
  W2[r + col * NBH] = acc;
}

__global__ void hh_identity_kernel(int64_t m, int64_t n, double2* __restrict__ Q, int64_t ldq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < m) Q[i + j * ldq] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// Q(:, j) *= sign(beta_j), so that diag(R) = |beta| > 0.
__global__ void hh_signs_kernel(int64_t m, const double* __restrict__ beta, double2* __restrict__ Q,
                                int64_t ldq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < m && beta[j] < 0.0) {
    double2& q = Q[i + j * ldq];
    q = make_double2(-q.x, -q.y);
  }
}

}  // namespace

cudaError_t householder_alloc(HouseholderWork& w, int64_t N, int64_t ne) {
  const int64_t npan = cdiv(ne, NBH);
  cudaError_t e;
  if ((e = cudaMalloc(&w.Vp, (size_t)N * NBH * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.T, (size_t)npan * NBH * NBH * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.S, (size_t)NBH * NBH * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.W, (size_t)NBH * ne * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.W2, (size_t)NBH * ne * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.dots, (size_t)kMaxRowBlocks * NBH * sizeof(double2))) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&w.norms, (size_t)kMaxRowBlocks * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.beta, (size_t)ne * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.tau, (size_t)ne * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.scale, 2 * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.bad, sizeof(int))) != cudaSuccess) return e;
  // the Gram products here have NB rows and up to max(NB, ne) columns
  w.gws_elems = gram_workspace_elems(NBH, std::max<int64_t>(NBH, ne));
  if ((e = cudaMalloc(&w.gws, w.gws_elems * sizeof(double2))) != cudaSuccess) return e;
  w.N = N;
  w.ne = ne;
  return cudaSuccess;
}

void householder_free(HouseholderWork& w) {
  void* bufs[] = {w.Vp, w.T, w.S, w.W, w.W2, w.dots, w.norms, w.beta, w.tau, w.scale, w.bad,
                  w.gws};
  for (void* b : bufs)
    if (b) cudaFree(b);
  w = HouseholderWork{};
}

int householder_qr(cudaStream_t s, int64_t m, int64_t n, double2* X, int64_t ldx, double2* Q,
                   int64_t ldq, HouseholderWork& w) {
  double2* const gram_ws = w.gws;
  const size_t gram_ws_elems = w.gws_elems;
  if (n <= 0) return CHASE_OK;
  if (m < n || m > w.N || n > w.ne) return CHASE_ERR_INVALID_ARG;
#define HK(call)                                          \
  do {                                                    \
    if ((call) != cudaSuccess) return CHASE_CUDA_FAIL();  \
  } while (0)
  HK(cudaMemsetAsync(w.bad, 0, sizeof(int), s));
  const int64_t npan = cdiv(n, NBH);
  // ------------------------------------------------------------ factorisation
  for (int64_t p = 0; p < npan; ++p) {
    const int64_t k0 = p * NBH;
    const int kb = (int)std::min<int64_t>(NBH, n - k0);
    const int64_t kend = k0 + kb;
    for (int64_t c = k0; c < kend; ++c) {
      const int nbn = row_blocks(m - c - 1);
      hh_norm_kernel<<<nbn, HT, 0, s>>>(m, X, ldx, c, w.norms);
      count_launch();
      hh_reflector_kernel<<<1, 32, 0, s>>>(X, ldx, c, nbn, w.norms, w.beta, w.tau, w.scale, w.bad);
      count_launch();
      const int ncols = (int)(kend - c - 1);
      const int nb = row_blocks(m - c);
      if (ncols > 0) {
        hh_dots_kernel<<<nb, HT, 0, s>>>(m, X, ldx, c, ncols, w.scale, w.dots);
        count_launch();
      }
      hh_update_kernel<<<nb, HT, 0, s>>>(m, X, ldx, c, ncols, w.tau, w.scale, w.dots, nb);
      count_launch();
    }
    // block reflector of the panel: explicit V, S = V^H V, T
    const int64_t rows = m - k0;
    hh_build_vp_kernel<<<dim3((unsigned)cdiv(rows, 256), NBH, 1), 256, 0, s>>>(m, X, ldx, k0, kb,
                                                                             w.Vp, m);
    count_launch();
    HK(zgram(s, rows, NBH, NBH, w.Vp, m, w.Vp, m, w.S, NBH, true, gram_ws, gram_ws_elems));
    double2* Tp = w.T + p * NBH * NBH;
    hh_larft_kernel<<<1, NBH, 0, s>>>(kb, w.S, w.tau + k0, Tp);
    count_launch();
    // trailing columns: C <- H^H C = C - V (T^H (V^H C))
    const int64_t nt = n - kend;
    if (nt > 0) {
      double2* C = X + k0 + kend * ldx;
      HK(zgram(s, rows, NBH, nt, w.Vp, m, C, ldx, w.W, NBH, false, gram_ws, gram_ws_elems));
      hh_tmul_kernel<<<(unsigned)nt, NBH, 0, s>>>(kb, nt, Tp, true, w.W, w.W2);
      count_launch();
      Epilogue ep{};
      ep.mode = EPI_FILTER;  // C = -(V W2) + C
      ep.alpha = -1.0;
      ep.beta = 1.0;
      ep.gamma = 0.0;
      ep.X = C;
      ep.ldx = ldx;
      ep.Y = C;
      ep.ldy = ldx;
      HK(zgemm_nn(s, rows, nt, NBH, w.Vp, m, w.W2, NBH, ep));
    }
  }
  // ------------------------------------------------ Q = H_1 ... H_p [I; 0]
  hh_identity_kernel<<<dim3((unsigned)cdiv(m, 256), (unsigned)n, 1), 256, 0, s>>>(m, n, Q, ldq);
  count_launch();
  for (int64_t p = npan - 1; p >= 0; --p) {
    const int64_t k0 = p * NBH;
    const int kb = (int)std::min<int64_t>(NBH, n - k0);
    const int64_t rows = m - k0, nq = n - k0;
    hh_build_vp_kernel<<<dim3((unsigned)cdiv(rows, 256), NBH, 1), 256, 0, s>>>(m, X, ldx, k0, kb,
                                                                             w.Vp, m);
    count_launch();
    double2* Qs = Q + k0 + k0 * ldq;
    HK(zgram(s, rows, NBH, nq, w.Vp, m, Qs, ldq, w.W, NBH, false, gram_ws, gram_ws_elems));
    hh_tmul_kernel<<<(unsigned)nq, NBH, 0, s>>>(kb, nq, w.T + p * NBH * NBH, false, w.W, w.W2);
    count_launch();
    Epilogue ep{};
    ep.mode = EPI_FILTER;  // Qs = -(V W2) + Qs
    ep.alpha = -1.0;
    ep.beta = 1.0;
    ep.gamma = 0.0;
    ep.X = Qs;
    ep.ldx = ldq;
    ep.Y = Qs;
    ep.ldy = ldq;
    HK(zgemm_nn(s, rows, nq, NBH, w.Vp, m, w.W2, NBH, ep));
  }
  hh_signs_kernel<<<dim3((unsigned)cdiv(m, 256), (unsigned)n, 1), 256, 0, s>>>(m, w.beta, Q, ldq);
  count_launch();
  HK(cudaGetLastError());
  int bad = 0;
  HK(cudaMemcpyAsync(&bad, w.bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  HK(cudaStreamSynchronize(s));
#undef HK
  if (bad) fprintf(stderr, "[chase] Householder QR: the block holds non-finite values\n");
  return bad ? CHASE_ERR_QR_BREAKDOWN : CHASE_OK;
}

}  // namespace chase
