// Column copies/gathers and the Lanczos spectral-bound estimate (Alg. 1 and
// Alg. 2 first line). Reductions are two-pass with a fixed order, so repeated
// runs give bit-identical results.
#include <algorithm>

#include "common.cuh"

namespace chase {
namespace {

constexpr int VT = 256;
constexpr int RB = 128;  // reduction blocks per vector

__global__ void copy_cols_kernel(int64_t m, const double2* src, int64_t lds, double2* dst,
                                 int64_t ldd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < m) dst[i + j * ldd] = src[i + j * lds];
}

__global__ void gather_cols_kernel(int64_t m, const double2* src, int64_t lds, const int* perm,
                                   double2* dst, int64_t ldd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < m) dst[i + j * ldd] = src[i + (int64_t)perm[j] * lds];
}

// partial[b + r * RB] = sum over this block's rows of f(r, i)
// mode 0: |Q0_i|^2            (start-vector norms)
// mode 1: W_i -= beta_prev Qp_i; partial Re(conj(Q_i) W_i)
// mode 2: W_i -= alpha Q_i;  partial |W_i|^2
__global__ void lz_partial_kernel(int mode, int64_t N, int nvec, const double2* Q0, int64_t ldq,
                                  const double2* Q, const double2* Qp, double2* W, const double* ab,
                                  int step, int kmax, double* partial) {
  __shared__ double red[VT];
  const int r = blockIdx.y;
  const int t = threadIdx.x;
  double s = 0.0;
  const double* alpha = ab;               // [r * kmax + step]
  const double* beta = ab + 8 * kmax;     // [r * kmax + step]
  double bprev = 0.0, al = 0.0;
  if (mode == 1 && step > 0) bprev = beta[r * kmax + step - 1];
  if (mode == 2) al = alpha[r * kmax + step];
  for (int64_t i = (int64_t)blockIdx.x * VT + t; i < N; i += (int64_t)RB * VT) {
    if (mode == 0) {
      s += cabs2(Q0[i + r * ldq]);
    } else if (mode == 1) {
      double2 w = W[i + r * N];
      if (step > 0) {
        const double2 qp = Qp[i + r * N];
        w.x = fma(-bprev, qp.x, w.x);
        w.y = fma(-bprev, qp.y, w.y);
        W[i + r * N] = w;
      }
      const double2 q = Q[i + r * N];
      s += q.x * w.x + q.y * w.y;
    } else {
      const double2 q = Q[i + r * N];
      double2 w = W[i + r * N];
      w.x = fma(-al, q.x, w.x);
      w.y = fma(-al, q.y, w.y);
      W[i + r * N] = w;
      s += cabs2(w);
    }
  }
  red[t] = s;
  __syncthreads();
  for (int w = VT / 2; w >= 1; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  if (t == 0) partial[blockIdx.x + r * RB] = red[0];
}

// dst[r * kmax + step] = (sqrt?)(sum_b partial[b + r RB])
__global__ void lz_final_kernel(int nvec, const double* partial, double* dst, int kmax, int step,
                                int take_sqrt) {
  const int r = threadIdx.x;
  if (r >= nvec) return;
  double s = 0.0;
  for (int b = 0; b < RB; ++b) s += partial[b + r * RB];
  dst[r * kmax + step] = take_sqrt ? sqrt(s) : s;
}

// out[:, r] = in[:, r] * (1 / scale[r * kmax + step])
__global__ void lz_scale_kernel(int64_t N, int nvec, const double2* in, int64_t ldi, double2* out,
                                const double* scale, int kmax, int step) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= N) return;
  const double inv = 1.0 / scale[r * kmax + step];
  out[i + r * N] = cscale(inv, in[i + r * ldi]);
}

__global__ void lz_zero_kernel(int64_t n, double2* x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = make_double2(0.0, 0.0);
}

// T_r = tridiag(alpha, beta) as a complex k x k matrix, column-major.
__global__ void lz_build_t_kernel(int nvec, int k, int kmax, const double* ab, double2* T) {
  const int r = blockIdx.x;
  const double* alpha = ab + r * kmax;
  const double* beta = ab + 8 * kmax + r * kmax;
  double2* Tr = T + (size_t)r * k * k;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    double v = 0.0;
    if (i == j) v = alpha[i];
    else if (i == j + 1) v = beta[j];
    else if (j == i + 1) v = beta[i];
    Tr[e] = make_double2(v, 0.0);
  }
}

// b_sup, mu_1, mu_ne, norm_est from the Ritz values and Gauss weights.
__global__ void lz_bounds_kernel(int nvec, int k, int kmax, const double* ab, const double* theta,
                                 const double2* Z, double target, double* out4) {
  __shared__ double th[8 * 64], wt[8 * 64];
  __shared__ int ord[8 * 64];
  const int tot = nvec * k;
  const int t = threadIdx.x;
  for (int e = t; e < tot; e += blockDim.x) {
    const int r = e / k, i = e % k;
    th[e] = theta[r * k + i];
    const double2 z = Z[(size_t)r * k * k + 0 + (size_t)i * k];  // first component of vector i
    wt[e] = cabs2(z) / nvec;
  }
  __syncthreads();
  for (int e = t; e < tot; e += blockDim.x) {
    int rk = 0;
    for (int j = 0; j < tot; ++j) rk += (th[j] < th[e]) || (th[j] == th[e] && j < e);
    ord[rk] = e;
  }
  __syncthreads();
  if (t != 0) return;
  const double* beta = ab + 8 * kmax;
  double b_sup = -1e300, mu1 = 1e300, nrm = 0.0;
  for (int r = 0; r < nvec; ++r) {
    const double tmin = theta[r * k], tmax = theta[r * k + k - 1];
    b_sup = fmax(b_sup, tmax + fabs(beta[r * kmax + k - 1]));
    mu1 = fmin(mu1, tmin);
    nrm = fmax(nrm, fmax(fabs(tmin), fabs(tmax)));
  }
  double cum = 0.0, mune = th[ord[tot - 1]];
  for (int j = 0; j < tot; ++j) {
    cum += wt[ord[j]];
    if (cum >= target) {
      mune = th[ord[j]];
      break;
    }
  }
  mune = fmin(fmax(mune, mu1), b_sup);
  out4[0] = b_sup;
  out4[1] = mu1;
  out4[2] = mune;
  out4[3] = nrm;
}

}  // namespace

cudaError_t copy_cols(cudaStream_t s, int64_t m, int64_t n, const double2* src, int64_t lds,
                      double2* dst, int64_t ldd) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  copy_cols_kernel<<<dim3((unsigned)cdiv(m, 256), (unsigned)n, 1), 256, 0, s>>>(m, src, lds, dst,
                                                                                 ldd); count_launch();
  return cudaGetLastError();
}

cudaError_t gather_cols(cudaStream_t s, int64_t m, int64_t n, const double2* src, int64_t lds,
                        const int* perm, double2* dst, int64_t ldd) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  gather_cols_kernel<<<dim3((unsigned)cdiv(m, 256), (unsigned)n, 1), 256, 0, s>>>(m, src, lds,
                                                                                   perm, dst, ldd); count_launch();
  return cudaGetLastError();
}

cudaError_t lanczos_bounds(cudaStream_t s, int64_t N, const double2* A, int64_t lda,
                           const double2* Q0, int64_t ldq, int nvec, int k, int64_t ne,
                           LanczosWork& w) {
  const int kmax = 64;
  if (nvec < 1 || nvec > 8 || k < 1 || k > kmax) return cudaErrorInvalidValue;
  double2* Qp = w.Q;
  double2* Q = w.Q + (size_t)N * 8;
  double2* W = w.Q + (size_t)2 * N * 8;
  double* norms = w.ab + 16 * kmax;  // scratch row for start norms: [r * kmax + 0]
  const dim3 gp(RB, (unsigned)nvec, 1);
  const dim3 ge((unsigned)cdiv(N, 256), (unsigned)nvec, 1);
  // q = q0 / ||q0||
  lz_partial_kernel<<<gp, VT, 0, s>>>(0, N, nvec, Q0, ldq, nullptr, nullptr, nullptr, w.ab, 0,
                                      kmax, w.red); count_launch();
  lz_final_kernel<<<1, 32, 0, s>>>(nvec, w.red, norms, kmax, 0, 1); count_launch();
  lz_scale_kernel<<<ge, 256, 0, s>>>(N, nvec, Q0, ldq, Q, norms, kmax, 0); count_launch();
  lz_zero_kernel<<<(unsigned)cdiv(N * 8, 256), 256, 0, s>>>(N * 8, Qp); count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int j = 0; j < k; ++j) {
    e = w.matmul ? w.matmul(w.matmul_ctx, Q, N, nvec, W, N)   // W = A q
                 : zgemm_skinny(s, N, nvec, A, lda, Q, N, W, N, w.ws);
    if (e != cudaSuccess) return e;
    // W -= beta_{j-1} q_prev ; alpha_j = Re(q^H W)
    lz_partial_kernel<<<gp, VT, 0, s>>>(1, N, nvec, nullptr, 0, Q, Qp, W, w.ab, j, kmax, w.red); count_launch();
    lz_final_kernel<<<1, 32, 0, s>>>(nvec, w.red, w.ab, kmax, j, 0); count_launch();
    // W -= alpha_j q ; beta_j = ||W||
    lz_partial_kernel<<<gp, VT, 0, s>>>(2, N, nvec, nullptr, 0, Q, Qp, W, w.ab, j, kmax, w.red); count_launch();
    lz_final_kernel<<<1, 32, 0, s>>>(nvec, w.red, w.ab + 8 * kmax, kmax, j, 1); count_launch();
    if (j + 1 < k) {
      // q_prev <- q ; q <- W / beta_j  (the old q_prev buffer receives the new q)
      lz_scale_kernel<<<ge, 256, 0, s>>>(N, nvec, W, N, Qp, w.ab + 8 * kmax, kmax, j); count_launch();
      std::swap(Qp, Q);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  lz_build_t_kernel<<<nvec, 256, 0, s>>>(nvec, k, kmax, w.ab, w.T); count_launch();
  e = jacobi_small_batched(s, k, nvec, w.T, w.theta, w.Z, w.status);
  if (e != cudaSuccess) return e;
  lz_bounds_kernel<<<1, 256, 0, s>>>(nvec, k, kmax, w.ab, w.theta, w.Z, (double)ne / (double)N,
                                     w.out4); count_launch();
  return cudaGetLastError();
}

}  // namespace chase
