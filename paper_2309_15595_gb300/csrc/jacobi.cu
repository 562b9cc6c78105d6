// Two-sided cyclic Jacobi eigensolver for the small Hermitian Rayleigh-Ritz
// problem (the paper's HEEVD step, Alg. 2) and the Lanczos tridiagonals.
//
// Rotation for a pair (p, q) with a = G_pp, d = G_qq (real), b = G_pq = |b| phi:
//   tau = (d - a) / (2|b|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
//   c = 1/sqrt(1 + t^2), s = t c,
//   J = [[c, s phi], [-s conj(phi), c]]  (identity elsewhere),
// so that J^H G J has a zero (p, q) entry, new G_pp = a - t|b|, G_qq = d + t|b|.
// Pairs follow the round-robin (tournament) order: index 0 stays, the others
// rotate, so each round holds n/2 disjoint pairs that are rotated in parallel
// and n - 1 rounds visit every pair once (one sweep).
#include <algorithm>

#include "common.cuh"

namespace chase {
namespace {

constexpr int kMaxSweeps = 40;

struct Rot {
  double c, s, px, py, app, aqq;  // px + i py = phi
};

__device__ __forceinline__ Rot make_rot(double a, double d, double2 b) {
  Rot r;
  const double ab = sqrt(cabs2(b));
  if (!(ab > 1e-300)) {
    r.c = 1.0; r.s = 0.0; r.px = 1.0; r.py = 0.0; r.app = a; r.aqq = d;
    return r;
  }
  r.px = b.x / ab;
  r.py = b.y / ab;
  const double tau = (d - a) / (2.0 * ab);
  double t;
  if (fabs(tau) > 1e150) {
    t = 0.5 / tau;
  } else {
    t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  }
  r.c = 1.0 / sqrt(1.0 + t * t);
  r.s = t * r.c;
  r.app = a - t * ab;
  r.aqq = d + t * ab;
  return r;
}

// (x_p, x_q) <- (x_p, x_q) J  (column rotation)
__device__ __forceinline__ void rot_cols(double2& xp, double2& xq, const Rot& r) {
  const double2 phi = make_double2(r.px, r.py);
  const double2 np_ = csub(cscale(r.c, xp), cscale(r.s, cmul(xq, conjz(phi))));
  const double2 nq = cadd(cscale(r.s, cmul(xp, phi)), cscale(r.c, xq));
  xp = np_;
  xq = nq;
}
// (y_p; y_q) <- J^H (y_p; y_q)  (row rotation)
__device__ __forceinline__ void rot_rows(double2& yp, double2& yq, const Rot& r) {
  const double2 phi = make_double2(r.px, r.py);
  const double2 np_ = csub(cscale(r.c, yp), cscale(r.s, cmul(phi, yq)));
  const double2 nq = cadd(cscale(r.s, cmul(conjz(phi), yp)), cscale(r.c, yq));
  yp = np_;
  yq = nq;
}

__device__ __forceinline__ void rr_pair(int m, int round, int k, int& p, int& q) {
  auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (m - 1); };
  p = pos(k);
  q = pos(m - 1 - k);
  if (p > q) { const int tmp = p; p = q; q = tmp; }
}

__device__ bool converged_rule(double off, double fro, double off_prev) {
  if (off == 0.0 || off <= 1e-15 * fro) return true;
  return off <= 1e-12 * fro && off > 0.25 * off_prev;
}

// ------------------------------------------------- single-CTA batched version
constexpr int SJ_MAX = 64, SJ_T = 256;

__global__ void __launch_bounds__(SJ_T)
    jacobi_small_kernel(int n, const double2* __restrict__ Gin, double* __restrict__ w,
                        double2* __restrict__ Zout, int* status) {
  extern __shared__ double2 sm[];
  double2* G = sm;                    // n x n, ld SJ_MAX
  double2* Z = sm + SJ_MAX * SJ_MAX;  // n x n
  __shared__ Rot rots[SJ_MAX / 2 + 1];
  __shared__ double red[SJ_T], red2[SJ_T];
  __shared__ int rank_s[SJ_MAX];
  const int t = threadIdx.x;
  const double2* Gb = Gin + (size_t)blockIdx.x * n * n;
  for (int e = t; e < n * n; e += SJ_T) {
    const int r = e % n, c = e / n;
    G[r + c * SJ_MAX] = Gb[e];
    Z[r + c * SJ_MAX] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  const int m = n + (n & 1);
  const int npairs = m / 2;
  double off_prev = 1e300;
  bool conv = false;
  for (int sweep = 0; sweep <= kMaxSweeps; ++sweep) {
    double so = 0.0, sf = 0.0;
    for (int e = t; e < n * n; e += SJ_T) {
      const int r = e % n, c = e / n;
      const double v = cabs2(G[r + c * SJ_MAX]);
      sf += v;
      if (r != c) so += v;
    }
    red[t] = so;
    red2[t] = sf;
    __syncthreads();
    for (int s = SJ_T / 2; s >= 1; s >>= 1) {
      if (t < s) { red[t] += red[t + s]; red2[t] += red2[t + s]; }
      __syncthreads();
    }
    const double off = sqrt(red[0]), fro = sqrt(red2[0]);
    __syncthreads();
    if (converged_rule(off, fro, off_prev)) {
      conv = true;
      break;
    }
    off_prev = off;
    if (sweep == kMaxSweeps) break;
    for (int round = 0; round < m - 1; ++round) {
      if (t < npairs) {
        int p, q;
        rr_pair(m, round, t, p, q);
        if (q < n) {
          rots[t] = make_rot(G[p + p * SJ_MAX].x, G[q + q * SJ_MAX].x, G[p + q * SJ_MAX]);
        } else {
          rots[t] = make_rot(0.0, 0.0, make_double2(0.0, 0.0));
        }
      }
      __syncthreads();
      for (int e = t; e < npairs * n; e += SJ_T) {  // column rotations of G and Z
        const int k = e / n, i = e % n;
        int p, q;
        rr_pair(m, round, k, p, q);
        if (q >= n) continue;
        rot_cols(G[i + p * SJ_MAX], G[i + q * SJ_MAX], rots[k]);
        rot_cols(Z[i + p * SJ_MAX], Z[i + q * SJ_MAX], rots[k]);
      }
      __syncthreads();
      for (int e = t; e < npairs * n; e += SJ_T) {  // row rotations of G
        const int k = e / n, j = e % n;
        int p, q;
        rr_pair(m, round, k, p, q);
        if (q >= n) continue;
        rot_rows(G[p + j * SJ_MAX], G[q + j * SJ_MAX], rots[k]);
      }
      __syncthreads();
      if (t < npairs) {
        int p, q;
        rr_pair(m, round, t, p, q);
        if (q < n && rots[t].s != 0.0) {
          G[p + q * SJ_MAX] = make_double2(0.0, 0.0);
          G[q + p * SJ_MAX] = make_double2(0.0, 0.0);
          G[p + p * SJ_MAX] = make_double2(rots[t].app, 0.0);
          G[q + q * SJ_MAX] = make_double2(rots[t].aqq, 0.0);
        }
      }
      __syncthreads();
    }
  }
  if (t == 0 && !conv) *status = 1;
  // rank sort of the diagonal (ties by index)
  if (t < n) {
    const double v = G[t + t * SJ_MAX].x;
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double u = G[j + j * SJ_MAX].x;
      rk += (u < v) || (u == v && j < t);
    }
    rank_s[t] = rk;
  }
  __syncthreads();
  double* wb = w + (size_t)blockIdx.x * n;
  double2* Zb = Zout + (size_t)blockIdx.x * n * n;
  if (t < n) wb[rank_s[t]] = G[t + t * SJ_MAX].x;
  for (int e = t; e < n * n; e += SJ_T) {
    const int r = e % n, c = e / n;
    Zb[r + rank_s[c] * n] = Z[r + c * SJ_MAX];
  }
}

// ------------------------------------------------------ multi-launch version
constexpr int LJ_T = 256;

__global__ void init_kernel(int64_t n, const double2* G, int64_t ldg, double2* Gw, double2* Zw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n) return;
  Gw[i + j * n] = G[i + j * ldg];
  Zw[i + j * n] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

__global__ void __launch_bounds__(LJ_T)
    col_round_kernel(int64_t n, int m, int round, double2* Gw, double2* Zw, double* params) {
  __shared__ Rot r;
  int p, q;
  rr_pair(m, round, blockIdx.x, p, q);
  if (q >= n) return;
  if (threadIdx.x == 0) {
    r = make_rot(Gw[p + p * n].x, Gw[q + q * n].x, Gw[p + (int64_t)q * n]);
    double* pp = params + 8 * blockIdx.x;
    pp[0] = r.c; pp[1] = r.s; pp[2] = r.px; pp[3] = r.py; pp[4] = r.app; pp[5] = r.aqq;
  }
  __syncthreads();
  if (r.s == 0.0) return;
  double2* gp = Gw + (int64_t)p * n;
  double2* gq = Gw + (int64_t)q * n;
  double2* zp = Zw + (int64_t)p * n;
  double2* zq = Zw + (int64_t)q * n;
  for (int64_t i = threadIdx.x; i < n; i += LJ_T) {
    double2 a = gp[i], b = gq[i];
    rot_cols(a, b, r);
    gp[i] = a;
    gq[i] = b;
    double2 x = zp[i], y = zq[i];
    rot_cols(x, y, r);
    zp[i] = x;
    zq[i] = y;
  }
}

__global__ void __launch_bounds__(LJ_T)
    row_round_kernel(int64_t n, int m, int round, double2* Gw, const double* params) {
  int p, q;
  rr_pair(m, round, blockIdx.x, p, q);
  if (q >= n) return;
  const double* pp = params + 8 * blockIdx.x;
  Rot r;
  r.c = pp[0]; r.s = pp[1]; r.px = pp[2]; r.py = pp[3]; r.app = pp[4]; r.aqq = pp[5];
  if (r.s == 0.0) return;
  for (int64_t j = threadIdx.x; j < n; j += LJ_T) {
    double2 a = Gw[p + j * n], b = Gw[q + j * n];
    rot_rows(a, b, r);
    Gw[p + j * n] = a;
    Gw[q + j * n] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Gw[p + (int64_t)q * n] = make_double2(0.0, 0.0);
    Gw[q + (int64_t)p * n] = make_double2(0.0, 0.0);
    Gw[p + (int64_t)p * n] = make_double2(r.app, 0.0);
    Gw[q + (int64_t)q * n] = make_double2(r.aqq, 0.0);
  }
}

constexpr int RED_BLOCKS = 256;
__global__ void offnorm_partial_kernel(int64_t n, const double2* Gw, double* red) {
  __shared__ double so[256], sf[256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  const int64_t tot = n * n;
  for (int64_t e = (int64_t)blockIdx.x * 256 + t; e < tot; e += (int64_t)RED_BLOCKS * 256) {
    const double v = cabs2(Gw[e]);
    b += v;
    if (e % n != e / n) a += v;
  }
  so[t] = a;
  sf[t] = b;
  __syncthreads();
  for (int s = 128; s >= 1; s >>= 1) {
    if (t < s) { so[t] += so[t + s]; sf[t] += sf[t + s]; }
    __syncthreads();
  }
  if (t == 0) { red[blockIdx.x] = so[0]; red[RED_BLOCKS + blockIdx.x] = sf[0]; }
}
__global__ void offnorm_final_kernel(const double* red, double* out2) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < RED_BLOCKS; ++i) { a += red[i]; b += red[RED_BLOCKS + i]; }
  out2[0] = sqrt(a);
  out2[1] = sqrt(b);
}

__global__ void rank_kernel(int64_t n, const double2* Gw, double* w, int* rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = Gw[i + i * n].x;
  int64_t rk = 0;
  for (int64_t j = 0; j < n; ++j) {
    const double u = Gw[j + j * n].x;
    rk += (u < v) || (u == v && j < i);
  }
  rank[i] = (int)rk;
  w[rk] = v;
}
__global__ void permute_cols_kernel(int64_t n, const double2* Zw, const int* rank, double2* Z,
                                    int64_t ldz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i >= n) return;
  Z[i + (int64_t)rank[c] * ldz] = Zw[i + c * n];
}

bool g_small_attr = false;

}  // namespace

size_t jacobi_params_elems(int64_t n) { return (size_t)8 * (n / 2 + 2) + 2 * RED_BLOCKS + 8 + n; }

cudaError_t jacobi_small_batched(cudaStream_t s, int n, int batch, const double2* G, double* w,
                                 double2* Z, int* status) {
  if (n > SJ_MAX || n < 1) return cudaErrorInvalidValue;
  const size_t smem = 2 * SJ_MAX * SJ_MAX * sizeof(double2);
  if (!g_small_attr) {
    cudaFuncSetAttribute(jacobi_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    g_small_attr = true;
  }
  jacobi_small_kernel<<<batch, SJ_T, smem, s>>>(n, G, w, Z, status); count_launch();
  return cudaGetLastError();
}

int jacobi_heev(cudaStream_t s, int64_t n, const double2* G, int64_t ldg, double* w, double2* Z,
                int64_t ldz, JacobiWork& wk, int* sweeps_out) {
  if (n <= 0) return CHASE_OK;
  cudaError_t e;
  int* status = reinterpret_cast<int*>(wk.red + 2 * RED_BLOCKS + 4);
  if (n <= SJ_MAX) {
    // pack G (ld n) into Gw, run the single-CTA kernel into Zw, copy to Z.
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return CHASE_ERR_CUDA;
    e = cudaMemcpy2DAsync(wk.Gw, n * sizeof(double2), G, ldg * sizeof(double2),
                          n * sizeof(double2), n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return CHASE_ERR_CUDA;
    e = jacobi_small_batched(s, (int)n, 1, wk.Gw, w, wk.Zw, status);
    if (e != cudaSuccess) return CHASE_ERR_CUDA;
    e = cudaMemcpy2DAsync(Z, ldz * sizeof(double2), wk.Zw, n * sizeof(double2),
                          n * sizeof(double2), n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return CHASE_ERR_CUDA;
    int hs = 0;
    e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return CHASE_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CHASE_ERR_CUDA;
    if (sweeps_out) *sweeps_out = -1;
    return hs ? CHASE_ERR_HEEV_NOCONV : CHASE_OK;
  }
  const int m = (int)(n + (n & 1));
  const int npairs = m / 2;
  init_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(n, G, ldg, wk.Gw, wk.Zw); count_launch();
  if (cudaGetLastError() != cudaSuccess) return CHASE_ERR_CUDA;
  double off_prev = 1e300;
  bool conv = false;
  int sweep = 0;
  for (; sweep <= kMaxSweeps; ++sweep) {
    offnorm_partial_kernel<<<RED_BLOCKS, 256, 0, s>>>(n, wk.Gw, wk.red); count_launch();
    offnorm_final_kernel<<<1, 32, 0, s>>>(wk.red, wk.red + 2 * RED_BLOCKS); count_launch();
    e = cudaMemcpyAsync(wk.host_red, wk.red + 2 * RED_BLOCKS, 2 * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CHASE_ERR_CUDA;
    const double off = wk.host_red[0], fro = wk.host_red[1];
    if (off == 0.0 || off <= 1e-15 * fro || (off <= 1e-12 * fro && off > 0.25 * off_prev)) {
      conv = true;
      break;
    }
    off_prev = off;
    if (sweep == kMaxSweeps) break;
    for (int round = 0; round < m - 1; ++round) {
      col_round_kernel<<<npairs, LJ_T, 0, s>>>(n, m, round, wk.Gw, wk.Zw, wk.params); count_launch();
      row_round_kernel<<<npairs, LJ_T, 0, s>>>(n, m, round, wk.Gw, wk.params); count_launch();
    }
    if (cudaGetLastError() != cudaSuccess) return CHASE_ERR_CUDA;
  }
  int* rank = reinterpret_cast<int*>(wk.params + 8 * (n / 2 + 2));
  rank_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(n, wk.Gw, w, rank); count_launch();
  permute_cols_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(n, wk.Zw, rank,
                                                                                    Z, ldz); count_launch();
  if (cudaGetLastError() != cudaSuccess) return CHASE_ERR_CUDA;
  if (sweeps_out) *sweeps_out = sweep;
  return conv ? CHASE_OK : CHASE_ERR_HEEV_NOCONV;
}

}  // namespace chase
