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
#include <cstdio>

#include "common.cuh"

namespace chase {
namespace {

constexpr int kMaxSweeps = 40;
constexpr int kCoopMaxGrid = 2048;  // reduction scratch holds 2 * kCoopMaxGrid partials

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

// Pair k of round `round`, G double-buffered: the owner of pair (p, q) writes
// the new columns p, q of J^H G J into Gnew, reading only the pre-round Gold,
// so owners never race. Its column rotation J_k mixes columns p and q row by
// row; then every pair's row rotation J_k'^H (each thread derives its pairs'
// rotations from Gold itself) mixes rows (p', q') of these two columns. Z is
// updated in place: its columns p, q belong to this owner alone.
__device__ void process_pair(int64_t n, int m, int round, int k, const double2* __restrict__ Gold,
                             double2* __restrict__ Gnew, double2* __restrict__ Zw, double2* colbuf) {
  int p, q;
  rr_pair(m, round, k, p, q);
  // odd n: the pair holding the padding index n has one real column, p, which
  // still receives every other pair's row rotation
  const bool single = q >= n;
  if (single) q = p;
  double2* gp = colbuf;
  double2* gq = colbuf + n;
  const Rot r = single ? make_rot(0.0, 0.0, make_double2(0.0, 0.0))
                       : make_rot(Gold[p + (int64_t)p * n].x, Gold[q + (int64_t)q * n].x,
                                  Gold[p + (int64_t)q * n]);
  const double2* Gp = Gold + (int64_t)p * n;
  const double2* Gq = Gold + (int64_t)q * n;
  double2* Zp = Zw + (int64_t)p * n;
  double2* Zq = Zw + (int64_t)q * n;
  for (int64_t i = threadIdx.x; i < n; i += LJ_T) {
    double2 a = Gp[i], b = Gq[i];
    rot_cols(a, b, r);
    gp[i] = a;
    gq[i] = b;
    if (r.s != 0.0) {
      double2 x = Zp[i], y = Zq[i];
      rot_cols(x, y, r);
      Zp[i] = x;
      Zq[i] = y;
    }
  }
  __syncthreads();
  for (int kk = threadIdx.x; kk < m / 2; kk += LJ_T) {
    int pr, qr;
    rr_pair(m, round, kk, pr, qr);
    if (qr >= n) continue;
    const Rot rk = make_rot(Gold[pr + (int64_t)pr * n].x, Gold[qr + (int64_t)qr * n].x,
                            Gold[pr + (int64_t)qr * n]);
    if (rk.s == 0.0) continue;
    rot_rows(gp[pr], gp[qr], rk);
    rot_rows(gq[pr], gq[qr], rk);
  }
  __syncthreads();
  if (threadIdx.x == 0 && r.s != 0.0) {  // exact 2 x 2 block of this pair
    gp[p] = make_double2(r.app, 0.0);
    gq[q] = make_double2(r.aqq, 0.0);
    gp[q] = make_double2(0.0, 0.0);
    gq[p] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  double2* Np_ = Gnew + (int64_t)p * n;
  double2* Nq_ = Gnew + (int64_t)q * n;
  for (int64_t i = threadIdx.x; i < n; i += LJ_T) {
    Np_[i] = gp[i];
    if (!single) Nq_[i] = gq[i];
  }
  __syncthreads();  // colbuf is reused by this block's next pair
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (all blocks are co-resident). The
// wait is bounded: after 2 s it records status[0] = 1 and returns false.
__device__ bool grid_sync(unsigned* bar, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok_s = 1;
    volatile unsigned* vgen = bar + 1;
    __threadfence();
    const unsigned gen = *vgen;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = gtimer();
      while (*vgen == gen) {
        if (*(volatile int*)status != 0) {  // another block gave up: leave at once
          ok_s = 0;
          break;
        }
        if (gtimer() - t0 > 2000000000ull) {
          atomicExch(status, 1);
          ok_s = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (*(volatile int*)status != 0) ok_s = 0;
  }
  __syncthreads();
  return ok_s != 0;
}

struct CoopArgs {
  int64_t n;
  int m, max_sweeps;
  double2* G0;
  double2* G1;
  double2* Z;
  double* red;      // 2 * gridDim.x partial sums
  unsigned* bar;    // barrier counter and generation
  int* status;      // [0] error, [1] sweeps, [2] converged, [3] result in G1
};

// The whole cyclic Jacobi in one cooperative launch: per sweep a fixed-order
// off-norm test (identical in every block, so the decision is uniform), then
// the m - 1 rounds, each followed by a grid barrier.
__global__ void __launch_bounds__(LJ_T) jacobi_coop_kernel(CoopArgs a) {
  extern __shared__ double2 colbuf[];
  __shared__ double so[LJ_T], sf[LJ_T];
  __shared__ int decide;
  const int64_t n = a.n;
  const int npairs = a.m / 2;
  double2* Gcur = a.G0;
  double2* Gnxt = a.G1;
  double off_prev = 1e300;
  int sweep = 0;
  bool conv = false, alive = true;
  for (; sweep <= a.max_sweeps && alive; ++sweep) {
    // off-norm and Frobenius norm of Gcur: block partials, then every block
    // sums all partials in the same order
    double o = 0.0, f = 0.0;
    const int64_t tot = n * n;
    for (int64_t e = (int64_t)blockIdx.x * LJ_T + threadIdx.x; e < tot; e += (int64_t)gridDim.x * LJ_T) {
      const double v = cabs2(Gcur[e]);
      f += v;
      if (e % n != e / n) o += v;
    }
    so[threadIdx.x] = o;
    sf[threadIdx.x] = f;
    __syncthreads();
    for (int w = LJ_T / 2; w >= 1; w >>= 1) {
      if (threadIdx.x < w) {
        so[threadIdx.x] += so[threadIdx.x + w];
        sf[threadIdx.x] += sf[threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      a.red[blockIdx.x] = so[0];
      a.red[gridDim.x + blockIdx.x] = sf[0];
    }
    if (!grid_sync(a.bar, a.status)) { alive = false; break; }
    if (threadIdx.x == 0) {
      double to = 0.0, tf = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) {
        to += a.red[b];
        tf += a.red[gridDim.x + b];
      }
      const double off = sqrt(to), fro = sqrt(tf);
      int d = 0;
      if (off == 0.0 || off <= 1e-15 * fro || (off <= 1e-12 * fro && off > 0.25 * off_prev)) d = 1;
      else if (sweep == a.max_sweeps) d = 2;
      off_prev = off;
      decide = d;
    }
    __syncthreads();
    // every block has read the partials before any block rewrites them
    if (!grid_sync(a.bar, a.status)) { alive = false; break; }
    if (decide == 1) { conv = true; break; }
    if (decide == 2) break;
    for (int round = 0; round < a.m - 1; ++round) {
      for (int k = blockIdx.x; k < npairs; k += gridDim.x)
        process_pair(n, a.m, round, k, Gcur, Gnxt, a.Z, colbuf);
      if (!grid_sync(a.bar, a.status)) { alive = false; break; }
      double2* t = Gcur;
      Gcur = Gnxt;
      Gnxt = t;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status[1] = sweep;
    a.status[2] = conv ? 1 : 0;
    a.status[3] = Gcur == a.G1 ? 1 : 0;
  }
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

size_t jacobi_red_elems() { return (size_t)2 * kCoopMaxGrid + 16; }

size_t jacobi_params_elems(int64_t n) { return (size_t)8 * (n / 2 + 2) + 8 + n; }

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
  int* status = reinterpret_cast<int*>(wk.red + 2 * kCoopMaxGrid + 8);
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
    if (sweeps_out) *sweeps_out = 0;
    return hs ? CHASE_ERR_HEEV_NOCONV : CHASE_OK;
  }
  const int m = (int)(n + (n & 1));
  const int npairs = m / 2;
  const size_t smem = (size_t)2 * n * sizeof(double2);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(jacobi_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return CHASE_ERR_CUDA;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel, LJ_T, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return CHASE_ERR_CUDA;
  const int grid = std::min(std::min(npairs, per_sm * nsm), kCoopMaxGrid);
  double2* Gcur = wk.Gw;
  init_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(n, G, ldg, Gcur, wk.Zw); count_launch();
  // barrier words and status live in the reduction scratch after the partials
  unsigned* bar = reinterpret_cast<unsigned*>(wk.red + 2 * kCoopMaxGrid);
  int* st = reinterpret_cast<int*>(wk.red + 2 * kCoopMaxGrid + 2);
  if (cudaMemsetAsync(wk.red + 2 * kCoopMaxGrid, 0, 8 * sizeof(double), s) != cudaSuccess)
    return CHASE_ERR_CUDA;
  CoopArgs args;
  args.n = n;
  args.m = m;
  args.max_sweeps = kMaxSweeps;
  args.G0 = wk.Gw;
  args.G1 = wk.Gw2;
  args.Z = wk.Zw;
  args.red = wk.red;
  args.bar = bar;
  args.status = st;
  void* kargs[] = {&args};
  if (cudaLaunchCooperativeKernel((const void*)jacobi_coop_kernel, dim3(grid), dim3(LJ_T), kargs,
                                  smem, s) != cudaSuccess)
    return CHASE_ERR_CUDA;
  count_launch();
  int hst[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CHASE_ERR_CUDA;
  if (hst[0] != 0) {
    fprintf(stderr, "[chase] Jacobi: grid barrier wait expired\n");
    return CHASE_ERR_CUDA;
  }
  if (hst[3]) Gcur = wk.Gw2;
  const int sweep = hst[1];
  const bool conv = hst[2] != 0;
  int* rank = reinterpret_cast<int*>(wk.params + 8 * (n / 2 + 2));
  rank_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(n, Gcur, w, rank); count_launch();
  permute_cols_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(n, wk.Zw, rank,
                                                                                    Z, ldz); count_launch();
  if (cudaGetLastError() != cudaSuccess) return CHASE_ERR_CUDA;
  if (sweeps_out) *sweeps_out = sweep;
  return conv ? CHASE_OK : CHASE_ERR_HEEV_NOCONV;
}

}  // namespace chase
