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
#include <vector>

#include "common.cuh"

namespace chase {
namespace {

#define RC_(call)                   \
  do {                              \
    const int _rc = (call);         \
    if (_rc != CHASE_OK) return _rc; \
  } while (0)
#define RC_NEG(call)                  \
  do {                                \
    const int _rc = (call);           \
    if (_rc != CHASE_OK) return -_rc; \
  } while (0)

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
                        double2* __restrict__ Zout, int* status, int max_sweeps) {
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
    // Hermitian part of the input (inputs formed as X^H (G X) are Hermitian
    // only up to rounding)
    const double2 a = Gb[e], b = Gb[c + r * n];
    G[r + c * SJ_MAX] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    Z[r + c * SJ_MAX] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  const int m = n + (n & 1);
  const int npairs = m / 2;
  double off_prev = 1e300;
  bool conv = false;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
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
    if (sweep == max_sweeps) break;
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

// ------------------------------------------------------ large-n version
// Templated on the real type T (float or double): the large-n solver first
// sweeps in FP32 (the FP64 pipe of this part is 1/58 of the FP32 one), then
// re-orthonormalises the FP32 eigenvectors in FP64, forms Z^H G Z in FP64
// (nearly diagonal) and finishes with a few FP64 sweeps.
constexpr int LJ_T = 256;

template <typename T> struct Cx;
// eps: threshold of the rotation skip, |b| <= eps sqrt(|a d|) (unit round-off)
template <> struct Cx<double> {
  using C = double2;
  static __device__ __forceinline__ C mk(double x, double y) { return make_double2(x, y); }
  static constexpr double tiny = 1e-300, huge = 1e150, eps = 1.1102230246251565e-16;
};
template <> struct Cx<float> {
  using C = float2;
  static __device__ __forceinline__ C mk(float x, float y) { return make_float2(x, y); }
  static constexpr float tiny = 1e-30f, huge = 1e15f, eps = 5.9604645e-8f;
};

template <typename T>
struct RotT {
  T c, s, px, py, app, aqq;
};

template <typename T>
__device__ __forceinline__ RotT<T> make_rot_t(T a, T d, typename Cx<T>::C b) {
  RotT<T> r;
  const T ab = sqrt(b.x * b.x + b.y * b.y);
  // threshold Jacobi: an entry below eps sqrt(|a d|) changes neither the
  // eigenvalues nor the eigenvectors at working precision; skip it
  if (!(ab > Cx<T>::tiny) || ab <= Cx<T>::eps * sqrt(fabs(a) * fabs(d))) {
    r.c = T(1); r.s = T(0); r.px = T(1); r.py = T(0); r.app = a; r.aqq = d;
    return r;
  }
  r.px = b.x / ab;
  r.py = b.y / ab;
  const T tau = (d - a) / (T(2) * ab);
  T t;
  if (fabs(tau) > Cx<T>::huge) t = T(0.5) / tau;
  else t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
  r.c = T(1) / sqrt(T(1) + t * t);
  r.s = t * r.c;
  r.app = a - t * ab;
  r.aqq = d + t * ab;
  return r;
}

// (x_p, x_q) <- (x_p, x_q) J   with J = [[c, s phi], [-s conj(phi), c]]
template <typename T, typename C>
__device__ __forceinline__ void rot_cols_t(C& xp, C& xq, const RotT<T>& r) {
  const T sx = r.s * r.px, sy = r.s * r.py;  // s phi
  // xp' = c xp - conj(s phi) xq ; xq' = (s phi) xp + c xq
  const T npx = r.c * xp.x - (sx * xq.x + sy * xq.y);
  const T npy = r.c * xp.y - (sx * xq.y - sy * xq.x);
  const T nqx = (sx * xp.x - sy * xp.y) + r.c * xq.x;
  const T nqy = (sx * xp.y + sy * xp.x) + r.c * xq.y;
  xp.x = npx; xp.y = npy; xq.x = nqx; xq.y = nqy;
}
// (y_p; y_q) <- J^H (y_p; y_q)
template <typename T, typename C>
__device__ __forceinline__ void rot_rows_t(C& yp, C& yq, const RotT<T>& r) {
  const T sx = r.s * r.px, sy = r.s * r.py;
  // yp' = c yp - (s phi) yq ; yq' = conj(s phi) yp + c yq
  const T npx = r.c * yp.x - (sx * yq.x - sy * yq.y);
  const T npy = r.c * yp.y - (sx * yq.y + sy * yq.x);
  const T nqx = (sx * yp.x + sy * yp.y) + r.c * yq.x;
  const T nqy = (sx * yp.y - sy * yp.x) + r.c * yq.y;
  yp.x = npx; yp.y = npy; yq.x = nqx; yq.y = nqy;
}

template <typename T>
__device__ __forceinline__ RotT<T> load_rot_t(const T* __restrict__ params, int k) {
  const T* pp = params + 8 * k;
  RotT<T> r;
  r.c = pp[0]; r.s = pp[1]; r.px = pp[2]; r.py = pp[3]; r.app = pp[4]; r.aqq = pp[5];
  return r;
}

__global__ void init32_kernel(int64_t n, const double2* G, int64_t ldg, float2* G32, float2* Z32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n) return;
  const double2 g = G[i + j * ldg];
  G32[i + j * n] = make_float2((float)g.x, (float)g.y);
  Z32[i + j * n] = make_float2(i == j ? 1.f : 0.f, 0.f);
}
__global__ void promote_kernel(int64_t n, const float2* Z32, double2* Z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n) return;
  const float2 z = Z32[i + j * n];
  Z[i + j * n] = make_double2((double)z.x, (double)z.y);
}
__global__ void identity_kernel(int64_t n, double2* Z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i < n) Z[i + j * n] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// Pair k of round `round`, G double-buffered: the owner of pair (p, q) writes
// the new columns p, q of J^H G J into Gnew, reading only the pre-round Gold,
// so owners never race. Its column rotation J_k mixes columns p and q row by
// row; then every pair's row rotation J_k'^H (computed once per round, in
// `params`) mixes rows (p', q') of these two columns. Z is updated in place:
// its columns p, q belong to this owner alone.
template <typename T>
__device__ void process_pair(int64_t n, int m, int round, int k,
                             const typename Cx<T>::C* __restrict__ Gold,
                             typename Cx<T>::C* __restrict__ Gnew, typename Cx<T>::C* __restrict__ Zw,
                             typename Cx<T>::C* colbuf, const T* __restrict__ params,
                             const T* sparams) {
  using C = typename Cx<T>::C;
  int p, q;
  rr_pair(m, round, k, p, q);
  // odd n: the pair holding the padding index n has one real column, p, which
  // still receives every other pair's row rotation
  const bool single = q >= n;
  if (single) q = p;
  C* gp = colbuf;
  C* gq = colbuf + n;
  RotT<T> r = load_rot_t(params, k);
  if (single) r.s = T(0);
  const C* Gp = Gold + (int64_t)p * n;
  const C* Gq = Gold + (int64_t)q * n;
  C* Zp = Zw + (int64_t)p * n;
  C* Zq = Zw + (int64_t)q * n;
  for (int64_t i = threadIdx.x; i < n; i += LJ_T) {
    C a = Gp[i], b = Gq[i];
    if (r.s != T(0)) rot_cols_t(a, b, r);
    gp[i] = a;
    gq[i] = b;
    if (r.s != T(0)) {
      C x = Zp[i], y = Zq[i];
      rot_cols_t(x, y, r);
      Zp[i] = x;
      Zq[i] = y;
    }
  }
  __syncthreads();
  for (int kk = threadIdx.x; kk < m / 2; kk += LJ_T) {
    int pr, qr;
    rr_pair(m, round, kk, pr, qr);
    if (qr >= n) continue;
    const RotT<T> rk = load_rot_t(sparams, kk);
    if (rk.s == T(0)) continue;
    rot_rows_t(gp[pr], gp[qr], rk);
    rot_rows_t(gq[pr], gq[qr], rk);
  }
  __syncthreads();
  if (threadIdx.x == 0 && r.s != T(0)) {  // exact 2 x 2 block of this pair
    gp[p] = Cx<T>::mk(r.app, T(0));
    gq[q] = Cx<T>::mk(r.aqq, T(0));
    gp[q] = Cx<T>::mk(T(0), T(0));
    gq[p] = Cx<T>::mk(T(0), T(0));
  }
  __syncthreads();
  C* Np_ = Gnew + (int64_t)p * n;
  C* Nq_ = Gnew + (int64_t)q * n;
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
      }
    }
    __threadfence();
    if (*(volatile int*)status != 0) ok_s = 0;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename T>
struct CoopArgs {
  int64_t n;
  int m, max_sweeps;
  double tol_conv, tol_stag;  // converged: off <= tol_conv fro, or <= tol_stag fro and stalled
  typename Cx<T>::C* G0;
  typename Cx<T>::C* G1;
  typename Cx<T>::C* Z;
  T* params;        // 8 values per pair of the current round
  double* red;      // 2 * gridDim.x partial sums
  unsigned* bar;    // barrier counter and generation
  int* status;      // [0] error, [1] sweeps, [2] converged, [3] result in G1
};

// A whole cyclic Jacobi in one cooperative launch: per sweep a fixed-order
// off-norm test (identical in every block, so the decision is uniform), then
// the m - 1 rounds; per round the rotations are computed once (phase A) and
// applied by the pair owners (phase B), each phase closed by a grid barrier.
template <typename T>
__global__ void __launch_bounds__(LJ_T) jacobi_coop_kernel(CoopArgs<T> a) {
  using C = typename Cx<T>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* colbuf = reinterpret_cast<C*>(smem_raw);
  // this round's rotations, staged once per block (8 values per pair)
  T* sparams = reinterpret_cast<T*>(colbuf + 2 * a.n);
  __shared__ double so[LJ_T], sf[LJ_T];
  __shared__ int decide;
  const int64_t n = a.n;
  const int npairs = a.m / 2;
  C* Gcur = a.G0;
  C* Gnxt = a.G1;
  double off_prev = 1e300;
  int sweep = 0;
  bool conv = false, alive = true;
  for (; sweep <= a.max_sweeps && alive; ++sweep) {
    double o = 0.0, f = 0.0;
    const int64_t tot = n * n;
    for (int64_t e = (int64_t)blockIdx.x * LJ_T + threadIdx.x; e < tot; e += (int64_t)gridDim.x * LJ_T) {
      const C g = Gcur[e];
      const double v = (double)g.x * g.x + (double)g.y * g.y;
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
      if (off == 0.0 || off <= a.tol_conv * fro || (off <= a.tol_stag * fro && off > 0.25 * off_prev))
        d = 1;
      else if (sweep == a.max_sweeps)
        d = 2;
      off_prev = off;
      decide = d;
    }
    __syncthreads();
    // every block has read the partials before any block rewrites them
    if (!grid_sync(a.bar, a.status)) { alive = false; break; }
    if (decide == 1) { conv = true; break; }
    if (decide == 2) break;
    for (int round = 0; round < a.m - 1; ++round) {
      if constexpr (sizeof(T) == 4) {
        // FP32: every block computes all of this round's rotations itself (cheap
        // in FP32), which saves the grid barrier between computing and applying
        for (int k = threadIdx.x; k < npairs; k += LJ_T) {
          int p, q;
          rr_pair(a.m, round, k, p, q);
          const RotT<T> r = q < n ? make_rot_t<T>(Gcur[p + (int64_t)p * n].x,
                                                  Gcur[q + (int64_t)q * n].x,
                                                  Gcur[p + (int64_t)q * n])
                                  : make_rot_t<T>(T(0), T(0), Cx<T>::mk(T(0), T(0)));
          T* pp = sparams + 8 * k;
          pp[0] = r.c; pp[1] = r.s; pp[2] = r.px; pp[3] = r.py; pp[4] = r.app; pp[5] = r.aqq;
        }
        __syncthreads();
        for (int k = blockIdx.x; k < npairs; k += gridDim.x)
          process_pair<T>(n, a.m, round, k, Gcur, Gnxt, a.Z, colbuf, sparams, sparams);
      } else {
        // FP64 rotations are expensive on this part: computed once (phase A),
        // published through global memory, then applied (phase B)
        for (int k = blockIdx.x * LJ_T + threadIdx.x; k < npairs; k += gridDim.x * LJ_T) {
          int p, q;
          rr_pair(a.m, round, k, p, q);
          const RotT<T> r = q < n ? make_rot_t<T>(Gcur[p + (int64_t)p * n].x,
                                                  Gcur[q + (int64_t)q * n].x,
                                                  Gcur[p + (int64_t)q * n])
                                  : make_rot_t<T>(T(0), T(0), Cx<T>::mk(T(0), T(0)));
          T* pp = a.params + 8 * k;
          pp[0] = r.c; pp[1] = r.s; pp[2] = r.px; pp[3] = r.py; pp[4] = r.app; pp[5] = r.aqq;
        }
        if (!grid_sync(a.bar, a.status)) { alive = false; break; }
        for (int e = threadIdx.x; e < 8 * npairs; e += LJ_T) sparams[e] = a.params[e];
        __syncthreads();
        for (int k = blockIdx.x; k < npairs; k += gridDim.x)
          process_pair<T>(n, a.m, round, k, Gcur, Gnxt, a.Z, colbuf, a.params, sparams);
      }
      if (!grid_sync(a.bar, a.status)) { alive = false; break; }
      C* t = Gcur;
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

// Runs one cooperative Jacobi on G0 (destroyed; the result may end in G1).
// Returns CHASE_OK and fills *sweeps, *conv, *in_g1; CHASE_ERR_CUDA on a
// launch failure or an expired barrier.
template <typename T>
int run_coop(cudaStream_t s, int64_t n, typename Cx<T>::C* G0, typename Cx<T>::C* G1,
             typename Cx<T>::C* Z, T* params, double* red, int max_sweeps, double tol_conv,
             double tol_stag, int* sweeps, bool* conv, bool* in_g1) {
  using C = typename Cx<T>::C;
  const int m = (int)(n + (n & 1));
  const int npairs = m / 2;
  const size_t smem = (size_t)2 * n * sizeof(C) + (size_t)8 * npairs * sizeof(T);
  // The opt-in limit covers dynamic + static shared memory (the kernel's static
  // reduction arrays add 4 KB, so sizes just under 48 KB need it too). It is a
  // process-wide property of the function that concurrent solves on other host
  // threads share, so it is set once per device to the largest size any
  // context can ask for (n <= 3500), never lowered.
  static std::once_flag attr_once[kMaxDevices];
  once_per_device(attr_once, []() {
    constexpr int64_t nmax = 3500;
    const size_t most = (size_t)2 * nmax * sizeof(C) + (size_t)8 * (nmax / 2) * sizeof(T);
    cudaFuncSetAttribute(jacobi_coop_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)most);
  });
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  const cudaError_t oe =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel<T>, LJ_T, smem);
  if (!coop || oe != cudaSuccess || per_sm < 1) {
    fprintf(stderr,
            "[chase] Jacobi (%s) n=%lld: no cooperative residency (coop %d, occupancy %s, "
            "blocks/SM %d, dynamic smem %zu B)\n",
            sizeof(T) == 4 ? "FP32" : "FP64", (long long)n, coop, cudaGetErrorString(oe), per_sm,
            smem);
    return CHASE_CUDA_FAIL();
  }
  // one pair per block where the blocks fit, so pairs run concurrently
  const int grid = std::min(std::min(npairs, per_sm * nsm), kCoopMaxGrid);
  unsigned* bar = reinterpret_cast<unsigned*>(red + 2 * kCoopMaxGrid);
  int* st = reinterpret_cast<int*>(red + 2 * kCoopMaxGrid + 2);
  if (cudaMemsetAsync(red + 2 * kCoopMaxGrid, 0, 8 * sizeof(double), s) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  CoopArgs<T> args;
  args.n = n;
  args.m = m;
  args.max_sweeps = max_sweeps;
  args.tol_conv = tol_conv;
  args.tol_stag = tol_stag;
  args.G0 = G0;
  args.G1 = G1;
  args.Z = Z;
  args.params = params;
  args.red = red;
  args.bar = bar;
  args.status = st;
  void* kargs[] = {&args};
  if (cudaLaunchCooperativeKernel((const void*)jacobi_coop_kernel<T>, dim3(grid), dim3(LJ_T), kargs,
                                  smem, s) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  count_launch();
  int hst[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  if (hst[0] != 0) {
    fprintf(stderr, "[chase] Jacobi: grid barrier wait expired\n");
    return CHASE_CUDA_FAIL();
  }
  *sweeps = hst[1];
  *conv = hst[2] != 0;
  *in_g1 = hst[3] != 0;
  return CHASE_OK;
}

// ------------------------------------------------------ blocked FP32 Jacobi
// The FP32 stage as a block Jacobi method: the columns are cut into blocks of
// BJ_B, the blocks are paired in round-robin order (as the scalar method pairs
// columns), and per round every block pair's 2 BJ_B x 2 BJ_B principal
// submatrix S is diagonalised by one cyclic Jacobi sweep in shared memory,
// which accumulates its rotations into R (S <- R^H S R). The pair's columns of
// G and Z are then multiplied by R and its rows of G by R^H, as small GEMMs.
// Pairs of one round touch disjoint columns (and rows), so they run in
// parallel; a sweep visits every block pair once. Compared with one scalar
// rotation per column pair and round, the matrix streams through memory
// BJ_B times less often.
constexpr int BJ_B = 32;          // block width
constexpr int BJ_M = 2 * BJ_B;    // order of a block pair
constexpr int BJ_T = 256;
constexpr int BJ_ROWS = 64;       // rows (or columns) of G per CTA in the update kernels
constexpr int BJ_UPD_SMEM = (BJ_M * (BJ_M + 1) + BJ_ROWS * (BJ_M + 1)) * (int)sizeof(float2);

__device__ __forceinline__ void bj_pair(int64_t n, int nb, int nbp, int round, int k, int64_t& i0,
                                        int& ni, int64_t& j0, int& nj) {
  auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (nbp - 1); };
  int p = pos(k), q = pos(nbp - 1 - k);
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  i0 = (int64_t)p * BJ_B;
  j0 = (int64_t)q * BJ_B;
  ni = p < nb ? (int)min((int64_t)BJ_B, n - i0) : 0;
  nj = q < nb ? (int)min((int64_t)BJ_B, n - j0) : 0;
}
// global index of local index a of a block pair (first block, then second)
__device__ __forceinline__ int64_t bj_gidx(int a, int64_t i0, int ni, int64_t j0) {
  return a < ni ? i0 + a : j0 + (a - ni);
}

constexpr int BJ_INNER_SMEM = 2 * BJ_M * (BJ_M + 1) * (int)sizeof(float2);

__global__ void __launch_bounds__(BJ_T)
    bj_inner_kernel(int64_t n, int nb, int nbp, int round, const float2* __restrict__ G,
                    float2* __restrict__ Rbuf) {
  extern __shared__ float2 bj_smem[];
  float2 (*S)[BJ_M + 1] = reinterpret_cast<float2 (*)[BJ_M + 1]>(bj_smem);
  float2 (*R)[BJ_M + 1] = reinterpret_cast<float2 (*)[BJ_M + 1]>(bj_smem + BJ_M * (BJ_M + 1));
  __shared__ RotT<float> rots[BJ_M / 2];
  __shared__ int pq[BJ_M / 2][2];  // this round's index pairs
  const int k = blockIdx.x, t = threadIdx.x;
  int64_t i0, j0;
  int ni, nj;
  bj_pair(n, nb, nbp, round, k, i0, ni, j0, nj);
  const int m = ni + nj;
  // a full pair (m = 64, the common case): thread t always takes row/column
  // t % 64 of the pairs t / 64, t / 64 + 4, ... (no index arithmetic per element)
  static_assert(BJ_T % BJ_M == 0, "fixed element mapping");
  const bool full = m == BJ_M;
  for (int e = t; e < m * m; e += BJ_T) {
    const int a = e % m, c = e / m;
    S[a][c] = G[bj_gidx(a, i0, ni, j0) + bj_gidx(c, i0, ni, j0) * n];
    R[a][c] = make_float2(a == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  const int mp = m + (m & 1);
  for (int rd = 0; rd < mp - 1; ++rd) {
    if (t < mp / 2) {
      int p, q;
      rr_pair(mp, rd, t, p, q);
      pq[t][0] = p;
      pq[t][1] = q;
      rots[t] = q < m ? make_rot_t<float>(S[p][p].x, S[q][q].x, S[p][q])
                      : make_rot_t<float>(0.f, 0.f, make_float2(0.f, 0.f));
    }
    __syncthreads();
    if (full) {  // column rotations of S and R
      const int i = t % BJ_M;
#pragma unroll 4
      for (int kk = t / BJ_M; kk < BJ_M / 2; kk += BJ_T / BJ_M) {
        const RotT<float> r = rots[kk];
        if (r.s == 0.f) continue;
        const int p = pq[kk][0], q = pq[kk][1];
        rot_cols_t(S[i][p], S[i][q], r);
        rot_cols_t(R[i][p], R[i][q], r);
      }
    } else {
      for (int e = t; e < (mp / 2) * m; e += BJ_T) {
        const int kk = e / m, i = e % m;
        const int p = pq[kk][0], q = pq[kk][1];
        if (q >= m || rots[kk].s == 0.f) continue;
        rot_cols_t(S[i][p], S[i][q], rots[kk]);
        rot_cols_t(R[i][p], R[i][q], rots[kk]);
      }
    }
    __syncthreads();
    if (full) {  // row rotations of S
      const int j = t % BJ_M;
#pragma unroll 4
      for (int kk = t / BJ_M; kk < BJ_M / 2; kk += BJ_T / BJ_M) {
        const RotT<float> r = rots[kk];
        if (r.s == 0.f) continue;
        rot_rows_t(S[pq[kk][0]][j], S[pq[kk][1]][j], r);
      }
    } else {
      for (int e = t; e < (mp / 2) * m; e += BJ_T) {
        const int kk = e / m, j = e % m;
        const int p = pq[kk][0], q = pq[kk][1];
        if (q >= m || rots[kk].s == 0.f) continue;
        rot_rows_t(S[p][j], S[q][j], rots[kk]);
      }
    }
    __syncthreads();
    if (t < mp / 2) {  // the rotated 2 x 2 block exactly
      const int p = pq[t][0], q = pq[t][1];
      if (q < m && rots[t].s != 0.f) {
        S[p][p] = make_float2(rots[t].app, 0.f);
        S[q][q] = make_float2(rots[t].aqq, 0.f);
        S[p][q] = make_float2(0.f, 0.f);
        S[q][p] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
  }
  float2* Rk = Rbuf + (int64_t)k * BJ_M * BJ_M;
  for (int e = t; e < m * m; e += BJ_T) Rk[(e % m) + (e / m) * BJ_M] = R[e % m][e / m];
}

// Columns of the pair: M(r0:r0+64, idx) <- M(r0:r0+64, idx) R for M = G and Z.
__global__ void __launch_bounds__(BJ_T)
    bj_cols_kernel(int64_t n, int nb, int nbp, int round, float2* __restrict__ G,
                   float2* __restrict__ Z, const float2* __restrict__ Rbuf) {
  extern __shared__ float2 bj_smem[];
  float2* R = bj_smem;                      // [BJ_M][BJ_M + 1]
  float2* T = bj_smem + BJ_M * (BJ_M + 1);  // [BJ_ROWS][BJ_M + 1]
  const int k = blockIdx.y, t = threadIdx.x;
  int64_t i0, j0;
  int ni, nj;
  bj_pair(n, nb, nbp, round, k, i0, ni, j0, nj);
  const int m = ni + nj;
  if (m == 0) return;
  const float2* Rk = Rbuf + (int64_t)k * BJ_M * BJ_M;
  for (int e = t; e < m * m; e += BJ_T) R[(e % m) * (BJ_M + 1) + e / m] = Rk[(e % m) + (e / m) * BJ_M];
  const int64_t r0 = (int64_t)blockIdx.x * BJ_ROWS;
  const int tx = t & 15, ty = t >> 4;  // columns tx + 16 c, rows ty + 16 r
  for (int mat = 0; mat < 2; ++mat) {
    float2* M = mat == 0 ? G : Z;
    __syncthreads();
    for (int e = t; e < BJ_ROWS * m; e += BJ_T) {
      const int i = e % BJ_ROWS, a = e / BJ_ROWS;
      const int64_t row = r0 + i;
      T[i * (BJ_M + 1) + a] =
          row < n ? M[row + bj_gidx(a, i0, ni, j0) * n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 o[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) o[r][c] = make_float2(0.f, 0.f);
    for (int a = 0; a < m; ++a) {
      float2 x[4], y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x[r] = T[(ty + 16 * r) * (BJ_M + 1) + a];
#pragma unroll
      for (int c = 0; c < 4; ++c) y[c] = R[a * (BJ_M + 1) + tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          o[r][c].x = fmaf(x[r].x, y[c].x, fmaf(-x[r].y, y[c].y, o[r][c].x));
          o[r][c].y = fmaf(x[r].x, y[c].y, fmaf(x[r].y, y[c].x, o[r][c].y));
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t row = r0 + ty + 16 * r;
      if (row >= n) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int cc = tx + 16 * c;
        if (cc < m) M[row + bj_gidx(cc, i0, ni, j0) * n] = o[r][c];
      }
    }
  }
}

// Rows of the pair: G(idx, c0:c0+64) <- R^H G(idx, c0:c0+64).
__global__ void __launch_bounds__(BJ_T)
    bj_rows_kernel(int64_t n, int nb, int nbp, int round, float2* __restrict__ G,
                   const float2* __restrict__ Rbuf) {
  extern __shared__ float2 bj_smem[];
  float2* R = bj_smem;                      // [BJ_M][BJ_M + 1]
  float2* T = bj_smem + BJ_M * (BJ_M + 1);  // [BJ_M][BJ_ROWS + 1] (rows of the pair x columns)
  const int k = blockIdx.y, t = threadIdx.x;
  int64_t i0, j0;
  int ni, nj;
  bj_pair(n, nb, nbp, round, k, i0, ni, j0, nj);
  const int m = ni + nj;
  if (m == 0) return;
  const float2* Rk = Rbuf + (int64_t)k * BJ_M * BJ_M;
  for (int e = t; e < m * m; e += BJ_T) R[(e % m) * (BJ_M + 1) + e / m] = Rk[(e % m) + (e / m) * BJ_M];
  const int64_t c0 = (int64_t)blockIdx.x * BJ_ROWS;
  for (int e = t; e < m * BJ_ROWS; e += BJ_T) {
    const int a = e % m, j = e / m;
    const int64_t col = c0 + j;
    T[a * (BJ_ROWS + 1) + j] = col < n ? G[bj_gidx(a, i0, ni, j0) + col * n] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int tx = t & 15, ty = t >> 4;  // columns tx + 16 c, pair rows ty + 16 r
  float2 o[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) o[r][c] = make_float2(0.f, 0.f);
  for (int b = 0; b < m; ++b) {
    float2 x[4], y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int a = ty + 16 * r;  // (R^H)(a, b) = conj(R(b, a))
      const float2 rv = a < m ? R[b * (BJ_M + 1) + a] : make_float2(0.f, 0.f);
      x[r] = make_float2(rv.x, -rv.y);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] = T[b * (BJ_ROWS + 1) + tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        o[r][c].x = fmaf(x[r].x, y[c].x, fmaf(-x[r].y, y[c].y, o[r][c].x));
        o[r][c].y = fmaf(x[r].x, y[c].y, fmaf(x[r].y, y[c].x, o[r][c].y));
      }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = ty + 16 * r;
    if (a >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t col = c0 + tx + 16 * c;
      if (col < n) G[bj_gidx(a, i0, ni, j0) + col * n] = o[r][c];
    }
  }
}

// Off-diagonal and total squared Frobenius norms of G (n x n, FP32): one
// partial pair per block, summed on the host in a fixed order.
__global__ void bj_norms_kernel(int64_t n, const float2* __restrict__ G, double* __restrict__ part) {
  __shared__ double so[256], sf[256];
  double o = 0.0, f = 0.0;
  const int64_t tot = n * n;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < tot; e += (int64_t)gridDim.x * 256) {
    const float2 g = G[e];
    const double v = (double)g.x * g.x + (double)g.y * g.y;
    f += v;
    if (e % n != e / n) o += v;
  }
  so[threadIdx.x] = o;
  sf[threadIdx.x] = f;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) {
      so[threadIdx.x] += so[threadIdx.x + w];
      sf[threadIdx.x] += sf[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = so[0];
    part[2 * blockIdx.x + 1] = sf[0];
  }
}

std::once_flag g_bj_attr[kMaxDevices];

// Blocked FP32 Jacobi on G (n x n, destroyed) with eigenvectors into Z (starts
// as I): sweeps until off(G) <= tol_conv ||G||_F, or <= tol_stag ||G||_F with
// less than a 4x decrease in the last sweep, or max_sweeps. part: 512 doubles
// of device scratch, host_part: 512 doubles of host memory.
int run_block_jacobi32(cudaStream_t s, int64_t n, float2* G, float2* Z, float2* Rbuf,
                       double* part, double* host_part, int max_sweeps, double tol_conv,
                       double tol_stag, int* sweeps, bool* conv) {
  once_per_device(g_bj_attr, []() {
    cudaFuncSetAttribute(bj_inner_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         BJ_INNER_SMEM);
    cudaFuncSetAttribute(bj_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BJ_UPD_SMEM);
    cudaFuncSetAttribute(bj_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BJ_UPD_SMEM);
  });
  const int nb = (int)cdiv(n, BJ_B);
  const int nbp = nb + (nb & 1);
  const int npair = nbp / 2;
  const unsigned gt = (unsigned)cdiv(n, BJ_ROWS);
  constexpr int kNormBlocks = 256;
  double off_prev = 1e300;
  *conv = false;
  int sw = 0;
  for (; sw <= max_sweeps; ++sw) {
    bj_norms_kernel<<<kNormBlocks, 256, 0, s>>>(n, G, part);
    count_launch();
    if (cudaMemcpyAsync(host_part, part, 2 * kNormBlocks * sizeof(double), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return CHASE_CUDA_FAIL();
    double o = 0.0, f = 0.0;
    for (int b = 0; b < kNormBlocks; ++b) {
      o += host_part[2 * b];
      f += host_part[2 * b + 1];
    }
    const double off = std::sqrt(o), fro = std::sqrt(f);
    if (off == 0.0 || off <= tol_conv * fro || (off <= tol_stag * fro && off > 0.25 * off_prev)) {
      *conv = true;
      break;
    }
    off_prev = off;
    if (sw == max_sweeps) break;
    for (int rd = 0; rd < nbp - 1; ++rd) {
      bj_inner_kernel<<<npair, BJ_T, BJ_INNER_SMEM, s>>>(n, nb, nbp, rd, G, Rbuf);
      bj_cols_kernel<<<dim3(gt, (unsigned)npair, 1), BJ_T, BJ_UPD_SMEM, s>>>(n, nb, nbp, rd, G, Z,
                                                                          Rbuf);
      bj_rows_kernel<<<dim3(gt, (unsigned)npair, 1), BJ_T, BJ_UPD_SMEM, s>>>(n, nb, nbp, rd, G,
                                                                          Rbuf);
      count_launch();
      count_launch();
      count_launch();
    }
    if (cudaGetLastError() != cudaSuccess) return CHASE_CUDA_FAIL();
  }
  *sweeps = sw;
  return CHASE_OK;
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

// ------------------------------------------ FP64 refinement of the FP32 pairs
// One step of the iterative refinement of Ogita and Aishima (2018) for an
// approximate eigenvector matrix X of Hermitian G, with S = X^H G X and
// R = I - X^H X: lambda_i = Re s_ii / (1 - Re r_ii) and
// E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) (i != j), E_ii = r_ii / 2,
// then X <- X (I + E). Quadratic convergence from the FP32 Jacobi vectors. A
// pair whose first-order correction would exceed 1e-3 (eigenvalues too close
// to separate at this accuracy; larger corrections made near-degenerate pairs
// oscillate in tests) is only orthogonalised (E_ij = r_ij / 2); the largest
// |s_ij| of such pairs is reported so that FP64 Jacobi sweeps can finish them.
__global__ void oa_lambda_kernel(int64_t n, const double2* __restrict__ S,
                                 const double2* __restrict__ XX, double* __restrict__ lam) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  lam[i] = S[i + i * n].x / XX[i + i * n].x;  // 1 - r_ii = (X^H X)_ii
}
__global__ void oa_e_kernel(int64_t n, const double2* __restrict__ S,
                            const double2* __restrict__ XX, const double* __restrict__ lam,
                            double2* __restrict__ E, double* __restrict__ partial,
                            int* __restrict__ pairs, int* __restrict__ npairs) {
  __shared__ double me[256], mc[256];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // row
  const int64_t j = blockIdx.y;                                        // column
  double emax = 0.0, cmax = 0.0;
  if (i < n) {
    const double2 x = XX[i + j * n];
    const double2 r = make_double2((i == j ? 1.0 : 0.0) - x.x, -x.y);
    double2 e;
    if (i == j) {
      e = make_double2(0.5 * r.x, 0.5 * r.y);
      emax = 0.5 * sqrt(r.x * r.x + r.y * r.y);
    } else {
      const double2 sv = S[i + j * n];
      const double lj = lam[j], d = lj - lam[i];
      const double2 num = make_double2(fma(lj, r.x, sv.x), fma(lj, r.y, sv.y));
      const double an = sqrt(num.x * num.x + num.y * num.y);
      if (an <= 1e-3 * fabs(d)) {
        e = make_double2(num.x / d, num.y / d);
        emax = an / fabs(d);
      } else {
        e = make_double2(0.5 * r.x, 0.5 * r.y);
        emax = 0.5 * sqrt(r.x * r.x + r.y * r.y);
        cmax = sqrt(sv.x * sv.x + sv.y * sv.y);
        // a pair left to the FP64 finish: recorded (capacity permitting; the
        // host takes the full FP64 sweeps when the list overflows)
        const int k = atomicAdd(npairs, 1);
        if (k < kMaxClusterPairs) {
          pairs[2 * k] = (int)i;
          pairs[2 * k + 1] = (int)j;
        }
      }
    }
    E[i + j * n] = e;
  }
  me[threadIdx.x] = emax;
  mc[threadIdx.x] = cmax;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) {
      me[threadIdx.x] = fmax(me[threadIdx.x], me[threadIdx.x + w]);
      mc[threadIdx.x] = fmax(mc[threadIdx.x], mc[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
    partial[2 * b] = me[0];
    partial[2 * b + 1] = mc[0];
  }
}
// E = (I - XX) / 2: one orthogonalisation step X <- X (I + E)
__global__ void half_residual_kernel(int64_t n, const double2* __restrict__ XX,
                                     double2* __restrict__ E) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const double2 x = XX[i + j * n];
  E[i + j * n] = make_double2(0.5 * ((i == j ? 1.0 : 0.0) - x.x), -0.5 * x.y);
}
__global__ void max2_kernel(int64_t nb, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double a[256], c[256];
  double x = 0.0, y = 0.0;
  for (int64_t b = threadIdx.x; b < nb; b += 256) {
    x = fmax(x, partial[2 * b]);
    y = fmax(y, partial[2 * b + 1]);
  }
  a[threadIdx.x] = x;
  c[threadIdx.x] = y;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) {
      a[threadIdx.x] = fmax(a[threadIdx.x], a[threadIdx.x + w]);
      c[threadIdx.x] = fmax(c[threadIdx.x], c[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = a[0];
    out[1] = c[0];
  }
}
// Block S_c = X_c^H (G X_c) of each cluster c of size k (clusters of one size,
// consecutive in XI / TI): one CTA per cluster, one warp per output entry at a
// time, lanes over rows, fixed-order reduction. Output k x k column-major.
__global__ void cluster_gram_kernel(int64_t n, int k, const double2* __restrict__ XI,
                                    const double2* __restrict__ TI, int64_t ld,
                                    double2* __restrict__ Sout) {
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2* X = XI + (int64_t)c * k * ld;
  const double2* T = TI + (int64_t)c * k * ld;
  for (int e = warp; e < k * k; e += blockDim.x >> 5) {
    const int a = e % k, b = e / k;
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t r = lane; r < n; r += 32) acc = cadd(acc, cmulc(X[r + a * ld], T[r + b * ld]));
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) Sout[(int64_t)c * k * k + a + b * k] = acc;
  }
}
// X(:, idx_c) = XI_c Z_c for each cluster (its FP64 eigenvectors), and the
// cluster's eigenvalues into lam at the same column indices.
__global__ void cluster_apply_kernel(int64_t n, int k, const double2* __restrict__ XI, int64_t ld,
                                     const double2* __restrict__ Z, const double* __restrict__ wz,
                                     const int* __restrict__ idx, double2* __restrict__ X,
                                     double* __restrict__ lam) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  const double2* Xc = XI + (int64_t)c * k * ld;
  const double2* Zc = Z + (int64_t)c * k * k;
  const int* ic = idx + (int64_t)c * k;
  if (blockIdx.x == 0 && threadIdx.x < k) lam[ic[threadIdx.x]] = wz[(int64_t)c * k + threadIdx.x];
  if (r >= n) return;
  for (int b = 0; b < k; ++b) {
    double2 acc = make_double2(0.0, 0.0);
    for (int a = 0; a < k; ++a) acc = cadd(acc, cmul(Xc[r + a * ld], Zc[a + b * k]));
    X[r + (int64_t)ic[b] * n] = acc;
  }
}

// X(:, idx[j]) = P(:, j) and lam[idx[j]] = Re S(j, j) for a large cluster's
// eigenvectors P (n x m, ld n) and its diagonalised block S (m x m, ld m).
__global__ void scatter_cluster_kernel(int64_t n, int64_t m, const double2* __restrict__ P,
                                       const int* __restrict__ idx, const double2* __restrict__ S,
                                       double2* __restrict__ X, double* __restrict__ lam) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) lam[idx[j]] = S[j + j * m].x;
  if (r < n) X[r + (int64_t)idx[j] * n] = P[r + j * n];
}

__global__ void rank_vec_kernel(int64_t n, const double* __restrict__ lam, double* w, int* rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = lam[i];
  int64_t rk = 0;
  for (int64_t j = 0; j < n; ++j) {
    const double u = lam[j];
    rk += (u < v) || (u == v && j < i);
  }
  rank[i] = (int)rk;
  w[rk] = v;
}
__global__ void frob2_kernel(int64_t n, const double2* __restrict__ G, int64_t ldg,
                             double* __restrict__ partial) {
  __shared__ double a[256];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  double v = 0.0;
  if (i < n) {
    const double2 g = G[i + j * ldg];
    v = g.x * g.x + g.y * g.y;
  }
  a[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) a[threadIdx.x] += a[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
    partial[2 * b] = sqrt(a[0]);  // max of column-block norms: a cheap scale of ||G||
    partial[2 * b + 1] = 0.0;
  }
}

std::once_flag g_small_attr[kMaxDevices];

}  // namespace

size_t jacobi_red_elems() { return (size_t)2 * kCoopMaxGrid + 16; }

namespace {
// refinement products: P = A B (n x n) or P = X^H Y, on the tensor cores when
// the context supplied a product, else with the CUDA-core kernels
cudaError_t heev_nn(cudaStream_t s, const JacobiWork& wk, bool tc, int64_t n, const double2* A,
                    int64_t lda, const double2* B, const Epilogue& ep, bool extended = false) {
  if (tc && wk.gemm) return wk.gemm(wk.gemm_ctx, n, n, A, lda, false, n, B, n, ep, extended);
  return zgemm_nn(s, n, n, n, A, lda, B, n, ep);
}
cudaError_t heev_cn(cudaStream_t s, const JacobiWork& wk, bool tc, int64_t n, const double2* X,
                    const double2* Y, double2* P, bool hermitian, bool extended = false) {
  if (tc && wk.gemm) {
    Epilogue ep{};
    ep.mode = EPI_STORE;
    ep.Y = P;
    ep.ldy = n;
    cudaError_t e = wk.gemm(wk.gemm_ctx, n, n, X, n, true, n, Y, n, ep, extended);
    if (e != cudaSuccess || !hermitian) return e;
    return hermitian_part(s, n, P, n);
  }
  return zgram(s, n, n, n, X, n, Y, n, P, n, hermitian, wk.gram_ws, wk.gram_ws_elems);
}
}  // namespace

size_t jacobi_rot_elems(int64_t n) {
  const int64_t nb = cdiv(n, BJ_B);
  return (size_t)((nb + 1) / 2) * BJ_M * BJ_M;
}

size_t jacobi_params_elems(int64_t n) { return (size_t)8 * (n / 2 + 2) + 8 + n; }

cudaError_t jacobi_small_batched(cudaStream_t s, int n, int batch, const double2* G, double* w,
                                 double2* Z, int* status, int max_sweeps) {
  if (n > SJ_MAX || n < 1) return cudaErrorInvalidValue;
  const size_t smem = 2 * SJ_MAX * SJ_MAX * sizeof(double2);
  once_per_device(g_small_attr, [smem]() {
    cudaFuncSetAttribute(jacobi_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  });
  const int cap = max_sweeps > 0 ? std::min(max_sweeps, kMaxSweeps) : kMaxSweeps;
  jacobi_small_kernel<<<batch, SJ_T, smem, s>>>(n, G, w, Z, status, cap); count_launch();
  return cudaGetLastError();
}

namespace {
// FP64 finish restricted to the clusters of pairs the refinement left coupled
// (connected components of the recorded pairs, union-find on the host). For
// each cluster I: S_I = X_I^H G X_I in FP64, its eigenvectors Z_I by Jacobi
// (clusters of up to 64 batched in the single-CTA kernel, larger ones one by
// one in the cooperative kernel on their m x m block), X_I <- X_I Z_I, and its
// eigenvalues into lam. A cluster's coupling to every other vector is already
// at FP64 rounding level after the refinement, so the blocks are independent.
// Returns 1 when done, 0 when not applicable (pair list overflowed, or a
// cluster above 0.7 n, where the full FP64 sweeps cost about the same),
// -status on an error. *sweeps64 receives the FP64 sweeps of the large clusters.
int cluster_finish(cudaStream_t s, int64_t n, const double2* G, int64_t ldg, double2* X,
                   double2* XI, double* lam, JacobiWork& wk, int* status, int* info,
                   int max_sweeps, int* sweeps64) {
  info[0] = info[1] = 0;
  *sweeps64 = 0;
  int np = 0;
  if (cudaMemcpyAsync(&np, wk.npairs, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -CHASE_CUDA_FAIL();
  info[1] = np;
  if (np <= 0 || np > kMaxClusterPairs) return 0;
  std::vector<int> pr(2 * (size_t)np);
  if (cudaMemcpy(pr.data(), wk.pairs, pr.size() * sizeof(int), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return -CHASE_CUDA_FAIL();
  std::vector<int> parent((size_t)n);
  for (int64_t i = 0; i < n; ++i) parent[i] = (int)i;
  auto find = [&](int x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
  };
  for (int k = 0; k < np; ++k) {
    const int a = find(pr[2 * k]), b = find(pr[2 * k + 1]);
    if (a != b) parent[std::max(a, b)] = std::min(a, b);
  }
  // members of each component in ascending index order, components by size
  std::vector<std::vector<int>> comp((size_t)n);
  for (int64_t i = 0; i < n; ++i) comp[find((int)i)].push_back((int)i);
  std::vector<int> roots;
  for (int64_t i = 0; i < n; ++i)
    if (comp[i].size() >= 2) {
      info[0] = std::max(info[0], (int)comp[i].size());
      roots.push_back((int)i);
    }
  // a large cluster's Jacobi rotations (m x m, ld m) live in G32a viewed as FP64
  if ((double)info[0] > 0.7 * (double)n) return 0;
  if (roots.empty()) return 0;
  std::stable_sort(roots.begin(), roots.end(),
                   [&](int a, int b) { return comp[a].size() < comp[b].size(); });
  std::vector<int> idx;
  struct Group { int k, count; int64_t off; };
  std::vector<Group> groups;
  for (int r : roots) {
    const int k = (int)comp[r].size();
    if (groups.empty() || groups.back().k != k) groups.push_back({k, 0, (int64_t)idx.size()});
    groups.back().count++;
    idx.insert(idx.end(), comp[r].begin(), comp[r].end());
  }
  const int64_t ktot = (int64_t)idx.size();
  if (cudaMemcpyAsync(wk.cl_idx, idx.data(), ktot * sizeof(int), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
    return -CHASE_CUDA_FAIL();
  // XI = X(:, idx), TI = G XI (FP64)
  if (gather_cols(s, n, ktot, X, n, wk.cl_idx, XI, n) != cudaSuccess) return -CHASE_CUDA_FAIL();
  Epilogue ep{};
  ep.mode = EPI_STORE;
  ep.Y = wk.T;
  ep.ldy = n;
  if (zgemm_nn(s, n, ktot, n, G, ldg, XI, n, ep) != cudaSuccess) return -CHASE_CUDA_FAIL();
  double* wz = reinterpret_cast<double*>(wk.G32b);  // ktot eigenvalues
  for (const Group& g : groups) {
    const int64_t off = g.off;
    if (g.k > SJ_MAX) {  // one large cluster at a time, FP64 cooperative Jacobi
      for (int q = 0; q < g.count; ++q) {
        const int64_t m = g.k, o = off + (int64_t)q * m;
        if (zgram(s, n, m, m, XI + o * n, n, wk.T + o * n, n, wk.Gw, m, false, wk.gram_ws,
                  wk.gram_ws_elems) != cudaSuccess ||
            hermitian_part(s, m, wk.Gw, m) != cudaSuccess)
          return -CHASE_CUDA_FAIL();
        double2* Zr = reinterpret_cast<double2*>(wk.G32a);
        identity_kernel<<<dim3((unsigned)cdiv(m, 128), (unsigned)m, 1), 128, 0, s>>>(m, Zr);
        count_launch();
        int sw = 0;
        bool conv = false, in_g1 = false;
        RC_NEG(run_coop<double>(s, m, wk.Gw, wk.Gw2, Zr, wz + n, wk.red, max_sweeps, 1e-15, 1e-12,
                                &sw, &conv, &in_g1));
        *sweeps64 += sw;
        if (!conv) return -CHASE_ERR_HEEV_NOCONV;
        Epilogue ez{};
        ez.mode = EPI_STORE;  // P = X_I Z into the cluster's (now free) columns of T
        ez.Y = wk.T + o * n;
        ez.ldy = n;
        if (zgemm_nn(s, n, m, m, XI + o * n, n, Zr, m, ez) != cudaSuccess) return -CHASE_CUDA_FAIL();
        scatter_cluster_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)m, 1), 128, 0, s>>>(
            n, m, wk.T + o * n, wk.cl_idx + o, in_g1 ? wk.Gw2 : wk.Gw, X, lam);
        count_launch();
      }
      continue;
    }
    cluster_gram_kernel<<<g.count, 256, 0, s>>>(n, g.k, XI + off * n, wk.T + off * n, n, wk.Gw);
    count_launch();
    if (jacobi_small_batched(s, g.k, g.count, wk.Gw, wz + off, wk.Gw2, status, wk.max_sweeps) !=
        cudaSuccess)
      return -CHASE_CUDA_FAIL();
    cluster_apply_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)g.count, 1), 128, 0, s>>>(
        n, g.k, XI + off * n, n, wk.Gw2, wz + off, wk.cl_idx + off, X, lam);
    count_launch();
  }
  int hs = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -CHASE_CUDA_FAIL();
  info[1] = (int)roots.size();
  return hs ? -CHASE_ERR_HEEV_NOCONV : 1;
}
}  // namespace

int jacobi_heev(cudaStream_t s, int64_t n, const double2* G, int64_t ldg, double* w, double2* Z,
                int64_t ldz, JacobiWork& wk, int* sweeps_out, int* fp64_sweeps_out,
                int* cluster_out) {
  if (cluster_out) cluster_out[0] = cluster_out[1] = cluster_out[2] = 0;
  if (n <= 0) return CHASE_OK;
  cudaError_t e;
  int* status = reinterpret_cast<int*>(wk.red + 2 * kCoopMaxGrid + 8);
  if (n <= SJ_MAX) {
    // pack G (ld n) into Gw, run the single-CTA kernel into Zw, copy to Z.
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return CHASE_CUDA_FAIL();
    e = cudaMemcpy2DAsync(wk.Gw, n * sizeof(double2), G, ldg * sizeof(double2),
                          n * sizeof(double2), n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return CHASE_CUDA_FAIL();
    e = jacobi_small_batched(s, (int)n, 1, wk.Gw, w, wk.Zw, status, wk.max_sweeps);
    if (e != cudaSuccess) return CHASE_CUDA_FAIL();
    e = cudaMemcpy2DAsync(Z, ldz * sizeof(double2), wk.Zw, n * sizeof(double2),
                          n * sizeof(double2), n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return CHASE_CUDA_FAIL();
    int hs = 0;
    e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return CHASE_CUDA_FAIL();
    if (cudaStreamSynchronize(s) != cudaSuccess) return CHASE_CUDA_FAIL();
    if (sweeps_out) *sweeps_out = 0;
    return hs ? CHASE_ERR_HEEV_NOCONV : CHASE_OK;
  }
  // --- FP32 sweeps on the converted matrix
  const dim3 g2((unsigned)cdiv(n, 128), (unsigned)n, 1);
  init32_kernel<<<g2, 128, 0, s>>>(n, G, ldg, wk.G32a, wk.Z32); count_launch();
  int sw32 = 0;
  bool conv32 = false;
  // stage caps: 30 FP32 sweeps, 8 refinement steps, kMaxSweeps FP64 sweeps, each
  // lowered to the caller's cap when one is set
  auto cap = [&](int def) { return wk.max_sweeps > 0 ? std::min(def, wk.max_sweeps) : def; };
  // blocked FP32 Jacobi: G32a is G (in place), Rb the block rotations
  if (jacobi_rot_elems(n) > wk.rb_elems) return CHASE_ERR_INVALID_ARG;
  RC_(run_block_jacobi32(s, n, wk.G32a, wk.Z32, wk.Rb, wk.red, wk.host_part, cap(30), 4e-6, 1e-4,
                         &sw32, &conv32));
  // --- FP64: refine the FP32 eigenvectors (Ogita-Aishima steps, FP64 GEMMs)
  promote_kernel<<<g2, 128, 0, s>>>(n, wk.Z32, wk.Zw); count_launch();
  const unsigned gb = (unsigned)cdiv(n, 256);
  const int64_t nb = (int64_t)gb * n;  // partial slots (2 doubles each) of the E kernel
  double* lam = wk.params;             // n eigenvalue estimates (params is free here)
  double* out2 = wk.red + 2 * kCoopMaxGrid + 12;
  double2* X = wk.Zw;
  double2* Xn = wk.Zw2;
  // scale of G for the cluster test
  frob2_kernel<<<dim3(gb, (unsigned)n, 1), 256, 0, s>>>(n, G, ldg, reinterpret_cast<double*>(wk.T));
  count_launch();
  max2_kernel<<<1, 256, 0, s>>>(nb, reinterpret_cast<double*>(wk.T), out2); count_launch();
  if (cudaMemcpyAsync(wk.host_red, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CHASE_CUDA_FAIL();
  // sqrt(n) times the largest norm of a 256-row column segment: within a factor
  // sqrt(n) of ||G||_2 either way, enough for the 1e-14 cluster test below
  const double gscale = wk.host_red[0] * std::sqrt((double)n);
  int refine = 0;
  double emax = 1.0, cmax = 0.0;
  // With the digit-sliced tensor-core products (when the context supplies them)
  // the first, coarse steps use the 21-pair products, whose error (about
  // sqrt(n) 2^-50 of max|G_i.| max|X_.j| per entry) is far above what the Ritz
  // values need. Once the corrections fall below 1e-6 the steps are fine ones:
  // G X, X^H (G X) and X^H X, whose off-diagonal parts cancel to the size of
  // the corrections, keep the level-8 digit pairs too (error near the digit
  // rounding of the operands, a few 2^-48 of ||G||, like the CUDA-core FP64
  // products' sqrt(n) 2^-53), and so does the final orthogonalisation. Without
  // them, all products are the CUDA-core FP64 ones.
  const bool tc = wk.gemm != nullptr;
  bool fine = false;
  const int max_refine = cap(8);
  for (; refine < max_refine; ++refine) {  // 2-4 steps from FP32 accuracy; a slow start gets more
    Epilogue ep{};
    ep.mode = EPI_STORE;
    ep.Y = wk.T;
    ep.ldy = n;
    if (heev_nn(s, wk, tc, n, G, ldg, X, ep, fine) != cudaSuccess ||         // T = G X
        heev_cn(s, wk, tc, n, X, wk.T, wk.Gw, false, fine) != cudaSuccess ||   // S = X^H T
        heev_cn(s, wk, tc, n, X, X, wk.Gw2, true, fine) != cudaSuccess)        // X^H X
      return CHASE_CUDA_FAIL();
    oa_lambda_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(n, wk.Gw, wk.Gw2, lam); count_launch();
    // E into T (T is free once S is formed)
    if (cudaMemsetAsync(wk.npairs, 0, sizeof(int), s) != cudaSuccess) return CHASE_CUDA_FAIL();
    oa_e_kernel<<<dim3(gb, (unsigned)n, 1), 256, 0, s>>>(n, wk.Gw, wk.Gw2, lam, wk.T,
                                                        reinterpret_cast<double*>(wk.G32a),
                                                        wk.pairs, wk.npairs);
    count_launch();
    max2_kernel<<<1, 256, 0, s>>>(nb, reinterpret_cast<double*>(wk.G32a), out2); count_launch();
    // Xn = X + X E
    if (cudaMemcpyAsync(Xn, X, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return CHASE_CUDA_FAIL();
    Epilogue eu{};
    eu.mode = EPI_FILTER;
    eu.alpha = 1.0;
    eu.beta = 1.0;
    eu.gamma = 0.0;
    eu.X = Xn;
    eu.ldx = n;
    eu.Y = Xn;
    eu.ldy = n;
    if (heev_nn(s, wk, tc, n, X, n, wk.T, eu) != cudaSuccess) return CHASE_CUDA_FAIL();
    std::swap(X, Xn);
    if (cudaMemcpyAsync(wk.host_red, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return CHASE_CUDA_FAIL();
    emax = wk.host_red[0];
    cmax = wk.host_red[1];
    // the applied correction was ~emax; the error left is ~emax^2 (plus the
    // products' own error, hence the last step with the accurate products)
    if (emax <= 1e-8 && (!tc || fine)) {
      ++refine;
      break;
    }
    if (emax <= 1e-6) fine = true;
  }
  {
    // the corrections of close pairs carry rounding of order u / gap; one more
    // orthogonalisation step brings X^H X back to I at working precision
    if (heev_cn(s, wk, tc, n, X, X, wk.Gw2, true, true) != cudaSuccess) return CHASE_CUDA_FAIL();
    half_residual_kernel<<<g2, 128, 0, s>>>(n, wk.Gw2, wk.T); count_launch();
    if (cudaMemcpyAsync(Xn, X, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return CHASE_CUDA_FAIL();
    Epilogue eo{};
    eo.mode = EPI_FILTER;
    eo.alpha = 1.0;
    eo.beta = 1.0;
    eo.gamma = 0.0;
    eo.X = Xn;
    eo.ldx = n;
    eo.Y = Xn;
    eo.ldy = n;
    if (heev_nn(s, wk, tc, n, X, n, wk.T, eo) != cudaSuccess) return CHASE_CUDA_FAIL();
    std::swap(X, Xn);
  }
  int sw64 = 0;
  bool conv = emax <= 1e-8 && (!tc || fine);
  double2* Zfinal = X;
  double* wsrc = lam;
  bool clustered = false;
  if (conv && cmax > 1e-14 * gscale) {
    // pairs the refinement could not separate: FP64 Jacobi on each cluster of
    // them alone (their couplings to every other vector are already at FP64
    // level); falls through to full FP64 sweeps when the clusters are too many
    // or too large for the single-CTA kernel
    int cinfo[2];
    const int rc = cluster_finish(s, n, G, ldg, X, Xn, lam, wk, status, cinfo, cap(kMaxSweeps),
                                  &sw64);
    if (rc < 0) return -rc;
    clustered = rc == 1;
    if (cluster_out) {
      cluster_out[0] = clustered ? 1 : 0;  // finished by the cluster path
      cluster_out[1] = cinfo[0];           // largest cluster
      cluster_out[2] = cinfo[1];           // clusters (or recorded pairs if not used)
    }
  }
  if (!conv || (cmax > 1e-14 * gscale && !clustered)) {
    // pairs the refinement could not separate (or no convergence): FP64 Jacobi
    // sweeps on G' = X^H G X finish them; eigenvectors X Z'
    Epilogue ep{};
    ep.mode = EPI_STORE;
    ep.Y = wk.T;
    ep.ldy = n;
    if (zgemm_nn(s, n, n, n, G, ldg, X, n, ep) != cudaSuccess ||
        zgram(s, n, n, n, X, n, wk.T, n, wk.Gw, n, false, wk.gram_ws, wk.gram_ws_elems) !=
            cudaSuccess ||
        hermitian_part(s, n, wk.Gw, n) != cudaSuccess)
      return CHASE_CUDA_FAIL();
    double2* Zrot = Xn;  // the buffer X does not use
    identity_kernel<<<g2, 128, 0, s>>>(n, Zrot); count_launch();
    bool in_g1_64 = false;
    RC_(run_coop<double>(s, n, wk.Gw, wk.Gw2, Zrot, wk.params, wk.red, cap(kMaxSweeps), 1e-15,
                         1e-12, &sw64, &conv, &in_g1_64));
    double2* Gcur = in_g1_64 ? wk.Gw2 : wk.Gw;
    Epilogue ez{};
    ez.mode = EPI_STORE;
    ez.Y = wk.T;
    ez.ldy = n;
    if (zgemm_nn(s, n, n, n, X, n, Zrot, n, ez) != cudaSuccess) return CHASE_CUDA_FAIL();
    Zfinal = wk.T;
    int* rank = reinterpret_cast<int*>(wk.params + 8 * (n / 2 + 2));
    rank_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(n, Gcur, w, rank); count_launch();
    permute_cols_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(
        n, Zfinal, rank, Z, ldz); count_launch();
    wsrc = nullptr;
  }
  if (wsrc) {
    int* rank = reinterpret_cast<int*>(wk.params + 8 * (n / 2 + 2));
    rank_vec_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(n, lam, w, rank); count_launch();
    permute_cols_kernel<<<dim3((unsigned)cdiv(n, 128), (unsigned)n, 1), 128, 0, s>>>(
        n, Zfinal, rank, Z, ldz); count_launch();
  }
  if (cudaGetLastError() != cudaSuccess) return CHASE_CUDA_FAIL();
  if (sweeps_out) *sweeps_out = sw32 + sw64 + refine;
  if (fp64_sweeps_out) *fp64_sweeps_out = sw64;
  return conv ? CHASE_OK : CHASE_ERR_HEEV_NOCONV;
}

}  // namespace chase
