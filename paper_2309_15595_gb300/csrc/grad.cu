// Adjoints of the filter (Eq. 1 run backwards) and of the lowest eigenpairs
// (Hellmann-Feynman plus first-order eigenvector perturbation, the complement
// of the Ritz basis solved by projected conjugate gradients).
//
// Convention: for a real loss L the adjoint of a complex array Z is
// Zbar = 2 dL/d conj(Z); A is Hermitian, so its adjoint is made Hermitian.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "ctx.cuh"

using namespace chase;

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    fprintf(stderr, "[chase] CUDA error in %s: %s\n", what, cudaGetErrorString(e));
    return CHASE_CUDA_FAIL();
  }
  return CHASE_OK;
}
#define CK(call)                                   \
  do {                                             \
    int _rc = cuda_fail((call), #call);            \
    if (_rc != CHASE_OK) return _rc;               \
  } while (0)
#define RC(call)                                   \
  do {                                             \
    int _rc = (call);                              \
    if (_rc != CHASE_OK) return _rc;               \
  } while (0)

// ------------------------------------------------------------------ kernels
// out (cols x rows, ldo) = scale[j / block] * conj(X[:, j])^T for X rows x cols.
__global__ void conj_transpose_kernel(int64_t rows, int64_t cols, const double2* __restrict__ X,
                                      int64_t ldx, const double* __restrict__ scale,
                                      int64_t block, double2* __restrict__ out, int64_t ldo) {
  __shared__ double2 t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = r0 + tx, col = c0 + k;
    t[k][tx] = (r < rows && col < cols) ? X[r + col * ldx] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t col = c0 + tx, r = r0 + k;
    if (r < rows && col < cols) {
      const double s = scale ? scale[col / block] : 1.0;
      const double2 v = t[tx][k];
      out[col + r * ldo] = make_double2(s * v.x, -s * v.y);
    }
  }
}

// out[j] = Re(a_j^H b_j), one CTA per column, fixed-order reduction.
__global__ void col_dot_kernel(int64_t N, const double2* __restrict__ a, int64_t lda,
                               const double2* __restrict__ b, int64_t ldb, double* __restrict__ out) {
  __shared__ double red[256];
  const int64_t j = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += 256) {
    const double2 x = a[i + j * lda], y = b[i + j * ldb];
    s = fma(x.x, y.x, fma(x.y, y.y, s));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k >= 1; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

// W[:, j] -= shift[j] * P[:, j]
__global__ void shift_cols_kernel(int64_t N, int64_t n, double2* __restrict__ W, int64_t ldw,
                                  const double2* __restrict__ P, int64_t ldp,
                                  const double* __restrict__ shift) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= N) return;
  const double s = shift[j];
  const double2 p = P[i + j * ldp];
  double2 w = W[i + j * ldw];
  w.x = fma(-s, p.x, w.x);
  w.y = fma(-s, p.y, w.y);
  W[i + j * ldw] = w;
}

// Per-column CG scalars. sc layout (n each): rs, rs0, pw, rsn, alpha, beta, active.
struct CgScalars {
  double *rs, *rs0, *pw, *rsn, *alpha, *beta, *active;
};
__global__ void cg_alpha_kernel(int64_t n, CgScalars s) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  s.alpha[j] = (s.active[j] != 0.0 && s.pw[j] > 0.0) ? s.rs[j] / s.pw[j] : 0.0;
}
__global__ void cg_beta_kernel(int64_t n, double tol2, CgScalars s) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (s.active[j] == 0.0) {
    s.beta[j] = 0.0;
    return;
  }
  s.beta[j] = s.rsn[j] / s.rs[j];
  s.rs[j] = s.rsn[j];
  if (!(s.rsn[j] > tol2 * s.rs0[j])) s.active[j] = 0.0;
}
// rs0 holds ||b||^2, rsn the initial ||r||^2
__global__ void cg_init_kernel(int64_t n, double tol2, CgScalars s) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  s.rs[j] = s.rsn[j];
  s.active[j] = (s.rsn[j] > tol2 * s.rs0[j]) ? 1.0 : 0.0;
}
// z += alpha p; r -= alpha w (alpha null: r -= w, z untouched)
__global__ void cg_update_kernel(int64_t N, double2* __restrict__ Z, double2* __restrict__ R,
                                 const double2* __restrict__ P, const double2* __restrict__ W,
                                 int64_t ld, const double* __restrict__ alpha) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= N) return;
  const double a = alpha ? alpha[j] : 1.0;
  if (a == 0.0) return;
  const int64_t k = i + j * ld;
  const double2 w = W[k];
  double2 r = R[k];
  r.x = fma(-a, w.x, r.x);
  r.y = fma(-a, w.y, r.y);
  R[k] = r;
  if (alpha) {
    const double2 p = P[k];
    double2 z = Z[k];
    z.x = fma(a, p.x, z.x);
    z.y = fma(a, p.y, z.y);
    Z[k] = z;
  }
}

// D[j, i] /= (ritz_x[j] - ritz_i): Galerkin solution of (A - ritz_i) z = b in
// the span of the extra Ritz vectors (nx x nev, ld)
__global__ void galerkin_kernel(int64_t nx, int64_t nev, double2* __restrict__ D, int64_t ldd,
                                const double* __restrict__ ritz_x,
                                const double* __restrict__ ritz) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= nx) return;
  const double f = 1.0 / (ritz_x[j] - ritz[i]);
  double2 v = D[j + i * ldd];
  D[j + i * ldd] = make_double2(f * v.x, f * v.y);
}
// p = r + beta p (active columns)
__global__ void cg_dir_kernel(int64_t N, const double2* __restrict__ R, double2* __restrict__ P,
                              int64_t ld, const double* __restrict__ beta,
                              const double* __restrict__ active) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= N || active[j] == 0.0) return;
  const int64_t k = i + j * ld;
  const double b = beta[j];
  const double2 r = R[k], p = P[k];
  P[k] = make_double2(fma(b, p.x, r.x), fma(b, p.y, r.y));
}

// C[j, i] *= 1 / (ritz_i - ritz_j) for j != i, 0 for j == i (ne x nev, ldc)
__global__ void divided_kernel(int64_t ne, int64_t nev, double2* __restrict__ C, int64_t ldc,
                               const double* __restrict__ ritz) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= ne) return;
  double2 v = C[j + i * ldc];
  const double f = (j == i) ? 0.0 : 1.0 / (ritz[i] - ritz[j]);
  C[j + i * ldc] = make_double2(f * v.x, f * v.y);
}

// M[:, i] = lam_bar_i x_i - Z[:, i]   (lam_bar, Z may be null)
__global__ void eig_base_kernel(int64_t N, const double2* __restrict__ X, int64_t ldx,
                                const double* __restrict__ lam_bar,
                                const double2* __restrict__ Z, int64_t ldz,
                                double2* __restrict__ M, int64_t ldm) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (r >= N) return;
  const double lb = lam_bar ? lam_bar[i] : 0.0;
  const double2 x = X[r + i * ldx];
  double2 m = make_double2(lb * x.x, lb * x.y);
  if (Z) {
    const double2 z = Z[r + i * ldz];
    m.x -= z.x;
    m.y -= z.y;
  }
  M[r + i * ldm] = m;
}

// ------------------------------------------------------------------ helpers
cudaError_t copy_block(cudaStream_t s, double2* dst, int64_t ldd, const double2* src, int64_t lds,
                       int64_t rows, int64_t cols) {
  if (cols == 0) return cudaSuccess;
  return cudaMemcpy2DAsync(dst, ldd * sizeof(double2), src, lds * sizeof(double2),
                           rows * sizeof(double2), cols, cudaMemcpyDeviceToDevice, s);
}

int ensure_workspace(chase_ctx* c, size_t elems, size_t scalars) {
  if (c->gw_elems < elems) {
    if (c->gw) cudaFree(c->gw);
    c->gw = nullptr;
    c->gw_elems = 0;
    if (cudaMalloc(&c->gw, elems * sizeof(double2)) != cudaSuccess) return CHASE_ERR_OOM;
    c->gw_elems = elems;
  }
  if (c->gd_elems < scalars) {
    if (c->gd) cudaFree(c->gd);
    c->gd = nullptr;
    c->gd_elems = 0;
    if (cudaMalloc(&c->gd, scalars * sizeof(double)) != cudaSuccess) return CHASE_ERR_OOM;
    c->gd_elems = scalars;
  }
  return CHASE_OK;
}

// out = alpha (A X - gamma X) + beta out, the filter step on the context's
// product path (X: N x n, ldx; out: N x n, ldo)
int filter_step(chase_ctx* c, const double2* A, int64_t lda, const double2* X, int64_t ldx,
                int64_t n, double alpha, double beta, double gamma, double2* out, int64_t ldo) {
  Epilogue ep{};
  ep.mode = EPI_FILTER;
  ep.alpha = alpha;
  ep.beta = beta;
  ep.gamma = gamma;
  ep.X = X;
  ep.ldx = ldx;
  ep.Y = out;
  ep.ldy = ldo;
  if (c->p.fp64_tensor) {
    CK(ozaki_gemm(c->stream, n, 0, X, ldx, ep, c->ow));
  } else {
    CK(zgemm_nn(c->stream, c->N, n, c->N, A, lda, X, ldx, ep));
  }
  return CHASE_OK;
}

int finish(chase_ctx* c) {
  if (c->p.fp64_tensor) RC(ozaki_check(c->stream, c->ow));
  CK(cudaStreamSynchronize(c->stream));
  return CHASE_OK;
}

}  // namespace

// ------------------------------------------------------------- filter VJP
extern "C" int chase_filter_vjp(chase_ctx* c, const chase_c128* Ac, int64_t lda,
                                const chase_c128* Vc, int64_t ldv, int64_t n, int32_t deg,
                                double cc, double e, double mu_1, const chase_c128* Ybc,
                                int64_t ldyb, chase_c128* Abc, int64_t ldab, chase_c128* Vbc,
                                int64_t ldvb, int32_t checkpoint) {
  if (!c || !Ac || !Vc || !Ybc || !Abc || !Vbc) return CHASE_ERR_INVALID_ARG;
  const int64_t N = c->N;
  if (lda < N || ldv < N || ldyb < N || ldab < N || ldvb < N || n < 1 || n > c->ne || deg < 1 ||
      deg > 64)
    return CHASE_ERR_INVALID_ARG;
  if (!(e > 0.0) || (c->p.scaled_filter && !(mu_1 <= cc - e))) return CHASE_ERR_INVALID_ARG;
  const double2* A = reinterpret_cast<const double2*>(Ac);
  const double2* V = reinterpret_cast<const double2*>(Vc);
  const double2* Yb = reinterpret_cast<const double2*>(Ybc);
  double2* Ab = reinterpret_cast<double2*>(Abc);
  double2* Vb = reinterpret_cast<double2*>(Vbc);
  cudaStream_t s = c->stream;

  const int m = deg;
  const int seg = checkpoint > 0 ? std::min(checkpoint, m)
                                 : std::max(1, (int)std::ceil(std::sqrt((double)m)));
  const int nseg = (m + seg - 1) / seg;
  std::vector<double> al, be;
  cheb_coefficients(m + 1, cc, e, mu_1, c->p.scaled_filter != 0, al, be);
  be[m + 1] = 0.0;  // Z_{m+1} = 0

  // workspace (blocks of N x n, ld N): checkpoints Y_{ks} and Y_{ks-1}
  // (k = 0..nseg-1), segment states Y_{ks..ks+seg-1}, segment adjoints
  // Z_{ks..ks+seg+1}, and the scaled conjugate transpose of the segment states
  const size_t blk = (size_t)N * n;
  const size_t nblk = 2 * (size_t)nseg + seg + (seg + 2) + seg;
  RC(ensure_workspace(c, nblk * blk, (size_t)seg + 8));
  double2* ck_cur = c->gw;
  double2* ck_prev = ck_cur + nseg * blk;
  double2* yseg = ck_prev + nseg * blk;
  double2* zseg = yseg + seg * blk;
  double2* wt = zseg + (seg + 2) * blk;  // (seg n) x N, ld seg n
  double* dscale = c->gd;
  RC(ctx_prepare_a(c, A, lda));

  // forward sweep, keeping only the checkpoints: ping-pong in yseg[0], yseg[1]
  // (seg >= 2) or ck slots directly
  CK(copy_block(s, ck_cur, N, V, ldv, N, n));  // Y_0
  {
    double2* cur = ck_cur;  // Y_{i-1}
    double2* prev = nullptr;  // Y_{i-2}
    double2* tmp[2] = {yseg, zseg};  // scratch (zseg unused until the reverse sweep)
    for (int i = 1; i < m; ++i) {
      double2* out = tmp[i & 1];
      const int k = i / seg;
      if (i % seg == 0) out = ck_cur + k * blk;                 // Y_{ks}
      else if ((i + 1) % seg == 0 && (i + 1) / seg < nseg) out = ck_prev + ((i + 1) / seg) * blk;
      // out <- beta_i Y_{i-2} first (in-place epilogue reads it)
      if (i >= 2 && out != prev) CK(copy_block(s, out, N, prev, N, N, n));
      RC(filter_step(c, A, lda, cur, N, n, al[i], i >= 2 ? be[i] : 0.0, cc, out, N));
      prev = cur;
      cur = out;
    }
  }

  // reverse sweep, segment by segment
  CK(cudaMemset2DAsync(Ab, ldab * sizeof(double2), 0, N * sizeof(double2), N, s));
  for (int k = nseg - 1; k >= 0; --k) {
    const int i0 = k * seg;                    // segment covers steps i0+1 .. i1
    const int i1 = std::min(i0 + seg, m);
    const int len = i1 - i0;
    // recompute Y_{i0} .. Y_{i1-1} into yseg[0 .. len-1]
    CK(copy_block(s, yseg, N, ck_cur + k * blk, N, N, n));
    for (int j = 1; j < len; ++j) {
      const int i = i0 + j;
      const double2* ym2 = (j >= 2) ? yseg + (j - 2) * blk : (i >= 2 ? ck_prev + k * blk : nullptr);
      if (i >= 2) CK(copy_block(s, yseg + j * blk, N, ym2, N, N, n));
      RC(filter_step(c, A, lda, yseg + (j - 1) * blk, N, n, al[i], i >= 2 ? be[i] : 0.0, cc,
                     yseg + j * blk, N));
    }
    // Z_{i1} and Z_{i1+1} sit in zseg[len], zseg[len+1]
    if (k == nseg - 1) {
      CK(copy_block(s, zseg + len * blk, N, Yb, ldyb, N, n));
      CK(cudaMemsetAsync(zseg + (len + 1) * blk, 0, blk * sizeof(double2), s));
    }
    for (int i = i1; i > i0; --i) {  // Z_{i-1} = alpha_i (A - cI) Z_i + beta_{i+1} Z_{i+1}
      double2* zi = zseg + (i - i0) * blk;
      double2* zo = zseg + (i - 1 - i0) * blk;
      const double2* zn = zseg + (i + 1 - i0) * blk;
      const double b = be[i + 1];
      if (b != 0.0) CK(copy_block(s, zo, N, zn, N, N, n));
      RC(filter_step(c, A, lda, zi, N, n, al[i], b, cc, zo, N));
    }
    // Abar += [Z_{i0+1} .. Z_{i1}] diag(alpha) [Y_{i0} .. Y_{i1-1}]^H
    std::vector<double> sc(len);
    for (int j = 0; j < len; ++j) sc[j] = al[i0 + 1 + j];
    CK(cudaMemcpyAsync(dscale, sc.data(), len * sizeof(double), cudaMemcpyHostToDevice, s));
    const int64_t K = (int64_t)len * n;
    conj_transpose_kernel<<<dim3((unsigned)cdiv(N, 32), (unsigned)cdiv(K, 32), 1), dim3(32, 8, 1),
                            0, s>>>(N, K, yseg, N, dscale, n, wt, K);
    count_launch();
    CK(cudaGetLastError());
    Epilogue ep{};
    ep.mode = EPI_FILTER;  // Abar = 1 * (P - 0) + 1 * Abar
    ep.alpha = 1.0;
    ep.beta = 1.0;
    ep.gamma = 0.0;
    ep.X = Ab;
    ep.ldx = ldab;
    ep.Y = Ab;
    ep.ldy = ldab;
    CK(zgemm_nn(s, N, N, K, zseg + blk, N, wt, K, ep));
    // the host copy of the scales must outlive the enqueued copy
    CK(cudaStreamSynchronize(s));
    // carry Z_{i0}, Z_{i0+1} to the next (earlier) segment's top slots
    if (k > 0) {
      CK(copy_block(s, zseg + (seg + 1) * blk, N, zseg + blk, N, N, n));
      CK(copy_block(s, zseg + seg * blk, N, zseg, N, N, n));
    }
  }
  CK(copy_block(s, Vb, ldvb, zseg, N, N, n));  // Vbar = Z_0
  CK(hermitian_part(s, N, Ab, ldab));
  return finish(c);
}

// ----------------------------------------------------------- eigenpair VJP
extern "C" int chase_eig_vjp(chase_ctx* c, const chase_c128* Ac, int64_t lda,
                             const chase_c128* Xc, int64_t ldx, const double* ritz, int64_t ne,
                             int64_t nev, const double* lam_bar, const chase_c128* Xbc,
                             int64_t ldxb, chase_c128* Abc, int64_t ldab, double cg_tol,
                             int32_t cg_max_iter, int32_t* cg_iters) {
  if (!c || !Ac || !Xc || !ritz || !Abc) return CHASE_ERR_INVALID_ARG;
  const int64_t N = c->N;
  if (lda < N || ldx < N || ldab < N || ne < 1 || ne > c->ne || nev < 1 || nev > ne ||
      (Xbc && ldxb < N) || !(cg_tol > 0.0) || cg_max_iter < 0)
    return CHASE_ERR_INVALID_ARG;
  const double2* A = reinterpret_cast<const double2*>(Ac);
  const double2* X = reinterpret_cast<const double2*>(Xc);
  const double2* Xb = reinterpret_cast<const double2*>(Xbc);
  double2* Ab = reinterpret_cast<double2*>(Abc);
  cudaStream_t s = c->stream;
  const int64_t nx = ne - nev;  // extra Ritz vectors: initial guess of the complement solves
  const size_t blk = (size_t)N * nev;
  RC(ensure_workspace(c, 5 * blk, 7 * (size_t)nev + 8));
  double2* Z = c->gw;
  double2* R = Z + blk;
  double2* P = R + blk;
  double2* W = P + blk;
  double2* M = W + blk;
  double2* C = c->G;     // nev x nev (ld ne): x_j^H xbar_i inside the wanted block
  double2* D = c->Yeig;  // ne x nev (ld ne): projections, Galerkin coefficients
  double* d = c->gd;
  CgScalars sc{d, d + nev, d + 2 * nev, d + 3 * nev, d + 4 * nev, d + 5 * nev, d + 6 * nev};
  int iters = 0;
  bool converged = true;
  const unsigned gN = (unsigned)cdiv(N, 256);

  // W = (I - Xw Xw^H)(A - ritz_i I) Q, column by column shift
  auto apply_op = [&](const double2* Q) -> int {
    Epilogue st{};
    st.mode = EPI_STORE;
    st.Y = W;
    st.ldy = N;
    if (c->p.fp64_tensor) {
      CK(ozaki_gemm(s, nev, 0, Q, N, st, c->ow));
    } else {
      CK(zgemm_nn(s, N, nev, N, A, lda, Q, N, st));
    }
    shift_cols_kernel<<<dim3(gN, (unsigned)nev, 1), 256, 0, s>>>(N, nev, W, N, Q, N, ritz);
    count_launch();
    CK(zgram(s, N, nev, nev, X, ldx, W, N, D, c->ne, false, c->gram_ws, c->gram_ws_elems));
    Epilogue pw{};
    pw.mode = EPI_FILTER;  // W = -Xw D + W
    pw.alpha = -1.0;
    pw.beta = 1.0;
    pw.gamma = 0.0;
    pw.X = W;
    pw.ldx = N;
    pw.Y = W;
    pw.ldy = N;
    CK(zgemm_nn(s, N, nev, nev, X, ldx, D, c->ne, pw));
    return CHASE_OK;
  };

  if (Xb) {
    RC(ctx_prepare_a(c, A, lda));
    // C = Xw^H Xbar; R = b = (I - Xw Xw^H) Xbar
    CK(zgram(s, N, nev, nev, X, ldx, Xb, ldxb, C, c->ne, false, c->gram_ws, c->gram_ws_elems));
    CK(copy_block(s, R, N, Xb, ldxb, N, nev));
    Epilogue pr{};
    pr.mode = EPI_FILTER;
    pr.alpha = -1.0;
    pr.beta = 1.0;
    pr.gamma = 0.0;
    pr.X = R;
    pr.ldx = N;
    pr.Y = R;
    pr.ldy = N;
    CK(zgemm_nn(s, N, nev, nev, X, ldx, C, c->ne, pr));
    col_dot_kernel<<<(unsigned)nev, 256, 0, s>>>(N, R, N, R, N, sc.rs0);
    count_launch();
    // initial guess from the extra Ritz pairs: z_i = sum_j x_j (x_j^H b_i) / (ritz_j - ritz_i)
    if (nx > 0) {
      const double2* Xx = X + nev * ldx;
      CK(zgram(s, N, nx, nev, Xx, ldx, R, N, D, c->ne, false, c->gram_ws, c->gram_ws_elems));
      galerkin_kernel<<<dim3((unsigned)cdiv(nx, 128), (unsigned)nev, 1), 128, 0, s>>>(
          nx, nev, D, c->ne, ritz + nev, ritz);
      count_launch();
      Epilogue ez{};
      ez.mode = EPI_STORE;
      ez.Y = Z;
      ez.ldy = N;
      CK(zgemm_nn(s, N, nev, nx, Xx, ldx, D, c->ne, ez));
      RC(apply_op(Z));  // r = b - op(z)
      cg_update_kernel<<<dim3(gN, (unsigned)nev, 1), 256, 0, s>>>(N, nullptr, R, nullptr, W, N,
                                                                  nullptr);
      count_launch();
    } else {
      CK(cudaMemsetAsync(Z, 0, blk * sizeof(double2), s));
    }
    CK(copy_block(s, P, N, R, N, N, nev));
    col_dot_kernel<<<(unsigned)nev, 256, 0, s>>>(N, R, N, R, N, sc.rsn);
    count_launch();
    const double tol2 = cg_tol * cg_tol;
    cg_init_kernel<<<(unsigned)cdiv(nev, 128), 128, 0, s>>>(nev, tol2, sc);
    count_launch();
    CK(cudaGetLastError());
    std::vector<double> act(nev);
    converged = false;
    for (iters = 0; iters < cg_max_iter; ++iters) {
      if (iters % 8 == 0) {
        CK(cudaMemcpyAsync(act.data(), sc.active, nev * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (std::all_of(act.begin(), act.end(), [](double v) { return v == 0.0; })) {
          converged = true;
          break;
        }
      }
      RC(apply_op(P));
      col_dot_kernel<<<(unsigned)nev, 256, 0, s>>>(N, P, N, W, N, sc.pw);
      cg_alpha_kernel<<<(unsigned)cdiv(nev, 128), 128, 0, s>>>(nev, sc);
      cg_update_kernel<<<dim3(gN, (unsigned)nev, 1), 256, 0, s>>>(N, Z, R, P, W, N, sc.alpha);
      col_dot_kernel<<<(unsigned)nev, 256, 0, s>>>(N, R, N, R, N, sc.rsn);
      cg_beta_kernel<<<(unsigned)cdiv(nev, 128), 128, 0, s>>>(nev, tol2, sc);
      cg_dir_kernel<<<dim3(gN, (unsigned)nev, 1), 256, 0, s>>>(N, R, P, N, sc.beta, sc.active);
      for (int q = 0; q < 6; ++q) count_launch();
      CK(cudaGetLastError());
    }
    if (!converged) {
      CK(cudaMemcpyAsync(act.data(), sc.active, nev * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      converged = std::all_of(act.begin(), act.end(), [](double v) { return v == 0.0; });
    }
    // in-block coefficients: C[j, i] / (ritz_i - ritz_j), j != i
    divided_kernel<<<dim3((unsigned)cdiv(nev, 128), (unsigned)nev, 1), 128, 0, s>>>(nev, nev, C,
                                                                                    c->ne, ritz);
    count_launch();
  }
  // M = Xw diag(lam_bar) - Z + Xw (F o C)
  eig_base_kernel<<<dim3(gN, (unsigned)nev, 1), 256, 0, s>>>(N, X, ldx, lam_bar, Xb ? Z : nullptr,
                                                             N, M, N);
  count_launch();
  CK(cudaGetLastError());
  if (Xb) {
    Epilogue ey{};
    ey.mode = EPI_FILTER;
    ey.alpha = 1.0;
    ey.beta = 1.0;
    ey.gamma = 0.0;
    ey.X = M;
    ey.ldx = N;
    ey.Y = M;
    ey.ldy = N;
    CK(zgemm_nn(s, N, nev, nev, X, ldx, C, c->ne, ey));
  }
  // Abar = herm(M Xw^H)
  double2* XwH = Z;  // nev x N, ld nev (Z no longer needed)
  conj_transpose_kernel<<<dim3((unsigned)cdiv(N, 32), (unsigned)cdiv(nev, 32), 1), dim3(32, 8, 1),
                          0, s>>>(N, nev, X, ldx, nullptr, 1, XwH, nev);
  count_launch();
  Epilogue ea{};
  ea.mode = EPI_STORE;
  ea.Y = Ab;
  ea.ldy = ldab;
  CK(zgemm_nn(s, N, N, nev, M, N, XwH, nev, ea));
  CK(hermitian_part(s, N, Ab, ldab));
  RC(finish(c));
  if (cg_iters) *cg_iters = iters;
  return converged ? CHASE_OK : CHASE_ERR_NOT_CONVERGED;
}
